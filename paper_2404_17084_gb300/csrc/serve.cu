// Serving loop: continuous batching of mapping requests on one GPU.
//
// A server owns `slots` workers.  Each worker has its own context (octree,
// pair-list and integral workspace), its own non-blocking CUDA stream and a
// host thread, so the requests of different slots overlap on the device.
// Requests are queued FIFO as they arrive; the admission step starts the
// oldest queued request as soon as a slot is idle AND its device-memory
// estimate fits the server's HBM budget next to what the running requests
// hold and what idle slots keep cached (idle caches are released when that
// makes room).  A running request copies its host inputs to the device,
// uploads and prepares its grid (resident for the request), solves h
// (Eq. 7-9) and maps the particles (Eq. 1-3) on its slot, then copies the
// cell masses back.  Each result depends only on its own request: a request
// gives the same bits alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

struct map_server {
  map_server_config cfg;
  struct Slot {
    map_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread thread;
    bool busy = false;
    int64_t ticket = -1;    // request being run
    size_t reserved = 0;    // its admission estimate
  };
  struct Rec {
    map_request req;
    map_request_result res;
    bool done = false;
    std::chrono::steady_clock::time_point t_submit, t_admit;
  };
  std::vector<Slot> slots;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Rec> recs;
  std::mutex mu;
  std::condition_variable cv_work;  // workers wait for an admitted request
  std::condition_variable cv_done;  // callers wait for results
  int64_t next_ticket = 0;
  int64_t completed = 0;
  bool stopping = false;
};

namespace {

double ms_between(std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes a request may hold: its input copies, the prepared grid, the
// octree, the pair list (160 pairs per particle assumed: FP64 fraction and
// two index arrays) and the per-cell outputs, with 25% headroom.
size_t request_bytes(const map_request& r, int precision) {
  const double parts = 48.0 * r.n + 200.0 * r.n + 160.0 * 16.0 * r.n;
  // per loop entry: the staged index and the edge records the precision keeps
  // (12 floats for the mixed build, 12 doubles for FP64)
  const double loop = precision != MAP_FP64 ? 64.0 : 112.0;
  const double grid = 96.0 * r.ncell + 146.0 * r.nface + loop * r.nloop + 48.0 * r.nvert;
  const double outs = 24.0 * r.ncell;
  return (size_t)(1.25 * (parts + grid + outs)) + (64u << 20);
}

// Context workspace kept by an idle slot.
size_t cached_bytes(const map_server::Slot& s) { return s.ctx ? s.ctx->bytes_in_use : 0; }

// Frees a context's workspace and its pool of released grid buffers (not
// its grids); the next request reallocates.
void trim(map_ctx* ctx) {
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  auto drop = [&](DevBuf& b) {
    if (b.p) { cudaFree(b.p); ctx->bytes_in_use -= b.cap; b.p = nullptr; b.cap = 0; }
  };
  for (auto& b : ctx->ws_tree) drop(b);
  for (auto& b : ctx->ws_pairs) drop(b);
  for (auto& b : ctx->ws_misc) drop(b);
  for (auto& b : ctx->ws_inv) drop(b);
  for (auto& b : ctx->ws_vor) drop(b);
  for (auto& b : ctx->ws_grid) drop(b);
  for (auto* v : {&ctx->batch_off, &ctx->batch_idx, &ctx->batch_itm, &ctx->batch_ioff, &ctx->batch_part})
    for (auto& b : *v) drop(b);
  drop(ctx->cub_tmp);
  grid_pool_drop(ctx);
  ctx->pair_off = nullptr;
  ctx->pair_idx = nullptr;
  ctx->pair_frac = nullptr;
  ctx->inv_ready = false;
  ctx->items = nullptr;
  ctx->item_off = nullptr;
  ctx->partial = nullptr;
  ctx->bsig.clear();
}

// Starts queued requests while a slot is idle and memory allows (mu held).
void admit(map_server* S) {
  while (!S->queue.empty()) {
    int free_slot = -1;
    for (int i = 0; i < (int)S->slots.size(); ++i)
      if (!S->slots[i].busy) { free_slot = i; break; }
    if (free_slot < 0) return;
    const int64_t t = S->queue.front();
    map_server::Rec& R = S->recs[t];
    const size_t need = request_bytes(R.req, S->cfg.precision);
    auto held = [&]() {
      size_t h = 0;
      for (auto& s : S->slots) h += s.busy ? (s.reserved > cached_bytes(s) ? s.reserved : cached_bytes(s)) : cached_bytes(s);
      return h;
    };
    size_t in_use = held() - cached_bytes(S->slots[free_slot]);
    if (S->cfg.hbm_budget && in_use + need > S->cfg.hbm_budget) {
      // release the caches of idle slots, then look again
      for (auto& s : S->slots)
        if (!s.busy && s.ctx) trim(s.ctx);
      in_use = held() - cached_bytes(S->slots[free_slot]);
      if (in_use + need > S->cfg.hbm_budget) {
        bool any_busy = false;
        for (auto& s : S->slots) any_busy = any_busy || s.busy;
        if (any_busy) return;  // wait for memory to free up
        // alone and still too large: it can never run
        S->queue.pop_front();
        R.res.status = MAP_ENOMEM;
        R.res.bytes_reserved = need;
        R.done = true;
        ++S->completed;
        S->cv_done.notify_all();
        continue;
      }
    }
    S->queue.pop_front();
    map_server::Slot& sl = S->slots[free_slot];
    sl.busy = true;
    sl.ticket = t;
    sl.reserved = need;
    R.t_admit = std::chrono::steady_clock::now();
    R.res.bytes_reserved = need;
    S->cv_work.notify_all();
  }
}

// Runs one request on a slot (no lock held).
int run_request(map_server::Slot& sl, const map_request& q, map_request_result& res) {
  map_ctx* ctx = sl.ctx;
  cudaStream_t s = sl.stream;
  CUDA_TRY(cudaSetDevice(ctx->device));
  // device copies of the inputs, stream-ordered
  const size_t sz_p = q.n * sizeof(double);
  double *x = nullptr, *y = nullptr, *z = nullptr, *m = nullptr, *h = nullptr, *mass = nullptr, *rho = nullptr;
  int64_t *cfo = nullptr, *fvo = nullptr;
  int32_t* fv = nullptr;
  double *plane = nullptr, *vx = nullptr, *vy = nullptr, *vz = nullptr, *site = nullptr;
  std::vector<void*> owned;
  auto get = [&](auto** p, size_t bytes) -> int {
    void* v = nullptr;
    if (cudaMallocAsync(&v, bytes > 0 ? bytes : 16, s) != cudaSuccess) { cudaGetLastError(); return MAP_ENOMEM; }
    owned.push_back(v);
    *p = reinterpret_cast<std::remove_pointer_t<decltype(p)>>(v);
    return MAP_OK;
  };
  int rc = MAP_OK;
  auto cleanup = [&]() {
    for (void* v : owned) cudaFreeAsync(v, s);
    cudaStreamSynchronize(s);
  };
  if ((rc = get(&x, sz_p)) || (rc = get(&y, sz_p)) || (rc = get(&z, sz_p)) || (rc = get(&m, sz_p)) ||
      (rc = get(&h, sz_p)) || (rc = get(&mass, q.ncell * sizeof(double))) ||
      (rc = get(&rho, q.ncell * sizeof(double))) || (rc = get(&cfo, (q.ncell + 1) * sizeof(int64_t))) ||
      (rc = get(&fvo, (q.nface + 1) * sizeof(int64_t))) || (rc = get(&fv, q.nloop * sizeof(int32_t))) ||
      (rc = get(&plane, 4 * q.nface * sizeof(double))) || (rc = get(&vx, q.nvert * sizeof(double))) ||
      (rc = get(&vy, q.nvert * sizeof(double))) || (rc = get(&vz, q.nvert * sizeof(double))) ||
      (rc = get(&site, 3 * q.ncell * sizeof(double)))) {
    cleanup();
    return rc;
  }
  auto h2d = [&](void* d, const void* hsrc, size_t bytes) {
    return cudaMemcpyAsync(d, hsrc, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  bool ok = h2d(x, q.x, sz_p) && h2d(y, q.y, sz_p) && h2d(z, q.z, sz_p) && h2d(m, q.m, sz_p) &&
            h2d(cfo, q.cell_face_off, (q.ncell + 1) * sizeof(int64_t)) &&
            h2d(fvo, q.face_vert_off, (q.nface + 1) * sizeof(int64_t)) &&
            h2d(fv, q.face_vert, q.nloop * sizeof(int32_t)) && h2d(plane, q.face_plane, 4 * q.nface * sizeof(double)) &&
            h2d(vx, q.vx, q.nvert * sizeof(double)) && h2d(vy, q.vy, q.nvert * sizeof(double)) &&
            h2d(vz, q.vz, q.nvert * sizeof(double)) && h2d(site, q.site, 3 * q.ncell * sizeof(double));
  if (!ok) { cudaGetLastError(); cleanup(); return MAP_ECUDA; }
  map_grid g{q.ncell, q.nface, q.nloop, q.nvert, cfo, fvo, fv, plane, vx, vy, vz, site};
  int handle = -1;
  rc = map_grid_upload(ctx, &g, &handle, s);
  map_particles p{q.n, x, y, z, m, h};
  if (rc == MAP_OK) rc = solve_h(ctx, &p, nullptr, s);
  map_outputs out{mass, rho, nullptr};
  if (rc == MAP_OK) rc = map_particles_to_cells(ctx, &p, handle, &out, s);
  map_stats st{};
  if (rc == MAP_OK) rc = map_get_stats(ctx, &st);
  if (rc == MAP_OK) {
    ok = cudaMemcpyAsync(q.cell_mass, mass, q.ncell * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok && q.cell_rho)
      ok = cudaMemcpyAsync(q.cell_rho, rho, q.ncell * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok && q.h) ok = cudaMemcpyAsync(q.h, h, sz_p, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); rc = MAP_ECUDA; }
  }
  if (handle >= 0) map_grid_release(ctx, handle);
  cleanup();
  res.n_pairs = st.n_pairs;
  res.total_mass = st.total_mass;
  return rc != MAP_OK ? rc : (st.status != MAP_OK ? st.status : MAP_OK);
}

void worker(map_server* S, int i) {
  for (;;) {
    int64_t t;
    map_request q;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stopping || (S->slots[i].busy && S->slots[i].ticket >= 0); });
      if (S->slots[i].ticket < 0) return;  // stopping with nothing to run
      t = S->slots[i].ticket;
      q = S->recs[t].req;
    }
    map_request_result res{};
    const int rc = run_request(S->slots[i], q, res);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      map_server::Rec& R = S->recs[t];
      const auto now = std::chrono::steady_clock::now();
      res.status = rc;
      res.bytes_reserved = R.res.bytes_reserved;
      res.queue_ms = ms_between(R.t_submit, R.t_admit);
      res.latency_ms = ms_between(R.t_submit, now);
      R.res = res;
      R.done = true;
      ++S->completed;
      S->slots[i].busy = false;
      S->slots[i].ticket = -1;
      S->slots[i].reserved = 0;
      admit(S);
      S->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

void map_server_config_default(map_server_config* cfg) {
  if (!cfg) return;
  cfg->device = 0;
  cfg->precision = MAP_MIXED;
  cfg->slots = 4;
  cfg->hbm_budget = 0;
  cfg->hfact = 1.2;
}

int map_server_create(const map_server_config* cfg, map_server** out) {
  if (!out) return MAP_EINVAL;
  *out = nullptr;
  map_server_config c;
  map_server_config_default(&c);
  if (cfg) c = *cfg;
  if (c.slots < 1 || c.slots > 64 || !(c.hfact > 0.0)) return MAP_EINVAL;
  CUDA_TRY(cudaSetDevice(c.device));
  if (c.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    c.hbm_budget = fr / 10 * 9;
  }
  map_server* S = new (std::nothrow) map_server();
  if (!S) return MAP_ENOMEM;
  S->cfg = c;
  S->slots.resize(c.slots);
  for (auto& sl : S->slots) {
    map_config mc;
    map_config_default(&mc);
    mc.device = c.device;
    mc.precision = c.precision;
    mc.hfact = c.hfact;
    int rc = map_init(&sl.ctx, &mc);
    if (rc == MAP_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) rc = MAP_ECUDA;
    if (rc != MAP_OK) {
      cudaGetLastError();
      for (auto& s2 : S->slots) {
        if (s2.ctx) map_destroy(s2.ctx);
        if (s2.stream) cudaStreamDestroy(s2.stream);
      }
      delete S;
      return rc;
    }
  }
  for (int i = 0; i < c.slots; ++i) S->slots[i].thread = std::thread(worker, S, i);
  *out = S;
  return MAP_OK;
}

int map_server_submit(map_server* S, const map_request* req, int64_t* ticket) {
  if (!S || !req || !ticket) return MAP_EINVAL;
  const map_request& r = *req;
  if (r.n <= 0 || !r.x || !r.y || !r.z || !r.m || r.ncell <= 0 || r.nface < 4 * r.ncell || r.nloop < 3 * r.nface ||
      r.nvert <= 0 || !r.cell_face_off || !r.face_vert_off || !r.face_vert || !r.face_plane || !r.vx || !r.vy ||
      !r.vz || !r.site || !r.cell_mass)
    return MAP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) return MAP_EINVAL;
  const int64_t t = S->next_ticket++;
  map_server::Rec& R = S->recs[t];
  R.req = r;
  R.res = map_request_result{};
  R.res.status = MAP_OK;
  R.t_submit = std::chrono::steady_clock::now();
  S->queue.push_back(t);
  admit(S);
  *ticket = t;
  return MAP_OK;
}

int map_server_wait(map_server* S, int64_t ticket, map_request_result* res) {
  if (!S) return MAP_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->recs.find(ticket);
  if (it == S->recs.end()) return MAP_EINVAL;
  S->cv_done.wait(lk, [&] { return S->recs[ticket].done; });
  if (res) *res = S->recs[ticket].res;
  S->recs.erase(ticket);
  return MAP_OK;
}

int map_server_stats(map_server* S, int64_t* completed, int* running, int64_t* queued, size_t* held_bytes) {
  if (!S) return MAP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  int run = 0;
  size_t held = 0;
  for (auto& s : S->slots) {
    run += s.busy ? 1 : 0;
    held += s.busy ? (s.reserved > cached_bytes(s) ? s.reserved : cached_bytes(s)) : cached_bytes(s);
  }
  if (completed) *completed = S->completed;
  if (running) *running = run;
  if (queued) *queued = (int64_t)S->queue.size();
  if (held_bytes) *held_bytes = held;
  return MAP_OK;
}

void map_server_destroy(map_server* S) {
  if (!S) return;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // queued requests that never started are failed; running ones finish
    for (int64_t t : S->queue) {
      S->recs[t].res.status = MAP_EINVAL;
      S->recs[t].done = true;
    }
    S->queue.clear();
    S->cv_done.notify_all();
    S->cv_done.wait(lk, [&] {
      for (auto& s : S->slots)
        if (s.busy) return false;
      return true;
    });
    S->stopping = true;
    S->cv_work.notify_all();
  }
  for (auto& sl : S->slots) {
    if (sl.thread.joinable()) sl.thread.join();
    if (sl.ctx) map_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete S;
}

}  // extern "C"
