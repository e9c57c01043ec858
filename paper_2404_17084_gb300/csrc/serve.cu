// Serving loop: continuous batching of mapping requests on one GPU.
//
// A server owns `slots` workers.  Each worker has its own context (octree,
// pair-list and integral workspace, kept allocated between requests), its own
// non-blocking CUDA stream, a pinned staging ring and a host thread, so the
// requests of different slots overlap on the device.  Requests are queued
// FIFO as they arrive; the admission step starts the oldest queued request
// as soon as a slot is idle AND its device-memory estimate fits the server's
// HBM budget next to what the running requests hold, what idle slots keep
// cached and the resident grids (idle caches, then the least recently used
// resident grids no running request uses, are released when that makes
// room).
//
// Grids stay resident on the device: a request with grid_id >= 0 uploads and
// prepares its grid only if no resident grid has that id; later requests on
// the same id map onto the resident copy (the server's grid context owns it),
// from any slot.  A request with a negative id gets a grid of its own for
// its duration.  A running request copies its particles in through its
// slot's pinned ring, solves h (Eq. 7-9), builds its octree and pair list
// and maps the particles (Eq. 1-3) on its slot, then copies the cell masses
// back through the ring.  Nothing waits for the whole device: allocation and
// release are stream-ordered on the slot's stream.  Each result depends only
// on its own request: a request gives the same bits alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {
constexpr size_t STAGE_BYTES = 8u << 20;  // each of a slot's two pinned staging buffers
}

struct map_server {
  map_server_config cfg;
  struct Slot {
    map_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread thread;
    bool busy = false;
    int64_t ticket = -1;    // request being run
    size_t reserved = 0;    // its admission estimate
    unsigned char* pin[2] = {nullptr, nullptr};  // pinned staging ring
    cudaEvent_t pev[2] = {nullptr, nullptr};     // last copy through each half
  };
  struct Rec {
    map_request req;
    map_request_result res;
    bool done = false;
    std::chrono::steady_clock::time_point t_submit, t_admit;
  };
  // A resident grid.  refs: running requests mapping onto it (it is not
  // evicted while > 0); ready: prepared (a request that finds it not ready
  // waits for the one preparing it).
  struct GridRec {
    PreparedGrid* g = nullptr;
    int refs = 0;
    bool ready = false;
    int status = MAP_OK;
    size_t bytes = 0;
    uint64_t last_use = 0;
  };
  std::vector<Slot> slots;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Rec> recs;
  std::unordered_map<int64_t, GridRec> grids;
  map_ctx* gctx = nullptr;           // owns the resident grids' device memory
  std::mutex gmu;                    // one grid preparation at a time in gctx
  std::mutex mu;
  std::condition_variable cv_work;   // workers wait for an admitted request
  std::condition_variable cv_done;   // callers wait for results
  std::condition_variable cv_grid;   // requests wait for a grid another one prepares
  int64_t next_ticket = 0;
  int64_t completed = 0;
  int64_t grid_uploads = 0, grid_hits = 0;
  uint64_t tick = 0;
  bool stopping = false;
};

namespace {

double ms_between(std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes of a prepared grid (its copy of the CSR and the geometry the
// precision keeps: 12 floats per loop entry for the mixed build, 12 doubles
// for FP64), with 25% headroom.
size_t grid_bytes(const map_request& r, int precision) {
  const double loop = precision != MAP_FP64 ? 64.0 : 112.0;
  return (size_t)(1.25 * (96.0 * r.ncell + 146.0 * r.nface + loop * r.nloop + 48.0 * r.nvert));
}

// Device bytes a request may hold beside its grid: its input copies, the
// octree, the pair list (160 pairs per particle assumed: FP64 fraction and
// two index arrays) and the per-cell outputs, with 25% headroom.
size_t work_bytes(const map_request& r) {
  const double parts = 48.0 * r.n + 200.0 * r.n + 160.0 * 16.0 * r.n;
  const double outs = 24.0 * r.ncell;
  return (size_t)(1.25 * (parts + outs)) + (64u << 20);
}

// Context workspace kept by an idle slot.
size_t cached_bytes(const map_server::Slot& s) { return s.ctx ? s.ctx->bytes_in_use : 0; }

// Frees an idle slot's workspace and its pool of released grid buffers (not
// its grids) in stream order on the slot's own stream, whose work has
// finished; the next request reallocates.  No other slot waits.
void trim(map_ctx* ctx, cudaStream_t s) {
  cudaSetDevice(ctx->device);
  ctx->cur_stream = s;
  auto drop = [&](DevBuf& b) {
    if (b.p) { dev_free(ctx, b.p); ctx->bytes_in_use -= b.cap; b.p = nullptr; b.cap = 0; }
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

// Frees a resident grid that no running request uses (mu held).  Its users
// have finished and synchronised their streams, so the buffers go back to
// the allocator's pool at once.
void evict(map_server* S, std::unordered_map<int64_t, map_server::GridRec>::iterator it) {
  PreparedGrid* g = it->second.g;
  if (g) {
    S->gctx->cur_stream = nullptr;
    for (const DevBuf& b : g->allocs) dev_free(S->gctx, b.p);
    S->gctx->bytes_in_use -= g->bytes;
    delete g;
  }
  S->grids.erase(it);
}

size_t resident_bytes(const map_server* S) {
  size_t b = 0;
  for (auto& kv : S->grids) b += kv.second.ready ? kv.second.bytes : 0;
  return b;
}

// Bytes held (mu held): running requests' estimates or their slots' caches,
// idle slots' caches, the resident grids.
size_t held_bytes(const map_server* S) {
  size_t h = resident_bytes(S);
  for (auto& s : S->slots) h += s.busy ? (s.reserved > cached_bytes(s) ? s.reserved : cached_bytes(s)) : cached_bytes(s);
  return h;
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
    // a grid already resident (or being prepared) costs nothing more
    const bool resident = R.req.grid_id >= 0 && S->grids.count(R.req.grid_id);
    const size_t need = work_bytes(R.req) + (resident ? 0 : grid_bytes(R.req, S->cfg.precision));
    auto in_use = [&]() { return held_bytes(S) - cached_bytes(S->slots[free_slot]); };
    if (S->cfg.hbm_budget && in_use() + need > S->cfg.hbm_budget) {
      // release the caches of idle slots, then unused resident grids, oldest first
      for (auto& s : S->slots)
        if (!s.busy && s.ctx) trim(s.ctx, s.stream);
      while (in_use() + need > S->cfg.hbm_budget) {
        auto victim = S->grids.end();
        for (auto it = S->grids.begin(); it != S->grids.end(); ++it)
          if (it->second.ready && it->second.refs == 0 && it->first != R.req.grid_id &&
              (victim == S->grids.end() || it->second.last_use < victim->second.last_use))
            victim = it;
        if (victim == S->grids.end()) break;
        evict(S, victim);
      }
      if (in_use() + need > S->cfg.hbm_budget) {
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

// Host -> device through the slot's pinned ring: a chunk is copied into one
// half while the other half's transfer runs.
int h2d_staged(map_server::Slot& sl, void* dst, const void* src, size_t bytes) {
  const unsigned char* in = static_cast<const unsigned char*>(src);
  unsigned char* out = static_cast<unsigned char*>(dst);
  int k = 0;
  for (size_t off = 0; off < bytes; off += STAGE_BYTES, k ^= 1) {
    const size_t n = bytes - off < STAGE_BYTES ? bytes - off : STAGE_BYTES;
    CUDA_TRY(cudaEventSynchronize(sl.pev[k]));  // this half's previous transfer is done
    std::memcpy(sl.pin[k], in + off, n);
    CUDA_TRY(cudaMemcpyAsync(out + off, sl.pin[k], n, cudaMemcpyHostToDevice, sl.stream));
    CUDA_TRY(cudaEventRecord(sl.pev[k], sl.stream));
  }
  return MAP_OK;
}

// Device -> host through the ring: the next chunk transfers while the last
// one is copied out.
int d2h_staged(map_server::Slot& sl, void* dst, const void* src, size_t bytes) {
  unsigned char* out = static_cast<unsigned char*>(dst);
  const unsigned char* in = static_cast<const unsigned char*>(src);
  size_t prev_off = 0, prev_n = 0;
  int prev_k = -1, k = 0;
  for (size_t off = 0; off < bytes; off += STAGE_BYTES, k ^= 1) {
    const size_t n = bytes - off < STAGE_BYTES ? bytes - off : STAGE_BYTES;
    CUDA_TRY(cudaEventSynchronize(sl.pev[k]));
    CUDA_TRY(cudaMemcpyAsync(sl.pin[k], in + off, n, cudaMemcpyDeviceToHost, sl.stream));
    CUDA_TRY(cudaEventRecord(sl.pev[k], sl.stream));
    if (prev_k >= 0) {
      CUDA_TRY(cudaEventSynchronize(sl.pev[prev_k]));
      std::memcpy(out + prev_off, sl.pin[prev_k], prev_n);
    }
    prev_off = off;
    prev_n = n;
    prev_k = k;
  }
  if (prev_k >= 0) {
    CUDA_TRY(cudaEventSynchronize(sl.pev[prev_k]));
    std::memcpy(out + prev_off, sl.pin[prev_k], prev_n);
  }
  return MAP_OK;
}

// Copies a request's grid in (through the ring, into temporary device
// arrays) and prepares it: into the slot's context (out_h: its handle) or,
// for a resident grid, into the server's grid context (out_g).
int upload_grid(map_server* S, map_server::Slot& sl, const map_request& q, map_ctx* into, PreparedGrid** out_g,
                int* out_h) {
  cudaStream_t s = sl.stream;
  int64_t *cfo = nullptr, *fvo = nullptr;
  int32_t* fv = nullptr;
  double *plane = nullptr, *vx = nullptr, *vy = nullptr, *vz = nullptr, *site = nullptr;
  std::vector<void*> tmp;
  auto tget = [&](auto** p, size_t bytes) -> int {
    void* v = nullptr;
    if (cudaMallocAsync(&v, bytes > 0 ? bytes : 16, s) != cudaSuccess) { cudaGetLastError(); return MAP_ENOMEM; }
    tmp.push_back(v);
    *p = reinterpret_cast<std::remove_pointer_t<decltype(p)>>(v);
    return MAP_OK;
  };
  int r = MAP_OK;
  if ((r = tget(&cfo, (q.ncell + 1) * sizeof(int64_t))) || (r = tget(&fvo, (q.nface + 1) * sizeof(int64_t))) ||
      (r = tget(&fv, q.nloop * sizeof(int32_t))) || (r = tget(&plane, 4 * q.nface * sizeof(double))) ||
      (r = tget(&vx, q.nvert * sizeof(double))) || (r = tget(&vy, q.nvert * sizeof(double))) ||
      (r = tget(&vz, q.nvert * sizeof(double))) || (r = tget(&site, 3 * q.ncell * sizeof(double)))) {
  } else if ((r = h2d_staged(sl, cfo, q.cell_face_off, (q.ncell + 1) * sizeof(int64_t))) ||
             (r = h2d_staged(sl, fvo, q.face_vert_off, (q.nface + 1) * sizeof(int64_t))) ||
             (r = h2d_staged(sl, fv, q.face_vert, q.nloop * sizeof(int32_t))) ||
             (r = h2d_staged(sl, plane, q.face_plane, 4 * q.nface * sizeof(double))) ||
             (r = h2d_staged(sl, vx, q.vx, q.nvert * sizeof(double))) ||
             (r = h2d_staged(sl, vy, q.vy, q.nvert * sizeof(double))) ||
             (r = h2d_staged(sl, vz, q.vz, q.nvert * sizeof(double))) ||
             (r = h2d_staged(sl, site, q.site, 3 * q.ncell * sizeof(double)))) {
  } else {
    const map_grid mg{q.ncell, q.nface, q.nloop, q.nvert, cfo, fvo, fv, plane, vx, vy, vz, site};
    if (out_h) {
      r = map_grid_upload(into, &mg, out_h, s);
    } else {
      // the server's grid context: one preparation at a time (its pool and
      // byte count are shared); preparation synchronises this stream
      std::lock_guard<std::mutex> lk(S->gmu);
      PreparedGrid* g = new (std::nothrow) PreparedGrid();
      if (!g) {
        r = MAP_ENOMEM;
      } else {
        into->cur_stream = s;
        r = grid_prepare(into, &mg, g, s);
        if (r != MAP_OK) {
          cudaStreamSynchronize(s);
          for (const DevBuf& b : g->allocs) dev_free(into, b.p);
          into->bytes_in_use -= g->bytes;
          delete g;
          g = nullptr;
        }
        *out_g = g;
      }
    }
  }
  for (void* v : tmp) cudaFreeAsync(v, s);
  if (r != MAP_OK) cudaGetLastError();
  return r;
}

// The resident grid of q.grid_id for this request: found (counted as a
// hit), waited for while another request prepares it, or prepared here.
int acquire_grid(map_server* S, map_server::Slot& sl, const map_request& q, PreparedGrid** g) {
  *g = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->grids.find(q.grid_id);
    if (it != S->grids.end()) {
      it->second.refs++;
      S->cv_grid.wait(lk, [&] {
        auto jt = S->grids.find(q.grid_id);
        return jt == S->grids.end() || jt->second.ready || jt->second.status != MAP_OK;
      });
      auto jt = S->grids.find(q.grid_id);
      if (jt == S->grids.end()) return MAP_ECUDA;
      if (jt->second.status != MAP_OK) {
        const int r = jt->second.status;
        if (--jt->second.refs == 0) S->grids.erase(jt);
        return r;
      }
      *g = jt->second.g;
      ++S->grid_hits;
      return MAP_OK;
    }
    S->grids[q.grid_id].refs = 1;  // not ready: later requests on this id wait
  }
  PreparedGrid* ng = nullptr;
  const int r = upload_grid(S, sl, q, S->gctx, &ng, nullptr);
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->grids.find(q.grid_id);
  if (r == MAP_OK) {
    it->second.g = ng;
    it->second.bytes = ng->bytes;
    it->second.ready = true;
    *g = ng;
    ++S->grid_uploads;
  } else {
    it->second.status = r;
    if (--it->second.refs == 0) S->grids.erase(it);
  }
  S->cv_grid.notify_all();
  return r;
}

void release_grid(map_server* S, int64_t id) {
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->grids.find(id);
  if (it != S->grids.end()) {
    it->second.refs--;
    it->second.last_use = ++S->tick;
  }
}

// Runs one request on a slot (no lock held).
int run_request(map_server* S, map_server::Slot& sl, const map_request& q, map_request_result& res) {
  map_ctx* ctx = sl.ctx;
  cudaStream_t s = sl.stream;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t sz_p = q.n * sizeof(double);
  double *x = nullptr, *y = nullptr, *z = nullptr, *m = nullptr, *h = nullptr, *mass = nullptr, *rho = nullptr;
  std::vector<void*> owned;
  auto get = [&](auto** p, size_t bytes) -> int {
    void* v = nullptr;
    if (cudaMallocAsync(&v, bytes > 0 ? bytes : 16, s) != cudaSuccess) { cudaGetLastError(); return MAP_ENOMEM; }
    owned.push_back(v);
    *p = reinterpret_cast<std::remove_pointer_t<decltype(p)>>(v);
    return MAP_OK;
  };
  int rc = MAP_OK;
  if ((rc = get(&x, sz_p)) || (rc = get(&y, sz_p)) || (rc = get(&z, sz_p)) || (rc = get(&m, sz_p)) ||
      (rc = get(&h, sz_p)) || (rc = get(&mass, q.ncell * sizeof(double))) ||
      (rc = get(&rho, q.ncell * sizeof(double)))) {
  } else if ((rc = h2d_staged(sl, x, q.x, sz_p)) || (rc = h2d_staged(sl, y, q.y, sz_p)) ||
             (rc = h2d_staged(sl, z, q.z, sz_p)) || (rc = h2d_staged(sl, m, q.m, sz_p))) {
  }
  // the grid: resident under q.grid_id, or the request's own
  PreparedGrid* rg = nullptr;
  int handle = -1;
  if (rc == MAP_OK) rc = q.grid_id >= 0 ? acquire_grid(S, sl, q, &rg) : upload_grid(S, sl, q, ctx, nullptr, &handle);
  map_particles p{q.n, x, y, z, m, h};
  map_stats st{};
  if (rc == MAP_OK) rc = solve_h(ctx, &p, nullptr, s);
  map_outputs out{mass, rho, nullptr};
  if (rc == MAP_OK) {
    if (rg) {
      rc = ctx_enter(ctx, s);
      if (rc == MAP_OK) {
        CallScope scope{ctx, s};
        rc = map_run(ctx, &p, rg, &out, s);
      }
    } else {
      rc = map_particles_to_cells(ctx, &p, handle, &out, s);
    }
  }
  if (rc == MAP_OK) rc = map_get_stats(ctx, &st);
  if (rc == MAP_OK) rc = d2h_staged(sl, q.cell_mass, mass, q.ncell * sizeof(double));
  if (rc == MAP_OK && q.cell_rho) rc = d2h_staged(sl, q.cell_rho, rho, q.ncell * sizeof(double));
  if (rc == MAP_OK && q.h) rc = d2h_staged(sl, q.h, h, sz_p);
  if (rc != MAP_OK) cudaGetLastError();
  if (handle >= 0) map_grid_release(ctx, handle);
  for (void* v : owned) cudaFreeAsync(v, s);
  cudaStreamSynchronize(s);
  if (rg) release_grid(S, q.grid_id);
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
    const int rc = run_request(S, S->slots[i], q, res);
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

void free_slot_resources(map_server::Slot& sl) {
  if (sl.ctx) map_destroy(sl.ctx);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  for (auto& e : sl.pev) if (e) cudaEventDestroy(e);
  for (auto& p : sl.pin) if (p) cudaFreeHost(p);
  sl.ctx = nullptr;
  sl.stream = nullptr;
  sl.pev[0] = sl.pev[1] = nullptr;
  sl.pin[0] = sl.pin[1] = nullptr;
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
  map_config gc;
  map_config_default(&gc);
  gc.device = c.device;
  gc.precision = c.precision;
  gc.hfact = c.hfact;
  int rc = map_init(&S->gctx, &gc);
  for (auto& sl : S->slots) {
    if (rc != MAP_OK) break;
    rc = map_init(&sl.ctx, &gc);
    if (rc == MAP_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) rc = MAP_ECUDA;
    for (int k = 0; k < 2 && rc == MAP_OK; ++k)
      if (cudaEventCreateWithFlags(&sl.pev[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaMallocHost(&sl.pin[k], STAGE_BYTES) != cudaSuccess)
        rc = MAP_ENOMEM;
  }
  if (rc != MAP_OK) {
    cudaGetLastError();
    for (auto& s2 : S->slots) free_slot_resources(s2);
    if (S->gctx) map_destroy(S->gctx);
    delete S;
    return rc;
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

int map_server_stats(map_server* S, int64_t* completed, int* running, int64_t* queued, size_t* held) {
  if (!S) return MAP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  int run = 0;
  for (auto& s : S->slots) run += s.busy ? 1 : 0;
  if (completed) *completed = S->completed;
  if (running) *running = run;
  if (queued) *queued = (int64_t)S->queue.size();
  if (held) *held = held_bytes(S);
  return MAP_OK;
}

int map_server_grid_stats(map_server* S, int64_t* uploads, int64_t* hits, int64_t* resident, size_t* bytes) {
  if (!S) return MAP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  int64_t n = 0;
  for (auto& kv : S->grids) n += kv.second.ready ? 1 : 0;
  if (uploads) *uploads = S->grid_uploads;
  if (hits) *hits = S->grid_hits;
  if (resident) *resident = n;
  if (bytes) *bytes = resident_bytes(S);
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
    free_slot_resources(sl);
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    while (!S->grids.empty()) evict(S, S->grids.begin());
  }
  if (S->gctx) map_destroy(S->gctx);
  delete S;
}

}  // extern "C"
