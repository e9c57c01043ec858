// Batched mapping: many independent snapshots (particle set + resident grid)
// in one persistent pair-integral launch.
//
// Each snapshot's octree and pair list are built by one of the context's
// workers: BATCH_WORKERS worker contexts, each with its own workspace,
// stream and host thread; worker w takes snapshots w, w + 8, ... of the
// largest-first order (these steps size their buffers from device counts and
// so synchronise their stream; running several at once keeps the GPU busy
// between those points).  A call that repeats an earlier one replays the
// whole step as one CUDA graph instead (see the graph section below).  The pair lists
// are written to per-snapshot buffers of the context, reused by later
// batches of the same shape.  solve_h_batch solves the snapshots' smoothing
// lengths on the same workers.  The pair
// integrals of every snapshot then run in ONE launch of the persistent
// kernel: its device work queue hands out the cells of all snapshots, the
// snapshots laid out largest pair count first (longest-processing-time
// order), so that the last cells handed out are those of the smallest
// snapshots and the tail of the launch is short.  The descriptor upload, the
// launch and the per-snapshot mass sums are captured once in a CUDA graph and
// replayed while the batch's descriptors are byte-identical.
//
// Autotuner: with map_config.autotune set, the first mapping call of a
// context in the mixed build (a batch, or a single snapshot) times the
// integral launch on its own inputs for every pair of a work-item size (the
// target number of items per resident warp, 16, 64 or 256: smaller items
// spread large cells over more warps) and a launch shape (warps per CTA and
// CTAs per SM, hence the register cap per thread), and keeps the fastest pair
// for every later call of the context.  Each choice is deterministic; two
// shapes are separate compilations of the same source and may round FP32
// differently, and two item sizes add a cell's pairs in different groups.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>

#include "internal.cuh"

namespace {

__global__ void sum_totals(int n, const double* __restrict__ v, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += v[i];
    *out = t;
  }
}

constexpr int BATCH_WORKERS = 8;

int ensure_workers(map_ctx* ctx) {
  if (!ctx->wev) CUDA_TRY(cudaEventCreateWithFlags(&ctx->wev, cudaEventDisableTiming));
  while ((int)ctx->workers.size() < BATCH_WORKERS) {
    map_config c = ctx->cfg;
    c.autotune = 0;
    c.count_work = 0;
    c.hbm_budget = 0;  // the workers' workspace is not counted against the budget
    BatchWorker w;
    MAP_TRY(map_init(&w.ctx, &c));
    if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (w.stream) cudaStreamDestroy(w.stream);
      map_destroy(w.ctx);
      return MAP_ECUDA;
    }
    ctx->workers.push_back(w);
  }
  return MAP_OK;
}

int ensure_stream(map_ctx* ctx) {
  if (!ctx->bstream) CUDA_TRY(cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking));
  for (auto& e : ctx->bev)
    if (!e) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return MAP_OK;
}

// Graph replays: each snapshot's item count (its pair and item counts
// checked against the buffers' capacities), the queue bases in queue order,
// and the step's totals -- [0] items, [1] pairs, then the flags word: 1 an
// invalid particle, 2 a list or item count beyond its buffer.
__global__ void batch_bases(const SnapDesc* __restrict__ d, int nsnap, const int64_t* __restrict__ caps,
                            const unsigned long long* __restrict__ invalid, int64_t* ibase, int64_t* totals) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t items = 0, pairs = 0, bad = 0;
  for (int q = 0; q < nsnap; ++q) {
    const SnapDesc& D = d[q];
    ibase[q] = items;
    const int64_t np = D.pair_off[D.ncell], ni = D.item_off[D.ncell];
    if (invalid[q]) bad |= 1;
    if (np > caps[2 * q] || ni > caps[2 * q + 1]) bad |= 2;
    items += ni;
    pairs += np;
  }
  ibase[nsnap] = items;
  totals[0] = items;
  totals[1] = pairs;
  totals[2] = bad;
}

}  // namespace

void destroy_workers(map_ctx* ctx) {
  for (BatchWorker& w : ctx->workers) {
    if (w.stream) cudaStreamSynchronize(w.stream);
    map_destroy(w.ctx);  // before its stream goes
    if (w.done) cudaEventDestroy(w.done);
    if (w.stream) cudaStreamDestroy(w.stream);
  }
  ctx->workers.clear();
  if (ctx->wev) cudaEventDestroy(ctx->wev);
  ctx->wev = nullptr;
}

int run_on_workers(map_ctx* ctx, int n, const int* order, cudaStream_t s,
                   const std::function<int(BatchWorker&, int)>& fn) {
  MAP_TRY(ensure_workers(ctx));
  CUDA_TRY(cudaEventRecord(ctx->wev, s));
  std::vector<int64_t> l0(ctx->workers.size());
  for (size_t w = 0; w < ctx->workers.size(); ++w) {
    CUDA_TRY(cudaStreamWaitEvent(ctx->workers[w].stream, ctx->wev, 0));
    l0[w] = ctx->workers[w].ctx->launches;
  }
  // static assignment: worker w takes order[w], order[w + W], ... (the same
  // snapshots every call, so that each worker's workspace settles at the
  // sizes of its own snapshots, which the whole-step graph bakes in)
  std::atomic<int> err{MAP_OK};
  const int nw = (int)ctx->workers.size();
  std::vector<std::thread> th;
  for (size_t w = 0; w < ctx->workers.size(); ++w)
    th.emplace_back([&, w]() {
      BatchWorker& W = ctx->workers[w];
      if (cudaSetDevice(ctx->device) != cudaSuccess) { int e = MAP_OK; err.compare_exchange_strong(e, MAP_ECUDA); }
      for (int i = (int)w;; i += nw) {
        if (err.load() != MAP_OK) break;
        if (i >= n) break;
        const int r = fn(W, order[i]);
        if (r != MAP_OK) {
          int e = MAP_OK;
          err.compare_exchange_strong(e, r);
          break;
        }
      }
      cudaEventRecord(W.done, W.stream);
    });
  for (auto& t : th) t.join();
  for (size_t w = 0; w < ctx->workers.size(); ++w) {
    CUDA_TRY(cudaStreamWaitEvent(s, ctx->workers[w].done, 0));
    ctx->launches += ctx->workers[w].ctx->launches - l0[w];
  }
  return err.load();
}

// Times every (work-item target, launch shape) pair of the integral launch on
// the call's own inputs (rebuilding the work items for each target) and keeps
// the fastest pair; the items are left built for the chosen target.
int integrals_autotune(map_ctx* ctx, const std::function<int(int, BatchArgs&)>& rebuild, BatchArgs& B,
                       cudaStream_t s) {
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int best_t = 0, best_v = 0;
  float best_ms = 0.f;
  int rc = MAP_OK;
  for (int t = 0; t < N_TARGETS && rc == MAP_OK; ++t) {
    BatchArgs Bt;
    rc = rebuild(ITEM_TARGETS[t], Bt);
    for (int v = 0; v < N_SHAPES && rc == MAP_OK; ++v) {
      cudaEventRecord(e0, s);
      rc = integrals_enqueue(ctx, Bt, v, s);
      cudaEventRecord(e1, s);
      if (rc != MAP_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = MAP_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ctx->tune_ms[t * N_SHAPES + v] = ms;
      if ((t == 0 && v == 0) || ms < best_ms) { best_t = t; best_v = v; best_ms = ms; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MAP_OK) return rc;
  MAP_TRY(rebuild(ITEM_TARGETS[best_t], B));
  ctx->item_target = ITEM_TARGETS[best_t];
  ctx->tuned[MAP_MIXED] = best_v;
  ctx->tune_done[MAP_MIXED] = true;
  return MAP_OK;
}

// ---------------------------------------------------------------- the step as one graph
// After an eager map_batch, the context captures the whole step -- per
// snapshot (on the workers' streams, each snapshot on the worker
// run_on_workers gives it): reset of its flag, particle validation, the octree
// (tree_build_graph), the pair list and work items (pairs_build_graph, into
// the snapshot's slots, sized a quarter above the eager call's counts); then
// on the batch stream: descriptors, the queue bases from the device counts
// (batch_bases), the one persistent integral launch, the cell and snapshot
// sums.  A later call that names the same particle buffers, grids, outputs
// and launch choices replays it with one graph launch and one read of three
// words (item and pair totals, flags).  Flags 1 (invalid particles): the call
// returns MAP_EINVAL.  Flags 2 (a list outgrew its slot): the integral launch
// skipped itself, the call falls back to the eager step, which captures
// anew.

static int64_t* gtot(map_ctx* ctx) { return static_cast<int64_t*>(ctx->bgraph.tot.p); }

static void graph_drop(map_ctx* ctx, map_ctx::BatchGraph& G) {
  if (G.exec) {
    if (ctx->bstream) cudaStreamSynchronize(ctx->bstream);  // a replay may still run
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  // freed on the context's own batch stream, where they were last used (the
  // caller's stream of the last call may no longer exist)
  for (DevBuf* b : {&G.desc, &G.base, &G.tot, &G.caps, &G.flags}) {
    if (b->p) {
      cudaFreeAsync(b->p, ctx->bstream);
      ctx->bytes_in_use -= b->cap;
    }
    *b = DevBuf();
  }
  G.sig.clear();
  G.bufs.clear();
}

void batch_graph_drop(map_ctx* ctx) {
  graph_drop(ctx, ctx->bgraph);
  graph_drop(ctx, ctx->hgraph);
}

namespace {

// what the graph bakes in from the call: every input and output pointer,
// sizes, grids, launch choices
std::vector<unsigned char> graph_sig(map_ctx* ctx, int nsnap, const map_particles* parts, const int* grids,
                                     const map_outputs* outs) {
  std::vector<unsigned char> v;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    v.insert(v.end(), c, c + n);
  };
  const int64_t head[6] = {nsnap, ctx->cfg.precision, ctx->tuned[ctx->cfg.precision == MAP_MIXED ? MAP_MIXED : MAP_FP64],
                           ctx->item_target, ctx->cfg.leaf_size, ctx->cfg.count_work};
  put(head, sizeof(head));
  for (int j = 0; j < nsnap; ++j) {
    const map_particles& p = parts[j];
    const void* ptr[9] = {p.x, p.y, p.z, p.m, p.h, ctx->grids[grids[j]], outs[j].cell_mass, outs[j].cell_rho,
                          reinterpret_cast<const void*>((intptr_t)grids[j])};
    put(ptr, sizeof(ptr));
    put(&p.n, sizeof(p.n));
  }
  return v;
}

// every workspace allocation the graph reads or writes
std::vector<const void*> graph_bufs(map_ctx* ctx, int nsnap, const map_ctx::BatchGraph& G) {
  std::vector<const void*> v;
  for (BatchWorker& W : ctx->workers) {
    map_ctx* c = W.ctx;
    for (auto& b : c->ws_tree) v.push_back(b.p);
    for (auto& b : c->ws_pairs) v.push_back(b.p);
    for (auto& b : c->ws_misc) v.push_back(b.p);
    v.push_back(c->cub_tmp.p);
    v.push_back(c->d_counters);
  }
  for (auto* vec : {&ctx->batch_off, &ctx->batch_idx, &ctx->batch_itm, &ctx->batch_ioff, &ctx->batch_part})
    for (int j = 0; j < nsnap; ++j) v.push_back((*vec)[j].p);
  for (const DevBuf* b : {&G.desc, &G.base, &G.tot, &G.caps, &G.flags}) v.push_back(b->p);
  v.push_back(ctx->d_counters);
  v.push_back(ctx->d_total);
  return v;
}

// a phase event inside a capture becomes an event-record node of the graph
inline void gphase(map_ctx* ctx, int k, bool end, cudaStream_t s, bool capturing) {
  cudaEvent_t e = ctx->ev[2 * k + (end ? 1 : 0)];
  if (!e) return;
  if (capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
  if (end) ctx->ev_used[k] = true;
}

// The step's work, enqueued on the batch stream and the workers' streams
// (eagerly, or into a capture on the batch stream).  order: the queue's
// snapshot order; caps: per queue position, pair and item capacities.
int graph_enqueue(map_ctx* ctx, int nsnap, const map_particles* parts, const int* grids, const map_outputs* outs,
                  const std::vector<int>& order, const std::vector<int64_t>& caps, bool capturing) {
  // snapshot -> worker as run_on_workers assigns them (largest first, w mod 8)
  std::vector<int> big(nsnap), wof(nsnap);
  std::iota(big.begin(), big.end(), 0);
  std::stable_sort(big.begin(), big.end(), [&](int a, int b) { return parts[a].n > parts[b].n; });
  auto& G = ctx->bgraph;
  cudaStream_t bs = ctx->bstream;
  const int W = (int)ctx->workers.size();
  for (int r = 0; r < nsnap; ++r) wof[big[r]] = r % W;
  SnapDesc* d_desc = static_cast<SnapDesc*>(G.desc.p);
  int64_t* d_ibase = static_cast<int64_t*>(G.base.p);
  int64_t* d_cbase = d_ibase + nsnap + 1;
  double* d_tot = reinterpret_cast<double*>(gtot(ctx) + 4);
  const int64_t* d_caps = static_cast<const int64_t*>(G.caps.p);
  unsigned long long* d_invalid = static_cast<unsigned long long*>(G.flags.p);
  gphase(ctx, 1, false, bs, capturing);
  CUDA_TRY(cudaEventRecord(ctx->wev, bs));
  for (BatchWorker& Wk : ctx->workers) CUDA_TRY(cudaStreamWaitEvent(Wk.stream, ctx->wev, 0));
  std::vector<SnapDesc> qd(nsnap);
  std::vector<int64_t> ib(nsnap + 1, 0), cb(nsnap + 1, 0);
  int64_t item_bound = 0;
  for (int q = 0; q < nsnap; ++q) {
    const int j = order[q];
    BatchWorker& Wk = ctx->workers[wof[j]];
    map_ctx* wc = Wk.ctx;
    wc->cur_stream = Wk.stream;  // no ctx_enter: this stream is ordered by the fork above
    wc->item_target = ctx->item_target;
    const map_particles* p = &parts[j];
    const PreparedGrid* g = ctx->grids[grids[j]];
    CUDA_TRY(cudaMemsetAsync(d_invalid + q, 0, sizeof(unsigned long long), Wk.stream));
    MAP_TRY(validate_enqueue(wc, p, true, true, d_invalid + q, Wk.stream));
    MAP_TRY(tree_build_graph(wc, p->x, p->y, p->z, p->m, p->h, p->n, Wk.stream));
    PairBufs pb;
    pb.off = &ctx->batch_off[j];
    pb.idx = &ctx->batch_idx[j];
    pb.items = &ctx->batch_itm[j];
    pb.ioff = &ctx->batch_ioff[j];
    pb.part = &ctx->batch_part[j];
    MAP_TRY(pairs_build_graph(wc, g, Wk.stream, pb, caps[2 * q], caps[2 * q + 1]));
    qd[q] = make_desc(wc, g, p, &outs[j], wc->pair_off, wc->pair_idx, nullptr, j);
    cb[q + 1] = cb[q] + g->ncell;
    item_bound += caps[2 * q + 1];
  }
  for (BatchWorker& Wk : ctx->workers) {
    CUDA_TRY(cudaEventRecord(Wk.done, Wk.stream));
    CUDA_TRY(cudaStreamWaitEvent(bs, Wk.done, 0));
  }
  gphase(ctx, 1, true, bs, capturing);
  MAP_TRY(integrals_upload(ctx, qd.data(), ib.data(), cb.data(), nsnap, d_desc, d_ibase, d_cbase, bs));
  batch_bases<<<1, 1, 0, bs>>>(d_desc, nsnap, d_caps, d_invalid, d_ibase, gtot(ctx)); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  BatchArgs B{d_desc, d_ibase, d_cbase, nsnap, item_bound, cb[nsnap], ctx->d_counters};
  B.total_dev = gtot(ctx);
  B.bad = gtot(ctx) + 2;
  const int prec = ctx->cfg.precision == MAP_MIXED ? MAP_MIXED : MAP_FP64;
  gphase(ctx, 2, false, bs, capturing);
  MAP_TRY(integrals_enqueue(ctx, B, ctx->tuned[prec], bs));
  gphase(ctx, 2, true, bs, capturing);
  MAP_TRY(integrals_sum(ctx, d_desc, nsnap, d_tot, bs));
  sum_totals<<<1, 32, 0, bs>>>(nsnap, d_tot, ctx->d_total); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

}  // namespace

namespace {

constexpr int GRAPH_FALLBACK = -1000;  // internal: the replay's lists outgrew their slots

// Captures the step after an eager call (np: the call's pair counts by
// snapshot; order: its queue order).  Any failure leaves no graph and the
// eager call's results in place.
int batch_graph_build(map_ctx* ctx, int nsnap, const map_particles* parts, const int* grids,
                      const map_outputs* outs, const std::vector<int64_t>& np, const std::vector<int>& order,
                      cudaStream_t s) {
  graph_drop(ctx, ctx->bgraph);
  auto& G = ctx->bgraph;
  MAP_TRY(ensure_workers(ctx));
  std::vector<int64_t> caps(2 * nsnap);
  for (int q = 0; q < nsnap; ++q) {
    const int j = order[q];
    const int64_t nc = ctx->grids[grids[j]]->ncell;
    const int64_t cp = np[j] + np[j] / 4 + 4096;
    caps[2 * q] = cp;
    caps[2 * q + 1] = nc + cp / 32 + 1;  // no more items than cells plus blocks of 32 pairs
  }
  SnapDesc* dd;
  int64_t *db, *dt, *dc;
  unsigned long long* df;
  MAP_TRY(ensure_t(ctx, G.desc, nsnap, &dd));
  MAP_TRY(ensure_t(ctx, G.base, 2 * (nsnap + 1), &db));
  MAP_TRY(ensure_t(ctx, G.tot, 4 + nsnap, &dt));
  MAP_TRY(ensure_t(ctx, G.caps, 2 * nsnap, &dc));
  MAP_TRY(ensure_t(ctx, G.flags, nsnap, &df));
  CUDA_TRY(cudaMemcpyAsync(dc, caps.data(), caps.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaEventRecord(ctx->bev[0], s));
  CUDA_TRY(cudaStreamWaitEvent(ctx->bstream, ctx->bev[0], 0));
  // 1. the step once, eagerly: every workspace gets its size here, not in
  // the capture (its results equal the eager call's)
  MAP_TRY(graph_enqueue(ctx, nsnap, parts, grids, outs, order, caps, false));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, gtot(ctx), 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->bstream));
  CUDA_TRY(cudaStreamSynchronize(ctx->bstream));
  if (ctx->h_scratch[2] != 0) return MAP_ECAPACITY;
  // 2. the same, captured
  const std::vector<const void*> bufs0 = graph_bufs(ctx, nsnap, ctx->bgraph);
  const int64_t l0 = ctx->launches;
  std::vector<int64_t> wl0;
  for (BatchWorker& W : ctx->workers) wl0.push_back(W.ctx->launches);
  CUDA_TRY(cudaStreamBeginCapture(ctx->bstream, cudaStreamCaptureModeThreadLocal));
  int rc = graph_enqueue(ctx, nsnap, parts, grids, outs, order, caps, true);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->bstream, &graph);
  int64_t launched = ctx->launches - l0;
  for (size_t w = 0; w < ctx->workers.size(); ++w) {
    launched += ctx->workers[w].ctx->launches - wl0[w];
    ctx->workers[w].ctx->launches = wl0[w];
  }
  ctx->launches = l0;
  if (rc != MAP_OK || ce != cudaSuccess || graph_bufs(ctx, nsnap, ctx->bgraph) != bufs0) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != MAP_OK ? rc : MAP_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    G.exec = nullptr;
    cudaGetLastError();
    return MAP_ECUDA;
  }
  G.sig = graph_sig(ctx, nsnap, parts, grids, outs);
  G.bufs = bufs0;
  G.launches = launched;
  ++G.captures;
  return MAP_OK;
}

// One graph launch and one read of the totals and flags.
int batch_graph_replay(map_ctx* ctx, int nsnap, const int* grids, const map_outputs* outs, double* totals,
                       cudaStream_t s) {
  auto& G = ctx->bgraph;
  CUDA_TRY(cudaEventRecord(ctx->bev[0], s));
  CUDA_TRY(cudaStreamWaitEvent(ctx->bstream, ctx->bev[0], 0));
  CUDA_TRY(cudaGraphLaunch(G.exec, ctx->bstream));
  ctx->launches += G.launches;
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, gtot(ctx), 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->bstream));
  CUDA_TRY(cudaStreamSynchronize(ctx->bstream));
  const int64_t bad = ctx->h_scratch[2];
  if (bad & 1) return MAP_EINVAL;
  if (bad & 2) {
    ++G.fallbacks;
    return GRAPH_FALLBACK;
  }
  ++G.replays;
  int64_t cells = 0;
  for (int j = 0; j < nsnap; ++j) cells += ctx->grids[grids[j]]->ncell;
  ctx->n_pairs = ctx->h_scratch[1];
  ctx->last_ncell = cells;
  ctx->pair_off = nullptr;  // no single pair list describes a batch
  ctx->pair_idx = nullptr;
  ctx->pair_frac = nullptr;
  ctx->inv_ready = false;
  ctx->items = nullptr;
  ctx->item_off = nullptr;
  ctx->partial = nullptr;
  const double* d_tot = reinterpret_cast<const double*>(gtot(ctx) + 4);
  if (totals) CUDA_TRY(cudaMemcpyAsync(totals, d_tot, nsnap * sizeof(double), cudaMemcpyDeviceToDevice, ctx->bstream));
  for (int j = 0; j < nsnap; ++j)
    if (outs[j].cell_vol) {
      const PreparedGrid* g = ctx->grids[grids[j]];
      CUDA_TRY(cudaMemcpyAsync(outs[j].cell_vol, g->vol, g->ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                               ctx->bstream));
    }
  CUDA_TRY(cudaEventRecord(ctx->bev[1], ctx->bstream));
  CUDA_TRY(cudaStreamWaitEvent(s, ctx->bev[1], 0));
  return MAP_OK;
}

}  // namespace

// ---------------------------------------------------------------- solve_h_batch as one graph
// The same scheme for solve_h_batch: per set (on the worker run_on_workers
// gives it) the validation and the h solve over an octree built without host
// reads; one flag word read back.  Replayed while the call names the same
// buffers (positions, h, routes) and sizes.

namespace {

__global__ void any_flag(int n, const unsigned long long* __restrict__ f, int64_t* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t b = 0;
  for (int i = 0; i < n; ++i) b |= f[i] ? 1 : 0;
  out[0] = b;
}

std::vector<unsigned char> hgraph_sig(map_ctx* ctx, int nsnap, const map_particles* parts, int32_t* const* routes) {
  std::vector<unsigned char> v;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    v.insert(v.end(), c, c + n);
  };
  const double hf = ctx->cfg.hfact;
  const int64_t head[3] = {nsnap, ctx->cfg.precision, ctx->cfg.leaf_size};
  put(head, sizeof(head));
  put(&hf, sizeof(hf));
  for (int j = 0; j < nsnap; ++j) {
    const void* ptr[5] = {parts[j].x, parts[j].y, parts[j].z, parts[j].h, routes ? routes[j] : nullptr};
    put(ptr, sizeof(ptr));
    put(&parts[j].n, sizeof(parts[j].n));
  }
  return v;
}

int hgraph_enqueue(map_ctx* ctx, int nsnap, map_particles* parts, int32_t* const* routes, bool capturing) {
  auto& G = ctx->hgraph;
  cudaStream_t bs = ctx->bstream;
  const int W = (int)ctx->workers.size();
  std::vector<int> big(nsnap);
  std::iota(big.begin(), big.end(), 0);
  std::stable_sort(big.begin(), big.end(), [&](int a, int b) { return parts[a].n > parts[b].n; });
  unsigned long long* flags = static_cast<unsigned long long*>(G.flags.p);
  gphase(ctx, 3, false, bs, capturing);
  CUDA_TRY(cudaEventRecord(ctx->wev, bs));
  for (BatchWorker& Wk : ctx->workers) CUDA_TRY(cudaStreamWaitEvent(Wk.stream, ctx->wev, 0));
  for (int r = 0; r < nsnap; ++r) {
    const int j = big[r];
    BatchWorker& Wk = ctx->workers[r % W];
    map_ctx* wc = Wk.ctx;
    wc->cur_stream = Wk.stream;
    map_particles* p = &parts[j];
    CUDA_TRY(cudaMemsetAsync(flags + j, 0, sizeof(unsigned long long), Wk.stream));
    MAP_TRY(validate_enqueue(wc, p, false, false, flags + j, Wk.stream));
    MAP_TRY(h_solve_run(wc, p->x, p->y, p->z, p->n, p->h, routes ? routes[j] : nullptr, nullptr, Wk.stream, true));
  }
  for (BatchWorker& Wk : ctx->workers) {
    CUDA_TRY(cudaEventRecord(Wk.done, Wk.stream));
    CUDA_TRY(cudaStreamWaitEvent(bs, Wk.done, 0));
  }
  any_flag<<<1, 1, 0, bs>>>(nsnap, flags, static_cast<int64_t*>(G.tot.p)); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  gphase(ctx, 3, true, bs, capturing);
  return MAP_OK;
}

int hgraph_build(map_ctx* ctx, int nsnap, map_particles* parts, int32_t* const* routes, cudaStream_t s) {
  auto& G = ctx->hgraph;
  graph_drop(ctx, G);
  MAP_TRY(ensure_workers(ctx));
  unsigned long long* f;
  int64_t* t;
  MAP_TRY(ensure_t(ctx, G.flags, nsnap, &f));
  MAP_TRY(ensure_t(ctx, G.tot, 4, &t));
  CUDA_TRY(cudaEventRecord(ctx->bev[0], s));
  CUDA_TRY(cudaStreamWaitEvent(ctx->bstream, ctx->bev[0], 0));
  MAP_TRY(hgraph_enqueue(ctx, nsnap, parts, routes, false));  // sizes every workspace
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, t, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->bstream));
  CUDA_TRY(cudaStreamSynchronize(ctx->bstream));
  if (ctx->h_scratch[0] != 0) return MAP_EINVAL;
  const std::vector<const void*> bufs0 = graph_bufs(ctx, 0, G);
  const int64_t l0 = ctx->launches;
  std::vector<int64_t> wl0;
  for (BatchWorker& W : ctx->workers) wl0.push_back(W.ctx->launches);
  CUDA_TRY(cudaStreamBeginCapture(ctx->bstream, cudaStreamCaptureModeThreadLocal));
  const int rc = hgraph_enqueue(ctx, nsnap, parts, routes, true);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->bstream, &graph);
  int64_t launched = ctx->launches - l0;
  for (size_t w = 0; w < ctx->workers.size(); ++w) {
    launched += ctx->workers[w].ctx->launches - wl0[w];
    ctx->workers[w].ctx->launches = wl0[w];
  }
  ctx->launches = l0;
  if (rc != MAP_OK || ce != cudaSuccess || graph_bufs(ctx, 0, G) != bufs0) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != MAP_OK ? rc : MAP_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    G.exec = nullptr;
    cudaGetLastError();
    return MAP_ECUDA;
  }
  G.sig = hgraph_sig(ctx, nsnap, parts, routes);
  G.bufs = bufs0;
  G.launches = launched;
  ++G.captures;
  return MAP_OK;
}

int hgraph_replay(map_ctx* ctx, cudaStream_t s) {
  auto& G = ctx->hgraph;
  CUDA_TRY(cudaEventRecord(ctx->bev[0], s));
  CUDA_TRY(cudaStreamWaitEvent(ctx->bstream, ctx->bev[0], 0));
  CUDA_TRY(cudaGraphLaunch(G.exec, ctx->bstream));
  ctx->launches += G.launches;
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, G.tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->bstream));
  CUDA_TRY(cudaStreamSynchronize(ctx->bstream));
  if (ctx->h_scratch[0] != 0) return MAP_EINVAL;
  ++G.replays;
  CUDA_TRY(cudaEventRecord(ctx->bev[1], ctx->bstream));
  CUDA_TRY(cudaStreamWaitEvent(s, ctx->bev[1], 0));
  return MAP_OK;
}

}  // namespace

// The host-side part of check_particles (pointers and count), for a batch
// before its workers start.
static bool check_sizes(const map_particles* p) {
  return p && p->n > 0 && p->n < (int64_t)INT32_MAX && p->x && p->y && p->z;
}

extern "C" {

int solve_h_batch(map_ctx* ctx, int nsnap, map_particles* parts, int32_t* const* routes, void* stream) {
  if (!ctx || nsnap < 1 || !parts) return MAP_EINVAL;
  for (int j = 0; j < nsnap; ++j)
    if (!check_sizes(&parts[j]) || !parts[j].h) return MAP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MAP_ENTER(ctx, s);
  MAP_TRY(ensure_stream(ctx));
  const bool graphable = ctx->cfg.count_work == 0;
  if (ctx->hgraph.exec) {
    if (graphable && ctx->hgraph.sig == hgraph_sig(ctx, nsnap, parts, routes) &&
        ctx->hgraph.bufs == graph_bufs(ctx, 0, ctx->hgraph))
      return hgraph_replay(ctx, s);
    graph_drop(ctx, ctx->hgraph);
  }
  std::vector<int> big(nsnap);
  std::iota(big.begin(), big.end(), 0);
  std::stable_sort(big.begin(), big.end(), [&](int a, int b) { return parts[a].n > parts[b].n; });
  phase_begin(ctx, 3, s);
  const int rc = run_on_workers(ctx, nsnap, big.data(), s, [&](BatchWorker& W, int j) -> int {
    map_particles* p = &parts[j];
    MAP_ENTER(W.ctx, W.stream);
    MAP_TRY(check_particles(W.ctx, p, false, false, W.stream));
    return h_solve_run(W.ctx, p->x, p->y, p->z, p->n, p->h, routes ? routes[j] : nullptr, nullptr, W.stream);
  });
  phase_end(ctx, 3, s);
  if (rc != MAP_OK) return rc;
  // capture the step for the calls that repeat this one (optional)
  if (graphable && hgraph_build(ctx, nsnap, parts, routes, s) != MAP_OK) {
    graph_drop(ctx, ctx->hgraph);
    cudaGetLastError();
  }
  return MAP_OK;
}


int map_batch(map_ctx* ctx, int nsnap, const map_particles* parts, const int* grids, const map_outputs* outs,
              double* totals, void* stream) {
  if (!ctx || nsnap < 1 || !parts || !grids || !outs) return MAP_EINVAL;
  for (int j = 0; j < nsnap; ++j) {
    if (grids[j] < 0 || grids[j] >= (int)ctx->grids.size() || !ctx->grids[grids[j]]) return MAP_EHANDLE;
    if (!outs[j].cell_mass) return MAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MAP_ENTER(ctx, s);
  MAP_TRY(ensure_stream(ctx));
  for (int j = 0; j < nsnap; ++j)
    if (!check_sizes(&parts[j]) || !parts[j].m || !parts[j].h) return MAP_EINVAL;
  // the whole step as one graph launch, when this call repeats the captured one
  const bool graphable = ctx->cfg.count_work == 0;
  if (ctx->bgraph.exec) {
    if (graphable && (int)ctx->batch_off.size() >= nsnap && ctx->bgraph.sig == graph_sig(ctx, nsnap, parts, grids, outs) &&
        ctx->bgraph.bufs == graph_bufs(ctx, nsnap, ctx->bgraph)) {
      const int rc = batch_graph_replay(ctx, nsnap, grids, outs, totals, s);
      if (rc != GRAPH_FALLBACK) return rc;
    }
    graph_drop(ctx, ctx->bgraph);
  }
  if ((int)ctx->batch_off.size() < nsnap) {
    ctx->batch_off.resize(nsnap);
    ctx->batch_idx.resize(nsnap);
    ctx->batch_itm.resize(nsnap);
    ctx->batch_ioff.resize(nsnap);
    ctx->batch_part.resize(nsnap);
  }
  // 1. octree and pair list per snapshot, kept in the batch slots, built on
  // the workers (largest snapshots first)
  std::vector<SnapDesc> hd(nsnap);
  std::vector<int64_t> np(nsnap);
  int64_t n_pairs = 0, total = 0;
  for (int j = 0; j < nsnap; ++j)
    if (!check_sizes(&parts[j])) return MAP_EINVAL;
  std::vector<int> big(nsnap);
  std::iota(big.begin(), big.end(), 0);
  std::stable_sort(big.begin(), big.end(), [&](int a, int b) { return parts[a].n > parts[b].n; });
  size_t slot_bytes0 = 0;
  for (auto* v : {&ctx->batch_off, &ctx->batch_idx, &ctx->batch_itm, &ctx->batch_ioff, &ctx->batch_part})
    for (int j = 0; j < nsnap; ++j) slot_bytes0 += (*v)[j].cap;
  phase_begin(ctx, 1, s);
  int rc = run_on_workers(ctx, nsnap, big.data(), s, [&](BatchWorker& W, int j) -> int {
    map_ctx* wc = W.ctx;
    const map_particles* p = &parts[j];
    MAP_ENTER(wc, W.stream);
    wc->item_target = ctx->item_target;
    MAP_TRY(check_particles(wc, p, true, true, W.stream));
    const PreparedGrid* g = ctx->grids[grids[j]];
    MAP_TRY(tree_build(wc, p->x, p->y, p->z, p->m, p->h, p->n, W.stream));
    // the list goes straight to the snapshot's slot (reused by later batches)
    PairBufs pb;
    pb.off = &ctx->batch_off[j];
    pb.idx = &ctx->batch_idx[j];
    pb.items = &ctx->batch_itm[j];
    pb.ioff = &ctx->batch_ioff[j];
    pb.part = &ctx->batch_part[j];
    MAP_TRY(pairs_build(wc, g, W.stream, pb));
    hd[j] = make_desc(wc, g, p, &outs[j], wc->pair_off, wc->pair_idx, nullptr, j);
    np[j] = wc->n_pairs;
    return MAP_OK;
  });
  // the slots belong to this context: count their growth here
  size_t slot_bytes1 = 0;
  for (auto* v : {&ctx->batch_off, &ctx->batch_idx, &ctx->batch_itm, &ctx->batch_ioff, &ctx->batch_part})
    for (int j = 0; j < nsnap; ++j) slot_bytes1 += (*v)[j].cap;
  ctx->bytes_in_use += slot_bytes1 - slot_bytes0;
  if (rc != MAP_OK) return rc;
  for (int j = 0; j < nsnap; ++j) {
    n_pairs += np[j];
    total += ctx->grids[grids[j]]->ncell;
  }
  phase_end(ctx, 1, s);
  ctx->pair_off = nullptr;  // no single pair list describes a batch
  ctx->pair_idx = nullptr;
  ctx->pair_frac = nullptr;
  ctx->inv_ready = false;
  ctx->items = nullptr;
  ctx->item_off = nullptr;
  ctx->partial = nullptr;
  ctx->n_pairs = n_pairs;
  ctx->last_ncell = total;

  // 2. longest-processing-time order of the queue
  std::vector<int> order(nsnap);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return np[a] > np[b]; });
  std::vector<SnapDesc> qd(nsnap);
  std::vector<int64_t> ibase(nsnap + 1), base(nsnap + 1);
  SnapDesc* d_desc;
  int64_t* d_base;
  double* d_tot;
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[5], nsnap, &d_desc));
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[6], 2 * (nsnap + 1), &d_base));
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[7], nsnap, &d_tot));
  int64_t* d_ibase = d_base;
  int64_t* d_cbase = d_base + nsnap + 1;
  auto layout = [&]() -> BatchArgs {
    ibase[0] = base[0] = 0;
    for (int i = 0; i < nsnap; ++i) {
      qd[i] = hd[order[i]];
      ibase[i + 1] = ibase[i] + qd[i].nitems;
      base[i + 1] = base[i] + qd[i].ncell;
    }
    return BatchArgs{d_desc, d_ibase, d_cbase, nsnap, ibase[nsnap], total, ctx->d_counters};
  };
  BatchArgs B = layout();
  const int prec = ctx->cfg.precision == MAP_MIXED ? MAP_MIXED : MAP_FP64;
  if (ctx->cfg.autotune && prec == MAP_MIXED && !ctx->tune_done[MAP_MIXED]) {
    // the trials run on the caller's stream, before the batch stream takes over;
    // each target rebuilds every snapshot's work items in its batch slots
    auto rebuild = [&](int target, BatchArgs& Bo) -> int {
      for (int j = 0; j < nsnap; ++j) {
        PairBufs pb;
        pb.items = &ctx->batch_itm[j];
        pb.ioff = &ctx->batch_ioff[j];
        pb.part = &ctx->batch_part[j];
        MAP_TRY(items_build(ctx, static_cast<const int64_t*>(ctx->batch_off[j].p), ctx->grids[grids[j]]->ncell,
                            np[j], target, s, pb));
        hd[j].items = ctx->items;
        hd[j].item_off = ctx->item_off;
        hd[j].partial = ctx->partial;
        hd[j].nitems = ctx->n_items;
      }
      Bo = layout();
      return integrals_upload(ctx, qd.data(), ibase.data(), base.data(), nsnap, d_desc, d_ibase, d_cbase, s);
    };
    MAP_TRY(integrals_autotune(ctx, rebuild, B, s));
    ctx->items = nullptr;
    ctx->item_off = nullptr;
    ctx->partial = nullptr;
  }

  // 3. the integral launch of the whole batch: ordered after the caller's
  // stream, on the context's own stream (graphs cannot be captured on the
  // legacy default stream)
  CUDA_TRY(cudaEventRecord(ctx->bev[0], s));
  CUDA_TRY(cudaStreamWaitEvent(ctx->bstream, ctx->bev[0], 0));
  const int variant = ctx->tuned[prec];
  // graph signature: descriptor bytes, queue layout, launch shape, targets
  std::vector<unsigned char> sig(sizeof(SnapDesc) * nsnap + 2 * sizeof(int64_t) * (nsnap + 1) + 4 * sizeof(void*));
  {
    unsigned char* q = sig.data();
    std::memcpy(q, qd.data(), sizeof(SnapDesc) * nsnap);
    q += sizeof(SnapDesc) * nsnap;
    std::memcpy(q, ibase.data(), sizeof(int64_t) * (nsnap + 1));
    q += sizeof(int64_t) * (nsnap + 1);
    std::memcpy(q, base.data(), sizeof(int64_t) * (nsnap + 1));
    q += sizeof(int64_t) * (nsnap + 1);
    const void* extra[4] = {d_desc, d_base, d_tot, reinterpret_cast<const void*>((intptr_t)(variant * 2 + prec))};
    std::memcpy(q, extra, sizeof(extra));
  }
  if (!ctx->bexec || sig != ctx->bsig) {
    if (ctx->bexec) {
      CUDA_TRY(cudaGraphExecDestroy(ctx->bexec));
      ctx->bexec = nullptr;
    }
    const int64_t l0 = ctx->launches;
    CUDA_TRY(cudaStreamBeginCapture(ctx->bstream, cudaStreamCaptureModeThreadLocal));
    int rc = integrals_upload(ctx, qd.data(), ibase.data(), base.data(), nsnap, d_desc, d_ibase, d_cbase,
                              ctx->bstream);
    if (rc == MAP_OK) rc = integrals_enqueue(ctx, B, variant, ctx->bstream);
    if (rc == MAP_OK) rc = integrals_sum(ctx, d_desc, nsnap, d_tot, ctx->bstream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->bstream, &graph);
    if (rc != MAP_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != MAP_OK ? rc : MAP_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&ctx->bexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      ctx->bexec = nullptr;
      cudaGetLastError();
      return MAP_ECUDA;
    }
    ctx->bexec_launches = ctx->launches - l0;
    ctx->launches = l0;
    ctx->bsig.swap(sig);
  }
  phase_begin(ctx, 2, ctx->bstream);
  CUDA_TRY(cudaGraphLaunch(ctx->bexec, ctx->bstream));
  phase_end(ctx, 2, ctx->bstream);
  ctx->launches += ctx->bexec_launches;
  sum_totals<<<1, 32, 0, ctx->bstream>>>(nsnap, d_tot, ctx->d_total); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  if (totals) CUDA_TRY(cudaMemcpyAsync(totals, d_tot, nsnap * sizeof(double), cudaMemcpyDeviceToDevice, ctx->bstream));
  for (int j = 0; j < nsnap; ++j)
    if (outs[j].cell_vol) {
      const PreparedGrid* g = ctx->grids[grids[j]];
      CUDA_TRY(cudaMemcpyAsync(outs[j].cell_vol, g->vol, g->ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                               ctx->bstream));
    }
  CUDA_TRY(cudaEventRecord(ctx->bev[1], ctx->bstream));
  CUDA_TRY(cudaStreamWaitEvent(s, ctx->bev[1], 0));
  // capture the step for the calls that repeat this one (optional: on any
  // failure there is no graph, and this call's results stand)
  if (graphable && batch_graph_build(ctx, nsnap, parts, grids, outs, np, order, s) != MAP_OK) {
    graph_drop(ctx, ctx->bgraph);
    cudaGetLastError();
  }
  return MAP_OK;
}

int map_batch_graph_stats(map_ctx* ctx, int64_t* captures, int64_t* replays, int64_t* fallbacks) {
  if (!ctx) return MAP_EINVAL;
  if (captures) *captures = ctx->bgraph.captures;
  if (replays) *replays = ctx->bgraph.replays;
  if (fallbacks) *fallbacks = ctx->bgraph.fallbacks;
  return MAP_OK;
}

int solve_h_batch_graph_stats(map_ctx* ctx, int64_t* captures, int64_t* replays) {
  if (!ctx) return MAP_EINVAL;
  if (captures) *captures = ctx->hgraph.captures;
  if (replays) *replays = ctx->hgraph.replays;
  return MAP_OK;
}

int map_get_autotune(map_ctx* ctx, int* chosen, float* ms, int* nvariants) {
  if (!ctx) return MAP_EINVAL;
  int t = 0;
  for (int k = 0; k < N_TARGETS; ++k)
    if (ITEM_TARGETS[k] == ctx->item_target) t = k;
  if (chosen) *chosen = t * N_SHAPES + ctx->tuned[MAP_MIXED];
  if (ms)
    for (int v = 0; v < N_TARGETS * N_SHAPES; ++v) ms[v] = ctx->tune_ms[v];
  if (nvariants) *nvariants = N_TARGETS * N_SHAPES;
  return MAP_OK;
}

int map_autotune_shapes(map_ctx* ctx, int* warps_per_cta, int* ctas_per_sm, int* registers, int* nshapes) {
  if (!ctx || !warps_per_cta || !ctas_per_sm) return MAP_EINVAL;
  for (int v = 0; v < N_SHAPES; ++v) {
    int r = 0;
    MAP_TRY(integrals_shape(ctx, v, &warps_per_cta[v], &ctas_per_sm[v], &r));
    if (registers) registers[v] = r;
  }
  if (nshapes) *nshapes = N_SHAPES;
  return MAP_OK;
}

}  // extern "C"
