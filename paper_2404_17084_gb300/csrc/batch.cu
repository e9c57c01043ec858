// Batched mapping: many independent snapshots (particle set + resident grid)
// in one persistent pair-integral launch.
//
// Each snapshot's octree and pair list are built by one of the context's
// workers: BATCH_WORKERS worker contexts, each with its own workspace,
// stream and host thread, take the snapshots largest first (these steps size
// their buffers from device counts and so synchronise their stream; running
// several at once keeps the GPU busy between those points).  The pair lists
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
  std::atomic<int> next{0}, err{MAP_OK};
  std::vector<std::thread> th;
  for (size_t w = 0; w < ctx->workers.size(); ++w)
    th.emplace_back([&, w]() {
      BatchWorker& W = ctx->workers[w];
      if (cudaSetDevice(ctx->device) != cudaSuccess) { int e = MAP_OK; err.compare_exchange_strong(e, MAP_ECUDA); }
      for (;;) {
        if (err.load() != MAP_OK) break;
        const int i = next.fetch_add(1);
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
  return rc;
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

}  // extern "C"
