// C ABI entry points (see include/exactmap.h for the contract of each call).
#include <cmath>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace {

__global__ void validate_particles(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                   const double* __restrict__ z, const double* __restrict__ m,
                                   const double* __restrict__ h, unsigned long long* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool ok = x[i] >= 0.0 && x[i] <= 1.0 && y[i] >= 0.0 && y[i] <= 1.0 && z[i] >= 0.0 && z[i] <= 1.0;
  if (m) ok = ok && m[i] > 0.0 && m[i] < INFINITY;
  if (h) ok = ok && h[i] > 0.0 && h[i] < INFINITY;
  if (!ok) atomicOr(status, 1ULL);
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

int validate_enqueue(map_ctx* ctx, const map_particles* p, bool need_m, bool need_h, unsigned long long* status,
                     cudaStream_t s) {
  const int tpb = 256;
  validate_particles<<<(unsigned)((p->n + tpb - 1) / tpb), tpb, 0, s>>>(p->n, p->x, p->y, p->z, need_m ? p->m : nullptr,
                                                                        need_h ? p->h : nullptr, status); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

int check_particles(map_ctx* ctx, const map_particles* p, bool need_m, bool need_h, cudaStream_t s) {
  if (!p || p->n <= 0 || !p->x || !p->y || !p->z) return MAP_EINVAL;
  if (need_m && !p->m) return MAP_EINVAL;
  if (need_h && !p->h) return MAP_EINVAL;
  if (p->n >= (int64_t)INT32_MAX) return MAP_EINVAL;
  CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(unsigned long long), s));
  const int tpb = 256;
  validate_particles<<<(unsigned)((p->n + tpb - 1) / tpb), tpb, 0, s>>>(p->n, p->x, p->y, p->z, need_m ? p->m : nullptr,
                                                                        need_h ? p->h : nullptr, ctx->d_counters); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, ctx->d_counters, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ctx->h_scratch[0] ? MAP_EINVAL : MAP_OK;
}

int ctx_enter(map_ctx* ctx, cudaStream_t s) {
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (!ctx->ord_ev) CUDA_TRY(cudaEventCreateWithFlags(&ctx->ord_ev, cudaEventDisableTiming));
  if (ctx->has_last && ctx->last_stream != s) CUDA_TRY(cudaStreamWaitEvent(s, ctx->ord_ev, 0));
  ctx->cur_stream = s;
  ctx->last_stream = s;
  ctx->has_last = true;
  return MAP_OK;
}

int dev_alloc(map_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (cudaMallocAsync(p, bytes > 0 ? bytes : 16, ctx->cur_stream) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MAP_ENOMEM;
  }
  return MAP_OK;
}

void dev_free(map_ctx* ctx, void* p) {
  if (p) cudaFreeAsync(p, ctx->cur_stream);
}

int ctx_ensure(map_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.cap >= bytes) return MAP_OK;
  size_t nb = bytes + bytes / 4 + 4096;
  size_t after = ctx->bytes_in_use - b.cap + nb;
  if (ctx->cfg.hbm_budget && after > ctx->cfg.hbm_budget) return MAP_ENOMEM;
  if (b.p) {
    // the contents are dead; earlier users of the buffer are ordered before
    // this call's stream (ctx_enter), so the free waits for them in stream order
    dev_free(ctx, b.p);
    ctx->bytes_in_use -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  MAP_TRY(dev_alloc(ctx, &b.p, nb));
  b.cap = nb;
  ctx->bytes_in_use += nb;
  return MAP_OK;
}

// The mapping of Eq. (1)-(3) on a prepared grid (the context already entered on s).
int map_run(map_ctx* ctx, const map_particles* p, PreparedGrid* g, map_outputs* out, cudaStream_t s) {
  MAP_TRY(check_particles(ctx, p, true, true, s));
  phase_begin(ctx, 0, s);
  MAP_TRY(tree_build(ctx, p->x, p->y, p->z, p->m, p->h, p->n, s));
  phase_end(ctx, 0, s);
  phase_begin(ctx, 1, s);
  MAP_TRY(pairs_build(ctx, g, s));
  phase_end(ctx, 1, s);
  MAP_TRY(integrals_run(ctx, g, p, out, s));
  ctx->last_npart = p->n;
  return MAP_OK;
}

extern "C" {

void map_config_default(map_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->precision = MAP_MIXED;
  cfg->device = 0;
  cfg->hbm_budget = 0;
  cfg->theta = 0.5;
  cfg->hfact = 1.2;
  cfg->leaf_size = 16;
  cfg->ngb_bruteforce_max = 10000;
  cfg->autotune = 0;
  cfg->queue_timeout_ns = 2000000000ULL;
  cfg->count_work = 0;
  cfg->table_n = 64;
}

const char* map_strerror(int code) {
  switch (code) {
    case MAP_OK: return "ok";
    case MAP_EINVAL: return "invalid argument";
    case MAP_ENOMEM: return "out of memory (HBM budget or cudaMalloc)";
    case MAP_ECUDA: return "CUDA runtime error";
    case MAP_ETIMEOUT: return "bounded device wait timed out";
    case MAP_EDEGENERATE: return "degenerate geometry";
    case MAP_EHANDLE: return "unknown grid handle";
    case MAP_ECAPACITY: return "output buffer too small";
    default: return "unknown status";
  }
}

int map_init(map_ctx** out, const map_config* cfg) {
  if (!out) return MAP_EINVAL;
  *out = nullptr;
  map_ctx* ctx = new (std::nothrow) map_ctx();
  if (!ctx) return MAP_ENOMEM;
  if (cfg) ctx->cfg = *cfg; else map_config_default(&ctx->cfg);
  if (ctx->cfg.precision != MAP_FP64 && ctx->cfg.precision != MAP_MIXED && ctx->cfg.precision != MAP_TABLE) {
    delete ctx;
    return MAP_EINVAL;
  }
  if (ctx->cfg.precision == MAP_TABLE && (ctx->cfg.table_n < 2 || ctx->cfg.table_n > 512)) {
    delete ctx;
    return MAP_EINVAL;
  }
  if (ctx->cfg.leaf_size < 1 || !(ctx->cfg.hfact > 0) || !(ctx->cfg.theta >= 0)) { delete ctx; return MAP_EINVAL; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ctx->cfg.device < 0 || ctx->cfg.device >= ndev) {
    cudaGetLastError();
    delete ctx;
    return MAP_ECUDA;
  }
  ctx->device = ctx->cfg.device;
  if (cudaSetDevice(ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
      cudaMalloc(&ctx->d_counters, 16 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&ctx->d_total, sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_stats, sizeof(map_stats)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_scratch, 8 * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    map_destroy(ctx);
    return MAP_ECUDA;
  }
  cudaMemset(ctx->d_counters, 0, 16 * sizeof(unsigned long long));
  for (auto& e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); map_destroy(ctx); return MAP_ECUDA; }
  if (ctx->cfg.precision == MAP_TABLE) {
    const int r = table_ensure(ctx, nullptr);
    if (r != MAP_OK) { cudaGetLastError(); map_destroy(ctx); return r; }
  }
  *out = ctx;
  return MAP_OK;
}

void map_destroy(map_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  // wait for the context's own work only (other contexts keep running): its
  // workers, its batch stream and the end of its last call -- an event, as
  // the caller's stream may no longer exist; then return the workspace
  if (ctx->bstream) {
    cudaStreamSynchronize(ctx->bstream);
    batch_graph_drop(ctx);
  }
  destroy_workers(ctx);
  if (ctx->bstream) cudaStreamSynchronize(ctx->bstream);
  if (ctx->ord_ev) cudaEventSynchronize(ctx->ord_ev);
  ctx->cur_stream = nullptr;
  for (PreparedGrid* g : ctx->grids)
    if (g) {
      for (const DevBuf& b : g->allocs) dev_free(ctx, b.p);
      delete g;
    }
  for (const DevBuf& b : ctx->grid_pool) dev_free(ctx, b.p);
  for (auto& b : ctx->ws_tree) dev_free(ctx, b.p);
  for (auto& b : ctx->ws_pairs) dev_free(ctx, b.p);
  for (auto& b : ctx->ws_misc) dev_free(ctx, b.p);
  for (auto& b : ctx->ws_inv) dev_free(ctx, b.p);
  for (auto& b : ctx->ws_vor) dev_free(ctx, b.p);
  table_free(ctx);
  for (auto& b : ctx->ws_grid) dev_free(ctx, b.p);
  dev_free(ctx, ctx->cub_tmp.p);
  for (auto* v : {&ctx->batch_off, &ctx->batch_idx, &ctx->batch_itm, &ctx->batch_ioff, &ctx->batch_part})
    for (auto& b : *v) dev_free(ctx, b.p);
  cudaStreamSynchronize(ctx->cur_stream);
  if (ctx->d_counters) cudaFree(ctx->d_counters);
  if (ctx->d_total) cudaFree(ctx->d_total);
  if (ctx->h_stats) cudaFreeHost(ctx->h_stats);
  if (ctx->h_scratch) cudaFreeHost(ctx->h_scratch);
  for (auto& e : ctx->ev) if (e) cudaEventDestroy(e);
  if (ctx->ord_ev) cudaEventDestroy(ctx->ord_ev);
  if (ctx->bexec) cudaGraphExecDestroy(ctx->bexec);
  for (auto& e : ctx->bev) if (e) cudaEventDestroy(e);
  if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
  delete ctx;
}

int map_grid_upload(map_ctx* ctx, const map_grid* grid, int* handle, void* stream) {
  if (!ctx || !grid || !handle) return MAP_EINVAL;
  if (grid->ncell <= 0 || grid->nface < 4 * grid->ncell || grid->nloop < 3 * grid->nface || grid->nvert <= 0)
    return MAP_EINVAL;
  if (grid->nvert >= (int64_t)INT32_MAX || !grid->cell_face_off || !grid->face_vert_off || !grid->face_vert ||
      !grid->face_plane || !grid->vx || !grid->vy || !grid->vz || !grid->site)
    return MAP_EINVAL;
  MAP_ENTER(ctx, S(stream));
  PreparedGrid* g = new (std::nothrow) PreparedGrid();
  if (!g) return MAP_ENOMEM;
  int r = grid_prepare(ctx, grid, g, S(stream));
  if (r != MAP_OK) {
    cudaStreamSynchronize(S(stream));
    grid_recycle(ctx, g);
    delete g;
    return r;
  }
  for (size_t i = 0; i < ctx->grids.size(); ++i)
    if (!ctx->grids[i]) { ctx->grids[i] = g; *handle = (int)i; return MAP_OK; }
  ctx->grids.push_back(g);
  *handle = (int)ctx->grids.size() - 1;
  return MAP_OK;
}

int map_grid_sizes(map_ctx* ctx, int handle, int64_t* ncell, int64_t* nface, int64_t* nloop, int64_t* nvert) {
  if (!ctx) return MAP_EINVAL;
  if (handle < 0 || handle >= (int)ctx->grids.size() || !ctx->grids[handle]) return MAP_EHANDLE;
  const PreparedGrid* g = ctx->grids[handle];
  if (ncell) *ncell = g->ncell;
  if (nface) *nface = g->nface;
  if (nloop) *nloop = g->nloop;
  if (nvert) *nvert = g->nvert;
  return MAP_OK;
}

int map_grid_copy(map_ctx* ctx, int handle, int64_t* cell_face_off, int64_t* face_vert_off, int32_t* face_vert,
                  double* face_plane, double* vx, double* vy, double* vz, double* site, void* stream) {
  if (!ctx) return MAP_EINVAL;
  if (handle < 0 || handle >= (int)ctx->grids.size() || !ctx->grids[handle]) return MAP_EHANDLE;
  const PreparedGrid* g = ctx->grids[handle];
  cudaStream_t s = S(stream);
  MAP_ENTER(ctx, s);
  auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && bytes) CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return MAP_OK;
  };
  MAP_TRY(cp(cell_face_off, g->cell_face_off, (g->ncell + 1) * sizeof(int64_t)));
  MAP_TRY(cp(face_vert_off, g->face_vert_off, (g->nface + 1) * sizeof(int64_t)));
  MAP_TRY(cp(face_vert, g->face_vert, g->nloop * sizeof(int32_t)));
  MAP_TRY(cp(face_plane, g->face_plane, g->nface * 4 * sizeof(double)));
  MAP_TRY(cp(vx, g->vx, g->nvert * sizeof(double)));
  MAP_TRY(cp(vy, g->vy, g->nvert * sizeof(double)));
  MAP_TRY(cp(vz, g->vz, g->nvert * sizeof(double)));
  MAP_TRY(cp(site, g->site, g->ncell * 3 * sizeof(double)));
  return MAP_OK;
}

int map_grid_release(map_ctx* ctx, int handle) {
  if (!ctx) return MAP_EINVAL;
  if (handle < 0 || handle >= (int)ctx->grids.size() || !ctx->grids[handle]) return MAP_EHANDLE;
  // no wait: the buffers go to the context's pool, and the calls that reuse
  // or free them are ordered after this context's earlier work (ctx_enter)
  PreparedGrid* g = ctx->grids[handle];
  if (ctx->bgraph.exec) batch_graph_drop(ctx);  // its graph may read this grid
  grid_recycle(ctx, g);  // kept for the next upload; freed by map_destroy or when room runs out
  delete g;
  ctx->grids[handle] = nullptr;
  return MAP_OK;
}

int map_grid_volumes(map_ctx* ctx, int handle, double* vol, void* stream) {
  if (!ctx || !vol) return MAP_EINVAL;
  if (handle < 0 || handle >= (int)ctx->grids.size() || !ctx->grids[handle]) return MAP_EHANDLE;
  const PreparedGrid* g = ctx->grids[handle];
  MAP_ENTER(ctx, S(stream));
  CUDA_TRY(cudaMemcpyAsync(vol, g->vol, g->ncell * sizeof(double), cudaMemcpyDeviceToDevice, S(stream)));
  return MAP_OK;
}

int map_particles_to_cells(map_ctx* ctx, const map_particles* p, int handle, map_outputs* out, void* stream) {
  if (!ctx || !p || !out || !out->cell_mass) return MAP_EINVAL;
  if (handle < 0 || handle >= (int)ctx->grids.size() || !ctx->grids[handle]) return MAP_EHANDLE;
  cudaStream_t s = S(stream);
  MAP_ENTER(ctx, s);
  return map_run(ctx, p, ctx->grids[handle], out, s);
}

int map_get_pairs(map_ctx* ctx, const int64_t** pair_off, const int32_t** pair_idx, const double** pair_frac,
                  int64_t* n_pairs) {
  if (!ctx) return MAP_EINVAL;
  if (pair_off || pair_idx || pair_frac) {
    CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->cur_stream = ctx->last_stream;
    MAP_TRY(pairs_sort_lists(ctx, ctx->last_stream));
  }
  if (pair_off) *pair_off = ctx->pair_off;
  if (pair_idx) *pair_idx = ctx->pair_idx;
  if (pair_frac) *pair_frac = ctx->pair_frac;
  if (n_pairs) *n_pairs = ctx->n_pairs;
  return MAP_OK;
}

int map_copy_pairs(map_ctx* ctx, int64_t* pair_off, int32_t* pair_idx, double* pair_frac, int64_t capacity,
                   void* stream) {
  if (!ctx || !pair_off || !pair_idx) return MAP_EINVAL;
  if (!ctx->pair_off) return MAP_EINVAL;
  if (capacity < ctx->n_pairs) return MAP_ECAPACITY;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  if (!ctx->pairs_sorted) {
    // sort on the mapping call's stream, then order this copy after it
    ctx->cur_stream = ctx->last_stream;
    MAP_TRY(pairs_sort_lists(ctx, ctx->last_stream));
  }
  MAP_ENTER(ctx, s);
  CUDA_TRY(cudaMemcpyAsync(pair_off, ctx->pair_off, (ctx->last_ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (ctx->n_pairs > 0) {
    CUDA_TRY(cudaMemcpyAsync(pair_idx, ctx->pair_idx, ctx->n_pairs * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (pair_frac && ctx->pair_frac)
      CUDA_TRY(cudaMemcpyAsync(pair_frac, ctx->pair_frac, ctx->n_pairs * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return MAP_OK;
}

int map_get_stats(map_ctx* ctx, map_stats* st) {
  if (!ctx || !st) return MAP_EINVAL;
  CUDA_TRY(cudaSetDevice(ctx->device));
  unsigned long long c[16];
  double tot = 0.0;
  CUDA_TRY(cudaMemcpyAsync(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->last_stream));
  CUDA_TRY(cudaMemcpyAsync(&tot, ctx->d_total, sizeof(double), cudaMemcpyDeviceToHost, ctx->last_stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->last_stream));
  st->n_pairs = ctx->n_pairs;
  st->n_edge_terms = (int64_t)c[1];
  st->n_fp64_terms = (int64_t)c[2];
  st->total_mass = tot;
  st->status = c[0] ? MAP_EINVAL : MAP_OK;
  for (int k = 0; k < 6; ++k) ctx->last_work[k] = (int64_t)c[8 + k];
  return MAP_OK;
}

int map_get_timing(map_ctx* ctx, float* ms) {
  if (!ctx || !ms) return MAP_EINVAL;
  CUDA_TRY(cudaSetDevice(ctx->device));
  for (int k = 0; k < 4; ++k) {
    ms[k] = -1.0f;
    if (!ctx->ev_used[k]) continue;
    CUDA_TRY(cudaEventSynchronize(ctx->ev[2 * k + 1]));
    CUDA_TRY(cudaEventElapsedTime(&ms[k], ctx->ev[2 * k], ctx->ev[2 * k + 1]));
  }
  return MAP_OK;
}

int map_get_work(map_ctx* ctx, int64_t* counts, int64_t* launches) {
  if (!ctx) return MAP_EINVAL;
  if (counts)
    for (int k = 0; k < 6; ++k) counts[k] = ctx->last_work[k];
  if (launches) *launches = ctx->launches;
  return MAP_OK;
}

int solve_h(map_ctx* ctx, map_particles* p, int32_t* route, void* stream) {
  if (!ctx || !p || !p->h) return MAP_EINVAL;
  cudaStream_t s = S(stream);
  MAP_ENTER(ctx, s);
  MAP_TRY(check_particles(ctx, p, false, false, s));
  phase_begin(ctx, 3, s);
  MAP_TRY(h_solve_run(ctx, p->x, p->y, p->z, p->n, p->h, route, nullptr, s));
  phase_end(ctx, 3, s);
  return MAP_OK;
}

int build_pseudo_particles_walk(map_ctx* ctx, const map_particles* full, const map_walk* walk, map_particles* out,
                                int32_t* kind, int64_t* ident, int64_t* n_pseudo, void* stream) {
  if (!ctx || !full || !walk || !walk->src || walk->nsrc < 1 || !out || !n_pseudo || !full->m || !full->h)
    return MAP_EINVAL;
  if (walk->nregion < 0 || (walk->nregion > 0 && !walk->regions)) return MAP_EINVAL;
  if (!(std::isfinite(walk->r_part) && walk->r_part >= 0.0 && std::isfinite(walk->r_leaf) && walk->r_leaf >= 0.0))
    return MAP_EINVAL;
  for (int k = 0; k < 3 * walk->nsrc; ++k)
    if (!std::isfinite(walk->src[k])) return MAP_EINVAL;
  for (int k = 0; k < 5 * walk->nregion; ++k)
    if (!std::isfinite(walk->regions[k]) || (k % 5 >= 3 && walk->regions[k] < 0.0)) return MAP_EINVAL;
  cudaStream_t s = S(stream);
  MAP_ENTER(ctx, s);
  MAP_TRY(check_particles(ctx, full, true, true, s));
  return pseudo_run(ctx, full, walk, out, kind, ident, n_pseudo, s);
}

int build_pseudo_particles(map_ctx* ctx, const map_particles* full, const double* src, int nsrc, map_particles* out,
                           int32_t* kind, int64_t* ident, int64_t* n_pseudo, void* stream) {
  const map_walk walk{src, nsrc, 0.0, 0.0, nullptr, 0};
  return build_pseudo_particles_walk(ctx, full, &walk, out, kind, ident, n_pseudo, stream);
}

}  // extern "C"
