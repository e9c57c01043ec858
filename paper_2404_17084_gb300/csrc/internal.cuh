// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "../../include/exactmap.h"

#define MAP_PI 3.14159265358979323846

#define CUDA_TRY(expr)                        \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return MAP_ECUDA;  \
  } while (0)

#define MAP_TRY(expr)            \
  do {                           \
    int _r = (expr);             \
    if (_r != MAP_OK) return _r; \
  } while (0)

// A device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// A grid prepared for the kernels (all device memory owned by the context).
struct PreparedGrid {
  int64_t ncell = 0, nface = 0, nloop = 0, nvert = 0;
  int64_t* cell_face_off = nullptr;  // [ncell+1]
  int64_t* face_vert_off = nullptr;  // [nface+1]
  double4_32a* face_plane = nullptr;     // absolute (nx,ny,nz,d) [nface]
  double4_32a* face64 = nullptr;         // site-relative (nx,ny,nz,d - n.s) [nface]
  float4* face32 = nullptr;          // same, FP32
  float4* fsph32 = nullptr;          // per face: bounding-sphere centre (site-relative) and radius, FP32
  double* edge64 = nullptr;          // EDGE_STRIDE doubles per loop entry (site-relative); FP64 contexts
  float* edge32 = nullptr;           // EDGE_STRIDE floats per loop entry, interleaved (m.x, t.x, m.y, t.y), (m.z, t.z, a_A, a_B), (delta); mixed contexts
  double* site = nullptr;            // [3*ncell]
  double* vol = nullptr;             // [ncell]
  double* rad = nullptr;             // [ncell] largest vertex distance from the site
  float* rin = nullptr;              // [ncell] smallest site-to-face-plane distance, rounded down
  double* vx = nullptr;              // vertices (for the pair rule bounding tests)
  double* vy = nullptr;
  double* vz = nullptr;
  int32_t* face_vert = nullptr;
  int max_faces = 0;                 // largest face count of a cell
  int max_loops = 0;                 // largest loop-entry count of a cell
  std::vector<DevBuf> allocs;
  size_t bytes = 0;
};

// Last word of a node's FP32 walk record (box32) when its first child does
// not fit in 28 bits.
#define NODE_LINK_FAR 0xffffffffu

// Per-edge record: in-plane inward normal m (3), delta = m.(v_a - s) (so that
// m.(p - v_a) = m.(r - s) - delta > 0 when p is on the inner side),
// unit direction e (3), eps_a = e.(v_a - s), eps_b = e.(v_b - s), pad (3).
#define EDGE_STRIDE 12

// The record of the directed edge from vertex A to vertex B (site-relative
// positions) of a face with unit outward normal (nx, ny, nz), in FP64, into
// rec[0..8]; dr = d - n.s sets the length below which the edge counts as
// zero-length (no wedge: R0 is then +huge, beyond any support).
__device__ __forceinline__ void edge_record64(double nx, double ny, double nz, double dr, double Ax, double Ay,
                                              double Az, double Bx, double By, double Bz, double* rec) {
  double ex = Bx - Ax, ey = By - Ay, ez = Bz - Az;
  const double len = sqrt(ex * ex + ey * ey + ez * ez);
  if (len > 1e-13 * (dr > 0 ? dr : 1.0)) {
    ex /= len; ey /= len; ez /= len;
    // in-plane inward normal (loops are CCW seen from outside): m = n x e
    const double mx = ny * ez - nz * ey, my = nz * ex - nx * ez, mz = nx * ey - ny * ex;
    rec[0] = mx; rec[1] = my; rec[2] = mz;
    rec[3] = mx * Ax + my * Ay + mz * Az;
    rec[4] = ex; rec[5] = ey; rec[6] = ez;
    rec[7] = ex * Ax + ey * Ay + ez * Az;
    rec[8] = ex * Bx + ey * By + ez * Bz;
  } else {
    for (int j = 0; j < 9; ++j) rec[j] = 0.0;
    rec[3] = -1e30;
  }
}

// Octree over a particle set (Morton order, level-synchronous build).
struct DevTree {
  int64_t n = 0;          // particles
  int64_t nnodes = 0;
  int nlevels = 0;
  std::vector<int64_t> level_begin;  // host: first node of each level (+ end)
  // particle arrays in Morton order
  uint64_t* keys = nullptr;
  int32_t* idx = nullptr;             // sorted position -> particle index
  double* xs = nullptr;               // positions/mass/h in sorted order
  double* ys = nullptr;
  double* zs = nullptr;
  double* ms = nullptr;
  double* hs = nullptr;
  float* hs32 = nullptr;             // h in sorted order, FP32 (trees built with h; the pair walk)
  int32_t* owner = nullptr;           // sorted position -> leaf node
  float* split = nullptr;             // 6 floats per sorted position: FP32 hi/lo of x, y, z
  // node arrays
  int64_t* label = nullptr;
  int32_t* level = nullptr;
  int64_t* begin = nullptr;           // range in sorted order
  int64_t* end = nullptr;
  int64_t* first_child = nullptr;
  int32_t* nchild = nullptr;
  int32_t* parent = nullptr;
  double* mass = nullptr;
  double* com = nullptr;              // 3 per node
  unsigned long long* size_bits = nullptr;  // FP64 bits of the node size (max distance to COM)
  unsigned long long* hmax_bits = nullptr;  // FP64 bits of max h in the subtree
  unsigned long long* bbox_bits = nullptr;  // 6 per node: FP64 bits of (minx,miny,minz) and (maxx,maxy,maxz)
  float* box32 = nullptr;             // 8 per node: FP32 box rounded outward, largest h rounded up, pad
};

// A work item of the pair-integral kernel: cnt pairs of one cell, starting
// at position lo of the pair list.  Cells with many pairs are split into
// several items so that grids of few, large cells still fill the GPU.
struct PairItem {
  int64_t lo;
  int32_t cell;
  int32_t cnt;
};

// A worker of a context: its own context (octree, pair-list and h-solve
// workspace), stream and completion event, for the per-snapshot preparation
// of batches.
struct BatchWorker {
  map_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

struct map_ctx {
  map_config cfg;
  int device = 0;
  int sm_count = 0;
  size_t bytes_in_use = 0;             // device bytes held (workspace, grids, grid pool)
  std::vector<PreparedGrid*> grids;
  std::vector<DevBuf> grid_pool;       // buffers of released grids, reused by later uploads
  // workspace
  DevBuf ws_tree[32];
  DevBuf ws_pairs[15];
  DevBuf ws_misc[8];
  DevBuf ws_grid[4];                   // grid preparation: face -> cell, per-face volume term and radius^2,
                                       // FP32 vertex copies
  DevBuf ws_vor[22];                   // grid construction: buckets, cell slots, CSR arrays
  DevBuf ws_inv[13];                   // particle-major copy of the pair list (inverse mapping, Eq. 4)
  DevBuf cub_tmp;
  DevTree tree;
  int64_t node_cap0 = 0;  // > 0: octree node arrays start at this capacity (a context whose workspace is fixed)
  int item_target = 16;   // work items per resident warp of the integral launch (the autotuner may raise it)
  // results of the last mapping call
  int64_t last_ncell = 0;
  int64_t n_pairs = 0;
  int64_t* pair_off = nullptr;
  int32_t* pair_idx = nullptr;        // in the walk's order until pairs_sort_lists
  double* pair_frac = nullptr;
  bool pairs_sorted = false;          // lists sorted by particle index within each cell
  int64_t last_npart = 0;             // particles of the last single mapping call
  // particle-major copy of the last call's pairs (cell and f_ai per entry,
  // ascending cell order within a particle), built by the first inverse
  // mapping after the call
  bool inv_ready = false;
  const int64_t* inv_off = nullptr;   // [last_npart+1]
  const int32_t* inv_cell = nullptr;  // per entry: the Morton rank of its cell's site
  const double* inv_frac = nullptr;
  const int32_t* inv_morton = nullptr; // [last_ncell]: cells in Morton order of their sites
  const int32_t* inv_order = nullptr; // particles by decreasing entry count
  const int64_t* inv_nlong = nullptr; // device: particles summed by a whole warp
  struct PairItem* items = nullptr;  // work items of the pair-integral kernel
  int64_t* item_off = nullptr;       // [ncell+1]: items of cell c
  double* partial = nullptr;         // per item: its pairs' mass
  int64_t n_items = 0;
  // device counters: [0] status, [1] edge terms, [2] fp64 terms, [3] work queue,
  // [4..7] scratch, [8] face tests, [9] edge records read, [10] inner-piece
  // antiderivative evaluations, [11] middle-piece Gauss-Legendre intervals
  unsigned long long* d_counters = nullptr;
  double* d_total = nullptr;
  map_stats* h_stats = nullptr;  // pinned
  cudaStream_t last_stream = nullptr;  // stream of the context's last call
  bool has_last = false;               // a call has run (ord_ev marks its end)
  cudaStream_t cur_stream = nullptr;   // stream of the call in progress: workspace is allocated and freed on it
  cudaEvent_t ord_ev = nullptr;        // the end of the context's last call, on its stream
  int64_t* h_scratch = nullptr;  // pinned scratch for small readbacks
  int64_t launches = 0;          // kernels this context has launched (own kernels only)
  int64_t last_work[6] = {0, 0, 0, 0, 0, 0};  // work tally of the last mapping call (see map_get_work)
  // phase events (start/stop pairs): 0 tree build, 1 pair list, 2 pair integrals, 3 h solve
  cudaEvent_t ev[8] = {};
  bool ev_used[4] = {false, false, false, false};
  // launch shape of the pair-integral kernel, per precision (the autotuner's choice)
  int tuned[2] = {0, 0};
  bool tune_done[2] = {false, false};
  float tune_ms[32] = {};             // [item target][shape]: ms of each trial (0 when not run)
  // batches: per-snapshot pair lists of the last batch, and the CUDA graph of
  // its integral launch with the descriptor bytes it was captured for
  std::vector<DevBuf> batch_off, batch_idx, batch_itm, batch_ioff, batch_part;
  cudaStream_t bstream = nullptr;
  cudaEvent_t bev[2] = {};
  cudaGraphExec_t bexec = nullptr;
  std::vector<unsigned char> bsig;
  int64_t bexec_launches = 0;  // kernels per replay of bexec
  // map_batch's whole step as one CUDA graph: the snapshots' validation,
  // octrees, pair lists and work items on the workers' streams, then the one
  // integral launch and the sums.  Captured after an eager call, replayed
  // while a call names the same buffers, grids and outputs (sig) and every
  // workspace it baked in is still the same allocation (bufs).
  struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> sig;
    std::vector<const void*> bufs;
    int64_t launches = 0;                 // kernels per replay
    DevBuf desc, base, tot, caps, flags;  // its own descriptors, queue bases, totals, capacities, flags
    int64_t captures = 0, replays = 0, fallbacks = 0;
  } bgraph, hgraph;  // map_batch's step; solve_h_batch's step (its flags in tot)
  std::vector<BatchWorker> workers;  // created by the first batch call that uses them
  cudaEvent_t wev = nullptr;         // the caller's stream, before the workers start
  // MAP_TABLE: the table of the pyramid integral (n^3 FP32 texels)
  cudaArray_t tab_arr = nullptr;
  cudaTextureObject_t tab_tex = 0;
};

inline void phase_begin(map_ctx* ctx, int k, cudaStream_t s) { if (ctx->ev[2 * k]) cudaEventRecord(ctx->ev[2 * k], s); }
inline void phase_end(map_ctx* ctx, int k, cudaStream_t s) {
  if (ctx->ev[2 * k + 1]) { cudaEventRecord(ctx->ev[2 * k + 1], s); ctx->ev_used[k] = true; }
}

// ---------------------------------------------------------------- allocation
// Every call of a context starts with MAP_ENTER on its stream: the stream is
// ordered after the end of the context's previous call (an event, no host
// wait) and becomes the context's last stream, so that the context's buffers
// can be freed and allocated in stream order on it.
// Workspace then comes from the stream-ordered allocator (dev_alloc /
// dev_free on the current call's stream): growing or releasing a buffer never
// waits for the device.
int ctx_enter(map_ctx* ctx, cudaStream_t s);
// Marks the end of a call on its stream (at every return of the entry
// point): the next call of the context, on any stream, waits for this point.
// An event outlives the caller's stream, which may be destroyed in between.
struct CallScope {
  map_ctx* ctx;
  cudaStream_t s;
  ~CallScope() {
    if (ctx->ord_ev) cudaEventRecord(ctx->ord_ev, s);
  }
};
#define MAP_ENTER(ctx, s)          \
  MAP_TRY(ctx_enter((ctx), (s)));  \
  CallScope call_scope_{(ctx), (s)}
int dev_alloc(map_ctx* ctx, void** p, size_t bytes);
void dev_free(map_ctx* ctx, void* p);
int ctx_ensure(map_ctx* ctx, DevBuf& b, size_t bytes);
int ctx_alloc_grid(map_ctx* ctx, PreparedGrid* g, void** p, size_t bytes);

template <typename T>
inline int ensure_t(map_ctx* ctx, DevBuf& b, size_t count, T** out) {
  int r = ctx_ensure(ctx, b, count * sizeof(T) + 256);
  if (r != MAP_OK) return r;
  *out = reinterpret_cast<T*>(b.p);
  return MAP_OK;
}

// One mapping problem of the pair-integral kernel: a resident grid, a
// particle set, its pair list and its outputs (device pointers).
struct SnapDesc {
  int64_t ncell;
  const int64_t* cfo;
  const int64_t* fvo;
  const double* site;
  const double* vol;
  const int64_t* pair_off;
  const int32_t* pair_idx;
  const double *x, *y, *z, *m, *h;
  double* frac;        // per-pair f_ai, or NULL
  double* cell_mass;
  double* cell_rho;    // or NULL
  const PairItem* items;     // work items
  const int64_t* item_off;   // [ncell+1]
  double* partial;           // per item
  int64_t nitems;
  const void* face;    // site-relative planes: float4 (mixed) or double4 (FP64)
  const void* edge;    // EDGE_STRIDE floats or doubles per loop entry
  const double4_32a* face64;
  const double* edge64;
  const float4* fsph;  // per face: bounding sphere (site-relative centre, radius), FP32
  const int32_t* face_vert;          // loop entries -> vertices (the FP64 faces of the mixed build)
  const double *vx, *vy, *vz;
  int64_t orig;        // the caller's index of this snapshot
};

// The queue of the pair-integral kernel: work items of nsnap snapshots,
// snapshot j owning queue positions [item_base[j], item_base[j+1]) and cells
// [cell_base[j], cell_base[j+1]) of the per-cell sums.
struct BatchArgs {
  const SnapDesc* snaps;
  const int64_t* item_base;
  const int64_t* cell_base;
  int nsnap;
  int64_t total;        // items (with total_dev: an upper bound, for the launch shape)
  int64_t total_cells;
  unsigned long long* counters;  // [1] edge terms, [2] FP64 terms, [3] queue, [8..13] work tally
  const int64_t* total_dev = nullptr;  // graph replays: the item count, written on the device
  const int64_t* bad = nullptr;        // graph replays: nonzero = skip the launch (invalid input, overflow)
};

// The queue length a launch of the pair-integral kernels serves: the host's
// count, or (graph replays) the device's, 0 when the replay is to be skipped.
__device__ __forceinline__ int64_t queue_total(const BatchArgs& B) {
  if (!B.total_dev) return B.total;
  return (B.bad && *B.bad) ? 0 : *B.total_dev;
}

// Launch shapes of the mixed pair-integral kernel: (warps per CTA, CTAs per
// SM) = (4, 5), (4, 4), (2, 9), (8, 2).  Each is compiled for its CTAs per SM
// (the register cap per thread follows) and launched with at most that many
// per SM; all four fit an SM's registers and shared memory at once, so the
// launched shape is the resident one (integrals_shape reports it).
// Work-item targets: items per resident warp of a launch.
constexpr int N_SHAPES = 4;
constexpr int N_TARGETS = 3;
constexpr int ITEM_TARGETS[N_TARGETS] = {16, 64, 256};

// ---------------------------------------------------------------- subsystems
int grid_prepare(map_ctx* ctx, const map_grid* in, PreparedGrid* g, cudaStream_t s);
// Returns a grid's buffers to the context's pool (the caller has synchronised
// the device), and frees the pool.
void grid_recycle(map_ctx* ctx, PreparedGrid* g);
void grid_pool_drop(map_ctx* ctx);
int tree_build(map_ctx* ctx, const double* x, const double* y, const double* z, const double* m,
               const double* h, int64_t n, cudaStream_t s, bool want_size = false);
// The same tree from launches of fixed shape and no host reads (capturable in
// a CUDA graph): node arrays sized for the largest possible tree of n
// particles, tree_nodes_max(n, leaf).  Same nodes, same order, same sums as
// tree_build.
int64_t tree_nodes_max(int64_t n, int leaf_size);
int tree_build_graph(map_ctx* ctx, const double* x, const double* y, const double* z, const double* m,
                     const double* h, int64_t n, cudaStream_t s);
// Output buffers of a pair-list build; nullptr members mean the context's
// workspace.
struct PairBufs {
  DevBuf* off = nullptr;    // pair offsets per cell
  DevBuf* idx = nullptr;    // pair list
  DevBuf* items = nullptr;  // work items
  DevBuf* ioff = nullptr;   // items per cell (offsets)
  DevBuf* part = nullptr;   // per-item partial masses
};

// Pair list of the grid against the current octree, and its work items.
int pairs_build(map_ctx* ctx, const PreparedGrid* g, cudaStream_t s, const PairBufs& out = PairBufs());
// The work items of a pair list (offsets off, nc cells, np pairs) for at least
// `target` items per resident warp; sets ctx->items, item_off, partial, n_items.
int items_build(map_ctx* ctx, const int64_t* off, int64_t nc, int64_t np, int target, cudaStream_t s,
                const PairBufs& out = PairBufs());
// pairs_build with no host reads (capturable): the list and the items go to
// out, which must hold cap_pairs pairs and cap_items items; when a build needs
// more, nothing is written beyond them and the counts (off[nc], ioff[nc])
// say so.  Sets the context's list pointers like pairs_build; n_pairs and
// n_items are left unknown (-1).
int pairs_build_graph(map_ctx* ctx, const PreparedGrid* g, cudaStream_t s, const PairBufs& out, int64_t cap_pairs,
                      int64_t cap_items);
// Sorts the last call's lists (and f_ai) by particle index within each cell.
int pairs_sort_lists(map_ctx* ctx, cudaStream_t s);
int check_particles(map_ctx* ctx, const map_particles* p, bool need_m, bool need_h, cudaStream_t s);
// The validation kernel of check_particles alone: ORs 1 into *status (device)
// when a particle is invalid; no host read.
int validate_enqueue(map_ctx* ctx, const map_particles* p, bool need_m, bool need_h, unsigned long long* status,
                     cudaStream_t s);
// map_particles_to_cells on a prepared grid (after ctx_enter on s)
int map_run(map_ctx* ctx, const map_particles* p, PreparedGrid* g, map_outputs* out, cudaStream_t s);
int integrals_run(map_ctx* ctx, const PreparedGrid* g, const map_particles* p, map_outputs* out, cudaStream_t s);
SnapDesc make_desc(map_ctx* ctx, const PreparedGrid* g, const map_particles* p, const map_outputs* out,
                   const int64_t* pair_off, const int32_t* pair_idx, double* frac, int orig);
int integrals_upload(map_ctx* ctx, const SnapDesc* h_desc, const int64_t* h_ibase, const int64_t* h_cbase,
                     int nsnap, SnapDesc* d_desc, int64_t* d_ibase, int64_t* d_cbase, cudaStream_t s);
int integrals_enqueue(map_ctx* ctx, const BatchArgs& B, int variant, cudaStream_t s);
// Launch geometry of shape v of the mixed kernel on the context's device:
// warps per CTA, CTAs per SM launched, registers per thread.
int integrals_shape(map_ctx* ctx, int v, int* warps, int* ctas, int* regs);
int integrals_sum(map_ctx* ctx, const SnapDesc* d_desc, int nsnap, double* totals, cudaStream_t s);
// Times every (work-item target, launch shape) pair on the call's inputs and
// keeps the fastest (ctx->tuned[MAP_MIXED], ctx->item_target).  rebuild(T, B)
// rebuilds the work items for target T and returns the launch arguments;
// on return B holds those of the chosen target.
int integrals_autotune(map_ctx* ctx, const std::function<int(int, BatchArgs&)>& rebuild, BatchArgs& B,
                       cudaStream_t s);
// MAP_TABLE: build the table (synchronises the stream), free it, and launch
// the table variant of the pair-integral kernel
int table_ensure(map_ctx* ctx, cudaStream_t s);
void table_free(map_ctx* ctx);
int launch_table(map_ctx* ctx, const BatchArgs& B, cudaStream_t s);
// Runs fn(worker, j) for j = order[0..n) on the context's workers, each on
// its own stream and host thread, after the work queued on s; s then waits
// for all of them.  Returns the first error.  Work is handed out in `order`.
int run_on_workers(map_ctx* ctx, int n, const int* order, cudaStream_t s,
                   const std::function<int(BatchWorker&, int)>& fn);
void destroy_workers(map_ctx* ctx);
// Drops the batch graph (its inputs changed place: a grid released, a
// workspace reallocated) and frees its buffers.
void batch_graph_drop(map_ctx* ctx);
// (graph: the octree from tree_build_graph, so that the call reads nothing
// back and can be captured; the same tree, the same h)
int h_solve_run(map_ctx* ctx, const double* x, const double* y, const double* z, int64_t n, double* h,
                int32_t* route, const double* h0_override, cudaStream_t s, bool graph = false);
int pseudo_run(map_ctx* ctx, const map_particles* full, const map_walk* walk, map_particles* out, int32_t* kind,
               int64_t* ident, int64_t* n_pseudo, cudaStream_t s);

// blocks of t threads covering n items
inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// FP64 bit helpers for atomic max/min on non-negative doubles
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }
