/*
 * exactmap.h -- C ABI of the GB300 (sm_103a) library for the Exact mapping of
 * SPH particle densities onto a Voronoi grid, with the tree-based
 * pseudo-particle front end (Lau, Petkova & Bonnell 2024).
 *
 * Conventions
 *  - Every function returns MAP_OK (0) or a negative MAP_E* code; none aborts,
 *    exits or traps.  map_strerror() names a code.
 *  - Array arguments are DEVICE pointers owned by the caller, unless a
 *    function says otherwise.  The library owns only its context workspace.
 *  - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *    stream) unless documented as synchronising; statistics are read back with
 *    map_get_stats(), which synchronises that stream.
 *  - The calls of one context run in stream order, one after the other: a call
 *    on another stream than the context's previous call first makes its
 *    stream wait for the previous call's stream (an event; the host does not
 *    wait).  Workspace is allocated and freed in the stream-ordered
 *    allocator's pool on the calling stream, so no call waits for the whole
 *    device (map_destroy waits for the context's own streams).
 *  - A context is not thread-safe: use one context per host thread.
 *  - Lengths are in the unit cube [0,1]^3; masses are arbitrary positive
 *    numbers; the kernel is the M4 cubic spline with support 2h.
 */
#ifndef EXACTMAP_H
#define EXACTMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MAP_OK 0
#define MAP_EINVAL (-1)      /* bad argument: NULL, bad CSR, NaN, h <= 0, point outside the cube */
#define MAP_ENOMEM (-2)      /* over the context's HBM budget or cudaMalloc failed; nothing was changed */
#define MAP_ECUDA (-3)       /* a CUDA runtime call failed */
#define MAP_ETIMEOUT (-4)    /* reserved: no call returns it -- no kernel of the library waits on a flag, a peer or
                                another kernel (work queues are drained by atomics, never polled) */
#define MAP_EDEGENERATE (-5) /* reserved: geometry not classifiable even in FP64 (result flagged) */
#define MAP_EHANDLE (-6)     /* unknown grid handle */
#define MAP_ECAPACITY (-7)   /* a caller-provided output buffer is too small */

/* ------------------------------------------------------------ configuration */
#define MAP_FP64 0  /* every wedge integral in FP64 (closed form) */
#define MAP_MIXED 1 /* wedge integrals in FP32, FP64 accumulation */
#define MAP_TABLE 2 /* pyramid integrals interpolated in a pre-computed table (the paper's production route,
                       Section II-B); FP32 geometry, FP64 per-pair sums; see table_n */

typedef struct {
  int precision;                     /* MAP_FP64 or MAP_MIXED */
  int device;                        /* CUDA device ordinal */
  size_t hbm_budget;                 /* max bytes of workspace + resident grids; 0 = no limit */
  double theta;                      /* opening angle of Eq. (5); default 0.5 */
  double hfact;                      /* h = hfact n^(-1/3), Eq. (7); default 1.2 */
  int leaf_size;                     /* octree leaf capacity; default 16 */
  int ngb_bruteforce_max;            /* Section III-D: k_mid neighbour search above this many nodes; default 10000 */
  int autotune;                      /* 1: the context's first mixed mapping call (map_batch or
                                        map_particles_to_cells) times the pair-integral launch for every
                                        work-item size and launch shape (map_get_autotune) and keeps the
                                        fastest pair; default 0 */
  unsigned long long queue_timeout_ns; /* reserved, ignored: the library has no device-side wait to bound
                                          (see MAP_ETIMEOUT); default 2e9 */
  int count_work;                    /* 1: the pair-integral kernel also tallies its work (map_get_work,
                                        map_stats.n_edge_terms / n_fp64_terms), in a separate compilation
                                        of one launch shape that keeps the tally in registers (slower, and
                                        its FP32 rounding may differ within the mixed build's tolerance);
                                        0: those counts read 0; default 0 */
  int table_n;                       /* MAP_TABLE: nodes per axis of the table of I(r0, R0, phi) over r0 in
                                        [0, 2], R0 / sqrt(4 - r0^2) in [0, 1], phi in [0, pi/2] (n^3 FP32
                                        texels, trilinear interpolation by the texture unit, whose weights
                                        carry 8 fractional bits), built by map_init in FP64 from the closed
                                        form; 2..512, default 64 */
} map_config;

/* Fill *cfg with the defaults listed above. */
void map_config_default(map_config* cfg);

/* ------------------------------------------------------------ data */

/* Particle set, structure of arrays, FP64 device pointers of length n.
 * h is input (map_particles_to_cells) or output (solve_h). */
typedef struct {
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  const double* m;
  double* h;
} map_particles;

/* Convex-cell grid in CSR form (device pointers).  Cell c owns faces
 * [cell_face_off[c], cell_face_off[c+1]); face f owns loop entries
 * [face_vert_off[f], face_vert_off[f+1]) of face_vert, whose values index
 * the vertex arrays.  Loops run counter-clockwise seen from outside the cell.
 * face_plane holds 4 doubles per face (nx, ny, nz, d) with a unit outward
 * normal: points of the cell satisfy n.x <= d.  site holds 3 doubles per
 * cell: a point strictly inside the cell (the generating site). */
typedef struct {
  int64_t ncell;
  int64_t nface;
  int64_t nloop;
  int64_t nvert;
  const int64_t* cell_face_off;
  const int64_t* face_vert_off;
  const int32_t* face_vert;
  const double* face_plane;
  const double* vx;
  const double* vy;
  const double* vz;
  const double* site;
} map_grid;

/* Per-cell outputs (device pointers of length ncell, caller-owned).
 * cell_mass is required; cell_rho and cell_vol may be NULL. */
typedef struct {
  double* cell_mass; /* M_i = sum_a m_a f_ai, Eq. (3) numerator */
  double* cell_rho;  /* rho_i = M_i / V_i, Eq. (1)-(3) */
  double* cell_vol;  /* V_i */
} map_outputs;

/* Statistics of the last mapping call on a context. */
typedef struct {
  int64_t n_pairs;      /* listed particle-cell pairs (one pair integral each) */
  int64_t n_edge_terms; /* edge integrals evaluated (two vertex pyramids each); count_work only */
  int64_t n_fp64_terms; /* mixed build: (pair, face) tests decided in FP64 (a face plane within 1e-4 h of the
                           particle); count_work only */
  double total_mass;    /* sum_i M_i */
  int status;           /* device-side status word (MAP_OK or a MAP_E* code) */
} map_stats;

typedef struct map_ctx map_ctx;

/* ------------------------------------------------------------ lifetime */

/* Create a context on cfg->device (NULL cfg = defaults).  Allocates a small
 * pinned host block and selects the device; no device workspace yet, except
 * the table of a MAP_TABLE context (built here, synchronously). */
int map_init(map_ctx** ctx, const map_config* cfg);

/* Free all device and host memory of the context (grids included). */
void map_destroy(map_ctx* ctx);

/* Static string naming a status code. */
const char* map_strerror(int code);

/* ------------------------------------------------------------ grids */

/* Copy a grid (device or page-locked host pointers, read during the call
 * only; host arrays are copied in by the call itself) into context memory and precompute its per-face and per-edge geometry, cell volumes and
 * cell radii (largest vertex distance from the site).  The geometry kept is
 * what the context's precision reads: FP32 face planes, face bounding
 * spheres and edge records for MAP_MIXED, FP64 edge records for MAP_FP64.  The grid stays
 * resident until map_grid_release / map_destroy.  Synchronises the stream.
 * Errors: MAP_EINVAL (empty or inconsistent sizes, a corrupted CSR: an
 * offset array that is not increasing, a loop of fewer than 3 entries, a
 * cell of fewer than 4 faces, a vertex index out of range, or last offsets
 * that disagree with nface / nloop -- checked on the device before any
 * kernel indexes with them), MAP_ENOMEM. */
int map_grid_upload(map_ctx* ctx, const map_grid* grid, int* handle, void* stream);

/* Release a resident grid.  Its device buffers stay with the context and
 * serve later uploads of the same or a smaller grid (no cudaMalloc then);
 * they are freed by map_destroy, or when an upload or the HBM budget needs
 * the room.  Returns at once: later calls of the context that reuse or free
 * those buffers are ordered after its earlier work.  MAP_EHANDLE if unknown. */
int map_grid_release(map_ctx* ctx, int handle);

/* Copy the volumes V_i of a resident grid into vol (device, ncell doubles). */
int map_grid_volumes(map_ctx* ctx, int handle, double* vol, void* stream);

/* Build a resident grid on the device from point sites (Section II-A): drop
 * every site that lies within merge_tol of a site of lower index (the merging
 * of tightly packed cells; 0 keeps all), move the sites `lloyd` times to
 * their cells' centroids (Lloyd iterations; the paper applies 5), then
 * tessellate: each cell is the unit cube cut by the bisector planes of its
 * neighbours, vertices within a relative 1e-11 welded.  The grid's sites are
 * the final (moved) sites; its cells keep their own vertices (none shared).
 *
 * x, y, z: device, n doubles in [0, 1].  kept (optional, device, capacity n
 * int64): the indices of the sites that survived the merge, in order;
 * *n_kept (optional): their number = the grid's cell count.  *handle: as
 * map_grid_upload.  Synchronises the stream.  Workspace: about 3 KB per site
 * (cells are built in fixed slots of 96 vertices, 48 faces and 320 loop
 * entries), kept by the context for later builds until map_destroy; the
 * first call also raises the per-thread stack to at least 17 KB for the
 * context's device.
 * Errors: MAP_EINVAL (n < 1, a site outside the cube or not finite, lloyd <
 * 0, merge_tol < 0), MAP_ECAPACITY (a cell outgrew its slot), MAP_ENOMEM,
 * MAP_ECUDA. */
int map_grid_build(map_ctx* ctx, const double* x, const double* y, const double* z, int64_t n, int lloyd,
                   double merge_tol, int* handle, int64_t* kept, int64_t* n_kept, void* stream);

/* Sizes of a resident grid (any pointer may be NULL), and a copy of its
 * arrays in the layout of map_grid (device or page-locked host buffers of
 * those sizes; a NULL destination is skipped; asynchronous on stream). */
int map_grid_sizes(map_ctx* ctx, int handle, int64_t* ncell, int64_t* nface, int64_t* nloop, int64_t* nvert);
int map_grid_copy(map_ctx* ctx, int handle, int64_t* cell_face_off, int64_t* face_vert_off, int32_t* face_vert,
                  double* face_plane, double* vx, double* vy, double* vz, double* site, void* stream);

/* ------------------------------------------------------------ the mapping (Section II-B, Eq. 1-3) */

/* For every cell i of the resident grid: build the list of particles a whose
 * support may reach the cell, compute every pair integral
 * f_ai = int_{V_i} W(|r'-r_a|, h_a) dV' in closed form from the cell's face
 * and edge wedges (vertex pyramids, Section II-B), and write
 * M_i = sum_a m_a f_ai and rho_i = M_i / V_i (Eq. 1-3).
 *
 * Pair rule (makes pair lists reproducible; the paper is silent): (i,a) is
 * listed iff |r_a - s_i| < 2 h_a + R_i and n_f.r_a - d_f < 2 h_a for every
 * face f of cell i, both evaluated in FP64 in a fixed order without FMA.
 * The lists, as map_get_pairs / map_copy_pairs return them, are sorted by
 * particle index within each cell.
 *
 * p->h must hold positive smoothing lengths.  Synchronises the stream once
 * (to size the pair list).  The pair list and the per-pair integrals stay in
 * the context until the next call (map_get_pairs).
 * Errors: MAP_EINVAL, MAP_EHANDLE, MAP_ENOMEM, MAP_ECUDA. */
int map_particles_to_cells(map_ctx* ctx, const map_particles* p, int grid, map_outputs* out, void* stream);

/* Device pointers to the last call's pair list: pair_off (ncell+1 int64),
 * pair_idx (n_pairs int32 particle indices, ascending within each cell),
 * pair_frac (n_pairs doubles, f_ai).  Owned by the context; valid until the
 * next mapping call.  The mapping itself keeps each cell's list in the order
 * of its octree walk; the first request for the pointers after a mapping
 * call sorts the lists in place on that call's stream and waits for it. */
int map_get_pairs(map_ctx* ctx, const int64_t** pair_off, const int32_t** pair_idx, const double** pair_frac,
                  int64_t* n_pairs);

/* Copy the last call's pair list into caller-owned device buffers:
 * pair_off (ncell+1 int64), pair_idx (n_pairs int32, ascending within each
 * cell), pair_frac (n_pairs doubles, may be NULL).  capacity = the length of
 * pair_idx / pair_frac; MAP_ECAPACITY if it is smaller than n_pairs.  Sorts
 * the lists first when map_get_pairs has not (waiting for the mapping call's
 * stream), then copies asynchronously on stream. */
int map_copy_pairs(map_ctx* ctx, int64_t* pair_off, int32_t* pair_idx, double* pair_frac, int64_t capacity,
                   void* stream);

/* ------------------------------------------------------------ the inverse mapping (Section II-B, Eq. 4) */

/* Carry a per-cell quantity back to the particles of the last
 * map_particles_to_cells call with that call's pair integrals:
 *     particle_value[a] = sum_i cell_value[i] f_ai
 * over the cells i whose pair list holds a (Eq. 4; the quantity there is the
 * ionic fraction the radiative transfer step leaves in each cell).  With the
 * same weights as M_i = sum_a m_a f_ai, the mass-weighted totals agree:
 * sum_a m_a particle_value[a] = sum_i cell_value[i] M_i (up to rounding and
 * to the particles' own mass outside the grid).
 *
 * cell_value: device, ncell doubles of that call's grid; particle_value:
 * device, n doubles, written; n must be that call's particle count.  Each
 * particle's terms are fused into its running sum one at a time in ascending
 * cell order, from +0, with one rounding per term (acc <- RN(acc + v_i f_ai),
 * an FMA): equal bit for bit to that sequential sum.  A particle in no pair
 * list gets 0.
 *
 * The first call after a mapping builds a particle-major copy of its pair
 * list (cell and f_ai of every pair, 12 bytes per pair, plus 12 bytes per
 * particle), kept by the context until the next mapping call; later calls
 * with other cell values reuse it.  The build's sort workspace (about 20
 * bytes per pair) also stays with the context, for the next mapping's build,
 * until map_destroy.  Asynchronous on stream (ordered after the mapping
 * call like every call of the context).
 * Errors: MAP_EINVAL (NULL pointer; no single mapping call with per-pair
 * integrals in this context: map_batch and the server keep none; n is not
 * that call's particle count; 2^32 or more pairs), MAP_ENOMEM, MAP_ECUDA. */
int map_cells_to_particles(map_ctx* ctx, const double* cell_value, double* particle_value, int64_t n, void* stream);

/* Statistics of the last mapping call; synchronises its stream. */
int map_get_stats(map_ctx* ctx, map_stats* stats);

/* Work tally of the last mapping call, read by the last map_get_stats().
 * counts must hold 6 entries: [0] face tests, [1] edge records read,
 * [2] inner-piece antiderivative evaluations, [3] middle-piece intervals,
 * [4] beyond-the-support intervals, [5] middle intervals of the mixed build
 * split at the foot (a second Gauss-Legendre panel); all per pair, summed.
 * The counts are tallied only by a context created with count_work = 1
 * (zeros otherwise).  *launches: kernels this context has launched so far (its own kernels;
 * library sort/scan primitives not counted).  These feed the algorithmic
 * operation count of the roofline. */
int map_get_work(map_ctx* ctx, int64_t* counts, int64_t* launches);

/* Device time (ms, CUDA events on the call's stream) of the most recent
 * phases: ms[0] octree build and ms[1] pair-list build and ms[2] the
 * pair-integral kernel (all of the last map_particles_to_cells), ms[3] the
 * last solve_h.  -1 for a phase not yet run.  Waits for those events. */
int map_get_timing(map_ctx* ctx, float* ms);

/* ------------------------------------------------------------ batches */

/* Map nsnap independent snapshots (configuration: many uneven instances in
 * one persistent launch).  Snapshot j is the particle set parts[j] (m, h
 * given) on the resident grid grids[j], with outputs outs[j], exactly as in
 * map_particles_to_cells; every snapshot's result equals what that call
 * gives.  Octrees and pair lists are built by the context's workers (worker
 * contexts with their own streams and host threads, several snapshots at
 * once, largest first; the workspace they hold is not counted against the
 * HBM budget); the pair integrals of all snapshots then run in ONE launch of
 * the persistent kernel, whose device work queue hands out the cells of every
 * snapshot, largest pair count first.  That launch, with its descriptor
 * upload and the per-snapshot sums, is captured in a CUDA graph and replayed
 * while the batch's pointers and sizes are unchanged.
 *
 * The whole step as one graph: after a call that ran eagerly (a context's
 * first call, or one whose inputs moved), the context captures the entire
 * step -- per snapshot the particle validation, the octree, the pair list
 * and the work items (built without host reads, on the workers' streams,
 * into buffers a quarter larger than that call's lists), then the integral
 * launch and the sums.  A later call with the same particle buffers (x, y,
 * z, m, h and n), grids, outputs and launch choices replays it: one graph
 * launch, then one read of three device words (the pair and item totals and
 * a flag), so such a call returns once its results are complete.  Values in
 * the buffers may change between calls (new positions, h, masses): the
 * replay computes from them.  A replay whose lists outgrow their buffers
 * skips its integral launch and the call runs eagerly instead (and captures
 * anew); invalid particles give MAP_EINVAL.  Releasing a grid drops the
 * graph.  Counting contexts (count_work) never capture.  Results of a replay
 * equal those of the eager step on the same inputs bit for bit.
 *
 * totals (optional,
 * device, nsnap doubles) receives sum_i M_i per snapshot.  Per-pair fractions
 * are not kept (map_get_pairs / map_copy_pairs then report no list);
 * map_get_stats covers the whole batch.  The batch runs on a stream of the
 * context, ordered after and before the given stream by events.
 * Errors: MAP_EINVAL, MAP_EHANDLE, MAP_ENOMEM, MAP_ECUDA. */
int map_batch(map_ctx* ctx, int nsnap, const map_particles* parts, const int* grids, const map_outputs* outs,
              double* totals, void* stream);

/* The autotuner's state.  Trials are pairs of a work-item target T (items
 * per resident warp of the integral launch: 16, 64, 256; a cell's pairs form
 * items of at most K blocks of 32, K = (pair blocks) / (T x warps)) and a
 * launch shape of the mixed kernel (warps per CTA, CTAs per SM: (4,5),
 * (4,4), (2,9), (8,2); see map_autotune_shapes); trial t * 4 + v is target t
 * with shape v.  *chosen = the trial in use for the mixed build,
 * ms[0..*nvariants) = each trial's time on the tuning call's inputs (0 when
 * not run).  ms must hold at least 32 floats. */
int map_get_autotune(map_ctx* ctx, int* chosen, float* ms, int* nvariants);

/* The autotuner's launch shapes as launched on the context's device: per
 * shape v < *nshapes, warps_per_cta[v], ctas_per_sm[v] (the CTAs per SM the
 * persistent launch uses: the shape's own count, lowered to what the device
 * keeps resident at once) and registers[v] per thread (registers may be
 * NULL).  The arrays must hold at least 8 ints.  Errors: MAP_EINVAL (NULL
 * ctx or array), MAP_ECUDA. */
int map_autotune_shapes(map_ctx* ctx, int* warps_per_cta, int* ctas_per_sm, int* registers, int* nshapes);

/* How map_batch's whole-step graph has been used by this context: captures,
 * replays, and replays that fell back to the eager step (lists outgrew their
 * buffers).  Any pointer may be NULL.  Errors: MAP_EINVAL (ctx NULL). */
int map_batch_graph_stats(map_ctx* ctx, int64_t* captures, int64_t* replays, int64_t* fallbacks);

/* ------------------------------------------------------------ serving */

/* A request loop with continuous batching (the paper has no counterpart: it
 * maps one snapshot at a time).  Requests carry host arrays; the server runs
 * up to `slots` of them at once, each on its own context (its octree and
 * pair-list workspace stays allocated between requests) and CUDA stream, so
 * their work overlaps on the device.  Queued requests are admitted in arrival
 * order as soon as a slot is idle and the request's device-memory estimate
 * fits hbm_budget next to what running requests, idle slots' cached
 * workspace and the resident grids hold (idle caches, then the least
 * recently used resident grids that no running request maps onto, are
 * released to make room).  Grids are kept resident by id: a request whose
 * grid_id is >= 0 uploads its grid only when no resident grid has that id,
 * and maps onto the resident copy otherwise.  A request runs: copy-in of its
 * particles (and of its grid when not resident) through its slot's pinned
 * staging buffers, solve_h, map_particles_to_cells, copy-out.  No step waits
 * for the whole device: allocations are stream-ordered on the slot's stream.
 * Its result depends on its own inputs only, so it is bit-identical alone and
 * in any mix.  Threads: submit, wait and stats may be called from any thread. */
typedef struct map_server map_server;

typedef struct {
  int device;        /* CUDA device ordinal */
  int precision;     /* MAP_FP64 or MAP_MIXED (default) */
  int slots;         /* requests on the device at once; default 4, 1..64 */
  size_t hbm_budget; /* bytes the server may hold; 0 = 90% of the free memory at creation */
  double hfact;      /* Eq. (7); default 1.2 */
} map_server_config;

/* One mapping request.  All pointers are HOST memory owned by the caller and
 * must stay valid until map_server_wait returns for the request.  The grid
 * arrays follow map_grid; cell_mass (ncell) is required, cell_rho (ncell) and
 * h (n, the solved smoothing lengths) are optional outputs.  grid_id >= 0:
 * the grid is kept resident under that id after the request (the caller
 * guarantees that every request with the same id carries the same grid; a
 * request that finds its id resident does not read its grid arrays); < 0:
 * the grid is uploaded for this request alone. */
typedef struct {
  int64_t n;
  const double *x, *y, *z, *m;
  int64_t ncell, nface, nloop, nvert;
  const int64_t* cell_face_off;
  const int64_t* face_vert_off;
  const int32_t* face_vert;
  const double *face_plane, *vx, *vy, *vz, *site;
  double* cell_mass;
  double* cell_rho;
  double* h;
  int64_t grid_id;
} map_request;

typedef struct {
  int status;            /* MAP_OK, or MAP_ENOMEM when the request alone exceeds the budget, or the
                            first error of its steps */
  int64_t n_pairs;       /* pair integrals of the request */
  double total_mass;     /* sum_i M_i */
  double queue_ms;       /* submit to admission */
  double latency_ms;     /* submit to results in host memory */
  size_t bytes_reserved; /* the admission estimate */
} map_request_result;

void map_server_config_default(map_server_config* cfg);

/* Start a server (its contexts, streams and worker threads).
 * Errors: MAP_EINVAL, MAP_ENOMEM, MAP_ECUDA. */
int map_server_create(const map_server_config* cfg, map_server** srv);

/* Queue a request; *ticket identifies it.  Returns at once.
 * Errors: MAP_EINVAL (missing arrays, inconsistent sizes, server stopping). */
int map_server_submit(map_server* srv, const map_request* req, int64_t* ticket);

/* Block until the request is done and fill *res (may be NULL).  A ticket can
 * be waited for once.  Errors: MAP_EINVAL (unknown ticket). */
int map_server_wait(map_server* srv, int64_t ticket, map_request_result* res);

/* Requests completed so far, running now, queued, and the bytes the server
 * holds or has reserved. */
int map_server_stats(map_server* srv, int64_t* completed, int* running, int64_t* queued, size_t* held_bytes);

/* Resident grids: uploads so far (requests that found no resident grid for
 * their id), hits (requests that mapped onto a resident grid), grids
 * resident now and their device bytes.  Any pointer may be NULL. */
int map_server_grid_stats(map_server* srv, int64_t* uploads, int64_t* hits, int64_t* resident, size_t* bytes);

/* Fail the queued requests, wait for the running ones, stop the workers and
 * free everything (resident grids included). */
void map_server_destroy(map_server* srv);

/* ------------------------------------------------------------ smoothing lengths (Section III-C, Eq. 7-9) */

/* Solve h_a = hfact * n_a(h_a)^(-1/3), n_a(h) = sum_b W(|r_a - r_b|, h)
 * (self term included) for every particle: Newton-Raphson (at most 30
 * iterations, converged at |dh|/h < 1e-10), else bisection on
 * [h0/16, 16 h0] (|dh|/h < 1e-12), else the estimate h0.  A MAP_MIXED
 * context sums the kernel in FP32 (on FP32 hi/lo splits of the coordinates),
 * in the bisection too, iterates Newton in FP32 (its converged step applied
 * in FP64) and stops it at |dh|/h < 1e-6, which gives h to ~1e-7 relative
 * (within 7e-7 of the FP64 context's h on a 2^20 clumpy cloud).  The initial
 * guess h0 is hfact * (side of the particle's octree leaf cube) /
 * (leaf count)^(1/3).
 * Writes p->h; route (optional, n int32) receives 0 Newton, 1 bisection,
 * 2 estimate.  Errors: MAP_EINVAL, MAP_ENOMEM, MAP_ECUDA. */
int solve_h(map_ctx* ctx, map_particles* p, int32_t* route, void* stream);

/* solve_h for nsnap independent particle sets (Eq. 7-9 for each; the
 * configuration of many uneven instances): parts[j].h receives exactly what
 * solve_h on parts[j] alone gives; routes (NULL, or nsnap pointers each NULL
 * or n int32) as in solve_h.  The sets are solved by the context's workers,
 * several at once, each on its own stream, ordered after and before
 * `stream`; the call returns when all are done.  As map_batch, the call
 * captures its whole step after running it (validation, octree built
 * without host reads, h solve, per set on its worker's stream) and a later
 * call naming the same buffers (x, y, z, h, routes) and sizes replays it as
 * one graph launch with one read of a flag word, computing from the
 * buffers' current values (the same h, bit for bit).  Counting contexts
 * never capture.  Errors: MAP_EINVAL, MAP_ENOMEM, MAP_ECUDA (the first one
 * met). */
int solve_h_batch(map_ctx* ctx, int nsnap, map_particles* parts, int32_t* const* routes, void* stream);

/* Captures and replays of solve_h_batch's graph.  Either pointer may be NULL.
 * Errors: MAP_EINVAL (ctx NULL). */
int solve_h_batch_graph_stats(map_ctx* ctx, int64_t* captures, int64_t* replays);


/* solve_h for callers that cannot allocate device memory (a process that has
 * handed all of the GPU's memory to its own pools, a pipeline that forbids
 * allocation after start-up).  The paper has no counterpart: this is a
 * deployment variant of solve_h (same octree and Newton/bisection kernels,
 * the same results bit for bit as solve_h on an MAP_FP64 context), taking
 * only caller arrays -- x, y, z (n doubles each, in the unit cube), h (n
 * doubles, out), route (n int32, out, may be NULL) -- and using as scratch one
 * fixed 24 MiB array in the library's device image, which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   - n is limited to 32768 particles; larger n returns MAP_ECAPACITY.  The
 *     octree's node arrays hold 65536 nodes and are used whole from the
 *     start; a tree that needs more returns MAP_ECAPACITY before anything is
 *     written past them, and the array stays ready for the next call.
 *     Ordinary inputs stay far below (about n/7 nodes at leaf size 16).  The
 *     largest tree we could construct from 32768 particles -- groups of 17
 *     spread over the eight cells of one deepest-level node, so that every
 *     group keeps a chain of nodes down to the deepest level and ends in
 *     eight leaves -- has about 48,000 nodes, and fits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and sets up a host-side table for that device.
 *   - The stream must not be capturing (MAP_EINVAL, the capture untouched):
 *     the call waits on its stream, which a capture does not allow.
 *   - All calls share the array and keep its last contents.  Calls whose work
 *     overlapped on the GPU would race on it, and calls from several host
 *     threads would also share the host table; so the library serialises them:
 *     a call holds a per-device lock until its own work on the GPU has
 *     finished (the call synchronises its stream before returning).
 *   - Errors: MAP_EINVAL, MAP_ECAPACITY, MAP_ECUDA. */
int solve_h_noalloc(const double* x, const double* y, const double* z, int64_t n, double hfact, double* h,
                    int32_t* route, void* stream);

/* ------------------------------------------------------------ pseudo-particles (Section III-A/B, Eq. 5) */

/* Build the octree of the full particle set (leaf capacity cfg.leaf_size),
 * walk it from the root and open a node when r_node = 0 or
 * s_node^2 > theta^2 r_node^2 with r_node the distance from the node's centre
 * of mass to the nearest of the nsrc sources (src: host array of 3*nsrc
 * doubles).  Accepted nodes become pseudo-particles (centre of mass, node
 * mass); an opened leaf yields its particles, which keep their h.  Then solve
 * the pseudo-particles' h as in solve_h over the node set (accepted nodes
 * plus opened leaves standing in for their particles, Section III-C), with
 * initial guess hfact * 2 s_node (Eq. 9).
 *
 * out: caller-owned device arrays of capacity out->n (x, y, z, m, h); on
 * return *n_pseudo holds the number written, ordered depth-first (children
 * in octant order).  kind (optional, capacity out->n int32): 0 node, 1
 * particle; ident (optional, int64): node label (leading-1 Morton prefix) or
 * particle index.  Synchronises the stream.
 * Errors: MAP_EINVAL, MAP_ECAPACITY (*n_pseudo = required count),
 * MAP_ENOMEM, MAP_ECUDA. */
int build_pseudo_particles(map_ctx* ctx, const map_particles* full, const double* src, int nsrc,
                           map_particles* out, int32_t* kind, int64_t* ident, int64_t* n_pseudo, void* stream);

/* Walk controls (Section III-B).  Besides Eq. (5), a node is opened when,
 * for some source, its bounding sphere (centre of mass, radius s_node)
 * reaches within r_part of it (r_node < r_part + s_node: around the sources
 * every leaf yields its particles), or when it is not a leaf and its
 * bounding sphere reaches within r_leaf (r_node < r_leaf + s_node: in the
 * annulus out to r_leaf the walk reaches at least the leaves).  It is also
 * opened when its centre of mass lies within the radius of a region recorded
 * in an earlier step and it is larger than the smallest size reached there
 * (|com - c| < R and s_node > s_min: the region memory of Section III-B,
 * whose recording needs the radiative transfer results and is the caller's).
 * Distances are compared squared, each product and sum rounded once, so the
 * walk is reproducible bit for bit.  0 turns r_part / r_leaf off. */
typedef struct {
  const double* src;     /* host, 3 doubles per source */
  int nsrc;              /* >= 1 */
  double r_part;         /* >= 0 */
  double r_leaf;         /* >= 0 */
  const double* regions; /* host, 5 doubles per region: centre x, y, z, radius R, smallest size s_min; may be NULL */
  int nregion;           /* >= 0 */
} map_walk;

/* build_pseudo_particles with the walk controls above (theta from the
 * context's configuration); the same outputs, ordering and errors, plus
 * MAP_EINVAL for a negative or non-finite control or region value. */
int build_pseudo_particles_walk(map_ctx* ctx, const map_particles* full, const map_walk* walk, map_particles* out,
                                int32_t* kind, int64_t* ident, int64_t* n_pseudo, void* stream);

/* ------------------------------------------------------------ measurement */

/* Measured issue rates of device `device`, in lane operations per second
 * (one FMA = one operation): FP32 FMA, the special-function unit
 * (reciprocal square root) and FP64 FMA, each from a grid of 16 blocks of
 * 256 threads per SM running eight independent dependency chains per thread,
 * timed with CUDA events after a warm-up launch (a few milliseconds each).
 * They are the denominators of the pair-integral kernel's roofline (its
 * operation model counts FP32 and special-function operations).  The paper
 * has no counterpart.  Synchronises the device.
 * Errors: MAP_EINVAL (NULL output), MAP_ECUDA. */
int map_device_peaks(int device, double* ffma, double* mufu, double* dfma);

#ifdef __cplusplus
}
#endif

#endif /* EXACTMAP_H */
