// Pair-list build: for every cell i, the particles a whose support may reach
// the cell.  The rule (the paper is silent; fixed so that lists are
// reproducible bit for bit) is
//     |r_a - s_i| < 2 h_a + R_i   and   n_f.r_a - d_f < 2 h_a for every face f,
// in FP64 with a fixed operation order and no FMA contraction
// (__dmul_rn/__dadd_rn/__dsqrt_rn).  Candidates come from a traversal of the
// particle octree pruned by node bounding box and largest h; lists are sorted
// by particle index within each cell.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace {

struct PairTree {
  const double *xs, *ys, *zs, *hs;
  const float* hs32;   // h in FP32 (the screen)
  const float* split;  // 6 per sorted position: FP32 hi/lo of x, y, z
  const int32_t* idx;
  const int64_t *nb, *ne, *fc;
  const int32_t* nch;
  const unsigned long long* bbox;
  const unsigned long long* hmax;
  const float* box32;  // outward-rounded FP32 boxes and largest h (8 floats per node)
};

struct PairGrid {
  const int64_t* cfo;
  const double4_32a* plane;  // absolute planes (the exact FP64 rule)
  const float4* face32;      // site-relative planes (n, d - n.s) in FP32 (screening)
  const double* site;
  const double* rad;
  const float* rin;  // inscribed radius: smallest site-to-face-plane distance, rounded down
};

// The exact rule, FP64, fixed order, no FMA contraction.
__device__ __forceinline__ bool exact_dist(double sx, double sy, double sz, double R, double x, double y, double z,
                                           double h) {
  const double dx = __dsub_rn(x, sx), dy = __dsub_rn(y, sy), dz = __dsub_rn(z, sz);
  const double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  return dist < __dadd_rn(__dmul_rn(2.0, h), R);
}
__device__ __forceinline__ bool exact_face(const double4_32a P, double x, double y, double z, double h) {
  const double s = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(P.x, x), __dmul_rn(P.y, y)), __dmul_rn(P.z, z)), P.w);
  return s < __dmul_rn(2.0, h);
}

// The pair rule, decided in FP32 wherever the FP32 value is farther from the
// threshold than a rigorous bound on its rounding error, and by the exact
// FP64 rule otherwise -- so the outcome is always the FP64 rule's.  The FP32
// separation comes from the hi/lo split of both points,
// (hi_a - hi_s) + (lo_a - lo_s), within a few ulp of the separation itself;
// with the rounding of h, R and the squares, all FP32 roundings together stay
// below 1e-6 of the magnitudes involved, and the margin is 1e-5.  No FP64
// operation runs unless a value falls inside the margin.
struct SiteSplit {
  float hx, lx, hy, ly, hz, lz, R, rin;
};

__device__ __forceinline__ bool pair_rule(const PairGrid& G, const PairTree& T, int64_t c, const SiteSplit& S,
                                          int64_t k) {
  const float* P = T.split + 6 * k;
  const float fx = (P[0] - S.hx) + (P[1] - S.lx);
  const float fy = (P[2] - S.hy) + (P[3] - S.ly);
  const float fz = (P[4] - S.hz) + (P[5] - S.lz);
  const float hf = T.hs32[k];
  const float reach = fmaf(2.f, hf, S.R);
  const float reach2 = reach * reach;
  const float d2 = fx * fx + fy * fy + fz * fz;
  if (d2 > reach2 * 1.00001f) return false;
  if (!(d2 < reach2 * 0.99999f) &&
      !exact_dist(G.site[3 * c], G.site[3 * c + 1], G.site[3 * c + 2], G.rad[c], T.xs[k], T.ys[k], T.zs[k], T.hs[k]))
    return false;
  const float thr = 2.f * hf;
  // every face test passes when the particle lies within 2h + r_in of the
  // site: each face plane is at least r_in from the site, so
  // n.r - d = n.(r - s) - (d - n.s) <= |r - s| - r_in < 2h for every face (the
  // 1e-4 relative margin covers the FP32 rounding many times over)
  const float tin = thr + S.rin;
  if (d2 < tin * tin * 0.9999f) return true;
  const float l1 = fabsf(fx) + fabsf(fy) + fabsf(fz);
  for (int64_t f = G.cfo[c]; f < G.cfo[c + 1]; ++f) {
    const float4 F = G.face32[f];
    const float sv = (F.x * fx + F.y * fy + F.z * fz) - F.w;
    const float marg = 1e-5f * (l1 + fabsf(F.w) + thr) + 1e-30f;
    if (sv > thr + marg) return false;
    if (sv >= thr - marg && !exact_face(G.plane[f], T.xs[k], T.ys[k], T.zs[k], T.hs[k])) return false;
  }
  return true;
}

// One warp walks the octree for 32 cells that are consecutive in Morton order
// of their sites (so close together), sharing the node loads: every lane
// tests each visited node against its own cell (FP32, outward-rounded box,
// 1e-6 absolute margin: 2 * largest h + cell radius) and the warp descends
// when any lane needs the node.  At a leaf, the (cell, particle) tests of the
// lanes that reach it are spread over all 32 lanes -- each lane's cell data
// sit in shared memory -- and every hit is appended to its cell's list
// (lanes with the same cell take consecutive places, in lane order).
// FILL = false: count pairs per cell, keeping the first PAIR_ROW of them in
// the cell's row of `out` (ncell x PAIR_ROW); FILL = true: write the pairs at
// off[c] (the cells of `order` whose count exceeded the row; their number is
// read from *n_dev).
constexpr int PAIR_ROW = 256;
constexpr int PT_WARPS = 4;  // warps per block of the traversal (1 and 2 measured: no faster)
// CTAs per SM the traversal is compiled for: 12 caps it at 40 registers (a
// few spilled) for 48 resident warps; the walk waits on its node and
// candidate loads, so the extra warps pay (2^20: 15.2 ms at 64 registers,
// 14.0 at 48, 13.6 at 40, 16.1 at 32)
constexpr int PT_MINB = 12;

struct WalkCells {  // per warp: the 32 lanes' cells, one entry per lane
  float hx[32], lx[32], hy[32], ly[32], hz[32], lz[32], R[32], rin[32];
  int64_t c[32], w[32], cnt[32];
  int32_t need[32];  // the lanes that reach the current leaf, in lane order
};

template <bool FILL>
__global__ void __launch_bounds__(PT_WARPS * 32, PT_MINB)
    pair_traverse(int64_t ncell, const int32_t* __restrict__ order, PairTree T, PairGrid G, int64_t* count,
                  const int64_t* __restrict__ off, int32_t* out, const unsigned long long* n_dev,
                  int64_t cap = INT64_MAX) {
  __shared__ int32_t s_stack[PT_WARPS][200];
  if (FILL && off[ncell] > cap) return;  // the list does not fit its buffer: nothing is written
  __shared__ WalkCells s_cells[PT_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const bool valid = t < (n_dev ? (int64_t)*n_dev : ncell);
  if (__all_sync(0xffffffffu, !valid)) return;
  const int64_t c = valid ? (order ? order[t] : t) : -1;
  double sx = 0, sy = 0, sz = 0, R = 0;
  if (valid) { sx = G.site[3 * c]; sy = G.site[3 * c + 1]; sz = G.site[3 * c + 2]; R = G.rad[c]; }
  const float fsx = (float)sx, fsy = (float)sy, fsz = (float)sz, fR = (float)R;
  WalkCells& W = s_cells[warp];
  W.hx[lane] = fsx; W.lx[lane] = (float)(sx - (double)fsx);
  W.hy[lane] = fsy; W.ly[lane] = (float)(sy - (double)fsy);
  W.hz[lane] = fsz; W.lz[lane] = (float)(sz - (double)fsz);
  W.R[lane] = fR;
  W.rin[lane] = valid ? G.rin[c] : 0.f;
  W.c[lane] = c;
  W.w[lane] = valid ? (FILL ? off[c] : c * PAIR_ROW) : 0;
  W.cnt[lane] = 0;
  int32_t* stack = s_stack[warp];
  int sp = 1;
  if (lane == 0) stack[0] = 0;
  __syncwarp();
  while (sp > 0) {
    const int32_t nd = stack[--sp];
    __syncwarp();
    const float4 b0 = reinterpret_cast<const float4*>(T.box32)[2 * (int64_t)nd];
    const float4 b1 = reinterpret_cast<const float4*>(T.box32)[2 * (int64_t)nd + 1];
    const float dx = fsx < b0.x ? b0.x - fsx : (fsx > b0.w ? fsx - b0.w : 0.f);
    const float dy = fsy < b0.y ? b0.y - fsy : (fsy > b1.x ? fsy - b1.x : 0.f);
    const float dz = fsz < b0.z ? b0.z - fsz : (fsz > b1.y ? fsz - b1.y : 0.f);
    const float reach = (2.f * b1.z + fR + 1e-6f) * 1.000001f;
    const bool need = valid && dx * dx + dy * dy + dz * dz <= reach * reach;
    const unsigned mneed = __ballot_sync(0xffffffffu, need);
    if (!mneed) continue;
    const unsigned link = __float_as_uint(b1.w);
    if (link == 0u) {
      const int64_t k0 = T.nb[nd];
      const int nl = (int)(T.ne[nd] - k0);
      const int nn = __popc(mneed);
      if (need) W.need[__popc(mneed & lt)] = lane;
      __syncwarp();
      // tests (needing cell i, particle j): chunks of up to 32 particles, g
      // cells per round, lane -> (i = r + lane / chunk, j = p + lane % chunk)
      const int chunk = nl < 32 ? nl : 32;
      const int g = chunk > 0 ? 32 / chunk : 1;
      const int li = chunk > 0 ? lane / chunk : 0, lj = chunk > 0 ? lane - li * chunk : 0;
      for (int p = 0; p < nl; p += chunk) {
        for (int r = 0; r < nn; r += g) {
          const int i = r + li, j = p + lj;
          const bool on = li < g && i < nn && j < nl;
          const int l = on ? W.need[i] : 0;
          bool hit = false;
          if (on) {
            SiteSplit SS;
            SS.hx = W.hx[l]; SS.lx = W.lx[l];
            SS.hy = W.hy[l]; SS.ly = W.ly[l];
            SS.hz = W.hz[l]; SS.lz = W.lz[l];
            SS.R = W.R[l];
            SS.rin = W.rin[l];
            hit = pair_rule(G, T, W.c[l], SS, k0 + j);
          }
          if (__any_sync(0xffffffffu, hit)) {
            const unsigned grp = __match_any_sync(0xffffffffu, hit ? l : 32 + lane);
            int64_t q = 0;
            if (hit) {
              q = W.cnt[l] + __popc(grp & lt);
              if (FILL || q < PAIR_ROW) out[W.w[l] + q] = T.idx[k0 + j];
            }
            __syncwarp();
            if (hit && (grp & lt) == 0) W.cnt[l] += __popc(grp);
            __syncwarp();
          }
        }
      }
    } else {
      const int nc = link == NODE_LINK_FAR ? T.nch[nd] : (int)(link & 15u);
      const int64_t c0 = link == NODE_LINK_FAR ? T.fc[nd] : (int64_t)(link >> 4);
      if (lane < nc) stack[sp + lane] = (int32_t)(c0 + nc - 1 - lane);
      sp += nc;
      __syncwarp();
    }
  }
  if (!FILL && valid) count[c] = W.cnt[lane];
}

// The same walk with one warp per cell, for grids with many particles per
// cell (few, large cells): lanes test a node's children in parallel, the
// particles of the leaves the cell reaches are gathered in a buffer, and all
// 32 lanes apply the pair rule to 32 candidates at a time.  Output as
// pair_traverse (any order: each cell's list is sorted afterwards).
constexpr int WALK_STK = 160;   // a popped node pushes at most 8 of its children; 22 levels at most
constexpr int WALK_CAND = 512;  // candidate positions gathered before they are tested

template <bool FILL>
__global__ void __launch_bounds__(128) pair_walk_warp(int64_t ncell, const int32_t* __restrict__ cells, PairTree T,
                                                      PairGrid G, int64_t* count, const int64_t* __restrict__ off,
                                                      int32_t* out, const unsigned long long* n_dev,
                                                      int64_t cap = INT64_MAX) {
  __shared__ int32_t s_stk[4][WALK_STK];
  if (FILL && off[ncell] > cap) return;  // the list does not fit its buffer: nothing is written
  __shared__ int32_t s_cand[4][WALK_CAND];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = blockIdx.x * 4 + warp;
  if (t >= (n_dev ? (int64_t)*n_dev : ncell)) return;  // whole warp
  const int64_t c = cells ? cells[t] : t;
  const double sx = G.site[3 * c], sy = G.site[3 * c + 1], sz = G.site[3 * c + 2], R = G.rad[c];
  const float fsx = (float)sx, fsy = (float)sy, fsz = (float)sz, fR = (float)R;
  SiteSplit SS;
  SS.hx = fsx; SS.lx = (float)(sx - (double)fsx);
  SS.hy = fsy; SS.ly = (float)(sy - (double)fsy);
  SS.hz = fsz; SS.lz = (float)(sz - (double)fsz);
  SS.R = fR;
  SS.rin = G.rin[c];
  int32_t* stk = s_stk[warp];
  int32_t* cand = s_cand[warp];
  int64_t w = FILL ? off[c] : c * PAIR_ROW;
  int64_t cnt = 0;
  int sp = 1, nc_ = 0;  // stack depth, candidates held
  if (lane == 0) stk[0] = 0;
  __syncwarp();
  // test the candidates held, 32 at a time
  auto flush = [&]() {
    __syncwarp();  // the candidates written by every lane are visible
    for (int b = 0; b < nc_; b += 32) {
      const int j = b + lane;
      const bool hit = j < nc_ && pair_rule(G, T, c, SS, cand[j]);
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int64_t q = cnt + __popc(m & ((1u << lane) - 1u));
        if (FILL || q < PAIR_ROW) out[w + q] = T.idx[cand[j]];
      }
      cnt += __popc(m);
    }
    __syncwarp();
    nc_ = 0;
  };
  while (sp > 0) {
    const int nd = stk[sp - 1];
    --sp;
    const int nch = T.nch[nd];
    if (nch == 0) {  // the root is a leaf
      const int64_t a0 = T.nb[nd], a1 = T.ne[nd];
      for (int64_t a = a0; a < a1; a += WALK_CAND) {
        const int k = (int)((a1 - a) < WALK_CAND ? (a1 - a) : WALK_CAND);
        __syncwarp();
        for (int i = lane; i < k; i += 32) cand[i] = (int32_t)(a + i);
        __syncwarp();
        nc_ = k;
        flush();
      }
      continue;
    }
    const int64_t c0 = T.fc[nd];
    bool need = false, leaf = false;
    if (lane < nch) {
      const float* b = T.box32 + 8 * (c0 + lane);
      const float dx = fsx < b[0] ? b[0] - fsx : (fsx > b[3] ? fsx - b[3] : 0.f);
      const float dy = fsy < b[1] ? b[1] - fsy : (fsy > b[4] ? fsy - b[4] : 0.f);
      const float dz = fsz < b[2] ? b[2] - fsz : (fsz > b[5] ? fsz - b[5] : 0.f);
      const float reach = (2.f * b[6] + fR + 1e-6f) * 1.000001f;
      need = dx * dx + dy * dy + dz * dz <= reach * reach;
      leaf = need && T.nch[c0 + lane] == 0;
    }
    const unsigned ml = __ballot_sync(0xffffffffu, leaf), mi = __ballot_sync(0xffffffffu, need && !leaf);
    const int ni = __popc(mi);
    __syncwarp();  // every lane has read the popped entry
    if (sp + ni > WALK_STK) break;  // unreachable for trees of at most 22 levels
    if (need && !leaf) stk[sp + ni - 1 - __popc(mi & ((1u << lane) - 1u))] = (int)(c0 + lane);
    sp += ni;
    // leaf children: gather their particles, testing whenever the buffer fills
    unsigned m = ml;
    while (m) {
      const int bl = __ffs(m) - 1;
      m &= m - 1;
      const int64_t a0 = T.nb[c0 + bl], a1 = T.ne[c0 + bl];
      for (int64_t a = a0; a < a1;) {
        if (nc_ == WALK_CAND) flush();
        const int room = WALK_CAND - nc_;
        const int k = (int)((a1 - a) < room ? (a1 - a) : room);
        for (int i = lane; i < k; i += 32) cand[nc_ + i] = (int32_t)(a + i);
        nc_ += k;
        a += k;
      }
    }
    __syncwarp();
  }
  flush();
  if (!FILL && lane == 0) count[c] = cnt;
}

// Move the rows kept by the counting pass to their place in the list (one
// warp per cell); cells whose count exceeded the row go to the overflow list
// for the filling pass.
__global__ void __launch_bounds__(128) place_rows(int64_t ncell, const int64_t* __restrict__ count,
                                                  const int64_t* __restrict__ off, const int32_t* __restrict__ rows,
                                                  int32_t* out, int32_t* ovf, unsigned long long* n_ovf,
                                                  int64_t cap = INT64_MAX) {
  const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ncell || off[ncell] > cap) return;
  const int64_t n = count[c];
  if (n > PAIR_ROW) {
    if (lane == 0) ovf[atomicAdd(n_ovf, 1ULL)] = (int32_t)c;
    return;
  }
  const int32_t* src = rows + c * PAIR_ROW;
  int32_t* dst = out + off[c];
  for (int64_t i = lane; i < n; i += 32) dst[i] = src[i];
}

// Work items: cell c's n pairs in max(1, ceil(ceil(n/32)/K)) items of at
// most K blocks of 32 pairs, K = max(1, (np/32 + ncell) / tgt) from the
// list's pair count np = off[ncell] (read on the device).
__device__ __forceinline__ int64_t item_blocks(int64_t ncell, const int64_t* __restrict__ off, int64_t tgt) {
  const int64_t blocks = off[ncell] / 32 + ncell;
  return blocks / tgt > 1 ? blocks / tgt : 1;
}
__global__ void item_count(int64_t ncell, const int64_t* __restrict__ off, int64_t tgt, int64_t* cnt) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int64_t K = item_blocks(ncell, off, tgt);
  const int64_t blocks = (off[c + 1] - off[c] + 31) / 32;
  cnt[c] = blocks > K ? (blocks + K - 1) / K : 1;
}
__global__ void item_fill(int64_t ncell, const int64_t* __restrict__ off, const int64_t* __restrict__ ioff,
                          int64_t tgt, PairItem* items, int64_t cap = INT64_MAX) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell || ioff[ncell] > cap) return;
  const int64_t K = item_blocks(ncell, off, tgt);
  const int64_t b = off[c], n = off[c + 1] - b, span = 32 * K;
  int64_t lo = 0;
  for (int64_t i = ioff[c]; i < ioff[c + 1]; ++i) {
    const int64_t k = n - lo < span ? n - lo : span;
    items[i] = PairItem{b + lo, (int32_t)c, (int32_t)k};
    lo += k;
  }
}

// Sort each cell's pair list (<= 1024 entries) by particle index in shared
// memory, one warp per cell, bitonic, carrying f_ai: the keys are (index,
// position in the list) in 64 bits, and f_ai is gathered by position from a
// copy.  Longer lists are left to the library segmented sort.
__global__ void __launch_bounds__(128) sort_small_segments(int64_t ncell, const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ idx_in,
                                                           const double* __restrict__ frac_in, int32_t* idx,
                                                           double* frac) {
  __shared__ unsigned long long buf[4][1024];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x * 4LL + warp;
  if (c >= ncell) return;
  const int64_t b = off[c], e = off[c + 1];
  const int L = (int)(e - b);
  if (L > 1024 || L == 0) return;
  int P = 1;
  while (P < L) P <<= 1;
  unsigned long long* v = buf[warp];
  for (int i = lane; i < P; i += 32)
    v[i] = i < L ? ((unsigned long long)(uint32_t)idx_in[b + i] << 32) | (unsigned)i : ~0ULL;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a0 = v[i], a1 = v[ixj];
          const bool up = (i & k) == 0;
          if ((a0 > a1) == up) { v[i] = a1; v[ixj] = a0; }
        }
      }
      __syncwarp();
    }
  for (int i = lane; i < L; i += 32) {
    const unsigned long long key = v[i];
    idx[b + i] = (int32_t)(key >> 32);
    if (frac) frac[b + i] = frac_in[b + (int)(key & 0xffffffffu)];
  }
}

__global__ void mark_large(int64_t ncell, const int64_t* __restrict__ off, int64_t* beg, int64_t* end,
                           unsigned long long* nlarge) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  if (off[c + 1] - off[c] > 1024) {
    const unsigned long long k = atomicAdd(nlarge, 1ULL);
    beg[k] = off[c];
    end[k] = off[c + 1];
  }
}

__global__ void site_keys(int64_t n, const double* __restrict__ site, uint64_t* keys, int32_t* idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto q = [](double v) -> uint64_t {
    double s = floor(v * 1024.0);
    s = s < 0 ? 0 : (s > 1023 ? 1023 : s);
    return (uint64_t)s;
  };
  uint64_t k = 0;
  uint64_t xi = q(site[3 * i]), yi = q(site[3 * i + 1]), zi = q(site[3 * i + 2]);
  for (int b = 9; b >= 0; --b) k = (k << 3) | (((xi >> b) & 1) << 2) | (((yi >> b) & 1) << 1) | ((zi >> b) & 1);
  keys[i] = k;
  idx[i] = (int32_t)i;
}


}  // namespace

int pairs_build(map_ctx* ctx, const PreparedGrid* g, cudaStream_t s, const PairBufs& out) {
  DevTree& T = ctx->tree;
  const int64_t nc = g->ncell;
  const int tpb = 128;
  // cells visited in Morton order of their sites for coherent traversals
  uint64_t *k_in, *k_out;
  int32_t *o_in, *order;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[4], nc, &k_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[5], nc, &k_out));
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[6], nc, &o_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[14], nc, &order));  // kept for the inverse mapping's gather order
  site_keys<<<nblk(nc, 256), 256, 0, s>>>(nc, g->site, k_in, o_in); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t tb = 0;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, k_in, k_out, o_in, order, nc, 0, 30, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tb, k_in, k_out, o_in, order, nc, 0, 30, s));

  PairTree PT{T.xs, T.ys, T.zs, T.hs, T.hs32, T.split, T.idx, T.begin, T.end, T.first_child, T.nchild, T.bbox_bits,
              T.hmax_bits, T.box32};
  PairGrid PG{g->cell_face_off, g->face_plane, g->face32, g->site, g->rad, g->rin};
  int64_t *count, *off;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[0], nc + 1, &count));
  MAP_TRY(ensure_t(ctx, out.off ? *out.off : ctx->ws_pairs[1], nc + 1, &off));
  int32_t* rows;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[8], (size_t)nc * PAIR_ROW, &rows));
  CUDA_TRY(cudaMemsetAsync(count + nc, 0, sizeof(int64_t), s));
  // many particles per cell (few, large cells): one warp per cell
  const bool per_warp = T.n > 16 * nc;
  if (per_warp)
    pair_walk_warp<false><<<(unsigned)((nc + 3) / 4), tpb, 0, s>>>(nc, nullptr, PT, PG, count, nullptr, rows, nullptr);
  else
    pair_traverse<false><<<nblk(nc, PT_WARPS * 32), PT_WARPS * 32, 0, s>>>(nc, order, PT, PG, count, nullptr, rows, nullptr);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, count, off, nc + 1, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, count, off, nc + 1, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, off + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t np = ctx->h_scratch[0];
  // the list in the walk's order (deterministic); map_get_pairs and
  // map_copy_pairs sort each cell's entries by particle index when read
  int32_t* list;
  MAP_TRY(ensure_t(ctx, out.idx ? *out.idx : ctx->ws_pairs[3], np + 1, &list));
  // rows that fit go straight to the list; the other cells are walked again
  int32_t* ovf;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[9], nc, &ovf));
  unsigned long long* d_novf = ctx->d_counters + 6;
  CUDA_TRY(cudaMemsetAsync(d_novf, 0, sizeof(unsigned long long), s));
  place_rows<<<nblk(nc * 32, tpb), tpb, 0, s>>>(nc, count, off, rows, list, ovf, d_novf); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  if (per_warp)
    pair_walk_warp<true><<<(unsigned)((nc + 3) / 4), tpb, 0, s>>>(nc, ovf, PT, PG, nullptr, off, list, d_novf);
  else
    pair_traverse<true><<<nblk(nc, PT_WARPS * 32), PT_WARPS * 32, 0, s>>>(nc, ovf, PT, PG, nullptr, off, list, d_novf);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  ctx->n_pairs = np;
  ctx->pair_off = off;
  ctx->pair_idx = list;
  ctx->pairs_sorted = false;
  ctx->inv_ready = false;
  ctx->last_ncell = nc;
  return items_build(ctx, off, nc, np, ctx->item_target, s, out);
}

// Work items of a pair list: K blocks of 32 pairs at most, K chosen so that
// the launch has at least `target` items per resident warp (4 warps x 6 CTAs
// per SM); the autotuner may raise the target (smaller items).
int items_build(map_ctx* ctx, const int64_t* off, int64_t nc, int64_t np, int target, cudaStream_t s,
                const PairBufs& out) {
  (void)np;
  const int64_t tgt = (int64_t)target * ctx->sm_count * 24;
  int64_t *icnt, *ioff;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[0], nc + 1, &icnt));  // the pair counts are no longer needed
  MAP_TRY(ensure_t(ctx, out.ioff ? *out.ioff : ctx->ws_pairs[11], nc + 1, &ioff));
  item_count<<<nblk(nc, 256), 256, 0, s>>>(nc, off, tgt, icnt); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(icnt + nc, 0, sizeof(int64_t), s));
  size_t tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, icnt, ioff, nc + 1, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, icnt, ioff, nc + 1, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, ioff + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nitems = ctx->h_scratch[0];
  PairItem* items;
  double* part;
  MAP_TRY(ensure_t(ctx, out.items ? *out.items : ctx->ws_pairs[10], nitems, &items));
  MAP_TRY(ensure_t(ctx, out.part ? *out.part : ctx->ws_pairs[12], nitems, &part));
  item_fill<<<nblk(nc, 256), 256, 0, s>>>(nc, off, ioff, tgt, items); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  ctx->items = items;
  ctx->item_off = ioff;
  ctx->partial = part;
  ctx->n_items = nitems;
  return MAP_OK;
}

// pairs_build with no host reads: the list's and the items' sizes stay on
// the device; the buffers hold cap_pairs and cap_items, and a build that
// needs more writes nothing beyond them (its off[nc] or ioff[nc] says so).
int pairs_build_graph(map_ctx* ctx, const PreparedGrid* g, cudaStream_t s, const PairBufs& out, int64_t cap_pairs,
                      int64_t cap_items) {
  if (!out.off || !out.idx || !out.items || !out.ioff || !out.part) return MAP_EINVAL;
  DevTree& T = ctx->tree;
  const int64_t nc = g->ncell;
  const int tpb = 128;
  uint64_t *k_in, *k_out;
  int32_t *o_in, *order;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[4], nc, &k_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[5], nc, &k_out));
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[6], nc, &o_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[14], nc, &order));
  site_keys<<<nblk(nc, 256), 256, 0, s>>>(nc, g->site, k_in, o_in); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t tb = 0;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, k_in, k_out, o_in, order, nc, 0, 30, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tb, k_in, k_out, o_in, order, nc, 0, 30, s));
  PairTree PT{T.xs, T.ys, T.zs, T.hs, T.hs32, T.split, T.idx, T.begin, T.end, T.first_child, T.nchild, T.bbox_bits,
              T.hmax_bits, T.box32};
  PairGrid PG{g->cell_face_off, g->face_plane, g->face32, g->site, g->rad, g->rin};
  int64_t *count, *off;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[0], nc + 1, &count));
  MAP_TRY(ensure_t(ctx, *out.off, nc + 1, &off));
  int32_t* rows;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[8], (size_t)nc * PAIR_ROW, &rows));
  CUDA_TRY(cudaMemsetAsync(count + nc, 0, sizeof(int64_t), s));
  const bool per_warp = T.n > 16 * nc;
  if (per_warp)
    pair_walk_warp<false><<<(unsigned)((nc + 3) / 4), tpb, 0, s>>>(nc, nullptr, PT, PG, count, nullptr, rows, nullptr);
  else
    pair_traverse<false><<<nblk(nc, PT_WARPS * 32), PT_WARPS * 32, 0, s>>>(nc, order, PT, PG, count, nullptr, rows, nullptr);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, count, off, nc + 1, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, count, off, nc + 1, s));
  int32_t* list;
  MAP_TRY(ensure_t(ctx, *out.idx, cap_pairs + 1, &list));
  int32_t* ovf;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[9], nc, &ovf));
  unsigned long long* d_novf = ctx->d_counters + 6;
  CUDA_TRY(cudaMemsetAsync(d_novf, 0, sizeof(unsigned long long), s));
  place_rows<<<nblk(nc * 32, tpb), tpb, 0, s>>>(nc, count, off, rows, list, ovf, d_novf, cap_pairs); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  if (per_warp)
    pair_walk_warp<true><<<(unsigned)((nc + 3) / 4), tpb, 0, s>>>(nc, ovf, PT, PG, nullptr, off, list, d_novf,
                                                                  cap_pairs);
  else
    pair_traverse<true><<<nblk(nc, PT_WARPS * 32), PT_WARPS * 32, 0, s>>>(nc, ovf, PT, PG, nullptr, off, list, d_novf, cap_pairs);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  // the work items (the item size from the device-side pair count)
  const int64_t tgt = (int64_t)ctx->item_target * ctx->sm_count * 24;
  int64_t *icnt, *ioff;
  MAP_TRY(ensure_t(ctx, ctx->ws_pairs[0], nc + 1, &icnt));
  MAP_TRY(ensure_t(ctx, *out.ioff, nc + 1, &ioff));
  item_count<<<nblk(nc, 256), 256, 0, s>>>(nc, off, tgt, icnt); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(icnt + nc, 0, sizeof(int64_t), s));
  tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, icnt, ioff, nc + 1, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, icnt, ioff, nc + 1, s));
  PairItem* items;
  double* part;
  MAP_TRY(ensure_t(ctx, *out.items, cap_items, &items));
  MAP_TRY(ensure_t(ctx, *out.part, cap_items, &part));
  item_fill<<<nblk(nc, 256), 256, 0, s>>>(nc, off, ioff, tgt, items, cap_items); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  ctx->n_pairs = -1;
  ctx->pair_off = off;
  ctx->pair_idx = list;
  ctx->pairs_sorted = false;
  ctx->inv_ready = false;
  ctx->last_ncell = nc;
  ctx->items = items;
  ctx->item_off = ioff;
  ctx->partial = part;
  ctx->n_items = -1;
  return MAP_OK;
}

// Sorts the last mapping call's lists by particle index within each cell,
// f_ai alongside, in place (through copies), on stream s.
int pairs_sort_lists(map_ctx* ctx, cudaStream_t s) {
  if (ctx->pairs_sorted || !ctx->pair_off || !ctx->pair_idx) return MAP_OK;
  const int64_t nc = ctx->last_ncell, np = ctx->n_pairs;
  if (np > 0) {
    int32_t* idx = const_cast<int32_t*>(ctx->pair_idx);
    double* frac = ctx->pair_frac;
    int32_t* idx_in;
    double* frac_in = nullptr;
    MAP_TRY(ensure_t(ctx, ctx->ws_pairs[2], np, &idx_in));
    CUDA_TRY(cudaMemcpyAsync(idx_in, idx, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (frac) {
      MAP_TRY(ensure_t(ctx, ctx->ws_pairs[13], np, &frac_in));
      CUDA_TRY(cudaMemcpyAsync(frac_in, frac, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    sort_small_segments<<<nblk(nc, 4), 128, 0, s>>>(nc, ctx->pair_off, idx_in, frac_in, idx, frac); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    int64_t *lb, *le;
    MAP_TRY(ensure_t(ctx, ctx->ws_misc[1], nc + 1, &lb));
    MAP_TRY(ensure_t(ctx, ctx->ws_misc[2], nc + 1, &le));
    unsigned long long* d_nl = ctx->d_counters + 5;
    CUDA_TRY(cudaMemsetAsync(d_nl, 0, sizeof(unsigned long long), s));
    mark_large<<<nblk(nc, 256), 256, 0, s>>>(nc, ctx->pair_off, lb, le, d_nl); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, d_nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nlarge = ctx->h_scratch[0];
    if (nlarge > 0) {
      size_t tb = 0;
      if (frac) {
        CUDA_TRY(cub::DeviceSegmentedSort::SortPairs(nullptr, tb, idx_in, idx, frac_in, frac, np, nlarge, lb, le, s));
        MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
        CUDA_TRY(cub::DeviceSegmentedSort::SortPairs(ctx->cub_tmp.p, tb, idx_in, idx, frac_in, frac, np, nlarge, lb,
                                                     le, s));
      } else {
        CUDA_TRY(cub::DeviceSegmentedSort::SortKeys(nullptr, tb, idx_in, idx, np, nlarge, lb, le, s));
        MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
        CUDA_TRY(cub::DeviceSegmentedSort::SortKeys(ctx->cub_tmp.p, tb, idx_in, idx, np, nlarge, lb, le, s));
      }
      CUDA_TRY(cudaStreamSynchronize(s));  // the lists are complete for any stream
    }
  }
  ctx->pairs_sorted = true;
  return MAP_OK;
}
