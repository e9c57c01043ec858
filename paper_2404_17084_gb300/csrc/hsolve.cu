// Smoothing-length solve (Section III-C, Eq. 7-9): h = hfact n(h)^(-1/3) with
// n(h) = sum_b W(r_ab, h), by Newton-Raphson on g(h) = h - hfact n(h)^(-1/3)
// from the estimate h0 = hfact side/count^(1/3) of the particle's leaf, then
// bisection on [h0/16, 16 h0] (bracket located from h0 outwards, see below),
// then the estimate itself.
//
// One warp per octree leaf.  The warp walks the tree once for the whole leaf
// (children of a node tested by parallel lanes) and keeps, in shared memory,
// the particle ranges of every leaf that comes within R = 2.5 max(h0) of the
// leaf's box.  Leaves are visited depth-first, i.e. in the Morton order of the
// sorted particle arrays, so adjacent accepted leaves merge into one range,
// and a node whose box lies wholly within R of the query box is taken as one
// range without descending (the same candidates its leaves would give).  The
// ranges are expanded into a list of positions that the particles of the leaf
// sum over with all 32 lanes.  A particle's first pass over that list also
// keeps, in a list of its own, the candidates within min(2.5 h, R) of it;
// its later steps sum over that shorter list while it covers the support
// (2h <= 0.999 of its radius).  When an iterate outgrows the leaf's list
// (2h > R), or the list is far larger than needed (R > 8h), it is gathered
// again with R = 2.5 h; the next particle keeps whatever list covers it.  A
// list longer than the buffer is expanded and summed chunk by chunk; ranges
// beyond their own buffer come from a resumable walk.  The Newton and
// bisection rules are those of the per-particle definition; only the order
// of the sums differs.
//
// Mixed build: Newton and bisection sums in FP32 (on hi/lo-split
// coordinates); the Newton iterate, its step and the list-coverage tests in
// FP32 too (hfact as an FP32 hi/lo pair), the converged step applied in FP64;
// stop at |dh| < 1e-6 h.  FP64 build: every sum in FP64 behind an FP32
// distance screen with a 1e-5 relative margin, stop at 1e-10.
#include <type_traits>

#include "internal.cuh"

namespace {

constexpr int HS_WARPS = 2;     // warps per block: small blocks free their SM slots as soon as their
                                // warps end, and a warp's leaves take very different times
constexpr int HS_RNG = 384;     // particle ranges held per warp
constexpr int HS_CAP = 1024;    // candidate positions held per warp (a multiple of 32)
// Depth-first stack: the tree has at most 22 levels and a popped node pushes at
// most its 8 children, so at most 8 + 7 * 21 = 155 entries are live.
constexpr int HS_STK = 160;
constexpr int HS_PCAP = 512;   // one particle's own candidates (within 2.5 h of it)
constexpr unsigned FULL = 0xffffffffu;

struct HsTree {
  const double *xs, *ys, *zs;
  const float* split;  // 6 per sorted position: FP32 hi/lo of x, y, z
  const int64_t *nb, *ne, *fc;
  const int32_t *nch, *owner, *idx;
  const float* box32;  // 8 per node: outward-rounded FP32 box, hmax, pad
};

struct HsWarp {
  int2 rng[HS_RNG];
  int32_t cand[HS_CAP];
  int32_t pcand[HS_PCAP];  // the current particle's candidates within pR of it
  int32_t stk[HS_STK];
};

// Candidate list held by one warp (values uniform across its lanes); S is
// the build's type for h (FP32 in the mixed build, FP64 in the FP64 build).
template <typename S>
struct HsBuf {
  float q[6];       // query box: the leaf's outward-rounded FP32 box
  S R;              // gather radius
  int nr;           // ranges held
  bool rng_done;    // the walk finished: the ranges cover every candidate
  int64_t total;    // positions in the ranges held
  bool expanded;    // cand holds all of them
  int64_t pk;       // the particle whose own list pcand holds (-1: none)
  S pR;             // its radius
  int pn;           // its length
};

__device__ __forceinline__ double w_m4(double q) {
  if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
  if (q < 2.0) { const double t = 2.0 - q; return 0.25 * t * t * t; }
  return 0.0;
}
__device__ __forceinline__ double dw_m4(double q) {
  if (q < 1.0) return -3.0 * q + 2.25 * q * q;
  if (q < 2.0) { const double t = 2.0 - q; return -0.75 * t * t; }
  return 0.0;
}

// True when no point of box b is within R of box q.  Both boxes are rounded
// outward; the FP32 arithmetic on coordinates in the unit cube is covered by
// the margin folded into Rm.
__device__ __forceinline__ bool box_far_box(const float* __restrict__ b, const float* q, float Rm) {
  const float dx = fmaxf(fmaxf(b[0] - q[3], q[0] - b[3]), 0.f);
  const float dy = fmaxf(fmaxf(b[1] - q[4], q[1] - b[4]), 0.f);
  const float dz = fmaxf(fmaxf(b[2] - q[5], q[2] - b[5]), 0.f);
  return dx * dx + dy * dy + dz * dz > Rm * Rm;
}

// True when every point of box b is within R of box q (then every leaf below
// the node would be gathered; taking the node whole gives the same set).
__device__ __forceinline__ bool box_within_box(const float* __restrict__ b, const float* q, float R) {
  const float dx = fmaxf(fmaxf(b[3] - q[3], q[0] - b[0]), 0.f);
  const float dy = fmaxf(fmaxf(b[4] - q[4], q[1] - b[1]), 0.f);
  const float dz = fmaxf(fmaxf(b[5] - q[5], q[2] - b[2]), 0.f);
  return dx * dx + dy * dy + dz * dz <= R * R;
}

// Resumable depth-first walk over the leaves whose box comes within R of the
// query box (state uniform across the warp; the stack lives in W.stk).
struct HsWalk {
  float Rm;       // R with the FP32 margin folded in
  float Rin;      // R for whole-node acceptance
  int sp;         // stack depth
  int64_t c0;     // first child of the node whose range children are pending
  unsigned m;     // pending range children (leaves, or nodes taken whole)
};

__device__ __forceinline__ float walk_margin(double R) { return (float)(R + 1e-6) * 1.000001f; }
__device__ __forceinline__ float walk_margin(float R) { return (R + 1e-6f) * 1.000001f; }

template <typename S>
__device__ __forceinline__ void walk_begin(const HsTree& T, HsWarp& W, HsWalk& it, S R, int& nr) {
  __syncwarp();
  it.Rm = walk_margin(R);
  it.Rin = (float)R;
  it.m = 0u;
  it.c0 = 0;
  it.sp = 0;
  nr = 0;
  if (T.nch[0] == 0) {
    if ((threadIdx.x & 31) == 0) W.rng[0] = make_int2((int)T.nb[0], (int)T.ne[0]);
    nr = 1;
  } else {
    if ((threadIdx.x & 31) == 0) W.stk[0] = 0;
    it.sp = 1;
  }
  __syncwarp();
}

__device__ __forceinline__ bool walk_done(const HsWalk& it) { return it.sp == 0 && it.m == 0u; }

// Appends to W.rng[nr, HS_RNG) the next particle ranges of the walk, merging
// ranges that touch.  Returns the new count; stops when the buffer is full.
__device__ int walk_next(const HsTree& T, HsWarp& W, HsWalk& it, const float* q, int nr) {
  const int lane = threadIdx.x & 31;
  int last = nr > 0 ? W.rng[nr - 1].y : -1;
  __syncwarp();
  while (true) {
    if (it.m) {
      const int b = __ffs(it.m) - 1;
      const int a0 = (int)T.nb[it.c0 + b], a1 = (int)T.ne[it.c0 + b];
      if (a0 == last) {
        if (lane == 0) W.rng[nr - 1].y = a1;
      } else {
        if (nr == HS_RNG) break;
        if (lane == 0) W.rng[nr] = make_int2(a0, a1);
        ++nr;
      }
      last = a1;
      it.m &= it.m - 1u;
      continue;
    }
    if (it.sp == 0) break;
    const int nd = W.stk[it.sp - 1];
    --it.sp;
    // the node's link word: first child << 4 | child count (see the tree build)
    const unsigned link = __float_as_uint(T.box32[8 * (int64_t)nd + 7]);
    const int nc = link == NODE_LINK_FAR ? T.nch[nd] : (int)(link & 15u);
    const int64_t c0 = link == NODE_LINK_FAR ? T.fc[nd] : (int64_t)(link >> 4);
    bool hit = false, take = false;
    if (lane < nc) {
      const float4 b0 = reinterpret_cast<const float4*>(T.box32)[2 * (c0 + lane)];
      const float4 b1 = reinterpret_cast<const float4*>(T.box32)[2 * (c0 + lane) + 1];
      const float bx[6] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
      hit = !box_far_box(bx, q, it.Rm);
      take = hit && (__float_as_uint(b1.w) == 0u || box_within_box(bx, q, it.Rin));
    }
    const unsigned mt = __ballot_sync(FULL, take), mi = __ballot_sync(FULL, hit && !take);
    const int ni = __popc(mi);
    __syncwarp();  // every lane has read the popped entry before it is overwritten
    if (it.sp + ni > HS_STK) { it.sp = 0; break; }  // unreachable for trees of at most 22 levels
    // descended children pushed in reverse so that they pop in child order;
    // the ranges of this node's children are taken first, which keeps the
    // walk depth-first only within a node -- merging is an optimisation, and
    // the set of positions is the same in any order
    if (hit && !take) W.stk[it.sp + ni - 1 - __popc(mi & ((1u << lane) - 1u))] = (int)(c0 + lane);
    it.sp += ni;
    it.c0 = c0;
    it.m = mt;
    __syncwarp();
  }
  __syncwarp();
  return nr;
}

// Lane partial sums of w(q) and 3 w + q w'(q) over list[0, cnt) for the
// particle at sorted position k.  A lane takes positions lane, lane + 32, ...
// in that order; two of them per pass, with the loads of both issued before
// either term is added (the order of the additions is unchanged).  With keep
// set, the candidates with q^2 < keep_q2 are also appended, in list order, to
// keep[*nkeep ...] (*nkeep = -1 when they do not fit in HS_PCAP).
template <bool F32, typename S>
__device__ __forceinline__ void warp_accum(const HsTree& T, const int32_t* list, int cnt, int64_t k, S h,
                                           float& s32, float& d32, double& s64, double& d64, int32_t* keep,
                                           float keep_q2, int* nkeep) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const float* P0 = T.split + 6 * k;
  const float hx = P0[0], lx = P0[1], hy = P0[2], ly = P0[3], hz = P0[4], lz = P0[5];
  const float inv_hf = 1.0f / (float)h;
  double x = 0.0, y = 0.0, z = 0.0, R2 = 0.0, inv_h = 0.0;
  if (!F32) {
    x = T.xs[k]; y = T.ys[k]; z = T.zs[k];
    R2 = 4.0 * (double)h * (double)h;
    inv_h = 1.0 / (double)h;
  }
  // q^2 of one candidate (FP32, as the screen), its terms added when inside
  auto term = [&](int64_t c, float2 a, float2 b, float2 cc) -> float {
    const float dx = ((a.x - hx) + (a.y - lx)) * inv_hf;
    const float dy = ((b.x - hy) + (b.y - ly)) * inv_hf;
    const float dz = ((cc.x - hz) + (cc.y - lz)) * inv_hf;
    const float q2 = dx * dx + dy * dy + dz * dz;
    if (F32) {
      if (q2 >= 4.f) return q2;
      const float q = sqrtf(q2);
      float w, dwq;
      if (q < 1.f) { w = 1.f - 1.5f * q2 + 0.75f * q2 * q; dwq = -3.f * q2 + 2.25f * q2 * q; }
      else { const float t = 2.f - q; w = 0.25f * t * t * t; dwq = -0.75f * t * t * q; }
      s32 += w;
      d32 += 3.f * w + dwq;
    } else {
      if (q2 > 4.00004f) return q2;  // FP32 screen, 1e-5 relative margin
      const double ex = T.xs[c] - x, ey = T.ys[c] - y, ez = T.zs[c] - z;
      const double r2 = ex * ex + ey * ey + ez * ez;
      if (r2 >= R2) return q2;
      const double q = sqrt(r2) * inv_h;
      const double w = w_m4(q);
      s64 += w;
      d64 += 3.0 * w + q * dw_m4(q);
    }
    return q2;
  };
  auto append = [&](bool pred, int32_t v) {
    const unsigned m = __ballot_sync(FULL, pred);
    if (*nkeep < 0) return;
    if (*nkeep + __popc(m) > HS_PCAP) { *nkeep = -1; return; }
    if (pred) keep[*nkeep + __popc(m & lt)] = v;
    *nkeep += __popc(m);
  };
  for (int j0 = 0; j0 < cnt; j0 += 64) {
    const int j = j0 + lane, j1 = j + 32;
    const bool v0 = j < cnt, v1 = j1 < cnt;
    int32_t c0 = 0, c1 = 0;
    float2 a = make_float2(0.f, 0.f), b = a, c = a, a1 = a, b1 = a, cc1 = a;
    if (v0) {
      c0 = list[j];
      const float2* P = reinterpret_cast<const float2*>(T.split + 6 * (int64_t)c0);
      a = P[0]; b = P[1]; c = P[2];
    }
    if (v1) {
      c1 = list[j1];
      const float2* Q = reinterpret_cast<const float2*>(T.split + 6 * (int64_t)c1);
      a1 = Q[0]; b1 = Q[1]; cc1 = Q[2];
    }
    const float q0 = v0 ? term(c0, a, b, c) : 1e30f;
    const float q1 = v1 ? term(c1, a1, b1, cc1) : 1e30f;
    if (keep) {
      append(v0 && q0 < keep_q2, c0);
      append(v1 && q1 < keep_q2, c1);
    }
  }
}

__device__ __forceinline__ float rcbrt_s(float v) { return rcbrtf(v); }
__device__ __forceinline__ double rcbrt_s(double v) { return rcbrt(v); }

template <typename V>
__device__ __forceinline__ V warp_total(V v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return __shfl_sync(FULL, v, 0);
}

// Expands ranges [r, nr) of W.rng, from offset off in range r, into W.cand
// (up to HS_CAP positions).  Returns the count; advances r and off.
__device__ int expand(HsWarp& W, int nr, int& r, int& off) {
  const int lane = threadIdx.x & 31;
  int c = 0;
  __syncwarp();
  while (r < nr && c < HS_CAP) {
    const int2 g = W.rng[r];
    const int len = g.y - g.x - off;
    const int t = len < HS_CAP - c ? len : HS_CAP - c;
    for (int j = lane; j < t; j += 32) W.cand[c + j] = g.x + off + j;
    c += t;
    off += t;
    if (off == g.y - g.x) { ++r; off = 0; }
  }
  __syncwarp();
  return c;
}

// Gathers the candidate ranges for radius R, and their positions when they fit.
template <typename S>
__device__ __forceinline__ void regather(const HsTree& T, HsWarp& W, HsBuf<S>& B, S R) {
  const int lane = threadIdx.x & 31;
  HsWalk it;
  B.R = R;
  walk_begin(T, W, it, R, B.nr);
  B.nr = walk_next(T, W, it, B.q, B.nr);
  B.rng_done = walk_done(it);
  int64_t tot = 0;
  for (int r = lane; r < B.nr; r += 32) tot += W.rng[r].y - W.rng[r].x;
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
  B.total = tot;
  B.expanded = false;
  if (B.rng_done && tot <= HS_CAP) {
    int r = 0, off = 0;
    expand(W, B.nr, r, off);
    B.expanded = true;
  }
}

// n(h) and dn/dh for the particle at sorted position k (warp-uniform result),
// in the build's type S for h (every test on h and the radii in S).
template <bool F32, typename S>
__device__ void warp_density(const HsTree& T, HsWarp& W, HsBuf<S>& B, int64_t k, S h, S& n, S& dn) {
  float s32 = 0.f, d32 = 0.f;
  double s64 = 0.0, d64 = 0.0;
  int none = 0;
  const bool own = B.pk == k && S(2) * h <= S(0.999) * B.pR && B.pR <= S(8) * h;
  if (own) {
    // the particle's own list covers its support at this h
    warp_accum<F32>(T, W.pcand, B.pn, k, h, s32, d32, s64, d64, nullptr, 0.f, &none);
  } else {
    if (S(2) * h > B.R || B.R > S(8) * h) regather(T, W, B, S(2.5) * h);
  }
  if (own) {
    // done above
  } else if (B.expanded) {
    // the leaf's list; the first pass for a particle also keeps its own
    // candidates within pR = min(2.5 h, R) of it for the next steps (the
    // leaf's list holds every candidate within R of the leaf's box, so of
    // the particle)
    if (B.pk != k) {
      const S pR = S(2.5) * h < B.R ? S(2.5) * h : B.R;
      const float kq = (float)(pR / h);
      int nk = 0;
      warp_accum<F32>(T, W.cand, (int)B.total, k, h, s32, d32, s64, d64, W.pcand, kq * kq * 1.00001f, &nk);
      __syncwarp();
      B.pk = k;
      B.pR = nk >= 0 ? pR : S(0);  // 0: nothing kept (it did not fit)
      B.pn = nk >= 0 ? nk : 0;
    } else {
      warp_accum<F32>(T, W.cand, (int)B.total, k, h, s32, d32, s64, d64, nullptr, 0.f, &none);
    }
  } else if (B.rng_done) {
    // the ranges are complete but longer than the position buffer
    int r = 0, off = 0;
    while (r < B.nr) {
      const int c = expand(W, B.nr, r, off);
      warp_accum<F32>(T, W.cand, c, k, h, s32, d32, s64, d64, nullptr, 0.f, &none);
    }
  } else {
    // more ranges than their buffer: one resumable walk, range chunk by chunk
    HsWalk it;
    int nr;
    walk_begin(T, W, it, B.R, nr);
    for (;;) {
      nr = walk_next(T, W, it, B.q, nr);
      int r = 0, off = 0;
      while (r < nr) {
        const int c = expand(W, nr, r, off);
        warp_accum<F32>(T, W.cand, c, k, h, s32, d32, s64, d64, nullptr, 0.f, &none);
      }
      if (walk_done(it)) break;
      nr = 0;
    }
    B.nr = 0;
    B.R = S(-1);  // the buffer no longer holds the first ranges: regather next time
  }
  if (F32) {
    const float ih = 1.0f / (float)h;
    const float norm = ih * ih * ih * (float)(1.0 / MAP_PI);
    n = (S)(warp_total(s32) * norm);
    dn = (S)(-warp_total(d32) * norm * ih);
  } else {
    const double ih = 1.0 / h;
    const double norm = ih * ih * ih * (1.0 / MAP_PI);
    n = warp_total(s64) * norm;
    dn = -warp_total(d64) * norm * ih;
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(HS_WARPS * 32)
    h_solve_leaves(int64_t n, HsTree T, const double* __restrict__ h0s, double hfact, double tol, double* hout,
                   int32_t* route) {
  // the build's type for h: the mixed build iterates in FP32 (its sums are
  // FP32, and GB300's FP64 rate is about 1/74 of its FP32 rate)
  using S = typename std::conditional<MIXED, float, double>::type;
  const S hf_s = (S)hfact, hf3_s = (S)(hfact / 3.0), tol_s = (S)tol;
  const S hf_lo = (S)(hfact - (double)hf_s);
  __shared__ HsWarp sw[HS_WARPS];
  HsWarp& W = sw[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t k0 = (blockIdx.x * (int64_t)HS_WARPS + (threadIdx.x >> 5)) * 32;
  if (k0 >= n) return;  // whole warp
  // leaves whose first particle lies in this warp's window of 32 positions
  int leaf = -1;
  bool head = false;
  if (k0 + lane < n) {
    leaf = T.owner[k0 + lane];
    head = T.nb[leaf] == k0 + lane;
  }
  unsigned heads = __ballot_sync(FULL, head);
  while (heads) {
    const int src = __ffs(heads) - 1;
    heads &= heads - 1;
    const int L = __shfl_sync(FULL, leaf, src);
    const int64_t a0 = T.nb[L], a1 = T.ne[L];
    double gmax = 0.0;
    for (int64_t k = a0 + lane; k < a1; k += 32) gmax = fmax(gmax, h0s[k]);
    for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(FULL, gmax, o));
    HsBuf<S> B;
#pragma unroll
    for (int i = 0; i < 6; ++i) B.q[i] = T.box32[8 * (int64_t)L + i];
    B.R = S(-1);
    B.nr = 0;
    B.total = 0;
    B.rng_done = false;
    B.expanded = false;
    B.pk = -1;
    B.pR = S(0);
    B.pn = 0;
    const S R0 = S(2.5) * (S)gmax;
    for (int64_t k = a0; k < a1; ++k) {
      // the leaf's list for its first particle; later particles keep the
      // list they find while it covers their support (warp_density
      // regathers when 2h > R or R > 8h)
      if (k == a0) regather(T, W, B, R0);
      // Newton in S: g = h - hfact t, g' = 1 + hfact/3 t^4 dn/dh with t = n^(-1/3)
      S hs = (S)h0s[k];
      const S lo_s = hs / S(16), hi_s = hs * S(16);
      double h = 0.0;
      bool ok = false;
      for (int it = 0; it < 30; ++it) {
        S nn, dn;
        warp_density<MIXED>(T, W, B, k, hs, nn, dn);
        const S t = rcbrt_s(nn);
        S f = hs - hf_s * t;
        if (MIXED) f -= hf_lo * t;  // hfact as an FP32 pair
        const S fp = S(1) + hf3_s * (t * t) * (t * t) * dn;
        const S d = f / fp;
        const S hn = hs - d;
        if (!(hn >= lo_s && hn <= hi_s)) break;
        if ((hn > hs ? hn - hs : hs - hn) < tol_s * hn) {
          // the mixed build applies its converged step in FP64 (the result
          // keeps FP64's spacing, not FP32's)
          h = MIXED ? (double)hs - (double)d : (double)hn;
          ok = true;
          break;
        }
        hs = hn;
      }
      int r = 0;
      if (!ok) {
        const double g0 = h0s[k];
        const double lo = g0 / 16.0, hi = g0 * 16.0;
        // (the mixed build bisects on its FP32 sums too: the root moves by
        // ~1e-7 relative, inside the build's 1e-6, and GB300's FP64 rate
        // is about 1/74 of its FP32 rate)
        auto g = [&](double hh) {
          S nn, dn;
          warp_density<MIXED>(T, W, B, k, (S)hh, nn, dn);
          return hh - hfact * rcbrt((double)nn);
        };
        // Bisection on [lo, hi] needs g(lo) < 0 < g(hi).  g(h)/h is
        // nondecreasing in h (w is nonincreasing in q, so sum_b w(r_ab/h)
        // grows with h), so the sign of g at either end follows from any
        // point between: step from h0 by factors of 2 towards the sign change
        // and bisect the first bracket found, evaluating g at lo or hi only
        // when the steps reach them.
        double a = lo, b = hi;
        bool bracket = true;
        if (g(g0) < 0.0) {
          a = g0;
          double y = 2.0 * g0;
          for (; y < hi; y *= 2.0) {
            if (g(y) < 0.0) a = y; else { b = y; break; }
          }
          if (y >= hi) bracket = g(hi) > 0.0;
        } else {
          b = g0;
          double y = 0.5 * g0;
          for (; y > lo; y *= 0.5) {
            if (g(y) < 0.0) { a = y; break; } else b = y;
          }
          if (y <= lo) bracket = g(lo) < 0.0;
        }
        if (!bracket) {
          h = g0;
          r = 2;
        } else {
          for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (a + b);
            if (g(mid) < 0.0) a = mid; else b = mid;
            if (b - a < 1e-12 * mid) break;
          }
          h = 0.5 * (a + b);
          r = 1;
        }
      }
      if (lane == 0) {
        const int32_t a = T.idx[k];
        hout[a] = h;
        if (route) route[a] = r;
      }
    }
  }
}

// Initial guess: hfact * side(leaf cube) / count^(1/3), per sorted position.
__global__ void h_guess_leaf(int64_t n, const int32_t* __restrict__ owner, const int32_t* __restrict__ lev,
                             const int64_t* __restrict__ nb, const int64_t* __restrict__ ne, double hfact,
                             double* h0s) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int32_t leaf = owner[k];
  double side = ldexp(1.0, -lev[leaf]);
  h0s[k] = hfact * side / cbrt((double)(ne[leaf] - nb[leaf]));
}

__global__ void gather_h0(int64_t n, const int32_t* __restrict__ idx, const double* __restrict__ h0, double* h0s) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  h0s[k] = h0[idx[k]];
}

}  // namespace

int h_solve_run(map_ctx* ctx, const double* x, const double* y, const double* z, int64_t n, double* h, int32_t* route,
                const double* h0_override, cudaStream_t s, bool graph) {
  if (graph) MAP_TRY(tree_build_graph(ctx, x, y, z, nullptr, nullptr, n, s));
  else MAP_TRY(tree_build(ctx, x, y, z, nullptr, nullptr, n, s));
  DevTree& T = ctx->tree;
  double* h0s;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[22], n, &h0s));
  const int tpb = 128;
  if (h0_override)
    gather_h0<<<nblk(n, tpb), tpb, 0, s>>>(n, T.idx, h0_override, h0s);
  else
    h_guess_leaf<<<nblk(n, tpb), tpb, 0, s>>>(n, T.owner, T.level, T.begin, T.end, ctx->cfg.hfact, h0s);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  const HsTree V{T.xs, T.ys, T.zs, T.split, T.begin, T.end, T.first_child, T.nchild, T.owner, T.idx, T.box32};
  const int64_t warps = (n + 31) / 32;
  const unsigned blocks = (unsigned)((warps + HS_WARPS - 1) / HS_WARPS);
  if (ctx->cfg.precision != MAP_FP64)
    h_solve_leaves<true><<<blocks, HS_WARPS * 32, 0, s>>>(n, V, h0s, ctx->cfg.hfact, 1e-6, h, route);
  else
    h_solve_leaves<false><<<blocks, HS_WARPS * 32, 0, s>>>(n, V, h0s, ctx->cfg.hfact, 1e-10, h, route);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
