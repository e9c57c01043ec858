// Pair integrals and cell sums (Section II-B, Eq. 1-3).
//
// Persistent kernel, one warp per cell at a time: a warp pulls a cell from a
// device work queue and takes the cell's pairs 32 at a time, one pair per
// lane.  Warps share nothing and never wait for one another.  The cell's
// site-relative face planes and edge records are read straight from global
// memory: every lane reads the same record, so each read is one broadcast
// transaction, served from L1 after the first block of pairs.
//
// For each face (r0 from the plane; the inside flag) and each directed edge
// of it (R0 and the along-edge coordinates of the vertices), every lane splits
// its edge integral K'_e into pieces -- at most one inner piece, two middle
// pieces and two pieces beyond the support -- as (r0, R0, lo, hi), the sign
// s_f s_e folded into the interval direction.  The pieces beyond the support
// (-r0 E(r0) dPhi, one atan2 for both) are added by the lane itself.  Inner
// and middle pieces are pushed onto two per-warp stacks, one per kind;
// whenever a stack holds 32 pieces the whole warp evaluates them together
// (every lane the same code), so the costly evaluations run with all lanes
// busy; the stacks carry over from edge to edge and are flushed after the
// last face.  Each result is added to its owner lane's compensated (Kahan)
// accumulator, lanes with the same owner in turn, so the order of additions
// is fixed and every result is bit-reproducible.
// (Mixed build: a face whose plane passes within 1e-4 h of the particle has
// its side and distance taken from the FP64 plane and position; its edges
// then run through the FP32 pipeline like any other.)
//
// Per pair: f_ai = [inside] + sum_f sum_e s_f s_e K'_e (see wedge.cuh).
// M_i = sum_a m_a f_ai is accumulated in FP64 and reduced across the warp;
// rho_i = M_i / V_i.
//
// That is the FP64 build's kernel (pair_integrals).  The mixed build's kernel
// (pair_integrals_mixed) adds a level of compaction between the face loop and
// the edges: only a lane whose face can reach its support queues the face's
// edges, as (pair, edge) records that the warp then splits 32 at a time.
#include <cub/cub.cuh>
#include <type_traits>

#include "internal.cuh"
#include "wedge.cuh"

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4_32a type; };

// Mixed build: a face whose plane passes within TAU (in units of h) of the
// particle has its side and distance decided in FP64: FP32 rounding (~1e-7 h)
// could otherwise put the particle on the wrong side of the plane; with the
// FP64 distance, the face's integrals are as accurate in FP32 as any other
// (they are smooth in r0, and continuous as the particle crosses the plane).
// A separate FP64 evaluation of such faces was measured: every cell of a
// 2^18 clumpy snapshot agreed with it and with the FP64 build to the same
// 3.1e-6, and the FP64 path's registers cost the kernel 15%.  Exact zeros (particle
// exactly on a plane or edge line) are moved to +EPS on the inner side in the
// FP64 build: the integral is continuous in the particle position, and
// treating every exact zero as 'inside' is one consistent displacement of the
// particle into the cell.
constexpr float TAU = 1e-4f;
constexpr double EPS = 1e-12;
constexpr unsigned FULL = 0xffffffffu;
constexpr int LCAP = 96;  // stack depth: < 32 left after a drain + up to 2 pieces per lane

// Exclusive warp prefix sum of v in {0, 1, 2} (two ballots); returns the
// warp total in *tot.
__device__ __forceinline__ int warp_excl2(int v, int* tot) {
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  const unsigned b0 = __ballot_sync(FULL, v & 1), b1 = __ballot_sync(FULL, v & 2);
  *tot = __popc(b0) + 2 * __popc(b1);
  return __popc(b0 & lt) + 2 * __popc(b1 & lt);
}

// One edge record (EDGE_STRIDE words, 16-byte aligned) in vector loads:
// e0..e2 the in-plane edge normal m, e3 its offset delta, e4..e6 the edge
// direction t, e7, e8 the vertices' positions along t.  The FP32 record is
// interleaved, (m.x, t.x, m.y, t.y), (m.z, t.z, a_A, a_B), (delta), so that
// the pairs the two-lane arithmetic takes sit in adjacent registers.
__device__ __forceinline__ void load_edge(const float* E, float& e0, float& e1, float& e2, float& e3, float& e4,
                                          float& e5, float& e6, float& e7, float& e8) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(E)), b = __ldg(reinterpret_cast<const float4*>(E) + 1);
  const float4 c = __ldg(reinterpret_cast<const float4*>(E) + 2);
  e0 = a.x; e4 = a.y; e1 = a.z; e5 = a.w; e2 = b.x; e6 = b.y; e7 = b.z; e8 = b.w; e3 = c.x;
}
__device__ __forceinline__ void load_edge(const double* E, double& e0, double& e1, double& e2, double& e3,
                                          double& e4, double& e5, double& e6, double& e7, double& e8) {
  const double2 a = reinterpret_cast<const double2*>(E)[0], b = reinterpret_cast<const double2*>(E)[1];
  const double2 c = reinterpret_cast<const double2*>(E)[2], d = reinterpret_cast<const double2*>(E)[3];
  const double2 f = reinterpret_cast<const double2*>(E)[4];
  e0 = a.x; e1 = a.y; e2 = b.x; e3 = b.y; e4 = c.x; e5 = c.y; e6 = d.x; e7 = d.y; e8 = f.x;
}

// Per-warp piece stacks (inner, middle) and the results' accumulators.
//
// FP32: col[o][l] sums the pieces of owner lane o that lane l evaluated, so
// that in a drain every lane adds into its own column (bank l, no conflicts
// and no ordering between lanes); after the last drain of a block each owner
// adds up its row (compensated) and clears it.  Every cell sees its own
// lane's pieces in program order, so the result is bit-reproducible.
// FP64: one accumulator per owner, lanes with the same owner adding in turn.
template <typename T>
struct WarpStacks {
  // FP32 adds the pieces beyond the support in the lane itself (one atan2
  // per edge); FP64, where an atan2 costs far more than the stacking, stacks
  // them as a third kind
  static constexpr int NK = sizeof(T) == 4 ? 2 : 3;
  static constexpr bool COL = sizeof(T) == 4;
  typename Vec4<T>::type e[NK][LCAP];  // (r0, R0, lo, hi): inner, middle[, beyond]
  unsigned char own[NK][LCAP];         // owner lane
  float col[COL ? 32 : 1][32];         // FP32: [owner][evaluating lane]
  T acc[COL ? 1 : 32];                 // FP64: per-owner sum of its pieces
  SnapDesc d;                          // the snapshot of the warp's current cell
};

// Evaluates the queued pieces: every stack holding 32 or more (all that is
// left when flush), 32 at a time from the top, and adds each result to its
// owner lane's accumulator.
template <typename T, bool MIXED>
__device__ __forceinline__ void drain(WarpStacks<T>& S, int& cnt0, int& cnt1, int& cnt2, bool flush,
                                   unsigned& t0, unsigned& t1, unsigned& t2) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int K, n;
    if (cnt1 >= 32 || (flush && cnt1 > 0)) { K = 1; n = cnt1 < 32 ? cnt1 : 32; cnt1 -= n; t1 += n; }
    else if (cnt0 >= 32 || (flush && cnt0 > 0)) { K = 0; n = cnt0 < 32 ? cnt0 : 32; cnt0 -= n; t0 += n; }
    else if (WarpStacks<T>::NK == 3 && (cnt2 >= 32 || (flush && cnt2 > 0))) {
      K = 2; n = cnt2 < 32 ? cnt2 : 32; cnt2 -= n; t2 += n;
    } else {
      break;
    }
    const int base = K == 0 ? cnt0 : (K == 1 ? cnt1 : cnt2);
    const bool on = lane < n;
    T v = T(0);
    int o = 32 + lane;  // a key no owner has, for idle lanes
    if constexpr (WarpStacks<T>::COL) {
      // every lane evaluates (an idle lane a copy of the first piece) and
      // adds its value or 0: no divergent region
      const int idx = base + (on ? lane : 0);
      const typename Vec4<T>::type P = S.e[K][idx];
      o = S.own[K][idx];
      if (K == 1) v = wedge::piece_mid<T, MIXED>(P.x, P.y, P.z, P.w);
      else v = wedge::piece_inner<T>(P.x, P.y, P.z, P.w);
      // FP32 pieces are stacked unfolded, their sign s_f s_e in the owner's bit 7
      v = __int_as_float(__float_as_int(v) ^ ((o & 0x80) << 24));
      S.col[o & 31][lane] += on ? v : 0.f;  // this lane's column: no other lane touches it
      __syncwarp();
    } else {
      if (on) {
        const typename Vec4<T>::type P = S.e[K][base + lane];
        o = S.own[K][base + lane];
        if (K == 1) v = wedge::piece_mid<T, MIXED>(P.x, P.y, P.z, P.w);
        else if (K == 0) v = wedge::piece_inner<T>(P.x, P.y, P.z, P.w);
        else if constexpr (WarpStacks<T>::NK == 3) v = -P.x * wedge::dphi(P.z, P.w, P.y);  // P.x = c0 (the push)
      }
      // lanes holding pieces of the same owner add in turn, in lane order
      const unsigned grp = __match_any_sync(FULL, o);
      const int rank = __popc(grp & ((1u << lane) - 1u));
      for (int r = 0;; ++r) {
        const bool mine = on && rank == r;
        if (!__any_sync(FULL, mine)) break;
        if (mine) S.acc[o] += v;  // FP64: plain sums are ample
        __syncwarp();
      }
    }
  }
}

// FP32: this lane's row of the column accumulators, summed with compensation
// (Kahan) in a fixed order and cleared for the next block.  Lane o starts at
// column o, so the 32 lanes read 32 different banks at every step.
__device__ __forceinline__ float take_row(float (*col)[32], int o, float& comp) {
  float s = 0.f, c = 0.f;
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    const int k = (j + o) & 31;
    const float y = col[o][k] - c;
    col[o][k] = 0.f;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  comp = c;
  return s;
}

// Mixed build: the particle in the cell's site-relative frame, in units of
// h, and its signed distance to a face plane (> 0 on the inner side), every
// rounding explicit (no contraction left to the compiler).
__device__ __forceinline__ void pair_frame(const SnapDesc& A, int32_t a, double sx, double sy, double sz, float& yx,
                                           float& yy, float& yz, float& hinv) {
  hinv = __frcp_rn((float)__ldg(A.h + a));
  yx = __fmul_rn((float)(__ldg(A.x + a) - sx), hinv);
  yy = __fmul_rn((float)(__ldg(A.y + a) - sy), hinv);
  yz = __fmul_rn((float)(__ldg(A.z + a) - sz), hinv);
}
__device__ __forceinline__ float face_r0s(const float4& F, float yx, float yy, float yz, float hinv) {
  return __fsub_rn(__fmul_rn(F.w, hinv), __fmaf_rn(F.x, yx, __fmaf_rn(F.y, yy, __fmul_rn(F.z, yz))));
}

// COUNT: also tally the work (face tests, edge records, pieces) for the
// operation count; a separate compilation, as the tally holds registers.
template <typename T, bool MIXED, int NW, int MINB, bool COUNT>
__global__ void __launch_bounds__(NW * 32, MINB) pair_integrals(BatchArgs B) {
  typedef typename Vec4<T>::type V4;
  __shared__ WarpStacks<T> stacks[NW];
  const int lane = threadIdx.x & 31;
  WarpStacks<T>& S = stacks[threadIdx.x >> 5];
  const SnapDesc& A = S.d;
  wedge::WorkCount wc;
  unsigned n_in = 0, n_mid = 0;  // stacked pieces evaluated by this warp
  unsigned n_out = 0;            // this lane's beyond-support intervals (FP32)
  unsigned n_out_st = 0;         // stacked beyond-support pieces evaluated by this warp (FP64)
  int n64 = 0;
  unsigned n_split = 0;  // middle intervals split at the foot (counted once, evaluated as two pieces)
  int cur = -1;          // snapshot held in S.d
  if constexpr (WarpStacks<T>::COL) {
    for (int r = 0; r < 32; ++r) S.col[r][lane] = 0.f;
    __syncwarp();
  }

  const int64_t total = queue_total(B);
  for (;;) {
    int64_t g = 0;
    if (lane == 0) g = (int64_t)atomicAdd(&B.counters[3], 1ULL);
    g = __shfl_sync(FULL, g, 0);
    if (g >= total) break;
    // the snapshot owning queue position g: last j with item_base[j] <= g
    int jl = 0, jh = B.nsnap - 1;
    while (jl < jh) {
      const int jm = (jl + jh + 1) >> 1;
      if (B.item_base[jm] <= g) jl = jm; else jh = jm - 1;
    }
    if (jl != cur) {
      __syncwarp();
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(B.snaps + jl);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&S.d);
      for (int i = lane; i < (int)(sizeof(SnapDesc) / 8); i += 32) dst[i] = src[i];
      __syncwarp();
      cur = jl;
    }
    const int64_t it = g - B.item_base[jl];
    const PairItem item = A.items[it];
    const int64_t c = item.cell;
    const V4* __restrict__ face = reinterpret_cast<const V4*>(A.face);
    const T* __restrict__ edge = reinterpret_cast<const T*>(A.edge);
    const int64_t f0 = A.cfo[c];
    const int nf = (int)(A.cfo[c + 1] - f0);
    const int64_t l0 = A.fvo[f0];
    const T* __restrict__ ecell = edge + l0 * EDGE_STRIDE;
    const int nedge = (int)(A.fvo[f0 + nf] - l0);
    double macc = 0.0;
    const int64_t pb = item.lo, pe = item.lo + item.cnt;
    for (int64_t p0 = pb; p0 < pe; p0 += 32) {
      const int64_t p = p0 + lane;
      const bool active = p < pe;
      T yx = T(0), yy = T(0), yz = T(0), hinv = T(0);
      int32_t a = 0;
      if (active) {
        a = A.pair_idx[p];
        const double hh = A.h[a];
        const double sx = A.site[3 * c], sy = A.site[3 * c + 1], sz = A.site[3 * c + 2];
        if (MIXED) {
          const float hi = 1.0f / (float)hh;
          yx = (float)(A.x[a] - sx) * hi;
          yy = (float)(A.y[a] - sy) * hi;
          yz = (float)(A.z[a] - sz) * hi;
          hinv = hi;
        } else {
          const double hi = 1.0 / hh;
          yx = (A.x[a] - sx) * hi;
          yy = (A.y[a] - sy) * hi;
          yz = (A.z[a] - sz) * hi;
          hinv = hi;
        }
      }
      if constexpr (!WarpStacks<T>::COL) S.acc[lane] = T(0);
      bool inside = true;
      double dacc = 0.0;
      int cnt0 = 0, cnt1 = 0, cnt2 = 0;  // stack heights (warp-uniform)
      T osum = T(0), ocmp = T(0);  // this lane's beyond-support terms (compensated)
      int kb = 0;
      int pk = -1;  // index of the edge record held in n0..n8
      T n0, n1, n2, n3, n4, n5, n6, n7, n8;
      for (int fi = 0; fi < nf; ++fi) {
        const V4 F = face[f0 + fi];
        const int ke = (int)(A.fvo[f0 + fi + 1] - l0);
        const T r0s = F.w * hinv - (F.x * yx + F.y * yy + F.z * yz);
        bool fin = r0s >= T(0);
        T r0 = fabs(r0s);
        if (!MIXED) r0 = r0 > T(EPS) ? r0 : T(EPS);
        bool inrange = active && r0 < T(2);
        const T c0f = wedge::c0_of(r0);
        if (COUNT && active) wc.faces++;
        inside = inside && fin;
        if (__any_sync(FULL, inrange)) {
          if (pk != kb) load_edge(ecell + kb * EDGE_STRIDE, n0, n1, n2, n3, n4, n5, n6, n7, n8);
          for (int k = kb; k < ke; ++k) {
            const T e0 = n0, e1 = n1, e2 = n2, e3 = n3, e4 = n4, e5 = n5, e6 = n6, e7 = n7, e8 = n8;
            // the next record (of this face or the next) loads while this one is used
            pk = k + 1;
            if (pk < nedge) load_edge(ecell + pk * EDGE_STRIDE, n0, n1, n2, n3, n4, n5, n6, n7, n8);
            // R0 = m.(p - v_a) (> 0 inside), along-edge vertex positions
            const T R0s = (e0 * yx + e1 * yy + e2 * yz) - e3 * hinv;
            const T base = e4 * yx + e5 * yy + e6 * yz;
            const bool ein = R0s >= T(0);
            T R0 = fabs(R0s);
            if (!MIXED) R0 = R0 > T(EPS) ? R0 : T(EPS);
            const wedge::EdgeSplit<T> P =
                wedge::split_edge_flat<T>(r0, R0, e7 * hinv - base, e8 * hinv - base, fin == ein, inrange);
            const int nin = P.v & 1u, nmid = ((P.v >> 1) & 1u) + ((P.v >> 2) & 1u);
            const int nout = ((P.v >> 3) & 1u) + ((P.v >> 4) & 1u);
            if (COUNT && inrange) {
              wc.edges++;
              if (P.v) wc.terms++;
              n_split += P.split;
            }
            // push this edge's pieces (warp-aggregated)
            int t0, t1, t2 = 0;
            const int o0 = cnt0 + warp_excl2(nin, &t0);
            const int o1 = cnt1 + warp_excl2(nmid, &t1);
            const unsigned char ln = (unsigned char)lane;
            T lo, hi;
            if (P.v & 1u) { P.get(0, lo, hi); S.e[0][o0] = V4{r0, R0, lo, hi}; S.own[0][o0] = ln; }
            if (P.v & 2u) { P.get(1, lo, hi); S.e[1][o1] = V4{r0, R0, lo, hi}; S.own[1][o1] = ln; }
            if (P.v & 4u) {
              const int q = o1 + ((P.v >> 1) & 1u);
              P.get(2, lo, hi); S.e[1][q] = V4{r0, R0, lo, hi}; S.own[1][q] = ln;
            }
            // beyond the support, in this lane: -c0 (dPhi_left + dPhi_right)
            // as the argument of the product of the two intervals' numbers
            // (R0^2 + lo hi) + i (hi - lo) R0 -- each angle lies in
            // (-pi/2, pi/2) and together they span less than pi -- one atan2
            // per edge, branch-free (an empty interval contributes 1)
            if constexpr (WarpStacks<T>::NK == 3) {
              const int o2 = cnt2 + warp_excl2(nout, &t2);
              if (P.v & 8u) { P.get(3, lo, hi); S.e[2][o2] = V4{c0f, R0, lo, hi}; S.own[2][o2] = ln; }
              if (P.v & 16u) {
                const int q = o2 + ((P.v >> 3) & 1u);
                P.get(4, lo, hi); S.e[2][q] = V4{c0f, R0, lo, hi}; S.own[2][q] = ln;
              }
            } else {
              T l3, h3, l4, h4;
              P.get(3, l3, h3);
              P.get(4, l4, h4);
              const bool v3 = P.v & 8u, v4 = P.v & 16u;
              const T R02 = R0 * R0;
              const T ar = v3 ? R02 + l3 * h3 : T(1), ai = v3 ? (h3 - l3) * R0 : T(0);
              const T br = v4 ? R02 + l4 * h4 : T(1), bi = v4 ? (h4 - l4) * R0 : T(0);
              const T re = ar * br - ai * bi, im = ar * bi + ai * br;
              const T y = -c0f * wedge::xatan2(im, re) - ocmp;
              const T t = osum + y;
              ocmp = (t - osum) - y;
              osum = t;
              if (COUNT) n_out += nout;
            }
            cnt0 += t0;
            cnt1 += t1;
            cnt2 += t2;
            __syncwarp();
            // evaluate full stacks, 32 pieces at a time from the top
            if (cnt0 >= 32 || cnt1 >= 32 || cnt2 >= 32)
              drain<T, MIXED>(S, cnt0, cnt1, cnt2, false, n_in, n_mid, n_out_st);
          }
        }
        kb = ke;
      }
      // flush what is left (fewer than 32 of each kind)
      if (cnt0 || cnt1 || cnt2) drain<T, MIXED>(S, cnt0, cnt1, cnt2, true, n_in, n_mid, n_out_st);
      __syncwarp();
      double pieces;
      if constexpr (WarpStacks<T>::COL) {
        float comp;
        const float s = take_row(S.col, lane, comp);
        pieces = (double)s - (double)comp;
      } else {
        pieces = (double)S.acc[lane];
      }
      if (active) {
        const double f = (inside ? 1.0 : 0.0) + dacc + pieces + ((double)osum - (double)ocmp);
        if (A.frac) A.frac[p] = f;
        macc += A.m[a] * f;
      }
      __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) macc += __shfl_down_sync(FULL, macc, o);
    if (lane == 0) A.partial[it] = macc;  // summed per cell by cell_sums
    __syncwarp();
  }
  if (!COUNT) return;
  // work tally: warp sums, one atomic per warp and counter
  auto wsum = [](unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;
  };
  const unsigned long long terms = wsum((unsigned long long)wc.terms), faces = wsum((unsigned long long)wc.faces);
  const unsigned long long edges = wsum((unsigned long long)wc.edges), fp64 = wsum((unsigned long long)n64);
  const unsigned long long split = wsum((unsigned long long)n_split);
  const unsigned long long outs = wsum((unsigned long long)n_out);
  if (lane == 0) {
    atomicAdd(&B.counters[1], terms);
    atomicAdd(&B.counters[2], fp64);
    atomicAdd(&B.counters[8], faces);
    atomicAdd(&B.counters[9], edges);
    atomicAdd(&B.counters[10], 2ull * n_in);
    atomicAdd(&B.counters[11], (unsigned long long)n_mid - split);  // a split interval: one interval, two pieces
    atomicAdd(&B.counters[12], outs + n_out_st);
    atomicAdd(&B.counters[13], split);
  }
}

// ---------------------------------------------------------------- mixed build
// The mixed build compacts the work twice.  The face loop runs with one pair
// per lane; a lane whose face is within its support -- plane within 2h and
// face bounding sphere not wholly beyond 2h (such a face contributes nothing:
// every point of it lies beyond the support, so the particle's projection is
// outside the polygon and the angles of its edges cancel) -- pushes one
// (pair, edge) record per edge of the face on a per-warp stack.  Every 32
// records the warp splits those 32 edges, one per lane, and pushes their
// inner and middle pieces on the piece stacks as before; the beyond-support
// part is evaluated in the lane.  All results go to the owner pair's row of
// the column accumulators.
constexpr int CCAP = 64;  // (pair, edge) records: < 32 left + up to 32 pushed per edge

// A work item's face records (plane, bounding sphere, loop end) are staged in
// the warp's shared memory when the cell has at most FSTAGE faces (read from
// global memory otherwise): the face loop then reads them as broadcasts,
// once per block of 32 pairs, without the global-memory latency.
constexpr int FSTAGE = 48;
struct MixWarp {
  float4 fpl[FSTAGE];    // the item's face planes (site-relative, FP32)
  float4 fsp[FSTAGE];    // their bounding spheres
  int fend[FSTAGE];      // loop end of each face, relative to the cell's first loop entry
  WarpStacks<float> st;  // piece stacks, column accumulators, snapshot
  uint4 cmb[CCAP];       // (r0 bits, c0 bits, edge record offset in floats, fin << 5 | owner)
  float4 py[2][32];      // per pair: (y.x, y.x, y.y, y.y), (y.z, y.z, 1/h, 1/h), y site-relative in units of h
};

// Splits the n (<= 32) records on top of the record stack, one per lane.
template <bool COUNT>
__device__ __forceinline__ void edge_round(MixWarp& M, const float* __restrict__ ecell, int base, int n, int& cnt0,
                                           int& cnt1, unsigned& n_in, unsigned& n_mid, wedge::WorkCount& wc,
                                           unsigned& n_split, unsigned& n_out) {
  WarpStacks<float>& S = M.st;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const bool on = lane < n;
  const uint4 C = M.cmb[base + (on ? lane : 0)];  // an idle lane takes a copy of the first record
  __syncwarp();  // the records are taken: new ones may overwrite them
  const int o = (int)(C.w & 31u);
  const bool fin = C.w & 32u;
  const float r0 = __uint_as_float(C.x), c0f = __uint_as_float(C.y);
  const float4 Y0 = M.py[0][o], Y1 = M.py[1][o];
  float e0, e1, e2, e3, e4, e5, e6, e7, e8;
  load_edge(ecell + C.z, e0, e1, e2, e3, e4, e5, e6, e7, e8);
  // R0 = m.y - delta/h and the foot's along-edge position e.y, side by side
  // in two-lane arithmetic, then the vertices' positions from the foot
  using wedge::f2;
  const f2 g = wedge::fma2(f2{e2, e6}, f2{Y1.x, Y1.y},
                           wedge::fma2(f2{e1, e5}, f2{Y0.z, Y0.w}, wedge::mul2(f2{e0, e4}, f2{Y0.x, Y0.y})));
  const float R0s = fmaf(-e3, Y1.z, g.x);
  const bool ein = R0s >= 0.f;
  const float R0 = fabsf(R0s);
  const f2 ab = wedge::fma2(f2{e7, e8}, f2{Y1.z, Y1.w}, wedge::sp(-g.y));
  // the edge's pieces as wedge::split_edge_flat cuts them, written with
  // min/max instructions for the clamps and one predicate per piece (the
  // same bounds: no value is NaN, and a +-0 bound gives the same integrals)
  const float aa = ab.x, bb = ab.y;
  const float c2 = fmaf(r0, r0, R0 * R0);
  const bool far = c2 >= 4.f, lt1 = c2 < 1.f;
  float s1, s2;
  {
    // the breakpoints sqrt(4 - c^2), sqrt(1 - c^2): reciprocal square root
    // and one Newton step y (3/2 - r y/2), both in two-lane arithmetic
    const f2 xs = f2{4.f - c2, 1.f - c2};
    const f2 r = f2{rsqrtf(xs.x), rsqrtf(xs.y)};
    const f2 y = wedge::mul2(xs, r);
    const f2 q = wedge::mul2(y, wedge::fma2(wedge::mul2(wedge::sp(-0.5f), r), y, wedge::sp(1.5f)));
    s2 = far ? 0.f : q.x;
    s1 = lt1 ? q.y : 0.f;
  }
  const float x0 = fmaxf(aa, -s2), x1 = fminf(bb, s2);
  const float len = x1 - x0;
  const bool whole = !lt1 && len * len <= c2;
  const float l0 = fmaxf(x0, -s1), h0 = fminf(x1, s1);
  const float h1 = whole ? x1 : fminf(x1, -s1);
  const float l2 = fmaxf(x0, s1);
  const float h3 = far ? bb : fminf(bb, -s2);
  const float l4 = fmaxf(aa, s2);
  const bool v0 = on && h0 > l0, v1 = on && h1 > x0, v2 = on && !whole && x1 > l2;
  const bool v3 = h3 > aa, v4 = !far && bb > l4;
  const bool pos = fin == ein;
  if (COUNT && on) {
    wc.edges++;
    if (v0 || v1 || v2 || v3 || v4) wc.terms++;
    n_split += v1 && v2 && !lt1;
    n_out += (unsigned)v3 + (unsigned)v4;
  }
  // inner pieces (0 or 1 per record): one ballot; middle pieces: two
  const unsigned lt = (1u << lane) - 1u;
  const unsigned bin = __ballot_sync(FULL, v0), bm1 = __ballot_sync(FULL, v1), bm2 = __ballot_sync(FULL, v2);
  const int t0 = __popc(bin), t1 = __popc(bm1) + __popc(bm2);
  const int o0 = cnt0 + __popc(bin & lt);
  const int o1 = cnt1 + __popc(bm1 & lt) + __popc(bm2 & lt);
  // pieces go unfolded; their sign s_f s_e rides in the owner's bit 7
  const unsigned char ow = (unsigned char)(o | (pos ? 0 : 0x80));
  if (v0) { S.e[0][o0] = float4{r0, R0, l0, h0}; S.own[0][o0] = ow; }
  if (v1) { S.e[1][o1] = float4{r0, R0, x0, h1}; S.own[1][o1] = ow; }
  if (v2) { const int q = o1 + (int)v1; S.e[1][q] = float4{r0, R0, l2, x1}; S.own[1][q] = ow; }
  // beyond the support: -c0 (dPhi_left + dPhi_right) as the argument of the
  // product of the two intervals' numbers (R0^2 + lo hi) + i (hi - lo) R0
  {
    const float R02 = R0 * R0;
    const float ar = v3 ? fmaf(aa, h3, R02) : 1.f, ai = v3 ? (h3 - aa) * R0 : 0.f;
    const float br = v4 ? fmaf(l4, bb, R02) : 1.f, bi = v4 ? (bb - l4) * R0 : 0.f;
    const f2 z = wedge::fma2(f2{-ai, ai}, f2{bi, br}, wedge::mul2(wedge::sp(ar), f2{br, bi}));
    S.col[o][lane] += on ? (pos ? -c0f : c0f) * wedge::xatan2(z.y, z.x) : 0.f;
  }
  cnt0 += t0;
  cnt1 += t1;
  __syncwarp();
  if (cnt0 >= 32 || cnt1 >= 32) {
    int cnt2 = 0;
    unsigned n_st = 0;
    drain<float, true>(S, cnt0, cnt1, cnt2, false, n_in, n_mid, n_st);
  }
}

template <int NW, int MINB, bool COUNT>
__global__ void __launch_bounds__(NW * 32, MINB) pair_integrals_mixed(BatchArgs B) {
  __shared__ MixWarp mw[NW];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  MixWarp& M = mw[threadIdx.x >> 5];
  WarpStacks<float>& S = M.st;
  const SnapDesc& A = S.d;
  wedge::WorkCount wc;
  unsigned n_in = 0, n_mid = 0, n_split = 0, n_out = 0;
  int n64 = 0;
  int cur = -1;
  for (int r = 0; r < 32; ++r) S.col[r][lane] = 0.f;
  __syncwarp();

  const int64_t total = queue_total(B);
  for (;;) {
    int64_t g = 0;
    if (lane == 0) g = (int64_t)atomicAdd(&B.counters[3], 1ULL);
    g = __shfl_sync(FULL, g, 0);
    if (g >= total) break;
    int jl = 0, jh = B.nsnap - 1;
    while (jl < jh) {
      const int jm = (jl + jh + 1) >> 1;
      if (B.item_base[jm] <= g) jl = jm; else jh = jm - 1;
    }
    if (jl != cur) {
      __syncwarp();
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(B.snaps + jl);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&S.d);
      for (int i = lane; i < (int)(sizeof(SnapDesc) / 8); i += 32) dst[i] = src[i];
      __syncwarp();
      cur = jl;
    }
    const int64_t it = g - B.item_base[jl];
    const PairItem item = A.items[it];
    const int64_t c = item.cell;
    const float4* __restrict__ face = reinterpret_cast<const float4*>(A.face);
    const float4* __restrict__ fsph = A.fsph;
    const int64_t f0 = A.cfo[c];
    const int nf = (int)(A.cfo[c + 1] - f0);
    const int64_t l0 = A.fvo[f0];
    const float* __restrict__ ecell = reinterpret_cast<const float*>(A.edge) + l0 * EDGE_STRIDE;
    const double sx = A.site[3 * c], sy = A.site[3 * c + 1], sz = A.site[3 * c + 2];
    const bool staged = nf <= FSTAGE;
    if (staged) {
      __syncwarp();
      for (int i = lane; i < nf; i += 32) {
        M.fpl[i] = face[f0 + i];
        M.fsp[i] = fsph[f0 + i];
        M.fend[i] = (int)(A.fvo[f0 + i + 1] - l0);
      }
      __syncwarp();
    }
    double macc = 0.0;
    // the block loop compiled twice: shared-memory face records (STAGED)
    // or global ones, so that each reads its own memory space
    auto blocks = [&](auto stag) {
      constexpr bool STAGED = decltype(stag)::value;
      const int64_t pb = item.lo, pe = item.lo + item.cnt;
      for (int64_t p0 = pb; p0 < pe; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool active = p < pe;
        float yx = 0.f, yy = 0.f, yz = 0.f, hinv = 0.f;
        int32_t a = 0;
        if (active) {
          a = __ldg(A.pair_idx + p);
          pair_frame(A, a, sx, sy, sz, yx, yy, yz, hinv);
        }
        M.py[0][lane] = make_float4(yx, yx, yy, yy);
        M.py[1][lane] = make_float4(yz, yz, hinv, hinv);
        bool inside = true;
        int cntc = 0, cnt0 = 0, cnt1 = 0;  // stack heights (warp-uniform)
        __syncwarp();
        int kb = 0;
        for (int fi = 0; fi < nf; ++fi) {
          const float4 F = STAGED ? M.fpl[fi] : face[f0 + fi];
          const int ke = STAGED ? M.fend[fi] : (int)(A.fvo[f0 + fi + 1] - l0);
          const float r0s = face_r0s(F, yx, yy, yz, hinv);
          bool fin = r0s >= 0.f;
          float r0 = fabsf(r0s);
          bool inrange = active && r0 < 2.f;
          if (COUNT && active) wc.faces++;
          if (inrange && r0 < TAU) {
            // the plane passes within TAU h: its side and distance from the
            // FP64 plane and position, so that FP32 rounding cannot put the
            // particle on the wrong side; its edges then run as any other
            const double hh = 1.0 / A.h[a];
            const double* st = A.site + 3 * c;
            const double4_32a G = A.face64[f0 + fi];
            const double rs = G.w * hh - (G.x * ((A.x[a] - st[0]) * hh) + G.y * ((A.y[a] - st[1]) * hh) +
                                          G.z * ((A.z[a] - st[2]) * hh));
            fin = rs >= 0.0;
            r0 = (float)fabs(rs);
            if (COUNT) ++n64;
          }
          inside = inside && fin;
          if (inrange) {
            // the face's bounding sphere wholly beyond the support: nothing to add
            const float4 Q = STAGED ? M.fsp[fi] : fsph[f0 + fi];
            const float dx = yx - Q.x * hinv, dy = yy - Q.y * hinv, dz = yz - Q.z * hinv;
            const float rr = 2.f + Q.w * hinv;
            if (dx * dx + dy * dy + dz * dz >= rr * rr * 1.00001f) inrange = false;
          }
          const unsigned mn = __ballot_sync(FULL, inrange);
          if (mn) {
            const int nn = __popc(mn), rank = __popc(mn & lt);
            const float c0f = wedge::c0_of(r0);
            const unsigned tag = (unsigned)lane | (fin ? 32u : 0u);
            for (int k = kb; k < ke; ++k) {
              if (inrange)
                M.cmb[cntc + rank] = make_uint4(__float_as_uint(r0), __float_as_uint(c0f), (unsigned)k * EDGE_STRIDE, tag);
              cntc += nn;
              if (cntc >= 32) {
                cntc -= 32;
                edge_round<COUNT>(M, ecell, cntc, 32, cnt0, cnt1, n_in, n_mid, wc, n_split, n_out);
              }
            }
          }
          kb = ke;
        }
        // what is left: fewer than 32 records, then fewer than 32 pieces of each kind
        if (cntc) edge_round<COUNT>(M, ecell, 0, cntc, cnt0, cnt1, n_in, n_mid, wc, n_split, n_out);
        if (cnt0 || cnt1) {
          int cnt2 = 0;
          unsigned n_st = 0;
          drain<float, true>(S, cnt0, cnt1, cnt2, true, n_in, n_mid, n_st);
        }
        __syncwarp();
        float comp;
        const float rs = take_row(S.col, lane, comp);
        if (active) {
          const double f = (inside ? 1.0 : 0.0) + ((double)rs - (double)comp);
          if (A.frac) A.frac[p] = f;
          macc += A.m[a] * f;
        }
        __syncwarp();
      }
    };
    if (staged) blocks(std::true_type{}); else blocks(std::false_type{});
    for (int o = 16; o > 0; o >>= 1) macc += __shfl_down_sync(FULL, macc, o);
    if (lane == 0) A.partial[it] = macc;
    __syncwarp();
  }
  if (!COUNT) return;
  auto wsum = [](unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;
  };
  const unsigned long long terms = wsum((unsigned long long)wc.terms), faces = wsum((unsigned long long)wc.faces);
  const unsigned long long edges = wsum((unsigned long long)wc.edges), fp64 = wsum((unsigned long long)n64);
  const unsigned long long split = wsum((unsigned long long)n_split);
  const unsigned long long outs = wsum((unsigned long long)n_out);
  if (lane == 0) {
    atomicAdd(&B.counters[1], terms);
    atomicAdd(&B.counters[2], fp64);
    atomicAdd(&B.counters[8], faces);
    atomicAdd(&B.counters[9], edges);
    atomicAdd(&B.counters[10], 2ull * n_in);
    atomicAdd(&B.counters[11], (unsigned long long)n_mid - split);
    atomicAdd(&B.counters[12], outs);
    atomicAdd(&B.counters[13], split);
  }
}

// CTAs per SM of a launch of shape (NW, MINB): as many as are resident at
// once, at most MINB (a persistent launch beyond residency would only queue).
template <int NW, int MINB, bool COUNT = false>
int mixed_per_sm(int* per_sm, int* regs) {
  auto kern = pair_integrals_mixed<NW, MINB, COUNT>;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, NW * 32, 0));
  if (*per_sm > MINB) *per_sm = MINB;
  if (*per_sm < 1) *per_sm = 1;
  if (regs) {
    cudaFuncAttributes a;
    CUDA_TRY(cudaFuncGetAttributes(&a, kern));
    *regs = a.numRegs;
  }
  return MAP_OK;
}

template <int NW, int MINB, bool COUNT = false>
int launch_mixed(map_ctx* ctx, const BatchArgs& B, cudaStream_t s) {
  auto kern = pair_integrals_mixed<NW, MINB, COUNT>;
  int per_sm = 0;
  MAP_TRY((mixed_per_sm<NW, MINB, COUNT>(&per_sm, nullptr)));
  int64_t blocks = (int64_t)per_sm * ctx->sm_count;
  const int64_t need = (B.total + NW - 1) / NW;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<(unsigned)blocks, NW * 32, 0, s>>>(B); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

template <typename T, bool MIXED, int NW, int MINB, bool COUNT = false>
int launch(map_ctx* ctx, const BatchArgs& B, cudaStream_t s) {
  auto kern = pair_integrals<T, MIXED, NW, MINB, COUNT>;
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, 0));
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)per_sm * ctx->sm_count;
  const int64_t need = (B.total + NW - 1) / NW;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<(unsigned)blocks, NW * 32, 0, s>>>(B); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

// Descriptor upload through kernel parameters: the values are captured at
// launch, so the host copy may be reused at once and the launch can sit in a
// CUDA graph.
constexpr int DESC_CHUNK = 16;  // 16 x 192 bytes of parameters per launch
struct DescChunk {
  SnapDesc d[DESC_CHUNK];
  int n;
};
__global__ void put_descs(DescChunk c, SnapDesc* dst) {
  if ((int)threadIdx.x < c.n) dst[threadIdx.x] = c.d[threadIdx.x];
}
constexpr int I64_CHUNK = 480;
struct I64Chunk {
  int64_t v[I64_CHUNK];
  int n;
};
__global__ void put_i64(I64Chunk c, int64_t* dst) {
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) dst[i] = c.v[i];
}

// M_i = sum of cell i's item partials, in item order; rho_i = M_i / V_i.
// One thread per cell over the cells of all snapshots.
__global__ void cell_sums(const SnapDesc* __restrict__ d, const int64_t* __restrict__ cell_base, int nsnap,
                          int64_t total_cells, const int64_t* bad) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= total_cells || (bad && *bad)) return;
  int jl = 0, jh = nsnap - 1;
  while (jl < jh) {
    const int jm = (jl + jh + 1) >> 1;
    if (cell_base[jm] <= g) jl = jm; else jh = jm - 1;
  }
  const SnapDesc& D = d[jl];
  const int64_t c = g - cell_base[jl];
  double M = 0.0;
  for (int64_t i = D.item_off[c]; i < D.item_off[c + 1]; ++i) M += D.partial[i];
  D.cell_mass[c] = M;
  if (D.cell_rho) D.cell_rho[c] = M / D.vol[c];
}

// sum_i M_i of each snapshot (one block per snapshot, fixed order)
__global__ void sum_snapshots(const SnapDesc* __restrict__ d, double* totals) {
  typedef cub::BlockReduce<double, 256> BR;
  __shared__ typename BR::TempStorage tmp;
  const SnapDesc& D = d[blockIdx.x];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < D.ncell; i += 256) acc += D.cell_mass[i];
  const double t = BR(tmp).Sum(acc);
  if (threadIdx.x == 0) totals[D.orig] = t;
}

}  // namespace

int integrals_upload(map_ctx* ctx, const SnapDesc* h_desc, const int64_t* h_ibase, const int64_t* h_cbase,
                     int nsnap, SnapDesc* d_desc, int64_t* d_ibase, int64_t* d_cbase, cudaStream_t s) {
  for (int j0 = 0; j0 < nsnap; j0 += DESC_CHUNK) {
    DescChunk c;
    c.n = nsnap - j0 < DESC_CHUNK ? nsnap - j0 : DESC_CHUNK;
    for (int i = 0; i < c.n; ++i) c.d[i] = h_desc[j0 + i];
    put_descs<<<1, DESC_CHUNK, 0, s>>>(c, d_desc + j0); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  }
  for (int k = 0; k < 2; ++k) {
    const int64_t* h = k == 0 ? h_ibase : h_cbase;
    int64_t* dd = k == 0 ? d_ibase : d_cbase;
    for (int j0 = 0; j0 <= nsnap; j0 += I64_CHUNK) {
      I64Chunk c;
      c.n = nsnap + 1 - j0 < I64_CHUNK ? nsnap + 1 - j0 : I64_CHUNK;
      for (int i = 0; i < c.n; ++i) c.v[i] = h[j0 + i];
      put_i64<<<1, 128, 0, s>>>(c, dd + j0); ++ctx->launches;
      CUDA_TRY(cudaGetLastError());
    }
  }
  return MAP_OK;
}

int integrals_enqueue(map_ctx* ctx, const BatchArgs& B, int variant, cudaStream_t s) {
  CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), s));
  CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 8, 0, 8 * sizeof(unsigned long long), s));
  const bool count = ctx->cfg.count_work != 0;
  if (ctx->cfg.precision == MAP_TABLE) {
    MAP_TRY(launch_table(ctx, B, s));
  } else if (ctx->cfg.precision == MAP_MIXED && count) {
    MAP_TRY((launch_mixed<4, 5, true>(ctx, B, s)));
  } else if (ctx->cfg.precision == MAP_MIXED) {
    switch (variant) {
      case 1: MAP_TRY((launch_mixed<4, 4>(ctx, B, s))); break;
      case 2: MAP_TRY((launch_mixed<2, 9>(ctx, B, s))); break;
      case 3: MAP_TRY((launch_mixed<8, 2>(ctx, B, s))); break;
      default: MAP_TRY((launch_mixed<4, 5>(ctx, B, s))); break;
    }
  } else if (count) {
    MAP_TRY((launch<double, false, 4, 4, true>(ctx, B, s)));
  } else {
    MAP_TRY((launch<double, false, 4, 4>(ctx, B, s)));
  }
  if (B.total_cells > 0) {
    cell_sums<<<nblk(B.total_cells, 256), 256, 0, s>>>(B.snaps, B.cell_base, B.nsnap, B.total_cells, B.bad);
    ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  }
  return MAP_OK;
}

int integrals_shape(map_ctx* ctx, int v, int* warps, int* ctas, int* regs) {
  CUDA_TRY(cudaSetDevice(ctx->device));
  switch (v) {
    case 0: *warps = 4; return mixed_per_sm<4, 5>(ctas, regs);
    case 1: *warps = 4; return mixed_per_sm<4, 4>(ctas, regs);
    case 2: *warps = 2; return mixed_per_sm<2, 9>(ctas, regs);
    case 3: *warps = 8; return mixed_per_sm<8, 2>(ctas, regs);
    default: return MAP_EINVAL;
  }
}

int integrals_sum(map_ctx* ctx, const SnapDesc* d_desc, int nsnap, double* totals, cudaStream_t s) {
  sum_snapshots<<<nsnap, 256, 0, s>>>(d_desc, totals); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

SnapDesc make_desc(map_ctx* ctx, const PreparedGrid* g, const map_particles* p, const map_outputs* out,
                   const int64_t* pair_off, const int32_t* pair_idx, double* frac, int orig) {
  SnapDesc d;
  d.ncell = g->ncell;
  d.cfo = g->cell_face_off;
  d.fvo = g->face_vert_off;
  d.site = g->site;
  d.vol = g->vol;
  d.pair_off = pair_off;
  d.pair_idx = pair_idx;
  d.x = p->x; d.y = p->y; d.z = p->z; d.m = p->m; d.h = p->h;
  d.frac = frac;
  d.cell_mass = out->cell_mass;
  d.cell_rho = out->cell_rho;
  const bool mixed = ctx->cfg.precision != MAP_FP64;  // the table variant reads the FP32 records too
  d.face = mixed ? (const void*)g->face32 : (const void*)g->face64;
  d.edge = mixed ? (const void*)g->edge32 : (const void*)g->edge64;
  d.face64 = g->face64;
  d.edge64 = g->edge64;
  d.fsph = g->fsph32;
  d.face_vert = g->face_vert;
  d.vx = g->vx;
  d.vy = g->vy;
  d.vz = g->vz;
  d.items = ctx->items;
  d.item_off = ctx->item_off;
  d.partial = ctx->partial;
  d.nitems = ctx->n_items;
  d.orig = orig;
  return d;
}

int integrals_run(map_ctx* ctx, const PreparedGrid* g, const map_particles* p, map_outputs* out, cudaStream_t s) {
  double* frac;
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[0], ctx->n_pairs + 1, &frac));
  ctx->pair_frac = frac;
  ctx->inv_ready = false;
  SnapDesc* d_desc;
  int64_t* d_base;
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[3], 1, &d_desc));
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[4], 4, &d_base));
  auto upload = [&](BatchArgs& Bo) -> int {
    const SnapDesc h = make_desc(ctx, g, p, out, ctx->pair_off, ctx->pair_idx, frac, 0);
    const int64_t ibase[2] = {0, ctx->n_items}, cbase[2] = {0, g->ncell};
    MAP_TRY(integrals_upload(ctx, &h, ibase, cbase, 1, d_desc, d_base, d_base + 2, s));
    Bo = BatchArgs{d_desc, d_base, d_base + 2, 1, ctx->n_items, g->ncell, ctx->d_counters};
    return MAP_OK;
  };
  BatchArgs B;
  MAP_TRY(upload(B));
  if (ctx->cfg.autotune && ctx->cfg.precision == MAP_MIXED && !ctx->tune_done[MAP_MIXED]) {
    auto rebuild = [&](int target, BatchArgs& Bo) -> int {
      MAP_TRY(items_build(ctx, ctx->pair_off, g->ncell, ctx->n_pairs, target, s));
      return upload(Bo);
    };
    MAP_TRY(integrals_autotune(ctx, rebuild, B, s));
  }
  phase_begin(ctx, 2, s);
  MAP_TRY(integrals_enqueue(ctx, B, ctx->tuned[ctx->cfg.precision == MAP_MIXED ? MAP_MIXED : MAP_FP64], s));
  phase_end(ctx, 2, s);
  if (out->cell_vol) CUDA_TRY(cudaMemcpyAsync(out->cell_vol, g->vol, g->ncell * sizeof(double), cudaMemcpyDeviceToDevice, s));
  MAP_TRY(integrals_sum(ctx, d_desc, 1, ctx->d_total, s));
  return MAP_OK;
}
