// Pair integrals and cell sums (Section II-B, Eq. 1-3).
//
// Persistent kernel: each CTA pulls cells from a device work queue and stages
// the cell's site-relative face planes and edge records in shared memory.
// Each warp then takes the cell's pairs 32 at a time, one pair per lane,
// independently of the other warps, in three phases per chunk of ECH
// directed edges:
//
//  phase 1 (per thread = pair): for each edge of the chunk compute r0 (face),
//    R0 and the along-edge coordinates of the vertices, update the inside
//    flag, and QUEUE each piece of the edge integral K'_e -- at most one
//    inner piece, two middle pieces and two pieces beyond the support -- as
//    (r0, R0, lo, hi); the sign s_f s_e is folded into the interval direction.
//    (Mixed build: a face whose plane passes within 1e-4 h of the particle is
//    decided and evaluated in FP64 in this thread instead.)
//  phase 2 (whole warp): evaluate the queued pieces kind by kind, every lane
//    running the same code, each result written to its piece's slot;
//  phase 3 (per lane): sum the lane's own piece results in a fixed order
//    (compensated), so that every result is bit-reproducible.
// Only __syncwarp separates the phases; CTA barriers fall at cell boundaries.
//
// Without the queue, lanes (different particles) branch into different
// pieces and a warp runs every path with a few lanes active (measured 5.3 of
// 32).  Per pair: f_ai = [inside] + sum_f sum_e s_f s_e K'_e (see wedge.cuh).  M_i = sum_a m_a f_ai is accumulated in
// FP64 and reduced across the CTA; rho_i = M_i / V_i.
#include <cub/cub.cuh>

#include "internal.cuh"
#include "wedge.cuh"

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4_32a type; };
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

struct IntegralArgs {
  int64_t ncell;
  const int64_t* cfo;
  const int64_t* fvo;
  const double* site;
  const double* vol;
  const int64_t* pair_off;
  const int32_t* pair_idx;
  const double *x, *y, *z, *m, *h;
  double* frac;
  double* cell_mass;
  double* cell_rho;
  unsigned long long* counters;  // [1] edge terms, [2] FP64 terms, [3] work queue, [8..11] work tally
  const double4_32a* face64;     // FP64 geometry for the near-degenerate fallback of the mixed build
  const double* edge64;
};

// Mixed build: a face whose plane, or an edge whose line, passes within TAU
// (in units of h) of the particle (resp. its projection) is evaluated in FP64:
// FP32 rounding (~1e-7 h) could otherwise give inconsistent signs to a plane
// seen from two faces.  Exact zeros (particle exactly on a plane or edge line)
// are moved to +EPS on the inner side in both builds: the integral is
// continuous in the particle position, and treating every exact zero as
// 'inside' is one consistent displacement of the particle into the cell.
constexpr float TAU = 1e-4f;
constexpr double EPS = 1e-12;

// Exclusive warp prefix sum of v; returns the warp total in *tot.
__device__ __forceinline__ int warp_excl(int v, int* tot) {
  const int lane = threadIdx.x & 31;
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += t;
  }
  *tot = __shfl_sync(0xffffffffu, s, 31);
  return s - v;
}

// Per-warp work area in shared memory for one chunk of ECH edges: every lane
// owns fixed slots -- (r0, R0) per edge, (lo, hi) and a result per piece (5
// pieces per edge: 1 inner, 2 middle, 2 beyond the support) -- and three
// compact lists name the occupied slots of each kind.
template <typename T, int ECH>
struct WarpArea {
  typename Vec2<T>::type rr[ECH][32];     // (r0, R0) per (edge, lane)
  typename Vec2<T>::type lh[ECH * 5][32]; // (lo, hi) per (piece slot, lane)
  T res[ECH * 5][32];                     // piece results
  unsigned short q[3][ECH * 64];          // occupied slots: inner, middle, beyond
};

template <typename T, bool MIXED, int NT, int ECH>
__global__ void __launch_bounds__(NT, 4) pair_integrals(IntegralArgs A, const typename Vec4<T>::type* __restrict__ face,
                                                     const T* __restrict__ edge, int smem_faces, int smem_loops) {
  typedef typename Vec4<T>::type V4;
  typedef typename Vec2<T>::type V2;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  WarpArea<T, ECH>* areas = reinterpret_cast<WarpArea<T, ECH>*>(smem);
  unsigned char* geo = smem + sizeof(WarpArea<T, ECH>) * NW;
  geo = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(geo) + 127) & ~uintptr_t(127));
  V4* s_face = reinterpret_cast<V4*>(geo);
  T* s_edge = reinterpret_cast<T*>(geo + sizeof(V4) * smem_faces);
  int* s_floop = reinterpret_cast<int*>(geo + sizeof(V4) * smem_faces + sizeof(T) * EDGE_STRIDE * smem_loops);
  unsigned short* s_fidx = reinterpret_cast<unsigned short*>(s_floop + smem_faces + 1);

  __shared__ int64_t s_cell;
  __shared__ unsigned long long s_work[8];
  typedef cub::BlockReduce<double, NT> BR;
  __shared__ typename BR::TempStorage s_br;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  WarpArea<T, ECH>& W = areas[warp];
  if (tid < 8) s_work[tid] = 0;
  wedge::WorkCount wc, wcd;
  int n64 = 0;
  unsigned long long n_in_tot = 0, n_mid_tot = 0, n_out_tot = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_cell = (int64_t)atomicAdd(&A.counters[3], 1ULL);
    __syncthreads();
    const int64_t c = s_cell;
    if (c >= A.ncell) break;
    const int64_t f0 = A.cfo[c];
    const int nf = (int)(A.cfo[c + 1] - f0);
    const int64_t l0 = A.fvo[f0];
    const int nl = (int)(A.fvo[f0 + nf] - l0);
    if (!(nf <= smem_faces && nl <= smem_loops)) continue;  // mapped by pair_integrals_large
    for (int i = tid; i <= nf; i += NT) s_floop[i] = (int)(A.fvo[f0 + i] - l0);
    for (int i = tid; i < nf; i += NT) s_face[i] = face[f0 + i];
    {
      const int ne = nl * EDGE_STRIDE;
      const T* src = edge + l0 * EDGE_STRIDE;
      for (int i = tid; i < ne; i += NT) s_edge[i] = src[i];
    }
    __syncthreads();
    for (int fi = tid; fi < nf; fi += NT)
      for (int k = s_floop[fi]; k < s_floop[fi + 1]; ++k) s_fidx[k] = (unsigned short)fi;
    __syncthreads();

    const double sx = A.site[3 * c], sy = A.site[3 * c + 1], sz = A.site[3 * c + 2];
    double macc = 0.0;
    const int64_t pb = A.pair_off[c], pe = A.pair_off[c + 1];
    // each warp takes 32 pairs at a time; warps proceed independently
    for (int64_t p0 = pb + warp * 32; p0 < pe; p0 += NT) {
      const int64_t p = p0 + lane;
      const bool active = p < pe;
      T yx = T(0), yy = T(0), yz = T(0), hinv = T(0);
      int32_t a = 0;
      if (active) {
        a = A.pair_idx[p];
        const double hh = A.h[a];
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
      bool inside = true;
      double dacc = 0.0;
      T fsum = T(0), fcomp = T(0);  // compensated sum of this pair's pieces
      int cur = -1;
      T r0 = T(0);
      bool fin = true, inrange = false;
      for (int kc = 0; kc < nl; kc += ECH) {
        // ---------------- phase 1: geometry, fixed slots, compact lists
        const int kend = min(kc + ECH, nl);
        unsigned long long mask = 0;  // 5 bits per edge of the chunk
        int cnt_in = 0, cnt_mid = 0, cnt_out = 0;
        for (int k = kc; k < kend; ++k) {
          const int kl = k - kc;
          const int fi = s_fidx[k];
          if (fi != cur) {
            const V4 F = s_face[fi];
            const T r0s = F.w * hinv - (F.x * yx + F.y * yy + F.z * yz);
            fin = r0s >= T(0);
            r0 = fabs(r0s);
            if (!MIXED) r0 = r0 > T(1e-12) ? r0 : T(1e-12);
            inrange = active && r0 < T(2);
            cur = fi;
            if (active) wc.faces++;
            if (MIXED && inrange && r0 < T(1e-4)) {
              // the face plane passes within 1e-4 h of the particle: decide
              // the side and evaluate the whole face in FP64 in this thread
              const double hh = 1.0 / A.h[a];
              const double ydx = (A.x[a] - sx) * hh, ydy = (A.y[a] - sy) * hh, ydz = (A.z[a] - sz) * hh;
              const double4_32a G = A.face64[f0 + fi];
              const double rs = G.w * hh - (G.x * ydx + G.y * ydy + G.z * ydz);
              fin = rs >= 0.0;
              const double r0d = fabs(rs) > 1e-12 ? fabs(rs) : 1e-12;
              for (int kk = s_floop[fi]; kk < s_floop[fi + 1]; ++kk) {
                const double* D = A.edge64 + (l0 + kk) * EDGE_STRIDE;
                const double R0sd = (D[0] * ydx + D[1] * ydy + D[2] * ydz) - D[3] * hh;
                const double based = D[4] * ydx + D[5] * ydy + D[6] * ydz;
                const bool eind = R0sd >= 0.0;
                const double R0d = fabs(R0sd) > 1e-12 ? fabs(R0sd) : 1e-12;
                const double K = wedge::kprime_edge<double, false>(r0d, R0d, D[7] * hh - based, D[8] * hh - based, wcd);
                dacc += (fin == eind) ? K : -K;
                ++n64;
              }
              inrange = false;  // its edges are done
            }
            inside = inside && fin;
          }
          int nin = 0, nmid = 0, nout = 0;
          if (inrange) {
            const T* E = s_edge + k * EDGE_STRIDE;
            const T R0s = (E[0] * yx + E[1] * yy + E[2] * yz) - E[3] * hinv;  // m.(p - v_a): > 0 inside
            const T base = E[4] * yx + E[5] * yy + E[6] * yz;
            const bool ein = R0s >= T(0);
            T R0 = fabs(R0s);
            if (!MIXED) R0 = R0 > T(1e-12) ? R0 : T(1e-12);
            wc.edges++;
            V2 rr;
            rr.x = r0;
            rr.y = R0;
            W.rr[kl][lane] = rr;
            // slots: 0 inner, 1-2 middle, 3-4 beyond the support
            wedge::split_edge<T>(
                r0, R0, E[7] * hinv - base, E[8] * hinv - base, fin == ein,
                [&](T l, T h) { V2 v; v.x = l; v.y = h; W.lh[kl * 5 + 0][lane] = v; nin = 1; },
                [&](T l, T h) { V2 v; v.x = l; v.y = h; W.lh[kl * 5 + 1 + nmid][lane] = v; ++nmid; },
                [&](T l, T h) { V2 v; v.x = l; v.y = h; W.lh[kl * 5 + 3 + nout][lane] = v; ++nout; });
            mask |= (unsigned long long)((nin) | (((1 << nmid) - 1) << 1) | (((1 << nout) - 1) << 3)) << (5 * kl);
            if (nin + nmid + nout) wc.terms++;
          }
          // warp-aggregated append of this edge's slot ids to the compact lists
          int tin, tmid, tout;
          const int oin = warp_excl(nin, &tin);
          const int omid = warp_excl(nmid, &tmid);
          const int oout = warp_excl(nout, &tout);
          if (nin) W.q[0][cnt_in + oin] = (unsigned short)((kl * 5 + 0) * 32 + lane);
          for (int j = 0; j < nmid; ++j) W.q[1][cnt_mid + omid + j] = (unsigned short)((kl * 5 + 1 + j) * 32 + lane);
          for (int j = 0; j < nout; ++j) W.q[2][cnt_out + oout + j] = (unsigned short)((kl * 5 + 3 + j) * 32 + lane);
          cnt_in += tin;
          cnt_mid += tmid;
          cnt_out += tout;
        }
        __syncwarp();
        // ---------------- phase 2: uniform evaluation, kind by kind
        for (int i = lane; i < cnt_in; i += 32) {
          const int sl = W.q[0][i], ow = sl & 31, ps = sl >> 5;
          const V2 rr = W.rr[ps / 5][ow], lh = W.lh[ps][ow];
          W.res[ps][ow] = wedge::piece_inner<T>(rr.x, rr.y, lh.x, lh.y);
        }
        for (int i = lane; i < cnt_mid; i += 32) {
          const int sl = W.q[1][i], ow = sl & 31, ps = sl >> 5;
          const V2 rr = W.rr[ps / 5][ow], lh = W.lh[ps][ow];
          W.res[ps][ow] = wedge::piece_mid<T, MIXED>(rr.x, rr.y, lh.x, lh.y);
        }
        for (int i = lane; i < cnt_out; i += 32) {
          const int sl = W.q[2][i], ow = sl & 31, ps = sl >> 5;
          const V2 rr = W.rr[ps / 5][ow], lh = W.lh[ps][ow];
          W.res[ps][ow] = wedge::piece_outer<T>(rr.x, rr.y, lh.x, lh.y);
        }
        n_in_tot += cnt_in;
        n_mid_tot += cnt_mid;
        n_out_tot += cnt_out;
        __syncwarp();
        // ---------------- phase 3: each lane sums its own pieces in a fixed order
        while (mask) {
          const int b = __ffsll((long long)mask) - 1;
          mask &= mask - 1;
          const T v = W.res[b][lane] - fcomp;
          const T t = fsum + v;
          fcomp = (t - fsum) - v;
          fsum = t;
        }
        __syncwarp();
      }
      if (active) {
        const double f = (inside ? 1.0 : 0.0) + dacc + (double)fsum;
        if (A.frac) A.frac[p] = f;
        macc += A.m[a] * f;
      }
    }
    const double M = BR(s_br).Sum(macc);
    if (tid == 0) {
      A.cell_mass[c] = M;
      if (A.cell_rho) A.cell_rho[c] = M / A.vol[c];
    }
  }
  if (lane == 0) {
    atomicAdd(&s_work[3], 2 * n_in_tot);
    atomicAdd(&s_work[4], n_mid_tot);
    atomicAdd(&s_work[6], n_out_tot);
  }
  atomicAdd(&s_work[0], (unsigned long long)wc.terms);
  atomicAdd(&s_work[1], (unsigned long long)wc.faces);
  atomicAdd(&s_work[2], (unsigned long long)wc.edges);
  atomicAdd(&s_work[5], (unsigned long long)n64);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&A.counters[1], s_work[0]);
    atomicAdd(&A.counters[2], s_work[5]);
    atomicAdd(&A.counters[8], s_work[1]);
    atomicAdd(&A.counters[9], s_work[2]);
    atomicAdd(&A.counters[10], s_work[3]);
    atomicAdd(&A.counters[11], s_work[4]);
    atomicAdd(&A.counters[12], s_work[6]);
  }
}

// Cells too large for the staging area (none in practice for Voronoi cells;
// kept so that any valid grid is mapped): one CTA per such cell, one thread
// per pair, geometry read from global memory, every edge evaluated in place.
template <typename T, bool MIXED>
__global__ void pair_integrals_large(IntegralArgs A, const typename Vec4<T>::type* __restrict__ face,
                                     const T* __restrict__ edge, int smem_faces, int smem_loops) {
  typedef typename Vec4<T>::type V4;
  typedef cub::BlockReduce<double, 128> BR;
  __shared__ typename BR::TempStorage s_br;
  const int64_t c = blockIdx.x;
  const int64_t f0 = A.cfo[c];
  const int nf = (int)(A.cfo[c + 1] - f0);
  const int64_t l0 = A.fvo[f0];
  const int nl = (int)(A.fvo[f0 + nf] - l0);
  if (nf <= smem_faces && nl <= smem_loops) return;
  const double sx = A.site[3 * c], sy = A.site[3 * c + 1], sz = A.site[3 * c + 2];
  double macc = 0.0;
  wedge::WorkCount wc;
  for (int64_t p = A.pair_off[c] + threadIdx.x; p < A.pair_off[c + 1]; p += 128) {
    const int32_t a = A.pair_idx[p];
    const double hh = 1.0 / A.h[a];
    const double ydx = (A.x[a] - sx) * hh, ydy = (A.y[a] - sy) * hh, ydz = (A.z[a] - sz) * hh;
    double tot = 0.0;
    bool inside = true;
    // always FP64 here: large cells are rare and this path has no queue
    for (int fi = 0; fi < nf; ++fi) {
      const double4_32a G = A.face64[f0 + fi];
      const double rs = G.w * hh - (G.x * ydx + G.y * ydy + G.z * ydz);
      const bool fin = rs >= 0.0;
      inside = inside && fin;
      const double r0 = fabs(rs) > 1e-12 ? fabs(rs) : 1e-12;
      if (r0 >= 2.0) continue;
      for (int64_t k = A.fvo[f0 + fi] - l0; k < A.fvo[f0 + fi + 1] - l0; ++k) {
        const double* D = A.edge64 + (l0 + k) * EDGE_STRIDE;
        const double R0s = (D[0] * ydx + D[1] * ydy + D[2] * ydz) - D[3] * hh;
        const double base = D[4] * ydx + D[5] * ydy + D[6] * ydz;
        const bool ein = R0s >= 0.0;
        const double R0 = fabs(R0s) > 1e-12 ? fabs(R0s) : 1e-12;
        const double K = wedge::kprime_edge<double, false>(r0, R0, D[7] * hh - base, D[8] * hh - base, wc);
        tot += (fin == ein) ? K : -K;
      }
    }
    const double f = (inside ? 1.0 : 0.0) + tot;
    if (A.frac) A.frac[p] = f;
    macc += A.m[a] * f;
  }
  const double M = BR(s_br).Sum(macc);
  if (threadIdx.x == 0) {
    A.cell_mass[c] = M;
    if (A.cell_rho) A.cell_rho[c] = M / A.vol[c];
  }
}

constexpr size_t SMEM_CAP = 200 * 1024;

template <typename T, bool MIXED, int NT, int ECH>
int launch(map_ctx* ctx, const PreparedGrid* g, const IntegralArgs& A, cudaStream_t s) {
  typedef typename Vec4<T>::type V4;
  const size_t queue = sizeof(WarpArea<T, ECH>) * (NT / 32) + 128;
  int sf = g->max_faces, sl = g->max_loops;
  auto geo_bytes = [](int f, int l) {
    return sizeof(V4) * f + sizeof(T) * EDGE_STRIDE * l + sizeof(int) * (f + 1) + sizeof(unsigned short) * l + 16;
  };
  size_t bytes = queue + geo_bytes(sf, sl);
  if (bytes > SMEM_CAP) {
    sf = sf < 128 ? sf : 128;
    sl = (int)((SMEM_CAP - queue - sizeof(V4) * sf - sizeof(int) * (sf + 1) - 16) /
               (sizeof(T) * EDGE_STRIDE + sizeof(unsigned short)));
    bytes = queue + geo_bytes(sf, sl);
  }
  auto kern = pair_integrals<T, MIXED, NT, ECH>;
  CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, bytes));
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)per_sm * ctx->sm_count;
  if (blocks > g->ncell) blocks = g->ncell > 0 ? g->ncell : 1;
  const V4* fp = reinterpret_cast<const V4*>(MIXED ? (const void*)g->face32 : (const void*)g->face64);
  const T* ep = reinterpret_cast<const T*>(MIXED ? (const void*)g->edge32 : (const void*)g->edge64);
  kern<<<(unsigned)blocks, NT, bytes, s>>>(A, fp, ep, sf, sl); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  if (sf < g->max_faces || sl < g->max_loops) {
    pair_integrals_large<T, MIXED><<<(unsigned)g->ncell, 128, 0, s>>>(A, fp, ep, sf, sl); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  }
  return MAP_OK;
}

__global__ void sum_cells(int64_t n, const double* __restrict__ v, double* out) {
  typedef cub::BlockReduce<double, 256> BR;
  __shared__ typename BR::TempStorage tmp;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) acc += v[i];
  double t = BR(tmp).Sum(acc);
  if (threadIdx.x == 0) *out = t;
}

}  // namespace

int integrals_run(map_ctx* ctx, const PreparedGrid* g, const map_particles* p, map_outputs* out, cudaStream_t s) {
  double* frac;
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[0], ctx->n_pairs + 1, &frac));
  ctx->pair_frac = frac;
  CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), s));
  CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 8, 0, 8 * sizeof(unsigned long long), s));
  IntegralArgs A;
  A.ncell = g->ncell;
  A.cfo = g->cell_face_off;
  A.fvo = g->face_vert_off;
  A.site = g->site;
  A.vol = g->vol;
  A.pair_off = ctx->pair_off;
  A.pair_idx = ctx->pair_idx;
  A.x = p->x; A.y = p->y; A.z = p->z; A.m = p->m; A.h = p->h;
  A.frac = frac;
  A.cell_mass = out->cell_mass;
  A.cell_rho = out->cell_rho;
  A.counters = ctx->d_counters;
  A.face64 = g->face64;
  A.edge64 = g->edge64;
  phase_begin(ctx, 2, s);
  if (ctx->cfg.precision == MAP_MIXED)
    MAP_TRY((launch<float, true, 128, 4>(ctx, g, A, s)));
  else
    MAP_TRY((launch<double, false, 128, 2>(ctx, g, A, s)));
  phase_end(ctx, 2, s);
  if (out->cell_vol) CUDA_TRY(cudaMemcpyAsync(out->cell_vol, g->vol, g->ncell * sizeof(double), cudaMemcpyDeviceToDevice, s));
  sum_cells<<<1, 256, 0, s>>>(g->ncell, out->cell_mass, ctx->d_total); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
