// Pair integrals and cell sums (Section II-B, Eq. 1-3).
//
// Persistent kernel: each CTA pulls cells from a device work queue, stages the
// cell's site-relative face planes and edge records in shared memory, and
// gives every thread one particle of the cell's pair list.  All threads of a
// CTA walk the same faces and edges in lockstep (broadcast shared-memory
// reads), so loop trip counts never diverge; only the per-edge pieces do.
// Per pair: f_ai = [inside] - sum_f s_f (2 pi r0 E(r0) [p in face] - sum_e s_e K_e)
// (see wedge.cuh).  M_i = sum_a m_a f_ai is accumulated in FP64 and reduced
// across the CTA; rho_i = M_i / V_i.
#include <cub/cub.cuh>

#include "internal.cuh"
#include "wedge.cuh"

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4_32a type; };

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
  unsigned long long* counters;  // [1] edge terms, [3] work queue
};

// Loop-entry offsets of a cell's faces, from shared memory or global memory.
struct SmemLoops {
  const int* p;
  __device__ __forceinline__ int operator[](int i) const { return p[i]; }
};
struct GlobalLoops {
  const int64_t* fvo;  // face_vert_off + first face of the cell
  int64_t l0;
  __device__ __forceinline__ int operator[](int i) const { return (int)(fvo[i] - l0); }
};

// f_ai for one particle (coordinates relative to the site, in units of h).
template <typename T, bool MIXED, typename Loops>
__device__ __forceinline__ T pair_fraction(const typename Vec4<T>::type* __restrict__ faces, Loops floop,
                                           const T* __restrict__ edges, int nf, T yx, T yy, T yz, T hinv,
                                           wedge::WorkCount& wc) {
  T tot = T(0);
  bool inside = true;
  wc.faces += nf;
  for (int fi = 0; fi < nf; ++fi) {
    const typename Vec4<T>::type F = faces[fi];
    const T r0s = F.w * hinv - (F.x * yx + F.y * yy + F.z * yz);
    const bool fin = r0s >= T(0);
    inside = inside && fin;
    const T r0 = fabs(r0s);
    if (r0 >= T(2)) continue;
    bool pin = true;
    T jsum = T(0);
    const int k1 = floop[fi + 1];
    wc.edges += k1 - floop[fi];
    for (int k = floop[fi]; k < k1; ++k) {
      const T* E = edges + k * EDGE_STRIDE;
      const T R0s = (E[0] * yx + E[1] * yy + E[2] * yz) - E[3] * hinv;  // m.(p - v_a): > 0 inside
      const T base = E[4] * yx + E[5] * yy + E[6] * yz;
      const bool ein = R0s >= T(0);
      pin = pin && ein;
      const T R0 = fabs(R0s);
      if (r0 * r0 + R0 * R0 < T(4)) {
        const T K = wedge::edge_integral<T, MIXED>(r0, R0, E[7] * hinv - base, E[8] * hinv - base, wc);
        jsum += ein ? K : -K;
        ++wc.terms;
      }
    }
    const T cf = (pin ? wedge::face_term<T>(r0) : T(0)) - jsum;
    tot += fin ? cf : -cf;
  }
  return (inside ? T(1) : T(0)) - tot;
}

template <typename T, bool MIXED, int NT>
__global__ void __launch_bounds__(NT) pair_integrals(IntegralArgs A, const typename Vec4<T>::type* __restrict__ face,
                                                     const T* __restrict__ edge, int smem_faces, int smem_loops) {
  typedef typename Vec4<T>::type V4;
  extern __shared__ __align__(128) unsigned char smem[];
  V4* s_face = reinterpret_cast<V4*>(smem);
  T* s_edge = reinterpret_cast<T*>(smem + sizeof(V4) * smem_faces);
  int* s_floop = reinterpret_cast<int*>(smem + sizeof(V4) * smem_faces + sizeof(T) * EDGE_STRIDE * smem_loops);
  __shared__ int64_t s_cell;
  __shared__ unsigned long long s_work[5];
  typedef cub::BlockReduce<double, NT> BR;
  __shared__ typename BR::TempStorage s_br;
  if (threadIdx.x < 5) s_work[threadIdx.x] = 0;
  wedge::WorkCount wc;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_cell = (int64_t)atomicAdd(&A.counters[3], 1ULL);
    __syncthreads();
    const int64_t c = s_cell;
    if (c >= A.ncell) break;
    const int64_t f0 = A.cfo[c];
    const int nf = (int)(A.cfo[c + 1] - f0);
    const int64_t l0 = A.fvo[f0];
    const int nl = (int)(A.fvo[f0 + nf] - l0);
    // stage the cell geometry (cells larger than the staging area read global memory)
    const bool fits = nf <= smem_faces && nl <= smem_loops;
    if (fits) {
      for (int i = threadIdx.x; i <= nf; i += NT) s_floop[i] = (int)(A.fvo[f0 + i] - l0);
      for (int i = threadIdx.x; i < nf; i += NT) s_face[i] = face[f0 + i];
      const int ne = nl * EDGE_STRIDE;
      const T* src = edge + l0 * EDGE_STRIDE;
      for (int i = threadIdx.x; i < ne; i += NT) s_edge[i] = src[i];
    }
    __syncthreads();
    const double sx = A.site[3 * c], sy = A.site[3 * c + 1], sz = A.site[3 * c + 2];
    double macc = 0.0;
    const int64_t p1 = A.pair_off[c + 1];
    for (int64_t p = A.pair_off[c] + threadIdx.x; p < p1; p += NT) {
      const int32_t a = A.pair_idx[p];
      const double hinv = 1.0 / A.h[a];
      const T yx = (T)((A.x[a] - sx) * hinv);
      const T yy = (T)((A.y[a] - sy) * hinv);
      const T yz = (T)((A.z[a] - sz) * hinv);
      T f;
      if (fits)
        f = pair_fraction<T, MIXED>(s_face, SmemLoops{s_floop}, s_edge, nf, yx, yy, yz, (T)hinv, wc);
      else
        f = pair_fraction<T, MIXED>(face + f0, GlobalLoops{A.fvo + f0, l0}, edge + l0 * EDGE_STRIDE, nf, yx, yy, yz,
                                    (T)hinv, wc);
      if (A.frac) A.frac[p] = (double)f;
      macc += A.m[a] * (double)f;
    }
    const double M = BR(s_br).Sum(macc);
    if (threadIdx.x == 0) {
      A.cell_mass[c] = M;
      if (A.cell_rho) A.cell_rho[c] = M / A.vol[c];
    }
  }
  atomicAdd(&s_work[0], (unsigned long long)wc.terms);
  atomicAdd(&s_work[1], (unsigned long long)wc.faces);
  atomicAdd(&s_work[2], (unsigned long long)wc.edges);
  atomicAdd(&s_work[3], (unsigned long long)wc.inner);
  atomicAdd(&s_work[4], (unsigned long long)wc.mid);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&A.counters[1], s_work[0]);
    atomicAdd(&A.counters[8], s_work[1]);
    atomicAdd(&A.counters[9], s_work[2]);
    atomicAdd(&A.counters[10], s_work[3]);
    atomicAdd(&A.counters[11], s_work[4]);
  }
}

template <typename T, bool MIXED, int NT>
int launch(map_ctx* ctx, const PreparedGrid* g, const IntegralArgs& A, cudaStream_t s) {
  typedef typename Vec4<T>::type V4;
  int sf = g->max_faces, sl = g->max_loops;
  size_t bytes = sizeof(V4) * sf + sizeof(T) * EDGE_STRIDE * sl + sizeof(int) * (sf + 1) + 16;
  const size_t cap = 160 * 1024;
  if (bytes > cap) {
    // stage only cells up to a fixed size; larger ones read global memory
    sf = 128;
    sl = (int)((cap - sizeof(V4) * sf - sizeof(int) * (sf + 1) - 16) / (sizeof(T) * EDGE_STRIDE));
    bytes = sizeof(V4) * sf + sizeof(T) * EDGE_STRIDE * sl + sizeof(int) * (sf + 1) + 16;
  }
  auto kern = pair_integrals<T, MIXED, NT>;
  CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, bytes));
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)per_sm * ctx->sm_count;
  if (blocks > g->ncell) blocks = g->ncell > 0 ? g->ncell : 1;
  kern<<<(unsigned)blocks, NT, bytes, s>>>(A, reinterpret_cast<const V4*>(MIXED ? (const void*)g->face32 : (const void*)g->face64),
                                           reinterpret_cast<const T*>(MIXED ? (const void*)g->edge32 : (const void*)g->edge64),
                                           sf, sl); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
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
  phase_begin(ctx, 2, s);
  if (ctx->cfg.precision == MAP_MIXED)
    MAP_TRY((launch<float, true, 128>(ctx, g, A, s)));
  else
    MAP_TRY((launch<double, false, 128>(ctx, g, A, s)));
  phase_end(ctx, 2, s);
  if (out->cell_vol) CUDA_TRY(cudaMemcpyAsync(out->cell_vol, g->vol, g->ncell * sizeof(double), cudaMemcpyDeviceToDevice, s));
  sum_cells<<<1, 256, 0, s>>>(g->ncell, out->cell_mass, ctx->d_total); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
