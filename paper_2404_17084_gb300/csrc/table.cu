// Table variant of the pair integrals (MAP_TABLE): Section II-B's production
// route, where the vertex-pyramid integral I(r0, R0, phi) is pre-computed on
// a grid and interpolated, here by the texture unit's trilinear filtering.
//
// Table: n nodes per axis over r0 in [0, 2], rho = R0 / sqrt(4 - r0^2) in
// [0, 1] and phi in [0, pi/2] (x: phi, y: rho, z: r0), FP32 texels built
// once per context in FP64 from the closed form: I = Omega/(4 pi) + K' over
// [0, R0 tan phi] (the solid angle of the pyramid plus its kernel part; 0 at
// r0 = 0 and at R0 = 0, the limits).  Beyond the table's box the pyramid
// integral is known exactly: for r0 >= 2 a face contributes nothing to the
// solid-angle-free sum, and for rho >= 1 the edge line lies beyond the
// support, where K' = -c0 dPhi.
//
// Sum per pair: f = [inside] + sum_faces sum_edges s_f s_e K'_e as in the
// closed-form builds, with K'_e = [I(phi_b) - I(phi_a)] - [Omega(phi_b) -
// Omega(phi_a)] / (4 pi) from two table lookups and the exact solid angles:
// over a closed cell the exact solid angles sum to [inside], so this equals
// the paper's sum of interpolated pyramid integrals, with faces wholly beyond
// the support skipped (their pyramids' interpolation errors would not
// cancel).  The texture unit's weights carry 8 fractional bits, so a lookup
// differs from exact trilinear interpolation by at most 3 * 2^-9 of the
// largest difference between neighbouring texels.
#include "internal.cuh"
#include "wedge.cuh"

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr float HALF_PI_F = 1.57079632679489662f;
constexpr double HALF_PI = 1.57079632679489661923;

__global__ void table_fill(int n, cudaSurfaceObject_t surf) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
  if (k >= n) return;
  const double r0 = 2.0 * i / (n - 1);
  const double span = sqrt(fmax(4.0 - r0 * r0, 0.0));
  const double R0 = span * j / (n - 1);
  const double phi = k == n - 1 ? HALF_PI - 1e-12 : HALF_PI * k / (n - 1);
  double I = 0.0;
  if (r0 > 0.0 && R0 > 0.0 && phi > 0.0) {
    const double s = R0 * tan(phi);
    const double U = sqrt(r0 * r0 + R0 * R0 + s * s);
    wedge::WorkCount wc;
    I = wedge::omega(r0, R0, s, U) * wedge::INV_4PI + wedge::kprime_edge<double, false>(r0, R0, 0.0, s, wc);
  }
  surf3Dwrite((float)I, surf, k * (int)sizeof(float), j, i);
}

// K' of one edge from the table: lo < hi are the vertices' signed positions
// along the edge from the foot, all lengths in units of h.
__device__ __forceinline__ float kprime_table(cudaTextureObject_t tab, float tn1, float r0, float R0, float lo,
                                              float hi, float inv_span, float c0) {
  const float pa = wedge::atan2_fast(lo, R0), pb = wedge::atan2_fast(hi, R0);
  const float rho = R0 * inv_span;
  if (rho >= 1.f) return -c0 * (pb - pa);
  const float zc = 0.5f * r0 * tn1 + 0.5f, yc = rho * tn1 + 0.5f, xs = tn1 / HALF_PI_F;
  const float Ia = copysignf(tex3D<float>(tab, fabsf(pa) * xs + 0.5f, yc, zc), pa);
  const float Ib = copysignf(tex3D<float>(tab, fabsf(pb) * xs + 0.5f, yc, zc), pb);
  // Omega = Phi - A, A = arg(R0 U + i r0 s) in (-pi/2, pi/2): the difference
  // of the A's as the argument of one product (it lies in (-pi, pi))
  const float r02 = r0 * r0, R02 = R0 * R0;
  const float Ua = sqrtf(r02 + R02 + lo * lo), Ub = sqrtf(r02 + R02 + hi * hi);
  const float re = R02 * Ua * Ub + r02 * lo * hi, im = r0 * R0 * (hi * Ua - lo * Ub);
  const float dA = wedge::atan2_fast(im, re);
  return (Ib - Ia) - ((pb - pa) - dA) * (float)wedge::INV_4PI;
}

template <int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) pair_integrals_table(BatchArgs B, cudaTextureObject_t tab, float tn1) {
  __shared__ SnapDesc descs[NW];
  const int lane = threadIdx.x & 31;
  SnapDesc& A = descs[threadIdx.x >> 5];
  int cur = -1;
  const int64_t total = queue_total(B);
  for (;;) {
    int64_t g = 0;
    if (lane == 0) g = (int64_t)atomicAdd(&B.counters[3], 1ULL);
    g = __shfl_sync(FULLM, g, 0);
    if (g >= total) break;
    int jl = 0, jh = B.nsnap - 1;
    while (jl < jh) {
      const int jm = (jl + jh + 1) >> 1;
      if (B.item_base[jm] <= g) jl = jm; else jh = jm - 1;
    }
    if (jl != cur) {
      __syncwarp();
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(B.snaps + jl);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&A);
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
    const float4* __restrict__ ecell = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(A.edge) +
                                                                       l0 * EDGE_STRIDE);
    const double sx = A.site[3 * c], sy = A.site[3 * c + 1], sz = A.site[3 * c + 2];
    double macc = 0.0;
    const int64_t pb = item.lo, pe = item.lo + item.cnt;
    for (int64_t p0 = pb; p0 < pe; p0 += 32) {
      const int64_t p = p0 + lane;
      const bool active = p < pe;
      float yx = 0.f, yy = 0.f, yz = 0.f, hinv = 0.f;
      int32_t a = 0;
      if (active) {
        a = A.pair_idx[p];
        hinv = 1.0f / (float)A.h[a];
        yx = (float)(A.x[a] - sx) * hinv;
        yy = (float)(A.y[a] - sy) * hinv;
        yz = (float)(A.z[a] - sz) * hinv;
      }
      bool inside = true;
      float acc = 0.f, cmp = 0.f;  // compensated sum of the edge terms
      int kb = 0;
      for (int fi = 0; fi < nf; ++fi) {
        const float4 F = face[f0 + fi];
        const int ke = (int)(A.fvo[f0 + fi + 1] - l0);
        const float r0s = F.w * hinv - (F.x * yx + F.y * yy + F.z * yz);
        const bool fin = r0s >= 0.f;
        const float r0 = fabsf(r0s);
        inside = inside && fin;
        bool inrange = active && r0 < 2.f;
        if (inrange) {
          // the face's bounding sphere wholly beyond the support: nothing to add
          const float4 Q = fsph[f0 + fi];
          const float dx = yx - Q.x * hinv, dy = yy - Q.y * hinv, dz = yz - Q.z * hinv;
          const float rr = 2.f + Q.w * hinv;
          if (dx * dx + dy * dy + dz * dz >= rr * rr * 1.00001f) inrange = false;
        }
        if (__any_sync(FULLM, inrange)) {
          const float inv_span = rsqrtf(fmaxf(4.f - r0 * r0, 1e-30f));
          const float c0 = wedge::c0_of(r0);
          for (int k = kb; k < ke; ++k) {
            const float4 E0 = ecell[3 * k], E1 = ecell[3 * k + 1], E2 = ecell[3 * k + 2];
            if (!inrange) continue;
            const float R0s = (E0.x * yx + E0.z * yy + E1.x * yz) - E2.x * hinv;
            const float base = E0.y * yx + E0.w * yy + E1.y * yz;
            const float lo = E1.z * hinv - base, hi = E1.w * hinv - base;
            const float kp = kprime_table(tab, tn1, r0, fabsf(R0s), lo, hi, inv_span, c0);
            const float y = ((R0s >= 0.f) == fin ? kp : -kp) - cmp;
            const float t = acc + y;
            cmp = (t - acc) - y;
            acc = t;
          }
        }
        kb = ke;
      }
      if (active) {
        const double f = (inside ? 1.0 : 0.0) + ((double)acc - (double)cmp);
        if (A.frac) A.frac[p] = f;
        macc += A.m[a] * f;
      }
    }
    for (int o = 16; o > 0; o >>= 1) macc += __shfl_down_sync(FULLM, macc, o);
    if (lane == 0) A.partial[it] = macc;
    __syncwarp();
  }
}

}  // namespace

int table_ensure(map_ctx* ctx, cudaStream_t s) {
  if (ctx->tab_tex) return MAP_OK;
  const int n = ctx->cfg.table_n;
  if (n < 2 || n > 512) return MAP_EINVAL;
  cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
  cudaArray_t arr = nullptr;
  CUDA_TRY(cudaMalloc3DArray(&arr, &ch, make_cudaExtent(n, n, n), cudaArraySurfaceLoadStore));
  ctx->tab_arr = arr;
  ctx->bytes_in_use += (size_t)n * n * n * sizeof(float);
  cudaResourceDesc rd{};
  rd.resType = cudaResourceTypeArray;
  rd.res.array.array = arr;
  cudaSurfaceObject_t surf = 0;
  CUDA_TRY(cudaCreateSurfaceObject(&surf, &rd));
  table_fill<<<dim3((n + 63) / 64, n, n), 64, 0, s>>>(n, surf); ++ctx->launches;
  const cudaError_t e = cudaGetLastError();
  // the surface is only needed by the fill: wait for it, then drop it
  const cudaError_t w = cudaStreamSynchronize(s);
  cudaDestroySurfaceObject(surf);
  if (e != cudaSuccess || w != cudaSuccess) return MAP_ECUDA;
  cudaTextureDesc td{};
  td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
  td.filterMode = cudaFilterModeLinear;
  td.readMode = cudaReadModeElementType;
  td.normalizedCoords = 0;
  cudaTextureObject_t tex = 0;
  CUDA_TRY(cudaCreateTextureObject(&tex, &rd, &td, nullptr));
  ctx->tab_tex = tex;
  return MAP_OK;
}

void table_free(map_ctx* ctx) {
  if (ctx->tab_tex) cudaDestroyTextureObject(ctx->tab_tex);
  if (ctx->tab_arr) cudaFreeArray(ctx->tab_arr);
  ctx->tab_tex = 0;
  ctx->tab_arr = nullptr;
}

int launch_table(map_ctx* ctx, const BatchArgs& B, cudaStream_t s) {
  constexpr int NW = 4, MINB = 6;
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_integrals_table<NW, MINB>, NW * 32, 0));
  const int64_t want = (B.total + NW - 1) / NW;
  int64_t blocks = (int64_t)ctx->sm_count * (per_sm > 0 ? per_sm : 1);
  if (blocks > want) blocks = want > 0 ? want : 1;
  pair_integrals_table<NW, MINB><<<(unsigned)blocks, NW * 32, 0, s>>>(B, ctx->tab_tex, (float)(ctx->cfg.table_n - 1));
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
