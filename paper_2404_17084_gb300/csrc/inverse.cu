// Inverse mapping (Section II-B, Eq. 4): a per-cell quantity (the ionic
// fraction f_ion,i the radiative transfer step leaves in every cell) back onto
// the particles,
//     f_ion,a = sum_i f_ion,i f_ai,   f_ai = int_{V_i} W(|r'-r_a|, h_a) dV',
// with the pair integrals f_ai of the last mapping call.  The same weights
// carry the particle masses forward (M_i = sum_a m_a f_ai), so the ionised
// mass is the same on both sides: sum_a m_a f_ion,a = sum_i f_ion,i M_i.
//
// The pair list is cell-major; the sum runs over particles.  The first call
// after a mapping builds a particle-major copy of the list (a stable radix
// sort by particle index, so each particle's entries stay in ascending cell
// order) holding the cell and f_ai of every entry; later calls with other
// cell values reuse it.  Each particle's terms are rounded products added in
// ascending cell order without FMA contraction, so the result equals a plain
// sequential FP64 sum in that order bit for bit.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace {

constexpr int INV_THREADS = 256;
constexpr int INV_CHUNK = 512;  // staged products per warp (4 KB)

// value of entry p of the cell-major list: its cell (high word) and position
__global__ void inv_pack(int64_t nc, const int64_t* __restrict__ off, unsigned long long* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nc; c += nw) {
    const int64_t b = off[c], e = off[c + 1];
    for (int64_t p = b + lane; p < e; p += 32)
      val[p] = ((unsigned long long)c << 32) | (unsigned long long)p;
  }
}

// sorted entry k: its cell and f_ai
__global__ void inv_gather(int64_t np, const unsigned long long* __restrict__ val, const double* __restrict__ frac,
                           int32_t* __restrict__ cell, double* __restrict__ f) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
    const unsigned long long v = val[k];
    cell[k] = (int32_t)(v >> 32);
    f[k] = frac[v & 0xffffffffull];
  }
}

// ioff[a] = number of entries whose particle index is below a (a = 0..n)
__global__ void inv_bounds(int64_t np, int64_t n, const int32_t* __restrict__ key, int64_t* __restrict__ ioff) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= np; k += stride) {
    const int64_t prev = k == 0 ? -1 : (int64_t)key[k - 1];
    const int64_t cur = k == np ? n : (int64_t)key[k];
    for (int64_t a = prev + 1; a <= cur; ++a) ioff[a] = k;
  }
}

// One warp per 32 consecutive particles: the warp stages the rounded
// products of a chunk of their (contiguous) entries in shared memory, loads
// coalesced, then every lane adds its own particle's products in order.
__global__ void __launch_bounds__(INV_THREADS) inv_apply(int64_t n, const int64_t* __restrict__ ioff,
                                                         const int32_t* __restrict__ cell,
                                                         const double* __restrict__ f,
                                                         const double* __restrict__ cv, double* __restrict__ out) {
  __shared__ double sprod[INV_THREADS / 32][INV_CHUNK];
  const int lane = threadIdx.x & 31;
  double* s = sprod[threadIdx.x >> 5];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; a0 < n; a0 += nw * 32) {
    const int64_t a = a0 + lane;
    const int64_t last = a0 + 32 < n ? a0 + 32 : n;
    const int64_t lo = a < n ? ioff[a] : 0, hi = a < n ? ioff[a + 1] : 0;
    const int64_t e0 = ioff[a0], e1 = ioff[last];
    double acc = 0.0;
    for (int64_t base = e0; base < e1; base += INV_CHUNK) {
      const int64_t top = e1 < base + INV_CHUNK ? e1 : base + INV_CHUNK;
      for (int64_t k = base + lane; k < top; k += 32) s[k - base] = __dmul_rn(cv[cell[k]], f[k]);
      __syncwarp();
      const int64_t kb = lo > base ? lo : base, ke = hi < top ? hi : top;
      for (int64_t k = kb; k < ke; ++k) acc = __dadd_rn(acc, s[k - base]);
      __syncwarp();
    }
    if (a < n) out[a] = acc;
  }
}

int bits_for(int64_t n) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < n) ++b;
  return b;
}

int build_index(map_ctx* ctx, cudaStream_t s) {
  const int64_t np = ctx->n_pairs, nc = ctx->last_ncell, n = ctx->last_npart;
  int64_t* ioff;
  MAP_TRY(ensure_t(ctx, ctx->ws_inv[0], n + 1, &ioff));
  ctx->inv_off = ioff;
  if (np > 0) {
    unsigned long long *val, *val_s;
    int32_t *key_s, *cell;
    double* f;
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[1], np, &cell));
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[2], np, &f));
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[3], np, &val));
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[4], np, &val_s));
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[5], np, &key_s));
    const unsigned g = (unsigned)ctx->sm_count * 8;
    inv_pack<<<g, 256, 0, s>>>(nc, ctx->pair_off, val); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    size_t tb = 0;
    const int nb = bits_for(n);
    CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, ctx->pair_idx, key_s, val, val_s, np, 0, nb, s));
    MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
    CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tb, ctx->pair_idx, key_s, val, val_s, np, 0, nb, s));
    inv_gather<<<g, 256, 0, s>>>(np, val_s, ctx->pair_frac, cell, f); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    inv_bounds<<<g, 256, 0, s>>>(np, n, key_s, ioff); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    ctx->inv_cell = cell;
    ctx->inv_frac = f;
  } else {
    CUDA_TRY(cudaMemsetAsync(ioff, 0, (n + 1) * sizeof(int64_t), s));
    ctx->inv_cell = nullptr;
    ctx->inv_frac = nullptr;
  }
  ctx->inv_ready = true;
  // the copy reads the pair list, which a later map_get_pairs sorts in place
  // on the mapping call's stream
  if (s != ctx->last_stream) CUDA_TRY(cudaStreamSynchronize(s));
  return MAP_OK;
}

}  // namespace

extern "C" int map_cells_to_particles(map_ctx* ctx, const double* cell_value, double* particle_value, int64_t n,
                                      void* stream) {
  if (!ctx || !particle_value || (!cell_value && ctx->last_ncell > 0)) return MAP_EINVAL;
  if (!ctx->pair_off || !ctx->pair_frac || n != ctx->last_npart) return MAP_EINVAL;
  if (ctx->n_pairs >= (int64_t(1) << 32) || ctx->last_ncell >= (int64_t(1) << 31)) return MAP_EINVAL;
  if (n == 0) return MAP_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ctx->inv_ready) MAP_TRY(build_index(ctx, s));
  const int64_t groups = (n + 31) / 32;
  const int64_t per_block = INV_THREADS / 32;
  int64_t blocks = (groups + per_block - 1) / per_block;
  const int64_t cap = (int64_t)ctx->sm_count * 8;
  if (blocks > cap) blocks = cap;
  inv_apply<<<(unsigned)blocks, INV_THREADS, 0, s>>>(n, ctx->inv_off, ctx->inv_cell, ctx->inv_frac, cell_value,
                                                      particle_value);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
