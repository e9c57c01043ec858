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
// cell values reuse it.  Each particle's terms are fused into its running sum
// one at a time in ascending cell order (acc <- RN(acc + v_i f_ai), one
// rounding per term), so the result equals that sequential FP64 sum bit for
// bit.
//
// Locality of the cell-value gather: the copy stores, per entry, the Morton
// rank of its cell's site (the order the pair walk visits cells in) instead
// of the cell index, and every call first permutes the caller's cell values
// into that order (one coalesced write per cell).  A particle's cells lie
// within its support, so their ranks are close and the gathers of one
// particle's entries share 32-byte sectors; the terms, their values and
// their order are unchanged.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace {

constexpr int INV_THREADS = 256;

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

// rank[morton[k]] = k: the Morton rank of every cell
__global__ void inv_rank(int64_t nc, const int32_t* __restrict__ morton, int32_t* __restrict__ rank) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += stride) rank[morton[k]] = (int32_t)k;
}

// sorted entry k: the Morton rank of its cell, and f_ai
__global__ void inv_gather(int64_t np, const unsigned long long* __restrict__ val, const double* __restrict__ frac,
                           const int32_t* __restrict__ rank, int32_t* __restrict__ cell, double* __restrict__ f) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
    const unsigned long long v = val[k];
    cell[k] = rank[v >> 32];
    f[k] = frac[v & 0xffffffffull];
  }
}

// the caller's cell values in Morton order: out[k] = v[morton[k]]
__global__ void inv_permute(int64_t nc, const int32_t* __restrict__ morton, const double* __restrict__ v,
                            double* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += stride) out[k] = __ldg(v + morton[k]);
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

// per particle: its number of entries, and its index (for the sort by count)
__global__ void inv_counts(int64_t n, const int64_t* __restrict__ ioff, unsigned* __restrict__ cnt,
                           int32_t* __restrict__ ids) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += stride) {
    cnt[a] = (unsigned)(ioff[a + 1] - ioff[a]);
    ids[a] = (int32_t)a;
  }
}

// number of particles with more than INV_LONG entries (counts sorted in
// decreasing order)
constexpr unsigned INV_LONG = 256;

__global__ void inv_count_long(int64_t n, const unsigned* __restrict__ cnt_sorted, int64_t* __restrict__ nlong) {
  int64_t lo = 0, hi = n;  // first index whose count is <= INV_LONG
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cnt_sorted[mid] > INV_LONG) lo = mid + 1; else hi = mid;
  }
  *nlong = lo;
}

// Work items in order of decreasing entry count: first one item per long
// particle (more than INV_LONG entries), then one item per 32 of the others.
//  * A long particle is summed by a whole warp: chunks of 256 entries loaded
//    coalesced (8 per lane), staged in shared memory, and fused into the
//    running sum by lane 0 in order.
//  * A group of 32 short particles is summed lane t by particle t, in rounds
//    of INV_R entries per particle: the warp stages entries
//    [INV_R j, INV_R (j + 1)) of its 32 particles (8 lanes load 8
//    consecutive entries of one particle), then every lane fuses its own.
//    The sorted order gives the 32 sums of a group nearly the same length.
// Staged entries are (cell value, f_ai) pairs, 16 bytes; rows are padded to
// an odd number of pairs, so the lanes read different rows without bank
// conflicts.  Both paths are software pipelined: the cell indices and f_ai
// of the next round or chunk are loaded while the current one is summed.
constexpr int INV_R = 8;
constexpr int INV_ROW = INV_R + 1;
constexpr int INV_CHUNK = 256;  // entries per chunk of a long particle (<= 32 * INV_ROW)
constexpr int INV_U = 8;        // loads per lane per round or chunk

struct Pending {
  int c[INV_U];
  double f[INV_U];
  bool ok[INV_U];
};

// issue the loads of cell index and f_ai of the entries entry(u) names
// (entry(u, k, kend): the entry's position k, loaded only if below kend)
template <class Entry>
__device__ __forceinline__ void issue(Pending& P, Entry entry, const int32_t* __restrict__ cell,
                                      const double* __restrict__ f) {
#pragma unroll
  for (int u = 0; u < INV_U; ++u) {
    int64_t k, kend;
    entry(u, k, kend);
    P.ok[u] = k < kend;
    P.c[u] = P.ok[u] ? __ldg(cell + k) : 0;
    P.f[u] = P.ok[u] ? __ldg(f + k) : 0.0;
  }
}

// gather the cell values of the pending entries and stage (value, f_ai) at
// dst + dstride * u
__device__ __forceinline__ void land(const Pending& P, const double* __restrict__ cv, double2* dst, int dstride) {
  double v[INV_U];
#pragma unroll
  for (int u = 0; u < INV_U; ++u) v[u] = P.ok[u] ? __ldg(cv + P.c[u]) : 0.0;
#pragma unroll
  for (int u = 0; u < INV_U; ++u) dst[dstride * u] = make_double2(v[u], P.f[u]);
}

__global__ void __launch_bounds__(INV_THREADS) inv_apply(int64_t n, const int64_t* __restrict__ nlong_p,
                                                         const int32_t* __restrict__ order,
                                                         const int64_t* __restrict__ ioff,
                                                         const int32_t* __restrict__ cell,
                                                         const double* __restrict__ f,
                                                         const double* __restrict__ cv, double* __restrict__ out) {
  constexpr int W = INV_THREADS / 32;
  __shared__ double2 sp[W][32 * INV_ROW];
  __shared__ int64_t slo[W][32], shi[W][32];
  const int lane = threadIdx.x & 31, sub = lane >> 3, e = lane & 7, w = threadIdx.x >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nlong = *nlong_p;
  const int64_t items = nlong + (n - nlong + 31) / 32;
  Pending P;
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nw) {
    if (it < nlong) {
      const int64_t a = order[it];
      const int64_t lo = ioff[a], hi = ioff[a + 1];
      double acc = 0.0;
      auto chunk = [&](int64_t base) {
        issue(P, [&](int u, int64_t& k, int64_t& kend) { k = base + 32 * u + lane; kend = hi; }, cell, f);
      };
      chunk(lo);
      for (int64_t base = lo; base < hi; base += INV_CHUNK) {
        land(P, cv, &sp[w][lane], 32);
        __syncwarp();
        if (base + INV_CHUNK < hi) chunk(base + INV_CHUNK);
        if (lane == 0) {
          const int m = hi - base < INV_CHUNK ? (int)(hi - base) : INV_CHUNK;
          for (int q = 0; q < m; ++q) {
            const double2 t = sp[w][q];
            acc = __fma_rn(t.x, t.y, acc);
          }
        }
        __syncwarp();
      }
      if (lane == 0) out[a] = acc;
      continue;
    }
    const int64_t g0 = nlong + 32 * (it - nlong);
    const int64_t a = g0 + lane < n ? (int64_t)order[g0 + lane] : -1;
    const int64_t lo = a >= 0 ? ioff[a] : 0, hi = a >= 0 ? ioff[a + 1] : 0;
    slo[w][lane] = lo;
    shi[w][lane] = hi;
    __syncwarp();
    const int cnt = (int)(hi - lo);
    const int rounds = (int)((__reduce_max_sync(0xffffffffu, (unsigned)cnt) + INV_R - 1) / INV_R);
    auto round = [&](int j) {
      issue(P, [&](int i, int64_t& k, int64_t& kend) {
        k = slo[w][4 * i + sub] + (int64_t)INV_R * j + e;
        kend = shi[w][4 * i + sub];
      }, cell, f);
    };
    if (rounds > 0) round(0);
    double acc = 0.0;
    for (int j = 0; j < rounds; ++j) {
      land(P, cv, &sp[w][sub * INV_ROW + e], 4 * INV_ROW);
      __syncwarp();
      if (j + 1 < rounds) round(j + 1);
      const int left = cnt - INV_R * j;
      const int m = left < INV_R ? left : INV_R;
      for (int q = 0; q < m; ++q) {
        const double2 t = sp[w][lane * INV_ROW + q];
        acc = __fma_rn(t.x, t.y, acc);
      }
      __syncwarp();
    }
    if (a >= 0) out[a] = acc;
    __syncwarp();  // slo/shi are rewritten by the next item
  }
}

// bits that hold every value below n (at most 32)
int bits_for(int64_t n) {
  int b = 1;
  while (b < 32 && (int64_t(1) << b) < n) ++b;
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
    // the pair walk's Morton order of the cells, sorted by pairs_build with
    // the list this copy is made from (a buffer no other step writes)
    if (ctx->ws_pairs[14].cap < (size_t)nc * sizeof(int32_t)) return MAP_EINVAL;
    const int32_t* morton = static_cast<const int32_t*>(ctx->ws_pairs[14].p);
    int32_t* rank;
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[11], nc, &rank));
    inv_rank<<<g, 256, 0, s>>>(nc, morton, rank); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    ctx->inv_morton = morton;
    inv_gather<<<g, 256, 0, s>>>(np, val_s, ctx->pair_frac, rank, cell, f); ++ctx->launches;
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
  // particles in order of decreasing entry count (stable: ties by index)
  unsigned *cnt, *cnt_s;
  int32_t *ids, *order;
  MAP_TRY(ensure_t(ctx, ctx->ws_inv[6], n, &cnt));
  MAP_TRY(ensure_t(ctx, ctx->ws_inv[7], n, &cnt_s));
  MAP_TRY(ensure_t(ctx, ctx->ws_inv[8], n, &ids));
  MAP_TRY(ensure_t(ctx, ctx->ws_inv[9], n, &order));
  inv_counts<<<(unsigned)ctx->sm_count * 8, 256, 0, s>>>(n, ioff, cnt, ids); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t tb2 = 0;
  const int cb = bits_for(np + 1);
  CUDA_TRY(cub::DeviceRadixSort::SortPairsDescending(nullptr, tb2, cnt, cnt_s, ids, order, n, 0, cb, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb2));
  CUDA_TRY(cub::DeviceRadixSort::SortPairsDescending(ctx->cub_tmp.p, tb2, cnt, cnt_s, ids, order, n, 0, cb, s));
  int64_t* nlong;
  MAP_TRY(ensure_t(ctx, ctx->ws_inv[10], 1, &nlong));
  inv_count_long<<<1, 1, 0, s>>>(n, cnt_s, nlong); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  ctx->inv_order = order;
  ctx->inv_nlong = nlong;
  ctx->inv_ready = true;
  // the copy reads the pair list, which a later map_get_pairs sorts in place:
  // that sort runs on this call's stream or one ordered after it (ctx_enter)
  return MAP_OK;
}

}  // namespace

extern "C" int map_cells_to_particles(map_ctx* ctx, const double* cell_value, double* particle_value, int64_t n,
                                      void* stream) {
  if (!ctx || !particle_value || (!cell_value && ctx->last_ncell > 0)) return MAP_EINVAL;
  if (!ctx->pair_off || !ctx->pair_frac || n != ctx->last_npart) return MAP_EINVAL;
  if (ctx->n_pairs >= (int64_t(1) << 32) || ctx->last_ncell >= (int64_t(1) << 31)) return MAP_EINVAL;
  if (n == 0) return MAP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MAP_ENTER(ctx, s);
  if (!ctx->inv_ready) MAP_TRY(build_index(ctx, s));
  const int64_t groups = (n + 31) / 32;
  const int64_t per_block = INV_THREADS / 32;
  int64_t blocks = (groups + per_block - 1) / per_block;
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inv_apply, INV_THREADS, 0));
  const int64_t cap = (int64_t)ctx->sm_count * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  const double* cv = cell_value;
  if (ctx->inv_cell) {
    const int64_t nc = ctx->last_ncell;
    double* cv_m;
    MAP_TRY(ensure_t(ctx, ctx->ws_inv[12], nc, &cv_m));
    inv_permute<<<(unsigned)ctx->sm_count * 8, 256, 0, s>>>(nc, ctx->inv_morton, cell_value, cv_m); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    cv = cv_m;
  }
  inv_apply<<<(unsigned)blocks, INV_THREADS, 0, s>>>(n, ctx->inv_nlong, ctx->inv_order, ctx->inv_off, ctx->inv_cell,
                                                      ctx->inv_frac, cv, particle_value);
  ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
