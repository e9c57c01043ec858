// Device octree over a particle set.
//
// Octree (Section III-A, built as an octree with a leaf capacity instead of
// the paper's RCB tree): 63-bit Morton keys (21 bits per axis) are radix
// sorted; nodes are built level by level from the sorted keys, a node at
// level L being the cube of side 2^-L holding a contiguous key range, split
// while it holds more than leaf_size particles (up to level 21).  Labels carry
// a leading 1 bit, so parent = label >> 3 (the paper's heap-style label
// arithmetic with eight children).  Node mass and centre of mass are summed
// bottom-up; node size (distance from the centre of mass to the furthest
// particle, Section III-A), largest h and bounding box are reduced over each
// node's particles.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace {

constexpr int MORTON_BITS = 21;
constexpr int64_t BIG_NODE = 4096;

struct MaxOp {
  __device__ __forceinline__ double operator()(double a, double b) const { return a > b ? a : b; }
};
struct MinOp {
  __device__ __forceinline__ double operator()(double a, double b) const { return a < b ? a : b; }
};

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

__device__ __forceinline__ uint64_t coord21(double v) {
  double s = floor(v * 2097152.0);
  if (!(s >= 0.0)) s = 0.0;
  if (s > 2097151.0) s = 2097151.0;
  return (uint64_t)s;
}

__global__ void morton_keys(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ z, uint64_t* keys, int32_t* idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = (spread3(coord21(x[i])) << 2) | (spread3(coord21(y[i])) << 1) | spread3(coord21(z[i]));
  idx[i] = (int32_t)i;
}

__global__ void gather_sorted(int64_t n, const int32_t* __restrict__ idx, const double* __restrict__ x,
                              const double* __restrict__ y, const double* __restrict__ z,
                              const double* __restrict__ m, const double* __restrict__ h, double* xs, double* ys,
                              double* zs, double* ms, double* hs, float* split, float* hs32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t a = idx[i];
  const double px = x[a] + 0.0, py = y[a] + 0.0, pz = z[a] + 0.0;  // + 0.0: -0.0 -> +0.0 (bit-ordered min/max)
  xs[i] = px;
  ys[i] = py;
  zs[i] = pz;
  ms[i] = m ? m[a] : 1.0;
  hs[i] = h ? h[a] : 0.0;
  if (hs32) hs32[i] = (float)h[a];  // set only for trees built with h
  // FP32 hi/lo split of the coordinates: x = hi + lo to ~2^-48, so that the
  // difference of two nearby points, (hi_j - hi_i) + (lo_j - lo_i), keeps
  // ~24 bits relative to the separation
  const float hx = (float)px, hy = (float)py, hz = (float)pz;
  split[6 * i + 0] = hx; split[6 * i + 1] = (float)(px - (double)hx);
  split[6 * i + 2] = hy; split[6 * i + 3] = (float)(py - (double)hy);
  split[6 * i + 4] = hz; split[6 * i + 5] = (float)(pz - (double)hz);
}

__device__ __forceinline__ int64_t lower_octant(const uint64_t* keys, int64_t b, int64_t e, int shift, int o) {
  // first position in [b,e) whose octant at this shift is >= o
  int64_t lo = b, hi = e;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int)((keys[mid] >> shift) & 7) < o) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void split_count(int64_t lb, int64_t le, const uint64_t* __restrict__ keys, const int64_t* __restrict__ nb,
                            const int64_t* __restrict__ ne, const int32_t* __restrict__ lev, int leaf_size,
                            int32_t* nchild) {
  int64_t i = lb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= le) return;
  int64_t b = nb[i], e = ne[i];
  int L = lev[i];
  int cnt = 0;
  if (e - b > leaf_size && L < MORTON_BITS) {
    int shift = 3 * (MORTON_BITS - L - 1);
    int64_t prev = b;
    for (int o = 1; o <= 8; ++o) {
      int64_t nx = (o == 8) ? e : lower_octant(keys, b, e, shift, o);
      if (nx > prev) ++cnt;
      prev = nx;
    }
  }
  nchild[i - lb] = cnt;
}

__global__ void split_write(int64_t lb, int64_t le, int64_t next_begin, const uint64_t* __restrict__ keys,
                            int64_t* nb, int64_t* ne, int32_t* lev, int64_t* label, int64_t* first_child,
                            int32_t* nchild_out, int32_t* parent, const int32_t* __restrict__ nchild,
                            const int64_t* __restrict__ choff) {
  int64_t i = lb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= le) return;
  int cnt = nchild[i - lb];
  nchild_out[i] = cnt;
  if (cnt == 0) { first_child[i] = -1; return; }
  int64_t b = nb[i], e = ne[i];
  int L = lev[i];
  int shift = 3 * (MORTON_BITS - L - 1);
  int64_t w = next_begin + choff[i - lb];
  first_child[i] = w;
  int64_t prev = b;
  for (int o = 1; o <= 8; ++o) {
    int64_t nx = (o == 8) ? e : lower_octant(keys, b, e, shift, o);
    if (nx > prev) {
      nb[w] = prev;
      ne[w] = nx;
      lev[w] = L + 1;
      label[w] = label[i] * 8 + (o - 1);
      parent[w] = (int32_t)i;
      ++w;
    }
    prev = nx;
  }
}

// Bottom-up pass for one level: leaves sum their particles in sorted order,
// internal nodes sum their children in octant order (mass, mass-weighted
// position); bounding box and largest h are the union / maximum over the
// particles (leaves) or the children (internal nodes), exact in any order.
__device__ __forceinline__ void node_sum_one(int64_t i, const int64_t* __restrict__ nb,
                                             const int64_t* __restrict__ ne, const int64_t* __restrict__ fc,
                                             const int32_t* __restrict__ nch, const double* __restrict__ xs,
                                             const double* __restrict__ ys, const double* __restrict__ zs,
                                             const double* __restrict__ ms, const double* __restrict__ hs,
                                             double* mass, double* msum, unsigned long long* hmax_bits,
                                             unsigned long long* bbox, int32_t* owner) {
  double M = 0, Sx = 0, Sy = 0, Sz = 0, hm = 0;
  double lo0 = 1e300, lo1 = 1e300, lo2 = 1e300, hi0 = 0, hi1 = 0, hi2 = 0;
  if (nch[i] == 0) {
    for (int64_t k = nb[i]; k < ne[i]; ++k) {
      const double mk = ms[k], x = xs[k], y = ys[k], z = zs[k];
      M += mk;
      Sx += mk * x;
      Sy += mk * y;
      Sz += mk * z;
      hm = fmax(hm, hs[k]);
      lo0 = fmin(lo0, x); lo1 = fmin(lo1, y); lo2 = fmin(lo2, z);
      hi0 = fmax(hi0, x); hi1 = fmax(hi1, y); hi2 = fmax(hi2, z);
      owner[k] = (int32_t)i;
    }
  } else {
    for (int64_t c = fc[i]; c < fc[i] + nch[i]; ++c) {
      M += mass[c];
      Sx += msum[3 * c];
      Sy += msum[3 * c + 1];
      Sz += msum[3 * c + 2];
      hm = fmax(hm, bitsd(hmax_bits[c]));
      lo0 = fmin(lo0, bitsd(bbox[6 * c])); lo1 = fmin(lo1, bitsd(bbox[6 * c + 1])); lo2 = fmin(lo2, bitsd(bbox[6 * c + 2]));
      hi0 = fmax(hi0, bitsd(bbox[6 * c + 3])); hi1 = fmax(hi1, bitsd(bbox[6 * c + 4])); hi2 = fmax(hi2, bitsd(bbox[6 * c + 5]));
    }
  }
  mass[i] = M;
  msum[3 * i] = Sx;
  msum[3 * i + 1] = Sy;
  msum[3 * i + 2] = Sz;
  hmax_bits[i] = dbits(hm);
  bbox[6 * i] = dbits(lo0); bbox[6 * i + 1] = dbits(lo1); bbox[6 * i + 2] = dbits(lo2);
  bbox[6 * i + 3] = dbits(hi0); bbox[6 * i + 4] = dbits(hi1); bbox[6 * i + 5] = dbits(hi2);
}

__global__ void node_sums(int64_t lb, int64_t le, const int64_t* __restrict__ nb, const int64_t* __restrict__ ne,
                          const int64_t* __restrict__ fc, const int32_t* __restrict__ nch,
                          const double* __restrict__ xs, const double* __restrict__ ys,
                          const double* __restrict__ zs, const double* __restrict__ ms,
                          const double* __restrict__ hs, double* mass, double* msum /* 3 per node: sum m x */,
                          unsigned long long* hmax_bits, unsigned long long* bbox, int32_t* owner) {
  int64_t i = lb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= le) return;
  node_sum_one(i, nb, ne, fc, nch, xs, ys, zs, ms, hs, mass, msum, hmax_bits, bbox, owner);
}

__global__ void node_com(int64_t nn, const double* __restrict__ mass, const double* __restrict__ msum, double* com,
                         unsigned long long* size_bits) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  double M = mass[i];
  com[3 * i] = msum[3 * i] / M;
  com[3 * i + 1] = msum[3 * i + 1] / M;
  com[3 * i + 2] = msum[3 * i + 2] / M;
  size_bits[i] = 0ULL;
}

// Node size (distance from the centre of mass to the furthest particle,
// Section III-A), needed by the pseudo-particle walk only.  Small nodes: every
// particle walks up from its leaf while the node holds at most BIG_NODE
// particles and reduces into it with atomics.
__global__ void node_extent_small(int64_t n, const int32_t* __restrict__ owner, const int32_t* __restrict__ parent,
                                  const int64_t* __restrict__ nb, const int64_t* __restrict__ ne,
                                  const double* __restrict__ xs, const double* __restrict__ ys,
                                  const double* __restrict__ zs, const double* __restrict__ com,
                                  unsigned long long* size_bits) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double x = xs[k], y = ys[k], z = zs[k];
  int32_t node = owner[k];
  while (node >= 0 && ne[node] - nb[node] <= BIG_NODE) {
    double dx = x - com[3 * node], dy = y - com[3 * node + 1], dz = z - com[3 * node + 2];
    atomicMax(&size_bits[node], dbits(sqrt(dx * dx + dy * dy + dz * dz)));
    node = parent[node];
  }
}

// Big nodes: several blocks per node, each reducing a slice of its range.
__global__ void node_extent_big(const int32_t* __restrict__ big, int slices, const int64_t* __restrict__ nb,
                                const int64_t* __restrict__ ne, const double* __restrict__ xs,
                                const double* __restrict__ ys, const double* __restrict__ zs,
                                const double* __restrict__ com, unsigned long long* size_bits) {
  const int32_t node = big[blockIdx.x / slices];
  const int slice = blockIdx.x % slices;
  const double cx = com[3 * node], cy = com[3 * node + 1], cz = com[3 * node + 2];
  double smax = 0;
  for (int64_t k = nb[node] + (int64_t)slice * blockDim.x + threadIdx.x; k < ne[node];
       k += (int64_t)slices * blockDim.x) {
    const double dx = xs[k] - cx, dy = ys[k] - cy, dz = zs[k] - cz;
    smax = fmax(smax, sqrt(dx * dx + dy * dy + dz * dz));
  }
  typedef cub::BlockReduce<double, 256> BR;
  __shared__ typename BR::TempStorage tmp;
  const double v = BR(tmp).Reduce(smax, MaxOp());
  if (threadIdx.x == 0) atomicMax(&size_bits[node], dbits(v));
}

// FP32 copy of each node's bounding box (rounded outward) and largest h
// (rounded up), for conservative FP32 pruning in traversals.
// The walks' node record, two 16-byte loads: the outward-rounded FP32 box,
// the largest h, and (bits of the last float) first child << 4 | child count
// for an internal node with a first child below 2^28, 0 for a leaf, and
// NODE_LINK_FAR when the index does not fit (read the arrays then).
__global__ void node_box32(int64_t nn, const unsigned long long* __restrict__ bbox,
                           const unsigned long long* __restrict__ hmax, const int64_t* __restrict__ fc,
                           const int32_t* __restrict__ nch, float* box32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  for (int k = 0; k < 3; ++k) {
    box32[8 * i + k] = __double2float_rd(bitsd(bbox[6 * i + k]));
    box32[8 * i + 3 + k] = __double2float_ru(bitsd(bbox[6 * i + 3 + k]));
  }
  box32[8 * i + 6] = __double2float_ru(bitsd(hmax[i]));
  const int nc = nch[i];
  const int64_t f = fc[i];
  const unsigned link = nc == 0 ? 0u : (f < (1LL << 28) ? ((unsigned)f << 4) | (unsigned)nc : NODE_LINK_FAR);
  box32[8 * i + 7] = __uint_as_float(link);
}

__global__ void collect_big(int64_t nn, const int64_t* __restrict__ nb, const int64_t* __restrict__ ne, int32_t* big,
                            unsigned long long* nbig) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  if (ne[i] - nb[i] > BIG_NODE) big[atomicAdd(nbig, 1ULL)] = (int32_t)i;
}

// ---------------------------------------------------------------- build with no host reads
// The level-synchronous build numbers the nodes level by level, each level in
// key order.  The same numbering follows from the sorted keys alone: with
// pfx_L(k) = k >> 3 (21 - L) the level-L prefix, the node (L, P) exists iff
// L = 0 or its parent prefix at level L - 1 holds more than leaf_size
// particles (then every ancestor holds more too, so all of them split), and
// it is flagged at the sorted position of its first particle.  The flags of
// all levels, laid out level-major ([L n + i], 22 n entries and a terminal
// 0), are scanned: the scan is the node number, scan[L n] the first node of
// level L, scan[22 n] the node count.

__device__ __forceinline__ uint64_t pfx(uint64_t key, int L) { return key >> (3 * (MORTON_BITS - L)); }

// first sorted position in [0, hi] whose level-L prefix equals P
__device__ __forceinline__ int64_t prefix_begin(const uint64_t* keys, int64_t hi, int L, uint64_t P) {
  int64_t lo = 0;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (pfx(keys[mid], L) < P) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// one past the last sorted position in [lo, n) whose level-L prefix equals P
__device__ __forceinline__ int64_t prefix_end(const uint64_t* keys, int64_t lo, int64_t n, int L, uint64_t P) {
  int64_t hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (pfx(keys[mid], L) <= P) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The levels at which sorted position i starts a node: d = the shallowest
// level where its prefix differs from position i - 1's (22: none); from d on
// it starts a node while the enclosing node one level up splits.  Calls
// visit(L, lo) for each, lo being the first position of the parent node.
template <typename F>
__device__ __forceinline__ void node_starts(const uint64_t* __restrict__ keys, int64_t n, int64_t i, int leaf,
                                            F visit) {
  const uint64_t k = keys[i];
  int d = 0;
  if (i > 0) {
    const uint64_t x = keys[i - 1] ^ k;
    d = x == 0 ? MORTON_BITS + 1 : MORTON_BITS - (63 - __clzll((long long)x)) / 3;
  }
  if (d > MORTON_BITS) return;
  // the parent of the level-d node starts before i (unless d = 0)
  const int64_t lo_d = d == 0 ? 0 : prefix_begin(keys, i, d - 1, pfx(k, d - 1));
  for (int L = d; L <= MORTON_BITS; ++L) {
    if (L > 0) {
      const int64_t lo = L - 1 >= d ? i : lo_d;  // first position of the parent
      if (!(lo + leaf < n && pfx(keys[lo + leaf], L - 1) == pfx(k, L - 1))) return;  // parent is a leaf
    }
    visit(L, L == 0 ? (int64_t)-1 : (L - 1 >= d ? i : lo_d));
  }
}

__global__ void tree_flags(int64_t n, const uint64_t* __restrict__ keys, int leaf, int32_t* __restrict__ flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int L = 0; L <= MORTON_BITS; ++L) flags[L * n + i] = 0;
    node_starts(keys, n, i, leaf, [&](int L, int64_t) { flags[L * n + i] = 1; });
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) flags[(int64_t)(MORTON_BITS + 1) * n] = 0;
}

// the node records from the scanned flags (id = scan[L n + i])
__global__ void tree_fill(int64_t n, const uint64_t* __restrict__ keys, int leaf, const int32_t* __restrict__ scan,
                          int64_t* nb, int64_t* ne, int32_t* lev, int64_t* label, int64_t* first_child,
                          int32_t* nchild, int32_t* parent) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t k = keys[i];
    node_starts(keys, n, i, leaf, [&](int L, int64_t lo_parent) {
      const int64_t id = scan[L * n + i];
      const int64_t e = prefix_end(keys, i, n, L, pfx(k, L));
      nb[id] = i;
      ne[id] = e;
      lev[id] = L;
      label[id] = (int64_t)((1ULL << (3 * L)) | pfx(k, L));
      parent[id] = L == 0 ? -1 : scan[(L - 1) * n + lo_parent];
      if (e - i > leaf && L < MORTON_BITS) {
        const int64_t f = scan[(L + 1) * n + i];
        first_child[id] = f;
        nchild[id] = (int32_t)(scan[(L + 1) * n + e] - f);
      } else {
        first_child[id] = -1;
        nchild[id] = 0;
      }
    });
  }
}

// bottom-up sums of one level whose node range is read on the device
__global__ void node_sums_level(int L, int64_t n, const int32_t* __restrict__ scan, const int64_t* __restrict__ nb,
                                const int64_t* __restrict__ ne, const int64_t* __restrict__ fc,
                                const int32_t* __restrict__ nch, const double* __restrict__ xs,
                                const double* __restrict__ ys, const double* __restrict__ zs,
                                const double* __restrict__ ms, const double* __restrict__ hs, double* mass,
                                double* msum, unsigned long long* hmax_bits, unsigned long long* bbox,
                                int32_t* owner) {
  const int64_t lb = scan[L * n], le = scan[(L + 1) * n];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = lb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < le; i += stride)
    node_sum_one(i, nb, ne, fc, nch, xs, ys, zs, ms, hs, mass, msum, hmax_bits, bbox, owner);
}

__global__ void node_com_box(int64_t n, const int32_t* __restrict__ scan, const double* __restrict__ mass,
                             const double* __restrict__ msum, double* com, unsigned long long* size_bits,
                             const unsigned long long* __restrict__ bbox, const unsigned long long* __restrict__ hmax,
                             const int64_t* __restrict__ fc, const int32_t* __restrict__ nch, float* box32) {
  const int64_t nn = scan[(int64_t)(MORTON_BITS + 1) * n];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    const double M = mass[i];
    com[3 * i] = msum[3 * i] / M;
    com[3 * i + 1] = msum[3 * i + 1] / M;
    com[3 * i + 2] = msum[3 * i + 2] / M;
    size_bits[i] = 0ULL;
    for (int k = 0; k < 3; ++k) {
      box32[8 * i + k] = __double2float_rd(bitsd(bbox[6 * i + k]));
      box32[8 * i + 3 + k] = __double2float_ru(bitsd(bbox[6 * i + 3 + k]));
    }
    box32[8 * i + 6] = __double2float_ru(bitsd(hmax[i]));
    const int nc = nch[i];
    const int64_t f = fc[i];
    const unsigned link = nc == 0 ? 0u : (f < (1LL << 28) ? ((unsigned)f << 4) | (unsigned)nc : NODE_LINK_FAR);
    box32[8 * i + 7] = __uint_as_float(link);
  }
}


}  // namespace

// ---------------------------------------------------------------- tree build

static int grow_nodes(map_ctx* ctx, int64_t need) {
  DevTree& T = ctx->tree;
  // node arrays live in ws_tree[8..19]; growing keeps the old contents
  struct Arr { int slot; size_t esz; void** p; };
  Arr arrs[] = {{8, sizeof(int64_t), (void**)&T.label},      {9, sizeof(int32_t), (void**)&T.level},
                {10, sizeof(int64_t), (void**)&T.begin},     {11, sizeof(int64_t), (void**)&T.end},
                {12, sizeof(int64_t), (void**)&T.first_child}, {13, sizeof(int32_t), (void**)&T.nchild},
                {14, sizeof(int32_t), (void**)&T.parent},    {15, sizeof(double), (void**)&T.mass},
                {16, 3 * sizeof(double), (void**)&T.com},    {17, sizeof(unsigned long long), (void**)&T.size_bits},
                {18, sizeof(unsigned long long), (void**)&T.hmax_bits},
                {19, 6 * sizeof(unsigned long long), (void**)&T.bbox_bits}};
  for (auto& a : arrs) {
    DevBuf& b = ctx->ws_tree[a.slot];
    size_t bytes = (size_t)need * a.esz;
    if (b.cap >= bytes) { *a.p = b.p; continue; }
    size_t nb = bytes + bytes / 2 + 4096;
    if (ctx->cfg.hbm_budget && ctx->bytes_in_use + nb > ctx->cfg.hbm_budget) return MAP_ENOMEM;
    void* np = nullptr;
    MAP_TRY(dev_alloc(ctx, &np, nb));
    ctx->bytes_in_use += nb;
    if (b.p) {
      CUDA_TRY(cudaMemcpyAsync(np, b.p, b.cap, cudaMemcpyDeviceToDevice, ctx->cur_stream));
      dev_free(ctx, b.p);
      ctx->bytes_in_use -= b.cap;
    }
    b.p = np;
    b.cap = nb;
    *a.p = np;
  }
  return MAP_OK;
}

int tree_build(map_ctx* ctx, const double* x, const double* y, const double* z, const double* m, const double* h,
               int64_t n, cudaStream_t s, bool want_size) {
  DevTree& T = ctx->tree;
  T.n = n;
  const int tpb = 256;
  uint64_t* keys_in;
  int32_t* idx_in;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[0], n, &keys_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[1], n, &idx_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[2], n, &T.keys));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[3], n, &T.idx));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[4], 5 * n, &T.xs));
  T.ys = T.xs + n; T.zs = T.xs + 2 * n; T.ms = T.xs + 3 * n; T.hs = T.xs + 4 * n;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[5], n, &T.owner));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[23], 6 * n, &T.split));
  T.hs32 = nullptr;
  if (h) MAP_TRY(ensure_t(ctx, ctx->ws_tree[27], n, &T.hs32));
  morton_keys<<<nblk(n, tpb), tpb, 0, s>>>(n, x, y, z, keys_in, idx_in); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t tmp_bytes = 0;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, T.keys, idx_in, T.idx, n, 0, 63, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tmp_bytes));
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tmp_bytes, keys_in, T.keys, idx_in, T.idx, n, 0, 63, s));
  gather_sorted<<<nblk(n, tpb), tpb, 0, s>>>(n, T.idx, x, y, z, m, h, T.xs, T.ys, T.zs, T.ms, T.hs, T.split,
                                             T.hs32); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());

  // level-synchronous build
  int64_t cap = n / 4 + 64;
  if (ctx->node_cap0 > cap) cap = ctx->node_cap0;  // node arrays sized up front (fixed-workspace contexts)
  MAP_TRY(grow_nodes(ctx, cap));
  int64_t root_label = 1, zero = 0;
  int32_t root_level = 0, root_parent = -1;
  CUDA_TRY(cudaMemcpyAsync(T.label, &root_label, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(T.level, &root_level, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(T.begin, &zero, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(T.end, &n, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(T.parent, &root_parent, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  T.level_begin.assign(1, 0);
  int64_t lb = 0, le = 1;
  while (le > lb) {
    T.level_begin.push_back(le);
    int64_t nf = le - lb;
    int32_t* nchild;
    int64_t* choff;
    MAP_TRY(ensure_t(ctx, ctx->ws_tree[6], nf + 1, &nchild));
    MAP_TRY(ensure_t(ctx, ctx->ws_tree[7], nf + 1, &choff));
    split_count<<<nblk(nf, tpb), tpb, 0, s>>>(lb, le, T.keys, T.begin, T.end, T.level, ctx->cfg.leaf_size, nchild); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    size_t sb = 0;
    CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, sb, nchild, choff, nf + 1, s));
    MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, sb));
    // the (nf+1)-th entry of nchild is set to 0 so that choff[nf] is the total
    CUDA_TRY(cudaMemsetAsync(nchild + nf, 0, sizeof(int32_t), s));
    CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, sb, nchild, choff, nf + 1, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, choff + nf, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    int64_t nnew = ctx->h_scratch[0];
    if (le + nnew > cap) {
      cap = (le + nnew) * 2;
      MAP_TRY(grow_nodes(ctx, cap));
    }
    split_write<<<nblk(nf, tpb), tpb, 0, s>>>(lb, le, le, T.keys, T.begin, T.end, T.level, T.label, T.first_child,
                                             T.nchild, T.parent, nchild, choff); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    lb = le;
    le = le + nnew;
  }
  T.nnodes = le;
  T.nlevels = (int)T.level_begin.size() - 1;
  // bottom-up sums, deepest level first
  double* msum;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[20], 3 * T.nnodes, &msum));
  for (int L = T.nlevels - 1; L >= 0; --L) {
    int64_t a = T.level_begin[L], b = T.level_begin[L + 1];
    node_sums<<<nblk(b - a, tpb), tpb, 0, s>>>(a, b, T.begin, T.end, T.first_child, T.nchild, T.xs, T.ys, T.zs,
                                               T.ms, T.hs, T.mass, msum, T.hmax_bits, T.bbox_bits, T.owner);
    ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  }
  node_com<<<nblk(T.nnodes, tpb), tpb, 0, s>>>(T.nnodes, T.mass, msum, T.com, T.size_bits); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  if (want_size) {
    node_extent_small<<<nblk(n, tpb), tpb, 0, s>>>(n, T.owner, T.parent, T.begin, T.end, T.xs, T.ys, T.zs, T.com,
                                                   T.size_bits); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    int32_t* big;
    MAP_TRY(ensure_t(ctx, ctx->ws_tree[21], T.nnodes, &big));
    unsigned long long* d_nbig = ctx->d_counters + 4;
    CUDA_TRY(cudaMemsetAsync(d_nbig, 0, sizeof(unsigned long long), s));
    collect_big<<<nblk(T.nnodes, tpb), tpb, 0, s>>>(T.nnodes, T.begin, T.end, big, d_nbig); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, d_nbig, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nbig = ctx->h_scratch[0];
    if (nbig > 0) {
      const int slices = 32;
      node_extent_big<<<(unsigned)(nbig * slices), 256, 0, s>>>(big, slices, T.begin, T.end, T.xs, T.ys, T.zs,
                                                                T.com, T.size_bits); ++ctx->launches;
      CUDA_TRY(cudaGetLastError());
    }
  }
  float* box32;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[24], 8 * T.nnodes, &box32));
  T.box32 = box32;
  node_box32<<<nblk(T.nnodes, tpb), tpb, 0, s>>>(T.nnodes, T.bbox_bits, T.hmax_bits, T.first_child, T.nchild,
                                                 box32); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

// ---------------------------------------------------------------- tree build with no host reads

int64_t tree_nodes_max(int64_t n, int leaf_size) {
  // internal nodes of one level hold disjoint sets of more than leaf_size
  // particles, so each level has at most n / (leaf_size + 1) of them (21
  // levels split); every leaf holds at least one particle; plus the root
  const int64_t per_level = n / ((int64_t)(leaf_size > 0 ? leaf_size : 0) + 1);
  return n + (int64_t)MORTON_BITS * per_level + 64;
}

int tree_build_graph(map_ctx* ctx, const double* x, const double* y, const double* z, const double* m,
                     const double* h, int64_t n, cudaStream_t s) {
  DevTree& T = ctx->tree;
  T.n = n;
  const int tpb = 256;
  const int leaf = ctx->cfg.leaf_size;
  uint64_t* keys_in;
  int32_t* idx_in;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[0], n, &keys_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[1], n, &idx_in));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[2], n, &T.keys));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[3], n, &T.idx));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[4], 5 * n, &T.xs));
  T.ys = T.xs + n; T.zs = T.xs + 2 * n; T.ms = T.xs + 3 * n; T.hs = T.xs + 4 * n;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[5], n, &T.owner));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[23], 6 * n, &T.split));
  T.hs32 = nullptr;
  if (h) MAP_TRY(ensure_t(ctx, ctx->ws_tree[27], n, &T.hs32));
  morton_keys<<<nblk(n, tpb), tpb, 0, s>>>(n, x, y, z, keys_in, idx_in); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t tmp_bytes = 0;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, T.keys, idx_in, T.idx, n, 0, 63, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tmp_bytes));
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tmp_bytes, keys_in, T.keys, idx_in, T.idx, n, 0, 63, s));
  gather_sorted<<<nblk(n, tpb), tpb, 0, s>>>(n, T.idx, x, y, z, m, h, T.xs, T.ys, T.zs, T.ms, T.hs, T.split,
                                             T.hs32); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());

  // node flags of every level, their scan, the node records
  const int64_t nflag = (int64_t)(MORTON_BITS + 1) * n + 1;
  if (nflag >= (int64_t)INT32_MAX) return MAP_ECAPACITY;
  int32_t *flags, *scan;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[25], nflag, &flags));
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[26], nflag, &scan));
  const int64_t cap = tree_nodes_max(n, leaf);
  MAP_TRY(grow_nodes(ctx, cap));
  const unsigned g = (unsigned)(ctx->sm_count * 8);
  tree_flags<<<g, tpb, 0, s>>>(n, T.keys, leaf, flags); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t sb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, sb, flags, scan, (int)nflag, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, sb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, sb, flags, scan, (int)nflag, s));
  tree_fill<<<g, tpb, 0, s>>>(n, T.keys, leaf, scan, T.begin, T.end, T.level, T.label, T.first_child, T.nchild,
                             T.parent); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  // bottom-up sums, deepest level first (empty levels launch and return)
  double* msum;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[20], 3 * cap, &msum));
  for (int L = MORTON_BITS; L >= 0; --L) {
    node_sums_level<<<g, tpb, 0, s>>>(L, n, scan, T.begin, T.end, T.first_child, T.nchild, T.xs, T.ys, T.zs, T.ms,
                                      T.hs, T.mass, msum, T.hmax_bits, T.bbox_bits, T.owner); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  }
  float* box32;
  MAP_TRY(ensure_t(ctx, ctx->ws_tree[24], 8 * cap, &box32));
  T.box32 = box32;
  node_com_box<<<g, tpb, 0, s>>>(n, scan, T.mass, msum, T.com, T.size_bits, T.bbox_bits, T.hmax_bits, T.first_child,
                                 T.nchild, box32); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  // host-side sizes are unknown without a read: an upper bound, no levels
  T.nnodes = cap;
  T.nlevels = MORTON_BITS + 1;
  T.level_begin.clear();
  return MAP_OK;
}
