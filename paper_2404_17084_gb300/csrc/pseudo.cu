// Pseudo-particles (Section III-A/B) and their smoothing lengths (Section III-C/D).
//
// Walk (Eq. 5): a node is opened when r_node = 0 or s_node^2 > theta^2 r_node^2,
// r_node being the distance from its centre of mass to the nearest source, or
// when one of the walk controls of Section III-B asks for it (r_part, r_leaf,
// regions of an earlier step; see the opening rule below).  A
// node is reached when all its ancestors are opened; reached nodes that are
// not opened become pseudo-particles (centre of mass, node mass); reached
// leaves that are opened yield their particles, which keep their h.  Because
// every node is a contiguous range of the Morton-sorted particles, the
// accepted nodes and extracted particles partition that order, and listing
// them by first sorted position is the depth-first order of the walk.
//
// h of the accepted nodes: h = hfact n^(-1/3), n = sum_b W(r_ab, h) over the
// node set (accepted nodes plus opened leaves standing in for their
// particles), initial guess hfact * 2 s_node (Eq. 9; a node of size 0 starts
// from its first particle's h).  Candidates are all members when there are at
// most ngb_bruteforce_max of them (Section III-D), otherwise the members whose
// ancestor on level k_mid (one level above the highest member) lies within
// r_cut of the target, r_cut = sqrt(3) s_mid, replaced by 4 hfact s_above
// (s_above: the target's ancestor two levels up) when that is larger (Eq. 10).
#include <cub/cub.cuh>

#include "internal.cuh"

namespace {


constexpr int64_t KIND_PARTICLE = (int64_t)1 << 62;

// Opening rule of the walk (Eq. 5 and the controls of Section III-B), every
// distance compared squared with each product and sum rounded once.
struct WalkRule {
  const double* src;  // 3 per source
  int nsrc;
  double theta, r_part, r_leaf;
  const double* reg;  // 5 per region: centre, radius, smallest size
  int nreg;
};

__device__ __forceinline__ double sq3(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__global__ void open_flags(int64_t nn, const double* __restrict__ com, const unsigned long long* __restrict__ size_bits,
                           const int32_t* __restrict__ nchild, WalkRule R, int8_t* open) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double s = bitsd(size_bits[i]);
  const bool leaf = nchild[i] == 0;
  const double s2 = __dmul_rn(s, s), th2 = __dmul_rn(R.theta, R.theta);
  const double tp = __dadd_rn(R.r_part, s), tl = __dadd_rn(R.r_leaf, s);
  const double tp2 = __dmul_rn(tp, tp), tl2 = __dmul_rn(tl, tl);
  const double cx = com[3 * i], cy = com[3 * i + 1], cz = com[3 * i + 2];
  bool op = false;
  for (int k = 0; k < R.nsrc; ++k) {
    const double r2 = sq3(__dsub_rn(cx, R.src[3 * k]), __dsub_rn(cy, R.src[3 * k + 1]), __dsub_rn(cz, R.src[3 * k + 2]));
    if (r2 == 0.0 || s2 > __dmul_rn(th2, r2)) op = true;
    else if (R.r_part > 0.0 && r2 < tp2) op = true;
    else if (!leaf && R.r_leaf > 0.0 && r2 < tl2) op = true;
  }
  for (int k = 0; k < R.nreg; ++k) {
    const double* g = R.reg + 5 * k;
    const double d2 = sq3(__dsub_rn(cx, g[0]), __dsub_rn(cy, g[1]), __dsub_rn(cz, g[2]));
    if (d2 < __dmul_rn(g[3], g[3]) && s > g[4]) op = true;
  }
  open[i] = op ? 1 : 0;
}

// Status per node: 0 not reached / opened internal, 1 accepted, 2 opened leaf.
__global__ void walk_status(int64_t nn, const int32_t* __restrict__ parent, const int8_t* __restrict__ open,
                            const int32_t* __restrict__ nchild, int8_t* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  bool reached = true;
  for (int32_t a = parent[i]; a >= 0; a = parent[a])
    if (!open[a]) { reached = false; break; }
  int8_t st = 0;
  if (reached) {
    if (!open[i]) st = 1;
    else if (nchild[i] == 0) st = 2;
  }
  status[i] = st;
}

__global__ void mark_heads(int64_t nn, const int8_t* __restrict__ status, const int64_t* __restrict__ nb,
                           const int64_t* __restrict__ ne, int64_t* head, int32_t* is_head) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  if (status[i] == 1) {
    head[nb[i]] = i;
    is_head[nb[i]] = 1;
  } else if (status[i] == 2) {
    for (int64_t p = nb[i]; p < ne[i]; ++p) {
      head[p] = KIND_PARTICLE | p;
      is_head[p] = 1;
    }
  }
}

__global__ void write_pseudo(int64_t n, const int64_t* __restrict__ head, const int32_t* __restrict__ is_head,
                             const int64_t* __restrict__ slot, const double* __restrict__ com,
                             const double* __restrict__ mass, const int64_t* __restrict__ label,
                             const double* __restrict__ xs, const double* __restrict__ ys, const double* __restrict__ zs,
                             const double* __restrict__ ms, const double* __restrict__ hs,
                             const int32_t* __restrict__ idx, double* ox, double* oy, double* oz, double* om, double* oh,
                             int32_t* kind, int64_t* ident, int32_t* node_of_slot) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n || !is_head[p]) return;
  const int64_t j = slot[p];
  const int64_t hd = head[p];
  if (hd & KIND_PARTICLE) {
    const int64_t q = hd & (KIND_PARTICLE - 1);
    ox[j] = xs[q]; oy[j] = ys[q]; oz[j] = zs[q]; om[j] = ms[q]; oh[j] = hs[q];
    if (kind) kind[j] = 1;
    if (ident) ident[j] = idx[q];
    node_of_slot[j] = -1;
  } else {
    ox[j] = com[3 * hd]; oy[j] = com[3 * hd + 1]; oz[j] = com[3 * hd + 2]; om[j] = mass[hd]; oh[j] = 0.0;
    if (kind) kind[j] = 0;
    if (ident) ident[j] = label[hd];
    node_of_slot[j] = (int32_t)hd;
  }
}

// The node set for the h solve: accepted nodes and opened leaves, in node order.
__global__ void member_flags(int64_t nn, const int8_t* __restrict__ status, int32_t* flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  flag[i] = status[i] != 0 ? 1 : 0;
}

__global__ void member_write(int64_t nn, const int32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                             int32_t* members) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn || !flag[i]) return;
  members[pos[i]] = (int32_t)i;
}

__device__ __forceinline__ double w_m4(double q) {
  if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
  if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
  return 0.0;
}
__device__ __forceinline__ double dw_m4(double q) {
  if (q < 1.0) return -3.0 * q + 2.25 * q * q;
  if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
  return 0.0;
}

struct NodeSet {
  int64_t nm;                 // members
  const int32_t* members;     // node ids
  const double* com;          // node centre of mass (3 per node)
  // k_mid candidates (used when use_kmid)
  int use_kmid;
  int64_t mid_begin, mid_end; // node id range of level k_mid
  const int64_t* mid_off;     // per mid node: member range in mid_sorted (size nmid+1)
  const int32_t* mid_sorted;  // members grouped by their k_mid ancestor
};

__device__ __forceinline__ void acc_member(const double* com, int32_t b, double x, double y, double z, double R2,
                                           double inv_h, double& s, double& ds) {
  const double dx = com[3 * b] - x, dy = com[3 * b + 1] - y, dz = com[3 * b + 2] - z;
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (r2 >= R2) return;
  const double q = sqrt(r2) * inv_h;
  const double w = w_m4(q);
  s += w;
  ds += 3.0 * w + q * dw_m4(q);
}

// n(h) and dn/dh at (x, y, z) over the candidates, summed by the 32 lanes of
// a warp (strided over the members or the level-k_mid nodes) and combined by
// a butterfly reduction, so that every lane holds the same sums.
__device__ void set_density(const NodeSet& S, int lane, double x, double y, double z, double rcut, double h, double& n,
                            double& dn) {
  const double R2 = 4.0 * h * h, inv_h = 1.0 / h, norm = 1.0 / (MAP_PI * h * h * h);
  double s = 0.0, ds = 0.0;
  if (!S.use_kmid) {
    for (int64_t j = lane; j < S.nm; j += 32) acc_member(S.com, S.members[j], x, y, z, R2, inv_h, s, ds);
  } else {
    // the lanes test 32 level-k_mid nodes at a time, then share out the
    // members of each flagged one
    const double rc2 = rcut * rcut;
    for (int64_t m0 = S.mid_begin; m0 < S.mid_end; m0 += 32) {
      const int64_t m = m0 + lane;
      bool flag = false;
      if (m < S.mid_end) {
        const double dx = S.com[3 * m] - x, dy = S.com[3 * m + 1] - y, dz = S.com[3 * m + 2] - z;
        flag = dx * dx + dy * dy + dz * dz < rc2;
      }
      for (unsigned bal = __ballot_sync(0xffffffffu, flag); bal; bal &= bal - 1) {
        const int64_t k = m0 + (__ffs(bal) - 1) - S.mid_begin;
        for (int64_t j = S.mid_off[k] + lane; j < S.mid_off[k + 1]; j += 32)
          acc_member(S.com, S.mid_sorted[j], x, y, z, R2, inv_h, s, ds);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    ds += __shfl_xor_sync(0xffffffffu, ds, o);
  }
  n = s * norm;
  dn = -ds * norm * inv_h;
}

// One warp per output slot holding an accepted node: Newton-Raphson on
// h = hfact n(h)^(-1/3) from Eq. (9)'s guess, bisection on [h0/16, 16 h0]
// when it fails, the guess itself when that has no sign change (Section
// III-C).  The lanes hold identical sums, so the iteration is warp-uniform.
__global__ void pseudo_h(int64_t nout, const int32_t* __restrict__ node_of_slot, NodeSet S,
                         const unsigned long long* __restrict__ size_bits, const int32_t* __restrict__ parent,
                         const int32_t* __restrict__ level, const int64_t* __restrict__ nb, const double* __restrict__ hs,
                         int kmid, double hfact, double* oh) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= nout) return;
  const int32_t nd = node_of_slot[j];
  if (nd < 0) return;  // extracted particle keeps its h
  const double x = S.com[3 * nd], y = S.com[3 * nd + 1], z = S.com[3 * nd + 2];
  const double s_node = bitsd(size_bits[nd]);
  const double g0 = s_node > 0.0 ? hfact * 2.0 * s_node : hs[nb[nd]];
  double rcut = 0.0;
  if (S.use_kmid) {
    int32_t a = nd;
    while (level[a] > kmid) a = parent[a];
    rcut = 1.7320508075688772 * bitsd(size_bits[a]);
    const double r2h = 4.0 * hfact * s_node;
    if (rcut < r2h) {
      int32_t up = nd;
      for (int k = 0; k < 2 && parent[up] >= 0; ++k) up = parent[up];
      rcut = 4.0 * hfact * bitsd(size_bits[up]);
    }
  }
  const double lo = g0 / 16.0, hi = g0 * 16.0;
  double h = g0;
  bool ok = false;
  for (int it = 0; it < 30; ++it) {
    double nn, dn;
    set_density(S, lane, x, y, z, rcut, h, nn, dn);
    const double f = h - hfact * pow(nn, -1.0 / 3.0);
    const double fp = 1.0 + hfact / 3.0 * pow(nn, -4.0 / 3.0) * dn;
    const double hn = h - f / fp;
    if (!(hn >= lo && hn <= hi)) break;
    if (fabs(hn - h) < 1e-10 * hn) { h = hn; ok = true; break; }
    h = hn;
  }
  if (!ok) {
    double nn, dn;
    set_density(S, lane, x, y, z, rcut, lo, nn, dn);
    const double flo = lo - hfact * pow(nn, -1.0 / 3.0);
    set_density(S, lane, x, y, z, rcut, hi, nn, dn);
    const double fhi = hi - hfact * pow(nn, -1.0 / 3.0);
    if (!(flo < 0.0 && fhi > 0.0)) {
      h = g0;
    } else {
      double a0 = lo, b0 = hi;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (a0 + b0);
        set_density(S, lane, x, y, z, rcut, mid, nn, dn);
        if (mid - hfact * pow(nn, -1.0 / 3.0) < 0.0) a0 = mid; else b0 = mid;
        if (b0 - a0 < 1e-12 * mid) break;
      }
      h = 0.5 * (a0 + b0);
    }
  }
  if (lane == 0) oh[j] = h;
}

__global__ void member_anc(int64_t nm, const int32_t* __restrict__ members, const int32_t* __restrict__ parent,
                           const int32_t* __restrict__ level, int kmid, int64_t mid_begin, uint64_t* key, int32_t* val) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nm) return;
  int32_t a = members[j];
  while (level[a] > kmid) a = parent[a];
  key[j] = (uint64_t)(a - mid_begin);
  val[j] = members[j];
}

__global__ void mid_ranges(int64_t nm, int64_t nmid, const uint64_t* __restrict__ key_sorted, int64_t* off) {
  // off[k] = first j with key >= k (lower bound), for k in [0, nmid]
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k > nmid) return;
  int64_t lo = 0, hi = nm;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if (key_sorted[m] < (uint64_t)k) lo = m + 1; else hi = m;
  }
  off[k] = lo;
}

__global__ void min_member_level(int64_t nm, const int32_t* __restrict__ members, const int32_t* __restrict__ level,
                                 unsigned long long* out) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nm) return;
  atomicMin(out, (unsigned long long)level[members[j]]);
}

}  // namespace

int pseudo_run(map_ctx* ctx, const map_particles* full, const map_walk* walk, map_particles* out, int32_t* kind,
               int64_t* ident, int64_t* n_pseudo, cudaStream_t s) {
  const int nsrc = walk->nsrc, nreg = walk->nregion;
  const int64_t n = full->n;
  MAP_TRY(tree_build(ctx, full->x, full->y, full->z, full->m, full->h, n, s, true));
  DevTree& T = ctx->tree;
  const int64_t nn = T.nnodes;
  const int tpb = 256;
  double* d_src;
  int8_t *open, *status;
  int64_t *head, *slot, *mpos;
  int32_t *is_head, *node_of_slot, *mflag, *members;
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[1], 3 * nsrc + 5 * nreg, &d_src));
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[2], 2 * nn, &open));
  status = open + nn;
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[3], 2 * (n + 1), &head));
  slot = head + (n + 1);
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[4], 2 * (n + 1), &is_head));
  node_of_slot = is_head + (n + 1);
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[5], 2 * (nn + 1), &mflag));
  members = mflag + (nn + 1);
  MAP_TRY(ensure_t(ctx, ctx->ws_misc[6], nn + 1, &mpos));
  CUDA_TRY(cudaMemcpyAsync(d_src, walk->src, 3 * nsrc * sizeof(double), cudaMemcpyHostToDevice, s));
  if (nreg > 0)
    CUDA_TRY(cudaMemcpyAsync(d_src + 3 * nsrc, walk->regions, 5 * nreg * sizeof(double), cudaMemcpyHostToDevice, s));
  const WalkRule rule{d_src, nsrc, ctx->cfg.theta, walk->r_part, walk->r_leaf, d_src + 3 * nsrc, nreg};
  open_flags<<<nblk(nn, tpb), tpb, 0, s>>>(nn, T.com, T.size_bits, T.nchild, rule, open); ++ctx->launches;
  walk_status<<<nblk(nn, tpb), tpb, 0, s>>>(nn, T.parent, open, T.nchild, status); ++ctx->launches;
  CUDA_TRY(cudaMemsetAsync(is_head, 0, (n + 1) * sizeof(int32_t), s));
  mark_heads<<<nblk(nn, tpb), tpb, 0, s>>>(nn, status, T.begin, T.end, head, is_head); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  size_t tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, is_head, slot, n + 1, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, is_head, slot, n + 1, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, slot + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nout = ctx->h_scratch[0];
  *n_pseudo = nout;
  if (nout > out->n) return MAP_ECAPACITY;
  if (!out->x || !out->y || !out->z || !out->h) return MAP_EINVAL;
  double* om = const_cast<double*>(out->m);
  if (!om) return MAP_EINVAL;
  write_pseudo<<<nblk(n, tpb), tpb, 0, s>>>(n, head, is_head, slot, T.com, T.mass, T.label, T.xs, T.ys, T.zs, T.ms,
                                           T.hs, T.idx, const_cast<double*>(out->x), const_cast<double*>(out->y),
                                           const_cast<double*>(out->z), om, out->h, kind, ident, node_of_slot); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  // node set for the h solve
  member_flags<<<nblk(nn, tpb), tpb, 0, s>>>(nn, status, mflag); ++ctx->launches;
  CUDA_TRY(cudaMemsetAsync(mflag + nn, 0, sizeof(int32_t), s));
  tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, mflag, mpos, nn + 1, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, mflag, mpos, nn + 1, s));
  member_write<<<nblk(nn, tpb), tpb, 0, s>>>(nn, mflag, mpos, members); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, mpos + nn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nm = ctx->h_scratch[0];
  NodeSet S{};
  S.nm = nm;
  S.members = members;
  S.com = T.com;
  S.use_kmid = nm > ctx->cfg.ngb_bruteforce_max ? 1 : 0;
  int kmid = 0;
  if (S.use_kmid) {
    unsigned long long* d_min = ctx->d_counters + 5;
    unsigned long long big = 1ULL << 40;
    CUDA_TRY(cudaMemcpyAsync(d_min, &big, sizeof(big), cudaMemcpyHostToDevice, s));
    min_member_level<<<nblk(nm, tpb), tpb, 0, s>>>(nm, members, T.level, d_min); ++ctx->launches;
    CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, d_min, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    kmid = (int)ctx->h_scratch[0] - 1;
    if (kmid < 0) kmid = 0;
    S.mid_begin = T.level_begin[kmid];
    S.mid_end = T.level_begin[kmid + 1];
    const int64_t nmid = S.mid_end - S.mid_begin;
    uint64_t *kin, *kout;
    int32_t *vin, *vout;
    int64_t* moff;
    MAP_TRY(ensure_t(ctx, ctx->ws_pairs[4], nm, &kin));
    MAP_TRY(ensure_t(ctx, ctx->ws_pairs[5], nm, &kout));
    MAP_TRY(ensure_t(ctx, ctx->ws_pairs[6], nm, &vin));
    MAP_TRY(ensure_t(ctx, ctx->ws_pairs[7], nm, &vout));
    MAP_TRY(ensure_t(ctx, ctx->ws_misc[7], nmid + 1, &moff));
    member_anc<<<nblk(nm, tpb), tpb, 0, s>>>(nm, members, T.parent, T.level, kmid, S.mid_begin, kin, vin); ++ctx->launches;
    tb = 0;
    CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, vout, nm, 0, 40, s));
    MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
    CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tb, kin, kout, vin, vout, nm, 0, 40, s));
    mid_ranges<<<nblk(nmid + 1, tpb), tpb, 0, s>>>(nm, nmid, kout, moff); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    S.mid_off = moff;
    S.mid_sorted = vout;
  }
  pseudo_h<<<nblk(nout * 32, 128), 128, 0, s>>>(nout, node_of_slot, S, T.size_bits, T.parent, T.level, T.begin, T.hs,
                                           kmid, ctx->cfg.hfact, out->h); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}
