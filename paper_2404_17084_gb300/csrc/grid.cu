// Grid upload: copy the CSR grid into context memory and precompute, per cell,
// the site-relative face planes and the per-edge records the pair-integral
// kernels read (Section II-B's r0, R0 and phi are affine in the particle
// position once these are known), a bounding sphere per face (centre
// site-relative, radius rounded up: a face whose sphere lies beyond a
// particle's support contributes nothing), plus the cell volume (divergence
// theorem) and the cell radius R_i used by the pair rule.
#include <cstring>

#include "internal.cuh"

namespace {

// Face -> cell map (one thread per cell).
__global__ void face_cells(int64_t ncell, const int64_t* __restrict__ cfo, int32_t* fcell) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  for (int64_t f = cfo[c]; f < cfo[c + 1]; ++f) fcell[f] = (int32_t)c;
}

// FP32 copies of the vertex coordinates, for the face spheres' centres.
__global__ void vert32(int64_t nv, const double* __restrict__ vx, const double* __restrict__ vy,
                       const double* __restrict__ vz, float4* v32) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nv) v32[k] = make_float4((float)vx[k], (float)vy[k], (float)vz[k], 0.f);
}

// One thread per face: site-relative planes, the face's bounding sphere and
// edge records, its term dr * area / 3 of the cell volume (divergence
// theorem) and the largest squared vertex distance from the site.  The
// FP64 pipe runs at about 1/74 of the FP32 rate, so FP64 work is kept to the
// site-relative differences, one component of the area sum and the exact
// squares of the few vertices that can be the farthest.
__global__ void prep_faces(int64_t nface, const int32_t* __restrict__ fcell, const int64_t* __restrict__ fvo,
                           const int32_t* __restrict__ fv, const double4_32a* __restrict__ plane,
                           const double* __restrict__ vx, const double* __restrict__ vy,
                           const double* __restrict__ vz, const float4* __restrict__ v32,
                           const double* __restrict__ site, double4_32a* face64,
                           float4* face32, float4* fsph32, double* edge64, float* edge32, double* volf, double* r2f,
                           unsigned long long* status) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nface) return;
  const int64_t c = fcell[f];
  const double sx = site[3 * c], sy = site[3 * c + 1], sz = site[3 * c + 2];
  const double4_32a P = plane[f];
  const double dr = P.w - (P.x * sx + P.y * sy + P.z * sz);
  if (!(dr > 0.0)) atomicExch(status, (unsigned long long)(-MAP_EINVAL));  // site must be strictly inside
  face64[f] = make_double4_32a(P.x, P.y, P.z, dr);
  face32[f] = make_float4((float)P.x, (float)P.y, (float)P.z, (float)dr);
  const int64_t b = fvo[f], e = fvo[f + 1];
  const int64_t L = e - b;
  // site-relative vertices: differences in FP64, FP32 copies for the mixed
  // build's records (their rounding, ~1e-7 of the cell size, is that of
  // rounding an FP64 record)
  // face sphere centre: the vertex mean from the FP32 copies (any centre
  // serves: the radius below is measured from it to the accurate
  // site-relative vertices)
  float mx = 0.f, my = 0.f, mz = 0.f;
  if (fsph32) {
    const float sx32 = (float)sx, sy32 = (float)sy, sz32 = (float)sz;
    for (int64_t k = 0; k < L; ++k) {
      const float4 V = v32[fv[b + k]];
      mx += V.x - sx32; my += V.y - sy32; mz += V.z - sz32;
    }
    const float il = 1.0f / (float)L;
    mx *= il; my *= il; mz *= il;
  }
  // The loop's cross-product sum is 2 area n (a planar loop, unit n): its
  // component on the normal's largest axis, over that normal component,
  // gives the area.
  const double anx = fabs(P.x), any = fabs(P.y), anz = fabs(P.z);
  const int axis = anx >= any && anx >= anz ? 0 : (any >= anz ? 1 : 2);
  const double n_axis = axis == 0 ? P.x : (axis == 1 ? P.y : P.z);
  float sr2 = 0.f;   // FP32 squared sphere radius
  float r2s = 0.f;   // largest FP32 squared vertex distance so far
  double R2 = 0.0;
  double acc = 0.0;
  const int32_t i0 = fv[b];
  const double X0 = vx[i0] - sx, Y0 = vy[i0] - sy, Z0 = vz[i0] - sz;
  double Ax = X0, Ay = Y0, Az = Z0;
  float ax32 = (float)Ax, ay32 = (float)Ay, az32 = (float)Az;
  const float x032 = ax32, y032 = ay32, z032 = az32;
  for (int64_t k = 0; k < L; ++k) {
    double Bx = X0, By = Y0, Bz = Z0;
    float bx32 = x032, by32 = y032, bz32 = z032;
    if (k + 1 < L) {
      const int32_t ib = fv[b + k + 1];
      Bx = vx[ib] - sx; By = vy[ib] - sy; Bz = vz[ib] - sz;
      bx32 = (float)Bx; by32 = (float)By; bz32 = (float)Bz;
    }
    // cell radius: fixed evaluation order, no FMA contraction; one
    // correctly rounded square root of the cell's largest square at the end.
    // Only a vertex whose FP32 square (within 5e-7 of its FP64 one) comes
    // within 1e-5 of the largest so far can be the farthest; the others
    // skip the FP64 square.
    const float q = ax32 * ax32 + ay32 * ay32 + az32 * az32;
    if (q >= r2s * (1.f - 1e-5f)) {
      r2s = fmaxf(r2s, q);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(Ax, Ax), __dmul_rn(Ay, Ay)), __dmul_rn(Az, Az));
      R2 = r2 > R2 ? r2 : R2;
    }
    // area: one component of the site-relative loop's cross-product sum
    acc += axis == 0 ? Ay * Bz - Az * By : (axis == 1 ? Az * Bx - Ax * Bz : Ax * By - Ay * Bx);
    // a zero-length edge gets R0s = m.y - delta*hinv = +huge: it never
    // makes p 'outside' and its r0^2 + R0^2 is beyond the support
    if (edge64) {
      double rec[9];
      edge_record64(P.x, P.y, P.z, dr, Ax, Ay, Az, Bx, By, Bz, rec);
      double* E = edge64 + (b + k) * EDGE_STRIDE;
      for (int j = 0; j < 9; ++j) E[j] = rec[j];
      for (int j = 9; j < EDGE_STRIDE; ++j) E[j] = 0;
    }
    if (edge32) {
      float rec[12];
      float ex = bx32 - ax32, ey = by32 - ay32, ez = bz32 - az32;
      const float len = sqrtf(ex * ex + ey * ey + ez * ez);
      if (len > 0.f) {
        const float il = 1.0f / len;
        ex *= il; ey *= il; ez *= il;
        const float nx = (float)P.x, ny = (float)P.y, nz = (float)P.z;
        const float gx = ny * ez - nz * ey, gy = nz * ex - nx * ez, gz = nx * ey - ny * ex;
        rec[0] = gx; rec[1] = gy; rec[2] = gz;
        rec[3] = gx * ax32 + gy * ay32 + gz * az32;
        rec[4] = ex; rec[5] = ey; rec[6] = ez;
        rec[7] = ex * ax32 + ey * ay32 + ez * az32;
        rec[8] = ex * bx32 + ey * by32 + ez * bz32;
      } else {
        for (int j = 0; j < 9; ++j) rec[j] = 0.f;
        rec[3] = -1e30f;
      }
      rec[9] = rec[10] = rec[11] = 0.f;
      float4* Ef = reinterpret_cast<float4*>(edge32 + (b + k) * EDGE_STRIDE);
      // interleaved: (m.x, t.x, m.y, t.y), (m.z, t.z, a_A, a_B), (delta, 0, 0, 0)
      Ef[0] = make_float4(rec[0], rec[4], rec[1], rec[5]);
      Ef[1] = make_float4(rec[2], rec[6], rec[7], rec[8]);
      Ef[2] = make_float4(rec[3], rec[9], rec[10], rec[11]);
      if (fsph32) {
        const float dx = ax32 - mx, dy = ay32 - my, dz = az32 - mz;
        sr2 = fmaxf(sr2, dx * dx + dy * dy + dz * dz);
      }
    }
    Ax = Bx; Ay = By; Az = Bz;
    ax32 = bx32; ay32 = by32; az32 = bz32;
  }
  // bounding sphere: centre at the vertex mean, radius the largest vertex
  // distance, rounded up (FP32 rounding is far inside the margin)
  if (fsph32) fsph32[f] = make_float4(mx, my, mz, sqrtf(sr2) * (1.0f + 1e-5f) + 1e-12f);
  const double area = 0.5 * acc / n_axis;
  volf[f] = dr * area / 3.0;
  r2f[f] = R2;
}

// One thread per cell: volume (the faces' terms in face order), radius R_i,
// the inscribed radius (the smallest distance from the site to a face
// plane, rounded down to FP32) and the largest face and loop counts.
__global__ void prep_cells(int64_t ncell, const int64_t* __restrict__ cfo, const int64_t* __restrict__ fvo,
                           const double* __restrict__ volf, const double* __restrict__ r2f,
                           const double4_32a* __restrict__ face64, double* vol, double* rad, float* rin, int* maxf,
                           int* maxl) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int64_t f0 = cfo[c], f1 = cfo[c + 1];
  double V = 0.0, R2 = 0.0, dmin = 1e300;
  for (int64_t f = f0; f < f1; ++f) {
    V += volf[f];
    R2 = r2f[f] > R2 ? r2f[f] : R2;
    dmin = face64[f].w < dmin ? face64[f].w : dmin;
  }
  vol[c] = V;
  rad[c] = __dsqrt_rn(R2);
  rin[c] = __double2float_rd(dmin);
  atomicMax(maxf, (int)(f1 - f0));
  atomicMax(maxl, (int)(fvo[f1] - fvo[f0]));
}

// CSR sanity: offsets start at 0, end at the totals, never decrease; every
// face has at least 3 loop entries, every cell at least 4 faces; vertex
// indices in range.  Any violation sets *bad; nothing is indexed with an
// unchecked value.
__global__ void check_csr(int64_t ncell, int64_t nface, int64_t nloop, int64_t nvert, const int64_t* __restrict__ cfo,
                          const int64_t* __restrict__ fvo, const int32_t* __restrict__ fv, unsigned long long* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = i; c < ncell; c += stride) {
    const int64_t a = cfo[c], b = cfo[c + 1];
    if (a < 0 || b > nface || b - a < 4) atomicOr(bad, 1ULL);
  }
  for (int64_t f = i; f < nface; f += stride) {
    const int64_t a = fvo[f], b = fvo[f + 1];
    if (a < 0 || b > nloop || b - a < 3) atomicOr(bad, 2ULL);
  }
  for (int64_t k = i; k < nloop; k += stride) {
    const int32_t v = fv[k];
    if (v < 0 || v >= nvert) atomicOr(bad, 4ULL);
  }
  if (i == 0 && (cfo[0] != 0 || cfo[ncell] != nface || fvo[0] != 0 || fvo[nface] != nloop)) atomicOr(bad, 8ULL);
}

}  // namespace

void grid_recycle(map_ctx* ctx, PreparedGrid* g) {
  for (const DevBuf& b : g->allocs) ctx->grid_pool.push_back(b);
  g->allocs.clear();
  g->bytes = 0;
}

void grid_pool_drop(map_ctx* ctx) {
  for (const DevBuf& b : ctx->grid_pool) {
    dev_free(ctx, b.p);
    ctx->bytes_in_use -= b.cap;
  }
  ctx->grid_pool.clear();
}

// A grid buffer: the smallest pooled buffer of a released grid that holds
// `bytes` (and wastes at most as much again), else a new allocation, after
// freeing the pool if the budget or the device has no room.
int ctx_alloc_grid(map_ctx* ctx, PreparedGrid* g, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  int best = -1;
  for (int i = 0; i < (int)ctx->grid_pool.size(); ++i) {
    const size_t c = ctx->grid_pool[i].cap;
    if (c >= bytes && c <= 2 * bytes + (1u << 20) && (best < 0 || c < ctx->grid_pool[best].cap)) best = i;
  }
  if (best >= 0) {
    const DevBuf b = ctx->grid_pool[best];
    ctx->grid_pool.erase(ctx->grid_pool.begin() + best);
    *p = b.p;
    g->bytes += b.cap;
    g->allocs.push_back(b);
    return MAP_OK;
  }
  if (ctx->cfg.hbm_budget && ctx->bytes_in_use + bytes > ctx->cfg.hbm_budget) grid_pool_drop(ctx);
  if (ctx->cfg.hbm_budget && ctx->bytes_in_use + bytes > ctx->cfg.hbm_budget) return MAP_ENOMEM;
  if (dev_alloc(ctx, p, bytes) != MAP_OK) {
    if (ctx->grid_pool.empty()) return MAP_ENOMEM;
    grid_pool_drop(ctx);
    MAP_TRY(dev_alloc(ctx, p, bytes));
  }
  ctx->bytes_in_use += bytes;
  g->bytes += bytes;
  g->allocs.push_back(DevBuf{*p, bytes});
  return MAP_OK;
}

int grid_prepare(map_ctx* ctx, const map_grid* in, PreparedGrid* g, cudaStream_t s) {
  g->ncell = in->ncell;
  g->nface = in->nface;
  g->nloop = in->nloop;
  g->nvert = in->nvert;
  const int64_t nc = in->ncell, nf = in->nface, nl = in->nloop, nv = in->nvert;
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->cell_face_off, (nc + 1) * sizeof(int64_t)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->face_vert_off, (nf + 1) * sizeof(int64_t)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->face_vert, nl * sizeof(int32_t)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->face_plane, nf * sizeof(double4_32a)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->face64, nf * sizeof(double4_32a)));
  // FP32 faces for the pair rule's screen; then the records a context's
  // integral kernel reads: face spheres and FP32 edges for the mixed build
  // (a face whose plane passes within 1e-4 h of a particle takes its side
  // from face64), FP64 edges for the FP64 build
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->face32, nf * sizeof(float4)));
  if (ctx->cfg.precision != MAP_FP64) {
    MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->fsph32, nf * sizeof(float4)));
    MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->edge32, nl * EDGE_STRIDE * sizeof(float)));
  } else {
    MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->edge64, nl * EDGE_STRIDE * sizeof(double)));
  }
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->site, nc * 3 * sizeof(double)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->vol, nc * sizeof(double)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->rad, nc * sizeof(double)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->rin, nc * sizeof(float)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->vx, nv * sizeof(double)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->vy, nv * sizeof(double)));
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&g->vz, nv * sizeof(double)));
  CUDA_TRY(cudaMemcpyAsync(g->cell_face_off, in->cell_face_off, (nc + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->face_vert_off, in->face_vert_off, (nf + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->face_vert, in->face_vert, nl * sizeof(int32_t), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->face_plane, in->face_plane, nf * sizeof(double4_32a), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->site, in->site, nc * 3 * sizeof(double), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->vx, in->vx, nv * sizeof(double), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->vy, in->vy, nv * sizeof(double), cudaMemcpyDefault, s));
  CUDA_TRY(cudaMemcpyAsync(g->vz, in->vz, nv * sizeof(double), cudaMemcpyDefault, s));
  // small device scratch: [0] max faces, [1] max loops, bytes 16..23 status, 24..31 CSR check
  int* d_small = nullptr;
  MAP_TRY(ctx_alloc_grid(ctx, g, (void**)&d_small, 64));
  CUDA_TRY(cudaMemsetAsync(d_small, 0, 64, s));
  unsigned long long* d_status = reinterpret_cast<unsigned long long*>(d_small + 4);
  unsigned long long* d_bad = reinterpret_cast<unsigned long long*>(d_small + 6);
  check_csr<<<1024, 256, 0, s>>>(nc, nf, nl, nv, g->cell_face_off, g->face_vert_off, g->face_vert, d_bad); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  unsigned long long bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (bad) return MAP_EINVAL;
  const int tpb = 128;
  const int64_t blocks = (nc + tpb - 1) / tpb;
  int32_t* fcell;
  double *volf, *r2f;
  MAP_TRY(ensure_t(ctx, ctx->ws_grid[0], nf, &fcell));
  MAP_TRY(ensure_t(ctx, ctx->ws_grid[1], nf, &volf));
  MAP_TRY(ensure_t(ctx, ctx->ws_grid[2], nf, &r2f));
  float4* v32 = nullptr;
  if (g->fsph32) {
    MAP_TRY(ensure_t(ctx, ctx->ws_grid[3], nv, &v32));
    vert32<<<nblk(nv, tpb), tpb, 0, s>>>(nv, g->vx, g->vy, g->vz, v32); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  }
  face_cells<<<(unsigned)blocks, tpb, 0, s>>>(nc, g->cell_face_off, fcell); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  prep_faces<<<nblk(nf, tpb), tpb, 0, s>>>(nf, fcell, g->face_vert_off, g->face_vert, g->face_plane, g->vx, g->vy,
                                           g->vz, v32, g->site, g->face64, g->face32, g->fsph32, g->edge64,
                                           g->edge32, volf, r2f, d_status); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  prep_cells<<<(unsigned)blocks, tpb, 0, s>>>(nc, g->cell_face_off, g->face_vert_off, volf, r2f, g->face64, g->vol,
                                              g->rad, g->rin,
                                              d_small, d_small + 1); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  int64_t hs[4] = {0, 0, 0, 0};
  CUDA_TRY(cudaMemcpyAsync(hs, d_small, 32, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  int hi[8];
  std::memcpy(hi, hs, sizeof(hi));
  g->max_faces = hi[0];
  g->max_loops = hi[1];
  // the mixed integral kernel keeps a cell-relative edge-record offset in 32
  // bits (loop index x EDGE_STRIDE); 2^26 loop entries per cell bounds it
  if (g->max_loops >= (1 << 26)) return MAP_EINVAL;
  unsigned long long st;
  std::memcpy(&st, &hi[4], sizeof(st));
  if (st != 0) return MAP_EINVAL;
  return MAP_OK;
}
