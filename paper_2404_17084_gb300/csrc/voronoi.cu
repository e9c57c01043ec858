// Grid construction on the device (Section II-A): the Voronoi grid generated
// by point sites, clipped to the unit cube, after merging tightly packed
// sites and a number of Lloyd iterations.
//
// Each cell is built by one thread: the cube, relative to the site, cut by the
// bisector planes of the neighbouring sites.  Neighbours come from a uniform
// bucket grid, ring by ring around the site's bucket; a site at distance D
// cuts along a plane at D/2, so once every unvisited site is at least twice
// the cell's largest vertex radius away the cell is final.  A cut keeps the
// part n.x <= d: each face loop is clipped in turn (a vertex within a relative
// 1e-13 of the plane counts as on it), and the vertices on the plane, ordered
// by angle around their mean, form the new face.  At the end vertices within a
// relative 1e-11 are welded and faces left with fewer than three vertices
// dropped.  Walls have exact planes; a bisector's plane passes through the
// midpoint of its two sites.
//
// Lloyd iteration: every site moves to its cell's centroid (the
// volume-weighted mean of the tetrahedra site / fan triangle of a face).
// Merging: a site within merge_tol of any site of lower index is dropped.
//
// The cells are written to fixed slots (VOR_MAXV vertices, VOR_MAXF faces,
// VOR_MAXL loop entries); a cell that outgrows them makes the call fail with
// MAP_ECAPACITY.  A scan then packs the slots into the CSR layout of map_grid,
// which the resident-grid preparation takes as it is.
#include <cub/cub.cuh>

#include "internal.cuh"

namespace {

constexpr int VOR_MAXV = 96;
constexpr int VOR_MAXF = 48;
constexpr int VOR_MAXL = 320;
constexpr int VOR_NEAR = 32;  // nearest sites of the surrounding 27 buckets, cut first and in order

struct Poly {
  int nv, nf, nl;
  double vx[VOR_MAXV], vy[VOR_MAXV], vz[VOR_MAXV];
  unsigned char loop[VOR_MAXL];
  short fs[VOR_MAXF];          // first loop entry of each face
  unsigned char fl[VOR_MAXF];  // loop length
  int nb[VOR_MAXF];            // neighbour site, or -1-w for wall w
  double rmax2;
};

// a cell as written to its slot (site-relative vertices)
struct Slot {
  int nv, nf, nl, ok;
};

__host__ __device__ __forceinline__ void poly_box(Poly& P, double sx, double sy, double sz) {
  const double lo[3] = {-sx, -sy, -sz}, hi[3] = {1.0 - sx, 1.0 - sy, 1.0 - sz};
  for (int i = 0; i < 8; ++i) {
    P.vx[i] = (i & 1) ? hi[0] : lo[0];
    P.vy[i] = (i & 2) ? hi[1] : lo[1];
    P.vz[i] = (i & 4) ? hi[2] : lo[2];
  }
  // loops counter-clockwise seen from outside: x<=1, x>=0, y<=1, y>=0, z<=1, z>=0
  const unsigned char L[24] = {1, 3, 7, 5, 0, 4, 6, 2, 2, 6, 7, 3, 0, 1, 5, 4, 4, 5, 7, 6, 0, 2, 3, 1};
  for (int k = 0; k < 24; ++k) P.loop[k] = L[k];
  for (int f = 0; f < 6; ++f) { P.fs[f] = (short)(4 * f); P.fl[f] = 4; P.nb[f] = -1 - f; }
  P.nv = 8; P.nf = 6; P.nl = 24;
  double r = 0.0;
  for (int i = 0; i < 8; ++i) r = fmax(r, P.vx[i] * P.vx[i] + P.vy[i] * P.vy[i] + P.vz[i] * P.vz[i]);
  P.rmax2 = r;
}

// Cut P by n.x <= d into Q.  Returns 0 when nothing changed (Q untouched), 1
// when Q holds the cut cell, -1 on overflow.
__host__ __device__ __forceinline__ int poly_clip(const Poly& P, Poly& Q, double nx, double ny, double nz, double d, int nbid) {
  const double tol = 1e-13 * sqrt(P.rmax2);
  signed char cls[VOR_MAXV];
  double s[VOR_MAXV];
  double smax = -1e300;
  for (int i = 0; i < P.nv; ++i) {
    s[i] = nx * P.vx[i] + ny * P.vy[i] + nz * P.vz[i] - d;
    smax = fmax(smax, s[i]);
  }
  if (smax <= tol) return 0;
  unsigned char remap[VOR_MAXV];
  unsigned char on[VOR_MAXV];
  int non = 0;
  Q.nv = 0;
  for (int i = 0; i < P.nv; ++i) {
    cls[i] = s[i] < -tol ? -1 : (s[i] > tol ? 1 : 0);
    if (cls[i] <= 0) {
      remap[i] = (unsigned char)Q.nv;
      Q.vx[Q.nv] = P.vx[i]; Q.vy[Q.nv] = P.vy[i]; Q.vz[Q.nv] = P.vz[i];
      if (cls[i] == 0) on[non++] = (unsigned char)Q.nv;
      ++Q.nv;
    }
  }
  // cut vertices, keyed by their edge
  unsigned short ckey[VOR_MAXV];
  unsigned char cid[VOR_MAXV];
  int ncut = 0;
  Q.nf = 0;
  Q.nl = 0;
  for (int f = 0; f < P.nf; ++f) {
    const int b = P.fs[f], L = P.fl[f];
    const int start = Q.nl;
    for (int k = 0; k < L; ++k) {
      const int a = P.loop[b + k], c = P.loop[b + (k + 1 == L ? 0 : k + 1)];
      int push[2], np = 0;
      if (cls[a] <= 0) push[np++] = remap[a];
      if (cls[a] * cls[c] < 0) {
        const unsigned short key = (unsigned short)((a < c ? a : c) << 8 | (a < c ? c : a));
        int id = -1;
        for (int q = 0; q < ncut; ++q)
          if (ckey[q] == key) { id = cid[q]; break; }
        if (id < 0) {
          if (Q.nv >= VOR_MAXV) return -1;
          const double t = s[a] / (s[a] - s[c]);
          id = Q.nv++;
          Q.vx[id] = P.vx[a] + (P.vx[c] - P.vx[a]) * t;
          Q.vy[id] = P.vy[a] + (P.vy[c] - P.vy[a]) * t;
          Q.vz[id] = P.vz[a] + (P.vz[c] - P.vz[a]) * t;
          ckey[ncut] = key;
          cid[ncut] = (unsigned char)id;
          ++ncut;
          on[non++] = (unsigned char)id;
        }
        push[np++] = id;
      }
      for (int q = 0; q < np; ++q) {
        // drop consecutive duplicates
        if (Q.nl > start && Q.loop[Q.nl - 1] == push[q]) continue;
        if (Q.nl >= VOR_MAXL) return -1;
        Q.loop[Q.nl++] = (unsigned char)push[q];
      }
    }
    while (Q.nl - start > 1 && Q.loop[start] == Q.loop[Q.nl - 1]) --Q.nl;
    if (Q.nl - start >= 3) {
      if (Q.nf >= VOR_MAXF) return -1;
      Q.fs[Q.nf] = (short)start;
      Q.fl[Q.nf] = (unsigned char)(Q.nl - start);
      Q.nb[Q.nf] = P.nb[f];
      ++Q.nf;
    } else {
      Q.nl = start;
    }
  }
  // the new face: the vertices on the plane (sorted by index, duplicates
  // dropped), ordered by angle around their mean
  for (int i = 1; i < non; ++i)
    for (int j = i; j > 0 && on[j - 1] > on[j]; --j) { const unsigned char t = on[j]; on[j] = on[j - 1]; on[j - 1] = t; }
  int m = 0;
  for (int i = 0; i < non; ++i)
    if (m == 0 || on[m - 1] != on[i]) on[m++] = on[i];
  non = m;
  if (non >= 3) {
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int i = 0; i < non; ++i) { cx += Q.vx[on[i]]; cy += Q.vy[on[i]]; cz += Q.vz[on[i]]; }
    cx /= non; cy /= non; cz /= non;
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (fabs(nx) < 0.6) ax = 1.0; else ay = 1.0;
    double ux = ny * az - nz * ay, uy = nz * ax - nx * az, uz = nx * ay - ny * ax;
    const double un = sqrt(ux * ux + uy * uy + uz * uz);
    ux /= un; uy /= un; uz /= un;
    const double wx = ny * uz - nz * uy, wy = nz * ux - nx * uz, wz = nx * uy - ny * ux;
    double ang[VOR_MAXV];
    for (int i = 0; i < non; ++i) {
      const double rx = Q.vx[on[i]] - cx, ry = Q.vy[on[i]] - cy, rz = Q.vz[on[i]] - cz;
      ang[i] = atan2(rx * wx + ry * wy + rz * wz, rx * ux + ry * uy + rz * uz);
    }
    for (int i = 1; i < non; ++i)
      for (int j = i; j > 0 && (ang[j - 1] > ang[j] || (ang[j - 1] == ang[j] && on[j - 1] > on[j])); --j) {
        const double ta = ang[j]; ang[j] = ang[j - 1]; ang[j - 1] = ta;
        const unsigned char t = on[j]; on[j] = on[j - 1]; on[j - 1] = t;
      }
    if (Q.nf >= VOR_MAXF || Q.nl + non > VOR_MAXL) return -1;
    Q.fs[Q.nf] = (short)Q.nl;
    Q.fl[Q.nf] = (unsigned char)non;
    Q.nb[Q.nf] = nbid;
    ++Q.nf;
    for (int i = 0; i < non; ++i) Q.loop[Q.nl++] = on[i];
  }
  // drop vertices no face refers to
  short used[VOR_MAXV];
  for (int i = 0; i < Q.nv; ++i) used[i] = -1;
  int nv = 0;
  double tx[VOR_MAXV], ty[VOR_MAXV], tz[VOR_MAXV];
  for (int k = 0; k < Q.nl; ++k) {
    const int id = Q.loop[k];
    if (used[id] < 0) { used[id] = (short)nv; tx[nv] = Q.vx[id]; ty[nv] = Q.vy[id]; tz[nv] = Q.vz[id]; ++nv; }
    Q.loop[k] = (unsigned char)used[id];
  }
  double r = 0.0;
  for (int i = 0; i < nv; ++i) {
    Q.vx[i] = tx[i]; Q.vy[i] = ty[i]; Q.vz[i] = tz[i];
    r = fmax(r, tx[i] * tx[i] + ty[i] * ty[i] + tz[i] * tz[i]);
  }
  Q.nv = nv;
  Q.rmax2 = r;
  return 1;
}

// weld vertices within a relative 1e-11, drop faces with fewer than three
// vertices and unused vertices (in place, through Q as scratch)
__host__ __device__ __forceinline__ void poly_compact(Poly& P, Poly& Q) {
  const double scale = sqrt(fmax(P.rmax2, 1e-300));
  const double tol2 = (1e-11 * scale) * (1e-11 * scale);
  unsigned char rep[VOR_MAXV];
  for (int i = 0; i < P.nv; ++i) {
    rep[i] = (unsigned char)i;
    for (int j = 0; j < i; ++j)
      if (rep[j] == j) {
        const double dx = P.vx[i] - P.vx[j], dy = P.vy[i] - P.vy[j], dz = P.vz[i] - P.vz[j];
        if (dx * dx + dy * dy + dz * dz < tol2) { rep[i] = (unsigned char)j; break; }
      }
  }
  Q.nf = 0;
  Q.nl = 0;
  for (int f = 0; f < P.nf; ++f) {
    const int start = Q.nl;
    for (int k = 0; k < P.fl[f]; ++k) {
      const unsigned char r = rep[P.loop[P.fs[f] + k]];
      if (Q.nl > start && Q.loop[Q.nl - 1] == r) continue;
      Q.loop[Q.nl++] = r;
    }
    while (Q.nl - start > 1 && Q.loop[start] == Q.loop[Q.nl - 1]) --Q.nl;
    if (Q.nl - start >= 3) {
      Q.fs[Q.nf] = (short)start;
      Q.fl[Q.nf] = (unsigned char)(Q.nl - start);
      Q.nb[Q.nf] = P.nb[f];
      ++Q.nf;
    } else {
      Q.nl = start;
    }
  }
  short used[VOR_MAXV];
  for (int i = 0; i < P.nv; ++i) used[i] = -1;
  int nv = 0;
  for (int k = 0; k < Q.nl; ++k) {
    const int id = Q.loop[k];
    if (used[id] < 0) { used[id] = (short)nv; Q.vx[nv] = P.vx[id]; Q.vy[nv] = P.vy[id]; Q.vz[nv] = P.vz[id]; ++nv; }
    Q.loop[k] = (unsigned char)used[id];
  }
  Q.nv = nv;
  Q.rmax2 = P.rmax2;
  P = Q;
}

struct Buckets {
  int G;
  const int64_t* off;    // [G^3 + 1]
  const int32_t* sites;  // site indices grouped by bucket
};

__host__ __device__ __forceinline__ int bucket_coord(double v, int G) {
  int b = (int)floor(v * G);
  return b < 0 ? 0 : (b >= G ? G - 1 : b);
}

__global__ void vor_bucket_keys(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                const double* __restrict__ z, int G, int32_t* key, int32_t* idx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = (bucket_coord(z[i], G) * G + bucket_coord(y[i], G)) * G + bucket_coord(x[i], G);
  idx[i] = (int32_t)i;
}

// off[b] = first position whose bucket is >= b
__global__ void vor_bucket_bounds(int64_t n, int64_t nb, const int32_t* __restrict__ key, int64_t* off) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k > n) return;
  const int64_t prev = k == 0 ? -1 : key[k - 1];
  const int64_t cur = k == n ? nb : key[k];
  for (int64_t b = prev + 1; b <= cur; ++b) off[b] = k;
}

// merging: drop site i when a site of lower index lies within tol
__global__ void vor_merge_flags(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                const double* __restrict__ z, Buckets B, double tol, int64_t* keep) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) { keep[n] = 0; return; }
  const int G = B.G;
  const int bx = bucket_coord(x[i], G), by = bucket_coord(y[i], G), bz = bucket_coord(z[i], G);
  bool k = true;
  for (int dz = -1; dz <= 1 && k; ++dz)
    for (int dy = -1; dy <= 1 && k; ++dy)
      for (int dx = -1; dx <= 1 && k; ++dx) {
        const int cx = bx + dx, cy = by + dy, cz = bz + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= G || cy >= G || cz >= G) continue;
        const int64_t b = ((int64_t)cz * G + cy) * G + cx;
        for (int64_t q = B.off[b]; q < B.off[b + 1]; ++q) {
          const int32_t j = B.sites[q];
          if (j >= i) continue;
          const double ex = x[j] - x[i], ey = y[j] - y[i], ez = z[j] - z[i];
          if (ex * ex + ey * ey + ez * ez < tol * tol) { k = false; break; }
        }
      }
  keep[i] = k ? 1 : 0;
}

__global__ void vor_merge_pack(int64_t n, const int64_t* __restrict__ keep, const int64_t* __restrict__ pos,
                               const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                               double* sx, double* sy, double* sz, int64_t* kept) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  const int64_t j = pos[i];
  sx[j] = x[i]; sy[j] = y[i]; sz[j] = z[i];
  if (kept) kept[j] = i;
}

struct SlotArrays {
  Slot* info;
  double* v;            // 3 * VOR_MAXV per cell (site-relative)
  unsigned char* loop;  // VOR_MAXL per cell
  short* fs;            // VOR_MAXF per cell
  unsigned char* fl;    // VOR_MAXF per cell
  int* nb;              // VOR_MAXF per cell
};

// The cell of site i, written to its slot (one thread; also callable on the
// host).  Returns false when the cell outgrew the slot.
__host__ __device__ __forceinline__ void build_cell(int64_t i, const double* __restrict__ x,
                                                    const double* __restrict__ y, const double* __restrict__ z,
                                                    const Buckets& B, const SlotArrays& S, int* overflow_local) {
  Poly A, C;
  Poly* P = &A;
  Poly* Q = &C;
  const double sx = x[i], sy = y[i], sz = z[i];
  poly_box(*P, sx, sy, sz);
  const int G = B.G;
  const double bw = 1.0 / G;
  const int bx = bucket_coord(sx, G), by = bucket_coord(sy, G), bz = bucket_coord(sz, G);
  bool bad = false;
  // first the VOR_NEAR nearest sites of the 27 surrounding buckets, nearest
  // first (they shape the cell; later cuts are then mostly skipped)
  double kd2[VOR_NEAR];
  int kj[VOR_NEAR];
  int kn = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int cx = bx + dx, cy = by + dy, cz = bz + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= G || cy >= G || cz >= G) continue;
        const int64_t b = ((int64_t)cz * G + cy) * G + cx;
        for (int64_t q = B.off[b]; q < B.off[b + 1]; ++q) {
          const int32_t j = B.sites[q];
          if (j == i) continue;
          const double ex = x[j] - sx, ey = y[j] - sy, ez = z[j] - sz;
          const double d2 = ex * ex + ey * ey + ez * ez;
          if (d2 <= 0.0 || (kn == VOR_NEAR && d2 >= kd2[VOR_NEAR - 1])) continue;
          int k = kn < VOR_NEAR ? kn++ : VOR_NEAR - 1;
          for (; k > 0 && (kd2[k - 1] > d2 || (kd2[k - 1] == d2 && kj[k - 1] > j)); --k) {
            kd2[k] = kd2[k - 1];
            kj[k] = kj[k - 1];
          }
          kd2[k] = d2;
          kj[k] = j;
        }
      }
  for (int k = 0; k < kn && !bad; ++k) {
    if (kd2[k] >= 4.0 * P->rmax2) break;
    const int j = kj[k];
    const double ex = x[j] - sx, ey = y[j] - sy, ez = z[j] - sz;
    const double len = sqrt(kd2[k]);
    const int rc = poly_clip(*P, *Q, ex / len, ey / len, ez / len, 0.5 * len, j);
    if (rc < 0) bad = true;
    else if (rc > 0) { Poly* t = P; P = Q; Q = t; }
  }
  // then every other site, ring by ring (the 27 buckets again only when the
  // nearest list was full: sites closer than its last entry are done)
  const double done2 = kn == VOR_NEAR ? kd2[VOR_NEAR - 1] : 1e300;
  for (int r = kn == VOR_NEAR ? 0 : 2; r <= G && !bad; ++r) {
    // every site outside rings 0..r-1 is at least (r-1) bucket widths away
    const double reach = (r - 1) * bw;
    if (r >= 2 && reach * reach >= 4.0 * P->rmax2) break;
    for (int dz = -r; dz <= r && !bad; ++dz)
      for (int dy = -r; dy <= r && !bad; ++dy)
        for (int dx = -r; dx <= r && !bad; ++dx) {
          const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
          if ((ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az)) != r) continue;
          const int cx = bx + dx, cy = by + dy, cz = bz + dz;
          if (cx < 0 || cy < 0 || cz < 0 || cx >= G || cy >= G || cz >= G) continue;
          const int64_t b = ((int64_t)cz * G + cy) * G + cx;
          for (int64_t q = B.off[b]; q < B.off[b + 1]; ++q) {
            const int32_t j = B.sites[q];
            if (j == i) continue;
            const double ex = x[j] - sx, ey = y[j] - sy, ez = z[j] - sz;
            const double d2 = ex * ex + ey * ey + ez * ez;
            if (d2 <= 0.0 || d2 >= 4.0 * P->rmax2 || (r <= 1 && d2 < done2)) continue;
            const double len = sqrt(d2);
            const int rc = poly_clip(*P, *Q, ex / len, ey / len, ez / len, 0.5 * len, j);
            if (rc < 0) { bad = true; break; }
            if (rc > 0) { Poly* t = P; P = Q; Q = t; }
          }
        }
  }
  Slot info{0, 0, 0, 0};
  if (!bad) {
    poly_compact(*P, *Q);
    info = Slot{P->nv, P->nf, P->nl, 1};
    double* v = S.v + (size_t)i * 3 * VOR_MAXV;
    for (int k = 0; k < P->nv; ++k) { v[3 * k] = P->vx[k]; v[3 * k + 1] = P->vy[k]; v[3 * k + 2] = P->vz[k]; }
    unsigned char* lp = S.loop + (size_t)i * VOR_MAXL;
    for (int k = 0; k < P->nl; ++k) lp[k] = P->loop[k];
    for (int f = 0; f < P->nf; ++f) {
      S.fs[(size_t)i * VOR_MAXF + f] = P->fs[f];
      S.fl[(size_t)i * VOR_MAXF + f] = P->fl[f];
      S.nb[(size_t)i * VOR_MAXF + f] = P->nb[f];
    }
  } else {
    ++*overflow_local;
  }
  S.info[i] = info;
}

// One thread per site, the sites taken in bucket order so that the threads
// of a warp build neighbouring cells (the same candidate buckets, similar
// work): its cell, written to its slot.
__global__ void __launch_bounds__(64, 16) vor_cells(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                                const double* __restrict__ z, Buckets B, SlotArrays S,
                                                unsigned long long* overflow) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t i = B.sites[t];
  int over = 0;
  build_cell(i, x, y, z, B, S, &over);
  if (over) atomicAdd(overflow, 1ULL);
}

// centroid of each cell (site + volume-weighted mean of the fan tetrahedra)
__global__ void vor_centroids(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ z, SlotArrays S, double* ox, double* oy, double* oz) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Slot info = S.info[i];
  const double* v = S.v + (size_t)i * 3 * VOR_MAXV;
  const unsigned char* lp = S.loop + (size_t)i * VOR_MAXL;
  double tv = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
  for (int f = 0; f < info.nf; ++f) {
    const int b = S.fs[(size_t)i * VOR_MAXF + f], L = S.fl[(size_t)i * VOR_MAXF + f];
    const double* a = v + 3 * lp[b];
    for (int k = 1; k + 1 < L; ++k) {
      const double* p = v + 3 * lp[b + k];
      const double* q = v + 3 * lp[b + k + 1];
      const double vol = (a[0] * (p[1] * q[2] - p[2] * q[1]) - a[1] * (p[0] * q[2] - p[2] * q[0]) +
                          a[2] * (p[0] * q[1] - p[1] * q[0])) / 6.0;
      tv += vol;
      cx += vol * (a[0] + p[0] + q[0]) * 0.25;
      cy += vol * (a[1] + p[1] + q[1]) * 0.25;
      cz += vol * (a[2] + p[2] + q[2]) * 0.25;
    }
  }
  ox[i] = x[i] + cx / tv;
  oy[i] = y[i] + cy / tv;
  oz[i] = z[i] + cz / tv;
}

__global__ void vor_counts(int64_t n, const Slot* __restrict__ info, int64_t* nf, int64_t* nl, int64_t* nv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) { nf[i] = 0; nl[i] = 0; nv[i] = 0; return; }
  nf[i] = info[i].nf; nl[i] = info[i].nl; nv[i] = info[i].nv;
}

// pack the slots into the CSR arrays of map_grid (absolute coordinates)
__global__ void vor_pack(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ z, SlotArrays S, const int64_t* __restrict__ fo,
                         const int64_t* __restrict__ lo, const int64_t* __restrict__ vo, int64_t* cell_face_off,
                         int64_t* face_vert_off, int32_t* face_vert, double* face_plane, double* vx, double* vy,
                         double* vz, double* site) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    cell_face_off[n] = fo[n];
    face_vert_off[fo[n]] = lo[n];
    return;
  }
  const Slot info = S.info[i];
  const double sx = x[i], sy = y[i], sz = z[i];
  site[3 * i] = sx; site[3 * i + 1] = sy; site[3 * i + 2] = sz;
  cell_face_off[i] = fo[i];
  const double* v = S.v + (size_t)i * 3 * VOR_MAXV;
  for (int k = 0; k < info.nv; ++k) {
    vx[vo[i] + k] = sx + v[3 * k];
    vy[vo[i] + k] = sy + v[3 * k + 1];
    vz[vo[i] + k] = sz + v[3 * k + 2];
  }
  const unsigned char* lp = S.loop + (size_t)i * VOR_MAXL;
  int64_t l = lo[i];
  for (int f = 0; f < info.nf; ++f) {
    const int64_t F = fo[i] + f;
    face_vert_off[F] = l;
    const int b = S.fs[(size_t)i * VOR_MAXF + f], L = S.fl[(size_t)i * VOR_MAXF + f];
    for (int k = 0; k < L; ++k) face_vert[l++] = (int32_t)(vo[i] + lp[b + k]);
    const int w = S.nb[(size_t)i * VOR_MAXF + f];
    double nx, ny, nz, d;
    if (w < 0) {
      const int ax = (-1 - w) / 2, sg = ((-1 - w) % 2 == 0) ? 1 : -1;
      nx = ax == 0 ? sg : 0.0; ny = ax == 1 ? sg : 0.0; nz = ax == 2 ? sg : 0.0;
      d = sg > 0 ? 1.0 : 0.0;
    } else {
      const double ex = x[w] - sx, ey = y[w] - sy, ez = z[w] - sz;
      const double len = sqrt(ex * ex + ey * ey + ez * ez);
      nx = ex / len; ny = ey / len; nz = ez / len;
      d = nx * (0.5 * (sx + x[w])) + ny * (0.5 * (sy + y[w])) + nz * (0.5 * (sz + z[w]));
    }
    face_plane[4 * F] = nx; face_plane[4 * F + 1] = ny; face_plane[4 * F + 2] = nz; face_plane[4 * F + 3] = d;
  }
}

template <typename T>
int scan_excl(map_ctx* ctx, const T* in, T* out, int64_t n, cudaStream_t s) {
  size_t tb = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(ctx->cub_tmp.p, tb, in, out, n, s));
  return MAP_OK;
}

// bucket grid over the sites x, y, z (n of them)
int vor_buckets(map_ctx* ctx, const double* x, const double* y, const double* z, int64_t n, Buckets& B,
                cudaStream_t s) {
  int G = (int)floor(cbrt((double)n / 2.0));
  G = G < 1 ? 1 : (G > 1024 ? 1024 : G);
  const int64_t nb = (int64_t)G * G * G;
  int32_t *key, *idx, *key_s, *idx_s;
  int64_t* off;
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[0], n, &key));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[1], n, &idx));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[2], n, &key_s));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[3], n, &idx_s));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[4], nb + 1, &off));
  vor_bucket_keys<<<nblk(n, 256), 256, 0, s>>>(n, x, y, z, G, key, idx); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  int bits = 1;
  while (bits < 31 && (int64_t(1) << bits) < nb) ++bits;
  size_t tb = 0;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, key, key_s, idx, idx_s, n, 0, bits, s));
  MAP_TRY(ctx_ensure(ctx, ctx->cub_tmp, tb));
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, tb, key, key_s, idx, idx_s, n, 0, bits, s));
  vor_bucket_bounds<<<nblk(n + 1, 256), 256, 0, s>>>(n, nb, key_s, off); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  B = Buckets{G, off, idx_s};
  return MAP_OK;
}

// the cells of the sites x, y, z into the slots; MAP_ECAPACITY on overflow
int vor_tessellate(map_ctx* ctx, const double* x, const double* y, const double* z, int64_t n, SlotArrays& S,
                   cudaStream_t s) {
  Buckets B;
  MAP_TRY(vor_buckets(ctx, x, y, z, n, B, s));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[5], n, &S.info));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[6], (size_t)n * 3 * VOR_MAXV, &S.v));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[7], (size_t)n * VOR_MAXL, &S.loop));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[8], (size_t)n * VOR_MAXF, &S.fs));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[9], (size_t)n * VOR_MAXF, &S.fl));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[10], (size_t)n * VOR_MAXF, &S.nb));
  unsigned long long* d_over = ctx->d_counters + 7;
  CUDA_TRY(cudaMemsetAsync(d_over, 0, sizeof(unsigned long long), s));
  // the cell builder keeps two polyhedra per thread in local memory (a frame
  // of about 14 KB): make sure the per-thread stack holds it, whatever the
  // function attributes report
  cudaFuncAttributes fa{};
  CUDA_TRY(cudaFuncGetAttributes(&fa, vor_cells));
  size_t stack = 0;
  CUDA_TRY(cudaDeviceGetLimit(&stack, cudaLimitStackSize));
  const size_t need = (fa.localSizeBytes > 16384 ? fa.localSizeBytes : 16384) + 1024;
  if (stack < need) CUDA_TRY(cudaDeviceSetLimit(cudaLimitStackSize, need));
  // refuse to launch a frame the per-thread stack does not hold (the limit
  // read back, as the driver may round or cap it)
  CUDA_TRY(cudaDeviceGetLimit(&stack, cudaLimitStackSize));
  if (stack < fa.localSizeBytes + 1024) return MAP_ECUDA;
  vor_cells<<<nblk(n, 64), 64, 0, s>>>(n, x, y, z, B, S, d_over); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, d_over, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ctx->h_scratch[0] == 0 ? MAP_OK : MAP_ECAPACITY;
}

__global__ void vor_iota_k(int64_t n, int64_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = i;
}

int vor_iota(map_ctx* ctx, int64_t* out, int64_t n, cudaStream_t s) {
  vor_iota_k<<<nblk(n, 256), 256, 0, s>>>(n, out); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  return MAP_OK;
}

}  // namespace

extern "C" int map_grid_build(map_ctx* ctx, const double* x, const double* y, const double* z, int64_t n, int lloyd,
                              double merge_tol, int* handle, int64_t* kept, int64_t* n_kept, void* stream) {
  if (!ctx || !x || !y || !z || n < 1 || n >= (int64_t(1) << 31) || lloyd < 0 || !handle) return MAP_EINVAL;
  if (!(merge_tol >= 0.0) || !std::isfinite(merge_tol)) return MAP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MAP_ENTER(ctx, s);
  map_particles chk{n, x, y, z, nullptr, nullptr};
  MAP_TRY(check_particles(ctx, &chk, false, false, s));  // finite, inside the cube
  // the sites, merged, in one of two ping-pong buffers (x block, y block, z block)
  double *sa, *sb;
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[11], 3 * n, &sa));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[12], 3 * n, &sb));
  int64_t m = n;
  if (merge_tol > 0.0) {
    Buckets B;
    MAP_TRY(vor_buckets(ctx, x, y, z, n, B, s));
    int64_t *keep, *pos;
    MAP_TRY(ensure_t(ctx, ctx->ws_vor[13], n + 1, &keep));
    MAP_TRY(ensure_t(ctx, ctx->ws_vor[14], n + 1, &pos));
    vor_merge_flags<<<nblk(n + 1, 256), 256, 0, s>>>(n, x, y, z, B, merge_tol, keep); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    MAP_TRY(scan_excl<int64_t>(ctx, keep, pos, n + 1, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    m = ctx->h_scratch[0];
    vor_merge_pack<<<nblk(n, 256), 256, 0, s>>>(n, keep, pos, x, y, z, sa, sa + m, sa + 2 * m, kept); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
  } else {
    CUDA_TRY(cudaMemcpyAsync(sa, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(sa + n, y, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(sa + 2 * n, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (kept) MAP_TRY(vor_iota(ctx, kept, n, s));
  }
  if (n_kept) *n_kept = m;
  // Lloyd iterations, then the final cells
  SlotArrays S;
  for (int it = 0; it <= lloyd; ++it) {
    MAP_TRY(vor_tessellate(ctx, sa, sa + m, sa + 2 * m, m, S, s));
    if (it == lloyd) break;
    vor_centroids<<<nblk(m, 128), 128, 0, s>>>(m, sa, sa + m, sa + 2 * m, S, sb, sb + m, sb + 2 * m); ++ctx->launches;
    CUDA_TRY(cudaGetLastError());
    double* t = sa; sa = sb; sb = t;
  }
  // CSR offsets and the packed arrays
  int64_t *cf, *cl, *cv, *fo, *lo, *vo;
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[15], 6 * (m + 1), &cf));
  cl = cf + (m + 1); cv = cl + (m + 1); fo = cv + (m + 1); lo = fo + (m + 1); vo = lo + (m + 1);
  vor_counts<<<nblk(m + 1, 256), 256, 0, s>>>(m, S.info, cf, cl, cv); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  MAP_TRY(scan_excl<int64_t>(ctx, cf, fo, m + 1, s));
  MAP_TRY(scan_excl<int64_t>(ctx, cl, lo, m + 1, s));
  MAP_TRY(scan_excl<int64_t>(ctx, cv, vo, m + 1, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, fo + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch + 1, lo + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch + 2, vo + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nf = ctx->h_scratch[0], nl = ctx->h_scratch[1], nv = ctx->h_scratch[2];
  int64_t *cfo, *fvo;
  int32_t* fv;
  double *fpl, *vx, *vy, *vz, *site;
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[16], m + 1, &cfo));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[17], nf + 1, &fvo));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[18], nl, &fv));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[19], 4 * nf, &fpl));
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[20], 3 * nv, &vx));
  vy = vx + nv; vz = vy + nv;
  MAP_TRY(ensure_t(ctx, ctx->ws_vor[21], 3 * m, &site));
  vor_pack<<<nblk(m + 1, 128), 128, 0, s>>>(m, sa, sa + m, sa + 2 * m, S, fo, lo, vo, cfo, fvo, fv, fpl, vx, vy, vz,
                                            site); ++ctx->launches;
  CUDA_TRY(cudaGetLastError());
  const map_grid grid{m, nf, nl, nv, cfo, fvo, fv, fpl, vx, vy, vz, site};
  return map_grid_upload(ctx, &grid, handle, stream);
}
