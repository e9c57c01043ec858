/*
 * FP64 CPU oracle for the Exact SPH -> Voronoi density mapping and its
 * pseudo-particle front end (Lau, Petkova & Bonnell 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header or constant table with the CUDA path.
 *
 * What it computes, and by which route:
 *
 *  - Cell density, Eq. (1)-(3): rho_i = (1/V_i) sum_a m_a f_ai with the pair
 *    integral f_ai = int_{V_i} W(|r'-r_a|, h_a) dV'.
 *  - The cell volume is split into vertex pyramids (Section II-B): for each
 *    face, the perpendicular distance r0 from the particle to the face plane;
 *    for each edge of that face, the in-plane distance R0 from the projection
 *    point to the edge line and the angles phi between the foot of that
 *    perpendicular and the edge's two vertices.  Each pyramid integral is
 *    I(r0,R0,phi) = r0 * int_0^phi [H(U(phi')) - H(r0)] dphi',
 *    U = sqrt(r0^2 + R0^2 sec^2 phi'), where H' = F/u^2 and 4 pi F(u) is the
 *    kernel mass inside radius u.  (Solid angle dOmega = r0 dA / r^3 turns the
 *    pyramid integral into this 1-D integral.)  The oracle evaluates the 1-D
 *    integral by adaptive Gauss-Kronrod quadrature, split at the radii 1 and
 *    2 where the kernel changes polynomial piece.  It does NOT use the
 *    closed form the CUDA path uses.
 *  - Table variant (the paper's production route, Section II-B): with a
 *    table set (or_table_set), each pyramid integral inside the table's box
 *    is interpolated trilinearly between pre-computed values of I.
 *  - Kernel: the standard 3-D M4 cubic spline with support 2h,
 *    W = w(q)/(pi h^3), w = 1 - 1.5q^2 + 0.75q^3 (q<1), 0.25(2-q)^3 (q<2).
 *    (The paper names the M4 kernel in Section III-C but prints no formula.)
 *  - Pair rule (the paper is silent; reading fixed here so that pair lists
 *    are reproducible): pair (i,a) is listed iff |r_a - s_i| < 2h_a + R_i
 *    (R_i = largest vertex distance from the site) and no face plane of cell
 *    i separates it: n_f.r_a - d_f < 2h_a for every face.  Evaluated with a
 *    fixed operation order and no FMA contraction.
 *  - Smoothing lengths, Eq. (7)-(9): h = hfact n^(-1/3), n = sum_b W(r_ab, h)
 *    (self term included), solved by Newton-Raphson, then bisection, then the
 *    estimate of Eq. (9).
 *  - Octree and adaptive walk, Section III-A/B and Eq. (5): a node is opened
 *    when (s_node/r_node)^2 > theta^2 (or r_node = 0); an opened leaf yields
 *    its particles.  Node position = centre of mass, size = distance from the
 *    centre of mass to the furthest particle (Section III-A).
 *
 * Build: cc -O2 -fopenmp -ffp-contract=off -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ kernel */

/* w(q) of the M4 cubic spline (Section III-C), unnormalised. */
double or_w(double q) {
  if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
  if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
  return 0.0;
}

/* dw/dq */
double or_dw(double q) {
  if (q < 1.0) return -3.0 * q + 2.25 * q * q;
  if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
  return 0.0;
}

/* W(r,h) = w(r/h)/(pi h^3) */
double or_W(double r, double h) { return or_w(r / h) / (OR_PI * h * h * h); }

/* F(u) = int_0^u W(r,1) r^2 dr, so that 4 pi F(u) is the kernel mass within u. */
double or_F(double u) {
  double u2 = u * u, u3 = u2 * u;
  if (u < 1.0) return (4.0 / 3.0 * u3 - 6.0 / 5.0 * u3 * u2 + 0.5 * u3 * u3) / (4.0 * OR_PI);
  if (u < 2.0)
    return (-1.0 / 15.0 + 8.0 / 3.0 * u3 - 3.0 * u3 * u + 6.0 / 5.0 * u3 * u2 - u3 * u3 / 6.0) / (4.0 * OR_PI);
  return 1.0 / (4.0 * OR_PI);
}

/* H(u) = int F(u)/u^2 du, H(0)=0, continuous at u=1 and u=2. */
double or_H(double u) {
  double u2 = u * u;
  if (u < 1.0) return (u2 / 6.0 - 3.0 * u2 * u2 / 40.0 + u2 * u2 * u / 40.0) / OR_PI;
  if (u < 2.0)
    return (1.0 / (15.0 * u) + 4.0 * u2 / 3.0 - u2 * u + 3.0 * u2 * u2 / 10.0 - u2 * u2 * u / 30.0) / (4.0 * OR_PI)
           - 1.0 / (20.0 * OR_PI);
  return (0.5 - 1.0 / u) / (4.0 * OR_PI) + 9.0 / (40.0 * OR_PI);
}

/* ---------------------------------------------------- vertex pyramid (Sec. II-B) */

typedef struct { double r0, R0, Hr0; } wedge_par;

static double wedge_integrand(double phi, const wedge_par* p) {
  double c = cos(phi);
  double U = sqrt(p->r0 * p->r0 + (p->R0 * p->R0) / (c * c));
  return p->r0 * (or_H(U) - p->Hr0);
}

/* Gauss-Kronrod 7/15 nodes and weights on [-1,1]. */
static const double gk_x[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double gk_wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk15(double a, double b, const wedge_par* p, double* err) {
  double c = 0.5 * (a + b), hw = 0.5 * (b - a);
  double fc = wedge_integrand(c, p);
  double rk = fc * gk_wk[7], rg = fc * gk_wg[3];
  for (int j = 0; j < 7; ++j) {
    double dx = hw * gk_x[j];
    double f1 = wedge_integrand(c - dx, p), f2 = wedge_integrand(c + dx, p);
    rk += gk_wk[j] * (f1 + f2);
    if (j % 2 == 1) rg += gk_wg[j / 2] * (f1 + f2);
  }
  *err = fabs((rk - rg) * hw);
  return rk * hw;
}

static double adapt(double a, double b, const wedge_par* p, double whole, double err, int depth) {
  if (err <= 1e-16 || err <= 1e-14 * fabs(whole) || depth > 40) return whole;
  double m = 0.5 * (a + b), e1, e2;
  double l = gk15(a, m, p, &e1), r = gk15(m, b, p, &e2);
  return adapt(a, m, p, l, e1, depth + 1) + adapt(m, b, p, r, e2, depth + 1);
}

static double integrate(double a, double b, const wedge_par* p) {
  if (!(b > a)) return 0.0;
  double e;
  double w = gk15(a, b, p, &e);
  return adapt(a, b, p, w, e, 0);
}

/* I(r0,R0,phi): kernel mass (h = 1) in the pyramid with apex at the particle
 * over the right triangle (projection point, foot on the edge line, point at
 * angle phi from the foot).  r0, R0 >= 0, 0 <= phi < pi/2. */
double or_wedge(double r0, double R0, double phi) {
  if (r0 <= 0.0 || R0 <= 0.0 || phi <= 0.0) return 0.0;
  wedge_par p = {r0, R0, or_H(r0)};
  /* split where U(phi') crosses 1 and 2 */
  double cuts[2];
  int nc = 0;
  for (int b = 1; b <= 2; ++b) {
    double bb = (double)b;
    if (r0 < bb) {
      double rho = sqrt(bb * bb - r0 * r0);
      if (R0 < rho) {
        double pb = acos(R0 / rho);
        if (pb > 0.0 && pb < phi) cuts[nc++] = pb;
      }
    }
  }
  double lo = 0.0, tot = 0.0;
  for (int k = 0; k < nc; ++k) { tot += integrate(lo, cuts[k], &p); lo = cuts[k]; }
  tot += integrate(lo, phi, &p);
  return tot;
}

/* ------------------------------------- table variant (Section II-B, production) */

/* The paper's production route: I(r0, R0, phi) pre-computed on a grid and
 * interpolated.  Here: n nodes per axis over r0 in [0, 2], rho = R0 /
 * sqrt(4 - r0^2) in [0, 1] (R0 beyond the support's reach of the edge line
 * needs no table) and phi in [0, pi/2], filled with or_wedge, and trilinear
 * interpolation between the eight surrounding nodes.  Outside that box
 * (r0 >= 2 or rho >= 1) or with no table set, the exact or_wedge is used. */
static int tab_n = 0;
static double* tab = NULL;

void or_table_set(int n) {
  free(tab);
  tab = NULL;
  tab_n = 0;
  if (n < 2) return;
  tab = (double*)malloc(sizeof(double) * (size_t)n * n * n);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) {
    double r0 = 2.0 * i / (n - 1);
    double span = sqrt(fmax(4.0 - r0 * r0, 0.0));
    for (int j = 0; j < n; ++j) {
      double R0 = span * j / (n - 1);
      for (int k = 0; k < n; ++k) {
        double phi = 0.5 * OR_PI * k / (n - 1);
        /* or_wedge takes phi < pi/2: the last node is the limit, approached
           within 1e-12 */
        if (k == n - 1) phi = 0.5 * OR_PI - 1e-12;
        tab[((size_t)i * n + j) * n + k] = or_wedge(r0, R0, phi);
      }
    }
  }
  tab_n = n;
}

double or_wedge_table(double r0, double R0, double phi) {
  if (!tab || r0 >= 2.0) return or_wedge(r0, R0, phi);
  double span = sqrt(4.0 - r0 * r0);
  double rho = R0 / span;
  if (rho >= 1.0) return or_wedge(r0, R0, phi);
  int n = tab_n;
  double u[3] = {r0 / 2.0 * (n - 1), rho * (n - 1), phi / (0.5 * OR_PI) * (n - 1)};
  int i0[3];
  double t[3];
  for (int d = 0; d < 3; ++d) {
    double x = u[d] < 0.0 ? 0.0 : u[d];
    int k = (int)floor(x);
    if (k > n - 2) k = n - 2;
    i0[d] = k;
    t[d] = x - k;
  }
  double v = 0.0;
  for (int c = 0; c < 8; ++c) {
    int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
    double wgt = (a ? t[0] : 1.0 - t[0]) * (b ? t[1] : 1.0 - t[1]) * (e ? t[2] : 1.0 - t[2]);
    v += wgt * tab[((size_t)(i0[0] + a) * n + (i0[1] + b)) * n + (i0[2] + e)];
  }
  return v;
}

/* ---------------------------------------------------------------- cells */

typedef struct {
  const int64_t* cell_face_off;
  const int64_t* face_vert_off;
  const int32_t* face_vert;
  const double* face_plane; /* nx,ny,nz,d per face */
  const double *vx, *vy, *vz;
  const double* site;       /* 3 per cell */
} or_grid;

/* Pair integral f_ai for cell c of the grid and a particle at (x,y,z) with
 * smoothing length h: signed sum of vertex-pyramid integrals (Section II-B).
 * For each face: s_f = +1 if the particle is on the inner side of the face
 * plane.  For each edge of the face (loop order, CCW from outside): s_e = +1
 * if the projection point is on the inner side of the edge; the two wedges
 * at the edge's vertices are added when the foot of the perpendicular lies
 * between them, otherwise the far one is added and the near one subtracted. */
double or_pair_fraction(const or_grid* g, int64_t c, double x, double y, double z, double h) {
  double tot = 0.0;
  for (int64_t f = g->cell_face_off[c]; f < g->cell_face_off[c + 1]; ++f) {
    const double* pl = g->face_plane + 4 * f;
    double nx = pl[0], ny = pl[1], nz = pl[2], d = pl[3];
    double sd = d - (nx * x + ny * y + nz * z); /* >0: particle on the inner side */
    if (sd == 0.0) continue;                    /* degenerate pyramid: zero volume */
    double sf = sd > 0.0 ? 1.0 : -1.0;
    double r0 = fabs(sd) / h;
    /* projection of the particle onto the face plane */
    double px = x + sd * nx, py = y + sd * ny, pz = z + sd * nz;
    int64_t b = g->face_vert_off[f], e = g->face_vert_off[f + 1];
    int64_t L = e - b;
    double face_sum = 0.0;
    for (int64_t k = 0; k < L; ++k) {
      int32_t ia = g->face_vert[b + k], ib = g->face_vert[b + (k + 1) % L];
      double ax = g->vx[ia], ay = g->vy[ia], az = g->vz[ia];
      double bx = g->vx[ib], by = g->vy[ib], bz = g->vz[ib];
      double ex = bx - ax, ey = by - ay, ez = bz - az;
      double len = sqrt(ex * ex + ey * ey + ez * ez);
      if (len == 0.0) continue;
      ex /= len; ey /= len; ez /= len;
      /* inward in-plane normal of the edge: n x e */
      double mx = ny * ez - nz * ey, my = nz * ex - nx * ez, mz = nx * ey - ny * ex;
      double sR = mx * (px - ax) + my * (py - ay) + mz * (pz - az); /* >0: p inside w.r.t. this edge */
      if (sR == 0.0) continue;
      double se = sR > 0.0 ? 1.0 : -1.0;
      double R0 = fabs(sR) / h;
      /* signed positions of the two vertices along the edge, from the foot q */
      double ta = (ex * (ax - px) + ey * (ay - py) + ez * (az - pz)) / h;
      double tb = (ex * (bx - px) + ey * (by - py) + ez * (bz - pz)) / h;
      double phia = atan(fabs(ta) / R0), phib = atan(fabs(tb) / R0);
      double Ia = or_wedge_table(r0, R0, phia), Ib = or_wedge_table(r0, R0, phib);
      double contrib;
      if (ta < 0.0 && tb > 0.0) contrib = Ia + Ib;      /* foot between the vertices */
      else if (ta >= 0.0) contrib = Ib - Ia;            /* foot before a: b is far */
      else contrib = Ia - Ib;                           /* foot after b: a is far */
      face_sum += se * contrib;
    }
    tot += sf * face_sum;
  }
  return tot;
}

/* Cell volume by the divergence theorem: V = (1/3) sum_f d_f' A_f where d_f'
 * is the distance from the site to the face plane. */
double or_cell_volume(const or_grid* g, int64_t c) {
  double sx = g->site[3 * c], sy = g->site[3 * c + 1], sz = g->site[3 * c + 2];
  double V = 0.0;
  for (int64_t f = g->cell_face_off[c]; f < g->cell_face_off[c + 1]; ++f) {
    const double* pl = g->face_plane + 4 * f;
    int64_t b = g->face_vert_off[f], e = g->face_vert_off[f + 1];
    int64_t L = e - b;
    double ax = 0, ay = 0, az = 0;
    for (int64_t k = 0; k < L; ++k) {
      int32_t i0 = g->face_vert[b + k], i1 = g->face_vert[b + (k + 1) % L];
      double x0 = g->vx[i0] - sx, y0 = g->vy[i0] - sy, z0 = g->vz[i0] - sz;
      double x1 = g->vx[i1] - sx, y1 = g->vy[i1] - sy, z1 = g->vz[i1] - sz;
      ax += y0 * z1 - z0 * y1; ay += z0 * x1 - x0 * z1; az += x0 * y1 - y0 * x1;
    }
    double area = 0.5 * (ax * pl[0] + ay * pl[1] + az * pl[2]);
    double dist = pl[3] - (pl[0] * sx + pl[1] * sy + pl[2] * sz);
    V += dist * area / 3.0;
  }
  return V;
}

/* R_i: largest vertex distance from the site, fixed evaluation order. */
double or_cell_radius(const or_grid* g, int64_t c) {
  double sx = g->site[3 * c], sy = g->site[3 * c + 1], sz = g->site[3 * c + 2];
  double R = 0.0;
  for (int64_t f = g->cell_face_off[c]; f < g->cell_face_off[c + 1]; ++f)
    for (int64_t k = g->face_vert_off[f]; k < g->face_vert_off[f + 1]; ++k) {
      int32_t v = g->face_vert[k];
      double dx = g->vx[v] - sx, dy = g->vy[v] - sy, dz = g->vz[v] - sz;
      double r = sqrt((dx * dx + dy * dy) + dz * dz);
      if (r > R) R = r;
    }
  return R;
}

/* The pair rule (see the header comment). */
int or_pair_test(const or_grid* g, int64_t c, double Ri, double x, double y, double z, double h) {
  double sx = g->site[3 * c], sy = g->site[3 * c + 1], sz = g->site[3 * c + 2];
  double dx = x - sx, dy = y - sy, dz = z - sz;
  double dist = sqrt((dx * dx + dy * dy) + dz * dz);
  double h2 = 2.0 * h;
  if (!(dist < h2 + Ri)) return 0;
  for (int64_t f = g->cell_face_off[c]; f < g->cell_face_off[c + 1]; ++f) {
    const double* pl = g->face_plane + 4 * f;
    double s = ((pl[0] * x + pl[1] * y) + pl[2] * z) - pl[3];
    if (!(s < h2)) return 0;
  }
  return 1;
}

static or_grid make_grid(const int64_t* cfo, const int64_t* fvo, const int32_t* fv, const double* fpl,
                         const double* vx, const double* vy, const double* vz, const double* site) {
  or_grid g = {cfo, fvo, fv, fpl, vx, vy, vz, site};
  return g;
}

/* Count pairs for the listed cells by brute force over all particles. */
void or_pair_count(const int64_t* cfo, const int64_t* fvo, const int32_t* fv, const double* fpl,
                   const double* vx, const double* vy, const double* vz, const double* site,
                   const int64_t* cells, int64_t ncells, const double* px, const double* py, const double* pz,
                   const double* ph, int64_t np, int64_t* count, int nthreads) {
  or_grid g = make_grid(cfo, fvo, fv, fpl, vx, vy, vz, site);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t k = 0; k < ncells; ++k) {
    int64_t c = cells[k];
    double Ri = or_cell_radius(&g, c);
    int64_t n = 0;
    for (int64_t a = 0; a < np; ++a) n += or_pair_test(&g, c, Ri, px[a], py[a], pz[a], ph[a]);
    count[k] = n;
  }
}

/* Fill pairs (ascending particle index per cell) into off[k]..off[k+1]. */
void or_pair_fill(const int64_t* cfo, const int64_t* fvo, const int32_t* fv, const double* fpl,
                  const double* vx, const double* vy, const double* vz, const double* site,
                  const int64_t* cells, int64_t ncells, const double* px, const double* py, const double* pz,
                  const double* ph, int64_t np, const int64_t* off, int32_t* idx, int nthreads) {
  or_grid g = make_grid(cfo, fvo, fv, fpl, vx, vy, vz, site);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t k = 0; k < ncells; ++k) {
    int64_t c = cells[k];
    double Ri = or_cell_radius(&g, c);
    int64_t w = off[k];
    for (int64_t a = 0; a < np; ++a)
      if (or_pair_test(&g, c, Ri, px[a], py[a], pz[a], ph[a])) idx[w++] = (int32_t)a;
  }
}

/* Pair integrals and cell sums for the listed cells, given their pair lists.
 * frac[p] = f_ai for every listed pair; mass[k] = sum_a m_a f_ai (long
 * double accumulation); vol[k] = V_i; rho = mass/vol. */
void or_map_cells(const int64_t* cfo, const int64_t* fvo, const int32_t* fv, const double* fpl,
                  const double* vx, const double* vy, const double* vz, const double* site,
                  const int64_t* cells, int64_t ncells, const double* px, const double* py, const double* pz,
                  const double* pm, const double* ph, const int64_t* off, const int32_t* idx,
                  double* frac, double* mass, double* vol, double* rho, int nthreads) {
  or_grid g = make_grid(cfo, fvo, fv, fpl, vx, vy, vz, site);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t k = 0; k < ncells; ++k) {
    int64_t c = cells[k];
    long double M = 0.0L;
    for (int64_t p = off[k]; p < off[k + 1]; ++p) {
      int32_t a = idx[p];
      double f = or_pair_fraction(&g, c, px[a], py[a], pz[a], ph[a]);
      if (frac) frac[p] = f;
      M += (long double)pm[a] * (long double)f;
    }
    double V = or_cell_volume(&g, c);
    mass[k] = (double)M;
    vol[k] = V;
    rho[k] = (double)M / V;
  }
}

/* Volumes and radii of all cells. */
void or_cell_geometry(const int64_t* cfo, const int64_t* fvo, const int32_t* fv, const double* fpl,
                      const double* vx, const double* vy, const double* vz, const double* site, int64_t ncell,
                      double* vol, double* radius) {
  or_grid g = make_grid(cfo, fvo, fv, fpl, vx, vy, vz, site);
  for (int64_t c = 0; c < ncell; ++c) {
    if (vol) vol[c] = or_cell_volume(&g, c);
    if (radius) radius[c] = or_cell_radius(&g, c);
  }
}

/* ------------------------------------------------- smoothing lengths (Sec. III-C) */

/* Uniform bucket grid over the points, used only to enumerate candidates
 * within a radius (every point of every bucket overlapping the query box is
 * tested exactly, so the sum is the plain sum over all neighbours). */
typedef struct {
  int G;
  int64_t* start; /* G^3 + 1 */
  int64_t* item;
  const double *x, *y, *z;
  int64_t n;
} or_buckets;

static int bclamp(int v, int G) { return v < 0 ? 0 : (v >= G ? G - 1 : v); }

static void buckets_init(or_buckets* B, const double* x, const double* y, const double* z, int64_t n) {
  int G = (int)cbrt((double)n / 2.0);
  if (G < 1) G = 1;
  if (G > 256) G = 256;
  B->G = G; B->x = x; B->y = y; B->z = z; B->n = n;
  int64_t nb = (int64_t)G * G * G;
  B->start = (int64_t*)calloc(nb + 1, sizeof(int64_t));
  B->item = (int64_t*)malloc((n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* cnt = (int64_t*)calloc(nb, sizeof(int64_t));
  int64_t* key = (int64_t*)malloc((n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    int bx = bclamp((int)(x[i] * G), G), by = bclamp((int)(y[i] * G), G), bz = bclamp((int)(z[i] * G), G);
    key[i] = ((int64_t)bx * G + by) * G + bz;
    cnt[key[i]]++;
  }
  for (int64_t b = 0; b < nb; ++b) B->start[b + 1] = B->start[b] + cnt[b];
  memset(cnt, 0, nb * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) B->item[B->start[key[i]] + cnt[key[i]]++] = i;
  free(cnt); free(key);
}

static void buckets_free(or_buckets* B) { free(B->start); free(B->item); }

/* n(h) = sum_b W(r_ab, h) over all points (self included), and dn/dh. */
static void number_density(const or_buckets* B, double x, double y, double z, double h, double* n, double* dn) {
  int G = B->G;
  double R = 2.0 * h;
  int x0 = bclamp((int)floor((x - R) * G), G), x1 = bclamp((int)floor((x + R) * G), G);
  int y0 = bclamp((int)floor((y - R) * G), G), y1 = bclamp((int)floor((y + R) * G), G);
  int z0 = bclamp((int)floor((z - R) * G), G), z1 = bclamp((int)floor((z + R) * G), G);
  double s = 0.0, ds = 0.0;
  double h3 = h * h * h;
  for (int bx = x0; bx <= x1; ++bx)
    for (int by = y0; by <= y1; ++by)
      for (int bz = z0; bz <= z1; ++bz) {
        int64_t b = ((int64_t)bx * G + by) * G + bz;
        for (int64_t k = B->start[b]; k < B->start[b + 1]; ++k) {
          int64_t j = B->item[k];
          double dx = B->x[j] - x, dy = B->y[j] - y, dz = B->z[j] - z;
          double r = sqrt(dx * dx + dy * dy + dz * dz);
          double q = r / h;
          if (q >= 2.0) continue;
          double w = or_w(q);
          s += w / (OR_PI * h3);
          /* dW/dh = -(3 w + q w') / (pi h^4) */
          ds += -(3.0 * w + q * or_dw(q)) / (OR_PI * h3 * h);
        }
      }
  *n = s; *dn = ds;
}

/* Solve h = hfact n(h)^(-1/3) for the targets (indices into the point set).
 * h0[k] is the initial guess and the Eq. (9) fallback.  Route per target:
 * 0 = Newton-Raphson, 1 = bisection, 2 = estimate.  Newton: at most 30
 * iterations, converged when |dh|/h < 1e-10; any iterate outside
 * [h0/16, 16 h0] or no convergence -> bisection on [h0/16, 16 h0] (200
 * iterations or |dh|/h < 1e-12); no sign change -> h = h0. */
void or_solve_h(const double* x, const double* y, const double* z, int64_t n, const int64_t* targets,
                int64_t nt, const double* h0, double hfact, double* hout, int32_t* route, int nthreads) {
  or_buckets B;
  buckets_init(&B, x, y, z, n);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t k = 0; k < nt; ++k) {
    int64_t a = targets[k];
    double g0 = h0[k];
    double lo = g0 / 16.0, hi = g0 * 16.0;
    double h = g0;
    int ok = 0;
    for (int it = 0; it < 30; ++it) {
      double nn, dn;
      number_density(&B, x[a], y[a], z[a], h, &nn, &dn);
      double f = h - hfact * pow(nn, -1.0 / 3.0);
      double fp = 1.0 + hfact / 3.0 * pow(nn, -4.0 / 3.0) * dn;
      double hn = h - f / fp;
      if (!(hn >= lo && hn <= hi)) break;
      if (fabs(hn - h) < 1e-10 * hn) { h = hn; ok = 1; break; }
      h = hn;
    }
    if (ok) { hout[k] = h; route[k] = 0; continue; }
    double nn, dn;
    number_density(&B, x[a], y[a], z[a], lo, &nn, &dn);
    double flo = lo - hfact * pow(nn, -1.0 / 3.0);
    number_density(&B, x[a], y[a], z[a], hi, &nn, &dn);
    double fhi = hi - hfact * pow(nn, -1.0 / 3.0);
    if (!(flo < 0.0 && fhi > 0.0)) { hout[k] = g0; route[k] = 2; continue; }
    double a0 = lo, b0 = hi;
    for (int it = 0; it < 200; ++it) {
      double m = 0.5 * (a0 + b0);
      number_density(&B, x[a], y[a], z[a], m, &nn, &dn);
      double fm = m - hfact * pow(nn, -1.0 / 3.0);
      if (fm < 0.0) a0 = m; else b0 = m;
      if (b0 - a0 < 1e-12 * m) break;
    }
    hout[k] = 0.5 * (a0 + b0);
    route[k] = 1;
  }
  buckets_free(&B);
}

/* SPH number density n(h) = sum_b W(r_ab,h) at given h (for checks and for
 * locating the densest particle). */
void or_number_density(const double* x, const double* y, const double* z, int64_t n, const int64_t* targets,
                       int64_t nt, const double* h, double* nout, int nthreads) {
  or_buckets B;
  buckets_init(&B, x, y, z, n);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t k = 0; k < nt; ++k) {
    double nn, dn;
    int64_t a = targets[k];
    number_density(&B, x[a], y[a], z[a], h[k], &nn, &dn);
    nout[k] = nn;
  }
  buckets_free(&B);
}

/* ------------------------------------------- octree and adaptive walk (Sec. III-A/B) */

/* Octree over the unit cube: a node is the cube of side 2^-level at integer
 * coordinates (ix,iy,iz); it is a leaf when it holds <= leaf_size particles
 * or level == 21.  Children are the 8 half-size cubes, visited in octant
 * order (bit 2 = x, bit 1 = y, bit 0 = z), empty ones omitted.  Labels carry
 * a leading 1 bit: root = 1, child = parent*8 + octant (Section III-A's
 * label arithmetic with 8 children: parent = label >> 3). */
typedef struct {
  int64_t label;
  int level;
  int64_t count;
  double mass, cx, cy, cz, size;
  int leaf;
  int64_t first_child, nchild; /* indices into the node array */
  int64_t pbegin, pend;        /* range in the node-ordered particle list */
} or_node;

typedef struct {
  or_node* nodes;
  int64_t nnodes, cap;
  int64_t* order; /* particle indices grouped by node (depth-first) */
} or_tree;

static int64_t cell_coord(double v, int level) {
  double s = ldexp(1.0, level);
  int64_t c = (int64_t)floor(v * s);
  int64_t m = ((int64_t)1 << level) - 1;
  if (c < 0) c = 0;
  if (c > m) c = m;
  return c;
}

static int64_t push_node(or_tree* T) {
  if (T->nnodes == T->cap) {
    T->cap = T->cap ? 2 * T->cap : 1024;
    T->nodes = (or_node*)realloc(T->nodes, T->cap * sizeof(or_node));
  }
  memset(&T->nodes[T->nnodes], 0, sizeof(or_node));
  return T->nnodes++;
}

/* Build the subtree for particles list[0..cnt) that lie in the node cube.
 * list is reordered in place so that each child's particles are contiguous. */
static void build_node(or_tree* T, int64_t id, int64_t* list, int64_t cnt, int64_t base, const double* x,
                       const double* y, const double* z, const double* m, int leaf_size) {
  or_node* nd = &T->nodes[id];
  nd->count = cnt;
  nd->pbegin = base;
  nd->pend = base + cnt;
  /* mass and centre of mass, summed in ascending particle index order in
   * extended precision, then rounded once */
  int64_t* sorted = (int64_t*)malloc(cnt * sizeof(int64_t));
  memcpy(sorted, list, cnt * sizeof(int64_t));
  for (int64_t i = 1; i < cnt; ++i) { /* insertion sort is fine: small lists dominate */
    int64_t v = sorted[i], j = i - 1;
    while (j >= 0 && sorted[j] > v) { sorted[j + 1] = sorted[j]; --j; }
    sorted[j + 1] = v;
  }
  long double M = 0, sx = 0, sy = 0, sz = 0;
  for (int64_t i = 0; i < cnt; ++i) {
    int64_t a = sorted[i];
    M += m[a]; sx += (long double)m[a] * x[a]; sy += (long double)m[a] * y[a]; sz += (long double)m[a] * z[a];
  }
  free(sorted);
  nd->mass = (double)M;
  nd->cx = (double)(sx / M); nd->cy = (double)(sy / M); nd->cz = (double)(sz / M);
  double s2 = 0.0;
  for (int64_t i = 0; i < cnt; ++i) {
    int64_t a = list[i];
    double dx = x[a] - nd->cx, dy = y[a] - nd->cy, dz = z[a] - nd->cz;
    double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 > s2) s2 = d2;
  }
  nd->size = sqrt(s2);
  if (cnt <= leaf_size || nd->level >= 21) { nd->leaf = 1; nd->nchild = 0; return; }
  /* partition into octants of the next level */
  int L = nd->level + 1;
  int64_t* tmp = (int64_t*)malloc(cnt * sizeof(int64_t));
  int64_t oc[8] = {0};
  int* oct = (int*)malloc(cnt * sizeof(int));
  for (int64_t i = 0; i < cnt; ++i) {
    int64_t a = list[i];
    int o = (int)(((cell_coord(x[a], L) & 1) << 2) | ((cell_coord(y[a], L) & 1) << 1) | (cell_coord(z[a], L) & 1));
    oct[i] = o;
    oc[o]++;
  }
  int64_t start[8], pos[8];
  start[0] = 0;
  for (int o = 1; o < 8; ++o) start[o] = start[o - 1] + oc[o - 1];
  for (int o = 0; o < 8; ++o) pos[o] = start[o];
  for (int64_t i = 0; i < cnt; ++i) tmp[pos[oct[i]]++] = list[i];
  memcpy(list, tmp, cnt * sizeof(int64_t));
  free(tmp); free(oct);
  /* children are allocated contiguously, then recursed into */
  int64_t nch = 0;
  for (int o = 0; o < 8; ++o) if (oc[o]) nch++;
  int64_t first = T->nnodes;
  int64_t lab = nd->label;
  for (int o = 0; o < 8; ++o)
    if (oc[o]) {
      int64_t cid = push_node(T);
      T->nodes[cid].label = lab * 8 + o;
      T->nodes[cid].level = L;
    }
  T->nodes[id].first_child = first;
  T->nodes[id].nchild = nch;
  int64_t k = 0;
  for (int o = 0; o < 8; ++o)
    if (oc[o]) {
      build_node(T, first + k, list + start[o], oc[o], base + start[o], x, y, z, m, leaf_size);
      ++k;
    }
}

static or_tree* g_tree = NULL;

/* Build the octree; returns the node count.  Node arrays are read with
 * or_tree_nodes and released with or_tree_free. */
int64_t or_tree_build(const double* x, const double* y, const double* z, const double* m, int64_t n,
                      int leaf_size) {
  if (g_tree) { free(g_tree->nodes); free(g_tree->order); free(g_tree); }
  g_tree = (or_tree*)calloc(1, sizeof(or_tree));
  g_tree->order = (int64_t*)malloc((n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) g_tree->order[i] = i;
  int64_t r = push_node(g_tree);
  g_tree->nodes[r].label = 1;
  g_tree->nodes[r].level = 0;
  if (n > 0) build_node(g_tree, r, g_tree->order, n, 0, x, y, z, m, leaf_size);
  return g_tree->nnodes;
}

void or_tree_nodes(int64_t* label, int32_t* level, int64_t* count, double* mass, double* com, double* size,
                   int32_t* leaf, int64_t* first_child, int64_t* nchild, int64_t* pbegin, int64_t* order) {
  for (int64_t i = 0; i < g_tree->nnodes; ++i) {
    or_node* d = &g_tree->nodes[i];
    label[i] = d->label; level[i] = d->level; count[i] = d->count; mass[i] = d->mass;
    com[3 * i] = d->cx; com[3 * i + 1] = d->cy; com[3 * i + 2] = d->cz;
    size[i] = d->size; leaf[i] = d->leaf; first_child[i] = d->first_child; nchild[i] = d->nchild;
    pbegin[i] = d->pbegin;
  }
  if (order) {
    int64_t n = g_tree->nodes[0].count;
    memcpy(order, g_tree->order, n * sizeof(int64_t));
  }
}

void or_tree_free(void) {
  if (g_tree) { free(g_tree->nodes); free(g_tree->order); free(g_tree); g_tree = NULL; }
}
