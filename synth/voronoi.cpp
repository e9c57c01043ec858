// Clipped Voronoi tessellation of point sites in the unit cube [0,1]^3.
//
// This is an input generator: it turns seeded particle positions into the
// grid the Exact mapping runs on (cells generated by the particles, as in
// Section II-A of Lau, Petkova & Bonnell 2024).  It holds none of the mapping
// arithmetic; the mapping library and the FP64 oracle both read its output.
//
// Each cell starts as the cube and is clipped by the bisector planes of its
// neighbours, visited nearest-first through a kd-tree, until no further site
// can cut it (a site at distance D gives a plane at D/2; once D/2 exceeds the
// largest vertex radius of the cell, the cell is final).
//
// Output layout (CSR, all arrays allocated by the caller after a sizing pass):
//   cell c owns faces [cell_face_off[c], cell_face_off[c+1])
//   face f owns loop entries [face_vert_off[f], face_vert_off[f+1]) of
//   face_vert, which index the global vertex arrays vx/vy/vz.  A cell's
//   vertices are its own (not shared with neighbours).  Loops are counter-
//   clockwise seen from outside the cell.  face_plane holds (nx,ny,nz,d) with
//   a unit outward normal: points x of the cell satisfy n.x <= d.
//   face_nb is the neighbouring site index, or -1-w for cube wall w
//   (w = 0..5 for x<=1, x>=0, y<=1, y>=0, z<=1, z>=0).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct V3 { double x, y, z; };
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 mul(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

// ---------------------------------------------------------------- kd-tree
struct KdNode { double lo[3], hi[3]; int begin, end, left, right; };

struct KdTree {
  std::vector<int> idx;
  std::vector<KdNode> nodes;
  const double* p;
  int build(int b, int e) {
    KdNode nd;
    for (int k = 0; k < 3; ++k) { nd.lo[k] = 1e300; nd.hi[k] = -1e300; }
    for (int i = b; i < e; ++i)
      for (int k = 0; k < 3; ++k) {
        double v = p[3 * idx[i] + k];
        nd.lo[k] = std::min(nd.lo[k], v); nd.hi[k] = std::max(nd.hi[k], v);
      }
    nd.begin = b; nd.end = e; nd.left = nd.right = -1;
    int id = (int)nodes.size();
    nodes.push_back(nd);
    if (e - b > 8) {
      int ax = 0; double ext = -1;
      for (int k = 0; k < 3; ++k) if (nd.hi[k] - nd.lo[k] > ext) { ext = nd.hi[k] - nd.lo[k]; ax = k; }
      int m = (b + e) / 2;
      std::nth_element(idx.begin() + b, idx.begin() + m, idx.begin() + e,
                       [&](int a, int c) { return p[3 * a + ax] < p[3 * c + ax]; });
      int l = build(b, m);
      int r = build(m, e);
      nodes[id].left = l; nodes[id].right = r;
    }
    return id;
  }
  void init(const double* pts, int n) {
    p = pts; idx.resize(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    nodes.reserve(2 * (n / 4 + 1));
    if (n > 0) build(0, n);
  }
  double mind2(int node, V3 q) const {
    const KdNode& nd = nodes[node];
    double qq[3] = {q.x, q.y, q.z}, d2 = 0;
    for (int k = 0; k < 3; ++k) {
      double t = 0;
      if (qq[k] < nd.lo[k]) t = nd.lo[k] - qq[k];
      else if (qq[k] > nd.hi[k]) t = qq[k] - nd.hi[k];
      d2 += t * t;
    }
    return d2;
  }
};

// ---------------------------------------------------------------- polyhedron
struct Poly {
  std::vector<V3> v;                 // vertices, relative to the site
  std::vector<std::vector<int>> f;   // loops (CCW from outside)
  std::vector<V3> fn;                // unit outward normals
  std::vector<double> fd;            // plane offsets (relative coords)
  std::vector<int> nb;               // neighbour / wall id
  double rmax2 = 0;

  void box(V3 s) {
    double lo[3] = {-s.x, -s.y, -s.z}, hi[3] = {1 - s.x, 1 - s.y, 1 - s.z};
    v.clear(); f.clear(); fn.clear(); fd.clear(); nb.clear();
    for (int i = 0; i < 8; ++i)
      v.push_back({(i & 1) ? hi[0] : lo[0], (i & 2) ? hi[1] : lo[1], (i & 4) ? hi[2] : lo[2]});
    // loops CCW seen from outside
    f.push_back({1, 3, 7, 5}); fn.push_back({1, 0, 0});  fd.push_back(hi[0]);  nb.push_back(-1);
    f.push_back({0, 4, 6, 2}); fn.push_back({-1, 0, 0}); fd.push_back(-lo[0]); nb.push_back(-2);
    f.push_back({2, 6, 7, 3}); fn.push_back({0, 1, 0});  fd.push_back(hi[1]);  nb.push_back(-3);
    f.push_back({0, 1, 5, 4}); fn.push_back({0, -1, 0}); fd.push_back(-lo[1]); nb.push_back(-4);
    f.push_back({4, 5, 7, 6}); fn.push_back({0, 0, 1});  fd.push_back(hi[2]);  nb.push_back(-5);
    f.push_back({0, 2, 3, 1}); fn.push_back({0, 0, -1}); fd.push_back(-lo[2]); nb.push_back(-6);
    update_rmax();
  }
  void update_rmax() {
    rmax2 = 0;
    for (auto& q : v) rmax2 = std::max(rmax2, dot(q, q));
  }

  // Keep the half-space n.y <= d (n unit).  Returns false if nothing changed.
  bool clip(V3 n, double d, int nbid) {
    const double scale = std::sqrt(rmax2);
    const double tol = 1e-13 * scale;
    const size_t nv = v.size();
    std::vector<double> s(nv);
    double smax = -1e300;
    for (size_t i = 0; i < nv; ++i) { s[i] = dot(n, v[i]) - d; smax = std::max(smax, s[i]); }
    if (smax <= tol) return false;
    // classify: -1 in, 0 on, +1 out
    std::vector<int> cls(nv);
    for (size_t i = 0; i < nv; ++i) cls[i] = s[i] < -tol ? -1 : (s[i] > tol ? 1 : 0);
    std::vector<int> remap(nv, -1);
    std::vector<V3> nvtx;
    std::vector<int> on_plane;  // new indices of vertices on the cutting plane
    for (size_t i = 0; i < nv; ++i)
      if (cls[i] <= 0) {
        remap[i] = (int)nvtx.size();
        nvtx.push_back(v[i]);
        if (cls[i] == 0) on_plane.push_back(remap[i]);
      }
    // intersection vertices keyed by the (sorted) edge
    std::vector<std::pair<uint64_t, int>> cut;
    auto cut_vertex = [&](int a, int b) -> int {
      int lo = std::min(a, b), hi = std::max(a, b);
      uint64_t key = ((uint64_t)lo << 32) | (uint32_t)hi;
      for (auto& kv : cut) if (kv.first == key) return kv.second;
      double t = s[a] / (s[a] - s[b]);
      V3 q = add(v[a], mul(sub(v[b], v[a]), t));
      int id = (int)nvtx.size();
      nvtx.push_back(q);
      cut.push_back({key, id});
      on_plane.push_back(id);
      return id;
    };
    std::vector<std::vector<int>> nf;
    std::vector<V3> nfn; std::vector<double> nfd; std::vector<int> nnb;
    for (size_t fi = 0; fi < f.size(); ++fi) {
      const auto& loop = f[fi];
      std::vector<int> out;
      const size_t L = loop.size();
      for (size_t k = 0; k < L; ++k) {
        int a = loop[k], b = loop[(k + 1) % L];
        if (cls[a] <= 0) out.push_back(remap[a]);
        if ((cls[a] < 0 && cls[b] > 0) || (cls[a] > 0 && cls[b] < 0)) out.push_back(cut_vertex(a, b));
      }
      // drop consecutive duplicates
      std::vector<int> o2;
      for (size_t k = 0; k < out.size(); ++k)
        if (o2.empty() || o2.back() != out[k]) o2.push_back(out[k]);
      while (o2.size() > 1 && o2.front() == o2.back()) o2.pop_back();
      if (o2.size() >= 3) { nf.push_back(o2); nfn.push_back(fn[fi]); nfd.push_back(fd[fi]); nnb.push_back(nb[fi]); }
    }
    // the new face on the cutting plane
    std::sort(on_plane.begin(), on_plane.end());
    on_plane.erase(std::unique(on_plane.begin(), on_plane.end()), on_plane.end());
    if (on_plane.size() >= 3) {
      V3 c{0, 0, 0};
      for (int id : on_plane) c = add(c, nvtx[id]);
      c = mul(c, 1.0 / on_plane.size());
      V3 a = std::fabs(n.x) < 0.6 ? V3{1, 0, 0} : V3{0, 1, 0};
      V3 u1 = cross(n, a); u1 = mul(u1, 1.0 / norm(u1));
      V3 u2 = cross(n, u1);
      std::vector<std::pair<double, int>> ang;
      for (int id : on_plane) { V3 r = sub(nvtx[id], c); ang.push_back({std::atan2(dot(r, u2), dot(r, u1)), id}); }
      std::sort(ang.begin(), ang.end());
      std::vector<int> loop;
      for (auto& p : ang) loop.push_back(p.second);
      nf.push_back(loop); nfn.push_back(n); nfd.push_back(d); nnb.push_back(nbid);
    }
    v.swap(nvtx); f.swap(nf); fn.swap(nfn); fd.swap(nfd); nb.swap(nnb);
    drop_unused();
    update_rmax();
    return true;
  }

  // remove vertices no face refers to (cheap; the O(V^2) weld runs once per cell)
  void drop_unused() {
    std::vector<int>& used = scratch_used;
    used.assign(v.size(), -1);
    std::vector<V3>& nvtx = scratch_v;
    nvtx.clear();
    for (auto& loop : f)
      for (int& id : loop) {
        if (used[id] < 0) { used[id] = (int)nvtx.size(); nvtx.push_back(v[id]); }
        id = used[id];
      }
    v.swap(nvtx);
  }
  std::vector<int> scratch_used;
  std::vector<V3> scratch_v;

  // weld near-coincident vertices, drop degenerate faces and unused vertices
  void compact() {
    const double scale = std::sqrt(std::max(rmax2, 1e-300));
    const double tol2 = (1e-11 * scale) * (1e-11 * scale);
    const size_t nv = v.size();
    std::vector<int> rep(nv);
    for (size_t i = 0; i < nv; ++i) {
      rep[i] = (int)i;
      for (size_t j = 0; j < i; ++j)
        if (rep[j] == (int)j) {
          V3 dd = sub(v[i], v[j]);
          if (dot(dd, dd) < tol2) { rep[i] = (int)j; break; }
        }
    }
    std::vector<std::vector<int>> nf;
    std::vector<V3> nfn; std::vector<double> nfd; std::vector<int> nnb;
    for (size_t fi = 0; fi < f.size(); ++fi) {
      std::vector<int> o;
      for (int id : f[fi]) { int r = rep[id]; if (o.empty() || o.back() != r) o.push_back(r); }
      while (o.size() > 1 && o.front() == o.back()) o.pop_back();
      if (o.size() >= 3) { nf.push_back(o); nfn.push_back(fn[fi]); nfd.push_back(fd[fi]); nnb.push_back(nb[fi]); }
    }
    std::vector<int> used(nv, -1);
    std::vector<V3> nvtx;
    for (auto& loop : nf)
      for (int& id : loop) {
        if (used[id] < 0) { used[id] = (int)nvtx.size(); nvtx.push_back(v[id]); }
        id = used[id];
      }
    v.swap(nvtx); f.swap(nf); fn.swap(nfn); fd.swap(nfd); nb.swap(nnb);
  }
};

struct CellOut {
  std::vector<V3> v;                 // absolute
  std::vector<std::vector<int>> f;
  std::vector<V3> fn; std::vector<double> fd; std::vector<int> nb;
};

void make_cell(const double* pts, int n, const KdTree& kd, int i, CellOut& out) {
  V3 s{pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
  Poly P;
  P.box(s);
  // best-first traversal over the kd-tree, nearest nodes first
  std::vector<std::pair<double, int>> heap;  // (min dist^2, node), min-heap
  auto cmp = [](const std::pair<double, int>& a, const std::pair<double, int>& b) { return a.first > b.first; };
  if (!kd.nodes.empty()) heap.push_back({kd.mind2(0, s), 0});
  std::vector<std::pair<double, int>> cand;
  while (!heap.empty()) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    auto top = heap.back(); heap.pop_back();
    if (top.first >= 4.0 * P.rmax2) break;   // (D/2)^2 >= rmax^2: no cut possible
    const KdNode& nd = kd.nodes[top.second];
    if (nd.left < 0) {
      cand.clear();
      for (int k = nd.begin; k < nd.end; ++k) {
        int j = kd.idx[k];
        if (j == i) continue;
        V3 q{pts[3 * j], pts[3 * j + 1], pts[3 * j + 2]};
        V3 dd = sub(q, s);
        cand.push_back({dot(dd, dd), j});
      }
      std::sort(cand.begin(), cand.end());
      for (auto& c : cand) {
        if (c.first >= 4.0 * P.rmax2) break;
        if (c.first <= 0) continue;  // coincident site: no bisector
        int j = c.second;
        V3 q{pts[3 * j], pts[3 * j + 1], pts[3 * j + 2]};
        V3 dd = sub(q, s);
        double len = std::sqrt(c.first);
        P.clip(mul(dd, 1.0 / len), 0.5 * len, j);
      }
    } else {
      heap.push_back({kd.mind2(nd.left, s), nd.left}); std::push_heap(heap.begin(), heap.end(), cmp);
      heap.push_back({kd.mind2(nd.right, s), nd.right}); std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
  P.compact();
  out.v.resize(P.v.size());
  for (size_t k = 0; k < P.v.size(); ++k) out.v[k] = add(s, P.v[k]);
  out.f = P.f; out.fn = P.fn; out.nb = P.nb;
  out.fd.resize(P.fd.size());
  for (size_t k = 0; k < P.fd.size(); ++k) {
    int w = P.nb[k];
    if (w < 0) {
      // walls are exact: x<=1, x>=0, ...
      out.fd[k] = ((-1 - w) % 2 == 0) ? 1.0 : 0.0;
    } else {
      // bisector through the midpoint of the two sites
      V3 q{pts[3 * w], pts[3 * w + 1], pts[3 * w + 2]};
      out.fd[k] = dot(P.fn[k], mul(add(s, q), 0.5));
    }
  }
}

struct Tess {
  std::vector<CellOut> cells;
};

}  // namespace

extern "C" {

// Phase 1: tessellate; returns an opaque handle and the sizes of the CSR arrays.
void* vor_build(const double* pts, int64_t n, int nthreads, int64_t* nface, int64_t* nloop, int64_t* nvert) {
  KdTree kd;
  kd.init(pts, (int)n);
  Tess* T = new Tess;
  T->cells.resize(n);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t i = 0; i < n; ++i) make_cell(pts, (int)n, kd, (int)i, T->cells[i]);
  int64_t F = 0, L = 0, V = 0;
  for (auto& c : T->cells) {
    F += c.f.size(); V += c.v.size();
    for (auto& lp : c.f) L += lp.size();
  }
  *nface = F; *nloop = L; *nvert = V;
  return T;
}

// Phase 2: copy into caller-allocated arrays and free the handle.
void vor_fill(void* h, int64_t* cell_face_off, int64_t* face_vert_off, int32_t* face_vert,
              int32_t* face_nb, double* face_plane, double* vx, double* vy, double* vz) {
  Tess* T = (Tess*)h;
  int64_t F = 0, L = 0, V = 0;
  cell_face_off[0] = 0; face_vert_off[0] = 0;
  for (size_t c = 0; c < T->cells.size(); ++c) {
    const CellOut& C = T->cells[c];
    for (size_t k = 0; k < C.v.size(); ++k) { vx[V + k] = C.v[k].x; vy[V + k] = C.v[k].y; vz[V + k] = C.v[k].z; }
    for (size_t fi = 0; fi < C.f.size(); ++fi) {
      for (int id : C.f[fi]) face_vert[L++] = (int32_t)(V + id);
      face_nb[F] = C.nb[fi];
      face_plane[4 * F + 0] = C.fn[fi].x; face_plane[4 * F + 1] = C.fn[fi].y;
      face_plane[4 * F + 2] = C.fn[fi].z; face_plane[4 * F + 3] = C.fd[fi];
      ++F;
      face_vert_off[F] = L;
    }
    V += C.v.size();
    cell_face_off[c + 1] = F;
  }
  delete T;
}

void vor_free(void* h) { delete (Tess*)h; }

}  // extern "C"
