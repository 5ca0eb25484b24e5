// Periodic Voronoi tessellation of a jittered cubic lattice, by half-space clipping.
//
// Input generator only: it builds the static unstructured mesh that the RT
// subcycle runs on (the paper's method works on AREPO's Voronoi mesh, Sec. 2.1,
// which is rebuilt once per hydro step and held fixed over the RT subcycles,
// Sec. 2.3).  It computes geometry (volumes, centroids, face areas, normals,
// face centroids) and nothing of the radiative-transfer arithmetic.
//
// Method.  Generator p lies inside lattice cell (i,j,k) of an n^3 lattice of
// spacing h = L/n.  Its Voronoi cell starts as a large cube centred on the
// generator and is clipped, in order of increasing distance, by the bisector
// half-space {x : x.d <= |d|^2/2} of every generator (periodic image) in the
// (2K+1)^3 block of lattice cells around it.  Clipping stops once the next
// candidate is farther than twice the cell's current circumradius ("security
// radius"); if generators outside the block could still cut, K grows.
// Each face keeps the index of the generator that made it.  Intersection
// vertices on an edge are shared between the two faces meeting there, so the
// new face made by a cut is chained from the cut segments without sorting.
//
// Output.  One record per cell (volume, centroid) and one per face pair i<j,
// with the geometry taken from cell i's polyhedron: left=i, right=j, unit
// normal from generator i towards generator j (image), area, centroid.
// All positions are wrapped into [0, L).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <algorithm>
#include <array>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using V3 = std::array<double, 3>;

inline V3 sub(const V3& a, const V3& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
inline V3 add(const V3& a, const V3& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
inline V3 scl(const V3& a, double s) { return {a[0] * s, a[1] * s, a[2] * s}; }
inline double dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline V3 cross(const V3& a, const V3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}

struct FaceOut {
  int32_t nbr;   // generator index of the neighbour (-1: initial box face)
  V3 d;          // neighbour image position relative to this generator
  double area;   // area (projected on d/|d|)
  V3 centroid;   // relative to this generator
};

struct CellOut {
  double volume;
  V3 centroid;   // relative to this generator
  std::vector<FaceOut> faces;
  int status;    // 0 ok, 1 open cell (K too small), 2 topology failure
};

// Convex polyhedron as vertex positions plus face loops (CCW seen from outside).
struct Poly {
  std::vector<V3> v;
  std::vector<int> loop;           // concatenated loops
  std::vector<int> fstart, flen;   // per face
  std::vector<int> fnbr;           // per face neighbour id (-1 = box)
  std::vector<V3> fd;              // per face: neighbour displacement

  void clear() { v.clear(); loop.clear(); fstart.clear(); flen.clear(); fnbr.clear(); fd.clear(); }

  void init_box(double H) {
    clear();
    for (int k = 0; k < 8; ++k)
      v.push_back({(k & 1) ? H : -H, (k & 2) ? H : -H, (k & 4) ? H : -H});
    // faces with outward CCW loops
    const int f[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
    for (int q = 0; q < 6; ++q) {
      fstart.push_back((int)loop.size());
      flen.push_back(4);
      fnbr.push_back(-1);
      fd.push_back({0, 0, 0});
      for (int t = 0; t < 4; ++t) loop.push_back(f[q][t]);
    }
  }

  double max_r2() const {
    double m = 0;
    for (const V3& p : v) m = std::max(m, dot(p, p));
    return m;
  }
};

struct Scratch {
  std::vector<double> sd;
  std::vector<int> remap;
  std::vector<std::array<int, 3>> ecache;  // (a, b, new id) with a<b
  std::vector<std::pair<int, int>> seg;    // cut-face edges: from -> to
  Poly out;
};

// Clip poly by {x : x.d <= |d|^2/2}.  Returns 0 ok / no-op, 2 on topology failure.
int clip(Poly& P, const V3& d, int nbr, Scratch& S, double eps) {
  const double c = 0.5 * dot(d, d);
  const int nv = (int)P.v.size();
  S.sd.resize(nv);
  bool any_out = false, any_in = false;
  for (int i = 0; i < nv; ++i) {
    S.sd[i] = dot(P.v[i], d) - c;
    if (S.sd[i] > eps) any_out = true; else any_in = true;
  }
  if (!any_out) return 0;
  if (!any_in) return 2;
  Poly& Q = S.out;
  Q.clear();
  S.remap.assign(nv, -1);
  for (int i = 0; i < nv; ++i)
    if (S.sd[i] <= eps) { S.remap[i] = (int)Q.v.size(); Q.v.push_back(P.v[i]); }
  S.ecache.clear();
  S.seg.clear();
  auto xvert = [&](int a, int b) -> int {
    int lo = std::min(a, b), hi = std::max(a, b);
    for (auto& e : S.ecache) if (e[0] == lo && e[1] == hi) return e[2];
    // interpolate from the lower id for a result independent of the traversal direction
    double sl = S.sd[lo], sh = S.sd[hi];
    double t = sl / (sl - sh);
    V3 p = add(P.v[lo], scl(sub(P.v[hi], P.v[lo]), t));
    int id = (int)Q.v.size();
    Q.v.push_back(p);
    S.ecache.push_back({lo, hi, id});
    return id;
  };
  const int nf = (int)P.fstart.size();
  for (int f = 0; f < nf; ++f) {
    const int s0 = P.fstart[f], n = P.flen[f];
    int start = (int)Q.loop.size();
    int xin = -1, xout = -1, ncross = 0;
    for (int t = 0; t < n; ++t) {
      int a = P.loop[s0 + t], b = P.loop[s0 + (t + 1) % n];
      bool ain = S.sd[a] <= eps, bin = S.sd[b] <= eps;
      if (ain) Q.loop.push_back(S.remap[a]);
      if (ain && !bin) { xout = xvert(a, b); Q.loop.push_back(xout); ++ncross; }
      else if (!ain && bin) { xin = xvert(a, b); Q.loop.push_back(xin); ++ncross; }
    }
    int len = (int)Q.loop.size() - start;
    if (ncross != 0 && ncross != 2) return 2;
    if (len < 3) { Q.loop.resize(start); continue; }  // face removed (or degenerate)
    Q.fstart.push_back(start);
    Q.flen.push_back(len);
    Q.fnbr.push_back(P.fnbr[f]);
    Q.fd.push_back(P.fd[f]);
    if (ncross == 2) S.seg.push_back({xin, xout});  // cut face runs xin -> xout
  }
  // chain the cut face
  if (S.seg.size() < 3) return 2;
  int start = (int)Q.loop.size();
  int first = S.seg[0].first, cur = first;
  for (size_t it = 0; it <= S.seg.size(); ++it) {
    Q.loop.push_back(cur);
    int nxt = -1;
    for (auto& sg : S.seg) if (sg.first == cur) { nxt = sg.second; break; }
    if (nxt < 0) return 2;
    cur = nxt;
    if (cur == first) break;
  }
  if (cur != first || (int)Q.loop.size() - start != (int)S.seg.size()) return 2;
  Q.fstart.push_back(start);
  Q.flen.push_back((int)S.seg.size());
  Q.fnbr.push_back(nbr);
  Q.fd.push_back(d);
  std::swap(P, Q);
  return 0;
}

void finish(const Poly& P, CellOut& co) {
  co.faces.clear();
  double vol = 0;
  V3 cen = {0, 0, 0};
  const int nf = (int)P.fstart.size();
  for (int f = 0; f < nf; ++f) {
    const int s0 = P.fstart[f], n = P.flen[f];
    V3 nrm;
    double h;  // distance of the face plane from the origin
    if (P.fnbr[f] >= 0) {
      double dl = std::sqrt(dot(P.fd[f], P.fd[f]));
      nrm = scl(P.fd[f], 1.0 / dl);
      h = 0.5 * dl;
    } else {
      V3 a = {0, 0, 0};
      for (int t = 0; t < n; ++t) a = add(a, cross(P.v[P.loop[s0 + t]], P.v[P.loop[s0 + (t + 1) % n]]));
      double al = std::sqrt(dot(a, a));
      nrm = scl(a, 1.0 / al);
      h = dot(P.v[P.loop[s0]], nrm);
    }
    const V3& p0 = P.v[P.loop[s0]];
    double area = 0;
    V3 fc = {0, 0, 0};
    for (int t = 1; t + 1 < n; ++t) {
      const V3& p1 = P.v[P.loop[s0 + t]];
      const V3& p2 = P.v[P.loop[s0 + t + 1]];
      double ak = 0.5 * dot(cross(sub(p1, p0), sub(p2, p0)), nrm);
      area += ak;
      fc = add(fc, scl(add(add(p0, p1), p2), ak / 3.0));
      double vk = ak * h / 3.0;  // tetrahedron (origin, p0, p1, p2)
      vol += vk;
      cen = add(cen, scl(add(add(p0, p1), p2), vk / 4.0));
    }
    if (area > 0) fc = scl(fc, 1.0 / area);
    co.faces.push_back({P.fnbr[f], P.fd[f], area, fc});
  }
  co.volume = vol;
  co.centroid = vol > 0 ? scl(cen, 1.0 / vol) : V3{0, 0, 0};
}

struct Built {
  int64_t C = 0;
  std::vector<double> vol, cx, cy, cz;
  std::vector<int32_t> left, right;
  std::vector<double> area, nx, ny, nz, fx, fy, fz;
  int64_t n_asym = 0;     // faces seen from one side only (tiny, dropped)
  double max_asym_area = 0;
};

inline double wrap(double x, double L) {
  double y = std::fmod(x, L);
  if (y < 0) y += L;
  if (y >= L) y -= L;
  return y;
}

}  // namespace

extern "C" {

// Build the tessellation.  Generators: C = n^3 points, p = i + n*(j + n*k) lies in
// lattice cell (i,j,k) of spacing L/n.  Returns an opaque handle (nullptr on error,
// message in err).  nthreads <= 0 uses the OpenMP default.
void* vor_build(int n, double L, const double* px, const double* py, const double* pz,
                int nthreads, char* err, int errlen) {
  auto fail = [&](const char* msg) -> void* {
    if (err && errlen > 0) { std::snprintf(err, errlen, "%s", msg); }
    return nullptr;
  };
  if (n < 5) return fail("vor_build: lattice must have n >= 5 per side");
  const int64_t C = (int64_t)n * n * n;
  const double h = L / n;
  // largest offset of a generator from its lattice-cell centre, in units of h
  double a = 0;
  for (int64_t p = 0; p < C; ++p) {
    int i = (int)(p % n), j = (int)((p / n) % n), k = (int)(p / ((int64_t)n * n));
    double ox = std::fabs(px[p] / h - (i + 0.5)), oy = std::fabs(py[p] / h - (j + 0.5)),
           oz = std::fabs(pz[p] / h - (k + 0.5));
    a = std::max(a, std::max(ox, std::max(oy, oz)));
  }
  if (a >= 0.5) return fail("vor_build: a generator lies outside its lattice cell");
  std::vector<CellOut> cells(C);
  int64_t nbad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : nbad)
  {
    Poly P;
    Scratch S;
    std::vector<std::pair<double, int64_t>> cand;   // (dist^2, packed index)
    std::vector<V3> cd;
    std::vector<int32_t> cid;
#pragma omp for schedule(dynamic, 256)
    for (int64_t p = 0; p < C; ++p) {
      const int i = (int)(p % n), j = (int)((p / n) % n), k = (int)(p / ((int64_t)n * n));
      const V3 s = {px[p], py[p], pz[p]};
      int status = 1;
      for (int K = 2; K <= (n - 1) / 2 && status == 1; ++K) {
        cand.clear(); cd.clear(); cid.clear();
        for (int dk = -K; dk <= K; ++dk)
          for (int dj = -K; dj <= K; ++dj)
            for (int di = -K; di <= K; ++di) {
              if (!di && !dj && !dk) continue;
              int ii = i + di, jj = j + dj, kk = k + dk;
              double shx = 0, shy = 0, shz = 0;
              if (ii < 0) { ii += n; shx = -L; } else if (ii >= n) { ii -= n; shx = L; }
              if (jj < 0) { jj += n; shy = -L; } else if (jj >= n) { jj -= n; shy = L; }
              if (kk < 0) { kk += n; shz = -L; } else if (kk >= n) { kk -= n; shz = L; }
              int64_t q = ii + (int64_t)n * (jj + (int64_t)n * kk);
              V3 d = {px[q] + shx - s[0], py[q] + shy - s[1], pz[q] + shz - s[2]};
              cand.push_back({dot(d, d), (int64_t)cd.size()});
              cd.push_back(d);
              cid.push_back((int32_t)q);
            }
        std::sort(cand.begin(), cand.end());
        P.init_box((K + 1) * h);
        const double eps = 1e-13 * h * h;
        int st = 0;
        for (auto& cnd : cand) {
          double r2 = P.max_r2();
          if (cnd.first > 4.0 * r2) break;  // cannot cut any more
          st = clip(P, cd[cnd.second], cid[cnd.second], S, eps);
          if (st) break;
        }
        if (st) { status = 2; break; }
        // completeness: generators outside the block are at least (K+1-2a)h away
        double dout = (K + 1 - 2 * a) * h;
        bool open = false;
        for (int f : P.fnbr) if (f < 0) open = true;
        if (!open && 4.0 * P.max_r2() < dout * dout) status = 0;
      }
      CellOut& co = cells[p];
      co.status = status;
      if (status == 0) finish(P, co);
      else ++nbad;
    }
  }
  if (nbad) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "vor_build: %lld cells failed (open or degenerate)", (long long)nbad);
    return fail(msg);
  }
  Built* B = new Built;
  B->C = C;
  B->vol.resize(C); B->cx.resize(C); B->cy.resize(C); B->cz.resize(C);
  for (int64_t p = 0; p < C; ++p) {
    B->vol[p] = cells[p].volume;
    B->cx[p] = wrap(px[p] + cells[p].centroid[0], L);
    B->cy[p] = wrap(py[p] + cells[p].centroid[1], L);
    B->cz[p] = wrap(pz[p] + cells[p].centroid[2], L);
  }
  // faces: pair (p, q) with p < q, geometry from p; check that q sees p
  const double tiny = 1e-9 * h * h;
  for (int64_t p = 0; p < C; ++p) {
    for (const FaceOut& f : cells[p].faces) {
      if (f.nbr < 0) continue;
      if (f.nbr == p) { delete B; return fail("vor_build: self neighbour (box too small)"); }
      const CellOut& other = cells[f.nbr];
      bool seen = false;
      for (const FaceOut& g : other.faces) if (g.nbr == p) { seen = true; break; }
      if (!seen) {
        ++B->n_asym;
        B->max_asym_area = std::max(B->max_asym_area, f.area);
        if (f.area > tiny) { delete B; return fail("vor_build: face seen from one side only"); }
        continue;
      }
      if (f.nbr < p) continue;
      if (f.area <= 0) continue;
      double dl = std::sqrt(dot(f.d, f.d));
      B->left.push_back((int32_t)p);
      B->right.push_back(f.nbr);
      B->area.push_back(f.area);
      B->nx.push_back(f.d[0] / dl); B->ny.push_back(f.d[1] / dl); B->nz.push_back(f.d[2] / dl);
      B->fx.push_back(wrap(px[p] + f.centroid[0], L));
      B->fy.push_back(wrap(py[p] + f.centroid[1], L));
      B->fz.push_back(wrap(pz[p] + f.centroid[2], L));
    }
  }
  return B;
}

int64_t vor_num_faces(void* h) { return h ? (int64_t)((Built*)h)->left.size() : -1; }
int64_t vor_num_asym(void* h) { return h ? ((Built*)h)->n_asym : -1; }

void vor_fetch(void* h, double* vol, double* cx, double* cy, double* cz, int32_t* left, int32_t* right,
               double* area, double* nx, double* ny, double* nz, double* fx, double* fy, double* fz) {
  Built* B = (Built*)h;
  const size_t C = (size_t)B->C, F = B->left.size();
  std::memcpy(vol, B->vol.data(), C * 8); std::memcpy(cx, B->cx.data(), C * 8);
  std::memcpy(cy, B->cy.data(), C * 8); std::memcpy(cz, B->cz.data(), C * 8);
  std::memcpy(left, B->left.data(), F * 4); std::memcpy(right, B->right.data(), F * 4);
  std::memcpy(area, B->area.data(), F * 8);
  std::memcpy(nx, B->nx.data(), F * 8); std::memcpy(ny, B->ny.data(), F * 8); std::memcpy(nz, B->nz.data(), F * 8);
  std::memcpy(fx, B->fx.data(), F * 8); std::memcpy(fy, B->fy.data(), F * 8); std::memcpy(fz, B->fz.data(), F * 8);
}

void vor_free(void* h) { delete (Built*)h; }

}  // extern "C"
