// Host side of libucns: mesh topology (periodic node identification, face
// pairing, Morton cell order) and the FP64 precompute of ucns_precompute
// (cell geometry, face quadrature, stencils, least-squares pseudo-inverses by
// Householder QR, Eq. 4).  Produces structure-of-arrays host buffers in the
// internal cell order; api.cu uploads them.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "basis.hpp"
#include "host_arrays.hpp"
#include "ucns_internal.hpp"

namespace ucns {
namespace {

// VTK hexahedron: reference corners and faces ordered so (p2-p0)x(p3-p1)
// points out of the cell.
const int kHexCorner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                              {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
const int kHexFace[6][4] = {{0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4},
                            {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};
// tetrahedron faces ordered so (p1-p0)x(p2-p0) points out of a positive tet
const int kTetFace[4][3] = {{0, 2, 1}, {0, 1, 3}, {1, 2, 3}, {0, 3, 2}};
// triangular prism (base 0 1 2 counter-clockwise seen from the top 3 4 5,
// node k + 3 above node k): two triangles, then the three side quads, each
// ordered so that its area vector points out of the cell
const int kPrismFace[5][4] = {{0, 2, 1, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
// pyramid (base 0 1 2 3 counter-clockwise seen from the apex 4): the base
// quad, then the four side triangles, outward
const int kPyramidFace[5][4] = {{0, 3, 2, 1}, {0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}};

const int* face_local_nodes(int npc, int lf) {
  switch (npc) {
    case 8: return kHexFace[lf];
    case 6: return kPrismFace[lf];
    case 5: return kPyramidFace[lf];
    default: return kTetFace[lf];
  }
}
// nodes of local face lf: 4 (quadrilateral) or 3 (triangle)
int face_node_count(int npc, int lf) {
  switch (npc) {
    case 8: return 4;
    case 6: return lf < 2 ? 3 : 4;
    case 5: return lf == 0 ? 4 : 3;
    default: return 3;
  }
}

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double comp(V3 a, int d) { return d == 0 ? a.x : (d == 1 ? a.y : a.z); }

// Gauss-Legendre points/weights on [0,1]: closed form for n = 1, 2, 3; for
// larger n the roots of P_n by Newton's iteration from Chebyshev guesses,
// w = 2 / ((1 - t^2) P_n'(t)^2) on [-1, 1], mapped to [0, 1].
void gauss01(int n, double* x, double* w) {
  if (n == 1) {
    x[0] = 0.5;
    w[0] = 1.0;
  } else if (n == 2) {
    double d = 0.5 / std::sqrt(3.0);
    x[0] = 0.5 - d; x[1] = 0.5 + d;
    w[0] = w[1] = 0.5;
  } else if (n == 3) {
    double d = 0.5 * std::sqrt(0.6);
    x[0] = 0.5 - d; x[1] = 0.5; x[2] = 0.5 + d;
    w[0] = 5.0 / 18.0; w[1] = 4.0 / 9.0; w[2] = 5.0 / 18.0;
  } else {
    for (int i = 0; i < n; i++) {
      double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
      for (int it = 0; it < 100; it++) {
        double p0 = 1.0, p1 = t;  // P_0, P_1; recurrence (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}
        for (int k = 1; k < n; k++) {
          const double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
          p0 = p1;
          p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        const double dt = p1 / dp;
        t -= dt;
        if (std::fabs(dt) < 1e-16) break;
      }
      // recompute the derivative at the converged root
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < n; k++) {
        const double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      x[n - 1 - i] = 0.5 * (1.0 + t);
      w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);
    }
  }
}

struct CellPts {
  V3 p[8];
};

CellPts load_cell(const ucns_mesh* m, int64_t user) {
  CellPts c;
  for (int a = 0; a < m->npc; a++) {
    const double* x = &m->X[3 * m->C[user * m->npc + a]];
    c.p[a] = {x[0], x[1], x[2]};
  }
  return c;
}

// Map the unit cube onto the cell: trilinear (hex) or collapsed (tet).
void map_point(int npc, const CellPts& c, double s, double t, double u, V3* x, double* jac) {
  if (npc == 8) {
    V3 xs{0, 0, 0}, ds{0, 0, 0}, dt{0, 0, 0}, du{0, 0, 0};
    for (int a = 0; a < 8; a++) {
      double fs = kHexCorner[a][0] ? s : 1 - s, ft = kHexCorner[a][1] ? t : 1 - t,
             fu = kHexCorner[a][2] ? u : 1 - u;
      double gs = kHexCorner[a][0] ? 1 : -1, gt = kHexCorner[a][1] ? 1 : -1,
             gu = kHexCorner[a][2] ? 1 : -1;
      xs = xs + (fs * ft * fu) * c.p[a];
      ds = ds + (gs * ft * fu) * c.p[a];
      dt = dt + (fs * gt * fu) * c.p[a];
      du = du + (fs * ft * gu) * c.p[a];
    }
    *x = xs;
    *jac = dot(ds, cross(dt, du));
  } else if (npc == 6) {
    // prism: the base and top triangles' collapsed maps B(s, t) = P0 + s e1 +
    // s t e2 (and T likewise), linear in between: x = (1 - u) B + u T
    const V3 e1 = c.p[1] - c.p[0], e2 = c.p[2] - c.p[1], f1 = c.p[4] - c.p[3], f2 = c.p[5] - c.p[4];
    const V3 B = c.p[0] + s * e1 + (s * t) * e2, T = c.p[3] + s * f1 + (s * t) * f2;
    *x = (1 - u) * B + u * T;
    const V3 ds = (1 - u) * (e1 + t * e2) + u * (f1 + t * f2);
    const V3 dt = (1 - u) * (s * e2) + u * (s * f2);
    const V3 du = T - B;
    *jac = dot(ds, cross(dt, du));
  } else if (npc == 5) {
    // pyramid: the base's bilinear map Q(s, t) shrunk onto the apex: x = (1 - u) Q + u P4
    const V3 Q = ((1 - s) * (1 - t)) * c.p[0] + (s * (1 - t)) * c.p[1] + (s * t) * c.p[2] + ((1 - s) * t) * c.p[3];
    const V3 Qs = (1 - t) * (c.p[1] - c.p[0]) + t * (c.p[2] - c.p[3]);
    const V3 Qt = (1 - s) * (c.p[3] - c.p[0]) + s * (c.p[2] - c.p[1]);
    *x = (1 - u) * Q + u * c.p[4];
    *jac = dot((1 - u) * Qs, cross((1 - u) * Qt, c.p[4] - Q));
  } else {
    V3 e1 = c.p[1] - c.p[0], e2 = c.p[2] - c.p[1], e3 = c.p[3] - c.p[2];
    *x = c.p[0] + s * e1 + (s * t) * e2 + (s * t * u) * e3;
    double vol6 = dot(c.p[1] - c.p[0], cross(c.p[2] - c.p[0], c.p[3] - c.p[0]));
    *jac = s * s * t * vol6;
  }
}

struct Geom {
  double V;
  V3 c;
  double h;
  double S[6];  // (1/V) int xi_a xi_b, xi = (x - c)/h: xx yy zz xy xz yz
};

Geom cell_geometry(const ucns_mesh* m, int64_t user) {
  CellPts cp = load_cell(m, user);
  double gx[3], gw[3];
  gauss01(3, gx, gw);  // exact: hex integrands are degree <= 4 per direction, tet <= 3
  Geom g{};
  double V = 0;
  V3 mx{0, 0, 0};
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int q = 0; q < 3; q++) {
        V3 x;
        double j;
        map_point(m->npc, cp, gx[a], gx[b], gx[q], &x, &j);
        double w = gw[a] * gw[b] * gw[q] * j;
        V += w;
        mx = mx + w * x;
      }
  g.V = V;
  g.c = (1.0 / V) * mx;
  g.h = std::cbrt(V);
  double S[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int q = 0; q < 3; q++) {
        V3 x;
        double j;
        map_point(m->npc, cp, gx[a], gx[b], gx[q], &x, &j);
        double w = gw[a] * gw[b] * gw[q] * j;
        V3 y = (1.0 / g.h) * (x - g.c);
        S[0] += w * y.x * y.x; S[1] += w * y.y * y.y; S[2] += w * y.z * y.z;
        S[3] += w * y.x * y.y; S[4] += w * y.x * y.z; S[5] += w * y.y * y.z;
      }
  for (int k = 0; k < 6; k++) g.S[k] = S[k] / V;
  return g;
}

// Central moments of a cell up to degree kMomDeg: mean over the cell of
// (x - c)^b, indexed by mom_index(b); degree kMomDeg = 6 suffices for the
// smoothness indicators of a quartic (products of two cubic derivatives).
constexpr int kMomDeg = 6;
int mom_index(int a, int b, int c) { return (a * (kMomDeg + 1) + b) * (kMomDeg + 1) + c; }
constexpr int kMomSlots = (kMomDeg + 1) * (kMomDeg + 1) * (kMomDeg + 1);

// mean over the cell of (x - c)^b for every |b| <= kMomDeg (slots with a
// larger total degree stay zero), by a 5-point Gauss rule per direction:
// exact for a degree-6 monomial times the trilinear Jacobian (degree <= 8
// per direction on the unit cube)
void central_moments(const ucns_mesh* m, int64_t user, const Geom& g, double* mu) {
  CellPts cp = load_cell(m, user);
  double gx[5], gw[5];
  gauss01(5, gx, gw);
  for (int k = 0; k < kMomSlots; k++) mu[k] = 0.0;
  for (int a = 0; a < 5; a++)
    for (int b = 0; b < 5; b++)
      for (int q = 0; q < 5; q++) {
        V3 x;
        double j;
        map_point(m->npc, cp, gx[a], gx[b], gx[q], &x, &j);
        const double w = gw[a] * gw[b] * gw[q] * j / g.V;
        const V3 y = x - g.c;
        double px[kMomDeg + 1], py[kMomDeg + 1], pz[kMomDeg + 1];
        px[0] = py[0] = pz[0] = 1.0;
        for (int e = 1; e <= kMomDeg; e++) {
          px[e] = px[e - 1] * y.x;
          py[e] = py[e - 1] * y.y;
          pz[e] = pz[e - 1] * y.z;
        }
        for (int ea = 0; ea <= kMomDeg; ea++)
          for (int eb = 0; ea + eb <= kMomDeg; eb++)
            for (int ec = 0; ea + eb + ec <= kMomDeg; ec++) mu[mom_index(ea, eb, ec)] += w * px[ea] * py[eb] * pz[ec];
      }
}

double binom(int n, int k) {
  double r = 1.0;
  for (int j = 1; j <= k; j++) r = r * (n - k + j) / j;
  return r;
}
// n (n-1) ... (n-k+1)
double falling(int n, int k) {
  double r = 1.0;
  for (int j = 0; j < k; j++) r *= (double)(n - j);
  return r;
}

// Face quadrature of an owner-local face: points and owner-outward area vectors.
int face_points(const ucns_mesh* m, int64_t owner_user, int lf, int order, V3* x, V3* dS) {
  CellPts cp = load_cell(m, owner_user);
  const int* fl = face_local_nodes(m->npc, lf);
  if (face_node_count(m->npc, lf) == 4) {
    V3 Q0 = cp.p[fl[0]], Q1 = cp.p[fl[1]], Q2 = cp.p[fl[2]], Q3 = cp.p[fl[3]];
    double gx[kMaxOrder], gw[kMaxOrder];
    gauss01(order, gx, gw);
    int q = 0;
    for (int ia = 0; ia < order; ia++)
      for (int ib = 0; ib < order; ib++, q++) {
        double s = gx[ia], t = gx[ib];
        x[q] = ((1 - s) * (1 - t)) * Q0 + (s * (1 - t)) * Q1 + (s * t) * Q2 + ((1 - s) * t) * Q3;
        V3 da = (1 - t) * (Q1 - Q0) + t * (Q2 - Q3);
        V3 db = (1 - s) * (Q3 - Q0) + s * (Q2 - Q1);
        dS[q] = (gw[ia] * gw[ib]) * cross(da, db);
      }
    return q;
  }
  V3 Q0 = cp.p[fl[0]], Q1 = cp.p[fl[1]], Q2 = cp.p[fl[2]];
  if (order == 1) {
    x[0] = (1.0 / 3.0) * (Q0 + Q1 + Q2);
    dS[0] = 0.5 * cross(Q1 - Q0, Q2 - Q0);
    return 1;
  }
  // collapsed 2x2 Gauss on the triangle (exact to degree 2)
  double gx[2], gw[2];
  gauss01(2, gx, gw);
  V3 e1 = Q1 - Q0, e2 = Q2 - Q1, nrm = cross(e1, e2);
  int q = 0;
  for (int ia = 0; ia < 2; ia++)
    for (int ib = 0; ib < 2; ib++, q++) {
      double a = gx[ia], b = gx[ib];
      x[q] = Q0 + a * e1 + (a * b) * e2;
      dS[q] = (gw[ia] * gw[ib] * a) * nrm;
    }
  return q;
}

// ---------------------------------------------------------------- topology
struct QKey {
  int64_t k[3];
  bool operator==(const QKey& o) const { return k[0] == o.k[0] && k[1] == o.k[1] && k[2] == o.k[2]; }
};
struct QKeyHash {
  size_t operator()(const QKey& q) const {
    uint64_t h = 1469598103934665603ull;
    for (int d = 0; d < 3; d++) {
      h ^= (uint64_t)q.k[d];
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

}  // namespace

int build_topology(ucns_mesh* m) {
  const int64_t N = m->N, nn = m->nn;
  const int npc = m->npc;
  for (int64_t k = 0; k < N * npc; k++)
    if (m->C[k] < 0 || m->C[k] >= nn) return fail(UCNS_ERR_MESH, "cell node id out of range");
  // periodic node identification: quantised wrapped coordinates
  double scale = std::max(std::max(m->L[0], m->L[1]), m->L[2]);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t n = 0; n < nn; n++)
    for (int d = 0; d < 3; d++) {
      lo[d] = std::min(lo[d], m->X[3 * n + d]);
      hi[d] = std::max(hi[d], m->X[3 * n + d]);
    }
  for (int d = 0; d < 3; d++) scale = std::max(scale, hi[d] - lo[d]);
  const double quantum = 1e-8 * (scale > 0 ? scale : 1.0);
  m->canon.assign(nn, 0);
  {
    std::unordered_map<QKey, int64_t, QKeyHash> first;
    first.reserve((size_t)nn * 2);
    for (int64_t n = 0; n < nn; n++) {
      QKey q;
      for (int d = 0; d < 3; d++) {
        double x = m->X[3 * n + d];
        if (m->per[d]) {
          x -= m->L[d] * std::floor(x / m->L[d]);
          if (x > m->L[d] * (1.0 - 1e-9)) x -= m->L[d];
        }
        q.k[d] = std::llround(x / quantum);
      }
      auto it = first.emplace(q, n);
      m->canon[n] = it.first->second;
    }
  }
  // Morton order of the vertex means (ties by user id)
  std::vector<std::pair<uint64_t, int64_t>> key(N);
  for (int64_t c = 0; c < N; c++) {
    double s[3] = {0, 0, 0};
    for (int a = 0; a < npc; a++)
      for (int d = 0; d < 3; d++) s[d] += m->X[3 * m->C[c * npc + a] + d];
    uint64_t code = 0;
    for (int d = 0; d < 3; d++) {
      double span = hi[d] - lo[d];
      double t = span > 0 ? (s[d] / npc - lo[d]) / span : 0.0;
      uint64_t q = (uint64_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
      code |= spread3(q) << d;
    }
    key[c] = {code, c};
  }
  std::sort(key.begin(), key.end());
  m->perm.resize(N);
  m->iperm.resize(N);
  for (int64_t k = 0; k < N; k++) {
    m->perm[k] = key[k].second;
    m->iperm[key[k].second] = k;
  }
  // faces: each element face is a sorted tuple of canonical nodes
  struct FE {
    std::array<int64_t, 4> k;
    int64_t user;
    int lf;
  };
  std::vector<FE> fe((size_t)N * m->nfc);
  for (int64_t c = 0; c < N; c++)
    for (int lf = 0; lf < m->nfc; lf++) {
      FE& e = fe[(size_t)c * m->nfc + lf];
      const int* fl = face_local_nodes(npc, lf);
      const int nfn = face_node_count(npc, lf);
      e.k = {-1, -1, -1, -1};
      for (int q = 0; q < nfn; q++) e.k[q] = m->canon[m->C[c * npc + fl[q]]];
      std::sort(e.k.begin(), e.k.begin() + nfn);
      e.user = c;
      e.lf = lf;
    }
  std::sort(fe.begin(), fe.end(), [](const FE& a, const FE& b) {
    if (a.k != b.k) return a.k < b.k;
    return a.user < b.user;
  });
  const size_t ne = fe.size();
  const bool open = !(m->per[0] && m->per[1] && m->per[2]);
  struct FP {
    int64_t o_int;
    int lf, nlf;
    int64_t n_int;  // -1: a face on a non-periodic side of the box
  };
  std::vector<FP> fp;
  fp.reserve(ne / 2 + 1);
  for (size_t j = 0; j < ne;) {
    const FE& a = fe[j];
    if (j + 1 < ne && fe[j + 1].k == a.k) {
      const FE& b = fe[j + 1];
      if (j + 2 < ne && fe[j + 2].k == a.k) return fail(UCNS_ERR_MESH, "unpaired or non-manifold face");
      if (a.user == b.user) return fail(UCNS_ERR_MESH, "a cell is its own face neighbour");
      fp.push_back({m->iperm[a.user], a.lf, b.lf, m->iperm[b.user]});  // a.user < b.user: owner
      j += 2;
    } else {
      if (!open) return fail(UCNS_ERR_MESH, "unpaired face (every axis of the box is periodic)");
      fp.push_back({m->iperm[a.user], a.lf, -1, -1});
      j += 1;
    }
  }
  m->F = (int64_t)fp.size();
  if (m->F >= (int64_t(1) << 30)) return fail(UCNS_ERR_MESH, "too many faces");
  m->n_boundary = 0;
  for (const FP& q : fp) m->n_boundary += q.n_int < 0;
  std::sort(fp.begin(), fp.end(), [](const FP& a, const FP& b) {
    return a.o_int != b.o_int ? a.o_int < b.o_int : a.lf < b.lf;
  });
  m->fo.resize(m->F);
  m->fn.resize(m->F);
  m->flf.resize(m->F);
  m->cf.assign((size_t)N * m->nfc, -1);
  for (int64_t f = 0; f < m->F; f++) {
    m->fo[f] = (int32_t)fp[f].o_int;
    m->fn[f] = (int32_t)fp[f].n_int;
    m->flf[f] = (int8_t)fp[f].lf;
    m->cf[(size_t)fp[f].o_int * m->nfc + fp[f].lf] = (int32_t)(f << 1);
    if (fp[f].n_int >= 0) m->cf[(size_t)fp[f].n_int * m->nfc + fp[f].nlf] = (int32_t)((f << 1) | 1);
  }
  for (int32_t e : m->cf)
    if (e < 0) return fail(UCNS_ERR_MESH, "element face without a partner");
  return UCNS_OK;
}

namespace {

struct Cand {
  int64_t id;  // internal
  int depth, shared;
  int64_t user;
};

// the cell across local face lf of cell i, -1 on a boundary face
int64_t face_nbr(const ucns_mesh* m, int64_t i, int lf) {
  int32_t e = m->cf[(size_t)i * m->nfc + lf];
  int32_t f = e >> 1;
  return (e & 1) ? m->fo[f] : m->fn[f];
}

// breadth-first search over face adjacency from `start`, never entering `avoid`
bool bfs(const ucns_mesh* m, int64_t start, int64_t avoid, int maxd, std::vector<Cand>& out) {
  out.clear();
  out.push_back({start, 0, 0, m->perm[start]});
  for (size_t head = 0; head < out.size(); head++) {
    Cand cur = out[head];
    if (cur.depth == maxd) continue;
    for (int lf = 0; lf < m->nfc; lf++) {
      int64_t n = face_nbr(m, cur.id, lf);
      if (n < 0 || n == avoid) continue;  // a boundary face, or the cell a directional search avoids
      bool seen = false;
      for (const Cand& c : out)
        if (c.id == n) { seen = true; break; }
      if (!seen) out.push_back({n, cur.depth + 1, 0, m->perm[n]});
    }
    if (out.size() > 512) return false;
  }
  return true;
}

int shared_nodes(const ucns_mesh* m, int64_t ui, int64_t um) {
  int s = 0;
  for (int a = 0; a < m->npc; a++) {
    int64_t ca = m->canon[m->C[ui * m->npc + a]];
    for (int b = 0; b < m->npc; b++)
      if (m->canon[m->C[um * m->npc + b]] == ca) { s++; break; }
  }
  return s;
}

// Householder QR of A (M x K, row-major); P[k][r] = (R^-1 Q^T)[k][r] * w[r].
bool pinv_householder(const double* Ain, int M, int K, const double* w, double* P) {
  double A[kMaxMc * kMaxK], v[kMaxK][kMaxMc], beta[kMaxK], colnorm[kMaxK];
  std::memcpy(A, Ain, sizeof(double) * M * K);
  for (int j = 0; j < K; j++) {
    double s = 0;
    for (int r = 0; r < M; r++) s += A[r * K + j] * A[r * K + j];
    colnorm[j] = std::sqrt(s);
  }
  for (int j = 0; j < K; j++) {
    double nx = 0;
    for (int r = j; r < M; r++) nx += A[r * K + j] * A[r * K + j];
    nx = std::sqrt(nx);
    if (!(nx > 1e-10 * colnorm[j])) return false;
    double alpha = A[j * K + j] > 0 ? -nx : nx;
    for (int r = 0; r < M; r++) v[j][r] = r < j ? 0.0 : A[r * K + j];
    v[j][j] -= alpha;
    double vv = 0;
    for (int r = j; r < M; r++) vv += v[j][r] * v[j][r];
    beta[j] = 2.0 / vv;
    for (int c = j; c < K; c++) {
      double d = 0;
      for (int r = j; r < M; r++) d += v[j][r] * A[r * K + c];
      d *= beta[j];
      for (int r = j; r < M; r++) A[r * K + c] -= d * v[j][r];
    }
  }
  // thin Q: apply the reflectors (last first) to the first K unit columns
  double Q[kMaxMc * kMaxK];
  for (int r = 0; r < M; r++)
    for (int c = 0; c < K; c++) Q[r * K + c] = (r == c) ? 1.0 : 0.0;
  for (int j = K - 1; j >= 0; j--)
    for (int c = 0; c < K; c++) {
      double d = 0;
      for (int r = j; r < M; r++) d += v[j][r] * Q[r * K + c];
      d *= beta[j];
      for (int r = j; r < M; r++) Q[r * K + c] -= d * v[j][r];
    }
  // P = R^-1 Q^T diag(w): solve R X = Q^T column by column (back substitution)
  for (int r = 0; r < M; r++) {
    double x[kMaxK];
    for (int k = K - 1; k >= 0; k--) {
      double s = Q[r * K + k];
      for (int l = k + 1; l < K; l++) s -= A[k * K + l] * x[l];
      x[k] = s / A[k * K + k];
    }
    for (int k = 0; k < K; k++) P[k * M + r] = x[k] * w[r];
  }
  return true;
}

}  // namespace

int host_precompute(ucns_mesh* m, const ucns_params* p, HostArrays* h) {
  const int64_t N = m->N, F = m->F;
  const int order = p->order;
  const int K = basis_count(order);
  const int Mc = 2 * K;
  const int nd = (order >= 2 && p->scheme == UCNS_SCHEME_CWENOZ) ? m->nfc : 0;
  // directional candidates: linear at P2 and P3, quadratic at P4 (Sec. 2.2)
  const int Kd = order == 4 ? 9 : 3;
  const int Md = 2 * Kd;
  const int nq = order * order;
  if (order >= 3 && m->npc != 8) return fail(UCNS_ERR_INVALID_ARG, "orders 3 and 4 are built for hexahedra only");
  if ((int64_t)F * nq >= (int64_t(1) << 31) || N * 5 >= (int64_t(1) << 31) ||
      (int64_t)(K + 1) * N * 5 >= (int64_t(1) << 31))
    return fail(UCNS_ERR_INVALID_ARG, "mesh too large for 32-bit kernel indexing");
  m->K = K; m->Mc = Mc; m->nd = nd; m->Md = Md; m->Kd = Kd; m->nq = nq; m->NC = K + 1;
  std::vector<Geom> g(N);  // internal order
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) g[i] = cell_geometry(m, m->perm[i]);
  for (int64_t i = 0; i < N; i++)
    if (!(g[i].V > 0)) return fail(UCNS_ERR_MESH, "cell with non-positive volume");
  // P3/P4: central moments of every cell (moment-form least-squares rows and
  // smoothness-indicator matrices)
  std::vector<double> cm;
  if (order >= 3) {
    cm.assign((size_t)N * kMomSlots, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) central_moments(m, m->perm[i], g[i], &cm[(size_t)i * kMomSlots]);
  }
  auto shift_of = [&](int64_t i, int64_t j, double s[3]) {  // nearest image of j seen from i
    for (int d = 0; d < 3; d++) {
      s[d] = 0.0;
      if (m->per[d]) s[d] = -m->L[d] * std::nearbyint((comp(g[j].c, d) - comp(g[i].c, d)) / m->L[d]);
    }
  };
  h->vol.resize(N); h->inv_vol.resize(N); h->inv_h.resize(N); h->dtlen.resize(N);
  h->mom.resize(6 * N);
  for (int64_t i = 0; i < N; i++) {
    h->vol[i] = g[i].V;
    h->inv_vol[i] = 1.0 / g[i].V;
    h->inv_h[i] = 1.0 / g[i].h;
    for (int k = 0; k < 6; k++) h->mom[k * N + i] = g[i].S[k];
  }
  // faces: quadrature in owner / neighbour local coordinates
  h->fq.assign((size_t)nq * 10 * F, 0.0);
  h->fpen.resize(F);
  std::vector<double> area(F);
  h->fkind.assign(F, -1);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < F; f++) {
    int64_t o = m->fo[f], n = m->fn[f];
    V3 x[16], dS[16];
    face_points(m, m->perm[o], m->flf[f], order, x, dS);
    double s[3] = {0.0, 0.0, 0.0};
    if (n >= 0) shift_of(o, n, s);
    V3 sv{s[0], s[1], s[2]};
    V3 tot{0, 0, 0};
    for (int q = 0; q < nq; q++) {
      double a = std::sqrt(dot(dS[q], dS[q]));
      V3 nh = (1.0 / a) * dS[q];
      V3 xl = x[q] - g[o].c;  // offset from the owner's centroid
      // offset from the neighbour image's centroid (a boundary face has none)
      V3 xr = n >= 0 ? x[q] - sv - g[n].c : V3{0, 0, 0};
      double vals[10] = {xl.x, xl.y, xl.z, xr.x, xr.y, xr.z, nh.x, nh.y, nh.z, a};
      for (int c = 0; c < 10; c++) h->fq[((size_t)q * 10 + c) * F + f] = vals[c];
      tot = tot + dS[q];
    }
    area[f] = std::sqrt(dot(tot, tot));
    if (n >= 0) {
      V3 dc = g[n].c + sv - g[o].c;
      h->fpen[f] = p->alpha / std::sqrt(dot(dc, dc));
    } else {
      // a face on a non-periodic side of the box: that side (the axis of the
      // largest component of its outward area vector, and its sign) and the
      // side's boundary kind
      const double t3[3] = {tot.x, tot.y, tot.z};
      int ax = 0;
      for (int d = 1; d < 3; d++)
        if (std::fabs(t3[d]) > std::fabs(t3[ax])) ax = d;
      h->fkind[f] = (int8_t)m->bc[2 * ax + (t3[ax] > 0 ? 1 : 0)];
      h->fpen[f] = 0.0;
    }
  }
  for (int64_t i = 0; i < N; i++) {
    double asum = 0;
    for (int lf = 0; lf < m->nfc; lf++) asum += area[m->cf[(size_t)i * m->nfc + lf] >> 1];
    h->dtlen[i] = 2.0 * g[i].V / asum;
  }
  // stencils and pseudo-inverses
  h->sc.assign((size_t)Mc * N, 0);
  h->Pc.assign((size_t)K * Mc * N, 0.0);
  h->sd.assign((size_t)nd * Md * N, 0);
  h->Pd.assign((size_t)nd * Kd * Md * N, 0.0);
  h->dvalid.assign(nd ? N : 0, (uint8_t)((1u << nd) - 1u));
  if (order >= 3) {
    // per cell: the means of the non-linear basis monomials (xi units) and
    // the smoothness-indicator matrix of Eq. 6's reading, SI(a) = a^T M a,
    // M_kl = sum_{1 <= |b|} (1/V) int d^b psi_k d^b psi_l (derivatives in xi,
    // each multi-index b once), from the xi-moments of the cell
    const int nm = K * (K + 1) / 2;
    h->psib.assign((size_t)(K - 3) * N, 0.0);
    h->Msi.assign((size_t)nm * N, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
      const double* mu = &cm[(size_t)i * kMomSlots];
      double ihp[2 * kMaxOrder + 1];  // (1/h)^e
      ihp[0] = 1.0;
      for (int e = 1; e <= 2 * kMaxOrder; e++) ihp[e] = ihp[e - 1] / g[i].h;
      auto xmu = [&](int a, int b, int c) { return mu[mom_index(a, b, c)] * ihp[a + b + c]; };
      for (int k = 3; k < K; k++)
        h->psib[(size_t)(k - 3) * N + i] = xmu(basis_exp(k, 0), basis_exp(k, 1), basis_exp(k, 2));
      int q = 0;
      for (int k = 0; k < K; k++)
        for (int l = k; l < K; l++, q++) {
          const int ak[3] = {basis_exp(k, 0), basis_exp(k, 1), basis_exp(k, 2)};
          const int al[3] = {basis_exp(l, 0), basis_exp(l, 1), basis_exp(l, 2)};
          double t = 0.0;
          for (int b0 = 0; b0 <= std::min(ak[0], al[0]); b0++)
            for (int b1 = 0; b1 <= std::min(ak[1], al[1]); b1++)
              for (int b2 = 0; b2 <= std::min(ak[2], al[2]); b2++) {
                if (b0 + b1 + b2 == 0) continue;
                const double f = falling(ak[0], b0) * falling(ak[1], b1) * falling(ak[2], b2) * falling(al[0], b0) *
                                 falling(al[1], b1) * falling(al[2], b2);
                t += f * xmu(ak[0] + al[0] - 2 * b0, ak[1] + al[1] - 2 * b1, ak[2] + al[2] - 2 * b2);
              }
          h->Msi[(size_t)q * N + i] = t;
        }
    }
  }
  int bad = 0;
  // A row of cell i's basis integrated over member j's image (moment form):
  // int_{V_j} phi_k = V_j [psi_k(d) + (h_j/h_i)^2 S_j,k - S_i,k], d = (c_j' - c_i)/h_i
  auto arow = [&](int64_t i, int64_t j, int KK, double* row) {
    double s[3];
    shift_of(i, j, s);
    double d[3];
    for (int q = 0; q < 3; q++) d[q] = (comp(g[j].c, q) + s[q] - comp(g[i].c, q)) / g[i].h;
    double r2 = (g[j].h / g[i].h) * (g[j].h / g[i].h);
    double V = g[j].V;
    row[0] = V * d[0]; row[1] = V * d[1]; row[2] = V * d[2];
    if (KK == 9) {
      const double* Sj = g[j].S;
      const double* Si = g[i].S;
      row[3] = V * (d[0] * d[0] + r2 * Sj[0] - Si[0]);
      row[4] = V * (d[1] * d[1] + r2 * Sj[1] - Si[1]);
      row[5] = V * (d[2] * d[2] + r2 * Sj[2] - Si[2]);
      row[6] = V * (d[0] * d[1] + r2 * Sj[3] - Si[3]);
      row[7] = V * (d[0] * d[2] + r2 * Sj[4] - Si[4]);
      row[8] = V * (d[1] * d[2] + r2 * Sj[5] - Si[5]);
    }
  };
  // P3/P4 rows (moment form from the member's central moments): the mean of
  // ((x - c_i)/h_i)^a over the member's image, expanded about its centroid c_j'
  // by the binomial theorem, less cell i's own mean of that monomial, times |V_j|
  double bin[kMaxOrder + 1][kMaxOrder + 1];  // binomial coefficients C(n, k)
  for (int n = 0; n <= kMaxOrder; n++)
    for (int k = 0; k <= kMaxOrder; k++) bin[n][k] = k <= n ? binom(n, k) : 0.0;
  auto arow_ho = [&](int64_t i, int64_t j, int KK, double* row) {
    double s[3];
    shift_of(i, j, s);
    double dp[3][kMaxOrder + 1];  // powers of the centroid offset, per coordinate
    for (int q = 0; q < 3; q++) {
      const double d = comp(g[j].c, q) + s[q] - comp(g[i].c, q);
      dp[q][0] = 1.0;
      for (int e = 1; e <= kMaxOrder; e++) dp[q][e] = dp[q][e - 1] * d;
    }
    double ihp[kMaxOrder + 1];
    ihp[0] = 1.0;
    for (int e = 1; e <= kMaxOrder; e++) ihp[e] = ihp[e - 1] / g[i].h;
    const double* muj = &cm[(size_t)j * kMomSlots];
    const double* mui = &cm[(size_t)i * kMomSlots];
    for (int k = 0; k < KK; k++) {
      const int a[3] = {basis_exp(k, 0), basis_exp(k, 1), basis_exp(k, 2)};
      double t = 0.0;
      for (int b0 = 0; b0 <= a[0]; b0++)
        for (int b1 = 0; b1 <= a[1]; b1++)
          for (int b2 = 0; b2 <= a[2]; b2++)
            t += bin[a[0]][b0] * bin[a[1]][b1] * bin[a[2]][b2] * dp[0][a[0] - b0] * dp[1][a[1] - b1] *
                 dp[2][a[2] - b2] * muj[mom_index(b0, b1, b2)];
      row[k] = g[j].V * (t - mui[mom_index(a[0], a[1], a[2])]) * ihp[a[0] + a[1] + a[2]];
    }
  };
  auto row_of = [&](int64_t i, int64_t j, int KK, double* row) {
    if (order >= 3) arow_ho(i, j, KK, row);
    else arow(i, j, KK, row);
  };
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
  for (int64_t i = 0; i < N; i++) {
    std::vector<Cand> c;
    if (!bfs(m, i, -1, order == 4 ? 4 : 3, c)) { bad |= 1; continue; }
    for (size_t q = 1; q < c.size(); q++) c[q].shared = shared_nodes(m, m->perm[i], c[q].user);
    std::sort(c.begin() + 1, c.end(), [](const Cand& a, const Cand& b) {
      if (a.depth != b.depth) return a.depth < b.depth;
      if (a.shared != b.shared) return a.shared > b.shared;
      return a.user < b.user;
    });
    if ((int)c.size() - 1 < Mc) { bad |= 2; continue; }
    double A[kMaxMc * kMaxK], w[kMaxMc], P[kMaxK * kMaxMc];
    for (int r = 0; r < Mc; r++) {
      int64_t j = c[1 + r].id;
      h->sc[(size_t)r * N + i] = (int32_t)j;
      row_of(i, j, K, &A[r * K]);
      w[r] = g[j].V;
    }
    if (!pinv_householder(A, Mc, K, w, P)) { bad |= 4; continue; }
    for (int k = 0; k < K; k++)
      for (int r = 0; r < Mc; r++) h->Pc[((size_t)k * Mc + r) * N + i] = P[k * Mc + r];
    for (int s = 0; s < nd; s++) {
      int64_t nb = face_nbr(m, i, s);
      if (nb < 0) {
        // a boundary face: no directional candidate there (its slot keeps the
        // cell itself as members and zero rows, and is marked invalid)
        h->dvalid[i] &= (uint8_t)~(1u << s);
        for (int r = 0; r < Md; r++) h->sd[((size_t)s * Md + r) * N + i] = (int32_t)i;
        continue;
      }
      if (!bfs(m, nb, i, Kd == 3 ? 2 : 3, c)) { bad |= 1; break; }
      std::sort(c.begin() + 1, c.end(), [](const Cand& a, const Cand& b) {
        if (a.depth != b.depth) return a.depth < b.depth;
        return a.user < b.user;
      });
      if ((int)c.size() < Md) { bad |= 2; break; }
      for (int r = 0; r < Md; r++) {
        int64_t j = c[r].id;
        h->sd[((size_t)s * Md + r) * N + i] = (int32_t)j;
        row_of(i, j, Kd, &A[r * Kd]);
        w[r] = g[j].V;
      }
      if (!pinv_householder(A, Md, Kd, w, P)) { bad |= 4; break; }
      for (int k = 0; k < Kd; k++)
        for (int r = 0; r < Md; r++) h->Pd[(((size_t)s * Kd + k) * Md + r) * N + i] = P[k * Md + r];
    }
  }
  if (bad & 1) return fail(UCNS_ERR_STENCIL, "stencil search overflow");
  if (bad & 2) return fail(UCNS_ERR_STENCIL, "too few cells for a stencil (mesh too small)");
  if (bad & 4) return fail(UCNS_ERR_STENCIL, "rank-deficient least-squares stencil");
  return UCNS_OK;
}

}  // namespace ucns
