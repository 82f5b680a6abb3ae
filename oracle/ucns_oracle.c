/*
 * ucns_oracle.c -- plain, slow FP64 CPU oracle of the explicit residual and
 * SSP Runge-Kutta update (SSP-RK3, SSP(5,4)) of the high-order cell-centred
 * finite-volume scheme
 * (Sec. 2.2: Eq. 1 conservation law, Eq. 2 semi-discretisation, Eqs. 3-4
 * k-exact least-squares reconstruction, Eqs. 5-6 CWENOZ, Eq. 7 viscous
 * interface gradient, HLLC inviscid flux, Eq. 8 explicit SSP Runge-Kutta).
 * Reconstruction degrees P1 and P2 on hexahedra, tetrahedra, triangular
 * prisms and pyramids, P3 and P4 (quadratic directional candidates) on
 * hexahedra.

 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library; the product path
 * (libucns + its CUDA kernels) neither links nor calls it, and the two share
 * no source.
 *
 * Everything is FP64, user cell order, no reordering, no blocking and no
 * fusion: mesh -> faces -> stencils -> least-squares operators -> per-cell
 * reconstruction -> per-face flux -> per-cell residual -> Runge-Kutta.
 * Every reading of a point where the paper is silent is listed in the
 * design notes and restated at the function that implements it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA
 * contraction, so each step rounds as written).  OpenMP only splits the
 * independent per-cell / per-face loops; every output element is written by
 * one iteration, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXK 34     /* non-constant modes of a quartic in 3-D (Eq. 3, K-1; P4) */
#define ORC_MAXM 68     /* central stencil size 2K */
#define ORC_MAXD 6      /* directional stencils: one per element face */
#define ORC_MD 18       /* largest directional stencil: 2 x 9 (quadratic candidates at P4) */

typedef struct {
  int64_t N, nn;
  int npc;  /* nodes per cell: 8 hex, 6 prism, 5 pyramid, 4 tet */
  int nfc;  /* faces per cell: 6 hex, 5 prism or pyramid, 4 tet */
  double L[3];
  int per[3];
  double *X;       /* [nn][3] */
  int64_t *C;      /* [N][npc] */
  int64_t *canon;  /* node -> canonical (periodic) node id */
  /* parameters */
  int order, scheme, inviscid;
  int rk;  /* 0: SSP-RK3, 1: SSP(5,4) */
  int bc[6];         /* per box side x-, x+, y-, y+, z-, z+ of a non-periodic axis:
                        0 or 1 slip wall, 2 supersonic outflow, 3 supersonic inflow */
  double uinf[5];    /* conserved inflow state */
  double gam, Pr, Re, Mach, cfl, lamc, eps, alpha;
  int K, nq, Mc, nd, Md;
  int Kd;  /* modes of a directional candidate: 3 (linear, P2 and P3) or 9 (quadratic, P4) */
  /* geometry */
  double *vol, *cen, *hh, *psib; /* psib [N][ORC_MAXK]: (1/V) int psi_k */
  /* faces */
  int64_t F;
  int64_t *fo, *fn;
  int *flf;
  signed char *fsh;  /* [F][3] image shift of the neighbour, in box lengths */
  int64_t *cf;       /* [N][nfc] face ids */
  signed char *cs;   /* [N][nfc] +1 owner, -1 neighbour */
  /* stencils and operators */
  int64_t *sc;       /* [N][Mc] */
  signed char *scsh; /* [N][Mc][3] */
  double *Pc;        /* [N][K][Mc] */
  int64_t *sd;       /* [N][nd][Md] */
  signed char *sdsh; /* [N][nd][Md][3] */
  double *Pd;        /* [N][nd][3][Md] */
  unsigned char *ready;
  unsigned char *dvalid;  /* [N][nd]: directional candidate s exists (no wall on face s) */
  int walls;              /* some box axis is not periodic: its unpaired faces are slip walls */
  unsigned char *mask;    /* [N] or NULL: per-cell scheme of a CWENOZ case (0: p_opt, the
                             linear weights; nonzero: CWENOZ), Sec. 2.2, Eqs. 5-6 */
  /* quadrature on [0,1] */
  int ngeo;
  double gx[8], gw[8];
} orc_case;

static char g_err[512];
static void set_err(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char *orc_last_error(void) { return g_err; }

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1] by Newton iteration on P_n.                  */
/* ------------------------------------------------------------------------ */
static void gauss_legendre01(int n, double *x, double *w) {
  for (int i = 0; i < n; i++) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  /* = (2/((1-z^2)P'^2)) / 2 */
  }
}

/* ------------------------------------------------------------------------ */
/* Element maps.  Hex: trilinear map of the unit cube (VTK node order).      */
/* Tet: collapsed (Duffy) map of the unit cube onto the tetrahedron.         */
/* Prism (nodes 0,1,2 counter-clockwise seen from the top triangle 3,4,5,   */
/* node 3+k above node k): the collapsed map of the base triangle times a   */
/* linear map in height, so its side faces are the bilinear quad patches.   */
/* Pyramid (base 0,1,2,3 counter-clockwise seen from the apex 4): the base's */
/* bilinear map shrunk linearly onto the apex, x = (1 - w) Q(a, b) + w x_4.   */
/* ------------------------------------------------------------------------ */
static const int HEXO[8][3] = {{0,0,0},{1,0,0},{1,1,0},{0,1,0},{0,0,1},{1,0,1},{1,1,1},{0,1,1}};
/* local faces, node lists ordered so (p2-p0)x(p3-p1) points outward */
static const int HEXF[6][4] = {{0,4,7,3},{1,2,6,5},{0,1,5,4},{3,7,6,2},{0,3,2,1},{4,5,6,7}};
/* tet faces ordered so (p1-p0)x(p2-p0) points outward for positive tets */
static const int TETF[4][3] = {{0,2,1},{0,1,3},{1,2,3},{0,3,2}};
/* prism faces: two triangles, then three quads, each ordered by the rules above */
static const int PRISMF[5][4] = {{0,2,1,-1},{3,4,5,-1},{0,1,4,3},{1,2,5,4},{2,0,3,5}};
/* pyramid faces: the base quad, then four triangles */
static const int PYRF[5][4] = {{0,3,2,1},{0,1,4,-1},{1,2,4,-1},{2,3,4,-1},{3,0,4,-1}};

static void cell_nodes(const orc_case *c, int64_t i, double P[8][3]) {
  for (int a = 0; a < c->npc; a++)
    for (int d = 0; d < 3; d++) P[a][d] = c->X[3 * c->C[i * c->npc + a] + d];
}

static double det3(const double a[3], const double b[3], const double e[3]) {
  return a[0] * (b[1] * e[2] - b[2] * e[1]) - a[1] * (b[0] * e[2] - b[2] * e[0]) +
         a[2] * (b[0] * e[1] - b[1] * e[0]);
}

static void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/* point x and Jacobian determinant at reference point r in [0,1]^3 */
static void cell_map(const orc_case *c, const double P[8][3], const double r[3], double x[3],
                     double *detJ) {
  if (c->npc == 8) {
    double s = r[0], t = r[1], u = r[2];
    double dx[3][3] = {{0}};
    x[0] = x[1] = x[2] = 0.0;
    for (int a = 0; a < 8; a++) {
      double fs = HEXO[a][0] ? s : 1.0 - s, ft = HEXO[a][1] ? t : 1.0 - t,
             fu = HEXO[a][2] ? u : 1.0 - u;
      double ds = HEXO[a][0] ? 1.0 : -1.0, dt = HEXO[a][1] ? 1.0 : -1.0,
             du = HEXO[a][2] ? 1.0 : -1.0;
      double N = fs * ft * fu;
      for (int d = 0; d < 3; d++) {
        x[d] += N * P[a][d];
        dx[0][d] += ds * ft * fu * P[a][d];
        dx[1][d] += fs * dt * fu * P[a][d];
        dx[2][d] += fs * ft * du * P[a][d];
      }
    }
    *detJ = det3(dx[0], dx[1], dx[2]);
  } else if (c->npc == 5) {
    double a = r[0], b = r[1], w = r[2], da[3], db[3], dw[3];
    for (int d = 0; d < 3; d++) {
      double Q = (1 - a) * (1 - b) * P[0][d] + a * (1 - b) * P[1][d] + a * b * P[2][d] + (1 - a) * b * P[3][d];
      double Qa = (1 - b) * (P[1][d] - P[0][d]) + b * (P[2][d] - P[3][d]);
      double Qb = (1 - a) * (P[3][d] - P[0][d]) + a * (P[2][d] - P[1][d]);
      x[d] = (1.0 - w) * Q + w * P[4][d];
      da[d] = (1.0 - w) * Qa;
      db[d] = (1.0 - w) * Qb;
      dw[d] = P[4][d] - Q;
    }
    *detJ = det3(da, db, dw);
  } else if (c->npc == 6) {
    /* x = (1 - w) B(a, b) + w T(a, b), B = P0 + a e1 + a b e2 on the base,
       T = P3 + a f1 + a b f2 on the top */
    double a = r[0], b = r[1], w = r[2], da[3], db[3], dw[3];
    for (int d = 0; d < 3; d++) {
      double e1 = P[1][d] - P[0][d], e2 = P[2][d] - P[1][d], f1 = P[4][d] - P[3][d], f2 = P[5][d] - P[4][d];
      double B = P[0][d] + a * e1 + a * b * e2, T = P[3][d] + a * f1 + a * b * f2;
      x[d] = (1.0 - w) * B + w * T;
      da[d] = (1.0 - w) * (e1 + b * e2) + w * (f1 + b * f2);
      db[d] = (1.0 - w) * a * e2 + w * a * f2;
      dw[d] = T - B;
    }
    *detJ = det3(da, db, dw);
  } else {
    double a = r[0], b = r[1], cc = r[2];
    double e1[3], e2[3], e3[3], v1[3], v2[3], v3[3];
    for (int d = 0; d < 3; d++) {
      e1[d] = P[1][d] - P[0][d];
      e2[d] = P[2][d] - P[1][d];
      e3[d] = P[3][d] - P[2][d];
      x[d] = P[0][d] + a * e1[d] + a * b * e2[d] + a * b * cc * e3[d];
      v1[d] = P[1][d] - P[0][d];
      v2[d] = P[2][d] - P[0][d];
      v3[d] = P[3][d] - P[0][d];
    }
    *detJ = a * a * b * det3(v1, v2, v3);
  }
}

/* quadrature over cell i: calls f(x, weight) with weight = w * detJ */
typedef void (*cell_fn)(void *ctx, const double x[3], double w);
static void cell_quad(const orc_case *c, int64_t i, int n, cell_fn f, void *ctx) {
  double gx[16], gw[16];
  gauss_legendre01(n, gx, gw);
  double P[8][3];
  cell_nodes(c, i, P);
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++)
      for (int q = 0; q < n; q++) {
        double r[3] = {gx[a], gx[b], gx[q]}, x[3], dj;
        cell_map(c, P, r, x, &dj);
        f(ctx, x, gw[a] * gw[b] * gw[q] * dj);
      }
}

/* ------------------------------------------------------------------------ */
/* Basis of Eq. 3: monomials psi_k of xi=(x-x_i)/h_i, h_i = V_i^(1/3),      */
/* k = x, y, z, xx, yy, zz, xy, xz, yz (P2: the first 9), then the cubics    */
/* xxx, yyy, zzz, xxy, xxz, xyy, yyz, xzz, yzz, xyz (P3: 19);                */
/* phi_k = psi_k - (1/V_i) int psi_k.                                        */
/* ------------------------------------------------------------------------ */
/* exponents of every basis monomial, in basis order */
static const int MONO[ORC_MAXK][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
    {3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1},
    {4, 0, 0}, {0, 4, 0}, {0, 0, 4}, {3, 1, 0}, {3, 0, 1}, {1, 3, 0}, {0, 3, 1}, {1, 0, 3}, {0, 1, 3},
    {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};
/* d^b of the monomial with exponents e at xi: the falling-factorial
   coefficient, then the remaining powers of x, y and z in that order */
static double mono_d(const int e[3], const int b[3], const double xi[3]) {
  double v = 1.0;
  for (int d = 0; d < 3; d++) {
    if (b[d] > e[d]) return 0.0;
    for (int j = 0; j < b[d]; j++) v *= (double)(e[d] - j);
  }
  for (int d = 0; d < 3; d++)
    for (int j = 0; j < e[d] - b[d]; j++) v *= xi[d];
  return v;
}
/* the derivative multi-indices of order 1..4, each once, in a fixed order */
static const int DER1[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
static const int DER3[10][3] = {{3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {2, 1, 0}, {2, 0, 1},
                                {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1}};
static const int DER4[15][3] = {{4, 0, 0}, {0, 4, 0}, {0, 0, 4}, {3, 1, 0}, {3, 0, 1}, {1, 3, 0}, {0, 3, 1}, {1, 0, 3},
                                {0, 1, 3}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};
static const int DER2[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
static const int ZERO3[3] = {0, 0, 0};

/* psi_eval / psi_grad / psi_hess fill the first nk entries (nk <= ORC_MAXK;
   the explicit P1-P3 entries are always written) */
static void psi_eval(const double xi[3], double p[ORC_MAXK], int nk) {
  const double x = xi[0], y = xi[1], z = xi[2];
  p[0] = x; p[1] = y; p[2] = z;
  p[3] = x * x; p[4] = y * y; p[5] = z * z;
  p[6] = x * y; p[7] = x * z; p[8] = y * z;
  p[9] = x * x * x; p[10] = y * y * y; p[11] = z * z * z;
  p[12] = x * x * y; p[13] = x * x * z; p[14] = x * y * y;
  p[15] = y * y * z; p[16] = x * z * z; p[17] = y * z * z; p[18] = x * y * z;
  for (int k = 19; k < nk; k++) p[k] = mono_d(MONO[k], ZERO3, xi);  /* quartics (P4) */
}
/* d psi_k / d xi_j */
static void psi_grad(const double xi[3], double g[ORC_MAXK][3], int nk) {
  const double x = xi[0], y = xi[1], z = xi[2];
  memset(g, 0, sizeof(double) * ORC_MAXK * 3);
  g[0][0] = 1; g[1][1] = 1; g[2][2] = 1;
  g[3][0] = 2 * x; g[4][1] = 2 * y; g[5][2] = 2 * z;
  g[6][0] = y; g[6][1] = x;
  g[7][0] = z; g[7][2] = x;
  g[8][1] = z; g[8][2] = y;
  g[9][0] = 3 * x * x; g[10][1] = 3 * y * y; g[11][2] = 3 * z * z;
  g[12][0] = 2 * x * y; g[12][1] = x * x;
  g[13][0] = 2 * x * z; g[13][2] = x * x;
  g[14][0] = y * y; g[14][1] = 2 * x * y;
  g[15][1] = 2 * y * z; g[15][2] = y * y;
  g[16][0] = z * z; g[16][2] = 2 * x * z;
  g[17][1] = z * z; g[17][2] = 2 * y * z;
  g[18][0] = y * z; g[18][1] = x * z; g[18][2] = x * y;
  for (int k = 19; k < nk; k++)
    for (int j = 0; j < 3; j++) g[k][j] = mono_d(MONO[k], DER1[j], xi);
}
/* second derivatives d2 psi_k / d xi_a d xi_b in the order xx,yy,zz,xy,xz,yz */
static void psi_hess(const double xi[3], double H[ORC_MAXK][6], int nk) {
  const double x = xi[0], y = xi[1], z = xi[2];
  memset(H, 0, sizeof(double) * ORC_MAXK * 6);
  H[3][0] = 2; H[4][1] = 2; H[5][2] = 2;
  H[6][3] = 1; H[7][4] = 1; H[8][5] = 1;
  H[9][0] = 6 * x; H[10][1] = 6 * y; H[11][2] = 6 * z;
  H[12][0] = 2 * y; H[12][3] = 2 * x;              /* xxy */
  H[13][0] = 2 * z; H[13][4] = 2 * x;              /* xxz */
  H[14][1] = 2 * x; H[14][3] = 2 * y;              /* xyy */
  H[15][1] = 2 * z; H[15][5] = 2 * y;              /* yyz */
  H[16][2] = 2 * x; H[16][4] = 2 * z;              /* xzz */
  H[17][2] = 2 * y; H[17][5] = 2 * z;              /* yzz */
  H[18][3] = z; H[18][4] = y; H[18][5] = x;        /* xyz */
  for (int k = 19; k < nk; k++)
    for (int j = 0; j < 6; j++) H[k][j] = mono_d(MONO[k], DER2[j], xi);
}
/* ------------------------------------------------------------------------ */
/* Geometry: volume, centroid, h, mean of each monomial.                     */
/* ------------------------------------------------------------------------ */
typedef struct { double v, m[3]; } vm_ctx;
static void f_volmom(void *ctx, const double x[3], double w) {
  vm_ctx *q = (vm_ctx *)ctx;
  q->v += w;
  for (int d = 0; d < 3; d++) q->m[d] += w * x[d];
}
typedef struct { double c[3], h, s[ORC_MAXK]; } pb_ctx;
static void f_psibar(void *ctx, const double x[3], double w) {
  pb_ctx *q = (pb_ctx *)ctx;
  double xi[3], p[ORC_MAXK];
  for (int d = 0; d < 3; d++) xi[d] = (x[d] - q->c[d]) / q->h;
  psi_eval(xi, p, ORC_MAXK);
  for (int k = 0; k < ORC_MAXK; k++) q->s[k] += w * p[k];
}

static int compute_geometry(orc_case *c) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < c->N; i++) {
    vm_ctx q = {0, {0, 0, 0}};
    cell_quad(c, i, c->ngeo, f_volmom, &q);
    if (!(q.v > 0)) { bad = 1; continue; }
    c->vol[i] = q.v;
    for (int d = 0; d < 3; d++) c->cen[3 * i + d] = q.m[d] / q.v;
    c->hh[i] = cbrt(q.v);
    pb_ctx b;
    memset(&b, 0, sizeof b);
    for (int d = 0; d < 3; d++) b.c[d] = c->cen[3 * i + d];
    b.h = c->hh[i];
    cell_quad(c, i, c->ngeo, f_psibar, &b);
    for (int k = 0; k < ORC_MAXK; k++) c->psib[ORC_MAXK * i + k] = b.s[k] / q.v;
  }
  if (bad) { set_err("cell with non-positive volume"); return -1; }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Periodic canonical nodes: nodes equal modulo the box lengths are one.     */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t k[3]; int64_t id; } nkey;
static int cmp_nkey(const void *a, const void *b) {
  const nkey *p = (const nkey *)a, *q = (const nkey *)b;
  for (int d = 0; d < 3; d++) {
    if (p->k[d] < q->k[d]) return -1;
    if (p->k[d] > q->k[d]) return 1;
  }
  return (p->id < q->id) ? -1 : (p->id > q->id);
}

static void compute_canon(orc_case *c) {
  nkey *a = (nkey *)malloc(sizeof(nkey) * c->nn);
  double scale = 0;
  for (int d = 0; d < 3; d++) scale = fmax(scale, c->L[d]);
  for (int64_t n = 0; n < c->nn; n++) {
    for (int d = 0; d < 3; d++) {
      double x = c->X[3 * n + d];
      if (c->per[d]) {
        x = x - c->L[d] * floor(x / c->L[d]);
        if (x > c->L[d] - 1e-9 * c->L[d]) x -= c->L[d];
      }
      a[n].k[d] = llround(x / (1e-8 * (scale > 0 ? scale : 1.0)));
    }
    a[n].id = n;
  }
  qsort(a, c->nn, sizeof(nkey), cmp_nkey);
  int64_t first = 0;
  for (int64_t n = 0; n < c->nn; n++) {
    if (n == 0 || memcmp(a[n].k, a[n - 1].k, sizeof a[n].k) != 0) first = a[n].id;
    c->canon[a[n].id] = first;
  }
  free(a);
}

/* ------------------------------------------------------------------------ */
/* Faces: each element face is a sorted tuple of canonical node ids; every  */
/* tuple must occur exactly twice.  Owner = lower cell id; the face normal  */
/* and quadrature points come from the owner's own nodes.                    */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t k[4]; int64_t cell; int lf; } fkey;
static int cmp_fkey(const void *a, const void *b) {
  const fkey *p = (const fkey *)a, *q = (const fkey *)b;
  for (int d = 0; d < 4; d++) {
    if (p->k[d] < q->k[d]) return -1;
    if (p->k[d] > q->k[d]) return 1;
  }
  if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
  return p->lf - q->lf;
}
static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

static const int *face_nodes(const orc_case *c, int lf) {
  return c->npc == 8 ? HEXF[lf] : (c->npc == 6 ? PRISMF[lf] : (c->npc == 5 ? PYRF[lf] : TETF[lf]));
}
/* nodes of local face lf: 4 (quad) or 3 (triangle) */
static int face_nn(const orc_case *c, int lf) {
  return c->npc == 8 ? 4 : (c->npc == 6 ? (lf < 2 ? 3 : 4) : (c->npc == 5 ? (lf == 0 ? 4 : 3) : 3));
}

/* nearest periodic image of cell m seen from cell i, as integer box shifts */
static void image_shift(const orc_case *c, int64_t i, int64_t m, signed char sh[3]) {
  for (int d = 0; d < 3; d++) {
    sh[d] = 0;
    if (c->per[d]) {
      double dd = c->cen[3 * m + d] - c->cen[3 * i + d];
      sh[d] = (signed char)(-llround(dd / c->L[d]));
    }
  }
}

static int build_faces(orc_case *c) {
  int64_t nk = c->N * c->nfc;
  fkey *a = (fkey *)malloc(sizeof(fkey) * nk);
  for (int64_t i = 0; i < c->N; i++)
    for (int lf = 0; lf < c->nfc; lf++) {
      fkey *f = &a[i * c->nfc + lf];
      const int *fnl = face_nodes(c, lf);
      for (int q = 0; q < 4; q++) f->k[q] = -1;
      const int nn = face_nn(c, lf);
      for (int q = 0; q < nn; q++) f->k[q] = c->canon[c->C[i * c->npc + fnl[q]]];
      qsort(f->k, nn, sizeof(int64_t), cmp_i64);
      f->cell = i;
      f->lf = lf;
    }
  qsort(a, nk, sizeof(fkey), cmp_fkey);
  if (nk % 2 && !c->walls) { free(a); set_err("unpaired face"); return -1; }
  /* pairs sorted by key; faces then ordered by (owner, local face).  With a
     non-periodic box axis, a face whose key occurs once lies on the box
     boundary: a slip wall, neighbour -1 */
  typedef struct { int64_t o, n; int lf, nlf; } pr;
  pr *p = (pr *)malloc(sizeof(pr) * nk);
  int64_t F = 0;
  for (int64_t j = 0; j < nk;) {
    fkey *x = &a[j];
    if (j + 1 < nk && memcmp(x->k, a[j + 1].k, sizeof x->k) == 0) {
      fkey *y = &a[j + 1];
      if (j + 2 < nk && memcmp(y->k, a[j + 2].k, sizeof y->k) == 0) {
        free(a); free(p); set_err("unpaired or non-manifold face"); return -1;
      }
      if (x->cell == y->cell) { free(a); free(p); set_err("cell is its own neighbour"); return -1; }
      p[F].o = x->cell; p[F].lf = x->lf; p[F].n = y->cell; p[F].nlf = y->lf;
      j += 2;
    } else {
      if (!c->walls) { free(a); free(p); set_err("unpaired or non-manifold face"); return -1; }
      p[F].o = x->cell; p[F].lf = x->lf; p[F].n = -1; p[F].nlf = -1;
      j += 1;
    }
    F++;
  }
  free(a);
  c->F = F;
  c->fo = (int64_t *)malloc(sizeof(int64_t) * c->F);
  c->fn = (int64_t *)malloc(sizeof(int64_t) * c->F);
  c->flf = (int *)malloc(sizeof(int) * c->F);
  c->fsh = (signed char *)malloc(3 * c->F);
  /* order by owner then owner-local face: counting sort on owner */
  int64_t *cnt = (int64_t *)calloc(c->N * c->nfc, sizeof(int64_t));
  for (int64_t f = 0; f < c->F; f++) cnt[p[f].o * c->nfc + p[f].lf] = f + 1;
  int64_t k = 0;
  for (int64_t s = 0; s < c->N * c->nfc; s++)
    if (cnt[s]) {
      pr *q = &p[cnt[s] - 1];
      c->fo[k] = q->o; c->fn[k] = q->n; c->flf[k] = q->lf;
      c->cf[q->o * c->nfc + q->lf] = k; c->cs[q->o * c->nfc + q->lf] = 1;
      if (q->n >= 0) {
        c->cf[q->n * c->nfc + q->nlf] = k; c->cs[q->n * c->nfc + q->nlf] = -1;
        image_shift(c, q->o, q->n, &c->fsh[3 * k]);
      } else {
        for (int d = 0; d < 3; d++) c->fsh[3 * k + d] = 0;
      }
      k++;
    }
  free(cnt);
  free(p);
  return 0;
}

/* face quadrature: points x[nq][3] and area vectors dS[nq][3] of face f,  */
/* oriented outward from the owner (Eq. 2: omega_alpha |S_f| per point).    */
static void face_quad(const orc_case *c, int64_t f, double x[][3], double dS[][3]) {
  double P[8][3];
  cell_nodes(c, c->fo[f], P);
  const int *fnl = face_nodes(c, c->flf[f]);
  if (face_nn(c, c->flf[f]) == 4) {
    double Q[4][3];
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) Q[a][d] = P[fnl[a]][d];
    int r = c->order;  /* r x r Gauss points: 1 at P1, 4 at P2 */
    double gx[8], gw[8];
    gauss_legendre01(r, gx, gw);
    int q = 0;
    for (int ia = 0; ia < r; ia++)
      for (int ib = 0; ib < r; ib++, q++) {
        double s = gx[ia], t = gx[ib], da[3], db[3], nrm[3];
        for (int d = 0; d < 3; d++) {
          x[q][d] = (1 - s) * (1 - t) * Q[0][d] + s * (1 - t) * Q[1][d] + s * t * Q[2][d] +
                    (1 - s) * t * Q[3][d];
          da[d] = (1 - t) * (Q[1][d] - Q[0][d]) + t * (Q[2][d] - Q[3][d]);
          db[d] = (1 - s) * (Q[3][d] - Q[0][d]) + s * (Q[2][d] - Q[1][d]);
        }
        cross3(da, db, nrm);
        for (int d = 0; d < 3; d++) dS[q][d] = gw[ia] * gw[ib] * nrm[d];
      }
  } else {
    double Q[3][3], e1[3], e2[3], n[3];
    for (int a = 0; a < 3; a++)
      for (int d = 0; d < 3; d++) Q[a][d] = P[fnl[a]][d];
    if (c->order == 1) {
      for (int d = 0; d < 3; d++) {
        x[0][d] = (Q[0][d] + Q[1][d] + Q[2][d]) / 3.0;
        e1[d] = Q[1][d] - Q[0][d];
        e2[d] = Q[2][d] - Q[0][d];
      }
      cross3(e1, e2, n);
      for (int d = 0; d < 3; d++) dS[0][d] = 0.5 * n[d];
    } else {
      /* collapsed 2x2 Gauss rule: x = Q0 + a(Q1-Q0) + ab(Q2-Q1), dS = a (Q1-Q0)x(Q2-Q1) */
      double gx[8], gw[8];
      gauss_legendre01(2, gx, gw);
      for (int d = 0; d < 3; d++) {
        e1[d] = Q[1][d] - Q[0][d];
        e2[d] = Q[2][d] - Q[1][d];
      }
      cross3(e1, e2, n);
      int q = 0;
      for (int ia = 0; ia < 2; ia++)
        for (int ib = 0; ib < 2; ib++, q++) {
          double a = gx[ia], b = gx[ib];
          for (int d = 0; d < 3; d++) {
            x[q][d] = Q[0][d] + a * e1[d] + a * b * e2[d];
            dS[q][d] = gw[ia] * gw[ib] * a * n[d];
          }
        }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Stencils.  Central (Sec. 2.2 compact stencil S_i): the first 2K cells of */
/* the face-graph neighbourhood of i ordered by (face-graph distance, nodes */
/* shared with i descending, cell id).  Directional (sectorial, one per     */
/* face f): breadth-first from the face neighbour n_f without entering i,   */
/* ordered by (distance from n_f, cell id), first 6 (linear polynomials).   */
/* ------------------------------------------------------------------------ */
static int shared_nodes(const orc_case *c, int64_t i, int64_t m) {
  int s = 0;
  for (int a = 0; a < c->npc; a++)
    for (int b = 0; b < c->npc; b++)
      if (c->canon[c->C[i * c->npc + a]] == c->canon[c->C[m * c->npc + b]]) { s++; break; }
  return s;
}
static int64_t face_nbr(const orc_case *c, int64_t i, int lf) {
  int64_t f = c->cf[i * c->nfc + lf];
  return c->fo[f] == i ? c->fn[f] : c->fo[f];
}

typedef struct { int64_t id; int depth, shared; } cand;
static int cmp_central(const void *a, const void *b) {
  const cand *p = (const cand *)a, *q = (const cand *)b;
  if (p->depth != q->depth) return p->depth - q->depth;
  if (p->shared != q->shared) return q->shared - p->shared;
  return (p->id > q->id) - (p->id < q->id);
}
static int cmp_dir(const void *a, const void *b) {
  const cand *p = (const cand *)a, *q = (const cand *)b;
  if (p->depth != q->depth) return p->depth - q->depth;
  return (p->id > q->id) - (p->id < q->id);
}

/* breadth-first search over face adjacency from `start`, never visiting
 * `avoid`, up to `maxd`; returns number of candidates (start included at depth 0) */
static int bfs(const orc_case *c, int64_t start, int64_t avoid, int maxd, cand *out, int cap) {
  int n = 0;
  out[n].id = start; out[n].depth = 0; out[n].shared = 0; n++;
  int head = 0;
  while (head < n) {
    cand cur = out[head++];
    if (cur.depth == maxd) continue;
    for (int lf = 0; lf < c->nfc; lf++) {
      int64_t m = face_nbr(c, cur.id, lf);
      if (m < 0 || m == avoid) continue;  /* a wall, or the cell a directional search avoids */
      int seen = 0;
      for (int q = 0; q < n; q++)
        if (out[q].id == m) { seen = 1; break; }
      if (seen) continue;
      if (n == cap) return -1;
      out[n].id = m; out[n].depth = cur.depth + 1; out[n].shared = 0; n++;
    }
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Least squares (Eq. 4): A_mk = int_{V_m} phi_k dV over the periodic image  */
/* of member m, rhs |V_m|(U_m - U_i); P' = A^+ diag(|V_m|) by QR (modified  */
/* Gram-Schmidt, each column orthogonalised twice).                          */
/* ------------------------------------------------------------------------ */
typedef struct { double c[3], h, sh[3], s[ORC_MAXK]; const double *pb; int K; } am_ctx;
static void f_arow(void *ctx, const double x[3], double w) {
  am_ctx *q = (am_ctx *)ctx;
  double xi[3], p[ORC_MAXK];
  for (int d = 0; d < 3; d++) xi[d] = (x[d] + q->sh[d] - q->c[d]) / q->h;
  psi_eval(xi, p, q->K);
  for (int k = 0; k < q->K; k++) q->s[k] += w * (p[k] - q->pb[k]);
}

static void lsq_matrix(const orc_case *c, int64_t i, int M, const int64_t *mem,
                       const signed char *sh, int K, double *A /* [M][K] */) {
  for (int r = 0; r < M; r++) {
    am_ctx q;
    memset(&q, 0, sizeof q);
    for (int d = 0; d < 3; d++) {
      q.c[d] = c->cen[3 * i + d];
      q.sh[d] = sh[3 * r + d] * c->L[d];
    }
    q.h = c->hh[i];
    q.pb = &c->psib[ORC_MAXK * i];
    q.K = K;
    cell_quad(c, mem[r], c->ngeo, f_arow, &q);
    for (int k = 0; k < K; k++) A[r * K + k] = q.s[k];
  }
}

/* P [K][M] = A^+ diag(V_m) */
static int lsq_pinv(const double *A, int M, int K, const double *Vm, double *P) {
  double Q[ORC_MAXM * ORC_MAXK], R[ORC_MAXK * ORC_MAXK];
  memset(R, 0, sizeof R);
  /* rank test against the largest column: a column that vanishes (every
     member shares the cell's mean of that mode) is as deficient as one that
     depends on the others */
  double amax = 0;
  for (int j = 0; j < K; j++) {
    double n = 0;
    for (int r = 0; r < M; r++) n += A[r * K + j] * A[r * K + j];
    amax = fmax(amax, n);
  }
  for (int j = 0; j < K; j++) {
    double v[ORC_MAXM], n0 = 0;
    for (int r = 0; r < M; r++) { v[r] = A[r * K + j]; n0 += v[r] * v[r]; }
    for (int pass = 0; pass < 2; pass++)
      for (int l = 0; l < j; l++) {
        double d = 0;
        for (int r = 0; r < M; r++) d += Q[r * K + l] * v[r];
        R[l * K + j] += d;
        for (int r = 0; r < M; r++) v[r] -= d * Q[r * K + l];
      }
    double nv = 0;
    for (int r = 0; r < M; r++) nv += v[r] * v[r];
    nv = sqrt(nv);
    if (!(nv > 1e-10 * sqrt(n0)) || !(nv > 1e-8 * sqrt(amax))) {
      set_err("rank-deficient least-squares stencil");
      return -1;
    }
    R[j * K + j] = nv;
    for (int r = 0; r < M; r++) Q[r * K + j] = v[r] / nv;
  }
  /* R^{-1} by back substitution, column by column */
  double Ri[ORC_MAXK * ORC_MAXK];
  memset(Ri, 0, sizeof Ri);
  for (int col = 0; col < K; col++)
    for (int row = col; row >= 0; row--) {
      double s = (row == col) ? 1.0 : 0.0;
      for (int l = row + 1; l <= col; l++) s -= R[row * K + l] * Ri[l * K + col];
      Ri[row * K + col] = s / R[row * K + row];
    }
  for (int k = 0; k < K; k++)
    for (int r = 0; r < M; r++) {
      double s = 0;
      for (int l = 0; l < K; l++) s += Ri[k * K + l] * Q[r * K + l];
      P[k * M + r] = s * Vm[r];
    }
  return 0;
}

static int ensure_cell(orc_case *c, int64_t i) {
  if (c->ready[i]) return 0;
  cand buf[256];
  int n = bfs(c, i, -1, c->order == 4 ? 4 : 3, buf, 256);  /* 2K = 68 members at P4 need 4 layers */
  if (n < 0) { set_err("stencil search overflow"); return -1; }
  for (int q = 1; q < n; q++) buf[q].shared = shared_nodes(c, i, buf[q].id);
  qsort(buf + 1, n - 1, sizeof(cand), cmp_central);
  if (n - 1 < c->Mc) { set_err("too few cells for the central stencil"); return -1; }
  int64_t *sc = &c->sc[i * c->Mc];
  signed char *ss = &c->scsh[i * c->Mc * 3];
  double Vm[ORC_MAXM], A[ORC_MAXM * ORC_MAXK];
  for (int r = 0; r < c->Mc; r++) {
    sc[r] = buf[1 + r].id;
    image_shift(c, i, sc[r], &ss[3 * r]);
    Vm[r] = c->vol[sc[r]];
  }
  lsq_matrix(c, i, c->Mc, sc, ss, c->K, A);
  if (lsq_pinv(A, c->Mc, c->K, Vm, &c->Pc[i * c->K * c->Mc])) return -1;
  for (int s = 0; s < c->nd; s++) {
    int64_t nf = face_nbr(c, i, s);
    c->dvalid[i * c->nd + s] = nf >= 0;
    if (nf < 0) continue;  /* a wall face: no directional candidate there */
    int m = bfs(c, nf, i, c->Kd == 3 ? 2 : 3, buf, 256);
    if (m < 0) { set_err("stencil search overflow"); return -1; }
    qsort(buf + 1, m - 1, sizeof(cand), cmp_dir);
    if (m < c->Md) { set_err("too few cells for a directional stencil"); return -1; }
    int64_t *sd = &c->sd[(i * c->nd + s) * c->Md];
    signed char *ds = &c->sdsh[(i * c->nd + s) * c->Md * 3];
    for (int r = 0; r < c->Md; r++) {
      sd[r] = buf[r].id;
      image_shift(c, i, sd[r], &ds[3 * r]);
      Vm[r] = c->vol[sd[r]];
    }
    lsq_matrix(c, i, c->Md, sd, ds, c->Kd, A);
    if (lsq_pinv(A, c->Md, c->Kd, Vm, &c->Pd[(i * c->nd + s) * c->Kd * c->Md])) return -1;
  }
  c->ready[i] = 1;
  return 0;
}

static int ensure_all(orc_case *c) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t i = 0; i < c->N; i++)
    if (ensure_cell(c, i)) bad = 1;
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Smoothness indicator (reading of Eq. 6): SI = sum over 1<=|beta|<=r of   */
/* V^(2|beta|/3 - 1) int_V (d^beta p)^2 dV, integrated by quadrature.        */
/* ------------------------------------------------------------------------ */
typedef struct { double c[3], h, w1, w2, w3, w4; const double *a; int deg; double s; } si_ctx;
static void f_si(void *ctx, const double x[3], double w) {
  si_ctx *q = (si_ctx *)ctx;
  double xi[3], g[ORC_MAXK][3], H[ORC_MAXK][6];
  for (int d = 0; d < 3; d++) xi[d] = (x[d] - q->c[d]) / q->h;
  int K = q->deg == 1 ? 3 : (q->deg == 2 ? 9 : (q->deg == 3 ? 19 : 34));
  psi_grad(xi, g, K);
  psi_hess(xi, H, K);
  for (int j = 0; j < 3; j++) {
    double d = 0;
    for (int k = 0; k < K; k++) d += q->a[k] * g[k][j] / q->h;
    q->s += w * q->w1 * d * d;
  }
  if (q->deg >= 2)
    for (int j = 0; j < 6; j++) {
      double d = 0;
      for (int k = 0; k < K; k++) d += q->a[k] * H[k][j] / (q->h * q->h);
      q->s += w * q->w2 * d * d;
    }
  if (q->deg >= 3)
    for (int j = 0; j < 10; j++) {
      double d = 0;
      for (int k = 0; k < K; k++) d += q->a[k] * mono_d(MONO[k], DER3[j], xi) / (q->h * q->h * q->h);
      q->s += w * q->w3 * d * d;
    }
  if (q->deg == 4)
    for (int j = 0; j < 15; j++) {
      double d = 0;
      for (int k = 0; k < K; k++) d += q->a[k] * mono_d(MONO[k], DER4[j], xi) / (q->h * q->h * q->h * q->h);
      q->s += w * q->w4 * d * d;
    }
}
static double smoothness(const orc_case *c, int64_t i, const double *a, int deg) {
  si_ctx q;
  for (int d = 0; d < 3; d++) q.c[d] = c->cen[3 * i + d];
  q.h = c->hh[i];
  q.w1 = pow(c->vol[i], 2.0 / 3.0 - 1.0);  /* |beta| = 1 */
  q.w2 = pow(c->vol[i], 4.0 / 3.0 - 1.0);  /* |beta| = 2 */
  q.w3 = c->vol[i];                        /* |beta| = 3: V^(6/3 - 1) */
  q.w4 = pow(c->vol[i], 8.0 / 3.0 - 1.0);  /* |beta| = 4 */
  q.a = a;
  q.deg = deg;
  q.s = 0;
  /* (d p)^2 of a cubic (quartic) is of degree 4 (6): one more point per direction */
  cell_quad(c, i, deg >= 3 ? c->ngeo + 1 : c->ngeo, f_si, &q);
  return q.s;
}

/* ------------------------------------------------------------------------ */
/* Reconstruction of cell i from gathered values (Eqs. 3-6).                 */
/* coef[5][K]: final polynomial p = U_i + sum_k coef_k phi_k.                */
/* ------------------------------------------------------------------------ */
static void recon_from_values(const orc_case *c, int64_t i, const double Ui[5],
                              const double *Uc /* [Mc][5] */, const double *Ud /* [nd][Md][5] */,
                              double coef[5][ORC_MAXK], double *wout /* [5][nd+1] or NULL */) {
  const double *Pc = &c->Pc[i * c->K * c->Mc];
  for (int v = 0; v < 5; v++) {
    double aopt[ORC_MAXK];
    for (int k = 0; k < c->K; k++) {
      double s = 0;
      for (int r = 0; r < c->Mc; r++) s += Pc[k * c->Mc + r] * (Uc[r * 5 + v] - Ui[v]);
      aopt[k] = s;
    }
    /* a cell that the mask routes to the linear weights keeps p_opt itself
       (omega_s = lambda_s makes sum_s lambda_s p_s = p_opt, Sec. 2.2) */
    if (c->scheme == 0 || c->nd == 0 || (c->mask && !c->mask[i])) {
      for (int k = 0; k < c->K; k++) coef[v][k] = aopt[k];
      if (wout) { wout[v * (c->nd + 1)] = 1.0; for (int s = 0; s < c->nd; s++) wout[v * (c->nd + 1) + 1 + s] = 0.0; }
      continue;
    }
    /* CWENOZ: s = 0 central (p_opt defines SI_1), s = 1..nd directional */
    int st = c->nd + 1;
    double as[ORC_MAXD + 1][ORC_MAXK], lam[ORC_MAXD + 1], SI[ORC_MAXD + 1], wt[ORC_MAXD + 1];
    /* candidates: the central one and the directional ones that exist (a
       wall face has none); linear weights normalised over those */
    const unsigned char *dv = &c->dvalid[i * c->nd];
    int nv = 0;
    for (int s = 1; s < st; s++) nv += dv[s - 1];
    double lsum = c->lamc + nv * 1.0;
    lam[0] = c->lamc / lsum;
    for (int s = 1; s < st; s++) lam[s] = dv[s - 1] ? 1.0 / lsum : 0.0;
    for (int s = 1; s < st; s++) {
      if (!dv[s - 1]) continue;
      const double *Pd = &c->Pd[(i * c->nd + (s - 1)) * c->Kd * c->Md];
      for (int k = 0; k < c->K; k++) as[s][k] = 0.0;
      for (int k = 0; k < c->Kd; k++) {
        double t = 0;
        for (int r = 0; r < c->Md; r++) t += Pd[k * c->Md + r] * (Ud[((s - 1) * c->Md + r) * 5 + v] - Ui[v]);
        as[s][k] = t;
      }
    }
    SI[0] = smoothness(c, i, aopt, c->order);
    for (int s = 1; s < st; s++) SI[s] = dv[s - 1] ? smoothness(c, i, as[s], c->Kd == 3 ? 1 : 2) : 0.0;
    /* central candidate p_1 = (p_opt - sum_{s>=2} lam_s p_s) / lam_1 */
    for (int k = 0; k < c->K; k++) {
      double t = aopt[k];
      for (int s = 1; s < st; s++)
        if (dv[s - 1]) t -= lam[s] * as[s][k];
      as[0][k] = t / lam[0];
    }
    double tau = 0;
    for (int s = 1; s < st; s++)
      if (dv[s - 1]) tau += fabs(SI[0] - SI[s]);
    tau /= (double)nv;
    double wsum = 0;
    for (int s = 0; s < st; s++) {
      wt[s] = (s == 0 || dv[s - 1]) ? lam[s] * (1.0 + tau / (c->eps + SI[s])) : 0.0;
      wsum += wt[s];
    }
    for (int s = 0; s < st; s++) wt[s] /= wsum;
    for (int k = 0; k < c->K; k++) {
      double t = 0;
      for (int s = 0; s < st; s++)
        if (s == 0 || dv[s - 1]) t += wt[s] * as[s][k];
      coef[v][k] = t;
    }
    if (wout)
      for (int s = 0; s < st; s++) wout[v * st + s] = wt[s];
  }
}

static void recon_cell(const orc_case *c, int64_t i, const double *U, double coef[5][ORC_MAXK],
                       double *wout) {
  int64_t N = c->N;
  double Ui[5], Uc[ORC_MAXM * 5], Ud[ORC_MAXD * ORC_MD * 5];
  for (int v = 0; v < 5; v++) Ui[v] = U[v * N + i];
  for (int r = 0; r < c->Mc; r++)
    for (int v = 0; v < 5; v++) Uc[r * 5 + v] = U[v * N + c->sc[i * c->Mc + r]];
  for (int s = 0; s < c->nd; s++)
    if (c->dvalid[i * c->nd + s])
      for (int r = 0; r < c->Md; r++)
        for (int v = 0; v < 5; v++)
          Ud[(s * c->Md + r) * 5 + v] = U[v * N + c->sd[(i * c->nd + s) * c->Md + r]];
  recon_from_values(c, i, Ui, Uc, Ud, coef, wout);
}

/* value and gradient of cell i's polynomial at point x (cell i's frame) */
static void eval_poly(const orc_case *c, int64_t i, const double Ui[5], double coef[5][ORC_MAXK],
                      const double x[3], double val[5], double grad[5][3]) {
  double xi[3], p[ORC_MAXK], g[ORC_MAXK][3];
  for (int d = 0; d < 3; d++) xi[d] = (x[d] - c->cen[3 * i + d]) / c->hh[i];
  psi_eval(xi, p, c->K);
  psi_grad(xi, g, c->K);
  const double *pb = &c->psib[ORC_MAXK * i];
  for (int v = 0; v < 5; v++) {
    double s = Ui[v];
    for (int k = 0; k < c->K; k++) s += coef[v][k] * (p[k] - pb[k]);
    val[v] = s;
    for (int j = 0; j < 3; j++) {
      double t = 0;
      for (int k = 0; k < c->K; k++) t += coef[v][k] * g[k][j];
      grad[v][j] = t / c->hh[i];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* HLLC flux (Toro, Spruce & Speares) with Einfeldt/Roe wave-speed bounds.  */
/* F = flux per unit area through unit normal n.                             */
/* ------------------------------------------------------------------------ */
static void phys_flux(const double U[5], const double n[3], double g, double F[5], double *p_out,
                      double *un_out) {
  double r = U[0], u[3] = {U[1] / r, U[2] / r, U[3] / r};
  double p = (g - 1.0) * (U[4] - 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  F[0] = r * un;
  for (int d = 0; d < 3; d++) F[1 + d] = r * u[d] * un + p * n[d];
  F[4] = (U[4] + p) * un;
  *p_out = p;
  *un_out = un;
}

void orc_hllc(const double UL[5], const double UR[5], const double n[3], double g, double F[5]) {
  double FL[5], FR[5], pL, pR, unL, unR;
  phys_flux(UL, n, g, FL, &pL, &unL);
  phys_flux(UR, n, g, FR, &pR, &unR);
  double rL = UL[0], rR = UR[0];
  double uL[3] = {UL[1] / rL, UL[2] / rL, UL[3] / rL}, uR[3] = {UR[1] / rR, UR[2] / rR, UR[3] / rR};
  double aL = sqrt(g * pL / rL), aR = sqrt(g * pR / rR);
  double HL = (UL[4] + pL) / rL, HR = (UR[4] + pR) / rR;
  double sL = sqrt(rL), sR = sqrt(rR);
  double ut[3], q2 = 0, utn = 0;
  for (int d = 0; d < 3; d++) {
    ut[d] = (sL * uL[d] + sR * uR[d]) / (sL + sR);
    q2 += ut[d] * ut[d];
    utn += ut[d] * n[d];
  }
  double Ht = (sL * HL + sR * HR) / (sL + sR);
  double at = sqrt((g - 1.0) * (Ht - 0.5 * q2));
  double SL = fmin(unL - aL, utn - at);
  double SR = fmax(unR + aR, utn + at);
  double Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) /
              (rL * (SL - unL) - rR * (SR - unR));
  if (0.0 <= SL) {
    memcpy(F, FL, sizeof FL);
  } else if (0.0 <= Ss) {
    double f = rL * (SL - unL) / (SL - Ss), Us[5];
    Us[0] = f;
    for (int d = 0; d < 3; d++) Us[1 + d] = f * (uL[d] + (Ss - unL) * n[d]);
    Us[4] = f * (UL[4] / rL + (Ss - unL) * (Ss + pL / (rL * (SL - unL))));
    for (int v = 0; v < 5; v++) F[v] = FL[v] + SL * (Us[v] - UL[v]);
  } else if (0.0 <= SR) {
    double f = rR * (SR - unR) / (SR - Ss), Us[5];
    Us[0] = f;
    for (int d = 0; d < 3; d++) Us[1 + d] = f * (uR[d] + (Ss - unR) * n[d]);
    Us[4] = f * (UR[4] / rR + (Ss - unR) * (Ss + pR / (rR * (SR - unR))));
    for (int v = 0; v < 5; v++) F[v] = FR[v] + SR * (Us[v] - UR[v]);
  } else {
    memcpy(F, FR, sizeof FR);
  }
}

/* ------------------------------------------------------------------------ */
/* Viscous flux F_v . n from a face state and conserved-variable gradient:  */
/* Newtonian stress with Stokes' hypothesis, Fourier heat flux, constant    */
/* mu = 1/Re, R = 1/(gamma M^2), kappa = mu c_p / Pr.                        */
/* ------------------------------------------------------------------------ */
void orc_viscous_flux(const double Uf[5], const double gU[15], const double n[3], double g,
                      double Re, double Pr, double Mach, double Fv[5]) {
  double mu = 1.0 / Re, Rg = 1.0 / (g * Mach * Mach), cp = g * Rg / (g - 1.0), kap = mu * cp / Pr;
  double r = Uf[0], u[3] = {Uf[1] / r, Uf[2] / r, Uf[3] / r}, E = Uf[4];
  double gu[3][3], gT[3];
  for (int a = 0; a < 3; a++)
    for (int j = 0; j < 3; j++) gu[a][j] = (gU[(1 + a) * 3 + j] - u[a] * gU[j]) / r;
  for (int j = 0; j < 3; j++) {
    double de = gU[12 + j] / r - E * gU[j] / (r * r);
    for (int a = 0; a < 3; a++) de -= u[a] * gu[a][j];
    gT[j] = (g - 1.0) / Rg * de;
  }
  double div = gu[0][0] + gu[1][1] + gu[2][2];
  Fv[0] = 0.0;
  double work = 0.0;
  for (int a = 0; a < 3; a++) {
    double t = 0;
    for (int j = 0; j < 3; j++) {
      double tau = mu * (gu[a][j] + gu[j][a]) - (a == j ? 2.0 / 3.0 * mu * div : 0.0);
      t += tau * n[j];
    }
    Fv[1 + a] = t;
    work += u[a] * t;
  }
  Fv[4] = work + kap * (gT[0] * n[0] + gT[1] * n[1] + gT[2] * n[2]);
}

/* ------------------------------------------------------------------------ */
/* Residual (Eq. 2): reconstruct every cell, integrate every face once,     */
/* then R_i = -(1/|V_i|) sum_f sigma_if G_f.                                 */
/* ------------------------------------------------------------------------ */
/* flux integral G_f of face f (owner-outward), from the reconstructions */
/* the box side of a boundary face from its outward area vector (the axis of
   its largest component and that component's sign), and that side's kind */
static int boundary_kind(const orc_case *c, double dS[][3]) {
  double s[3] = {0, 0, 0};
  for (int q = 0; q < c->nq; q++)
    for (int d = 0; d < 3; d++) s[d] += dS[q][d];
  int ax = 0;
  for (int d = 1; d < 3; d++)
    if (fabs(s[d]) > fabs(s[ax])) ax = d;
  return c->bc[2 * ax + (s[ax] > 0 ? 1 : 0)];
}

static void face_flux(const orc_case *c, int64_t f, const double *U, const double *coef, double g[5]) {
  int64_t N = c->N, o = c->fo[f], nb = c->fn[f];
  double x[32][3], dS[32][3], Uo[5], Un[5], shv[3];
  for (int v = 0; v < 5; v++) g[v] = 0.0;
  if (nb < 0) {
    /* a boundary face: the ghost state at each Gauss point is, by the kind of
       its box side, the mirror of the owner's reconstructed state (slip wall:
       same density and energy, normal momentum reversed), that state itself
       (supersonic outflow: extrapolation), or the given inflow state
       (supersonic inflow); HLLC between the two (inviscid flows only) */
    for (int v = 0; v < 5; v++) Uo[v] = U[v * N + o];
    face_quad(c, f, x, dS);
    const int kind = boundary_kind(c, dS);
    for (int q = 0; q < c->nq; q++) {
      double UL[5], UR[5], gL[5][3], nh[3], A, Fc[5];
      eval_poly(c, o, Uo, (double(*)[ORC_MAXK]) & coef[o * 5 * ORC_MAXK], x[q], UL, gL);
      A = sqrt(dS[q][0] * dS[q][0] + dS[q][1] * dS[q][1] + dS[q][2] * dS[q][2]);
      for (int d = 0; d < 3; d++) nh[d] = dS[q][d] / A;
      if (kind == 2) {
        for (int v = 0; v < 5; v++) UR[v] = UL[v];
      } else if (kind == 3) {
        for (int v = 0; v < 5; v++) UR[v] = c->uinf[v];
      } else {
        double mn = UL[1] * nh[0] + UL[2] * nh[1] + UL[3] * nh[2];
        UR[0] = UL[0];
        for (int d = 0; d < 3; d++) UR[1 + d] = UL[1 + d] - 2.0 * mn * nh[d];
        UR[4] = UL[4];
      }
      orc_hllc(UL, UR, nh, c->gam, Fc);
      for (int v = 0; v < 5; v++) g[v] += Fc[v] * A;
    }
    return;
  }
  for (int d = 0; d < 3; d++) shv[d] = c->fsh[3 * f + d] * c->L[d];
  for (int v = 0; v < 5; v++) { Uo[v] = U[v * N + o]; Un[v] = U[v * N + nb]; }
  face_quad(c, f, x, dS);
  double Lint = 0;
  for (int d = 0; d < 3; d++) {
    double dd = c->cen[3 * nb + d] + shv[d] - c->cen[3 * o + d];
    Lint += dd * dd;
  }
  Lint = sqrt(Lint);
  for (int q = 0; q < c->nq; q++) {
    double UL[5], UR[5], gL[5][3], gR[5][3], xr[3], nh[3], A, Fc[5], Fv[5] = {0, 0, 0, 0, 0};
    eval_poly(c, o, Uo, (double(*)[ORC_MAXK]) & coef[o * 5 * ORC_MAXK], x[q], UL, gL);
    for (int d = 0; d < 3; d++) xr[d] = x[q][d] - shv[d];
    eval_poly(c, nb, Un, (double(*)[ORC_MAXK]) & coef[nb * 5 * ORC_MAXK], xr, UR, gR);
    A = sqrt(dS[q][0] * dS[q][0] + dS[q][1] * dS[q][1] + dS[q][2] * dS[q][2]);
    for (int d = 0; d < 3; d++) nh[d] = dS[q][d] / A;
    orc_hllc(UL, UR, nh, c->gam, Fc);
    if (!c->inviscid) {
      double Uf[5], gf[15];
      for (int v = 0; v < 5; v++) {
        Uf[v] = 0.5 * (UL[v] + UR[v]);
        for (int j = 0; j < 3; j++)
          gf[v * 3 + j] = 0.5 * (gL[v][j] + gR[v][j]) + c->alpha / Lint * (UR[v] - UL[v]) * nh[j];
      }
      orc_viscous_flux(Uf, gf, nh, c->gam, c->Re, c->Pr, c->Mach, Fv);
    }
    for (int v = 0; v < 5; v++) g[v] += (Fc[v] - Fv[v]) * A;
  }
}

/* R_i = -(1/|V_i|) sum_f sigma_if G_f; optionally also the magnitude of the
 * summed terms, S_i = (1/|V_i|) sum_f |G_f| (the scale of the rounding error
 * of the signed sum). */
static int residual_terms(orc_case *c, const double *U, double *R, double *S) {
  if (ensure_all(c)) return -1;
  int64_t N = c->N;
  double *coef = (double *)malloc(sizeof(double) * N * 5 * ORC_MAXK);
  double *G = (double *)malloc(sizeof(double) * c->F * 5);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++)
    recon_cell(c, i, U, (double(*)[ORC_MAXK]) & coef[i * 5 * ORC_MAXK], NULL);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < c->F; f++) face_flux(c, f, U, coef, &G[f * 5]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++)
    for (int v = 0; v < 5; v++) {
      double s = 0;
      for (int j = 0; j < c->nfc; j++) s += c->cs[i * c->nfc + j] * G[c->cf[i * c->nfc + j] * 5 + v];
      R[v * N + i] = -s / c->vol[i];
      if (S) {
        double a = 0;
        for (int j = 0; j < c->nfc; j++) a += fabs(G[c->cf[i * c->nfc + j] * 5 + v]);
        S[v * N + i] = a / c->vol[i];
      }
    }
  free(coef);
  free(G);
  return 0;
}

static int residual(orc_case *c, const double *U, double *R) { return residual_terms(c, U, R, NULL); }

/* Residual of a sample of cells only (same arithmetic as residual(); used to
 * time the oracle on a bounded part of a large mesh).  R: [5][ns]. */
int orc_residual_subset_terms(orc_case *c, const double *U, int64_t ns, const int64_t *sel, double *R,
                              double *S);
int orc_residual_subset(orc_case *c, const double *U, int64_t ns, const int64_t *sel, double *R) {
  return orc_residual_subset_terms(c, U, ns, sel, R, NULL);
}
/* ... and S_k = (1/|V_i|) sum_f |G_f| of each sampled cell (may be NULL) */
int orc_residual_subset_terms(orc_case *c, const double *U, int64_t ns, const int64_t *sel, double *R,
                              double *S) {
  int64_t N = c->N;
  unsigned char *need = (unsigned char *)calloc(N, 1);
  for (int64_t k = 0; k < ns; k++) {
    if (sel[k] < 0 || sel[k] >= N) { free(need); set_err("cell id out of range"); return -1; }
    need[sel[k]] = 1;
    for (int j = 0; j < c->nfc; j++) {
      int64_t m = face_nbr(c, sel[k], j);
      if (m >= 0) need[m] = 1;
    }
  }
  int64_t nl = 0;
  int64_t *list = (int64_t *)malloc(sizeof(int64_t) * N);
  for (int64_t i = 0; i < N; i++)
    if (need[i]) list[nl++] = i;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t k = 0; k < nl; k++)
    if (ensure_cell(c, list[k])) bad = 1;
  double *coef = bad ? NULL : (double *)malloc(sizeof(double) * N * 5 * ORC_MAXK);
  int64_t *fid = NULL, nf = 0;
  double *G = NULL;
  if (!bad) {
    /* each face of the sample once */
    unsigned char *fneed = (unsigned char *)calloc(c->F, 1);
    for (int64_t k = 0; k < ns; k++)
      for (int j = 0; j < c->nfc; j++) fneed[c->cf[sel[k] * c->nfc + j]] = 1;
    fid = (int64_t *)malloc(sizeof(int64_t) * c->F);
    int64_t *fpos = (int64_t *)malloc(sizeof(int64_t) * c->F);
    for (int64_t f = 0; f < c->F; f++)
      if (fneed[f]) { fpos[f] = nf; fid[nf++] = f; }
    G = (double *)malloc(sizeof(double) * 5 * (nf ? nf : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nl; k++)
      recon_cell(c, list[k], U, (double(*)[ORC_MAXK]) & coef[list[k] * 5 * ORC_MAXK], NULL);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nf; q++) face_flux(c, fid[q], U, coef, &G[5 * q]);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < ns; k++) {
      int64_t i = sel[k];
      double s[5] = {0, 0, 0, 0, 0};
      for (int j = 0; j < c->nfc; j++) {
        const double *g = &G[5 * fpos[c->cf[i * c->nfc + j]]];
        for (int v = 0; v < 5; v++) s[v] += c->cs[i * c->nfc + j] * g[v];
      }
      for (int v = 0; v < 5; v++) R[v * ns + k] = -s[v] / c->vol[i];
      if (S)
        for (int v = 0; v < 5; v++) {
          double t = 0;
          for (int j = 0; j < c->nfc; j++) t += fabs(G[5 * fpos[c->cf[i * c->nfc + j]] + v]);
          S[v * ns + k] = t / c->vol[i];
        }
    }
    free(fneed);
    free(fpos);
  }
  free(fid);
  free(G);
  free(coef);
  free(list);
  free(need);
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Time step: dt = CFL * min_i min(h_i/(|u_i|+a_i), rho_i h_i^2 Pr/(2 g mu)) */
/* with h_i = 2 |V_i| / sum_f |S_f| (cube: side/3).                         */
/* ------------------------------------------------------------------------ */
static double face_area(const orc_case *c, int64_t f) {
  double x[32][3], dS[32][3], s[3] = {0, 0, 0};
  face_quad(c, f, x, dS);
  for (int q = 0; q < c->nq; q++)
    for (int d = 0; d < 3; d++) s[d] += dS[q][d];
  return sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
}

static double time_step(const orc_case *c, const double *U) {
  int64_t N = c->N;
  double dt = INFINITY;
  for (int64_t i = 0; i < N; i++) {
    double r = U[i], u[3] = {U[N + i] / r, U[2 * N + i] / r, U[3 * N + i] / r};
    double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double p = (c->gam - 1.0) * (U[4 * N + i] - 0.5 * r * q2);
    double a = sqrt(c->gam * p / r), asum = 0;
    for (int j = 0; j < c->nfc; j++) asum += face_area(c, c->cf[i * c->nfc + j]);
    double h = 2.0 * c->vol[i] / asum;
    double d = h / (sqrt(q2) + a);
    if (!c->inviscid) {
      double dv = r * h * h * c->Pr / (2.0 * c->gam * (1.0 / c->Re));
      if (dv < d) d = dv;
    }
    if (d < dt) dt = d;
  }
  return c->cfl * dt;
}

/* ------------------------------------------------------------------------ */
/* SSP-RK3 (Shu-Osher form) on a generic residual.                           */
/* ------------------------------------------------------------------------ */
typedef int (*res_fn)(void *ctx, const double *U, double *R);
int orc_ssprk3_generic(res_fn f, void *ctx, double *U, int64_t n, double dt) {
  double *U0 = (double *)malloc(sizeof(double) * n), *U1 = (double *)malloc(sizeof(double) * n),
         *R = (double *)malloc(sizeof(double) * n);
  memcpy(U0, U, sizeof(double) * n);
  int rc = f(ctx, U0, R);
  for (int64_t k = 0; k < n && !rc; k++) U1[k] = U0[k] + dt * R[k];
  if (!rc) rc = f(ctx, U1, R);
  for (int64_t k = 0; k < n && !rc; k++) U1[k] = 0.75 * U0[k] + 0.25 * (U1[k] + dt * R[k]);
  if (!rc) rc = f(ctx, U1, R);
  for (int64_t k = 0; k < n && !rc; k++) U[k] = U0[k] / 3.0 + 2.0 / 3.0 * (U1[k] + dt * R[k]);
  free(U0); free(U1); free(R);
  return rc;
}

/* scalar linear test equation dU/dt = lambda U through the same stepper */
static int lin_res(void *ctx, const double *U, double *R) {
  R[0] = *(const double *)ctx * U[0];
  return 0;
}
double orc_ssprk3_linear(double lambda, double dt, double u0) {
  double u = u0;
  orc_ssprk3_generic(lin_res, &lambda, &u, 1, dt);
  return u;
}

/* ------------------------------------------------------------------------ */
/* SSP(5,4) of Spiteri and Ruuth (the fourth-order SSP scheme of Eq. 8) in   */
/* Shu-Osher form: u_0 = U^n and, for i = 1..5,                              */
/*   u_i = sum_{j<i} ( alpha_ij u_j + dt beta_ij L(u_j) ),  U^{n+1} = u_5,    */
/* with the published 15-digit coefficients (zero entries omitted there).    */
/* ------------------------------------------------------------------------ */
static const double SSP54_ALPHA[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0, 0, 0, 0, 0},
    {0.444370493651235, 0.555629506348765, 0, 0, 0},
    {0.620101851488403, 0, 0.379898148511597, 0, 0},
    {0.178079954393132, 0, 0, 0.821920045606868, 0},
    {0, 0, 0.517231671970585, 0.096059710526147, 0.386708617503269}};
static const double SSP54_BETA[6][5] = {
    {0, 0, 0, 0, 0},
    {0.391752226571890, 0, 0, 0, 0},
    {0, 0.368410593050371, 0, 0, 0},
    {0, 0, 0.251891774271694, 0, 0},
    {0, 0, 0, 0.544974750228521, 0},
    {0, 0, 0, 0.063692468666290, 0.226007483236906}};

int orc_ssp54_generic(res_fn f, void *ctx, double *U, int64_t n, double dt) {
  double *u[5], *L[5];
  int rc = 0;
  for (int j = 0; j < 5; j++) {
    u[j] = (double *)malloc(sizeof(double) * n);
    L[j] = (double *)malloc(sizeof(double) * n);
  }
  memcpy(u[0], U, sizeof(double) * n);
  for (int i = 1; i <= 5 && !rc; i++) {
    rc = f(ctx, u[i - 1], L[i - 1]);  /* every stage value is needed once its stage exists */
    double *dst = i < 5 ? u[i] : U;
    for (int64_t k = 0; k < n && !rc; k++) {
      double v = 0.0;
      for (int j = 0; j < i; j++) v += SSP54_ALPHA[i][j] * u[j][k] + dt * SSP54_BETA[i][j] * L[j][k];
      dst[k] = v;
    }
  }
  for (int j = 0; j < 5; j++) { free(u[j]); free(L[j]); }
  return rc;
}

/* the Shu-Osher coefficients as stored, alpha then beta, row-major [6][5] each */
void orc_ssp54_coeffs(double *out) {
  memcpy(out, SSP54_ALPHA, sizeof SSP54_ALPHA);
  memcpy(out + 30, SSP54_BETA, sizeof SSP54_BETA);
}

double orc_ssp54_linear(double lambda, double dt, double u0) {
  double u = u0;
  orc_ssp54_generic(lin_res, &lambda, &u, 1, dt);
  return u;
}

/* logistic equation u' = u (1 - u), a nonlinear scalar test problem:
   n steps of size T/n from u0 with SSP(5,4) */
static int logistic_res(void *ctx, const double *U, double *R) {
  (void)ctx;
  R[0] = U[0] * (1.0 - U[0]);
  return 0;
}
double orc_ssp54_logistic(double u0, double T, int n) {
  double u = u0;
  for (int k = 0; k < n; k++) orc_ssp54_generic(logistic_res, NULL, &u, 1, T / n);
  return u;
}
double orc_ssprk3_logistic(double u0, double T, int n) {
  double u = u0;
  for (int k = 0; k < n; k++) orc_ssprk3_generic(logistic_res, NULL, &u, 1, T / n);
  return u;
}

static int case_res(void *ctx, const double *U, double *R) { return residual((orc_case *)ctx, U, R); }

/* ------------------------------------------------------------------------ */
/* Public entry points.                                                      */
/* ------------------------------------------------------------------------ */
/* params: [order, scheme(0 linear,1 cwenoz), gamma, Pr, Re(<=0 inviscid),   */
/*          Mach, cfl, lambda_central, eps, alpha]                           */
void orc_destroy(orc_case *c);
orc_case *orc_create(const double *nodes, int64_t nn, const int64_t *cells, int64_t N, int npc,
                     const double *box, const double *params) {
  if (!(npc == 8 || npc == 6 || npc == 5 || npc == 4) || N < 1 || nn < 1) { set_err("bad arguments"); return NULL; }
  orc_case *c = (orc_case *)calloc(1, sizeof(orc_case));
  c->N = N; c->nn = nn; c->npc = npc;
  c->nfc = npc == 8 ? 6 : (npc == 6 || npc == 5 ? 5 : 4);
  for (int d = 0; d < 3; d++) {
    c->L[d] = box ? box[d] : 0.0;
    c->per[d] = box && box[d] > 0;
  }
  c->order = (int)params[0];
  c->scheme = (int)params[1];
  c->gam = params[2]; c->Pr = params[3]; c->Re = params[4];
  c->inviscid = !(params[4] > 0);
  c->Mach = params[5]; c->cfl = params[6]; c->lamc = params[7]; c->eps = params[8];
  c->alpha = params[9];
  c->rk = (int)params[10];
  for (int k = 0; k < 6; k++) c->bc[k] = (int)params[11 + k];
  for (int v = 0; v < 5; v++) c->uinf[v] = params[17 + v];
  if (c->order < 1 || c->order > 4) { set_err("order must be 1, 2, 3 or 4"); free(c); return NULL; }
  if (c->order >= 3 && npc != 8) { set_err("orders 3 and 4 are built for hexahedra only"); free(c); return NULL; }
  if (c->rk != 0 && c->rk != 1) { set_err("integrator must be 0 (SSP-RK3) or 1 (SSP(5,4))"); free(c); return NULL; }
  c->K = c->order == 1 ? 3 : (c->order == 2 ? 9 : (c->order == 3 ? 19 : 34));
  c->Mc = 2 * c->K;
  c->nd = (c->order >= 2 && c->scheme == 1) ? c->nfc : 0;  /* directional candidates: linear (P2, P3) */
  c->Kd = c->order == 4 ? 9 : 3;  /* quadratic directional candidates at P4 (Sec. 2.2) */
  c->Md = 2 * c->Kd;
  c->nq = c->order * c->order;
  c->ngeo = npc == 8 ? (c->order == 4 ? 4 : 3) : 4;  /* exact for the A-matrix integrands */
  c->X = (double *)malloc(sizeof(double) * 3 * nn);
  memcpy(c->X, nodes, sizeof(double) * 3 * nn);
  c->C = (int64_t *)malloc(sizeof(int64_t) * npc * N);
  memcpy(c->C, cells, sizeof(int64_t) * npc * N);
  for (int64_t k = 0; k < npc * N; k++)
    if (c->C[k] < 0 || c->C[k] >= nn) { set_err("node index out of range"); orc_destroy(c); return NULL; }
  c->canon = (int64_t *)malloc(sizeof(int64_t) * nn);
  c->vol = (double *)malloc(sizeof(double) * N);
  c->cen = (double *)malloc(sizeof(double) * 3 * N);
  c->hh = (double *)malloc(sizeof(double) * N);
  c->psib = (double *)malloc(sizeof(double) * ORC_MAXK * N);
  c->cf = (int64_t *)malloc(sizeof(int64_t) * c->nfc * N);
  c->cs = (signed char *)malloc(c->nfc * N);
  c->sc = (int64_t *)malloc(sizeof(int64_t) * c->Mc * N);
  c->scsh = (signed char *)malloc(3 * c->Mc * N);
  c->Pc = (double *)malloc(sizeof(double) * c->K * c->Mc * N);
  if (c->nd) {
    c->sd = (int64_t *)malloc(sizeof(int64_t) * c->nd * c->Md * N);
    c->sdsh = (signed char *)malloc(3 * c->nd * c->Md * N);
    c->Pd = (double *)malloc(sizeof(double) * c->nd * c->Kd * c->Md * N);
  }
  c->ready = (unsigned char *)calloc(N, 1);
  c->dvalid = (unsigned char *)calloc(c->nd > 0 ? c->nd * N : 1, 1);
  c->walls = !(c->per[0] && c->per[1] && c->per[2]);
  if (c->walls && !c->inviscid) { set_err("slip walls are built for inviscid flows (Re <= 0) only"); orc_destroy(c); return NULL; }
  compute_canon(c);
  if (compute_geometry(c) || build_faces(c)) { orc_destroy(c); return NULL; }
  return c;
}

void orc_destroy(orc_case *c) {
  if (!c) return;
  free(c->X); free(c->C); free(c->canon); free(c->vol); free(c->cen); free(c->hh); free(c->psib);
  free(c->fo); free(c->fn); free(c->flf); free(c->fsh); free(c->cf); free(c->cs);
  free(c->sc); free(c->scsh); free(c->Pc); free(c->sd); free(c->sdsh); free(c->Pd); free(c->ready); free(c->dvalid);
  free(c->mask);
  free(c);
}

/* counts: [N, F, K, Mc, nd, Md, nq, faces per cell] */
void orc_counts(const orc_case *c, int64_t *out) {
  out[0] = c->N; out[1] = c->F; out[2] = c->K; out[3] = c->Mc; out[4] = c->nd; out[5] = c->Md;
  out[6] = c->nq; out[7] = c->nfc;
}

void orc_geometry(const orc_case *c, double *vol, double *cen, double *hh) {
  memcpy(vol, c->vol, sizeof(double) * c->N);
  memcpy(cen, c->cen, sizeof(double) * 3 * c->N);
  memcpy(hh, c->hh, sizeof(double) * c->N);
}

/* faces: owner, neighbour, shift; and per-cell closed-surface sums */
void orc_faces(const orc_case *c, int64_t *fo, int64_t *fn, int32_t *fsh) {
  for (int64_t f = 0; f < c->F; f++) {
    fo[f] = c->fo[f]; fn[f] = c->fn[f];
    for (int d = 0; d < 3; d++) fsh[3 * f + d] = c->fsh[3 * f + d];
  }
}
void orc_face_quad(const orc_case *c, int64_t f, double *x, double *dS) {
  face_quad(c, f, (double(*)[3])x, (double(*)[3])dS);
}
void orc_surface_sums(const orc_case *c, double *out /* [N][3] */) {
  memset(out, 0, sizeof(double) * 3 * c->N);
  for (int64_t f = 0; f < c->F; f++) {
    double x[32][3], dS[32][3];
    face_quad(c, f, x, dS);
    for (int q = 0; q < c->nq; q++)
      for (int d = 0; d < 3; d++) {
        out[3 * c->fo[f] + d] += dS[q][d];
        if (c->fn[f] >= 0) out[3 * c->fn[f] + d] -= dS[q][d];
      }
  }
}

/* stencil members and operators of one cell (which = -1 central, s >= 0 directional) */
int orc_stencil(orc_case *c, int64_t i, int which, int64_t *mem, int32_t *sh, double *A, double *P) {
  if (ensure_cell(c, i)) return -1;
  if (which >= 0 && !c->dvalid[i * c->nd + which]) { set_err("no directional candidate on a wall face"); return -1; }
  int M = which < 0 ? c->Mc : c->Md, K = which < 0 ? c->K : c->Kd;
  const int64_t *m = which < 0 ? &c->sc[i * c->Mc] : &c->sd[(i * c->nd + which) * c->Md];
  const signed char *s = which < 0 ? &c->scsh[i * c->Mc * 3] : &c->sdsh[(i * c->nd + which) * c->Md * 3];
  const double *PP = which < 0 ? &c->Pc[i * c->K * c->Mc] : &c->Pd[(i * c->nd + which) * c->Kd * c->Md];
  for (int r = 0; r < M; r++) {
    mem[r] = m[r];
    for (int d = 0; d < 3; d++) sh[3 * r + d] = s[3 * r + d];
  }
  lsq_matrix(c, i, M, m, s, K, A);
  memcpy(P, PP, sizeof(double) * K * M);
  return 0;
}

/* Per-cell choice of the reconstruction in a CWENOZ case (Sec. 2.2, Eqs.
   5-6): mask[i] != 0 keeps cell i's CWENOZ polynomial, mask[i] == 0 gives it
   the optimal central polynomial p_opt (the linear weights).  Copied; NULL
   restores CWENOZ everywhere.  Every later residual, reconstruction and step
   of the case follows it. */
int orc_set_scheme_mask(orc_case *c, const unsigned char *mask) {
  free(c->mask);
  c->mask = NULL;
  if (!mask) return 0;
  if (c->nd == 0) { set_err("a scheme mask needs a CWENOZ case"); return -1; }
  c->mask = (unsigned char *)malloc(c->N);
  memcpy(c->mask, mask, c->N);
  return 0;
}

int orc_residual(orc_case *c, const double *U, double *R) { return residual(c, U, R); }
int orc_residual_terms(orc_case *c, const double *U, double *R, double *S) {
  return residual_terms(c, U, R, S);
}

/* one step of the case's integrator (SSP-RK3 or SSP(5,4)); dt <= 0 computes
   it from the CFL condition; returns dt */
double orc_rk_step(orc_case *c, double *U, double dt) {
  if (ensure_all(c)) return -1.0;
  if (!(dt > 0)) dt = time_step(c, U);
  int rc = c->rk == 1 ? orc_ssp54_generic(case_res, c, U, 5 * c->N, dt)
                      : orc_ssprk3_generic(case_res, c, U, 5 * c->N, dt);
  if (rc) return -1.0;
  return dt;
}

double orc_time_step(orc_case *c, const double *U) { return time_step(c, U); }

/* final reconstruction coefficients [N][5][K] and, for CWENOZ, weights [N][5][nd+1] */
int orc_reconstruct(orc_case *c, const double *U, double *coef, double *w) {
  if (ensure_all(c)) return -1;
  int st = c->nd + 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->N; i++) {
    double cc[5][ORC_MAXK];
    recon_cell(c, i, U, cc, w ? &w[i * 5 * st] : NULL);
    for (int v = 0; v < 5; v++)
      for (int k = 0; k < c->K; k++) coef[(i * 5 + v) * c->K + k] = cc[v][k];
  }
  return 0;
}

/* evaluate cell i's reconstruction at npts points (cell i's own frame) */
int orc_eval(orc_case *c, const double *U, int64_t i, int npts, const double *x, double *val,
             double *grad) {
  if (ensure_cell(c, i)) return -1;
  for (int64_t q = 0; q < c->Mc; q++)
    if (ensure_cell(c, c->sc[i * c->Mc + q])) return -1;
  double cc[5][ORC_MAXK], Ui[5], g[5][3];
  recon_cell(c, i, U, cc, NULL);
  for (int v = 0; v < 5; v++) Ui[v] = U[v * c->N + i];
  for (int p = 0; p < npts; p++) eval_poly(c, i, Ui, cc, &x[3 * p], &val[5 * p], g), memcpy(&grad[15 * p], g, sizeof g);
  return 0;
}

/* smoothness indicator of a polynomial with coefficients a[K] on cell i */
double orc_smoothness(orc_case *c, int64_t i, const double *a, int deg) {
  return smoothness(c, i, a, deg);
}

/* cell averages of an analytic field (for the k-exactness probe):        */
/* poly[5][10] = constant, x, y, z, xx, yy, zz, xy, xz, yz in absolute x    */
typedef struct { const double *poly; double sh[3], s[5], v; } pa_ctx;
static void f_polyavg(void *ctx, const double x[3], double w) {
  pa_ctx *q = (pa_ctx *)ctx;
  double X = x[0] + q->sh[0], Y = x[1] + q->sh[1], Z = x[2] + q->sh[2];
  double m[10] = {1, X, Y, Z, X * X, Y * Y, Z * Z, X * Y, X * Z, Y * Z};
  for (int v = 0; v < 5; v++) {
    double t = 0;
    for (int k = 0; k < 10; k++) t += q->poly[v * 10 + k] * m[k];
    q->s[v] += w * t;
  }
  q->v += w;
}
static void poly_avg(const orc_case *c, int64_t m, const signed char *sh, const double *poly, double out[5]) {
  pa_ctx q;
  memset(&q, 0, sizeof q);
  q.poly = poly;
  for (int d = 0; d < 3; d++) q.sh[d] = sh ? sh[d] * c->L[d] : 0.0;
  cell_quad(c, m, 5, f_polyavg, &q);
  for (int v = 0; v < 5; v++) out[v] = q.s[v] / q.v;
}

/* the same with a polynomial of degree <= 4 in the physical coordinates:
   nterm = 20 (cubic) or 35 (quartic) terms per variable, 1 then the basis
   monomials in basis order (MONO) of (X, Y, Z) */
typedef struct { const double *poly; int nterm; double sh[3], s[5], v; } pan_ctx;
static void f_polyavgN(void *ctx, const double x[3], double w) {
  pan_ctx *q = (pan_ctx *)ctx;
  double X[3] = {x[0] + q->sh[0], x[1] + q->sh[1], x[2] + q->sh[2]}, m[ORC_MAXK + 1];
  m[0] = 1.0;
  for (int k = 0; k + 1 < q->nterm; k++) m[k + 1] = mono_d(MONO[k], ZERO3, X);
  for (int v = 0; v < 5; v++) {
    double t = 0;
    for (int k = 0; k < q->nterm; k++) t += q->poly[v * q->nterm + k] * m[k];
    q->s[v] += w * t;
  }
  q->v += w;
}
static void poly_avgN(const orc_case *c, int64_t m, const signed char *sh, const double *poly, int nterm,
                      double out[5]) {
  pan_ctx q;
  memset(&q, 0, sizeof q);
  q.poly = poly;
  q.nterm = nterm;
  for (int d = 0; d < 3; d++) q.sh[d] = sh ? sh[d] * c->L[d] : 0.0;
  cell_quad(c, m, 6, f_polyavgN, &q);
  for (int v = 0; v < 5; v++) out[v] = q.s[v] / q.v;
}
int orc_kexact_probeN(orc_case *c, int64_t i, const double *poly, int nterm, int npts, const double *x,
                      double *val, double *grad) {
  if (nterm != 20 && nterm != 35) { set_err("nterm must be 20 or 35"); return -1; }
  if (ensure_cell(c, i)) return -1;
  double Ui[5], Uc[ORC_MAXM * 5], Ud[ORC_MAXD * ORC_MD * 5], cc[5][ORC_MAXK], g[5][3];
  poly_avgN(c, i, NULL, poly, nterm, Ui);
  for (int r = 0; r < c->Mc; r++)
    poly_avgN(c, c->sc[i * c->Mc + r], &c->scsh[(i * c->Mc + r) * 3], poly, nterm, &Uc[5 * r]);
  for (int s = 0; s < c->nd; s++)
    for (int r = 0; r < c->Md && c->dvalid[i * c->nd + s]; r++) {
      int64_t k = (i * c->nd + s) * c->Md + r;
      poly_avgN(c, c->sd[k], &c->sdsh[3 * k], poly, nterm, &Ud[(s * c->Md + r) * 5]);
    }
  recon_from_values(c, i, Ui, Uc, Ud, cc, NULL);
  for (int p = 0; p < npts; p++) eval_poly(c, i, Ui, cc, &x[3 * p], &val[5 * p], g), memcpy(&grad[15 * p], g, sizeof g);
  return 0;
}

/* k-exactness probe: the stencil values of cell i are the averages of the */
/* polynomial over each member's periodic image; reconstruct and evaluate.  */
int orc_kexact_probe(orc_case *c, int64_t i, const double *poly, int npts, const double *x,
                     double *val, double *grad) {
  if (ensure_cell(c, i)) return -1;
  double Ui[5], Uc[ORC_MAXM * 5], Ud[ORC_MAXD * ORC_MD * 5], cc[5][ORC_MAXK], g[5][3];
  poly_avg(c, i, NULL, poly, Ui);
  for (int r = 0; r < c->Mc; r++) poly_avg(c, c->sc[i * c->Mc + r], &c->scsh[(i * c->Mc + r) * 3], poly, &Uc[5 * r]);
  for (int s = 0; s < c->nd; s++)
    for (int r = 0; r < c->Md && c->dvalid[i * c->nd + s]; r++) {
      int64_t k = (i * c->nd + s) * c->Md + r;
      poly_avg(c, c->sd[k], &c->sdsh[3 * k], poly, &Ud[(s * c->Md + r) * 5]);
    }
  recon_from_values(c, i, Ui, Uc, Ud, cc, NULL);
  for (int p = 0; p < npts; p++) eval_poly(c, i, Ui, cc, &x[3 * p], &val[5 * p], g), memcpy(&grad[15 * p], g, sizeof g);
  return 0;
}

/* cell averages of analytic initial fields by an n^3-point rule            */
/* kind 0: Taylor-Green (p[0]=Mach, p[1]=gamma)                             */
/* kind 1: density wave rho = p0 + p1 sin(x+y+z - (ux+uy+uz) t), uniform    */
/*         velocity (p2,p3,p4) and pressure p5, time p6, gamma p7           */
/* kind 2: isentropic vortex of strength p0, core radius p1, centre (p2,p3) */
/*         advected by (p4,p5) for time p6, gamma p7; x-y periodic box      */
typedef struct { int kind; const double *p; double s[5], v; } ic_ctx;
static void ic_point(int kind, const double *p, const double x[3], double U[5]) {
  double r, u, v, w, pr;
  if (kind == 0) {
    double M = p[0], g = p[1];
    u = sin(x[0]) * cos(x[1]) * cos(x[2]);
    v = -cos(x[0]) * sin(x[1]) * cos(x[2]);
    w = 0;
    pr = 1.0 / (g * M * M) + (cos(2 * x[2]) + 2.0) * (cos(2 * x[0]) + cos(2 * x[1])) / 16.0;
    r = g * M * M * pr;
    U[0] = r; U[1] = r * u; U[2] = r * v; U[3] = r * w;
    U[4] = pr / (g - 1.0) + 0.5 * r * (u * u + v * v + w * w);
  } else if (kind == 1) {
    double g = p[7];
    u = p[2]; v = p[3]; w = p[4]; pr = p[5];
    r = p[0] + p[1] * sin(x[0] + x[1] + x[2] - (u + v + w) * p[6]);
    U[0] = r; U[1] = r * u; U[2] = r * v; U[3] = r * w;
    U[4] = pr / (g - 1.0) + 0.5 * r * (u * u + v * v + w * w);
  } else {
    double beta = p[0], sig = p[1], g = p[7];
    double xc = p[2] + p[4] * p[6], yc = p[3] + p[5] * p[6];
    double dx = (x[0] - xc) / sig, dy = (x[1] - yc) / sig, r2 = dx * dx + dy * dy;
    double e = exp(0.5 * (1.0 - r2));
    u = p[4] - beta / (2.0 * M_PI) * e * dy;
    v = p[5] + beta / (2.0 * M_PI) * e * dx;
    w = 0;
    double T = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * M_PI * M_PI) * e * e;
    r = pow(T, 1.0 / (g - 1.0));
    pr = r * T;
    U[0] = r; U[1] = r * u; U[2] = r * v; U[3] = r * w;
    U[4] = pr / (g - 1.0) + 0.5 * r * (u * u + v * v + w * w);
  }
}
static void f_ic(void *ctx, const double x[3], double w) {
  ic_ctx *q = (ic_ctx *)ctx;
  double U[5];
  ic_point(q->kind, q->p, x, U);
  for (int v = 0; v < 5; v++) q->s[v] += w * U[v];
  q->v += w;
}
void orc_cell_average(const orc_case *c, int kind, const double *p, int nq1d, double *U) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->N; i++) {
    ic_ctx q;
    memset(&q, 0, sizeof q);
    q.kind = kind;
    q.p = p;
    cell_quad(c, i, nq1d, f_ic, &q);
    for (int v = 0; v < 5; v++) U[v * c->N + i] = q.s[v] / q.v;
  }
}

/* Troubled-cell indicator features (32 per cell), from the cell average and  */
/* the optimal central polynomial p_opt (Eq. 4) of cell i:                    */
/*  0..17  (rho_m - rho_i)/rho_i over the central stencil, in stencil order   */
/*  18..23 (p_m - p_i)/p_i over its first 6 members                          */
/*  24..28 SI_v/(SI_v + q_v^2), SI of p_opt per variable (Eq. 6 reading),      */
/*         q = 0.1 (rho, rho a, rho a, rho a, rho a^2)                         */
/*  29 |u|/a, 30 h |div u|/a, 31 h |curl u|/a, h = |V_i|^(1/3), grad u from     */
/*         p_opt at the centroid                                              */
int orc_features(orc_case *c, const double *U, double *Fout /* [N][32] */) {
  if (ensure_all(c)) return -1;
  int64_t N = c->N;
  if (c->Mc < 18) { set_err("features need a 18-cell central stencil (P2)"); return -1; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    double *F = &Fout[i * 32];
    double Ui[5], aopt[5][ORC_MAXK], val[5], g[5][3];
    for (int v = 0; v < 5; v++) Ui[v] = U[v * N + i];
    const double *Pc = &c->Pc[i * c->K * c->Mc];
    for (int v = 0; v < 5; v++)
      for (int k = 0; k < c->K; k++) {
        double s = 0;
        for (int r = 0; r < c->Mc; r++) s += Pc[k * c->Mc + r] * (U[v * N + c->sc[i * c->Mc + r]] - Ui[v]);
        aopt[v][k] = s;
      }
    double r = Ui[0], u[3] = {Ui[1] / r, Ui[2] / r, Ui[3] / r};
    double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double p = (c->gam - 1.0) * (Ui[4] - 0.5 * r * q2), a = sqrt(c->gam * p / r);
    for (int m = 0; m < 18; m++) {
      int64_t j = c->sc[i * c->Mc + m];
      F[m] = (U[j] - r) / r;
    }
    for (int m = 0; m < 6; m++) {
      int64_t j = c->sc[i * c->Mc + m];
      double rj = U[j], mj2 = U[N + j] * U[N + j] + U[2 * N + j] * U[2 * N + j] + U[3 * N + j] * U[3 * N + j];
      double pj = (c->gam - 1.0) * (U[4 * N + j] - 0.5 * mj2 / rj);
      F[18 + m] = (pj - p) / p;
    }
    double sc[5] = {r, r * a, r * a, r * a, r * a * a};
    for (int v = 0; v < 5; v++) {
      double SI = smoothness(c, i, aopt[v], c->order), q = 0.1 * sc[v];
      F[24 + v] = SI / (SI + q * q);
    }
    eval_poly(c, i, Ui, aopt, &c->cen[3 * i], val, g);
    double gu[3][3];
    for (int A = 0; A < 3; A++)
      for (int j = 0; j < 3; j++) gu[A][j] = (g[1 + A][j] - u[A] * g[0][j]) / r;
    double wx = gu[2][1] - gu[1][2], wy = gu[0][2] - gu[2][0], wz = gu[1][0] - gu[0][1];
    double dv = gu[0][0] + gu[1][1] + gu[2][2];
    F[29] = sqrt(q2) / a;
    F[30] = c->hh[i] * fabs(dv) / a;
    F[31] = c->hh[i] * sqrt(wx * wx + wy * wy + wz * wz) / a;
  }
  return 0;
}

/* diagnostics: [KE, eps_s, eps_d] with cell-centroid gradients of the      */
/* reconstruction: KE = sum V rho|u|^2/2 / sum V,                           */
/* eps_s = sum V |curl u|^2 /(Re sum V), eps_d = 4/3 sum V (div u)^2/(Re sum V) */
int orc_diagnostics(orc_case *c, const double *U, double *out) {
  if (ensure_all(c)) return -1;
  int64_t N = c->N;
  double *coef = (double *)malloc(sizeof(double) * N * 5 * c->K);
  if (orc_reconstruct(c, U, coef, NULL)) { free(coef); return -1; }
  double ke = 0, es = 0, ed = 0, vt = 0;
  for (int64_t i = 0; i < N; i++) {
    double cc[5][ORC_MAXK], Ui[5], val[5], g[5][3];
    for (int v = 0; v < 5; v++) {
      Ui[v] = U[v * N + i];
      for (int k = 0; k < c->K; k++) cc[v][k] = coef[(i * 5 + v) * c->K + k];
    }
    eval_poly(c, i, Ui, cc, &c->cen[3 * i], val, g);
    double r = Ui[0], u[3] = {Ui[1] / r, Ui[2] / r, Ui[3] / r}, gu[3][3];
    for (int a = 0; a < 3; a++)
      for (int j = 0; j < 3; j++) gu[a][j] = (g[1 + a][j] - u[a] * g[0][j]) / r;
    double wx = gu[2][1] - gu[1][2], wy = gu[0][2] - gu[2][0], wz = gu[1][0] - gu[0][1];
    double dv = gu[0][0] + gu[1][1] + gu[2][2];
    double V = c->vol[i];
    ke += V * 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    es += V * (wx * wx + wy * wy + wz * wz);
    ed += V * dv * dv;
    vt += V;
  }
  double mu = c->inviscid ? 1.0 : 1.0 / c->Re;
  out[0] = ke / vt;
  out[1] = mu * es / vt;
  out[2] = 4.0 / 3.0 * mu * ed / vt;
  free(coef);
  return 0;
}
