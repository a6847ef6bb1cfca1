/*
 * FP64 CPU oracle: the pressure (Schur) operator of the IMEX-DG
 * compressible-Euler scheme, its Helmholtz / internal-energy Jacobi
 * preconditioners and the Krylov solves around it.
 *
 * Source: G. Orlando, T. Benacchio, L. Bonaventura, "Improving the
 * scalability of a high-order atmospheric dynamics solver based on the
 * deal.II library", arXiv:2505.00384 -- Sec. 2 (Eqs. for the IMEX stage,
 * the block system A U + B P = F, C U + D P = G, Eq. for A^(l), the Schur
 * form D P + C A^-1 (F - B P) = G), Sec. 3.1 (GMRES + Jacobi, Helmholtz
 * preconditioner entries) and Sec. 3.3 (fast block-diagonal inverse
 * S^-T J^-1 S^-1 with r+1 Gauss points; consistent integration with 2r+1
 * Gauss points).
 *
 * TEST INFRASTRUCTURE.  This file is the independent checker of the CUDA
 * library.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, table or constant
 * generator with the CUDA path.
 *
 * Everything here is the plain definition, written for a reader to check
 * against the paper by eye:
 *   - every field is evaluated at every quadrature point by summing over
 *     all (r+1)^3 nodal basis functions (no sum factorisation);
 *   - the geometry is the isoparametric map x(xi) = sum_nodes X_node psi(xi),
 *     differentiated directly; face normals are cross products of tangents;
 *   - cell inverses of the density-weighted mass are dense LU solves of the
 *     matrix assembled with r+1 Gauss points (algebraically S^-T J^-1 S^-1);
 *   - FGMRES is Saad's flexible GMRES, CG the textbook preconditioned CG.
 *
 * Readings of points the paper leaves open (numerical fluxes, boundary
 * conditions, terrain mapping) are stated where they are used.
 *
 * Layout: DoF index = cell * (r+1)^3 + a + (r+1) b + (r+1)^2 c (x fastest),
 * cell = cx + nx (cy + ny cz); vector fields are three consecutive N-blocks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 8   /* degree r <= 7 */
#define ORC_MAXQ 16  /* quadrature points per direction */

typedef struct {
  int nx, ny, nz;
  int r;          /* polynomial degree                                         */
  int q;          /* Gauss points per direction of the consistent rule (2r+1)  */
  int terrain;    /* 0 flat, 1 bell h_c/(1+d^2/a_c^2), 2 bell with power -3/2  */
  int bc_lateral; /* 0 slip wall, 1 far field on the four lateral faces        */
  int pad;
  double Lx, Ly, Lz;
  double hc, ac, xc, yc;
} orc_mesh;

/* ------------------------------------------------------------------ */
/* 1D rules (textbook: Newton iteration on Legendre polynomials)       */
/* ------------------------------------------------------------------ */

/* P_k(x) and P_k'(x) by the three-term recurrence; |x| < 1 for P'. */
static void legendre(int k, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x;
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int j = 1; j < k; ++j) {
    double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
    p0 = p1; p1 = p2;
  }
  *P = p1;
  *dP = k * (x * p1 - p0) / (x * x - 1.0);
}

/* Gauss-Legendre points and weights on [0,1], ascending. */
int orc_gauss(int q, double *x, double *w) {
  if (q < 1 || q > ORC_MAXQ) return -1;
  for (int i = 0; i < q; ++i) {
    double t = -cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre(q, t, &P, &dP);
    x[i] = 0.5 * (1.0 + t);
    w[i] = 1.0 / ((1.0 - t * t) * dP * dP);
  }
  return 0;
}

/* Gauss-Lobatto-Legendre points and weights on [0,1] (n >= 2 points):
 * the end points and the roots of P'_{n-1}. */
int orc_gll(int n, double *x, double *w) {
  if (n < 2 || n > ORC_MAXN) return -1;
  int k = n - 1;
  double t[ORC_MAXN];
  t[0] = -1.0; t[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double s = -cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(k, s, &P, &dP);
      double d2P = (2.0 * s * dP - k * (k + 1.0) * P) / (1.0 - s * s);
      double ds = dP / d2P;
      s -= ds;
      if (fabs(ds) < 1e-16) break;
    }
    t[i] = s;
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    if (i == 0 || i == k) P = (i == 0 && (k % 2)) ? -1.0 : 1.0;
    else legendre(k, t[i], &P, &dP);
    x[i] = 0.5 * (1.0 + t[i]);
    w[i] = 1.0 / (k * (k + 1.0) * P * P);
  }
  return 0;
}

/* Lagrange cardinal polynomials on the nodes xn and their derivatives. */
void orc_lagrange(int n, const double *xn, double x, double *l, double *dl) {
  for (int a = 0; a < n; ++a) {
    double prod = 1.0;
    for (int b = 0; b < n; ++b)
      if (b != a) prod *= (x - xn[b]) / (xn[a] - xn[b]);
    l[a] = prod;
    if (dl) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) {
        if (c == a) continue;
        double t = 1.0 / (xn[a] - xn[c]);
        for (int b = 0; b < n; ++b)
          if (b != a && b != c) t *= (x - xn[b]) / (xn[a] - xn[b]);
        s += t;
      }
      dl[a] = s;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Mesh and geometry                                                    */
/* ------------------------------------------------------------------ */

/* Bottom height of the terrain-following mesh. */
double orc_terrain_height(const orc_mesh *m, double x, double y) {
  if (m->terrain == 0) return 0.0;
  double s = 1.0 + ((x - m->xc) * (x - m->xc) + (y - m->yc) * (y - m->yc)) / (m->ac * m->ac);
  if (m->terrain == 1) return m->hc / s;
  return m->hc * pow(s, -1.5);
}

typedef struct {
  int n, q, n3, q3, q2;
  double gll[ORC_MAXN], gllw[ORC_MAXN];
  double gq[ORC_MAXQ], gw[ORC_MAXQ];   /* consistent rule, q points   */
  double ga[ORC_MAXN], gaw[ORC_MAXN];  /* fast-inverse rule, r+1 pts  */
  double *psi, *dpsi;                  /* volume points: [q3][n3], [q3][3][n3] */
  double *wq;                          /* volume weights [q3]          */
  double *psia, *dpsia, *wa;           /* fast points: [n3][n3], [n3][3][n3], [n3] */
  double *fpsi[6], *fdpsi[6], *fw[6];  /* faces (k,s) -> 2k+s: [q2][n3], [q2][3][n3], [q2] */
} tabs;

static void basis3(const tabs *T, const double xi[3], double *psi, double *dpsi) {
  int n = T->n, n3 = T->n3;
  double l[3][ORC_MAXN], dl[3][ORC_MAXN];
  for (int d = 0; d < 3; ++d) orc_lagrange(n, T->gll, xi[d], l[d], dl[d]);
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        int i = a + n * (b + n * c);
        psi[i] = l[0][a] * l[1][b] * l[2][c];
        if (dpsi) {
          dpsi[0 * n3 + i] = dl[0][a] * l[1][b] * l[2][c];
          dpsi[1 * n3 + i] = l[0][a] * dl[1][b] * l[2][c];
          dpsi[2 * n3 + i] = l[0][a] * l[1][b] * dl[2][c];
        }
      }
}

static int tabs_init(tabs *T, const orc_mesh *m) {
  memset(T, 0, sizeof(*T));
  int n = m->r + 1, q = m->q;
  if (m->r < 1 || n > ORC_MAXN || q < 1 || q > ORC_MAXQ) return -1;
  T->n = n; T->q = q; T->n3 = n * n * n; T->q3 = q * q * q; T->q2 = q * q;
  orc_gll(n, T->gll, T->gllw);
  orc_gauss(q, T->gq, T->gw);
  orc_gauss(n, T->ga, T->gaw);
  int n3 = T->n3, q3 = T->q3, q2 = T->q2;
  T->psi = malloc(sizeof(double) * q3 * n3);
  T->dpsi = malloc(sizeof(double) * q3 * 3 * n3);
  T->wq = malloc(sizeof(double) * q3);
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i) {
        int p = i + q * (j + q * k);
        double xi[3] = {T->gq[i], T->gq[j], T->gq[k]};
        basis3(T, xi, T->psi + (size_t)p * n3, T->dpsi + (size_t)p * 3 * n3);
        T->wq[p] = T->gw[i] * T->gw[j] * T->gw[k];
      }
  T->psia = malloc(sizeof(double) * n3 * n3);
  T->dpsia = malloc(sizeof(double) * n3 * 3 * n3);
  T->wa = malloc(sizeof(double) * n3);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int p = i + n * (j + n * k);
        double xi[3] = {T->ga[i], T->ga[j], T->ga[k]};
        basis3(T, xi, T->psia + (size_t)p * n3, T->dpsia + (size_t)p * 3 * n3);
        T->wa[p] = T->gaw[i] * T->gaw[j] * T->gaw[k];
      }
  for (int f = 0; f < 6; ++f) {
    int k = f / 2, s = f % 2;
    int t1 = (k == 0) ? 1 : 0, t2 = (k == 2) ? 1 : 2;
    T->fpsi[f] = malloc(sizeof(double) * q2 * n3);
    T->fdpsi[f] = malloc(sizeof(double) * q2 * 3 * n3);
    T->fw[f] = malloc(sizeof(double) * q2);
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i) {
        int p = i + q * j;
        double xi[3];
        xi[k] = (double)s; xi[t1] = T->gq[i]; xi[t2] = T->gq[j];
        basis3(T, xi, T->fpsi[f] + (size_t)p * n3, T->fdpsi[f] + (size_t)p * 3 * n3);
        T->fw[f][p] = T->gw[i] * T->gw[j];
      }
  }
  return 0;
}

static void tabs_free(tabs *T) {
  free(T->psi); free(T->dpsi); free(T->wq);
  free(T->psia); free(T->dpsia); free(T->wa);
  for (int f = 0; f < 6; ++f) { free(T->fpsi[f]); free(T->fdpsi[f]); free(T->fw[f]); }
}

long orc_num_cells(const orc_mesh *m) { return (long)m->nx * m->ny * m->nz; }

/* Physical coordinates of the (r+1)^3 GLL nodes of a cell.  Reading of the
 * terrain-following mapping: Gal-Chen, z = zeta + h(x,y) (1 - zeta/Lz) with
 * zeta uniform on [0, Lz]; x, y affine. */
static void cell_nodes(const orc_mesh *m, const tabs *T, long cell, double *Xn /* [3][n3] */) {
  int n = T->n, n3 = T->n3;
  long cx = cell % m->nx, cy = (cell / m->nx) % m->ny, cz = cell / ((long)m->nx * m->ny);
  double dx = m->Lx / m->nx, dy = m->Ly / m->ny, dz = m->Lz / m->nz;
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        int i = a + n * (b + n * c);
        double x = (cx + T->gll[a]) * dx, y = (cy + T->gll[b]) * dy;
        double zeta = (cz + T->gll[c]) * dz;
        Xn[i] = x;
        Xn[n3 + i] = y;
        Xn[2 * n3 + i] = zeta + orc_terrain_height(m, x, y) * (1.0 - zeta / m->Lz);
      }
}

/* Jacobian J_ij = dX_i/dxi_j of the isoparametric map at a point whose basis
 * gradients are dpsi [3][n3]. */
static void jacobian(int n3, const double *Xn, const double *dpsi, double J[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int a = 0; a < n3; ++a) s += Xn[i * n3 + a] * dpsi[j * n3 + a];
      J[i][j] = s;
    }
}

static double det3(double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
       - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
       + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* Ji[j][d] = (J^-1)_{jd} = d xi_j / d x_d. */
static void inv3(double J[3][3], double det, double Ji[3][3]) {
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

/* Per-cell geometry at the quadrature points. */
typedef struct {
  double *wdet;   /* [q3]  w_q det J                                   */
  double *Ji;     /* [q3][9] (J^-1)_{jd}                               */
  double *nA[6];  /* [q2][3] outward normal * area element * w          */
  double *wdeta;  /* [n3]  fast rule: w_q det J                        */
  double Xn[3 * ORC_MAXN * ORC_MAXN * ORC_MAXN];
} cgeo;

static void cgeo_alloc(cgeo *G, const tabs *T) {
  G->wdet = malloc(sizeof(double) * T->q3);
  G->Ji = malloc(sizeof(double) * T->q3 * 9);
  for (int f = 0; f < 6; ++f) G->nA[f] = malloc(sizeof(double) * T->q2 * 3);
  G->wdeta = malloc(sizeof(double) * T->n3);
}
static void cgeo_free(cgeo *G) {
  free(G->wdet); free(G->Ji);
  for (int f = 0; f < 6; ++f) free(G->nA[f]);
  free(G->wdeta);
}

static void cell_geometry(const orc_mesh *m, const tabs *T, long cell, cgeo *G) {
  int n3 = T->n3;
  cell_nodes(m, T, cell, G->Xn);
  for (int p = 0; p < T->q3; ++p) {
    double J[3][3], Ji[3][3];
    jacobian(n3, G->Xn, T->dpsi + (size_t)p * 3 * n3, J);
    double det = det3(J);
    inv3(J, det, Ji);
    G->wdet[p] = T->wq[p] * det;
    for (int j = 0; j < 3; ++j)
      for (int d = 0; d < 3; ++d) G->Ji[p * 9 + 3 * j + d] = Ji[j][d];
  }
  for (int p = 0; p < n3; ++p) {
    double J[3][3];
    jacobian(n3, G->Xn, T->dpsia + (size_t)p * 3 * n3, J);
    G->wdeta[p] = T->wa[p] * det3(J);
  }
  for (int f = 0; f < 6; ++f) {
    int k = f / 2, s = f % 2;
    int t1 = (k == 0) ? 1 : 0, t2 = (k == 2) ? 1 : 2;
    for (int p = 0; p < T->q2; ++p) {
      double J[3][3];
      jacobian(n3, G->Xn, T->fdpsi[f] + (size_t)p * 3 * n3, J);
      double a[3] = {J[0][t1], J[1][t1], J[2][t1]};
      double b[3] = {J[0][t2], J[1][t2], J[2][t2]};
      double N[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      /* outward: along +xi_k on side 1, -xi_k on side 0 */
      double dk = N[0] * J[0][k] + N[1] * J[1][k] + N[2] * J[2][k];
      double sg = ((dk > 0) == (s == 1)) ? 1.0 : -1.0;
      for (int d = 0; d < 3; ++d) G->nA[f][3 * p + d] = sg * N[d] * T->fw[f][p];
    }
  }
}

/* Neighbour across face (k, s); -1 on the domain boundary. */
static long neighbour(const orc_mesh *m, long cell, int k, int s) {
  long c[3] = {cell % m->nx, (cell / m->nx) % m->ny, cell / ((long)m->nx * m->ny)};
  long nn[3] = {m->nx, m->ny, m->nz};
  c[k] += s ? 1 : -1;
  if (c[k] < 0 || c[k] >= nn[k]) return -1;
  return c[0] + m->nx * (c[1] + m->ny * c[2]);
}

/* Boundary kind of face direction k: 0 slip wall, 1 far field. */
static int boundary_kind(const orc_mesh *m, int k) { return (k == 2) ? 0 : m->bc_lateral; }

static double dotn(int n3, const double *f, const double *psi) {
  double s = 0.0;
  for (int i = 0; i < n3; ++i) s += f[i] * psi[i];
  return s;
}

/* ------------------------------------------------------------------ */
/* Cell operators                                                       */
/* ------------------------------------------------------------------ */

/* (B P) on one cell, 3 components [3][n3]:
 *   alpha [ - int_K p div(phi) + int_dK p_hat phi.n ]
 * Reading of the flux: p_hat = {p} = (p- + p+)/2 on interior faces,
 * p_hat = p- on every boundary face (p+ = p-). */
static void cell_B(const orc_mesh *m, const tabs *T, const cgeo *G, long cell, double alpha,
                   const double *p, double *out) {
  int n3 = T->n3;
  const double *pc = p + cell * n3;
  memset(out, 0, sizeof(double) * 3 * n3);
  for (int qp = 0; qp < T->q3; ++qp) {
    const double *ps = T->psi + (size_t)qp * n3, *dps = T->dpsi + (size_t)qp * 3 * n3;
    const double *Ji = G->Ji + qp * 9;
    double pq = dotn(n3, pc, ps) * G->wdet[qp];
    for (int i = 0; i < n3; ++i) {
      double g0 = dps[i], g1 = dps[n3 + i], g2 = dps[2 * n3 + i];
      for (int d = 0; d < 3; ++d) {
        double gd = g0 * Ji[d] + g1 * Ji[3 + d] + g2 * Ji[6 + d];
        out[d * n3 + i] -= pq * gd;
      }
    }
  }
  for (int f = 0; f < 6; ++f) {
    int k = f / 2, s = f % 2;
    long nb = neighbour(m, cell, k, s);
    const double *fps = T->fpsi[f], *fpsn = T->fpsi[2 * k + (1 - s)];
    for (int qp = 0; qp < T->q2; ++qp) {
      double pm = dotn(n3, pc, fps + (size_t)qp * n3);
      double ph = pm;
      if (nb >= 0) ph = 0.5 * (pm + dotn(n3, p + nb * n3, fpsn + (size_t)qp * n3));
      const double *nA = G->nA[f] + 3 * qp;
      for (int i = 0; i < n3; ++i) {
        double v = ph * fps[(size_t)qp * n3 + i];
        for (int d = 0; d < 3; ++d) out[d * n3 + i] += v * nA[d];
      }
    }
  }
  for (int i = 0; i < 3 * n3; ++i) out[i] *= alpha;
}

/* Dense density-weighted mass of one cell with the r+1 point Gauss rule,
 * A_ij = sum_q rho(x_q) psi_i(x_q) psi_j(x_q) w_q det J(x_q). */
static void cell_A_matrix(const tabs *T, const cgeo *G, long cell, const double *rho, double *A) {
  int n3 = T->n3;
  const double *rc = rho + cell * n3;
  memset(A, 0, sizeof(double) * n3 * n3);
  for (int qp = 0; qp < n3; ++qp) {
    const double *ps = T->psia + (size_t)qp * n3;
    double c = dotn(n3, rc, ps) * G->wdeta[qp];
    for (int i = 0; i < n3; ++i)
      for (int j = 0; j < n3; ++j) A[i * n3 + j] += c * ps[i] * ps[j];
  }
}

/* LU with partial pivoting, in place; solves A x = b for nrhs right-hand
 * sides stored as rows of B ([nrhs][n]). */
static int lu_solve(int n, double *A, int nrhs, double *B) {
  int piv[ORC_MAXN * ORC_MAXN * ORC_MAXN];
  for (int k = 0; k < n; ++k) {
    int pk = k;
    double mx = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > mx) { mx = fabs(A[i * n + k]); pk = i; }
    if (mx == 0.0) return -1;
    piv[k] = pk;
    if (pk != k)
      for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[pk * n + j]; A[pk * n + j] = t; }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  for (int r = 0; r < nrhs; ++r) {
    double *b = B + (size_t)r * n;
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) b[i] -= A[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) b[i] -= A[i * n + j] * b[j];
      b[i] /= A[i * n + i];
    }
  }
  return 0;
}

/* (C V) on one cell: alpha [ - int_K kappa V.grad(psi) + int_dK (kappa V)^.n psi ],
 * kappa = gamma p_k / (gamma - 1)  (h rho with h = gamma p / ((gamma-1) rho)).
 * Reading of the flux: (kappa V)^ = average of both traces on interior faces;
 * zero normal flux on slip walls ((V.n)+ = -(V.n)-); far-field faces are
 * transmissive in the pressure operator ((kappa V)+ = (kappa V)-). */
static void cell_C(const orc_mesh *m, const tabs *T, const cgeo *G, long cell, double alpha,
                   double gamma, const double *pk, const double *V, long N, double *out) {
  int n3 = T->n3;
  double kf = gamma / (gamma - 1.0);
  const double *kc = pk + cell * n3;
  const double *V0 = V + cell * n3, *V1 = V + N + cell * n3, *V2 = V + 2 * N + cell * n3;
  memset(out, 0, sizeof(double) * n3);
  for (int qp = 0; qp < T->q3; ++qp) {
    const double *ps = T->psi + (size_t)qp * n3, *dps = T->dpsi + (size_t)qp * 3 * n3;
    const double *Ji = G->Ji + qp * 9;
    double kq = kf * dotn(n3, kc, ps) * G->wdet[qp];
    double v[3] = {dotn(n3, V0, ps), dotn(n3, V1, ps), dotn(n3, V2, ps)};
    for (int i = 0; i < n3; ++i) {
      double g0 = dps[i], g1 = dps[n3 + i], g2 = dps[2 * n3 + i];
      double s = 0.0;
      for (int d = 0; d < 3; ++d) s += v[d] * (g0 * Ji[d] + g1 * Ji[3 + d] + g2 * Ji[6 + d]);
      out[i] -= kq * s;
    }
  }
  for (int f = 0; f < 6; ++f) {
    int k = f / 2, s = f % 2;
    long nb = neighbour(m, cell, k, s);
    int bk = boundary_kind(m, k);
    if (nb < 0 && bk == 0) continue; /* slip wall: no normal flux */
    const double *fps = T->fpsi[f], *fpsn = T->fpsi[2 * k + (1 - s)];
    for (int qp = 0; qp < T->q2; ++qp) {
      const double *ps = fps + (size_t)qp * n3;
      const double *nA = G->nA[f] + 3 * qp;
      double km = kf * dotn(n3, kc, ps);
      double vm = dotn(n3, V0, ps) * nA[0] + dotn(n3, V1, ps) * nA[1] + dotn(n3, V2, ps) * nA[2];
      double flux = km * vm;
      if (nb >= 0) {
        const double *pn = fpsn + (size_t)qp * n3;
        double kp = kf * dotn(n3, pk + nb * n3, pn);
        double vp = dotn(n3, V + nb * n3, pn) * nA[0] + dotn(n3, V + N + nb * n3, pn) * nA[1] +
                    dotn(n3, V + 2 * N + nb * n3, pn) * nA[2];
        flux = 0.5 * (km * vm + kp * vp);
      }
      for (int i = 0; i < n3; ++i) out[i] += flux * ps[i];
    }
  }
  for (int i = 0; i < n3; ++i) out[i] *= alpha;
}

/* Consistent mass on one cell, scaled: out_i = scale * int_K f psi_i. */
static void cell_M(const tabs *T, const cgeo *G, long cell, double scale, const double *f, double *out) {
  int n3 = T->n3;
  const double *fc = f + cell * n3;
  memset(out, 0, sizeof(double) * n3);
  for (int qp = 0; qp < T->q3; ++qp) {
    const double *ps = T->psi + (size_t)qp * n3;
    double fq = dotn(n3, fc, ps) * G->wdet[qp] * scale;
    for (int i = 0; i < n3; ++i) out[i] += fq * ps[i];
  }
}

/* ------------------------------------------------------------------ */
/* Global drivers (OpenMP over cells; each cell writes only its DoFs)   */
/* ------------------------------------------------------------------ */

typedef struct { tabs T; long nc, N; int ok; } orc_setup;

static int setup(orc_setup *S, const orc_mesh *m) {
  S->ok = tabs_init(&S->T, m) == 0;
  S->nc = orc_num_cells(m);
  S->N = S->nc * S->T.n3;
  return S->ok ? 0 : -1;
}

int orc_node_coords(const orc_mesh *m, double *X) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < S.nc; ++c) {
    double Xn[3 * ORC_MAXN * ORC_MAXN * ORC_MAXN];
    cell_nodes(m, &S.T, c, Xn);
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < n3; ++i) X[d * S.N + c * n3 + i] = Xn[d * n3 + i];
  }
  tabs_free(&S.T);
  return 0;
}

int orc_apply_B(const orc_mesh *m, double alpha, const double *p, double *out) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
    double *loc = malloc(sizeof(double) * 3 * n3);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      cell_geometry(m, &S.T, c, &G);
      cell_B(m, &S.T, &G, c, alpha, p, loc);
      for (int d = 0; d < 3; ++d) memcpy(out + d * S.N + c * n3, loc + d * n3, sizeof(double) * n3);
    }
    free(loc); cgeo_free(&G);
  }
  tabs_free(&S.T);
  return 0;
}

/* inverse = 0: out = A_rho in ; inverse = 1: out = A_rho^-1 in (per component). */
static int apply_A_impl(const orc_mesh *m, const double *rho, const double *in, double *out, int inverse) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
  int err = 0;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
    double *A = malloc(sizeof(double) * n3 * n3);
    double *B = malloc(sizeof(double) * 3 * n3);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      cell_geometry(m, &S.T, c, &G);
      cell_A_matrix(&S.T, &G, c, rho, A);
      for (int d = 0; d < 3; ++d) memcpy(B + d * n3, in + d * S.N + c * n3, sizeof(double) * n3);
      if (inverse) {
        if (lu_solve(n3, A, 3, B)) err = -2;
      } else {
        double t[3 * ORC_MAXN * ORC_MAXN * ORC_MAXN];
        for (int d = 0; d < 3; ++d)
          for (int i = 0; i < n3; ++i) {
            double s = 0.0;
            for (int j = 0; j < n3; ++j) s += A[i * n3 + j] * B[d * n3 + j];
            t[d * n3 + i] = s;
          }
        memcpy(B, t, sizeof(double) * 3 * n3);
      }
      for (int d = 0; d < 3; ++d) memcpy(out + d * S.N + c * n3, B + d * n3, sizeof(double) * n3);
    }
    free(A); free(B); cgeo_free(&G);
  }
  tabs_free(&S.T);
  return err;
}

int orc_apply_A(const orc_mesh *m, const double *rho, const double *in, double *out) {
  return apply_A_impl(m, rho, in, out, 0);
}
int orc_apply_Ainv(const orc_mesh *m, const double *rho, const double *in, double *out) {
  return apply_A_impl(m, rho, in, out, 1);
}

int orc_apply_C(const orc_mesh *m, double alpha, double gamma, const double *pk, const double *V, double *out) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      cell_geometry(m, &S.T, c, &G);
      cell_C(m, &S.T, &G, c, alpha, gamma, pk, V, S.N, out + c * n3);
    }
    cgeo_free(&G);
  }
  tabs_free(&S.T);
  return 0;
}

/* out = scale * M f with the consistent (q-point) rule; D = M / (gamma - 1). */
int orc_apply_M(const orc_mesh *m, double scale, const double *f, double *out) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      cell_geometry(m, &S.T, c, &G);
      cell_M(&S.T, &G, c, scale, f, out + c * n3);
    }
    cgeo_free(&G);
  }
  tabs_free(&S.T);
  return 0;
}

/* y = S P = D P - C A^-1 B P on the cells flagged in mask (all cells when
 * mask is NULL); y is left untouched elsewhere.  Needs V = A^-1 B P on the
 * flagged cells and on their face neighbours. */
int orc_apply_S_masked(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
                       const double *p, const unsigned char *mask, double *y) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
  long nc = S.nc, N = S.N;
  unsigned char *need = calloc(nc, 1);
  for (long c = 0; c < nc; ++c) {
    if (mask && !mask[c]) continue;
    need[c] = 1;
    for (int f = 0; f < 6; ++f) {
      long nb = neighbour(m, c, f / 2, f % 2);
      if (nb >= 0) need[nb] = 1;
    }
  }
  double *V = calloc((size_t)3 * N, sizeof(double));
  int err = 0;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
    double *A = malloc(sizeof(double) * n3 * n3);
    double *B = malloc(sizeof(double) * 3 * n3);
    double *loc = malloc(sizeof(double) * 2 * n3);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < nc; ++c) {
      if (!need[c]) continue;
      cell_geometry(m, &S.T, c, &G);
      cell_B(m, &S.T, &G, c, alpha, p, B);
      cell_A_matrix(&S.T, &G, c, rho, A);
      if (lu_solve(n3, A, 3, B)) err = -2;
      for (int d = 0; d < 3; ++d) memcpy(V + d * N + c * n3, B + d * n3, sizeof(double) * n3);
    }
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < nc; ++c) {
      if (mask && !mask[c]) continue;
      cell_geometry(m, &S.T, c, &G);
      cell_M(&S.T, &G, c, 1.0 / (gamma - 1.0), p, loc);
      cell_C(m, &S.T, &G, c, alpha, gamma, pk, V, N, loc + n3);
      for (int i = 0; i < n3; ++i) y[c * n3 + i] = loc[i] - loc[n3 + i];
    }
    free(A); free(B); free(loc); cgeo_free(&G);
  }
  free(V); free(need);
  tabs_free(&S.T);
  return err;
}

int orc_apply_S(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
                const double *p, double *y) {
  return orc_apply_S_masked(m, alpha, gamma, rho, pk, p, NULL, y);
}

/* Jacobi diagonal (Sec. 3.1):
 *   kind 1 (Helmholtz):       d_i = int psi_i^2/(gamma-1) + alpha^2 int h |grad psi_i|^2,
 *                              h = e + p/rho = gamma p_k / ((gamma-1) rho), volume terms only;
 *   kind 2 (internal energy): d_i = int psi_i^2/(gamma-1)  (the diagonal of D).
 * Integrals with the consistent rule. */
int orc_precond_diag(const orc_mesh *m, int kind, double alpha, double gamma, const double *rho,
                     const double *pk, double *dg) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      cell_geometry(m, &S.T, c, &G);
      double *o = dg + c * n3;
      for (int i = 0; i < n3; ++i) o[i] = 0.0;
      for (int qp = 0; qp < S.T.q3; ++qp) {
        const double *ps = S.T.psi + (size_t)qp * n3, *dps = S.T.dpsi + (size_t)qp * 3 * n3;
        const double *Ji = G.Ji + qp * 9;
        double hq = 0.0;
        if (kind == 1)
          hq = gamma * dotn(n3, pk + c * n3, ps) / ((gamma - 1.0) * dotn(n3, rho + c * n3, ps));
        for (int i = 0; i < n3; ++i) {
          double v = ps[i] * ps[i] / (gamma - 1.0);
          if (kind == 1) {
            double g2 = 0.0;
            for (int d = 0; d < 3; ++d) {
              double gd = dps[i] * Ji[d] + dps[n3 + i] * Ji[3 + d] + dps[2 * n3 + i] * Ji[6 + d];
              g2 += gd * gd;
            }
            v += alpha * alpha * hq * g2;
          }
          o[i] += v * G.wdet[qp];
        }
      }
    }
    cgeo_free(&G);
  }
  tabs_free(&S.T);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Krylov solvers                                                       */
/* ------------------------------------------------------------------ */

static double vdot(long n, const double *a, const double *b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

typedef struct {
  const orc_mesh *m;
  double alpha, gamma;
  const double *rho, *pk;
} sctx;

static void S_apply(const sctx *c, const double *x, double *y) {
  orc_apply_S(c->m, c->alpha, c->gamma, c->rho, c->pk, x, y);
}

/* Flexible GMRES(restart), right preconditioned by the diagonal scaling
 * z = dinv .* v (dinv NULL: identity), classical Gram-Schmidt applied twice.
 * Convergence: true residual ||b - S x|| / ||b|| <= tol, checked at every
 * restart (the Arnoldi estimate ends a cycle early).  Returns 0 converged,
 * 1 not converged within maxit, <0 error. */
int orc_fgmres(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
               const double *dinv, const double *b, double *x, double tol, int restart, int maxit,
               int *its_out, double *relres_out) {
  sctx c = {m, alpha, gamma, rho, pk};
  long N = orc_num_cells(m) * (long)(m->r + 1) * (m->r + 1) * (m->r + 1);
  int mm = restart;
  double *Vb = malloc(sizeof(double) * N * (mm + 1));
  double *Zb = malloc(sizeof(double) * N * mm);
  double *w = malloc(sizeof(double) * N);
  double *H = calloc((size_t)(mm + 1) * mm, sizeof(double));
  double *cs = malloc(sizeof(double) * mm), *sn = malloc(sizeof(double) * mm);
  double *g = malloc(sizeof(double) * (mm + 1)), *yv = malloc(sizeof(double) * mm);
  double *h = malloc(sizeof(double) * (mm + 1));
  double bn = sqrt(vdot(N, b, b));
  int its = 0, status = 1;
  double rel = 0.0;
  if (bn == 0.0) {
    for (long i = 0; i < N; ++i) x[i] = 0.0;
    status = 0;
    goto done;
  }
  for (;;) {
    S_apply(&c, x, w);
    for (long i = 0; i < N; ++i) w[i] = b[i] - w[i];
    double beta = sqrt(vdot(N, w, w));
    rel = beta / bn;
    if (rel <= tol) { status = 0; break; }
    if (its >= maxit) { status = 1; break; }
    for (long i = 0; i < N; ++i) Vb[i] = w[i] / beta;
    for (int i = 0; i <= mm; ++i) g[i] = 0.0;
    g[0] = beta;
    int jj = 0;
    for (int j = 0; j < mm; ++j) {
      double *z = Zb + (size_t)j * N, *vj = Vb + (size_t)j * N;
      for (long i = 0; i < N; ++i) z[i] = dinv ? dinv[i] * vj[i] : vj[i];
      S_apply(&c, z, w);
      for (int i = 0; i <= j; ++i) H[i * mm + j] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i <= j; ++i) h[i] = vdot(N, Vb + (size_t)i * N, w);
        for (int i = 0; i <= j; ++i) {
          const double *vi = Vb + (size_t)i * N;
          for (long t = 0; t < N; ++t) w[t] -= h[i] * vi[t];
          H[i * mm + j] += h[i];
        }
      }
      double hn = sqrt(vdot(N, w, w));
      H[(j + 1) * mm + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * mm + j], bb = H[(i + 1) * mm + j];
        H[i * mm + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * mm + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[j * mm + j], bb = H[(j + 1) * mm + j];
      double rr = hypot(a, bb);
      cs[j] = a / rr; sn[j] = bb / rr;
      H[j * mm + j] = rr; H[(j + 1) * mm + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      jj = j + 1;
      if (hn == 0.0) break; /* happy breakdown */
      double *vn = Vb + (size_t)(j + 1) * N;
      for (long i = 0; i < N; ++i) vn[i] = w[i] / hn;
      if (fabs(g[j + 1]) / bn <= tol || its >= maxit) break;
    }
    for (int i = jj - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jj; ++k) s -= H[i * mm + k] * yv[k];
      yv[i] = s / H[i * mm + i];
    }
    for (int k = 0; k < jj; ++k) {
      const double *z = Zb + (size_t)k * N;
      for (long i = 0; i < N; ++i) x[i] += yv[k] * z[i];
    }
  }
done:
  if (its_out) *its_out = its;
  if (relres_out) *relres_out = rel;
  free(Vb); free(Zb); free(w); free(H); free(cs); free(sn); free(g); free(yv); free(h);
  return status;
}

/* Preconditioned conjugate gradients (for the symmetric positive definite
 * case); same stopping rule on the true recursive residual. */
int orc_cg(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
           const double *dinv, const double *b, double *x, double tol, int maxit, int *its_out,
           double *relres_out) {
  sctx c = {m, alpha, gamma, rho, pk};
  long N = orc_num_cells(m) * (long)(m->r + 1) * (m->r + 1) * (m->r + 1);
  double *r = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N);
  double *p = malloc(sizeof(double) * N), *q = malloc(sizeof(double) * N);
  double bn = sqrt(vdot(N, b, b));
  int its = 0, status = 1;
  double rel = 0.0;
  S_apply(&c, x, q);
  for (long i = 0; i < N; ++i) r[i] = b[i] - q[i];
  if (bn == 0.0) bn = 1.0;
  rel = sqrt(vdot(N, r, r)) / bn;
  if (rel <= tol) status = 0;
  for (long i = 0; i < N; ++i) { z[i] = dinv ? dinv[i] * r[i] : r[i]; p[i] = z[i]; }
  double rz = vdot(N, r, z);
  while (status != 0 && its < maxit) {
    S_apply(&c, p, q);
    double a = rz / vdot(N, p, q);
    for (long i = 0; i < N; ++i) { x[i] += a * p[i]; r[i] -= a * q[i]; }
    ++its;
    rel = sqrt(vdot(N, r, r)) / bn;
    if (rel <= tol) { status = 0; break; }
    for (long i = 0; i < N; ++i) z[i] = dinv ? dinv[i] * r[i] : r[i];
    double rz2 = vdot(N, r, z);
    double be = rz2 / rz;
    rz = rz2;
    for (long i = 0; i < N; ++i) p[i] = z[i] + be * p[i];
  }
  if (its_out) *its_out = its;
  if (relres_out) *relres_out = rel;
  free(r); free(z); free(p); free(q);
  return status;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
