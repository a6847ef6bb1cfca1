/*
 * Shared internals of the FP64 CPU oracle (TEST INFRASTRUCTURE): 1D rules,
 * tables of basis values at quadrature points, the isoparametric geometry
 * of the terrain-following cells, neighbour lookup and a dense LU solve.
 * Included by orc.c and orc_imex.c only.
 */
#ifndef ORC_CORE_H
#define ORC_CORE_H
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
  int bc_lateral; /* 0 slip wall, 1 far field, 2 periodic (lateral faces)      */
  int pad;
  double Lx, Ly, Lz;
  double hc, ac, xc, yc;
  /* 2:1 refinement box in base cells, [ref[0], ref[1]) x [ref[2], ref[3]) x
   * [ref[4], ref[5]); no refinement when the box is empty */
  int ref[6];
} orc_mesh;

/* exported 1D rules and helpers (defined in orc.c) */
int orc_gauss(int q, double *x, double *w);
int orc_gll(int n, double *x, double *w);
void orc_lagrange(int n, const double *xn, double x, double *l, double *dl);
double orc_terrain_height(const orc_mesh *m, double x, double y);
long orc_num_cells(const orc_mesh *m);


/* ------------------------------------------------------------------ */
/* 1D rules (textbook: Newton iteration on Legendre polynomials)       */
/* ------------------------------------------------------------------ */

/* P_k(x) and P_k'(x) by the three-term recurrence; |x| < 1 for P'. */
static inline void legendre(int k, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x;
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int j = 1; j < k; ++j) {
    double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
    p0 = p1; p1 = p2;
  }
  *P = p1;
  *dP = k * (x * p1 - p0) / (x * x - 1.0);
}



/* (orc_gauss and orc_gll, defined in orc.c, use legendre() above.) */

/* ------------------------------------------------------------------ */
/* Basis tables at the quadrature points, mesh and geometry            */
/* ------------------------------------------------------------------ */

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

static double dotn(int n3, const double *f, const double *psi) {
  double s = 0.0;
  for (int i = 0; i < n3; ++i) s += f[i] * psi[i];
  return s;
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



/* ------------------------------------------------------------------ */
/* Non-conforming meshes (Sec. 3: neighbouring cells of different        */
/* resolution horizontally and vertically)                              */
/* ------------------------------------------------------------------ */
/* The nx*ny*nz base mesh with the cells of the box ref[] split into
 * 2 x 2 x 2 children.  Cell numbering: the base cells first, x fastest (those
 * inside the box are "dead": they hold no unknowns and every operator gives 0
 * there), then the (2bx)(2by)(2bz) children as one structured block, x
 * fastest.  A face between a child and a base cell is "hanging": the base
 * cell's face is the union of four children's faces (2:1 in both tangential
 * directions).  Reading of the geometry: a child's map is its parent's
 * isoparametric map restricted to the child, so hanging faces are watertight. */
static int refined(const orc_mesh *m) {
  return m->ref[1] > m->ref[0] && m->ref[3] > m->ref[2] && m->ref[5] > m->ref[4];
}
static long base_cells(const orc_mesh *m) { return (long)m->nx * m->ny * m->nz; }
static void fine_dims(const orc_mesh *m, long fd[3]) {
  for (int d = 0; d < 3; ++d) fd[d] = refined(m) ? 2L * (m->ref[2 * d + 1] - m->ref[2 * d]) : 0;
}
static void base_coords(const orc_mesh *m, long cell, long c[3]) {
  c[0] = cell % m->nx; c[1] = (cell / m->nx) % m->ny; c[2] = cell / ((long)m->nx * m->ny);
}
static int in_box(const orc_mesh *m, const long c[3]) {
  if (!refined(m)) return 0;
  for (int d = 0; d < 3; ++d)
    if (c[d] < m->ref[2 * d] || c[d] >= m->ref[2 * d + 1]) return 0;
  return 1;
}
/* a base cell replaced by its children */
static int cell_dead(const orc_mesh *m, long cell) {
  if (cell >= base_cells(m)) return 0;
  long c[3];
  base_coords(m, cell, c);
  return in_box(m, c);
}
static int cell_fine(const orc_mesh *m, long cell) { return cell >= base_cells(m); }
static void fine_coords(const orc_mesh *m, long cell, long f[3]) {
  long fd[3], l = cell - base_cells(m);
  fine_dims(m, fd);
  f[0] = l % fd[0]; f[1] = (l / fd[0]) % fd[1]; f[2] = l / (fd[0] * fd[1]);
}
static long fine_index(const orc_mesh *m, const long f[3]) {
  long fd[3];
  fine_dims(m, fd);
  return base_cells(m) + f[0] + fd[0] * (f[1] + fd[1] * f[2]);
}
static long base_index(const orc_mesh *m, const long c[3]) { return c[0] + m->nx * (c[1] + (long)m->ny * c[2]); }

/* Physical coordinates of the (r+1)^3 GLL nodes of a cell.  Reading of the
 * terrain-following mapping: Gal-Chen, z = zeta + h(x,y) (1 - zeta/Lz) with
 * zeta uniform on [0, Lz]; x, y affine.  A child's nodes are its parent's
 * isoparametric map evaluated at the child's nodes, xi = (sigma + x_a) / 2. */
static void cell_nodes(const orc_mesh *m, const tabs *T, long cell, double *Xn /* [3][n3] */) {
  int n = T->n, n3 = T->n3;
  if (cell_fine(m, cell)) {
    long f[3], pc[3];
    fine_coords(m, cell, f);
    for (int d = 0; d < 3; ++d) pc[d] = m->ref[2 * d] + f[d] / 2;
    double Xp[3 * ORC_MAXN * ORC_MAXN * ORC_MAXN], ps[ORC_MAXN * ORC_MAXN * ORC_MAXN];
    cell_nodes(m, T, base_index(m, pc), Xp);
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          double xi[3] = {0.5 * (f[0] % 2 + T->gll[a]), 0.5 * (f[1] % 2 + T->gll[b]), 0.5 * (f[2] % 2 + T->gll[c])};
          basis3(T, xi, ps, NULL);
          int i = a + n * (b + n * c);
          for (int d = 0; d < 3; ++d) Xn[d * n3 + i] = dotn(n3, Xp + d * n3, ps);
        }
    return;
  }
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

/* Outward normal times area element times weight, nA [q2][3], at the face
 * points of face f = 2k+s of a cell with nodes Xn. */
static void face_normals(const tabs *T, const double *Xn, int f, double *nA) {
  int n3 = T->n3;
  int k = f / 2, s = f % 2;
  int t1 = (k == 0) ? 1 : 0, t2 = (k == 2) ? 1 : 2;
  for (int p = 0; p < T->q2; ++p) {
    double J[3][3];
    jacobian(n3, Xn, T->fdpsi[f] + (size_t)p * 3 * n3, J);
    double a[3] = {J[0][t1], J[1][t1], J[2][t1]};
    double b[3] = {J[0][t2], J[1][t2], J[2][t2]};
    double N[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    /* outward: along +xi_k on side 1, -xi_k on side 0 */
    double dk = N[0] * J[0][k] + N[1] * J[1][k] + N[2] * J[2][k];
    double sg = ((dk > 0) == (s == 1)) ? 1.0 : -1.0;
    for (int d = 0; d < 3; ++d) nA[3 * p + d] = sg * N[d] * T->fw[f][p];
  }
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
  for (int f = 0; f < 6; ++f) face_normals(T, G->Xn, f, G->nA[f]);
}

/* Neighbour across face (k, s); -1 on the domain boundary.  With periodic
 * lateral boundaries (bc_lateral 2) the x and y directions wrap around (a
 * refinement box must then stay clear of the periodic faces).  -2: a hanging
 * face (see hanging_points). */
static long base_neighbour(const orc_mesh *m, const long c0[3], int k, int s, long c[3]) {
  long nn[3] = {m->nx, m->ny, m->nz};
  for (int d = 0; d < 3; ++d) c[d] = c0[d];
  c[k] += s ? 1 : -1;
  if (c[k] < 0 || c[k] >= nn[k]) {
    if (k == 2 || m->bc_lateral != 2) return -1;
    c[k] = (c[k] + nn[k]) % nn[k];
  }
  return base_index(m, c);
}
static long neighbour(const orc_mesh *m, long cell, int k, int s) {
  long c[3], nc[3];
  if (cell_fine(m, cell)) {
    long f[3], fd[3];
    fine_coords(m, cell, f);
    fine_dims(m, fd);
    f[k] += s ? 1 : -1;
    if (f[k] >= 0 && f[k] < fd[k]) return fine_index(m, f);
    for (int d = 0; d < 3; ++d) c[d] = m->ref[2 * d] + (d == k ? (s ? fd[k] / 2 - 1 : 0) : f[d] / 2);
    return base_neighbour(m, c, k, s, nc) < 0 ? -1 : -2;
  }
  base_coords(m, cell, c);
  long nb = base_neighbour(m, c, k, s, nc);
  if (nb >= 0 && in_box(m, nc)) return -2;
  return nb;
}

/* Cells across the hanging face f = 2k+s of `cell`: for a base cell the four
 * children nb[sig1 + 2 sig2] whose faces make up its face (sig1, sig2 the
 * children's positions along the face's tangential directions t1, t2),
 * returns 4; for a child the base cell nb[0], with the child's position
 * *sig = sig1 + 2 sig2, returns 1. */
static int hanging_cells(const orc_mesh *m, long cell, int f, long *nb, int *sig) {
  int k = f / 2, s = f % 2;
  int t1 = (k == 0) ? 1 : 0, t2 = (k == 2) ? 1 : 2;
  long c[3], nc[3];
  if (cell_fine(m, cell)) {
    long fc[3], fd[3];
    fine_coords(m, cell, fc);
    fine_dims(m, fd);
    for (int d = 0; d < 3; ++d) c[d] = m->ref[2 * d] + (d == k ? (s ? fd[k] / 2 - 1 : 0) : fc[d] / 2);
    nb[0] = base_neighbour(m, c, k, s, nc);
    *sig = (int)(fc[t1] % 2 + 2 * (fc[t2] % 2));
    return 1;
  }
  base_coords(m, cell, c);
  base_neighbour(m, c, k, s, nc);
  for (int sg2 = 0; sg2 < 2; ++sg2)
    for (int sg1 = 0; sg1 < 2; ++sg1) {
      long fc[3];
      fc[k] = 2 * (nc[k] - m->ref[2 * k]) + (s ? 0 : 1);
      fc[t1] = 2 * (c[t1] - m->ref[2 * t1]) + sg1;
      fc[t2] = 2 * (c[t2] - m->ref[2 * t2]) + sg2;
      nb[sg1 + 2 * sg2] = fine_index(m, fc);
    }
  *sig = -1;
  return 4;
}

/* Quadrature points of the hanging face f = 2k+s of `cell`: the face rule of
 * each child face it consists of (four for a base cell, its own for a child).
 * Per point: the neighbour cell nb, this cell's basis ps [n3] and the
 * neighbour's basis psn [n3] there, and nA [3] outward from this cell (the
 * child's face geometry on both sides, so the two sides' fluxes cancel).
 * The child face at position (sig1, sig2) covers the base face's reference
 * square [sig1/2, (sig1+1)/2] x [sig2/2, (sig2+1)/2].  Returns the number of
 * points; the arrays hold 4 q2 points. */
static int hanging_points(const orc_mesh *m, const tabs *T, long cell, int f, long *nb, double *ps, double *psn,
                          double *nA) {
  int k = f / 2, s = f % 2, q = T->q, q2 = T->q2, n3 = T->n3;
  int t1 = (k == 0) ? 1 : 0, t2 = (k == 2) ? 1 : 2;
  int fo = 2 * k + (1 - s); /* the same face seen from the other side */
  double Xn[3 * ORC_MAXN * ORC_MAXN * ORC_MAXN];
  long cells[4];
  int sig;
  int nh = hanging_cells(m, cell, f, cells, &sig);
  if (nh == 1) {
    int sg1 = sig % 2, sg2 = sig / 2;
    cell_nodes(m, T, cell, Xn);
    face_normals(T, Xn, f, nA);
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i) {
        int p = i + q * j;
        double xi[3];
        xi[k] = (double)(1 - s); xi[t1] = 0.5 * (sg1 + T->gq[i]); xi[t2] = 0.5 * (sg2 + T->gq[j]);
        nb[p] = cells[0];
        memcpy(ps + (size_t)p * n3, T->fpsi[f] + (size_t)p * n3, sizeof(double) * n3);
        basis3(T, xi, psn + (size_t)p * n3, NULL);
      }
    return q2;
  }
  double nAc[3 * ORC_MAXQ * ORC_MAXQ];
  for (int sg2 = 0; sg2 < 2; ++sg2)
    for (int sg1 = 0; sg1 < 2; ++sg1) {
      long child = cells[sg1 + 2 * sg2];
      cell_nodes(m, T, child, Xn);
      face_normals(T, Xn, fo, nAc);
      for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
          int p = (sg1 + 2 * sg2) * q2 + i + q * j;
          double xi[3];
          xi[k] = (double)s; xi[t1] = 0.5 * (sg1 + T->gq[i]); xi[t2] = 0.5 * (sg2 + T->gq[j]);
          nb[p] = child;
          basis3(T, xi, ps + (size_t)p * n3, NULL);
          memcpy(psn + (size_t)p * n3, T->fpsi[fo] + (size_t)(i + q * j) * n3, sizeof(double) * n3);
          for (int d = 0; d < 3; ++d) nA[3 * p + d] = -nAc[3 * (i + q * j) + d];
        }
    }
  return 4 * q2;
}

/* Scratch of hanging_points for one face. */
typedef struct { long *nb; double *ps, *psn, *nA; } hang_buf;
static void hang_alloc(hang_buf *H, const tabs *T) {
  H->nb = malloc(sizeof(long) * 4 * T->q2);
  H->ps = malloc(sizeof(double) * 4 * T->q2 * T->n3);
  H->psn = malloc(sizeof(double) * 4 * T->q2 * T->n3);
  H->nA = malloc(sizeof(double) * 4 * T->q2 * 3);
}
static void hang_free(hang_buf *H) { free(H->nb); free(H->ps); free(H->psn); free(H->nA); }

/* Boundary kind of face direction k: 0 slip wall, 1 far field (periodic
 * lateral faces have neighbours and never reach this). */
static int boundary_kind(const orc_mesh *m, int k) { return (k == 2) ? 0 : m->bc_lateral; }



/* LU with partial pivoting, in place; solves A x = b for nrhs right-hand
 * sides stored as rows of B ([nrhs][n]). */
static inline int lu_solve(int n, double *A, int nrhs, double *B) {
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

#endif
