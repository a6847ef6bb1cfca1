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
#include "orc_core.h"

/* ------------------------------------------------------------------ */
/* 1D rules (textbook: Newton iteration on Legendre polynomials)       */
/* ------------------------------------------------------------------ */

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

/* Bottom height of the terrain-following mesh. */
double orc_terrain_height(const orc_mesh *m, double x, double y) {
  if (m->terrain == 0) return 0.0;
  double s = 1.0 + ((x - m->xc) * (x - m->xc) + (y - m->yc) * (y - m->yc)) / (m->ac * m->ac);
  if (m->terrain == 1) return m->hc / s;
  return m->hc * pow(s, -1.5);
}

long orc_num_cells(const orc_mesh *m) {
  long fd[3];
  fine_dims(m, fd);
  return base_cells(m) + fd[0] * fd[1] * fd[2];
}

/* Face relation for the tests: -1 domain boundary, 0 conforming neighbour
 * nb[0], 1 hanging face of a base cell (the four children nb[sig1 + 2 sig2]),
 * 2 hanging face of a child (the base cell nb[0], the child's position
 * sig1 + 2 sig2 in nb[1]), 3 dead cell. */
int orc_face_info(const orc_mesh *m, long cell, int f, long *nb) {
  if (cell_dead(m, cell)) return 3;
  long r = neighbour(m, cell, f / 2, f % 2);
  if (r >= -1) { nb[0] = r; return r < 0 ? -1 : 0; }
  int sig;
  if (hanging_cells(m, cell, f, nb, &sig) == 4) return 1;
  nb[1] = sig;
  return 2;
}

/* ------------------------------------------------------------------ */
/* Cell operators                                                       */
/* ------------------------------------------------------------------ */

/* (B P) on one cell, 3 components [3][n3]:
 *   alpha [ - int_K p div(phi) + int_dK p_hat phi.n ]
 * Reading of the flux: p_hat = {p} = (p- + p+)/2 on interior faces,
 * p_hat = p- on slip walls (p+ = p-), and on far-field faces the far-field
 * datum of the perturbation pressure, p_hat = 0, imposed weakly (the
 * transmissive choice p+ = p- there makes the acoustic subsystem gain energy
 * through the boundary). */
static void cell_B(const orc_mesh *m, const tabs *T, const cgeo *G, hang_buf *H, long cell, double alpha,
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
    if (nb == -2) { /* hanging face: central p_hat at the child faces' points */
      int np = hanging_points(m, T, cell, f, H->nb, H->ps, H->psn, H->nA);
      for (int qp = 0; qp < np; ++qp) {
        const double *ps = H->ps + (size_t)qp * n3;
        double ph = 0.5 * (dotn(n3, pc, ps) + dotn(n3, p + H->nb[qp] * n3, H->psn + (size_t)qp * n3));
        for (int i = 0; i < n3; ++i)
          for (int d = 0; d < 3; ++d) out[d * n3 + i] += ph * ps[i] * H->nA[3 * qp + d];
      }
      continue;
    }
    const double *fps = T->fpsi[f], *fpsn = T->fpsi[2 * k + (1 - s)];
    int ff = nb < 0 && boundary_kind(m, k) == 1;
    for (int qp = 0; qp < T->q2; ++qp) {
      double pm = dotn(n3, pc, fps + (size_t)qp * n3);
      double ph = pm;
      if (nb >= 0) ph = 0.5 * (pm + dotn(n3, p + nb * n3, fpsn + (size_t)qp * n3));
      if (ff) ph = 0.0; /* far field: the background pressure, p' = 0, imposed weakly */
      const double *nA = G->nA[f] + 3 * qp;
      for (int i = 0; i < n3; ++i) {
        double v = ph * fps[(size_t)qp * n3 + i];
        for (int d = 0; d < 3; ++d) out[d * n3 + i] += v * nA[d];
      }
    }
  }
  for (int i = 0; i < 3 * n3; ++i) out[i] *= alpha;
}

/* Dense density-weighted mass of one cell,
 * A_ij = sum_q rho(x_q) psi_i(x_q) psi_j(x_q) w_q det J(x_q),
 * with the r+1 point Gauss rule of the fast inverse (consistent = 0, Sec. 3.3)
 * or the consistent 2r+1 point rule of the other integrals (consistent = 1,
 * the integration the fast inverse replaces). */
static void cell_A_matrix(const tabs *T, const cgeo *G, long cell, const double *rho, double *A, int consistent) {
  int n3 = T->n3;
  int nq = consistent ? T->q3 : n3;
  const double *rc = rho + cell * n3;
  memset(A, 0, sizeof(double) * n3 * n3);
  for (int qp = 0; qp < nq; ++qp) {
    const double *ps = (consistent ? T->psi : T->psia) + (size_t)qp * n3;
    double c = dotn(n3, rc, ps) * (consistent ? G->wdet[qp] : G->wdeta[qp]);
    for (int i = 0; i < n3; ++i)
      for (int j = 0; j < n3; ++j) A[i * n3 + j] += c * ps[i] * ps[j];
  }
}


/* (C V) on one cell: alpha [ - int_K kappa V.grad(psi) + int_dK (kappa V)^.n psi ],
 * kappa = gamma p_k / (gamma - 1)  (h rho with h = gamma p / ((gamma-1) rho)).
 * Reading of the flux: (kappa V)^ = average of both traces on interior faces;
 * zero normal flux on slip walls ((V.n)+ = -(V.n)-); far-field faces are
 * transmissive in the pressure operator ((kappa V)+ = (kappa V)-). */
static void cell_C(const orc_mesh *m, const tabs *T, const cgeo *G, hang_buf *H, long cell, double alpha,
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
    if (nb == -2) { /* hanging face: central flux at the child faces' points */
      int np = hanging_points(m, T, cell, f, H->nb, H->ps, H->psn, H->nA);
      for (int qp = 0; qp < np; ++qp) {
        const double *ps = H->ps + (size_t)qp * n3, *pn = H->psn + (size_t)qp * n3, *nA = H->nA + 3 * qp;
        long o = H->nb[qp] * n3;
        double vm = dotn(n3, V0, ps) * nA[0] + dotn(n3, V1, ps) * nA[1] + dotn(n3, V2, ps) * nA[2];
        double vp = dotn(n3, V + o, pn) * nA[0] + dotn(n3, V + N + o, pn) * nA[1] + dotn(n3, V + 2 * N + o, pn) * nA[2];
        double flux = 0.5 * (kf * dotn(n3, kc, ps) * vm + kf * dotn(n3, pk + o, pn) * vp);
        for (int i = 0; i < n3; ++i) out[i] += flux * ps[i];
      }
      continue;
    }
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
    hang_buf H; hang_alloc(&H, &S.T);
    double *loc = malloc(sizeof(double) * 3 * n3);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      if (cell_dead(m, c)) memset(loc, 0, sizeof(double) * 3 * n3);
      else {
        cell_geometry(m, &S.T, c, &G);
        cell_B(m, &S.T, &G, &H, c, alpha, p, loc);
      }
      for (int d = 0; d < 3; ++d) memcpy(out + d * S.N + c * n3, loc + d * n3, sizeof(double) * n3);
    }
    free(loc); hang_free(&H); cgeo_free(&G);
  }
  tabs_free(&S.T);
  return 0;
}

/* inverse = 0: out = A_rho in ; inverse = 1: out = A_rho^-1 in (per component);
 * consistent selects the quadrature of A_rho (see cell_A_matrix). */
static int apply_A_impl(const orc_mesh *m, const double *rho, const double *in, double *out, int inverse,
                        int consistent) {
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
      if (cell_dead(m, c)) {
        for (int d = 0; d < 3; ++d) memset(out + d * S.N + c * n3, 0, sizeof(double) * n3);
        continue;
      }
      cell_geometry(m, &S.T, c, &G);
      cell_A_matrix(&S.T, &G, c, rho, A, consistent);
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
  return apply_A_impl(m, rho, in, out, 0, 0);
}
int orc_apply_Ainv(const orc_mesh *m, const double *rho, const double *in, double *out) {
  return apply_A_impl(m, rho, in, out, 1, 0);
}
/* A_rho or its inverse with either quadrature (consistent = 1: 2r+1 points). */
int orc_apply_mass(const orc_mesh *m, int consistent, int inverse, const double *rho, const double *in,
                   double *out) {
  return apply_A_impl(m, rho, in, out, inverse, consistent);
}

int orc_apply_C(const orc_mesh *m, double alpha, double gamma, const double *pk, const double *V, double *out) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
    hang_buf H; hang_alloc(&H, &S.T);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < S.nc; ++c) {
      if (cell_dead(m, c)) { memset(out + c * n3, 0, sizeof(double) * n3); continue; }
      cell_geometry(m, &S.T, c, &G);
      cell_C(m, &S.T, &G, &H, c, alpha, gamma, pk, V, S.N, out + c * n3);
    }
    hang_free(&H); cgeo_free(&G);
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
      if (cell_dead(m, c)) { memset(out + c * n3, 0, sizeof(double) * n3); continue; }
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
 * flagged cells and on their face neighbours.  consistent selects the
 * quadrature of A (see cell_A_matrix). */
int orc_apply_S_rule(const orc_mesh *m, int consistent, double alpha, double gamma, const double *rho,
                     const double *pk, const double *p, const unsigned char *mask, double *y) {
  orc_setup S;
  if (setup(&S, m)) return -1;
  int n3 = S.T.n3;
  long nc = S.nc, N = S.N;
  unsigned char *need = calloc(nc, 1);
  for (long c = 0; c < nc; ++c) {
    if ((mask && !mask[c]) || cell_dead(m, c)) continue;
    need[c] = 1;
    for (int f = 0; f < 6; ++f) {
      long nb[4];
      int rel = orc_face_info(m, c, f, nb);
      if (rel == 0) need[nb[0]] = 1;
      if (rel == 1) for (int j = 0; j < 4; ++j) need[nb[j]] = 1;
      if (rel == 2) need[nb[0]] = 1;
    }
  }
  double *V = calloc((size_t)3 * N, sizeof(double));
  int err = 0;
#pragma omp parallel
  {
    cgeo G; cgeo_alloc(&G, &S.T);
    hang_buf H; hang_alloc(&H, &S.T);
    double *A = malloc(sizeof(double) * n3 * n3);
    double *B = malloc(sizeof(double) * 3 * n3);
    double *loc = malloc(sizeof(double) * 2 * n3);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < nc; ++c) {
      if (!need[c]) continue;
      cell_geometry(m, &S.T, c, &G);
      cell_B(m, &S.T, &G, &H, c, alpha, p, B);
      cell_A_matrix(&S.T, &G, c, rho, A, consistent);
      if (lu_solve(n3, A, 3, B)) err = -2;
      for (int d = 0; d < 3; ++d) memcpy(V + d * N + c * n3, B + d * n3, sizeof(double) * n3);
    }
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < nc; ++c) {
      if (mask && !mask[c]) continue;
      if (cell_dead(m, c)) { memset(y + c * n3, 0, sizeof(double) * n3); continue; }
      cell_geometry(m, &S.T, c, &G);
      cell_M(&S.T, &G, c, 1.0 / (gamma - 1.0), p, loc);
      cell_C(m, &S.T, &G, &H, c, alpha, gamma, pk, V, N, loc + n3);
      for (int i = 0; i < n3; ++i) y[c * n3 + i] = loc[i] - loc[n3 + i];
    }
    free(A); free(B); free(loc); hang_free(&H); cgeo_free(&G);
  }
  free(V); free(need);
  tabs_free(&S.T);
  return err;
}

int orc_apply_S_masked(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
                       const double *p, const unsigned char *mask, double *y) {
  return orc_apply_S_rule(m, 0, alpha, gamma, rho, pk, p, mask, y);
}

int orc_apply_S(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
                const double *p, double *y) {
  return orc_apply_S_rule(m, 0, alpha, gamma, rho, pk, p, NULL, y);
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
      double *o = dg + c * n3;
      if (cell_dead(m, c)) { for (int i = 0; i < n3; ++i) o[i] = 1.0; continue; } /* no unknowns */
      cell_geometry(m, &S.T, c, &G);
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
  int consistent;  /* quadrature of A in S */
} sctx;

static void S_apply(const sctx *c, const double *x, double *y) {
  orc_apply_S_rule(c->m, c->consistent, c->alpha, c->gamma, c->rho, c->pk, x, NULL, y);
}

/* Flexible GMRES(restart), right preconditioned by the diagonal scaling
 * z = dinv .* v (dinv NULL: identity), classical Gram-Schmidt applied twice.
 * Convergence: true residual ||b - S x|| / ||b|| <= tol, checked at every
 * restart (the Arnoldi estimate ends a cycle early).  Returns 0 converged,
 * 1 not converged within maxit, <0 error. */
int orc_fgmres_rule(const orc_mesh *m, int consistent, double alpha, double gamma, const double *rho,
                    const double *pk, const double *dinv, const double *b, double *x, double tol, int restart,
                    int maxit, int *its_out, double *relres_out) {
  sctx c = {m, alpha, gamma, rho, pk, consistent};
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

int orc_fgmres(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
               const double *dinv, const double *b, double *x, double tol, int restart, int maxit,
               int *its_out, double *relres_out) {
  return orc_fgmres_rule(m, 0, alpha, gamma, rho, pk, dinv, b, x, tol, restart, maxit, its_out, relres_out);
}

/* Preconditioned conjugate gradients (for the symmetric positive definite
 * case); same stopping rule on the true recursive residual. */
int orc_cg(const orc_mesh *m, double alpha, double gamma, const double *rho, const double *pk,
           const double *dinv, const double *b, double *x, double tol, int maxit, int *its_out,
           double *relres_out) {
  sctx c = {m, alpha, gamma, rho, pk, 0};
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
