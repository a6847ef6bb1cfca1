"""Geometric multigrid for the pressure system, FP64 numpy (oracle).

TEST INFRASTRUCTURE: the plain checker of the CUDA library's multigrid
preconditioner; only ``tests/`` and the bench's CPU legs may import it.  It
shares no code with the CUDA path.

The paper solves its SPD systems with conjugate gradients preconditioned by
geometric multigrid and, for the non-symmetric Schur system, names the lack
of theory for multigrid (Sec. 3.1, Sec. 4).  This module writes out one
V-cycle as the textbook defines it, level by level, for the structured
terrain-following meshes of the operator:

* levels: the mesh with nx, ny, nz halved each time (same domain, degree,
  terrain and boundaries), so each coarse cell is the union of 2 x 2 x 2 fine
  cells (children) and the reference coordinates nest exactly;
* prolongation P: the coarse cell's polynomial evaluated at the fine GLL nodes
  of each child (nodal interpolation, exact for the coarse polynomial);
  restriction R = P^T (residuals are dual vectors);
* coarse coefficients (rho, p_k): the fine field evaluated at the coarse
  nodes, each coarse node taking the child that holds it (the first child at
  a child interface);
* operator on each level: the Schur operator S of that level's mesh and
  coefficients (rediscretisation), the Helmholtz Jacobi diagonal d of Sec. 3.1;
* smoother: Chebyshev iteration on D^-1 S (Saad, Iterative Methods for Sparse
  Linear Systems, 2nd ed., Algorithm 12.1) over [lambda_max / range, 1.1
  lambda_max], lambda_max from power iteration on D^-1 S from a fixed start
  vector v_i = frac(0.6180339887498949 (i + 1)) - 1/2;
* coarsest level: conjugate gradients preconditioned by D^-1 (SPD systems) or
  FGMRES(30) with D^-1, to a relative residual (at most coarse_its iterations);
* V-cycle with zero initial guess: pre-smooth, restrict the residual, cycle on
  the next level, prolong and correct, post-smooth.
"""
import numpy as np

from . import apply_S, gll, lagrange, make_mesh, ndofs, precond_diag, solve, PC_HELMHOLTZ

GOLDEN = 0.6180339887498949


def start_vector(n):
    """The fixed start vector of the power iteration (no random draws)."""
    i = np.arange(n, dtype=np.float64)
    v = GOLDEN * (i + 1.0)
    return v - np.floor(v) - 0.5


def child_matrices(r):
    """E[s][a_f][a_c] = l_{a_c}((x_{a_f} + s) / 2): the coarse 1D basis at the
    GLL nodes of child s (s = 0 the lower half of the coarse interval)."""
    x, _ = gll(r + 1)
    E = np.zeros((2, r + 1, r + 1))
    for s in range(2):
        for af in range(r + 1):
            E[s, af], _ = lagrange(x, 0.5 * (x[af] + s))
    return E


def inject_matrices(r):
    """For each coarse node a_c: the child s(a_c) that holds it (s = 1 for a
    node above the interval's middle) and F[a_c][i_f] = l_{i_f}(2 x_{a_c} - s):
    the fine child's 1D basis at that node."""
    x, _ = gll(r + 1)
    side = (x > 0.5).astype(int)
    F = np.zeros((r + 1, r + 1))
    for a in range(r + 1):
        F[a], _ = lagrange(x, 2.0 * x[a] - side[a])
    return side, F


def coarse_mesh(m):
    assert m.nx % 2 == 0 and m.ny % 2 == 0 and m.nz % 2 == 0, "each level halves nx, ny, nz"
    return make_mesh(m.nx // 2, m.ny // 2, m.nz // 2, m.r, Lx=m.Lx, Ly=m.Ly, Lz=m.Lz, terrain=m.terrain,
                     hc=m.hc, ac=m.ac, xc=m.xc, yc=m.yc, bc_lateral=m.bc_lateral)


def _cells(m):
    return m.nx * m.ny * m.nz


def prolong(mc, mf, xc):
    """Fine nodal vector of the coarse field xc (one scalar field)."""
    n = mf.r + 1
    E = child_matrices(mf.r)
    X = xc.reshape(mc.nz, mc.ny, mc.nx, n, n, n)  # [cz][cy][cx][c][b][a]
    out = np.zeros((mf.nz, mf.ny, mf.nx, n, n, n))
    for sz in range(2):
        for sy in range(2):
            for sx in range(2):
                # child values: sum over coarse nodes (k, j, i) of Ez[c,k] Ey[b,j] Ex[a,i] X[..., k, j, i]
                child = np.einsum("ck,bj,ai,zyxkji->zyxcba", E[sz], E[sy], E[sx], X)
                out[sz::2, sy::2, sx::2] = child
    return out.reshape(-1)


def restrict(mc, mf, rf):
    """R = P^T applied to a fine dual vector."""
    n = mf.r + 1
    E = child_matrices(mf.r)
    Rf = rf.reshape(mf.nz, mf.ny, mf.nx, n, n, n)
    out = np.zeros((mc.nz, mc.ny, mc.nx, n, n, n))
    for sz in range(2):
        for sy in range(2):
            for sx in range(2):
                out += np.einsum("ck,bj,ai,zyxcba->zyxkji", E[sz], E[sy], E[sx], Rf[sz::2, sy::2, sx::2])
    return out.reshape(-1)


def inject(mc, mf, vf):
    """Coarse nodal values of the fine field vf (coefficients)."""
    n = mf.r + 1
    side, F = inject_matrices(mf.r)
    Vf = vf.reshape(mf.nz, mf.ny, mf.nx, n, n, n)
    out = np.zeros((mc.nz, mc.ny, mc.nx, n, n, n))
    for c in range(n):
        for b in range(n):
            for a in range(n):
                child = Vf[side[c]::2, side[b]::2, side[a]::2]  # [cz][cy][cx][k][j][i]
                out[:, :, :, c, b, a] = np.einsum("k,j,i,zyxkji->zyx", F[c], F[b], F[a], child)
    return out.reshape(-1)


def power_lambda(apply, dinv, its):
    """Largest eigenvalue estimate of D^-1 S: its power steps from start_vector,
    lambda = |w| / |v| of the last step."""
    v = start_vector(len(dinv))
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(its):
        w = dinv * apply(v)
        lam = np.linalg.norm(w)  # |v| = 1
        v = w / lam
    return lam


def chebyshev(apply, dinv, b, x, lmax, lmin, degree):
    """Saad Alg. 12.1 on D^-1 S x = D^-1 b: degree steps from x (updated copy)."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    x = x.copy()
    r = b - apply(x)
    rho = 1.0 / sigma
    d = dinv * r / theta
    for k in range(degree):
        x = x + d
        if k + 1 == degree:
            break
        r = r - apply(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x


def pcg(apply, dinv, b, tol, maxit):
    """Jacobi-preconditioned CG from zero (coarsest level)."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for _ in range(maxit):
        q = apply(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * bn:
            break
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


class Hierarchy:
    """Levels 0 (the given mesh) .. L-1 with their coefficients, Jacobi
    diagonals and eigenvalue bounds."""

    def __init__(self, m, alpha, gamma, rho, pk, levels, degree=3, smooth_range=15.0, power_its=15,
                 coarse_tol=1e-10, coarse_its=500, coarse="cg"):
        self.alpha, self.gamma, self.degree = alpha, gamma, degree
        self.coarse_tol, self.coarse_its, self.coarse = coarse_tol, coarse_its, coarse
        self.meshes, self.rho, self.pk, self.dinv, self.lmax = [m], [rho], [pk], [], []
        for _ in range(levels - 1):
            mc = coarse_mesh(self.meshes[-1])
            self.rho.append(inject(mc, self.meshes[-1], self.rho[-1]))
            self.pk.append(inject(mc, self.meshes[-1], self.pk[-1]))
            self.meshes.append(mc)
        for l, ml in enumerate(self.meshes):
            d = precond_diag(ml, PC_HELMHOLTZ, alpha, gamma, self.rho[l], self.pk[l])
            self.dinv.append(1.0 / d)
            self.lmax.append(power_lambda(self.op(l), self.dinv[l], power_its))
        self.smooth_range = smooth_range

    def op(self, l):
        m, rho, pk = self.meshes[l], self.rho[l], self.pk[l]
        return lambda v: apply_S(m, self.alpha, self.gamma, rho, pk, v)

    def vcycle(self, b, l=0):
        """z = M^-1 b: one V-cycle from zero."""
        S = self.op(l)
        if l == len(self.meshes) - 1:
            if self.coarse == "fgmres":  # the library's FGMRES(30) with the Helmholtz Jacobi
                x, _, _, _ = solve(self.meshes[l], self.alpha, self.gamma, self.rho[l], self.pk[l], b,
                                   method="fgmres", tol=self.coarse_tol, maxit=self.coarse_its)
                return x
            return pcg(S, self.dinv[l], b, self.coarse_tol, self.coarse_its)
        lmax = 1.1 * self.lmax[l]
        lmin = self.lmax[l] / self.smooth_range
        x = chebyshev(S, self.dinv[l], b, np.zeros_like(b), lmax, lmin, self.degree)
        r = b - S(x)
        ec = self.vcycle(restrict(self.meshes[l + 1], self.meshes[l], r), l + 1)
        x = x + prolong(self.meshes[l + 1], self.meshes[l], ec)
        return chebyshev(S, self.dinv[l], b, x, lmax, lmin, self.degree)


def mg_pcg(h, b, tol=1e-10, maxit=500):
    """CG preconditioned by one V-cycle per iteration (SPD systems).
    Returns (x, iterations, relative residual)."""
    S = h.op(0)
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    z = h.vcycle(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit and np.linalg.norm(r) > tol * bn:
        q = S(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        it += 1
        z = h.vcycle(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, np.linalg.norm(r) / bn
