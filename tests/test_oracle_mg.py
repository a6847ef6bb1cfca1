"""Pins of the geometric multigrid oracle (oracle/mg.py) against what the
mathematics fixes: nodal prolongation reproduces the coarse polynomial
exactly, restriction is its transpose, the coarse coefficients are the fine
field's values at the coarse nodes (with the stated child at an interface),
the Chebyshev smoother's error is the scaled Chebyshev polynomial of the
operator (Saad, Alg. 12.1) in closed form, power iteration finds the top
eigenvalue of a diagonal matrix, and the V-cycle preconditions CG on the SPD
special case of the Schur operator (uniform coefficients, slip walls: S SPD,
Sec. 3.1).  Planted mistakes (swapped children, a flipped interface rule, a
sign error in the Chebyshev recurrence) each fail a named pin."""
import numpy as np
import pytest

import oracle as O
from oracle import mg

A_DT = 0.29289321881345254
GAMMA = 1.4


def _poly(X, Lx, Ly, Lz, r):
    """A polynomial of degree r in each coordinate (tensor-product space)."""
    x, y, z = X[0] / Lx, X[1] / Ly, X[2] / Lz
    px = sum((k + 1) * x ** k for k in range(r + 1))
    py = sum((-1) ** k * (k + 2) * y ** k for k in range(r + 1))
    pz = sum(0.5 ** k * z ** k for k in range(r + 1))
    return px * py * pz


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_prolongation_reproduces_coarse_polynomials(r):
    mf = O.make_mesh(4, 2, 6, r, Lx=2000.0, Ly=1000.0, Lz=3000.0)
    mc = mg.coarse_mesh(mf)
    fc = _poly(O.node_coords(mc), 2000.0, 1000.0, 3000.0, r)
    ff = _poly(O.node_coords(mf), 2000.0, 1000.0, 3000.0, r)
    assert np.abs(mg.prolong(mc, mf, fc) - ff).max() <= 1e-12 * np.abs(ff).max()


def test_restriction_is_the_transpose():
    mf = O.make_mesh(4, 4, 2, 3, terrain=1, hc=200.0, ac=500.0)
    mc = mg.coarse_mesh(mf)
    rng = np.random.default_rng(3)
    xc, yf = rng.standard_normal(O.ndofs(mc)), rng.standard_normal(O.ndofs(mf))
    lhs = mg.prolong(mc, mf, xc) @ yf
    rhs = xc @ mg.restrict(mc, mf, yf)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("r", [2, 3, 4])
def test_injection_of_polynomial_coefficients(r):
    mf = O.make_mesh(2, 4, 2, r, Lx=1000.0, Ly=2000.0, Lz=1000.0)
    mc = mg.coarse_mesh(mf)
    vf = _poly(O.node_coords(mf), 1000.0, 2000.0, 1000.0, r)
    vc = _poly(O.node_coords(mc), 1000.0, 2000.0, 1000.0, r)
    assert np.abs(mg.inject(mc, mf, vf) - vc).max() <= 1e-12 * np.abs(vc).max()


@pytest.mark.parametrize("r", [2, 3])
def test_injection_takes_the_child_that_holds_the_node(r):
    """A field constant on each fine cell (value = the cell's index): a coarse
    node strictly inside child s gets that child's value; a node on the
    children's interface (the middle GLL node, even r) gets the lower child's."""
    mf = O.make_mesh(2, 2, 2, r)
    mc = mg.coarse_mesh(mf)
    n = r + 1
    vf = np.repeat(np.arange(8, dtype=float), n ** 3)
    vc = mg.inject(mc, mf, vf).reshape(n, n, n)  # [c][b][a]
    x, _ = O.gll(n)
    side = [1 if xi > 0.5 else 0 for xi in x]
    for c in range(n):
        for b in range(n):
            for a in range(n):
                assert vc[c, b, a] == pytest.approx(side[a] + 2 * side[b] + 4 * side[c], abs=1e-12)


def test_chebyshev_error_is_the_scaled_chebyshev_polynomial():
    lam = np.linspace(0.3, 4.0, 41)
    b = np.cos(np.arange(41.0))
    A = lambda v: lam * v
    lmin, lmax = 0.3, 4.0
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    for degree in (1, 2, 3, 5):
        x = mg.chebyshev(A, np.ones(41), b, np.zeros(41), lmax, lmin, degree)
        e0 = b / lam  # exact solution minus the zero start
        T = np.polynomial.chebyshev.Chebyshev.basis(degree)
        pk = T((theta - lam) / delta) / T(theta / delta)
        assert np.allclose(b / lam - x, pk * e0, rtol=1e-12, atol=1e-14)


def test_power_iteration_finds_the_top_eigenvalue():
    lam = np.concatenate([np.linspace(0.1, 1.0, 50), [2.0]])
    lest = mg.power_lambda(lambda v: lam * v, np.ones(51), 200)
    assert lest == pytest.approx(2.0, rel=1e-12)


def test_vcycle_preconditions_cg_on_the_spd_case():
    """Uniform coefficients and slip walls make S SPD (Sec. 3.1's CG case):
    CG with one V-cycle (3 levels) per iteration reaches 1e-10 in at most half
    the Jacobi-CG iterations and agrees with the Jacobi-CG solution."""
    m = O.make_mesh(8, 8, 4, 2, Lx=4000.0, Ly=4000.0, Lz=2000.0)
    N = O.ndofs(m)
    rho, pk = np.full(N, 1.2), np.full(N, 1e5)
    b = np.random.default_rng(5).standard_normal(N)
    h = mg.Hierarchy(m, A_DT, GAMMA, rho, pk, levels=3, degree=3)
    x, its, rel = mg.mg_pcg(h, b, tol=1e-10)
    xj, st, jits, _ = O.solve(m, A_DT, GAMMA, rho, pk, b, method="cg", tol=1e-10, maxit=5000)
    assert st == 0 and rel <= 1e-10
    assert its * 2 <= jits, (its, jits)
    assert np.abs(x - xj).max() <= 1e-7 * np.abs(xj).max()


# ---- planted mistakes: each must make a named pin fail

def test_planted_swapped_children_fails_the_polynomial_pin(monkeypatch):
    real = mg.child_matrices
    monkeypatch.setattr(mg, "child_matrices", lambda r: real(r)[::-1])
    with pytest.raises(AssertionError):
        test_prolongation_reproduces_coarse_polynomials(2)


def test_planted_flipped_interface_rule_fails_the_child_pin(monkeypatch):
    def flipped(r):
        x, _ = O.gll(r + 1)
        side = (x >= 0.5).astype(int)
        F = np.zeros((r + 1, r + 1))
        for a in range(r + 1):
            F[a], _ = O.lagrange(x, 2.0 * x[a] - side[a])
        return side, F
    monkeypatch.setattr(mg, "inject_matrices", flipped)
    with pytest.raises(AssertionError):
        test_injection_takes_the_child_that_holds_the_node(2)


def test_planted_chebyshev_sign_fails_the_closed_form(monkeypatch):
    def wrong(apply, dinv, b, x, lmax, lmin, degree):
        theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
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
            rho_new = 1.0 / (2.0 * sigma + rho)  # planted: + instead of -
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
            rho = rho_new
        return x
    monkeypatch.setattr(mg, "chebyshev", wrong)
    with pytest.raises(AssertionError):
        test_chebyshev_error_is_the_scaled_chebyshev_polynomial()
