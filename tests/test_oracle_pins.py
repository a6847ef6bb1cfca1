"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: exact quadrature
of monomials, exact 1D element matrices integrated symbolically (sympy),
closed-form results of the weak operators on fields they must reproduce,
the invariants and the symmetry / definiteness the formulation implies, and
manufactured-solution convergence rates.  The paper is arXiv:2505.00384;
Sec. 2 defines the block system and the Schur form, Sec. 3.1 the Helmholtz
preconditioner, Sec. 3.3 the fast block-diagonal inverse and the 2r+1 point
consistent integration.
"""
import numpy as np
import pytest
import sympy as sp

import oracle as O

GAMMA = 1.4
ALPHA = 0.3


# --------------------------------------------------------------- 1D rules
@pytest.mark.parametrize("q", [1, 2, 3, 5, 9, 11])
def test_gauss_exactness(q):
    # q-point Gauss-Legendre integrates x^k exactly for k <= 2q-1 (Sec. 3.3)
    x, w = O.gauss(q)
    for k in range(2 * q):
        assert abs(w @ x**k - 1.0 / (k + 1)) < 1e-14
    # same rule as numpy's Gauss-Legendre routine mapped to [0,1]
    t, v = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, 0.5 * (1 + t), atol=1e-15, rtol=0) and np.allclose(w, 0.5 * v, atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_gll_exactness(n):
    # n-point Gauss-Lobatto integrates x^k exactly for k <= 2n-3
    x, w = O.gll(n)
    assert x[0] == 0.0 and abs(x[-1] - 1.0) < 1e-15
    for k in range(2 * n - 2):
        assert abs(w @ x**k - 1.0 / (k + 1)) < 1e-14
    # interior nodes are the roots of P'_{n-1} (numpy Legendre series)
    dP = np.polynomial.legendre.Legendre.basis(n - 1).deriv()
    if n > 2:
        assert np.abs(dP(2 * x[1:-1] - 1)).max() < 1e-12 * max(1.0, np.abs(dP.coef).max())


def test_gll_known_values():
    x, w = O.gll(4)
    s = 1 / np.sqrt(5)
    assert np.allclose(x, [0, (1 - s) / 2, (1 + s) / 2, 1], atol=1e-15)
    assert np.allclose(w, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)
    x, w = O.gll(5)
    t = np.sqrt(3 / 7)
    assert np.allclose(x, [0, (1 - t) / 2, 0.5, (1 + t) / 2, 1], atol=1e-15)
    assert np.allclose(w, [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5, 6])
def test_lagrange(n):
    xn, _ = O.gll(n)
    for b in range(n):
        l, _ = O.lagrange(xn, xn[b])
        assert np.allclose(l, np.eye(n)[b], atol=1e-14)
    for x in [0.1, 0.37, 0.9]:
        l, dl = O.lagrange(xn, x)
        assert abs(l.sum() - 1) < 1e-14 and abs(dl.sum()) < 1e-12
        # derivative exact on x^k, k <= r
        for k in range(1, n):
            assert abs(dl @ xn**k - k * x ** (k - 1)) < 1e-11


# ------------------------------------------------ exact 1D element matrices
def _sym_1d(r):
    """Exact 1D GLL-basis matrices on [0,1]: mass M1, G1[a,b] = int l_a l_b',
    stiffness K1, and int l_a."""
    t = sp.symbols("t")
    nodes = {1: [0, 1], 2: [0, sp.Rational(1, 2), 1],
             3: [0, (5 - sp.sqrt(5)) / 10, (5 + sp.sqrt(5)) / 10, 1]}[r]
    n = r + 1
    L = []
    for a in range(n):
        e = sp.Integer(1)
        for b in range(n):
            if b != a:
                e *= (t - nodes[b]) / (nodes[a] - nodes[b])
        L.append(sp.expand(e))
    f = lambda e: float(sp.integrate(e, (t, 0, 1)))
    M1 = np.array([[f(L[a] * L[b]) for b in range(n)] for a in range(n)])
    G1 = np.array([[f(L[a] * sp.diff(L[b], t)) for b in range(n)] for a in range(n)])
    K1 = np.array([[f(sp.diff(L[a], t) * sp.diff(L[b], t)) for b in range(n)] for a in range(n)])
    W1 = np.array([f(L[a]) for a in range(n)])
    return M1, G1, K1, W1


def _k3(Ax, Ay, Az):
    # DoF index a + n b + n^2 c (x fastest)
    return np.kron(Az, np.kron(Ay, Ax))


@pytest.mark.parametrize("r", [1, 2, 3])
def test_single_cell_matrices_closed_form(r):
    hx, hy, hz = 700.0, 500.0, 300.0
    m = O.make_mesh(1, 1, 1, r, Lx=hx, Ly=hy, Lz=hz)
    N = O.ndofs(m)
    M1, G1, K1, _ = _sym_1d(r)
    Mref = hx * hy * hz * _k3(M1, M1, M1)
    M = O.assemble(lambda v: O.apply_M(m, v), N, N)
    assert np.abs(M - Mref).max() <= 1e-13 * np.abs(Mref).max()
    D = O.assemble(lambda v: O.apply_D(m, GAMMA, v), N, N)
    assert np.abs(D - Mref / (GAMMA - 1)).max() <= 1e-13 * np.abs(Mref).max()
    # B (one cell, all faces walls): B = alpha int grad(p).phi, e.g. x part
    # alpha hy hz (M1 x M1 x G1); y, z analogous.
    B = O.assemble(lambda v: O.apply_B(m, ALPHA, v), N, 3 * N)
    I = np.eye(r + 1)
    Bref = [ALPHA * hy * hz * _k3(G1, M1, M1), ALPHA * hx * hz * _k3(M1, G1, M1), ALPHA * hx * hy * _k3(M1, M1, G1)]
    for d in range(3):
        assert np.abs(B[d * N:(d + 1) * N] - Bref[d]).max() <= 1e-12 * np.abs(Bref[d]).max()
    # C with constant kappa and wall faces: C = -kappa B^T
    pk = np.full(N, 1e5)
    kappa = GAMMA * 1e5 / (GAMMA - 1)
    Cm = O.assemble(lambda v: O.apply_C(m, ALPHA, GAMMA, pk, v), 3 * N, N)
    Bfull = np.vstack(Bref)
    assert np.abs(Cm + kappa * Bfull.T).max() <= 1e-12 * kappa * np.abs(Bfull).max()
    # fast rho-mass (r+1 Gauss points) with constant rho equals rho * M exactly
    rho = np.full(N, 1.3)
    A = O.assemble(lambda v: O.apply_A(m, rho, v), 3 * N, 3 * N)
    for d in range(3):
        blk = A[d * N:(d + 1) * N, d * N:(d + 1) * N]
        assert np.abs(blk - 1.3 * Mref).max() <= 1e-13 * np.abs(Mref).max()
    # Helmholtz diagonal: M_ii/(g-1) + alpha^2 h (stiffness)_ii, uniform h
    h = GAMMA * 1e5 / ((GAMMA - 1) * 1.3)
    Kref = hx * hy * hz * (_k3(K1, M1, M1) / hx**2 + _k3(M1, K1, M1) / hy**2 + _k3(M1, M1, K1) / hz**2)
    dref = np.diag(Mref) / (GAMMA - 1) + ALPHA**2 * h * np.diag(Kref)
    d = O.precond_diag(m, O.PC_HELMHOLTZ, ALPHA, GAMMA, rho, pk)
    assert np.abs(d - dref).max() <= 1e-12 * dref.max()
    d2 = O.precond_diag(m, O.PC_INTERNAL_ENERGY, ALPHA, GAMMA, rho, pk)
    assert np.abs(d2 - np.diag(Mref) / (GAMMA - 1)).max() <= 1e-13 * dref.max()


@pytest.mark.parametrize("r", [1, 2])
def test_interior_face_fluxes_closed_form(r):
    """2x1x1 cells, piecewise-constant fields: the central averages on the
    shared face give closed forms (weak forms integrated by parts)."""
    hx, hy, hz = 400.0, 300.0, 200.0
    m = O.make_mesh(2, 1, 1, r, Lx=2 * hx, Ly=hy, Lz=hz)
    n = r + 1
    n3 = n**3
    N = O.ndofs(m)
    _, _, _, W1 = _sym_1d(r)
    ea0 = np.eye(n)[0]
    ean = np.eye(n)[n - 1]
    # p = 1 on cell 0, 0 on cell 1: B p = alpha int grad p . phi + alpha/2 int [p] phi.n
    p = np.zeros(N)
    p[:n3] = 1.0
    Bp = O.apply_B(m, ALPHA, p)
    ref0 = -0.5 * ALPHA * hy * hz * np.kron(W1, np.kron(W1, ean))
    ref1 = -0.5 * ALPHA * hy * hz * np.kron(W1, np.kron(W1, ea0))
    sc = np.abs(ref0).max()
    assert np.abs(Bp[:n3] - ref0).max() <= 1e-13 * sc
    assert np.abs(Bp[n3:N] - ref1).max() <= 1e-13 * sc
    assert np.abs(Bp[N:]).max() <= 1e-13 * sc
    # V = (1,0,0) on cell 0, 0 on cell 1, constant kappa
    V = np.zeros(3 * N)
    V[:n3] = 1.0
    pk = np.full(N, 1e5)
    kappa = GAMMA * 1e5 / (GAMMA - 1)
    CV = O.apply_C(m, ALPHA, GAMMA, pk, V)
    ref0 = ALPHA * kappa * hy * hz * np.kron(W1, np.kron(W1, ea0 - 0.5 * ean))
    ref1 = ALPHA * kappa * hy * hz * np.kron(W1, np.kron(W1, -0.5 * ea0))
    sc = np.abs(ref0).max()
    assert np.abs(CV[:n3] - ref0).max() <= 1e-13 * sc
    assert np.abs(CV[n3:] - ref1).max() <= 1e-13 * sc


@pytest.mark.parametrize("r", [1, 2])
def test_far_field_pressure_flux_closed_form(r):
    """One cell with far-field lateral faces and slip walls at bottom and top,
    constant p = c: the far-field datum p^ = 0 (the perturbation pressure of the
    background) leaves only the far-field faces' term, B p = -alpha c int_ff phi.n,
    i.e. the x part -alpha c hy hz (W x W x (e_n - e_0)), y analogous, z zero."""
    hx, hy, hz = 700.0, 500.0, 300.0
    m = O.make_mesh(1, 1, 1, r, Lx=hx, Ly=hy, Lz=hz, bc_lateral=1)
    N = O.ndofs(m)
    n = r + 1
    _, _, _, W1 = _sym_1d(r)
    de = np.eye(n)[n - 1] - np.eye(n)[0]
    c = 2.0
    Bp = O.apply_B(m, ALPHA, np.full(N, c))
    refx = -ALPHA * c * hy * hz * _k3(de, W1, W1)
    refy = -ALPHA * c * hx * hz * _k3(W1, de, W1)
    sc = np.abs(refx).max()
    assert np.abs(Bp[:N] - refx).max() <= 1e-13 * sc
    assert np.abs(Bp[N:2 * N] - refy).max() <= 1e-13 * sc
    assert np.abs(Bp[2 * N:]).max() <= 1e-13 * sc


def test_far_field_divergence_of_constant_field():
    """Flat box, far-field lateral faces (transmissive (kappa V)^ in C) and
    slip walls at bottom and top: a constant horizontal kappa V has zero weak
    divergence, C V = 0 (the volume term and the far-field face terms cancel;
    V.n = 0 on the walls)."""
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=1600.0, Lz=1500.0, bc_lateral=1)
    N = O.ndofs(m)
    V = np.concatenate([np.full(N, 3.0), np.full(N, -2.0), np.zeros(N)])
    CV = O.apply_C(m, ALPHA, GAMMA, np.full(N, 1e5), V)
    kappa = GAMMA * 1e5 / (GAMMA - 1)
    assert np.abs(CV).max() <= 1e-13 * ALPHA * kappa * 3.0 * 1e6


# ------------------------------------------------------- curved geometry
CURVED = [dict(terrain=1, hc=300.0, ac=800.0), dict(terrain=2, hc=250.0, ac=600.0, xc=1100.0, yc=900.0)]


@pytest.mark.parametrize("geo", CURVED)
@pytest.mark.parametrize("r", [1, 2, 3])
def test_B_reproduces_gradient_of_linear_fields(geo, r):
    """For p = x, y or z (exactly representable on the isoparametric mesh),
    central {p} equals the trace, so B p = alpha M grad p: the x-, y- or
    z-component of B p equals alpha M 1 and the others vanish.  This pins the
    volume metric terms and the face normals of the curved cells."""
    m = O.make_mesh(3, 2, 2, r, Lx=3000.0, Ly=2000.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    X = O.node_coords(m)
    M1 = O.apply_M(m, np.ones(N))
    for d in range(3):
        Bp = O.apply_B(m, ALPHA, X[d].copy())
        for e in range(3):
            ref = ALPHA * M1 if e == d else np.zeros(N)
            assert np.abs(Bp[e * N:(e + 1) * N] - ref).max() <= 1e-13 * np.abs(ALPHA * M1).max()


@pytest.mark.parametrize("geo", CURVED)
def test_terrain_following_map(geo):
    """Node coordinates of the terrain-following mesh: x and y on the uniform
    lateral grid of each cell's GLL nodes, the bottom surface on the terrain
    h(x, y), the top flat at Lz, and z affine in the computational vertical
    coordinate along every vertical node column (the Gal-Chen map)."""
    import oracle.learned as NL
    nx, ny, nz, r = 3, 2, 4, 2
    Lx, Ly, Lz = 3000.0, 2000.0, 1500.0
    m = O.make_mesh(nx, ny, nz, r, Lx=Lx, Ly=Ly, Lz=Lz, **geo)
    n = r + 1
    shape = (nz * n, ny * n, nx * n)
    perm = NL.dof_to_grid_index(nx, ny, nz, r)
    Xg = [NL.to_grid(c, shape, perm) for c in O.node_coords(m)]
    xn, _ = O.gll(n)
    xs = ((np.arange(nx)[:, None] + xn[None, :]) * Lx / nx).ravel()
    ys = ((np.arange(ny)[:, None] + xn[None, :]) * Ly / ny).ravel()
    zeta = ((np.arange(nz)[:, None] + xn[None, :]) * Lz / nz).ravel()
    assert np.array_equal(Xg[0], np.broadcast_to(xs, shape))
    assert np.array_equal(Xg[1], np.broadcast_to(ys[None, :, None], shape))
    h = np.array([[O.terrain_height(m, x, y) for x in xs] for y in ys])
    assert h.max() > 0.5 * geo["hc"]
    assert np.abs(Xg[2][0] - h).max() <= 1e-12 * Lz
    assert np.abs(Xg[2][-1] - Lz).max() <= 1e-12 * Lz
    # affine in zeta along each column: second differences vanish
    Z = Xg[2].reshape(shape[0], -1)
    ok = np.diff(zeta) > 0  # skip the repeated interface nodes
    slope = (Z[1:] - Z[:-1])[ok] / np.diff(zeta)[ok][:, None]
    assert np.abs(slope - slope[0]).max() <= 1e-12


@pytest.mark.parametrize("geo", CURVED)
def test_C_is_minus_kappa_B_transpose_on_curved_walls(geo):
    """With uniform kappa and slip walls the weak divergence with central
    fluxes is the negative adjoint of the weak gradient: C = -kappa B^T (cell
    integration by parts, interior face terms pair up, wall terms cancel).
    B being pinned by the linear-field test, this pins the volume metric
    terms, face normals and the sign of every term of C on curved cells."""
    m = O.make_mesh(2, 2, 1, 2, Lx=2000.0, Ly=1600.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    pk = np.full(N, 1e5)
    kappa = GAMMA * 1e5 / (GAMMA - 1)
    B = O.assemble(lambda v: O.apply_B(m, ALPHA, v), N, 3 * N)
    Cm = O.assemble(lambda v: O.apply_C(m, ALPHA, GAMMA, pk, v), 3 * N, N)
    assert np.abs(Cm + kappa * B.T).max() <= 1e-13 * kappa * np.abs(B).max()


@pytest.mark.parametrize("geo", [dict(terrain=0)] + CURVED)
def test_S_invariants(geo):
    """S 1 = D 1 (constant pressure has zero weak gradient) and
    1^T S = 1^T D (interior fluxes cancel, walls carry no normal flux) for any
    positive coefficient fields, on wall-bounded meshes."""
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=1600.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    rng = np.random.default_rng(1)
    rho = 1.2 * (1 + 0.2 * rng.random(N))
    pk = 1e5 * (1 + 0.2 * rng.random(N))
    one = np.ones(N)
    S1 = O.apply_S(m, ALPHA, GAMMA, rho, pk, one)
    D1 = O.apply_D(m, GAMMA, one)
    assert np.abs(S1 - D1).max() <= 1e-13 * np.abs(D1).max()
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v), N, N)
    assert np.abs(S.sum(axis=0) - D1).max() <= 1e-12 * np.abs(D1).max()
    # non-uniform kappa: S is not symmetric (hence GMRES, Sec. 3.1)
    assert np.abs(S - S.T).max() > 1e-6 * np.abs(S).max()


@pytest.mark.parametrize("geo", [dict(terrain=0)] + CURVED)
@pytest.mark.parametrize("r", [1, 2])
def test_S_symmetric_positive_definite_uniform(geo, r):
    """Uniform rho, p_k and slip walls: -C = kappa B^T, so
    S = D + kappa B^T A^-1 B is symmetric positive definite."""
    m = O.make_mesh(2, 2, 1, r, Lx=2000.0, Ly=1600.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    rho = np.full(N, 1.1)
    pk = np.full(N, 9e4)
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v), N, N)
    assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    D = O.assemble(lambda v: O.apply_D(m, GAMMA, v), N, N)
    # S - D = kappa B^T A^-1 B is positive semi-definite
    evd = np.linalg.eigvalsh(S - D)
    assert ev.min() > 0 and evd.min() > -1e-10 * ev.max()


def test_fast_inverse_is_tensor_product_form():
    """A^-1 = S^-T J^-1 S^-1 (Sec. 3.3) with S = S1 x S1 x S1,
    S1[a,q] = l_a(g_q) at r+1 Gauss points, J = rho(x_q) det J w_q: on an
    affine cell with random rho the oracle's dense LU inverse matches."""
    r = 3
    hx, hy, hz = 500.0, 400.0, 300.0
    m = O.make_mesh(1, 1, 1, r, Lx=hx, Ly=hy, Lz=hz)
    N = O.ndofs(m)
    n = r + 1
    xn, _ = O.gll(n)
    g, w = O.gauss(n)
    S1 = np.array([O.lagrange(xn, gq)[0] for gq in g]).T  # [a, q]
    S3 = _k3(S1, S1, S1)
    rng = np.random.default_rng(3)
    rho = 1.0 + rng.random(N)
    rho_q = S3.T @ rho
    J = rho_q * _k3(np.diag(w), np.diag(w), np.diag(w)).diagonal() * hx * hy * hz
    Si = np.linalg.inv(S3)
    Ainv = Si.T @ np.diag(1 / J) @ Si
    v = rng.standard_normal(3 * N)
    out = O.apply_Ainv(m, rho, v)
    for d in range(3):
        ref = Ainv @ v[d * N:(d + 1) * N]
        assert np.abs(out[d * N:(d + 1) * N] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fast_mass_aliasing_for_variable_density():
    """With rho of degree r > 1 the r+1 point rule is not exact for the
    triple product (Sec. 3.3): the fast A differs from the exact
    density-weighted mass, here integrated symbolically in 1D."""
    r = 2
    m = O.make_mesh(1, 1, 1, r, Lx=1.0, Ly=1.0, Lz=1.0)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rho = (1 + X[0] ** 2)  # degree 2 in x, exactly representable
    A = O.assemble(lambda v: O.apply_A(m, rho, v), 3 * N, 3 * N)[:N, :N]
    t = sp.symbols("t")
    nodes = [0, sp.Rational(1, 2), 1]
    L = []
    for a in range(3):
        e = sp.Integer(1)
        for b in range(3):
            if b != a:
                e *= (t - nodes[b]) / (nodes[a] - nodes[b])
        L.append(e)
    Mx = np.array([[float(sp.integrate((1 + t**2) * L[a] * L[b], (t, 0, 1))) for b in range(3)] for a in range(3)])
    M1 = np.array([[float(sp.integrate(L[a] * L[b], (t, 0, 1))) for b in range(3)] for a in range(3)])
    exact = _k3(Mx, M1, M1)
    err = np.abs(A - exact).max() / np.abs(exact).max()
    assert err > 1e-4  # aliasing present
    # and consistent with a 3-point Gauss rule applied to the degree-6 integrand
    g, w = O.gauss(3)
    Ma = np.array([[sum(w[k] * (1 + g[k] ** 2) * O.lagrange(np.array([0, .5, 1.]), g[k])[0][a]
                        * O.lagrange(np.array([0, .5, 1.]), g[k])[0][b] for k in range(3)) for b in range(3)] for a in range(3)])
    assert np.abs(A - _k3(Ma, M1, M1)).max() <= 1e-13 * np.abs(exact).max()
    # the consistent 2r+1 point rule integrates the degree-3r integrand exactly
    Ac = O.assemble(lambda v: O.apply_A(m, rho, v, consistent=True), 3 * N, 3 * N)[:N, :N]
    assert np.abs(Ac - exact).max() <= 1e-13 * np.abs(exact).max()


@pytest.mark.parametrize("geo", [dict(terrain=0)] + CURVED)
def test_consistent_mass_and_its_inverse(geo):
    """The consistent density-weighted mass (2r+1 points, the integration the
    fast inverse replaces, Sec. 3.3) is the mass matrix M for rho = 1 on
    curved cells, is symmetric positive definite for positive rho, and its
    inverse inverts it; the fast (r+1 point) mass differs from it on curved
    cells (aliasing of the metric) and for variable rho."""
    m = O.make_mesh(2, 1, 2, 2, Lx=2000.0, Ly=1000.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    one = np.ones(N)
    Mfull = O.assemble(lambda v: O.apply_M(m, v), N, N)
    A1 = O.assemble(lambda v: O.apply_A(m, one, v, consistent=True), 3 * N, 3 * N)
    for d in range(3):
        assert np.abs(A1[d * N:(d + 1) * N, d * N:(d + 1) * N] - Mfull).max() <= 1e-13 * np.abs(Mfull).max()
    rng = np.random.default_rng(12)
    rho = 1.2 * (1 + 0.3 * rng.random(N))
    A = O.assemble(lambda v: O.apply_A(m, rho, v, consistent=True), 3 * N, 3 * N)[:N, :N]
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max() and np.linalg.eigvalsh(A).min() > 0
    v = rng.standard_normal(3 * N)
    back = O.apply_A(m, rho, O.apply_Ainv(m, rho, v, consistent=True), consistent=True)
    assert np.abs(back - v).max() <= 1e-11 * np.abs(v).max()
    Af = O.assemble(lambda v: O.apply_A(m, rho, v), 3 * N, 3 * N)[:N, :N]
    assert np.abs(Af - A).max() > 1e-6 * np.abs(A).max()


@pytest.mark.parametrize("geo", [dict(terrain=0)] + CURVED)
def test_S_with_consistent_mass(geo):
    """With the consistent mass the Schur operator keeps its structure: S 1 =
    D 1 and 1^T S = 1^T D for random coefficients, and S is symmetric positive
    definite for uniform coefficients with slip walls."""
    m = O.make_mesh(2, 2, 1, 2, Lx=2000.0, Ly=1600.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    rng = np.random.default_rng(13)
    rho, pk = 1.2 * (1 + 0.2 * rng.random(N)), 1e5 * (1 + 0.2 * rng.random(N))
    one = np.ones(N)
    D1 = O.apply_D(m, GAMMA, one)
    assert np.abs(O.apply_S(m, ALPHA, GAMMA, rho, pk, one, consistent=True) - D1).max() <= 1e-13 * np.abs(D1).max()
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v, consistent=True), N, N)
    assert np.abs(S.sum(axis=0) - D1).max() <= 1e-12 * np.abs(D1).max()
    Su = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, np.full(N, 1.1), np.full(N, 9e4), v, consistent=True), N, N)
    assert np.abs(Su - Su.T).max() <= 1e-13 * np.abs(Su).max() and np.linalg.eigvalsh(Su).min() > 0
    b = rng.standard_normal(N)
    x, st, its, rel = O.solve(m, ALPHA, GAMMA, rho, pk, b, tol=1e-12, consistent=True)
    assert st == 0 and np.abs(x - np.linalg.solve(S, b)).max() <= 1e-9 * np.abs(x).max()


# ------------------------------------------------ convergence (MMS)
def _mms_error(m, rho, pk, pex, f, method):
    b = O.apply_M(m, f)
    x, st, its, rel = O.solve(m, ALPHA, GAMMA, rho, pk, b, method=method, tol=1e-13, maxit=4000)
    assert st == 0
    e = x - pex
    return np.sqrt(e @ O.apply_M(m, e))


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_mms_convergence_uniform(r):
    """p/(g-1) - alpha^2 h lap p = f with p = cos(pi x / L), walls (Neumann):
    central fluxes give order r+1 for even r and r for odd r."""
    L = 1000.0
    rho0, p0 = 1.2, 1e5
    h = GAMMA * p0 / ((GAMMA - 1) * rho0)
    errs = []
    for mm in [2, 4, 8]:
        m = O.make_mesh(mm, 1, 1, r, Lx=L, Ly=L, Lz=L)
        N = O.ndofs(m)
        X = O.node_coords(m)
        pex = np.cos(np.pi * X[0] / L)
        f = pex * (1 / (GAMMA - 1) + ALPHA**2 * h * (np.pi / L) ** 2)
        errs.append(_mms_error(m, np.full(N, rho0), np.full(N, p0), pex, f, "cg"))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    expect = r + 1 if r % 2 == 0 else r
    assert orders[-1] >= expect - 0.25, orders


@pytest.mark.parametrize("r", [2, 3])
def test_mms_convergence_variable_coefficients(r):
    """rho and p_k with different scale heights make S non-symmetric;
    p/(g-1) - alpha^2 div(h grad p) = f, h = g p_k/((g-1) rho), by FGMRES."""
    L, H1, H2, rho0, p0 = 1000.0, 3000.0, 1500.0, 1.2, 1e5
    errs = []
    for mm in [2, 4, 8]:
        m = O.make_mesh(mm, 1, mm, r, Lx=L, Ly=L, Lz=L)
        X = O.node_coords(m)
        x, z = X[0], X[2]
        rho = rho0 * np.exp(-z / H1)
        pk = p0 * np.exp(-z / H2)
        a = 1 / H2 - 1 / H1
        h = GAMMA * p0 / ((GAMMA - 1) * rho0) * np.exp(-a * z)
        k = np.pi / L
        pex = np.cos(k * x) * np.cos(k * z)
        f = pex / (GAMMA - 1) - ALPHA**2 * (h * (-2 * k * k * pex) + (-a * h) * (-k * np.cos(k * x) * np.sin(k * z)))
        errs.append(_mms_error(m, rho, pk, pex, f, "fgmres"))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    expect = r + 1 if r % 2 == 0 else r
    assert orders[-1] >= expect - 0.25, orders


# ------------------------------------------------------------ solvers
@pytest.mark.parametrize("geo", [dict(terrain=0, bc_lateral=0), dict(terrain=1, hc=300.0, ac=700.0, bc_lateral=1)])
def test_fgmres_matches_dense_solve(geo):
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=2000.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    rng = np.random.default_rng(5)
    rho = 1.2 * (1 + 0.2 * rng.random(N))
    pk = 1e5 * (1 + 0.2 * rng.random(N))
    b = rng.standard_normal(N)
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v), N, N)
    xref = np.linalg.solve(S, b)
    for pc in [O.PC_HELMHOLTZ, O.PC_INTERNAL_ENERGY, O.PC_NONE]:
        x, st, its, rel = O.solve(m, ALPHA, GAMMA, rho, pk, b, method="fgmres", pc=pc, tol=1e-12, restart=20)
        assert st == 0 and rel <= 1e-12
        assert np.linalg.norm(b - S @ x) <= 1.01e-12 * np.linalg.norm(b)
        assert np.abs(x - xref).max() <= 1e-9 * np.abs(xref).max()


@pytest.mark.parametrize("pc", [O.PC_NONE, O.PC_HELMHOLTZ])
@pytest.mark.parametrize("k", [3, 8])
def test_fgmres_cycle_minimises_residual_over_krylov_space(pc, k):
    """One FGMRES cycle of k steps from x = 0 with the fixed right
    preconditioner M = diag(dinv) returns the x in M K_k(S M, b) that minimises
    ||b - S x|| (Saad's minimal-residual property); the minimum is computed
    here by a dense least-squares solve on an orthonormal Krylov basis."""
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0)
    N = O.ndofs(m)
    rng = np.random.default_rng(11)
    rho = 1.2 * (1 + 0.2 * rng.random(N))
    pk = 1e5 * (1 + 0.2 * rng.random(N))
    b = rng.standard_normal(N)
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v), N, N)
    Md = np.ones(N) if pc == O.PC_NONE else 1.0 / O.precond_diag(m, pc, ALPHA, GAMMA, rho, pk)
    SM = S * Md[None, :]
    K = [b / np.linalg.norm(b)]
    for _ in range(k - 1):  # modified Gram-Schmidt, twice
        w = SM @ K[-1]
        for _ in range(2):
            for q in K:
                w = w - (q @ w) * q
        K.append(w / np.linalg.norm(w))
    Q = np.array(K).T
    y = np.linalg.lstsq(SM @ Q, b, rcond=None)[0]
    rmin = np.linalg.norm(b - SM @ Q @ y) / np.linalg.norm(b)
    x, st, its, rel = O.solve(m, ALPHA, GAMMA, rho, pk, b, method="fgmres", pc=pc, tol=1e-14, restart=k, maxit=k)
    assert st == 1 and its == k
    assert rmin < 0.9 and abs(rel - rmin) <= 1e-8 * rmin
    assert np.linalg.norm(x - Md * (Q @ y)) <= 1e-7 * np.linalg.norm(x)


def test_cg_matches_dense_solve_spd():
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=2000.0, Lz=1500.0)
    N = O.ndofs(m)
    rho = np.full(N, 1.2)
    pk = np.full(N, 1e5)
    b = np.random.default_rng(6).standard_normal(N)
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v), N, N)
    x, st, its, rel = O.solve(m, ALPHA, GAMMA, rho, pk, b, method="cg", tol=1e-12)
    assert st == 0
    assert np.abs(x - np.linalg.solve(S, b)).max() <= 1e-9 * np.abs(x).max()


def test_helmholtz_preconditioner_beats_internal_energy():
    """The Helmholtz diagonal (Sec. 3.1) accounts for the elliptic part and
    needs fewer iterations than the internal-energy (D-only) diagonal once
    alpha^2 h / dx^2 is not small."""
    m = O.make_mesh(4, 4, 4, 2, Lx=1000.0, Ly=1000.0, Lz=1000.0)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rho = 1.2 * np.exp(-X[2] / 7314.0)
    pk = 1e5 * np.exp(-X[2] / 7314.0)
    b = np.random.default_rng(7).standard_normal(N)
    a = 1.0
    _, st1, it1, _ = O.solve(m, a, GAMMA, rho, pk, b, pc=O.PC_HELMHOLTZ, tol=1e-10)
    _, st2, it2, _ = O.solve(m, a, GAMMA, rho, pk, b, pc=O.PC_INTERNAL_ENERGY, tol=1e-10)
    assert st1 == 0 and st2 == 0 and it1 < it2


def test_sampled_apply_matches_full():
    m = O.make_mesh(3, 3, 2, 2, Lx=3000.0, Ly=3000.0, Lz=1500.0, terrain=1, hc=400.0, ac=900.0, bc_lateral=1)
    N = O.ndofs(m)
    rng = np.random.default_rng(8)
    rho = 1.2 * (1 + 0.1 * rng.random(N))
    pk = 1e5 * (1 + 0.1 * rng.random(N))
    p = rng.standard_normal(N)
    y = O.apply_S(m, ALPHA, GAMMA, rho, pk, p)
    cells = [0, 4, 17]
    ys = O.apply_S(m, ALPHA, GAMMA, rho, pk, p, cells=cells)
    n3 = 27
    for c in cells:
        assert np.array_equal(ys[c * n3:(c + 1) * n3], y[c * n3:(c + 1) * n3])


@pytest.mark.parametrize("geo", [dict(terrain=0), dict(terrain=1, hc=300.0, ac=700.0)])
def test_periodic_lateral_boundaries(geo):
    """Periodic x, y (centred hill) and slip walls top and bottom: no boundary
    flux remains, so S is symmetric positive definite for uniform
    coefficients and S 1 = D 1, 1^T S = 1^T D for random coefficients."""
    m = O.make_mesh(3, 2, 2, 2, Lx=3000.0, Ly=2000.0, Lz=1500.0, bc_lateral=2, **geo)
    N = O.ndofs(m)
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, np.full(N, 1.1), np.full(N, 9e4), v), N, N)
    assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    rng = np.random.default_rng(9)
    rho, pk = 1.2 * (1 + 0.2 * rng.random(N)), 1e5 * (1 + 0.2 * rng.random(N))
    D1 = O.apply_D(m, GAMMA, np.ones(N))
    assert np.abs(O.apply_S(m, ALPHA, GAMMA, rho, pk, np.ones(N)) - D1).max() <= 1e-13 * np.abs(D1).max()
    S = O.assemble(lambda v: O.apply_S(m, ALPHA, GAMMA, rho, pk, v), N, N)
    assert np.abs(S.sum(axis=0) - D1).max() <= 1e-12 * np.abs(D1).max()
