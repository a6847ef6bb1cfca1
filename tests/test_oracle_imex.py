"""Pins of the oracle's explicit fluxes, background states and IMEX step.

The explicit tendencies are the DG weak forms of -div(rho u), -div(rho u_d u),
-div(rho k u) (+ rho g.u) with a local Lax-Friedrichs flux; the IMEX step is
the stage scheme of Sec. 2 of arXiv:2505.00384 with ARS(2,2,2).  Pins:
free-stream preservation on terrain-following cells, linear-field
reproduction, the upwind closed form of the Lax-Friedrichs flux, discrete mass
conservation, the hydrostatic background formulas of Sec. 3 (hydrostatic
balance and the buoyancy frequency by finite differences), rest-state
preservation, mass conservation and second-order temporal convergence of the
IMEX step.
"""
import numpy as np
import pytest
import sympy as sp

import oracle as O

G = 9.81


def _interior_idx(m, cells):
    n3 = (m.r + 1) ** 3
    return np.concatenate([np.arange(c * n3, (c + 1) * n3) for c in cells])


def _curved(bc_lateral=1, r=2):
    return O.make_mesh(3, 3, 3, r, Lx=3000.0, Ly=3000.0, Lz=1500.0, terrain=1, hc=300.0, ac=800.0,
                       bc_lateral=bc_lateral)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_free_stream_preserved_on_curved_cells(r):
    """Uniform rho and horizontal u (g = 0): every interior cell has zero
    tendency (the discrete metric identities hold because the Jacobian
    cofactors are polynomials integrated exactly)."""
    m = _curved(r=r)
    N = O.ndofs(m)
    bg = O.make_bg(g=0.0, ubar=10.0)
    rho = np.full(N, 1.1)
    u = np.concatenate([np.full(N, 10.0), np.full(N, 3.0), np.zeros(N)])
    Er, Em, Ee = O.explicit(m, bg, rho, u, rho)
    rng = np.random.default_rng(1)
    Er2, _, _ = O.explicit(m, bg, rho * (1 + 0.1 * rng.random(N)), u, rho)
    scale = np.abs(Er2).max()
    idx = _interior_idx(m, [13])
    assert np.abs(Er[idx]).max() <= 1e-13 * scale
    for d in range(3):
        assert np.abs(Em[d * N + idx]).max() <= 1e-13 * scale * 10.0
    assert np.abs(Ee[idx]).max() <= 1e-13 * scale * 60.0


def test_linear_density_constant_velocity():
    """Continuous linear rho, constant u: -div(rho u) = -u.grad(rho) and the
    jump terms vanish, so Erho = -M (u.grad rho); momentum and kinetic energy
    tendencies are u_d Erho and k Erho, plus the gravity work -g w M rho."""
    m = _curved(r=2)
    N = O.ndofs(m)
    X = O.node_coords(m)
    a = np.array([1e-4, -2e-4, 3e-4])
    rho = 1.0 + a[0] * X[0] + a[1] * X[1] + a[2] * X[2]
    uc = np.array([10.0, 3.0, -2.0])
    u = np.concatenate([np.full(N, uc[0]), np.full(N, uc[1]), np.full(N, uc[2])])
    bg = O.make_bg(g=G)
    Er, Em, Ee = O.explicit(m, bg, rho, u, rho)
    ref = -O.apply_M(m, np.full(N, uc @ a))
    idx = _interior_idx(m, [13])
    sc = np.abs(ref[idx]).max()
    assert np.abs(Er[idx] - ref[idx]).max() <= 1e-12 * sc
    for d in range(3):
        assert np.abs(Em[d * N + idx] - uc[d] * ref[idx]).max() <= 1e-12 * sc * 10
    k = 0.5 * uc @ uc
    grav = -G * uc[2] * O.apply_M(m, rho)
    assert np.abs(Ee[idx] - (k * ref[idx] + grav[idx])).max() <= 1e-12 * np.abs(Ee[idx]).max()


@pytest.mark.parametrize("r", [1, 2])
def test_lax_friedrichs_upwind_closed_form(r):
    """Two cells, rho = rho_L | rho_R piecewise constant, u = (U, 0, 0): the
    Lax-Friedrichs flux with lambda = |U| is the upwind flux U rho_L on the
    shared face; the mirror state gives zero flux through slip walls."""
    hx, hy, hz = 400.0, 300.0, 200.0
    m = O.make_mesh(2, 1, 1, r, Lx=2 * hx, Ly=hy, Lz=hz)
    n = r + 1
    n3 = n ** 3
    N = O.ndofs(m)
    t = sp.symbols("t")
    nodes = {1: [0, 1], 2: [0, sp.Rational(1, 2), 1]}[r]
    W = []
    for a in range(n):
        e = sp.Integer(1)
        for b in range(n):
            if b != a:
                e *= (t - nodes[b]) / (nodes[a] - nodes[b])
        W.append(float(sp.integrate(e, (t, 0, 1))))
    W = np.array(W)
    e0, en = np.eye(n)[0], np.eye(n)[n - 1]
    rL, rR, U = 1.3, 0.7, 5.0
    rho = np.concatenate([np.full(n3, rL), np.full(n3, rR)])
    u = np.concatenate([np.full(N, U), np.zeros(2 * N)])
    Er, _, _ = O.explicit(m, O.make_bg(g=0.0), rho, u, rho)
    A = hy * hz
    ref0 = -rL * U * A * np.kron(W, np.kron(W, e0))
    ref1 = rR * U * A * np.kron(W, np.kron(W, en - e0)) + U * rL * A * np.kron(W, np.kron(W, e0))
    sc = np.abs(ref1).max()
    assert np.abs(Er[:n3] - ref0).max() <= 1e-13 * sc
    assert np.abs(Er[n3:] - ref1).max() <= 1e-13 * sc


def test_mass_conservation_of_explicit_tendency():
    """Slip walls all round: interior fluxes cancel pairwise and walls carry
    no mass, so the tendencies of the continuity equation sum to zero."""
    m = _curved(bc_lateral=0)
    N = O.ndofs(m)
    rng = np.random.default_rng(2)
    rho = 1.0 + 0.1 * rng.random(N)
    u = rng.standard_normal(3 * N)
    Er, _, _ = O.explicit(m, O.make_bg(g=G), rho, u, rho)
    assert abs(Er.sum()) <= 1e-13 * np.abs(Er).max() * N ** 0.5


@pytest.mark.parametrize("kind", [0, 1])
def test_background_states(kind):
    """Isothermal: p = p0 exp(-g z/(R T)), rho = p/(R T).  Constant-N state
    of Sec. 3: p(0) = p_ref, rho(0) = p_ref/(R T_ref), hydrostatic dp/dz = -rho g
    and buoyancy frequency g d(ln theta)/dz = N^2 (finite differences)."""
    bg = O.make_bg(kind=kind, T=293.15 if kind else 250.0, p0=1e5, Nbv=0.01, R=287.0, gamma=1.4, g=G)
    m = O.make_mesh(1, 1, 40, 1, Lx=100.0, Ly=100.0, Lz=16000.0)
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    z = X[2]
    if kind == 0:
        assert np.allclose(pb, 1e5 * np.exp(-G * z / (287.0 * 250.0)), rtol=1e-14)
        assert np.allclose(rb, pb / (287.0 * 250.0), rtol=1e-14)
        return
    o = np.argsort(z, kind="stable")
    zs, ps, rs = z[o], pb[o], rb[o]
    keep = np.concatenate([[True], np.diff(zs) > 1e-9])
    zs, ps, rs = zs[keep], ps[keep], rs[keep]
    assert abs(ps[0] - 1e5) < 1e-9 and abs(rs[0] - 1e5 / (287.0 * 293.15)) < 1e-12
    # central differences on the (uniform) node column
    dz = np.diff(zs)
    dpdz = (ps[2:] - ps[:-2]) / (zs[2:] - zs[:-2])
    assert np.abs(dpdz + rs[1:-1] * G).max() <= 2e-4 * np.abs(rs * G).max()
    theta = ps / (rs * 287.0) * (1e5 / ps) ** (0.4 / 1.4)
    n2 = G * (np.log(theta[2:]) - np.log(theta[:-2])) / (zs[2:] - zs[:-2])
    assert np.abs(n2 - 1e-4).max() <= 1e-6
    assert dz.min() > 0


@pytest.mark.parametrize("kind", [0, 1])
def test_hydrostatic_rest_is_preserved(kind):
    """u = 0, p = p_bar, rho = rho_bar: all perturbations vanish, so one IMEX
    step leaves the state unchanged (the background pair -grad p_bar +
    rho_bar g is removed analytically)."""
    bg = O.make_bg(kind=kind, T=293.15 if kind else 250.0, g=G)
    m = _curved(bc_lateral=0)
    N = O.ndofs(m)
    rb, pb = O.background(m, bg)
    r, u, p, st, its = O.imex_step(m, bg, rb, np.zeros(3 * N), pb, 1.0)
    assert st == 0 and np.array_equal(r, rb) and np.array_equal(p, pb) and np.abs(u).max() == 0.0


def test_imex_step_conserves_mass_with_walls():
    bg = O.make_bg(g=G)
    m = O.make_mesh(3, 2, 2, 2, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=800.0)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    p = pb + 30.0 * np.exp(-((X[0] - 1500) ** 2 + (X[2] - 700) ** 2) / (2 * 300.0 ** 2))
    u = np.concatenate([2.0 * np.sin(np.pi * X[0] / 3000.0), np.zeros(N), np.zeros(N)])
    ones = np.ones(N)

    def mass(r):
        return O.apply_A(m, ones, np.concatenate([r, 0 * r, 0 * r]))[:N].sum()

    m0 = mass(rb)
    r, u2, p2, st, its = O.imex_step(m, bg, rb, u, p, 1.0)
    assert st == 0
    assert abs(mass(r) - m0) <= 1e-13 * m0
    assert np.abs(r - rb).max() > 0  # the flow did move mass around


@pytest.mark.slow
def test_imex_second_order_in_time():
    """Smooth pressure pulse in a wall-bounded isothermal atmosphere, ARS(2,2,2)
    with two fixed-point iterations: errors against a dt/8 reference halve
    twice per halving of dt (second order)."""
    bg = O.make_bg(g=G, ubar=0.0)
    m = O.make_mesh(4, 1, 4, 2, Lx=2000.0, Ly=500.0, Lz=2000.0)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    p0 = pb + 50.0 * np.exp(-((X[0] - 1000) ** 2 + (X[2] - 1000) ** 2) / (2 * 300.0 ** 2))

    def run(dt, T=0.5):
        r, u, p = rb.copy(), np.zeros(3 * N), p0.copy()
        for _ in range(int(round(T / dt))):
            r, u, p, st, _ = O.imex_step(m, bg, r, u, p, dt, K=2, tol=1e-13)
            assert st == 0
        return p, u

    pref, uref = run(1.0 / 128)
    e = []
    for dt in (0.0625, 0.03125):
        p, u = run(dt)
        e.append(np.abs(p - pref).max())
    order = np.log2(e[0] / e[1])
    assert order >= 1.8, (e, order)


def test_periodic_uniform_wind_is_steady():
    """Flat periodic domain, hydrostatic background and a uniform horizontal
    wind: an exact steady state; the explicit tendencies vanish and an IMEX
    step leaves the state unchanged to roundoff."""
    bg = O.make_bg(g=G, ubar=10.0)
    m = O.make_mesh(3, 2, 3, 3, Lx=3000.0, Ly=2000.0, Lz=1500.0, bc_lateral=2)
    N = O.ndofs(m)
    rb, pb = O.background(m, bg)
    u = np.concatenate([np.full(N, 10.0), np.full(N, -4.0), np.zeros(N)])
    Er, Em, Ee = O.explicit(m, bg, rb, u, rb)
    rng = np.random.default_rng(3)
    sc = np.abs(O.explicit(m, bg, rb * (1 + 0.01 * rng.random(N)), u, rb)[0]).max()
    assert np.abs(Er).max() <= 1e-12 * sc and np.abs(Em).max() <= 1e-12 * sc * 10 and np.abs(Ee).max() <= 1e-12 * sc * 60
    r, u2, p, st, _ = O.imex_step(m, bg, rb, u, pb, 1.0)
    assert st == 0
    assert np.abs(r - rb).max() <= 1e-12 * rb.max()
    assert np.abs(u2 - u).max() <= 1e-10 * 10.0
    assert np.abs(p - pb).max() <= 1e-10 * pb.max()


def test_periodic_mass_conservation():
    bg = O.make_bg(g=G, ubar=10.0)
    m = O.make_mesh(3, 2, 2, 2, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=200.0, ac=800.0, bc_lateral=2)
    N = O.ndofs(m)
    rb, pb = O.background(m, bg)
    u = np.concatenate([np.full(N, 10.0), np.zeros(N), np.zeros(N)])
    ones = np.ones(N)
    mass = lambda r: O.apply_A(m, ones, np.concatenate([r, 0 * r, 0 * r]))[:N].sum()
    r, _, _, st, _ = O.imex_step(m, bg, rb, u, pb, 1.0)
    assert st == 0 and abs(mass(r) - mass(rb)) <= 1e-13 * mass(rb) and np.abs(r - rb).max() > 0


def test_acoustic_standing_wave_closed_form():
    """Linear acoustics (g = 0, uniform isothermal state, periodic in x):
    p' = eps cos(k x) cos(w t), u = eps/(rho0 c) sin(k x) sin(w t) with
    c^2 = gamma p0 / rho0 is the exact solution of the linearised equations
    (rho0 u_t = -p'_x, p'_t = -gamma p0 u_x from the energy equation with
    rho E = p/(gamma-1) + rho k).  The IMEX step converges to it at second
    order in dt; a wrong enthalpy factor kappa, a flipped pressure-gradient or
    enthalpy-flux sign, or a wrong velocity recovery changes the wave speed or
    makes the wave grow."""
    R, T, gam, p0 = 287.0, 250.0, 1.4, 1e5
    bg = O.make_bg(kind=0, T=T, p0=p0, R=R, gamma=gam, g=0.0, ubar=0.0)
    Lx, nx = 1000.0, 16
    m = O.make_mesh(nx, 1, 1, 3, Lx=Lx, Ly=Lx / nx, Lz=Lx / nx, bc_lateral=2)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    rho0 = p0 / (R * T)
    assert np.allclose(rb, rho0, rtol=1e-15) and np.allclose(pb, p0, rtol=1e-15)
    c = np.sqrt(gam * p0 / rho0)
    k = 2 * np.pi / Lx
    w = c * k
    eps, t_end = 1.0, 0.8
    ua = eps / (rho0 * c)

    def errors(dt):
        r, u, p = rb.copy(), np.zeros(3 * N), pb + eps * np.cos(k * X[0])
        n = int(round(t_end / dt))
        for _ in range(n):
            r, u, p, st, _ = O.imex_step(m, bg, r, u, p, dt, K=2, tol=1e-12)
            assert st == 0
        t = n * dt
        ep = np.abs((p - pb) - eps * np.cos(k * X[0]) * np.cos(w * t)).max() / eps
        eu = np.abs(u[:N] - ua * np.sin(k * X[0]) * np.sin(w * t)).max() / ua
        eyz = np.abs(u[N:]).max() / ua
        return ep, eu, eyz

    e1, e2 = errors(0.1), errors(0.05)  # w dt = 0.20 and 0.10
    assert e1[0] < 4e-3 and e2[0] < 1e-3, (e1, e2)
    assert e1[0] / e2[0] > 3.5, (e1, e2)  # second order towards the closed form
    assert e1[1] < 1e-3 and e2[1] < 1e-3, (e1, e2)
    assert e1[2] < 1e-8 and e2[2] < 1e-8, (e1, e2)


@pytest.mark.parametrize("consistent", [False, True])
def test_buoyancy_initial_acceleration(consistent):
    """A density anomaly rho' at rest with p' = 0 accelerates vertically at
    w_t = -g rho' / rho and not horizontally: after one short step,
    w = -g rho'/rho dt up to the projection of the weak buoyancy term and
    O(dt^2) (the pressure answers the compression at second order).  Holds
    with the fast and with the consistent density-weighted mass."""
    bg = O.make_bg(kind=0, T=250.0, g=G, ubar=0.0)
    m = O.make_mesh(4, 1, 4, 2, Lx=2000.0, Ly=500.0, Lz=2000.0, bc_lateral=2)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    delta = 1e-3 * np.exp(-((X[0] - 1000) ** 2 + (X[2] - 1000) ** 2) / (2 * 300.0 ** 2))
    dt = 0.01
    _, u, _, st, _ = O.imex_step(m, bg, rb * (1 + delta), np.zeros(3 * N), pb, dt, consistent=consistent)
    assert st == 0
    wref = -G * delta / (1 + delta) * dt
    sc = np.abs(wref).max()
    assert np.abs(u[2 * N:] - wref).max() <= 5e-3 * sc
    assert np.abs(u[:N]).max() <= 1e-4 * sc and np.abs(u[N:2 * N]).max() <= 1e-12 * sc


def test_fast_and_consistent_mass_agree():
    """Sec. 3.3: the fast inverse (r+1 point rule for every density-weighted
    mass) changes the solution of the hill flow only by its aliasing error:
    after two steps the vertical velocities of the fast and the consistent
    variants agree to a small fraction of the flow's own w, and differ."""
    bg = O.make_bg(g=G, ubar=10.0)
    m = O.make_mesh(4, 2, 3, 3, Lx=4000.0, Ly=2000.0, Lz=3000.0, terrain=1, hc=300.0, ac=800.0, bc_lateral=2)
    N = O.ndofs(m)
    rb, pb = O.background(m, bg)
    u0 = np.concatenate([np.full(N, 10.0), np.zeros(2 * N)])
    out = []
    for consistent in (False, True):
        r, u, p = rb.copy(), u0.copy(), pb.copy()
        for _ in range(2):
            r, u, p, st, _ = O.imex_step(m, bg, r, u, p, 1.0, consistent=consistent)
            assert st == 0
        out.append(u[2 * N:])
    wmax = np.abs(out[0]).max()
    diff = np.abs(out[0] - out[1]).max()
    assert wmax > 0.1 and 0 < diff <= 0.01 * wmax, (wmax, diff)  # measured 1.8e-3


def test_explicit_momentum_and_energy_budgets():
    """Periodic lateral faces and flat slip walls, random rho and u: the
    interior Lax-Friedrichs fluxes cancel pairwise and the mirror state at a
    horizontal wall carries vertical momentum only, so the x and y momentum
    tendencies sum to zero; the kinetic-energy tendencies sum to the gravity
    work -g int rho w (no energy crosses the walls).  On a curved bottom the
    wall flux has horizontal components, so the check uses a flat mesh."""
    m = O.make_mesh(3, 3, 3, 2, Lx=3000.0, Ly=3000.0, Lz=1500.0, bc_lateral=2)
    N = O.ndofs(m)
    rng = np.random.default_rng(14)
    rho = 1.0 + 0.1 * rng.random(N)
    u = rng.standard_normal(3 * N)
    Er, Em, Ee = O.explicit(m, O.make_bg(g=G), rho, u, rho)
    sc = np.abs(Em).max()
    assert abs(Em[:N].sum()) <= 1e-13 * sc * N ** 0.5 and abs(Em[N:2 * N].sum()) <= 1e-13 * sc * N ** 0.5
    assert abs(Em[2 * N:].sum()) > 1e-3 * sc  # the walls do act on vertical momentum
    # int rho w with the consistent rule (exact for the degree-3r integrand)
    rw = O.apply_A(m, rho, np.concatenate([u[2 * N:], np.zeros(2 * N)]), consistent=True)[:N].sum()
    assert abs(Ee.sum() + G * rw) <= 1e-13 * np.abs(Ee).max() * N ** 0.5


def test_far_field_free_stream():
    """Uniform density rho_bar and wind (u_bar, 0, 0) equal to the far-field
    ghost state, g = 0, far-field lateral faces and flat walls: every cell's
    tendencies vanish, the boundary cells included."""
    bg = O.make_bg(g=0.0, ubar=10.0)
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=2000.0, Lz=1500.0, bc_lateral=1)
    N = O.ndofs(m)
    rho = np.full(N, 1.1)
    u = np.concatenate([np.full(N, 10.0), np.zeros(2 * N)])
    Er, Em, Ee = O.explicit(m, bg, rho, u, rho)
    sc = np.abs(O.explicit(m, bg, rho * (1 + 0.01 * np.random.default_rng(15).random(N)), u, rho)[0]).max()
    assert np.abs(Er).max() <= 1e-12 * sc and np.abs(Em).max() <= 1e-11 * sc and np.abs(Ee).max() <= 1e-10 * sc


def test_far_field_inflow_mass_budget():
    """Uniform rho = 1.1 and wind (u_bar, 0, 0) against a far-field density
    rho_bar = 1.0 (g = 0, flat walls): the Lax-Friedrichs flux at the far-field
    faces is the upwind flux, so the inflow face brings rho_bar and the outflow
    face takes rho; the continuity tendencies sum to -(rho - rho_bar) u_bar Ly Lz."""
    bg = O.make_bg(g=0.0, ubar=10.0)
    Ly, Lz = 1600.0, 1500.0
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=Ly, Lz=Lz, bc_lateral=1)
    N = O.ndofs(m)
    u = np.concatenate([np.full(N, 10.0), np.zeros(2 * N)])
    Er, _, _ = O.explicit(m, bg, np.full(N, 1.1), u, np.full(N, 1.0))
    ref = -(1.1 - 1.0) * 10.0 * Ly * Lz
    assert abs(Er.sum() - ref) <= 1e-12 * abs(ref) * N ** 0.5


def test_imex_euler_acoustics_closed_form():
    """The IMEX Euler pair (explicit stage, then one implicit stage: A =
    [[0, 0], [1, 0]], A~ = [[0, 0], [0, 1]]) is backward Euler for linear
    acoustics: each step multiplies the mode (p', i rho0 c u) by
    g = 1 / (1 - i w dt), so after n steps p' = eps cos(kx) Re(g^n) and
    u = eps/(rho0 c) sin(kx) Im(g^n).  Pins the stage machinery with a
    tableau other than ARS(2,2,2)."""
    R, T, gam, p0 = 287.0, 250.0, 1.4, 1e5
    bg = O.make_bg(kind=0, T=T, p0=p0, R=R, gamma=gam, g=0.0, ubar=0.0)
    Lx, nx = 1000.0, 16
    m = O.make_mesh(nx, 1, 1, 3, Lx=Lx, Ly=Lx / nx, Lz=Lx / nx, bc_lateral=2)
    N = O.ndofs(m)
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    rho0 = p0 / (R * T)
    c = np.sqrt(gam * p0 / rho0)
    k = 2 * np.pi / Lx
    wdt, n = 0.5, 4
    A = np.array([[0.0, 0.0], [1.0, 0.0]])
    At = np.array([[0.0, 0.0], [0.0, 1.0]])
    r, u, p = rb.copy(), np.zeros(3 * N), pb + np.cos(k * X[0])
    for _ in range(n):
        r, u, p, st, _ = O.imex_step(m, bg, r, u, p, wdt / (c * k), A=A, At=At, K=2, tol=1e-12)
        assert st == 0
    gn = (1.0 / (1.0 - 1j * wdt)) ** n
    assert np.abs((p - pb) - gn.real * np.cos(k * X[0])).max() <= 2e-4
    assert np.abs(u[:N] * rho0 * c - gn.imag * np.sin(k * X[0])).max() <= 2e-4
    assert np.abs(u[N:]).max() * rho0 * c <= 1e-8


@pytest.mark.parametrize("geo", [dict(terrain=0), dict(terrain=1, hc=300.0, ac=800.0)])
def test_kinetic_mass_closed_form(geo):
    """int rho |u|^2/2 psi_i for constant rho and u = (x, y, 0): the
    integrand rho (x^2 + y^2)/2 is the degree-2 polynomial the r = 2 nodal
    basis holds exactly, so the result is rho/2 M (x^2 + y^2) with M the
    (pinned) consistent mass, on flat and terrain-following cells."""
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=1600.0, Lz=1500.0, **geo)
    N = O.ndofs(m)
    X = O.node_coords(m)
    u = np.concatenate([X[0], X[1], np.zeros(N)])
    out = O.kinetic_mass(m, np.full(N, 1.3), u)
    ref = O.apply_M(m, 0.65 * (X[0] ** 2 + X[1] ** 2))
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()
