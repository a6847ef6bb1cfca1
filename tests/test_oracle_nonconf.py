"""Pins of the oracle on non-conforming meshes (2:1 hanging faces).

The paper runs its hill case on a non-conforming mesh whose neighbouring
cells differ in resolution horizontally and vertically (Sec. 3), and reports
the Helmholtz preconditioner's largest gain there (Sec. 3.1).  The oracle's
non-conforming meshes split the base cells of a box 2 x 2 x 2; a child's map
is its parent's isoparametric map restricted to it, and the face terms on a
hanging face are integrated with the children's face rule on both sides.
Each pin ties that to a property the formulation fixes:

* the cells partition the domain (volume of the conforming base mesh);
* face relations are mutual (a base cell's four children see it back at the
  positions it lists);
* B reproduces the gradient of linear fields exactly (p_hat = p on every
  hanging point, watertight geometry), so S 1 = D 1 on walls;
* C = -kappa B^T for uniform kappa on walls (adjointness across hanging
  faces), and 1^T S = 1^T D (the hanging fluxes cancel);
* refining every base cell gives the conforming fine mesh's operator and
  explicit tendencies exactly (the child block's numbering and neighbours);
* the explicit fluxes preserve a free stream, conserve mass across hanging
  faces and upwind there (closed form for a density jump);
* the weak gradient converges at order r on refined non-conforming meshes.
"""
import numpy as np
import pytest

import oracle as O

GAMMA = 1.4
ALPHA = 0.3
HILL = dict(terrain=1, hc=200.0, ac=400.0, xc=380.0, yc=610.0)  # off-centre: no symmetry between children


def _mesh(nb=4, r=2, bc=0, geo=HILL, box=None, nz=3):
    box = box or (1, 3, 1, 3, 0, 2)
    return O.make_mesh(nb, nb, nz, r, bc_lateral=bc, refine=box, **geo)


def test_numbering_and_dead_cells():
    m = _mesh()
    assert O.num_cells(m) == 4 * 4 * 3 + 8 * 2 * 2 * 2
    dead = O.dead_cells(m)
    assert sorted(dead) == sorted(x + 4 * (y + 4 * z) for z in (0, 1) for y in (1, 2) for x in (1, 2))
    assert O.active_mask(m).sum() == (O.num_cells(m) - 8) * 27
    for c in dead:
        assert O.face_info(m, int(c), 0)[0] == 3


def test_face_relations_are_mutual():
    m = _mesh()
    counts = {-1: 0, 0: 0, 1: 0, 2: 0, 3: 0}
    for c in range(O.num_cells(m)):
        for f in range(6):
            rel, nb = O.face_info(m, c, f)
            counts[rel] += 1
            if rel == 0:
                assert O.face_info(m, nb[0], f ^ 1) == (0, [c] + O.face_info(m, nb[0], f ^ 1)[1][1:])
            elif rel == 1:
                for s in range(4):
                    r2, nb2 = O.face_info(m, nb[s], f ^ 1)
                    assert r2 == 2 and nb2[0] == c and nb2[1] == s
    # box 2 x 2 x 2 base cells on the bottom: 4 side faces of 2 x 2 base faces + the top 2 x 2
    assert counts[1] == 4 * 4 + 4 and counts[2] == 4 * counts[1]


@pytest.mark.parametrize("geo", [dict(terrain=0), HILL, dict(terrain=2, hc=150.0, ac=300.0, xc=420.0, yc=300.0)])
def test_cells_partition_the_domain(geo):
    """The children's maps restrict their parents' maps, so the volume of a
    refined mesh is the base mesh's to rounding."""
    m = _mesh(geo=geo)
    base = O.make_mesh(4, 4, 3, 2, **geo)
    vol = O.apply_M(m, O.active_mask(m).astype(float)).sum()
    vb = O.apply_M(base, np.ones(O.ndofs(base))).sum()
    assert abs(vol / vb - 1) <= 1e-14


@pytest.mark.parametrize("r", [1, 2, 3])
def test_B_reproduces_gradient_of_linear_fields(r):
    """p = a.x + c (exact in every cell, coarse or fine): B p = alpha a_d M 1
    on slip walls; in particular B 1 = 0, so S 1 = D 1."""
    m = _mesh(r=r)
    X = O.node_coords(m)
    act = O.active_mask(m)
    a = np.array([0.3, -0.7, 1.1])
    p = (a @ X + 5.0) * act
    Bp = O.apply_B(m, ALPHA, p).reshape(3, -1)
    M1 = O.apply_M(m, act.astype(float))
    for d in range(3):
        assert np.abs(Bp[d] - ALPHA * a[d] * M1).max() <= 1e-13 * np.abs(M1).max()
    rng = np.random.default_rng(3)
    N = O.ndofs(m)
    rho = (1.2 + 0.2 * rng.random(N)) * act + (1 - act)
    pk = (1e5 * (1 + 0.2 * rng.random(N))) * act
    S1 = O.apply_S(m, ALPHA, GAMMA, rho, pk, act.astype(float))
    D1 = O.apply_D(m, GAMMA, act.astype(float))
    assert np.abs(S1 - D1).max() <= 1e-12 * np.abs(D1).max()
    assert np.all(S1[~act] == 0)


def test_C_is_minus_kappa_B_transpose_across_hanging_faces():
    m = O.make_mesh(2, 2, 2, 2, Lx=2000.0, Ly=1600.0, Lz=1500.0, bc_lateral=0, refine=(0, 1, 0, 1, 0, 1), **HILL)
    N = O.ndofs(m)
    act = O.active_mask(m)
    pk = np.full(N, 1e5)
    kappa = GAMMA * 1e5 / (GAMMA - 1)
    B = O.assemble(lambda v: O.apply_B(m, ALPHA, v), N, 3 * N)
    Cm = O.assemble(lambda v: O.apply_C(m, ALPHA, GAMMA, pk, v), 3 * N, N)
    a3 = np.tile(act, 3)
    B, Cm = B[np.ix_(a3, act)], Cm[np.ix_(act, a3)]
    assert np.abs(Cm + kappa * B.T).max() <= 1e-13 * kappa * np.abs(B).max()


def test_hanging_fluxes_cancel():
    """1^T C V = 0 for any V, pk on walls, hence 1^T S = 1^T D."""
    m = _mesh(r=2)
    N = O.ndofs(m)
    act = O.active_mask(m)
    rng = np.random.default_rng(4)
    V = rng.standard_normal(3 * N) * np.tile(act, 3)
    pk = (1e5 + 1e3 * rng.standard_normal(N)) * act
    CV = O.apply_C(m, ALPHA, GAMMA, pk, V)
    assert abs(CV.sum()) <= 1e-14 * np.abs(CV).sum()
    rho = (1.2 + 0.2 * rng.random(N)) * act + (1 - act)
    p = rng.standard_normal(N) * act
    S = O.apply_S(m, ALPHA, GAMMA, rho, pk, p)
    D = O.apply_D(m, GAMMA, p)
    assert abs(S.sum() - D.sum()) <= 1e-12 * np.abs(D).sum()


def test_fully_refined_mesh_is_the_conforming_fine_mesh():
    """Box = the whole (flat) domain: every base cell is dead and the children
    form the conforming 2nx x 2ny x 2nz mesh, cell for cell."""
    nb, r = 2, 2
    m = O.make_mesh(nb, nb, nb, r, bc_lateral=1, refine=(0, nb, 0, nb, 0, nb))
    f = O.make_mesh(2 * nb, 2 * nb, 2 * nb, r, bc_lateral=1)
    n3 = (r + 1) ** 3
    off = nb ** 3 * n3
    N, Nf = O.ndofs(m), O.ndofs(f)
    assert N == off + Nf
    rng = np.random.default_rng(5)
    pf = rng.standard_normal(Nf)
    rhof = 1.2 + 0.2 * rng.random(Nf)
    pkf = 1e5 * (1 + 0.2 * rng.random(Nf))
    ext = lambda v, fill=0.0: np.concatenate([np.full(off, fill), v])
    Sf = O.apply_S(f, ALPHA, GAMMA, rhof, pkf, pf)
    Sm = O.apply_S(m, ALPHA, GAMMA, ext(rhof, 1.0), ext(pkf, 1.0), ext(pf))
    assert np.all(Sm[:off] == 0)
    assert np.abs(Sm[off:] - Sf).max() <= 1e-13 * np.abs(Sf).max()
    bg = O.make_bg(ubar=7.0)
    uf = rng.standard_normal(3 * Nf)
    rbf = 1.1 + 0.1 * rng.random(Nf)
    Ef = O.explicit(f, bg, rhof, uf, rbf)
    um = np.concatenate([ext(uf[d * Nf:(d + 1) * Nf]) for d in range(3)])
    Em = O.explicit(m, bg, ext(rhof), um, ext(rbf))
    for a, b, k in zip(Em, Ef, (1, 3, 1)):
        a = a.reshape(k, -1)[:, off:].reshape(-1)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_explicit_free_stream():
    """Uniform density and wind, no gravity, far-field lateral faces carrying
    the same wind: zero tendencies in every cell off the terrain-following
    bottom (where the mirror state turns the wind)."""
    m = _mesh(bc=1)
    bg = O.make_bg(g=0.0, ubar=10.0)
    act = O.active_mask(m)
    rho = 1.2 * act
    u = np.concatenate([10.0 * act, 0 * act, 0 * act])
    Er, Em, Ee = O.explicit(m, bg, rho, u, rho.copy())
    keep = np.repeat([O.face_info(m, c, 4)[0] != -1 for c in range(O.num_cells(m))], 27)
    sc = 1.2 * 10.0 * np.abs(O.apply_M(m, act.astype(float))).max()
    assert np.abs(Er[keep]).max() <= 1e-13 * sc
    assert np.abs(Em.reshape(3, -1)[:, keep]).max() <= 1e-13 * sc * 10
    assert np.abs(Ee[keep]).max() <= 1e-13 * sc * 100
    assert np.abs(Er[~keep & act]).max() > 1e-6 * sc  # the bottom does turn the wind


def test_explicit_mass_conservation_across_hanging_faces():
    """Slip walls everywhere: the mass tendency sums to zero for any state."""
    m = _mesh(bc=0)
    N = O.ndofs(m)
    act = O.active_mask(m)
    rng = np.random.default_rng(6)
    rho = (1.0 + 0.3 * rng.random(N)) * act
    u = rng.standard_normal(3 * N) * np.tile(act, 3)
    Er, _, _ = O.explicit(m, O.make_bg(), rho, u, rho.copy())
    assert abs(Er.sum()) <= 1e-14 * np.abs(Er).sum()


def test_explicit_upwinds_a_density_jump_across_hanging_faces():
    """Flat mesh, walls, density 1 on base cells and 2 on children, wind
    (U, 0, 0): the volume term of sum_i Erho_i vanishes, and each interior
    x face carries the upwind density times U times its area, so a cell's
    sum is -U (rho_up,right A_right - rho_up,left A_left) (walls: zero)."""
    m = O.make_mesh(4, 4, 2, 2, Lx=4000.0, Ly=4000.0, Lz=2000.0, bc_lateral=0, refine=(1, 3, 1, 3, 0, 1))
    n3, U = 27, 3.0
    nc = O.num_cells(m)
    fine = np.arange(nc) >= 32
    act = O.active_mask(m)
    rho = np.repeat(np.where(fine, 2.0, 1.0), n3) * act
    u = np.concatenate([U * act, 0 * act, 0 * act])
    Er, _, _ = O.explicit(m, O.make_bg(g=0.0), rho, u, rho.copy())
    sums = Er.reshape(nc, n3).sum(axis=1)
    A = lambda c: (1000.0 if c < 32 else 500.0) * (1000.0 if c < 32 else 500.0)
    for c in range(nc):
        rel, _ = O.face_info(m, c, 0)
        if rel == 3:
            continue
        own = 2.0 if fine[c] else 1.0
        # x- face: inflow; the upwind density is the left neighbour's
        rl, nl = O.face_info(m, c, 0)
        inflow = 0.0
        if rl == 0:
            inflow = (2.0 if fine[nl[0]] else 1.0) * A(c)
        elif rl == 1:
            inflow = 2.0 * A(c)
        elif rl == 2:
            inflow = 1.0 * A(c)
        rr, _ = O.face_info(m, c, 1)
        outflow = own * A(c) if rr != -1 else 0.0
        assert abs(sums[c] + U * (outflow - inflow)) <= 1e-12 * U * 2e6, c


@pytest.mark.parametrize("r", [2, 3])
def test_weak_gradient_converges_at_order_r(r):
    """||A^-1 B p - grad p|| on a curved non-conforming mesh and on its
    uniform refinement (base mesh and box doubled): observed order >= r - 0.1."""
    def err(nb):
        m = O.make_mesh(nb, nb, nb, r, terrain=1, hc=150.0, ac=400.0, bc_lateral=0,
                        refine=(nb // 4, 3 * nb // 4, nb // 4, 3 * nb // 4, 0, nb // 2))
        X = O.node_coords(m)
        act = O.active_mask(m)
        k = 2 * np.pi / 1000.0
        p = np.sin(k * X[0]) * np.cos(k * X[1]) * np.cos(0.5 * k * X[2]) * act
        g = np.stack([k * np.cos(k * X[0]) * np.cos(k * X[1]) * np.cos(0.5 * k * X[2]),
                      -k * np.sin(k * X[0]) * np.sin(k * X[1]) * np.cos(0.5 * k * X[2]),
                      -0.5 * k * np.sin(k * X[0]) * np.cos(k * X[1]) * np.sin(0.5 * k * X[2])]) * act
        rho = act + (1.0 - act)
        e = O.apply_Ainv(m, rho, O.apply_B(m, 1.0, p)).reshape(3, -1) - g
        return np.sqrt(sum((e[d] * O.apply_M(m, e[d])).sum() for d in range(3)))
    e1, e2 = err(4), err(8)
    assert np.log2(e1 / e2) >= r - 0.1


def test_imex_step_conserves_mass_across_hanging_faces():
    """One IMEX step on a wall-bounded non-conforming hill mesh: the continuity
    update rho^(l) = rho^n + M^-1 dt sum a Erho (fast mass) keeps the total mass
    1^T M rho exactly, because the mass tendency sums to zero over the cells
    (hanging fluxes cancel, walls carry none); dead cells keep the state given."""
    m = _mesh(bc=0)
    act = O.active_mask(m)
    bg = O.make_bg(ubar=0.0)
    rb, pb = O.background(m, bg)
    X = O.node_coords(m)
    bump = np.exp(-((X[0] - 380.0) ** 2 + (X[2] - 300.0) ** 2) / (2 * 200.0 ** 2)) * act
    rho = rb * (1.0 + 0.01 * bump)
    p = pb + 80.0 * bump
    u = np.concatenate([3.0 * bump, -2.0 * bump, 1.0 * bump])
    ones = np.ones(O.ndofs(m))
    mass = lambda r: O.apply_A(m, ones, np.concatenate([r, 0 * r, 0 * r]))[:O.ndofs(m)].sum()
    r1, u1, p1, st, _ = O.imex_step(m, bg, rho, u, p, 1.0, K=2, tol=1e-12)
    assert st == 0
    assert abs(mass(r1) - mass(rho)) <= 1e-13 * abs(mass(rho))
    assert np.abs(r1 - rho).max() > 1e-9 * np.abs(rho).max()  # the step did move the density
    assert np.all(r1[~act] == rho[~act]) and np.all(u1[np.tile(~act, 3)] == u[np.tile(~act, 3)])
