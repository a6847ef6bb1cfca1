"""Parity of the CUDA library on non-conforming meshes (2:1 hanging faces)
with the oracle, through the C ABI.

Non-conforming meshes (Sec. 3) split a box of base cells 2 x 2 x 2; the
per-patch kernels skip the faces between the children and the base cells and
the hanging-face kernels add their terms.  Bars as on conforming meshes: FP64
results within 1e-12 of the oracle (max-norm relative), FP32 within 2e-5,
explicit tendencies 1e-12; every launch variant of the operator is checked;
solves agree with the oracle's solution to the solve tolerance; dead cells
(base cells replaced by their children) read and write exact zeros.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import GAMMA, Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 0.29289321881345254
G, UBAR = 9.81, 10.0

MESHES = [
    dict(nx=4, ny=4, nz=3, r=2, Lx=4000.0, Ly=4000.0, Lz=3000.0, terrain=1, hc=300.0, ac=900.0, xc=1700.0,
         yc=2300.0, refine=(1, 3, 1, 3, 0, 2)),
    dict(nx=4, ny=3, nz=3, r=3, Lx=4000.0, Ly=3000.0, Lz=3000.0, terrain=2, hc=250.0, ac=800.0, bc_lateral=1,
         refine=(0, 2, 1, 2, 1, 3)),
    dict(nx=5, ny=3, nz=2, r=4, Lx=5000.0, Ly=3000.0, Lz=2000.0, terrain=1, hc=300.0, ac=900.0, bc_lateral=1,
         refine=(2, 4, 1, 3, 0, 1)),
    dict(nx=5, ny=4, nz=3, r=2, Lx=5000.0, Ly=4000.0, Lz=3000.0, bc_lateral=2, refine=(1, 3, 1, 3, 1, 2)),
    dict(nx=3, ny=3, nz=2, r=5, Lx=3000.0, Ly=3000.0, Lz=2000.0, terrain=1, hc=200.0, ac=800.0,
         refine=(1, 2, 1, 2, 0, 1)),
]


def _ids(m):
    return "%dx%dx%d_r%d_t%d_bc%d_box%s" % (m["nx"], m["ny"], m["nz"], m["r"], m.get("terrain", 0),
                                            m.get("bc_lateral", 0), "".join(map(str, m["refine"])))


@pytest.fixture(params=MESHES, ids=[_ids(m) for m in MESHES])
def case(request):
    c = Case(**request.param)
    c.act = O.active_mask(c.m)
    rho, pk = c.random_coefficients(seed=17)
    # dead cells hold no unknowns: the oracle never reads them; the library sets its own copies to 1
    rho, pk = rho * c.act, pk * c.act
    c.set_coefficients(rho, pk, A_DT)
    c.rho, c.pk = rho, pk
    yield c
    c.close()


def _field(c, seed, n=1, scale=1.0):
    return inputs.random_field(n * c.N, seed, scale=scale) * np.tile(c.act, n)


def test_layout_and_node_coords(case):
    import torch
    assert case.N == O.ndofs(case.m)
    X = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_node_coords(case.ctx, X.data_ptr())
    act3 = np.tile(case.act, 3)
    ref = case.coords().reshape(-1)
    assert np.abs(host(X)[act3] - ref[act3]).max() <= 1e-9


def test_preconditioner_diagonals(case):
    import torch
    for pc in (dgx.DGX_PC_HELMHOLTZ, dgx.DGX_PC_INTERNAL_ENERGY):
        d = torch.zeros(case.N, dtype=torch.float64, device="cuda")
        dgx.dgx_preconditioner_diagonal(case.ctx, pc, d.data_ptr())
        ref = O.precond_diag(case.m, pc, A_DT, GAMMA, case.rho, case.pk)
        h = host(d)
        assert rel_max_err(h[case.act], ref[case.act]) <= 1e-12
        assert np.all(np.isfinite(h)) and np.all(h[~case.act] > 0)


def test_grad_and_div(case):
    import torch
    p = _field(case, 21, scale=100.0)
    V = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    pd = dev(p)
    dgx.dgx_apply_grad(case.ctx, dgx.DGX_F64, pd.data_ptr(), V.data_ptr())
    rho1 = case.rho + (1 - case.act)  # the oracle's inverse needs no dead-cell density, but keeps it finite
    ref = O.apply_Ainv(case.m, rho1, O.apply_B(case.m, A_DT, p))
    assert rel_max_err(host(V), ref) <= 1e-12
    Vr = _field(case, 32, n=3)
    y = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    Vd = dev(Vr)
    dgx.dgx_apply_div(case.ctx, dgx.DGX_F64, Vd.data_ptr(), pd.data_ptr(), y.data_ptr())
    ref = O.apply_D(case.m, GAMMA, p) - O.apply_C(case.m, A_DT, GAMMA, case.pk, Vr)
    h = host(y)
    assert rel_max_err(h, ref) <= 1e-12 and np.all(h[~case.act] == 0)


def test_operator_every_variant(case):
    """Every launch variant (one cell per CTA at three thread counts, the fused
    multi-cell kernels, the double-word kernels) against the oracle, FP64 and FP32."""
    import torch
    p = _field(case, 41, scale=100.0)
    pd = dev(p)
    ref = O.apply_S(case.m, A_DT, GAMMA, case.rho + (1 - case.act), case.pk + (1 - case.act), p)
    tried = 0
    for prec, tol, dt in ((dgx.DGX_F64, 1e-12, torch.float64), (dgx.DGX_F32, 2e-5, torch.float32)):
        x = pd if prec == dgx.DGX_F64 else pd.float()
        for v in range(dgx.DGX_OP_VARIANTS):
            if dgx.load().dgx_set_operator_variant(case.ctx, prec, v) != dgx.DGX_OK:
                continue
            y = torch.zeros(case.N, dtype=dt, device="cuda")
            dgx.dgx_apply_operator(case.ctx, prec, x.data_ptr(), y.data_ptr())
            h = host(y).astype(np.float64)
            assert rel_max_err(h, ref) <= tol, (prec, v)
            assert np.all(h[~case.act] == 0), (prec, v)
            tried += 1
        dgx.load().dgx_set_operator_variant(case.ctx, prec, -1)
    assert tried >= 5


def test_explicit_tendencies(case):
    import torch
    bg = dgx.background(kind=0, T=250.0, p0=1e5, R=287.0, gamma=1.4, g=G, u_bar=UBAR)
    dgx.dgx_set_background(case.ctx, bg)
    obg = O.make_bg(kind=0, T=250.0, p0=1e5, R=287.0, gamma=1.4, g=G, ubar=UBAR)
    rb, pb = O.background(case.m, obg)
    rbg = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_background_fields(case.ctx, rbg.data_ptr(), None)
    assert rel_max_err(host(rbg)[case.act], rb[case.act]) <= 1e-13
    X = case.coords()
    Lx, Lz = case.m.Lx, case.m.Lz
    bump = np.exp(-((X[0] - 0.4 * Lx) ** 2 + (X[2] - 0.3 * Lz) ** 2) / (2 * (0.25 * Lx) ** 2))
    rho = rb * (1.0 + 0.01 * bump) * case.act
    u = np.concatenate([(UBAR + 3.0 * bump) * case.act, (1.0 - bump) * case.act, 0.5 * bump * case.act])
    rd, ud = dev(rho), dev(u)
    Er = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    Em = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    Ee = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_explicit_tendencies(case.ctx, rd.data_ptr(), ud.data_ptr(), Er.data_ptr(), Em.data_ptr(), Ee.data_ptr())
    er, em, ee = O.explicit(case.m, obg, rho, u, rb)
    for a, b in ((Er, er), (Em, em), (Ee, ee)):
        assert rel_max_err(host(a), b) <= 1e-12


@pytest.mark.parametrize("method", [dgx.DGX_SOLVER_FGMRES, dgx.DGX_SOLVER_MIXED])
def test_solve_matches_oracle(case, method):
    import torch
    b = O.apply_S(case.m, A_DT, GAMMA, case.rho + (1 - case.act), case.pk + (1 - case.act), _field(case, 51))
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit, o.restart = method, dgx.DGX_PC_HELMHOLTZ, 1e-10, 600, 30
    x = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    bd = dev(b)
    st, info = dgx.dgx_solve_pressure(case.ctx, bd.data_ptr(), x.data_ptr(), o)
    assert st == dgx.DGX_OK and info.relres <= 1e-10
    xh = host(x)
    r = b - O.apply_S(case.m, A_DT, GAMMA, case.rho + (1 - case.act), case.pk + (1 - case.act), xh)
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)
    assert np.all(xh[~case.act] == 0)
    xo, st_o, its_o, rel_o = O.solve(case.m, A_DT, GAMMA, case.rho + (1 - case.act), case.pk + (1 - case.act), b,
                                     method="fgmres", tol=1e-12)
    assert rel_max_err(xh, xo) <= 1e-7


def test_unsupported_features_refuse():
    c = Case(**MESHES[0])
    try:
        L = dgx.load()
        assert L.dgx_set_mass_rule(c.ctx, dgx.DGX_MASS_CONSISTENT, 1e-12, 50) == dgx.DGX_ERR_STATE
        assert L.dgx_mg_setup(c.ctx, None) in (dgx.DGX_ERR_STATE,)
    finally:
        c.close()


def test_refinement_box_validation():
    for box, ok in (((1, 3, 1, 3, 0, 2), True), ((0, 4, 0, 4, 0, 3), False), ((2, 1, 0, 1, 0, 1), False),
                    ((0, 5, 0, 1, 0, 1), False)):
        d = dgx.mesh_desc(4, 4, 3, 2, 4000.0, 4000.0, 3000.0, refine=box)
        ctx = dgx.dgx_create(0, 0)
        try:
            r = dgx.load().dgx_mesh_build(ctx, dgx.C.byref(d))
            assert (r == dgx.DGX_OK) == ok, box
        finally:
            dgx.dgx_destroy(ctx)
    d = dgx.mesh_desc(4, 4, 3, 2, 4000.0, 4000.0, 3000.0, bc_lateral=2, refine=(0, 2, 1, 3, 0, 1))
    ctx = dgx.dgx_create(0, 0)
    try:
        assert dgx.load().dgx_mesh_build(ctx, dgx.C.byref(d)) == dgx.DGX_ERR_ARG  # box on a periodic face
    finally:
        dgx.dgx_destroy(ctx)


IMEX_MESHES = [
    dict(MESHES[0], bc_lateral=1),
    dict(nx=3, ny=2, nz=2, r=3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=2, hc=200.0, ac=700.0, bc_lateral=1,
         refine=(1, 2, 0, 1, 0, 1)),
]


@pytest.mark.parametrize("mesh", IMEX_MESHES, ids=[_ids(m) for m in IMEX_MESHES])
def test_imex_step_matches_oracle(mesh):
    """Two IMEX steps (ARS(2,2,2), K = 2, solves to 1e-13 on both sides) on a
    non-conforming hill mesh: the live cells' perturbations within 1e-9 of the
    oracle's; the dead cells stay at the background at rest."""
    c = Case(**mesh)
    act = O.active_mask(c.m)
    bg = dgx.background(kind=0, T=250.0, p0=1e5, R=287.0, gamma=1.4, g=G, u_bar=UBAR)
    dgx.dgx_set_background(c.ctx, bg)
    obg = O.make_bg(kind=0, T=250.0, p0=1e5, R=287.0, gamma=1.4, g=G, ubar=UBAR)
    rb, pb = O.background(c.m, obg)
    X = c.coords()
    Lx, Lz = c.m.Lx, c.m.Lz
    bump = np.exp(-((X[0] - 0.45 * Lx) ** 2 + (X[2] - 0.3 * Lz) ** 2) / (2 * (0.2 * Lx) ** 2)) * act
    rho = rb * (1.0 + 0.005 * bump)
    p = pb + 50.0 * bump
    u = np.concatenate([(UBAR + 2.0 * bump) * act, 0.5 * bump, 0.3 * bump])
    A, At = dgx.ars222()
    dgx.dgx_set_imex(c.ctx, A, At, 1.0, 2)
    rd, ud, pd = dev(rho), dev(u), dev(p)
    o = dgx.dgx_default_solve_opts()
    o.method, o.tol, o.maxit = dgx.DGX_SOLVER_FGMRES, 1e-13, 3000
    st, info = dgx.dgx_imex_step(c.ctx, rd.data_ptr(), ud.data_ptr(), pd.data_ptr(), 2, o)
    assert st == dgx.DGX_OK and info.max_relres <= 1e-13
    r1, u1, p1 = host(rd), host(ud), host(pd)
    ro, uo, po = rho, u, p
    for _ in range(2):
        ro, uo, po, sto, _ = O.imex_step(c.m, obg, ro, uo, po, 1.0, K=2, tol=1e-13)
        assert sto == 0
    a3 = np.tile(act, 3)
    assert rel_max_err((r1 - rb)[act], (ro - rb)[act]) <= 1e-9
    assert rel_max_err(u1[a3], uo[a3]) <= 1e-9
    assert rel_max_err((p1 - pb)[act], (po - pb)[act]) <= 1e-9
    import torch
    rg, pg = torch.zeros(c.N, dtype=torch.float64, device="cuda"), torch.zeros(c.N, dtype=torch.float64, device="cuda")
    dgx.dgx_background_fields(c.ctx, rg.data_ptr(), pg.data_ptr())
    rg, pg = host(rg), host(pg)  # the library's own background (equal to the oracle's to 1e-13)
    assert np.all(r1[~act] == rg[~act]) and np.all(u1[~a3] == 0) and np.all(p1[~act] == pg[~act])
    c.close()
