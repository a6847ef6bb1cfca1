"""Parity of the consistent-mass path (2r+1 point density-weighted mass, its
inverse by per-cell PCG preconditioned by the fast inverse; arXiv:2505.00384,
Sec. 3.3) with the FP64 oracle's consistent rule.

Bar: FP64 forward mass within 1e-12 of the oracle; FP64 inverse and the
operator S within 1e-11 (PCG to 1e-13 relative residual, times the
conditioning of the cell mass); FP32 inverse (PCG to 1e-5) within 1e-4; one IMEX step
within 1e-7 (solver tolerance bound, as for the fast rule).
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import GAMMA, Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 0.29289321881345254

MESHES = [
    dict(nx=2, ny=1, nz=1, r=2),
    dict(nx=2, ny=3, nz=2, r=3, Lx=2000.0, Ly=3000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0),
    dict(nx=2, ny=2, nz=3, r=4, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=2, hc=250.0, ac=600.0, bc_lateral=1),
    dict(nx=2, ny=1, nz=2, r=6, Lx=2000.0, Ly=1000.0, Lz=1000.0, terrain=1, hc=150.0, ac=500.0, bc_lateral=1),
    dict(nx=3, ny=2, nz=2, r=3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=200.0, ac=800.0, bc_lateral=2),
]


def _ids(m):
    return "%dx%dx%d_r%d_t%d" % (m["nx"], m["ny"], m["nz"], m["r"], m.get("terrain", 0))


@pytest.fixture(params=MESHES, ids=[_ids(m) for m in MESHES])
def case(request):
    c = Case(**request.param)
    rho, pk = c.random_coefficients(seed=21, rel=0.3)
    c.set_coefficients(rho, pk, A_DT)
    c.rho, c.pk = rho, pk
    dgx.dgx_set_mass_rule(c.ctx, dgx.DGX_MASS_CONSISTENT, 1e-13, 50)
    yield c
    c.close()


def _stats_ok(c, max_its=40):
    its, bad = dgx.dgx_mass_cg_stats(c.ctx)
    assert bad == 0 and its <= max_its, (its, bad)
    return its


def test_consistent_mass_forward(case):
    import torch
    v = inputs.random_field(3 * case.N, 31)
    out = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    rd = dev(case.rho)
    dgx.dgx_apply_mass(case.ctx, rd.data_ptr(), dev(v).data_ptr(), out.data_ptr())
    assert rel_max_err(host(out), O.apply_A(case.m, case.rho, v, consistent=True)) <= 1e-12


def test_consistent_mass_inverse_f64(case):
    import torch
    v = inputs.random_field(3 * case.N, 32)
    out = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_apply_mass_inverse(case.ctx, dgx.DGX_F64, dev(v).data_ptr(), out.data_ptr())
    ref = O.apply_Ainv(case.m, case.rho, v, consistent=True)
    assert rel_max_err(host(out), ref) <= 1e-11
    its = _stats_ok(case)
    assert its >= 1  # the fast inverse alone is not the consistent inverse
    # and differs from the fast inverse by the aliasing error
    dgx.dgx_set_mass_rule(case.ctx, dgx.DGX_MASS_FAST, 1e-13, 50)
    dgx.dgx_apply_mass_inverse(case.ctx, dgx.DGX_F64, dev(v).data_ptr(), out.data_ptr())
    assert rel_max_err(host(out), ref) > 1e-8


def test_consistent_mass_inverse_f32(case):
    import torch
    v = inputs.random_field(3 * case.N, 33)
    out = torch.zeros(3 * case.N, dtype=torch.float32, device="cuda")
    dgx.dgx_apply_mass_inverse(case.ctx, dgx.DGX_F32, dev(v, torch.float32).data_ptr(), out.data_ptr())
    assert rel_max_err(host(out), O.apply_Ainv(case.m, case.rho, v, consistent=True)) <= 1e-4
    _stats_ok(case)


def test_consistent_operator(case):
    import torch
    p = inputs.random_field(case.N, 34)
    y = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_apply_operator(case.ctx, dgx.DGX_F64, dev(p).data_ptr(), y.data_ptr())
    ref = O.apply_S(case.m, A_DT, GAMMA, case.rho, case.pk, p, consistent=True)
    assert rel_max_err(host(y), ref) <= 1e-11
    _stats_ok(case)


def test_consistent_solve(case):
    import torch
    b = inputs.random_field(case.N, 35)
    x = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit = dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_HELMHOLTZ, 1e-10, 2000
    st, info = dgx.dgx_solve_pressure(case.ctx, dev(b).data_ptr(), x.data_ptr(), o)
    assert st == dgx.DGX_OK and info.relres <= 1e-10
    r = b - O.apply_S(case.m, A_DT, GAMMA, case.rho, case.pk, host(x), consistent=True)
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(b)


def test_consistent_imex_step():
    """One IMEX step with every density-weighted mass consistent equals the
    oracle's consistent step (hill box, far-field lateral faces)."""
    import torch
    c = Case(2, 2, 2, 3, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=2, hc=250.0, ac=600.0, bc_lateral=1)
    G, UBAR = 9.81, 10.0
    bg = dgx.background(kind=0, T=250.0, p0=1e5, R=287.0, gamma=GAMMA, g=G, u_bar=UBAR)
    dgx.dgx_set_background(c.ctx, bg)
    obg = O.make_bg(kind=0, T=250.0, p0=1e5, R=287.0, gamma=GAMMA, g=G, ubar=UBAR)
    A, At = dgx.ars222()
    dgx.dgx_set_imex(c.ctx, A, At, 1.0, 2)
    dgx.dgx_set_mass_rule(c.ctx, dgx.DGX_MASS_CONSISTENT, 1e-13, 50)
    rb, pb = O.background(c.m, obg)
    X = c.coords()
    p0 = pb + 20.0 * np.exp(-((X[0] - 1000) ** 2 + (X[2] - 600) ** 2) / (2 * 300.0 ** 2))
    u0 = np.concatenate([np.full(c.N, UBAR), np.zeros(2 * c.N)])
    rd, ud, pd = dev(rb), dev(u0), dev(p0)
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit = dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_HELMHOLTZ, 1e-11, 3000
    st, info = dgx.dgx_imex_step(c.ctx, rd.data_ptr(), ud.data_ptr(), pd.data_ptr(), 1, o)
    assert st == dgx.DGX_OK
    ro, uo, po, sto, _ = O.imex_step(c.m, obg, rb, u0, p0, 1.0, K=2, tol=1e-11, consistent=True)
    assert sto == 0
    assert rel_max_err(host(pd) - pb, po - pb) <= 1e-7
    assert rel_max_err(host(ud), uo) <= 1e-7
    assert rel_max_err(host(rd) - rb, ro - rb) <= 1e-7
    _stats_ok(c)
    c.close()


def test_mass_rule_arguments():
    c = Case(1, 1, 1, 2)
    for args in [(2, 1e-13, 50), (dgx.DGX_MASS_CONSISTENT, 0.0, 50), (dgx.DGX_MASS_CONSISTENT, 1e-13, 0)]:
        with pytest.raises(dgx.DgxError):
            dgx.dgx_set_mass_rule(c.ctx, *args)
    assert dgx.dgx_mass_cg_stats(c.ctx) == (0, 0)
    c.close()
