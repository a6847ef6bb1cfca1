"""Parity of the CUDA geometric-multigrid preconditioner (dgx_mg_*) with the
multigrid oracle (oracle/mg.py): eigenvalue bounds per level, one V-cycle on
a random residual, CG with the V-cycle on the SPD case (Sec. 3.1) and FGMRES
with it on the non-symmetric Schur system (an experiment: the paper notes no
theory for multigrid there).

Bars: lambda_max per level 1e-10 (the same power steps from the same fixed
vector); V-cycle output 1e-8 (the coarsest solves run to 1e-12 on both sides,
their rounding differences scaled by the coarse conditioning); solutions 1e-8.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mg as OMG
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import GAMMA, Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 0.29289321881345254

CASES = [
    dict(geo=dict(nx=4, ny=4, nz=4, r=2), levels=2, uniform=True, coarse=0),
    dict(geo=dict(nx=8, ny=4, nz=4, r=3, Lx=4000.0, Ly=2000.0, Lz=2000.0), levels=3, uniform=True, coarse=0),
    dict(geo=dict(nx=4, ny=4, nz=4, r=2, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=250.0, ac=600.0,
                  bc_lateral=1), levels=2, uniform=False, coarse=1),
    dict(geo=dict(nx=8, ny=4, nz=4, r=4, Lx=4000.0, Ly=2000.0, Lz=2000.0, terrain=2, hc=300.0, ac=900.0,
                  bc_lateral=2), levels=3, uniform=False, coarse=1),
]


def _ids(c):
    g = c["geo"]
    return "%dx%dx%d_r%d_t%d_L%d" % (g["nx"], g["ny"], g["nz"], g["r"], g.get("terrain", 0), c["levels"])


def _setup(spec, seed=31):
    c = Case(**spec["geo"])
    if spec["uniform"]:
        rho, pk = np.full(c.N, 1.2), np.full(c.N, 1e5)
    else:
        rho, pk = c.random_coefficients(seed=seed, rel=0.05)
    c.set_coefficients(rho, pk, A_DT)
    o = dgx.dgx_default_mg_opts()
    o.levels, o.coarse_tol, o.coarse_maxit, o.coarse_solver = spec["levels"], 1e-12, 3000, spec["coarse"]
    dgx.dgx_mg_setup(c.ctx, o)
    h = OMG.Hierarchy(c.m, A_DT, GAMMA, rho, pk, levels=spec["levels"], coarse_tol=1e-12, coarse_its=3000,
                      coarse="fgmres" if spec["coarse"] else "cg")
    return c, rho, pk, h


@pytest.fixture(params=CASES, ids=[_ids(c) for c in CASES])
def mgcase(request):
    c, rho, pk, h = _setup(request.param)
    yield c, rho, pk, h, request.param
    c.close()


def test_eigenvalue_bounds_per_level(mgcase):
    c, _, _, h, spec = mgcase
    n, lam = dgx.dgx_mg_levels(c.ctx)
    assert n == spec["levels"]
    for l in range(n):
        assert lam[l] == pytest.approx(h.lmax[l], rel=1e-10), l


def test_one_vcycle(mgcase):
    import torch
    c, _, _, h, _ = mgcase
    r = inputs.random_field(c.N, 41)
    rd = dev(r)
    z = torch.zeros_like(rd)
    dgx.dgx_mg_vcycle(c.ctx, rd.data_ptr(), z.data_ptr())
    assert rel_max_err(host(z), h.vcycle(r)) <= 1e-8


def test_mg_cg_on_the_spd_case():
    """Uniform coefficients, slip walls (S SPD): CG + one V-cycle per iteration
    to 1e-10 from zero, iteration count and solution as the oracle's MG-CG, and
    at most half the iterations of Jacobi CG on the GPU."""
    import torch
    c, rho, pk, h = _setup(CASES[1])
    b = inputs.random_field(c.N, 42)
    bd = dev(b)
    x = torch.zeros_like(bd)
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit = dgx.DGX_SOLVER_CG, dgx.DGX_PC_MULTIGRID, 1e-10, 500
    st, info = dgx.dgx_solve_pressure(c.ctx, bd.data_ptr(), x.data_ptr(), o)
    xo, its_o, rel_o = OMG.mg_pcg(h, b, tol=1e-10)
    assert st == dgx.DGX_OK and info.relres <= 1e-10
    assert abs(info.iterations - its_o) <= 1, (info.iterations, its_o)
    assert rel_max_err(host(x), xo) <= 1e-8
    xj = torch.zeros_like(bd)
    o.pc = dgx.DGX_PC_HELMHOLTZ
    st, infj = dgx.dgx_solve_pressure(c.ctx, bd.data_ptr(), xj.data_ptr(), o)
    assert st == dgx.DGX_OK and 2 * info.iterations <= infj.iterations
    c.close()


def test_mg_fgmres_on_the_schur_system():
    """Curved hill mesh, non-uniform coefficients (S non-symmetric): FGMRES
    with the V-cycle reaches 1e-10, checked with the oracle's S."""
    import torch
    c, rho, pk, h = _setup(CASES[3])
    b = inputs.random_field(c.N, 43)
    bd = dev(b)
    x = torch.zeros_like(bd)
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit = dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_MULTIGRID, 1e-10, 300
    st, info = dgx.dgx_solve_pressure(c.ctx, bd.data_ptr(), x.data_ptr(), o)
    assert st == dgx.DGX_OK
    r = b - O.apply_S(c.m, A_DT, GAMMA, rho, pk, host(x))
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)
    c.close()


def test_vcycle_follows_new_coefficients():
    """dgx_set_coefficients after the set-up: the next V-cycle restricts the new
    coefficients and re-estimates the bounds (oracle hierarchy built afresh)."""
    import torch
    spec = CASES[2]
    c, _, _, _ = _setup(spec)
    rho2, pk2 = c.random_coefficients(seed=77, rel=0.05)
    c.set_coefficients(rho2, pk2, A_DT)
    h2 = OMG.Hierarchy(c.m, A_DT, GAMMA, rho2, pk2, levels=spec["levels"], coarse_tol=1e-12, coarse_its=3000,
                       coarse="fgmres")
    r = inputs.random_field(c.N, 44)
    rd = dev(r)
    z = torch.zeros_like(rd)
    dgx.dgx_mg_vcycle(c.ctx, rd.data_ptr(), z.data_ptr())
    assert rel_max_err(host(z), h2.vcycle(r)) <= 1e-8
    c.close()


def test_mg_errors():
    import torch
    c = Case(3, 2, 2, 2)
    rho, pk = c.random_coefficients(seed=5)
    c.set_coefficients(rho, pk, A_DT)
    with pytest.raises(dgx.DgxError) as e:  # 3 cells not divisible by 2
        dgx.dgx_mg_setup(c.ctx)
    assert e.value.code == dgx.DGX_ERR_ARG
    b = dev(inputs.random_field(c.N, 6))
    x = torch.zeros_like(b)
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc = dgx.DGX_SOLVER_CG, dgx.DGX_PC_MULTIGRID
    with pytest.raises(dgx.DgxError) as e:  # no hierarchy
        dgx.dgx_solve_pressure(c.ctx, b.data_ptr(), x.data_ptr(), o)
    assert e.value.code == dgx.DGX_ERR_ARG
    c.close()
    c = Case(2, 2, 2, 2)
    c.set_coefficients(np.full(c.N, 1.2), np.full(c.N, 1e5), A_DT)
    bad = dgx.dgx_default_mg_opts()
    bad.levels = 1
    with pytest.raises(dgx.DgxError):
        dgx.dgx_mg_setup(c.ctx, bad)
    with pytest.raises(dgx.DgxError):  # the default 3 levels need nx, ny, nz divisible by 4
        dgx.dgx_mg_setup(c.ctx)
    ok = dgx.dgx_default_mg_opts()
    ok.levels = 2
    dgx.dgx_mg_setup(c.ctx, ok)
    assert dgx.dgx_mg_levels(c.ctx)[0] == 2
    b = dev(inputs.random_field(c.N, 7))
    x = torch.zeros_like(b)
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc = dgx.DGX_SOLVER_MIXED, dgx.DGX_PC_MULTIGRID
    with pytest.raises(dgx.DgxError) as e:  # not inside the mixed-precision solver
        dgx.dgx_solve_pressure(c.ctx, b.data_ptr(), x.data_ptr(), o)
    assert e.value.code == dgx.DGX_ERR_ARG
    c.close()
