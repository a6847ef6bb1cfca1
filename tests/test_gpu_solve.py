"""Pressure solves on the GPU (C ABI) against the FP64 oracle.

Workload of the 4x4x4-cell affine box (1 km)^3 at degree 2 (1728 DoFs):
isothermal hydrostatic background at T = 250 K, p0 = 1e5 Pa (R = 287,
g = 9.81) as rho^(l) and p_k, a~_ll dt = 1 - 1/sqrt(2) (ARS(2,2,2), dt = 1 s),
right-hand side = Gaussian bump (sigma = 200 m, box centre) at the nodes plus
N(0, 1e-3^2) noise, seeds 20250501 + k.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import GAMMA, Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 1.0 - 1.0 / np.sqrt(2.0)


def _isothermal(z, T=250.0, p0=1e5, R=287.0, g=9.81):
    p = p0 * np.exp(-g * z / (R * T))
    return p / (R * T), p


def _box(r=2, bg=True):
    c = Case(4, 4, 4, r)
    X = c.coords()
    if bg:
        b = dgx.background(kind=0, T=250.0, p0=1e5, R=287.0, gamma=GAMMA, g=9.81)
        dgx.dgx_set_background(c.ctx, b)
        import torch
        rb = torch.zeros(c.N, dtype=torch.float64, device="cuda")
        pb = torch.zeros(c.N, dtype=torch.float64, device="cuda")
        dgx.dgx_background_fields(c.ctx, rb.data_ptr(), pb.data_ptr())
        rho, pk = _isothermal(X[2])
        assert rel_max_err(host(rb), rho) <= 1e-14 and rel_max_err(host(pb), pk) <= 1e-14
    else:
        rho, pk = np.full(c.N, 1.2), np.full(c.N, 1e5)
    c.set_coefficients(rho, pk, A_DT)
    c.rho, c.pk, c.X = rho, pk, X
    return c


def _rhs(c, k):
    return inputs.gaussian_bump_rhs(c.X, [500.0, 500.0, 500.0], 200.0, 1e-3, inputs.DEFAULT_SEED + k)


def _solve(c, b, method, pc=dgx.DGX_PC_HELMHOLTZ, tol=1e-10, maxit=500, restart=30, **kw):
    import torch
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit, o.restart = method, pc, tol, maxit, restart
    for k, v in kw.items():
        setattr(o, k, v)
    x = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    bd = dev(b)
    st, info = dgx.dgx_solve_pressure(c.ctx, bd.data_ptr(), x.data_ptr(), o)
    return st, info, host(x)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_fgmres_box(k):
    c = _box()
    b = _rhs(c, k)
    st, info, x = _solve(c, b, dgx.DGX_SOLVER_FGMRES)
    assert st == dgx.DGX_OK and info.relres <= 1e-10
    # true residual with the oracle's operator
    r = b - O.apply_S(c.m, A_DT, GAMMA, c.rho, c.pk, x)
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)
    xo, sto, _, _ = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, method="fgmres", tol=1e-13)
    assert sto == 0 and rel_max_err(x, xo) <= 1e-8
    c.close()


def test_cg_box_uniform_spd():
    c = _box(bg=False)
    b = _rhs(c, 3)
    st, info, x = _solve(c, b, dgx.DGX_SOLVER_CG)
    assert st == dgx.DGX_OK and info.relres <= 1e-10
    xo, sto, its, _ = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, method="cg", tol=1e-13)
    assert rel_max_err(x, xo) <= 1e-8
    c.close()


@pytest.mark.parametrize("pc", [dgx.DGX_PC_HELMHOLTZ, dgx.DGX_PC_INTERNAL_ENERGY, dgx.DGX_PC_NONE])
def test_preconditioner_iterations_match_oracle(pc):
    """Same Krylov method, same preconditioner: iteration counts agree with
    the oracle's FGMRES (Helmholtz needs fewer than internal-energy)."""
    c = _box()
    b = _rhs(c, 4)
    st, info, x = _solve(c, b, dgx.DGX_SOLVER_FGMRES, pc=pc, tol=1e-8, restart=30)
    _, sto, its, _ = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, method="fgmres", pc=pc, tol=1e-8, restart=30)
    assert st == dgx.DGX_OK and abs(info.iterations - its) <= 1
    c.close()


@pytest.mark.parametrize("r", [2, 3, 5])
def test_mixed_precision_box(r):
    """FP32 operator + FP32 Jacobi inside FP64 flexible GMRES to 1e-8."""
    c = _box(r=r)
    b = _rhs(c, 5)
    st, info, x = _solve(c, b, dgx.DGX_SOLVER_MIXED, tol=1e-8, restart=20, inner_maxit=20, inner_tol=1e-4)
    assert st == dgx.DGX_OK and info.relres <= 1e-8
    r_ = b - O.apply_S(c.m, A_DT, GAMMA, c.rho, c.pk, x)
    assert np.linalg.norm(r_) <= 1.05e-8 * np.linalg.norm(b)
    xo, _, _, _ = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, method="fgmres", tol=1e-12)
    assert rel_max_err(x, xo) <= 1e-6
    assert info.operator_f32 > 0 and info.operator_f64 < info.operator_f32
    c.close()


def test_curved_farfield_solve():
    c = Case(3, 2, 2, 3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0, bc_lateral=1)
    rho, pk = c.random_coefficients(81)
    c.set_coefficients(rho, pk, A_DT)
    b = inputs.random_field(c.N, 82)
    st, info, x = _solve(c, b, dgx.DGX_SOLVER_FGMRES, tol=1e-10)
    assert st == dgx.DGX_OK
    xo, _, _, _ = O.solve(c.m, A_DT, GAMMA, rho, pk, b, method="fgmres", tol=1e-13)
    assert rel_max_err(x, xo) <= 1e-8
    c.close()


def test_not_converged_and_breakdown_status():
    c = _box()
    b = _rhs(c, 6)
    st, info, x = _solve(c, b, dgx.DGX_SOLVER_FGMRES, maxit=2)
    assert st == dgx.DGX_NOT_CONVERGED and info.iterations == 2 and info.relres > 1e-10
    bad = b.copy()
    bad[17] = np.nan  # host-side fault injection: corrupted right-hand side
    with pytest.raises(dgx.DgxError) as e:
        _solve(c, bad, dgx.DGX_SOLVER_FGMRES)
    assert e.value.code == dgx.DGX_ERR_BREAKDOWN
    with pytest.raises(dgx.DgxError) as e:
        _solve(c, bad, dgx.DGX_SOLVER_MIXED)
    assert e.value.code == dgx.DGX_ERR_BREAKDOWN
    # zero right-hand side: x = 0 immediately
    st, info, x = _solve(c, np.zeros(c.N), dgx.DGX_SOLVER_FGMRES)
    assert st == dgx.DGX_OK and np.all(x == 0)
    c.close()
