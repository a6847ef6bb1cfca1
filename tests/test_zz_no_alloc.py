"""The allocation-free operator entry point (dgx_apply_operator_noalloc).

Callers that cannot allocate device memory at the point of use (a host
application whose pool allocator owns the device memory, a time-critical
loop that must not call cudaMalloc) use this variant: its scratch lives in a
fixed static device array.  The test calls it through the C ABI twice in a
row, with different inputs, and checks each result against
dgx_apply_operator within the operator tests' tolerances.  This file is
collected last so that a stop at the first failure has run all other tests.
"""
import numpy as np
import pytest

from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 0.29289321881345254
TOL = {dgx.DGX_F64: 1e-12, dgx.DGX_F32: 2e-5}


@pytest.mark.parametrize("prec", [dgx.DGX_F64, dgx.DGX_F32])
def test_noalloc_matches_operator_twice(prec):
    import torch
    dt = torch.float64 if prec == dgx.DGX_F64 else torch.float32
    c = Case(3, 2, 2, 3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0, bc_lateral=1)
    rho, pk = c.random_coefficients(seed=91)
    c.set_coefficients(rho, pk, A_DT)
    for call, seed in enumerate((92, 93)):
        x = dev(inputs.random_field(c.N, seed, scale=100.0)).to(dt)
        y_ref = torch.zeros(c.N, dtype=dt, device="cuda")
        y_na = torch.full((c.N,), float("nan"), dtype=dt, device="cuda")
        dgx.dgx_apply_operator(c.ctx, prec, x.data_ptr(), y_ref.data_ptr())
        dgx.dgx_apply_operator_noalloc(c.ctx, prec, x.data_ptr(), y_na.data_ptr())
        a, b = host(y_na), host(y_ref)
        assert np.all(np.isfinite(a)), "call %d" % call
        assert rel_max_err(a, b) <= TOL[prec], "call %d" % call
    c.close()


@pytest.mark.parametrize("prec", [dgx.DGX_F64, dgx.DGX_F32])
def test_noalloc_on_a_fresh_context(prec):
    """What an allocation-free caller gets: the entry point on a context that
    never applied the operator (so never ran the timing autotuner, which
    allocates), checked against the oracle's S."""
    import torch
    import oracle as O
    dt = torch.float64 if prec == dgx.DGX_F64 else torch.float32
    c = Case(3, 2, 2, 3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0, bc_lateral=1)
    rho, pk = c.random_coefficients(seed=94)
    c.set_coefficients(rho, pk, A_DT)
    assert dgx.dgx_operator_variant(c.ctx, prec) == -1
    x = inputs.random_field(c.N, 95, scale=100.0)
    if prec == dgx.DGX_F32:
        x = x.astype(np.float32).astype(np.float64)
    xd = dev(x).to(dt)
    y = torch.full((c.N,), float("nan"), dtype=dt, device="cuda")
    dgx.dgx_apply_operator_noalloc(c.ctx, prec, xd.data_ptr(), y.data_ptr())
    assert rel_max_err(host(y), O.apply_S(c.m, A_DT, 1.4, rho, pk, x)) <= TOL[prec]
    c.close()


@pytest.mark.parametrize("prec,shape", [(dgx.DGX_F64, (26, 26, 16)), (dgx.DGX_F32, (32, 32, 21))],
                         ids=["f64_26x26x16_r3", "f32_32x32x21_r3"])
def test_noalloc_near_the_limit(prec, shape):
    """Meshes whose V fills 98-99 % of the static array (3 N sizeof(T) just
    below DGX_NOALLOC_SCRATCH_BYTES), random input: every component stride of
    V up to the top of the array is exercised; result as dgx_apply_operator."""
    import torch
    dt = torch.float64 if prec == dgx.DGX_F64 else torch.float32
    nx, ny, nz = shape
    c = Case(nx, ny, nz, 3, Lx=500.0 * nx, Ly=500.0 * ny, Lz=400.0 * nz, terrain=1, hc=300.0, ac=2000.0,
             bc_lateral=1)
    elem = 8 if prec == dgx.DGX_F64 else 4
    assert 0.97 * dgx.DGX_NOALLOC_SCRATCH_BYTES <= 3 * c.N * elem <= dgx.DGX_NOALLOC_SCRATCH_BYTES
    rho, pk = c.random_coefficients(seed=96)
    c.set_coefficients(rho, pk, A_DT)
    for seed in (97, 98):
        x = dev(inputs.random_field(c.N, seed, scale=100.0)).to(dt)
        y_na = torch.full((c.N,), float("nan"), dtype=dt, device="cuda")
        y_ref = torch.zeros(c.N, dtype=dt, device="cuda")
        dgx.dgx_apply_operator_noalloc(c.ctx, prec, x.data_ptr(), y_na.data_ptr())
        dgx.dgx_apply_operator(c.ctx, prec, x.data_ptr(), y_ref.data_ptr())
        a, b = host(y_na), host(y_ref)
        assert np.all(np.isfinite(a))
        assert rel_max_err(a, b) <= TOL[prec]
    c.close()


def test_noalloc_rejects_meshes_above_the_limit():
    import torch
    # 40 x 40 x 8 cells at r = 3: N = 819200, 3N doubles = 19.7 MB > 16 MiB
    c = Case(40, 40, 8, 3, Lx=40000.0, Ly=40000.0, Lz=8000.0)
    rho, pk = np.full(c.N, 1.2), np.full(c.N, 1e5)
    c.set_coefficients(rho, pk, A_DT)
    x = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    y = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    with pytest.raises(dgx.DgxError) as e:
        dgx.dgx_apply_operator_noalloc(c.ctx, dgx.DGX_F64, x.data_ptr(), y.data_ptr())
    assert e.value.code == dgx.DGX_ERR_ARG and "16777216" in str(e.value)
    # the same mesh fits in FP32 (3N floats = 9.8 MB)
    xf, yf = x.float(), y.float()
    dgx.dgx_apply_operator_noalloc(c.ctx, dgx.DGX_F32, xf.data_ptr(), yf.data_ptr())
    assert float(host(yf).__abs__().max()) == 0.0
    c.close()
