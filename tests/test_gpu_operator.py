"""Parity of the CUDA pressure operator (through the C ABI) with the FP64 oracle.

Bar (per result): FP64 operator action within 1e-12 of the oracle, measured
as max |y_gpu - y_oracle| / max |y_oracle|; FP32 action within 2e-5 (FP32
unit roundoff 6e-8 times the sum-factorisation depth and the conditioning
of D - C A^-1 B).
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import GAMMA, Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
A_DT = 0.29289321881345254  # a~_22 dt of ARS(2,2,2) with dt = 1 s

MESHES = [
    dict(nx=1, ny=1, nz=1, r=1),
    dict(nx=2, ny=1, nz=1, r=2),
    dict(nx=3, ny=2, nz=2, r=2),
    dict(nx=2, ny=3, nz=2, r=3, Lx=2000.0, Ly=3000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0),
    dict(nx=2, ny=2, nz=3, r=4, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=2, hc=250.0, ac=600.0, bc_lateral=1),
    dict(nx=3, ny=2, nz=1, r=5, Lx=3000.0, Ly=2000.0, Lz=800.0, terrain=1, hc=200.0, ac=900.0),
    dict(nx=2, ny=1, nz=2, r=6, Lx=2000.0, Ly=1000.0, Lz=1000.0, terrain=1, hc=150.0, ac=500.0, bc_lateral=1),
    dict(nx=3, ny=2, nz=2, r=3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=200.0, ac=800.0, bc_lateral=2),
    dict(nx=1, ny=1, nz=2, r=2, Lx=1000.0, Ly=1000.0, Lz=1000.0, bc_lateral=2),
]


def _ids(m):
    return "%dx%dx%d_r%d_t%d_bc%d" % (m["nx"], m["ny"], m["nz"], m["r"], m.get("terrain", 0), m.get("bc_lateral", 0))


@pytest.fixture(params=MESHES, ids=[_ids(m) for m in MESHES])
def case(request):
    c = Case(**request.param)
    rho, pk = c.random_coefficients(seed=11)
    c.set_coefficients(rho, pk, A_DT)
    c.rho, c.pk = rho, pk
    yield c
    c.close()


def test_node_coords(case):
    import torch
    X = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_node_coords(case.ctx, X.data_ptr())
    ref = case.coords()
    assert np.abs(host(X).reshape(3, -1) - ref).max() <= 1e-9


def test_preconditioner_diagonals(case):
    import torch
    for pc in (dgx.DGX_PC_HELMHOLTZ, dgx.DGX_PC_INTERNAL_ENERGY):
        d = torch.zeros(case.N, dtype=torch.float64, device="cuda")
        dgx.dgx_preconditioner_diagonal(case.ctx, pc, d.data_ptr())
        ref = O.precond_diag(case.m, pc, A_DT, GAMMA, case.rho, case.pk)
        assert rel_max_err(host(d), ref) <= TOL64
    x = dev(inputs.random_field(case.N, 5))
    y = torch.zeros_like(x)
    dgx.dgx_apply_preconditioner(case.ctx, dgx.DGX_PC_HELMHOLTZ, dgx.DGX_F64, x.data_ptr(), y.data_ptr())
    ref = host(x) / O.precond_diag(case.m, 1, A_DT, GAMMA, case.rho, case.pk)
    assert rel_max_err(host(y), ref) <= TOL64


def test_fp32_preconditioner_diagonals(case):
    """Before any FP64 use, an FP32 preconditioner application computes the
    diagonals with the FP32 kernel (the mixed solver's inner GMRES): both
    Jacobi preconditioners against the oracle's diagonals to FP32 accuracy."""
    import torch
    x = dev(inputs.random_field(case.N, 6)).float()
    for pc in (dgx.DGX_PC_HELMHOLTZ, dgx.DGX_PC_INTERNAL_ENERGY):
        y = torch.zeros_like(x)
        dgx.dgx_apply_preconditioner(case.ctx, pc, dgx.DGX_F32, x.data_ptr(), y.data_ptr())
        ref = host(x).astype(np.float64) / O.precond_diag(case.m, pc, A_DT, GAMMA, case.rho, case.pk)
        assert rel_max_err(host(y), ref) <= TOL32


def test_grad_and_mass_inverse(case):
    import torch
    p = inputs.random_field(case.N, 21, scale=100.0)
    V = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    pd = dev(p)  # keep a reference: the library reads it asynchronously
    dgx.dgx_apply_grad(case.ctx, dgx.DGX_F64, pd.data_ptr(), V.data_ptr())
    ref = O.apply_Ainv(case.m, case.rho, O.apply_B(case.m, A_DT, p))
    assert rel_max_err(host(V), ref) <= TOL64
    w = inputs.random_field(3 * case.N, 22)
    out = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    wd = dev(w)
    dgx.dgx_apply_mass_inverse(case.ctx, dgx.DGX_F64, wd.data_ptr(), out.data_ptr())
    assert rel_max_err(host(out), O.apply_Ainv(case.m, case.rho, w)) <= TOL64


def test_div(case):
    import torch
    p = inputs.random_field(case.N, 31, scale=100.0)
    V = inputs.random_field(3 * case.N, 32)
    y = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    Vd, pd = dev(V), dev(p)
    dgx.dgx_apply_div(case.ctx, dgx.DGX_F64, Vd.data_ptr(), pd.data_ptr(), y.data_ptr())
    ref = O.apply_D(case.m, GAMMA, p) - O.apply_C(case.m, A_DT, GAMMA, case.pk, V)
    assert rel_max_err(host(y), ref) <= TOL64


def test_operator_f64(case):
    import torch
    for seed in (41, 42):
        p = inputs.random_field(case.N, seed, scale=100.0)
        y = torch.zeros(case.N, dtype=torch.float64, device="cuda")
        pd = dev(p)
        dgx.dgx_apply_operator(case.ctx, dgx.DGX_F64, pd.data_ptr(), y.data_ptr())
        ref = O.apply_S(case.m, A_DT, GAMMA, case.rho, case.pk, p)
        assert rel_max_err(host(y), ref) <= TOL64


def test_operator_f32(case):
    import torch
    p = inputs.random_field(case.N, 51, scale=100.0)
    y = torch.zeros(case.N, dtype=torch.float32, device="cuda")
    pd = dev(p.astype(np.float32))
    dgx.dgx_apply_operator(case.ctx, dgx.DGX_F32, pd.data_ptr(), y.data_ptr())
    ref = O.apply_S(case.m, A_DT, GAMMA, case.rho, case.pk, p.astype(np.float32).astype(np.float64))
    assert rel_max_err(host(y), ref) <= TOL32


def _pin(c, prec, variant):
    """Pin a launch variant; False when it does not fit this mesh (shared memory)."""
    try:
        dgx.dgx_set_operator_variant(c.ctx, prec, variant)
    except dgx.DgxError as e:
        assert e.code == dgx.DGX_ERR_ARG
        return False
    assert dgx.dgx_operator_variant(c.ctx, prec) == variant
    return True


@pytest.mark.parametrize("variant", list(range(dgx.DGX_OP_VARIANTS)))
def test_operator_variants(case, variant):
    """Every launch variant of the operator kernels (one cell per CTA at three
    thread counts, the fused multi-cell kernels in two configurations) against
    the oracle: both halves and S in FP64 (1e-12), S in FP32 (2e-5)."""
    import torch
    ok64 = _pin(case, dgx.DGX_F64, variant)
    ok32 = _pin(case, dgx.DGX_F32, variant)
    assert ok64 or ok32 or variant >= 3
    p = inputs.random_field(case.N, 81, scale=100.0)
    pd = dev(p)
    if ok64:
        V = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
        dgx.dgx_apply_grad(case.ctx, dgx.DGX_F64, pd.data_ptr(), V.data_ptr())
        assert rel_max_err(host(V), O.apply_Ainv(case.m, case.rho, O.apply_B(case.m, A_DT, p))) <= TOL64
        W = inputs.random_field(3 * case.N, 82)
        Wd = dev(W)
        y = torch.zeros(case.N, dtype=torch.float64, device="cuda")
        dgx.dgx_apply_div(case.ctx, dgx.DGX_F64, Wd.data_ptr(), pd.data_ptr(), y.data_ptr())
        ref = O.apply_D(case.m, GAMMA, p) - O.apply_C(case.m, A_DT, GAMMA, case.pk, W)
        assert rel_max_err(host(y), ref) <= TOL64
        dgx.dgx_apply_operator(case.ctx, dgx.DGX_F64, pd.data_ptr(), y.data_ptr())
        assert rel_max_err(host(y), O.apply_S(case.m, A_DT, GAMMA, case.rho, case.pk, p)) <= TOL64
    if ok32:
        p32 = p.astype(np.float32)
        pf = dev(p32)
        yf = torch.zeros(case.N, dtype=torch.float32, device="cuda")
        dgx.dgx_apply_operator(case.ctx, dgx.DGX_F32, pf.data_ptr(), yf.data_ptr())
        ref = O.apply_S(case.m, A_DT, GAMMA, case.rho, case.pk, p32.astype(np.float64))
        assert rel_max_err(host(yf), ref) <= TOL32


def test_variant_pinning_errors():
    c = Case(2, 2, 2, 2)
    for bad in (-3, dgx.DGX_OP_VARIANTS, 99):
        with pytest.raises(dgx.DgxError) as e:
            dgx.dgx_set_operator_variant(c.ctx, dgx.DGX_F64, bad)
        assert e.value.code == dgx.DGX_ERR_ARG
    with pytest.raises(dgx.DgxError):
        dgx.dgx_set_operator_variant(c.ctx, 7, 0)
    dgx.dgx_set_operator_variant(c.ctx, dgx.DGX_F64, 3)
    assert dgx.dgx_operator_variant(c.ctx, dgx.DGX_F64) == 3
    assert dgx.dgx_operator_threads(c.ctx, dgx.DGX_F64) == 128
    dgx.dgx_set_operator_variant(c.ctx, dgx.DGX_F64, -1)
    assert dgx.dgx_operator_variant(c.ctx, dgx.DGX_F64) == -1
    dgx.dgx_set_operator_variant(c.ctx, dgx.DGX_F32, 4)
    dgx.dgx_mesh_build(c.ctx, c.desc)  # a new mesh resets the choice
    assert dgx.dgx_operator_variant(c.ctx, dgx.DGX_F32) == -1
    c.close()


def test_operator_is_deterministic(case):
    import torch
    p = dev(inputs.random_field(case.N, 61))
    y1 = torch.zeros_like(p)
    y2 = torch.zeros_like(p)
    dgx.dgx_apply_operator(case.ctx, dgx.DGX_F64, p.data_ptr(), y1.data_ptr())
    dgx.dgx_apply_operator(case.ctx, dgx.DGX_F64, p.data_ptr(), y2.data_ptr())
    assert np.array_equal(host(y1), host(y2))


def test_errors_are_reported():
    import torch
    c = Case(2, 2, 2, 2)
    x = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    with pytest.raises(dgx.DgxError) as e:  # no coefficients yet
        dgx.dgx_apply_operator(c.ctx, dgx.DGX_F64, x.data_ptr(), x.data_ptr() + 8)
    assert e.value.code == dgx.DGX_ERR_STATE
    rho, pk = c.random_coefficients(3)
    c.set_coefficients(rho, pk, A_DT)
    with pytest.raises(dgx.DgxError) as e:  # aliasing input and output
        dgx.dgx_apply_operator(c.ctx, dgx.DGX_F64, x.data_ptr(), x.data_ptr())
    assert e.value.code == dgx.DGX_ERR_ARG
    with pytest.raises(dgx.DgxError):
        dgx.dgx_mesh_build(c.ctx, dgx.mesh_desc(2, 2, 2, 9, 1.0, 1.0, 1.0))  # degree too high
    with pytest.raises(dgx.DgxError):
        bad = dgx.mesh_desc(2, 2, 2, 2, 1000.0, 1000.0, 100.0, terrain=1, h_c=500.0, a_c=300.0)
        dgx.dgx_mesh_build(c.ctx, bad)  # terrain above the model top
    c.close()


def _sampled_cells(nx, ny, nz, seed):
    """Corners, edges, the hill top and random cells of an nx x ny x nz mesh."""
    cells = [0, nx - 1, nx * ny - 1, nx * ny * nz - 1, nx // 2 + nx * (ny // 2), nx // 2 + nx * ny * (nz - 1),
             nx // 2 - 1 + nx * (ny // 2 - 1 + ny * (nz // 2 - 1)), nx * (ny - 1) + nx * ny * (nz // 2)]
    rng = np.random.default_rng(seed)
    cells += list(rng.integers(0, nx * ny * nz, 9))
    return sorted(set(int(cc) for cc in cells))


def _sampled_parity(c, nx, ny, nz, n3, precs, variants=(None,), seed=71):
    """Apply S over the whole mesh with each pinned variant (None: the
    autotuner's choice, as the bench runs it) and compare sampled cells with the
    oracle's cell-by-cell evaluation."""
    import torch
    X = torch.zeros(3 * c.N, dtype=torch.float64, device="cuda")
    dgx.dgx_node_coords(c.ctx, X.data_ptr())
    z = host(X)[2 * c.N:]
    rho = inputs.perturbed_profile(z, 1.2, 7314.0, 0.05, seed)
    pk = inputs.perturbed_profile(z, 1e5, 7314.0, 0.05, seed + 1)
    c.set_coefficients(rho, pk, A_DT)
    p = inputs.random_field(c.N, seed + 2, scale=50.0)
    cells = _sampled_cells(nx, ny, nz, seed + 3)
    idx = np.concatenate([np.arange(cc * n3, (cc + 1) * n3) for cc in cells])
    ref = {}
    for prec in precs:
        pin = p if prec == dgx.DGX_F64 else p.astype(np.float32).astype(np.float64)
        ref[prec] = O.apply_S(c.m, A_DT, GAMMA, rho, pk, pin, cells=cells)[idx]
    tried = 0
    for v in variants:
        for prec in precs:
            dt = torch.float64 if prec == dgx.DGX_F64 else torch.float32
            if v is not None and not _pin(c, prec, v):
                continue
            pd = dev(p).to(dt)
            y = torch.zeros(c.N, dtype=dt, device="cuda")
            dgx.dgx_apply_operator(c.ctx, prec, pd.data_ptr(), y.data_ptr())
            tol = TOL64 if prec == dgx.DGX_F64 else TOL32
            err = rel_max_err(host(y)[idx], ref[prec])
            assert err <= tol, (v, prec, dgx.dgx_operator_variant(c.ctx, prec), err)
            tried += 1
    assert tried > 0


@pytest.mark.parametrize("terrain", [0, 1])
def test_full_size_sampled(terrain):
    """64 x 64 x 32 cells, r = 4 (16 384 000 DoFs), terrain-following hill,
    far-field lateral faces: GPU apply over the whole mesh in FP64 and FP32
    with the variant the autotuner picks (the bench's launch configuration),
    compared on sampled cells (corners, edges, the hill top, random) with the
    oracle's cell-by-cell evaluation."""
    c = Case(64, 64, 32, 4, Lx=60000.0, Ly=60000.0, Lz=20000.0, terrain=terrain, hc=400.0, ac=1000.0,
             bc_lateral=1)
    _sampled_parity(c, 64, 64, 32, 125, (dgx.DGX_F64, dgx.DGX_F32))
    assert dgx.dgx_operator_variant(c.ctx, dgx.DGX_F64) >= 0
    assert dgx.dgx_operator_variant(c.ctx, dgx.DGX_F32) >= 0
    c.close()


@pytest.mark.parametrize("geo", [dict(nx=16, ny=16, nz=8, r=4, bc_lateral=1, terrain=1),
                                 dict(nx=16, ny=16, nz=8, r=3, bc_lateral=2, terrain=2),
                                 dict(nx=13, ny=11, nz=15, r=2, bc_lateral=0, terrain=0)],
                         ids=["16x16x8_r4_hill_farfield", "16x16x8_r3_hill32_periodic", "13x11x15_r2_flat_walls"])
def test_every_variant_on_a_tuned_size_mesh(geo):
    """Meshes of at least 2048 cells (where the autotuner chooses among the
    variants), the last one with a ragged cell count for the multi-cell CTAs:
    every launch variant in FP64 and FP32 against the oracle on sampled cells."""
    n = geo["nx"]
    c = Case(geo["nx"], geo["ny"], geo["nz"], geo["r"], Lx=1000.0 * n, Ly=1000.0 * geo["ny"], Lz=5000.0,
             terrain=geo["terrain"], hc=400.0, ac=2000.0, bc_lateral=geo["bc_lateral"])
    _sampled_parity(c, geo["nx"], geo["ny"], geo["nz"], (geo["r"] + 1) ** 3, (dgx.DGX_F64, dgx.DGX_F32),
                    variants=list(range(dgx.DGX_OP_VARIANTS)), seed=91)
    c.close()


@pytest.mark.parametrize("geo", [dict(nx=1, ny=1, nz=1, r=2), dict(nx=2, ny=1, nz=1, r=2),
                                 dict(nx=2, ny=2, nz=2, r=2, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0,
                                      ac=700.0)],
                         ids=["1x1x1_r2", "2x1x1_r2", "2x2x2_r2_terrain"])
def test_operator_assembled_entry_by_entry(geo):
    """The library's operator applied to every unit vector equals the oracle's
    assembled S = D - C A^-1 B entry by entry (tiny meshes, affine and
    terrain-following)."""
    import torch
    c = Case(**geo)
    rho, pk = c.random_coefficients(seed=71)
    c.set_coefficients(rho, pk, A_DT)
    N = c.N
    S_gpu = np.zeros((N, N))
    e = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(e)
    for j in range(N):
        e.zero_()
        e[j] = 1.0
        dgx.dgx_apply_operator(c.ctx, dgx.DGX_F64, e.data_ptr(), y.data_ptr())
        S_gpu[:, j] = host(y)
    S_ref = O.assemble(lambda v: O.apply_S(c.m, A_DT, GAMMA, rho, pk, v), N, N)
    assert np.abs(S_gpu - S_ref).max() <= TOL64 * np.abs(S_ref).max()
    # the Schur complement formed from the separately assembled blocks of Sec. 2:
    # S = D - C A^-1 B with A the fast-rule density-weighted mass (3N x 3N),
    # B (3N x N), C (N x 3N), D (N x N), and a dense solve for A^-1 B
    D = O.assemble(lambda v: O.apply_D(c.m, GAMMA, v), N, N)
    B = O.assemble(lambda v: O.apply_B(c.m, A_DT, v), N, 3 * N)
    Cm = O.assemble(lambda v: O.apply_C(c.m, A_DT, GAMMA, pk, v), 3 * N, N)
    A = O.assemble(lambda v: O.apply_A(c.m, rho, v), 3 * N, 3 * N)
    S_blocks = D - Cm @ np.linalg.solve(A, B)
    scale = np.abs(S_blocks).max()
    assert np.abs(S_ref - S_blocks).max() <= TOL64 * scale
    assert np.abs(S_gpu - S_blocks).max() <= TOL64 * scale
    c.close()
