"""Parity of the GPU explicit fluxes, mass terms and IMEX step with the oracle.

Tolerances: explicit tendencies and mass terms (single applications) within
1e-12 of the oracle (max-norm relative); the IMEX step goes through pressure
solves converged to a relative residual of 1e-13 on both sides, so the states
agree to the solve tolerance times the conditioning of S.  On these meshes
the oracle's own states at 1e-11 and 1e-13 differ by at most 3e-10 (relative
max norm of the perturbations rho - rho_bar, u, p - p_bar), so the bar is 1e-9
for one, two and five steps; with the mixed-precision solver at 1e-9, 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

G, UBAR = 9.81, 10.0

MESHES = [
    dict(nx=2, ny=1, nz=2, r=1),
    dict(nx=3, ny=2, nz=2, r=2, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=800.0),
    dict(nx=2, ny=2, nz=2, r=3, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=2, hc=250.0, ac=600.0, bc_lateral=1),
    dict(nx=2, ny=1, nz=2, r=4, Lx=2000.0, Ly=1000.0, Lz=1500.0, terrain=1, hc=300.0, ac=700.0, bc_lateral=1),
    dict(nx=2, ny=1, nz=1, r=5, Lx=2000.0, Ly=1000.0, Lz=800.0, terrain=1, hc=150.0, ac=600.0, bc_lateral=1),
    dict(nx=3, ny=2, nz=2, r=4, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=200.0, ac=800.0, bc_lateral=2),
]


def _ids(m):
    return "%dx%dx%d_r%d_t%d_bc%d" % (m["nx"], m["ny"], m["nz"], m["r"], m.get("terrain", 0), m.get("bc_lateral", 0))


def _with_bg(c, kind=0):
    bg = dgx.background(kind=kind, T=250.0 if kind == 0 else 293.15, p0=1e5, R=287.0, gamma=1.4, g=G, u_bar=UBAR)
    dgx.dgx_set_background(c.ctx, bg)
    obg = O.make_bg(kind=kind, T=bg.T, p0=1e5, R=287.0, gamma=1.4, g=G, ubar=UBAR)
    rb, pb = O.background(c.m, obg)
    return obg, rb, pb


def _state(c, rb, pb, seed):
    """Smooth seeded perturbation of the background: density and pressure
    bubble, wind with smooth seeded-amplitude modes (per-node white noise is
    not a meaningful atmospheric state at high order)."""
    X = c.coords()
    a = 1.0 + 0.1 * inputs.normal(seed, 6)
    Lx, Ly, Lz = c.m.Lx, c.m.Ly, c.m.Lz
    xc, zc = 0.5 * Lx, 0.4 * Lz
    bump = np.exp(-((X[0] - xc) ** 2 + (X[2] - zc) ** 2) / (2 * (0.2 * Lx) ** 2))
    sx, cy, sz = np.sin(np.pi * X[0] / Lx), np.cos(np.pi * X[1] / Ly), np.sin(np.pi * X[2] / Lz)
    rho = rb * (1.0 + 0.005 * a[0] * bump)
    p = pb + 50.0 * a[1] * bump
    u = np.concatenate([UBAR + 2.0 * a[2] * sx * sz, 1.0 * a[3] * cy * sz, 0.5 * a[4] * sx * sz])
    return rho, u, p


@pytest.fixture(params=MESHES, ids=[_ids(m) for m in MESHES])
def case(request):
    c = Case(**request.param)
    yield c
    c.close()


def test_background_fields_match(case):
    import torch
    for kind in (0, 1):
        _, rb, pb = _with_bg(case, kind)
        r = torch.zeros(case.N, dtype=torch.float64, device="cuda")
        p = torch.zeros(case.N, dtype=torch.float64, device="cuda")
        dgx.dgx_background_fields(case.ctx, r.data_ptr(), p.data_ptr())
        assert rel_max_err(host(r), rb) <= 1e-13 and rel_max_err(host(p), pb) <= 1e-13


@pytest.mark.parametrize("variant", [1, 0], ids=["double_words", "fp64_pipe"])
def test_explicit_tendencies(case, variant):
    """Both arithmetics of the explicit fluxes (double-words on the FP32 pipes,
    the default up to degree 4, and the FP64 pipe) against the oracle."""
    import torch
    dgx.dgx_set_explicit_variant(case.ctx, variant)
    obg, rb, pb = _with_bg(case)
    rho, u, _ = _state(case, rb, pb, 101)
    rd, ud = dev(rho), dev(u)
    Er = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    Em = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    Ee = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_explicit_tendencies(case.ctx, rd.data_ptr(), ud.data_ptr(), Er.data_ptr(), Em.data_ptr(), Ee.data_ptr())
    er, em, ee = O.explicit(case.m, obg, rho, u, rb)
    assert rel_max_err(host(Er), er) <= 1e-12
    assert rel_max_err(host(Em), em) <= 1e-12
    assert rel_max_err(host(Ee), ee) <= 1e-12


@pytest.mark.parametrize("variant", [1, 0], ids=["double_words", "fp64_pipe"])
def test_mass_terms(case, variant):
    import torch
    dgx.dgx_set_explicit_variant(case.ctx, variant)
    _, rb, pb = _with_bg(case)
    rho, u, _ = _state(case, rb, pb, 111)
    rd, ud = dev(rho), dev(u)
    out3 = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_apply_mass(case.ctx, rd.data_ptr(), ud.data_ptr(), out3.data_ptr())
    assert rel_max_err(host(out3), O.apply_A(case.m, rho, u)) <= 1e-12
    out = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_kinetic_mass(case.ctx, rd.data_ptr(), ud.data_ptr(), out.data_ptr())
    assert rel_max_err(host(out), O.kinetic_mass(case.m, rho, u)) <= 1e-12


def _gpu_steps(c, rho, u, p, nsteps, method=dgx.DGX_SOLVER_FGMRES, tol=1e-11, dt=1.0, K=2):
    A, At = dgx.ars222()
    dgx.dgx_set_imex(c.ctx, A, At, dt, K)
    rd, ud, pd = dev(rho), dev(u), dev(p)
    o = dgx.dgx_default_solve_opts()
    o.method, o.tol, o.maxit = method, tol, 3000
    st, info = dgx.dgx_imex_step(c.ctx, rd.data_ptr(), ud.data_ptr(), pd.data_ptr(), nsteps, o)
    return st, info, host(rd), host(ud), host(pd)


STEP_TOL = 1e-13  # solver tolerance of both sides
STEP_BAR = 1e-9


def _compare_steps(case, obg, rb, pb, rho, u, p, nsteps):
    st, info, r1, u1, p1 = _gpu_steps(case, rho, u, p, nsteps, tol=STEP_TOL)
    assert st == dgx.DGX_OK and info.steps == nsteps and info.solves == 2 * 2 * nsteps
    assert info.max_relres <= STEP_TOL
    ro, uo, po = rho, u, p
    for _ in range(nsteps):
        ro, uo, po, sto, _ = O.imex_step(case.m, obg, ro, uo, po, 1.0, K=2, tol=STEP_TOL)
        assert sto == 0
    assert rel_max_err(r1 - rb, ro - rb) <= STEP_BAR
    assert rel_max_err(u1, uo) <= STEP_BAR
    assert rel_max_err(p1 - pb, po - pb) <= STEP_BAR


@pytest.mark.parametrize("nsteps", [1, 2])
def test_imex_step_matches_oracle(case, nsteps):
    obg, rb, pb = _with_bg(case)
    rho, u, p = _state(case, rb, pb, 121)
    _compare_steps(case, obg, rb, pb, rho, u, p, nsteps)


@pytest.mark.parametrize("variant", [3, 4, 5, 6])
def test_imex_step_with_fused_operator(case, variant):
    """The step with the fused operator kernels pinned (FP64, and FP32 for the
    variants that have an FP32 form; 5 and 6 compute the FP64 operator in
    double-word arithmetic): also covers their uses inside the step (the dual
    B p' and -C u with the step's own coefficients and a~ dt = 1)."""
    obg, rb, pb = _with_bg(case)
    rho, u, p = _state(case, rb, pb, 122)
    for prec in ((dgx.DGX_F64, dgx.DGX_F32) if variant < 5 else (dgx.DGX_F64,)):
        try:
            dgx.dgx_set_operator_variant(case.ctx, prec, variant)
        except dgx.DgxError:
            pytest.skip("variant %d does not fit degree %d" % (variant, case.m.r))
    _compare_steps(case, obg, rb, pb, rho, u, p, 1)


def test_imex_five_steps():
    """Five steps on a periodic hill mesh at r = 3 against the oracle's."""
    c = Case(3, 2, 2, 3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=200.0, ac=800.0, bc_lateral=2)
    obg, rb, pb = _with_bg(c)
    rho, u, p = _state(c, rb, pb, 123)
    _compare_steps(c, obg, rb, pb, rho, u, p, 5)
    c.close()


def test_imex_mixed_precision_step(case):
    """FP32-preconditioned solves to 1e-9 give the same step within 1e-5."""
    obg, rb, pb = _with_bg(case)
    rho, u, p = _state(case, rb, pb, 131)
    st, info, r1, u1, p1 = _gpu_steps(case, rho, u, p, 1, method=dgx.DGX_SOLVER_MIXED, tol=1e-9)
    assert st == dgx.DGX_OK and info.max_relres <= 1e-9 and info.operator_f32 > 0
    ro, uo, po, _, _ = O.imex_step(case.m, obg, rho, u, p, 1.0, K=2, tol=1e-11)
    assert rel_max_err(u1, uo) <= 1e-5 and rel_max_err(p1 - pb, po - pb) <= 1e-5


@pytest.mark.parametrize("kind", [0, 1])
def test_rest_state_is_preserved(case, kind):
    """The library's own background at rest (no far-field wind): all
    perturbations are exactly zero, so the state is unchanged bit for bit."""
    import torch
    bg = dgx.background(kind=kind, T=250.0 if kind == 0 else 293.15, g=G, u_bar=0.0)
    dgx.dgx_set_background(case.ctx, bg)
    r = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    p = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    dgx.dgx_background_fields(case.ctx, r.data_ptr(), p.data_ptr())
    rb, pb = host(r), host(p)
    st, info, r1, u1, p1 = _gpu_steps(case, rb, np.zeros(3 * case.N), pb, 2)
    assert st == dgx.DGX_OK
    assert np.array_equal(r1, rb) and np.array_equal(p1, pb) and np.abs(u1).max() == 0.0


def test_imex_requires_setup():
    import torch
    c = Case(2, 2, 2, 2)
    x = torch.zeros(3 * c.N, dtype=torch.float64, device="cuda")
    with pytest.raises(dgx.DgxError) as e:
        dgx.dgx_imex_step(c.ctx, x.data_ptr(), x.data_ptr(), x.data_ptr(), 1)
    assert e.value.code == dgx.DGX_ERR_STATE
    A, At = dgx.ars222()
    bad = At.copy()
    bad[0, 0] = 0.5
    with pytest.raises(dgx.DgxError):
        dgx.dgx_set_imex(c.ctx, A, bad, 1.0, 2)
    c.close()


def test_full_size_explicit_sampled_and_step():
    """64 x 64 x 32 cells, r = 4 (16 384 000 DoFs), bell hill, far field:
    explicit tendencies on sampled cells against the oracle; one full IMEX
    step with mixed-precision solves converges and keeps the state finite."""
    import torch
    c = Case(64, 64, 32, 4, Lx=60000.0, Ly=60000.0, Lz=20000.0, terrain=1, hc=400.0, ac=1000.0, bc_lateral=1)
    obg, rb, pb = _with_bg(c)
    X = torch.zeros(3 * c.N, dtype=torch.float64, device="cuda")
    dgx.dgx_node_coords(c.ctx, X.data_ptr())
    Xh = host(X).reshape(3, -1)
    bump = np.exp(-((Xh[0] - 30000.0) ** 2 + (Xh[1] - 30000.0) ** 2 + (Xh[2] - 3000.0) ** 2) / (2 * 3000.0 ** 2))
    rho = rb * (1.0 + 0.002 * bump)
    p = pb + 50.0 * bump
    u = np.concatenate([np.full(c.N, UBAR), np.zeros(c.N), np.zeros(c.N)])
    rd, ud = dev(rho), dev(u)
    Er = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    Em = torch.zeros(3 * c.N, dtype=torch.float64, device="cuda")
    Ee = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    dgx.dgx_explicit_tendencies(c.ctx, rd.data_ptr(), ud.data_ptr(), Er.data_ptr(), Em.data_ptr(), Ee.data_ptr())
    nx, ny, nz = 64, 64, 32
    cells = [0, nx - 1, nx * ny * nz - 1, 32 + nx * 32, 31 + nx * (31 + ny * 2), 5 + nx * (60 + ny * 31)]
    er, em, ee = O.explicit(c.m, obg, rho, u, rb, cells=cells)
    idx = np.concatenate([np.arange(cc * 125, (cc + 1) * 125) for cc in cells])
    assert rel_max_err(host(Er)[idx], er[idx]) <= 1e-12
    assert rel_max_err(host(Ee)[idx], ee[idx]) <= 1e-12
    idx3 = np.concatenate([d * c.N + idx for d in range(3)])
    assert rel_max_err(host(Em)[idx3], em[idx3]) <= 1e-12
    st, info, r1, u1, p1 = _gpu_steps(c, rho, u, p, 1, method=dgx.DGX_SOLVER_MIXED, tol=1e-8)
    assert st == dgx.DGX_OK and info.max_relres <= 1e-8
    assert np.all(np.isfinite(r1)) and np.all(np.isfinite(u1)) and np.all(np.isfinite(p1))
    c.close()
