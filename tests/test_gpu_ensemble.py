"""Batched ensemble of pressure solves against the oracle, member by member.

Members differ in mesh size, degree (3, 4, 5), terrain and lateral boundary
conditions.  Operator: FP64 within 1e-12 of the oracle, FP32 within 2e-5
(max-norm relative per member).  Solve: each member reaches the FP64 relative
residual 1e-8 (checked with the oracle's operator) and agrees with the
oracle's FGMRES solution within 1e-6.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

from _util import GAMMA, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 1.0 - 1.0 / np.sqrt(2.0)
SPECS = [
    dict(nx=3, ny=2, nz=2, r=3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=800.0, bc=2),
    dict(nx=2, ny=2, nz=2, r=4, Lx=2000.0, Ly=2000.0, Lz=1500.0, terrain=2, hc=250.0, ac=600.0, bc=1),
    dict(nx=2, ny=1, nz=2, r=5, Lx=2000.0, Ly=1000.0, Lz=1500.0, terrain=1, hc=200.0, ac=700.0, bc=0),
    dict(nx=4, ny=2, nz=1, r=3, Lx=4000.0, Ly=2000.0, Lz=800.0, terrain=0, hc=0.0, ac=1000.0, bc=0),
]


@pytest.fixture(scope="module")
def ens():
    import torch
    meshes = [O.make_mesh(s["nx"], s["ny"], s["nz"], s["r"], Lx=s["Lx"], Ly=s["Ly"], Lz=s["Lz"], terrain=s["terrain"],
                          hc=s["hc"], ac=s["ac"], bc_lateral=s["bc"]) for s in SPECS]
    descs = [dgx.mesh_desc(s["nx"], s["ny"], s["nz"], s["r"], s["Lx"], s["Ly"], s["Lz"], terrain=s["terrain"],
                           h_c=s["hc"], a_c=s["ac"], x_c=m.xc, y_c=m.yc, bc_lateral=s["bc"])
             for s, m in zip(SPECS, meshes)]
    e = dgx.dgx_ensemble_create(0, torch.cuda.current_stream().cuda_stream, descs)
    offs = [dgx.dgx_ensemble_offset(e, i) for i in range(len(SPECS))]
    Ns = [dgx.dgx_ensemble_num_dofs(e, i) for i in range(len(SPECS))]
    assert Ns == [O.ndofs(m) for m in meshes] and dgx.dgx_ensemble_num_dofs(e) == sum(Ns)
    rho, pk = [], []
    for i, m in enumerate(meshes):
        z = O.node_coords(m)[2]
        rho.append(inputs.perturbed_profile(z, 1.2, 7314.0, 0.05, 300 + i))
        pk.append(inputs.perturbed_profile(z, 1e5, 7314.0, 0.05, 400 + i))
    rd, pd = dev(np.concatenate(rho)), dev(np.concatenate(pk))
    dgx.dgx_ensemble_set_coefficients(e, rd.data_ptr(), pd.data_ptr(), A_DT, GAMMA)
    dgx.dgx_ensemble_autotune(e)  # every check below runs with the tuned tile shapes
    yield dict(e=e, meshes=meshes, offs=offs, Ns=Ns, rho=rho, pk=pk, keep=(rd, pd))
    torch.cuda.synchronize()
    dgx.dgx_ensemble_destroy(e)


def _split(E, v):
    return [v[o:o + n] for o, n in zip(E["offs"], E["Ns"])]


@pytest.mark.parametrize("prec", [dgx.DGX_F64, dgx.DGX_F32])
def test_ensemble_operator(ens, prec):
    import torch
    dt = torch.float64 if prec == dgx.DGX_F64 else torch.float32
    x = np.concatenate([inputs.random_field(n, 500 + i, 100.0) for i, n in enumerate(ens["Ns"])])
    if prec == dgx.DGX_F32:
        x = x.astype(np.float32).astype(np.float64)
    xd = dev(x).to(dt)
    y = torch.zeros_like(xd)
    dgx.dgx_ensemble_apply_operator(ens["e"], prec, xd.data_ptr(), y.data_ptr())
    yh = host(y)
    for i, (m, xs, ys) in enumerate(zip(ens["meshes"], _split(ens, x), _split(ens, yh))):
        ref = O.apply_S(m, A_DT, GAMMA, ens["rho"][i], ens["pk"][i], xs)
        assert rel_max_err(ys, ref) <= (1e-12 if prec == dgx.DGX_F64 else 2e-5), i


def test_ensemble_autotuner_choices(ens):
    dgx.dgx_ensemble_autotune(ens["e"])
    degrees = set()
    for g in range(3):
        deg, nmem, t64, t32 = dgx.dgx_ensemble_tuning(ens["e"], g)
        degrees.add(deg)
        assert nmem >= 1
        for prec, t in ((dgx.DGX_F64, t64), (dgx.DGX_F32, t32)):
            fused, cells = dgx.dgx_ensemble_tile(ens["e"], g, prec)
            if not fused:
                assert cells == 1 and t in (128, 192, 256)
            else:  # fused kernels: cells x (2r+1)^2 Gauss-point columns, whole warps
                assert cells in ((1, 2) if deg >= 3 else (4, 8))
                assert t % 32 == 0 and t >= cells * (2 * deg + 1) ** 2 > t - 32
    assert degrees == {3, 4, 5}


@pytest.mark.parametrize("seed", [600, 700])
def test_ensemble_solve(ens, seed):
    """Two solves in a row (the second replays the captured CUDA graph)."""
    import torch
    b = np.concatenate([inputs.random_field(n, seed + i) for i, n in enumerate(ens["Ns"])])
    b[ens["offs"][3]:ens["offs"][3] + ens["Ns"][3]] *= 1e3  # very different scales per member
    bd = dev(b)
    x = torch.zeros_like(bd)
    o = dgx.dgx_default_solve_opts()
    o.tol, o.maxit, o.inner_maxit, o.inner_tol = 1e-8, 50, 30, 1e-5
    st, infos = dgx.dgx_ensemble_solve(ens["e"], bd.data_ptr(), x.data_ptr(), len(SPECS), o)
    assert st == dgx.DGX_OK
    xh = host(x)
    for i, (m, bs, xs) in enumerate(zip(ens["meshes"], _split(ens, b), _split(ens, xh))):
        assert infos[i].status == dgx.DGX_OK and infos[i].relres <= 1e-8
        r = bs - O.apply_S(m, A_DT, GAMMA, ens["rho"][i], ens["pk"][i], xs)
        assert np.linalg.norm(r) <= 1.05e-8 * np.linalg.norm(bs), i
        xo, _, _, _ = O.solve(m, A_DT, GAMMA, ens["rho"][i], ens["pk"][i], bs, method="fgmres", tol=1e-12)
        assert rel_max_err(xs, xo) <= 1e-6, i


def test_ensemble_zero_member(ens):
    import torch
    b = np.concatenate([inputs.random_field(n, 800 + i) for i, n in enumerate(ens["Ns"])])
    b[ens["offs"][1]:ens["offs"][1] + ens["Ns"][1]] = 0.0
    bd = dev(b)
    x = torch.zeros_like(bd)
    o = dgx.dgx_default_solve_opts()
    o.tol, o.maxit, o.inner_maxit, o.inner_tol = 1e-8, 50, 30, 1e-5
    st, infos = dgx.dgx_ensemble_solve(ens["e"], bd.data_ptr(), x.data_ptr(), len(SPECS), o)
    assert st == dgx.DGX_OK
    assert np.all(host(x)[ens["offs"][1]:ens["offs"][1] + ens["Ns"][1]] == 0.0)


def test_ensemble_with_a_full_size_member():
    """A member of the 16-member benchmark ensemble's size (32 x 32 x 32 cells
    at r = 3, 2 097 152 DoFs, 30 x 30 x 10 km, hill, far-field faces) beside a
    small one: after the autotuner has chosen the tile shapes, the operator in
    FP64 and FP32 against the oracle on sampled cells, then one solve of both to
    1e-8 (the whole refinement loop one graph launch), its residual checked with
    the FP64 operator."""
    import torch
    specs = [dict(nx=32, ny=32, nz=32, r=3, Lx=30000.0, Ly=30000.0, Lz=10000.0, terrain=1, hc=500.0, ac=1500.0, bc=1),
             dict(nx=3, ny=2, nz=2, r=3, Lx=3000.0, Ly=2000.0, Lz=1500.0, terrain=1, hc=300.0, ac=800.0, bc=2)]
    meshes = [O.make_mesh(s["nx"], s["ny"], s["nz"], s["r"], Lx=s["Lx"], Ly=s["Ly"], Lz=s["Lz"], terrain=s["terrain"],
                          hc=s["hc"], ac=s["ac"], bc_lateral=s["bc"]) for s in specs]
    descs = [dgx.mesh_desc(s["nx"], s["ny"], s["nz"], s["r"], s["Lx"], s["Ly"], s["Lz"], terrain=s["terrain"],
                           h_c=s["hc"], a_c=s["ac"], x_c=m.xc, y_c=m.yc, bc_lateral=s["bc"])
             for s, m in zip(specs, meshes)]
    e = dgx.dgx_ensemble_create(0, torch.cuda.current_stream().cuda_stream, descs)
    Ns = [dgx.dgx_ensemble_num_dofs(e, i) for i in range(2)]
    offs = [dgx.dgx_ensemble_offset(e, i) for i in range(2)]
    rho, pk = [], []
    for i, m in enumerate(meshes):
        z = O.node_coords(m)[2]
        rho.append(inputs.perturbed_profile(z, 1.2, 7314.0, 0.05, 310 + i))
        pk.append(inputs.perturbed_profile(z, 1e5, 7314.0, 0.05, 410 + i))
    rd, pd = dev(np.concatenate(rho)), dev(np.concatenate(pk))
    dgx.dgx_ensemble_set_coefficients(e, rd.data_ptr(), pd.data_ptr(), A_DT, GAMMA)
    dgx.dgx_ensemble_autotune(e)
    x = np.concatenate([inputs.random_field(n, 520 + i, 100.0) for i, n in enumerate(Ns)])
    n3 = 64
    rng = np.random.default_rng(530)
    cells = sorted(set([0, 31, 32 * 32 - 1, 32 ** 3 - 1, 16 + 32 * 16, 16 + 32 * (16 + 32 * 31)]
                       + list(rng.integers(0, 32 ** 3, 8))))
    idx = np.concatenate([np.arange(cc * n3, (cc + 1) * n3) for cc in cells])
    for prec in (dgx.DGX_F64, dgx.DGX_F32):
        dt = torch.float64 if prec == dgx.DGX_F64 else torch.float32
        xin = x if prec == dgx.DGX_F64 else x.astype(np.float32).astype(np.float64)
        xd = dev(xin).to(dt)
        y = torch.zeros_like(xd)
        dgx.dgx_ensemble_apply_operator(e, prec, xd.data_ptr(), y.data_ptr())
        yh = host(y)
        tol = 1e-12 if prec == dgx.DGX_F64 else 2e-5
        ref0 = O.apply_S(meshes[0], A_DT, GAMMA, rho[0], pk[0], xin[:Ns[0]], cells=cells)[idx]
        assert rel_max_err(yh[:Ns[0]][idx], ref0) <= tol, prec
        ref1 = O.apply_S(meshes[1], A_DT, GAMMA, rho[1], pk[1], xin[offs[1]:])
        assert rel_max_err(yh[offs[1]:], ref1) <= tol, prec
    b = np.concatenate([inputs.random_field(n, 540 + i) for i, n in enumerate(Ns)])
    bd = dev(b)
    xs = torch.zeros_like(bd)
    o = dgx.dgx_default_solve_opts()
    o.tol, o.maxit, o.inner_maxit, o.inner_tol = 1e-8, 50, 30, 1e-5
    st, infos = dgx.dgx_ensemble_solve(e, bd.data_ptr(), xs.data_ptr(), 2, o)
    assert st == dgx.DGX_OK and all(i.relres <= 1e-8 and i.iterations >= 1 for i in infos)
    Sx = torch.zeros_like(bd)
    dgx.dgx_ensemble_apply_operator(e, dgx.DGX_F64, xs.data_ptr(), Sx.data_ptr())
    r = host(bd - Sx)
    for i in range(2):
        sl = slice(offs[i], offs[i] + Ns[i])
        assert np.linalg.norm(r[sl]) <= 1.05e-8 * np.linalg.norm(b[sl]), i
    # a second solve with other arguments (a new graph) from the first solution
    o.use_x0 = 1
    st, infos2 = dgx.dgx_ensemble_solve(e, bd.data_ptr(), xs.data_ptr(), 2, o)
    assert st == dgx.DGX_OK and all(i.iterations == 0 for i in infos2)
    torch.cuda.synchronize()
    dgx.dgx_ensemble_destroy(e)
