"""Learned preconditioner on the GPU (C ABI) against the FP64 oracle of the
network (oracle/learned.py) and the operator oracle.

Inputs: seeded coefficient profiles (perturbed hydrostatic, 10 % relative
noise), seeded random vectors, seeded network parameters (He-normal, every
layer non-zero); meshes with a Gal-Chen bell hill and periodic lateral faces
whose grid extents leave ragged 4x4x4 tiles (9 x 6 x 6) or fill them (12^3).
The network's weights are bfloat16 on the GPU: the oracle evaluates the same
network with the weights rounded to bfloat16 (biases FP32) in FP64; the rest
of the difference is FP32 accumulation, bounded here by 1e-4 relative.
"""
import numpy as np
import pytest

import oracle as O
import oracle.learned as NL
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs
from paper_2505_00384_gb300 import learned as LP

from _util import GAMMA, Case, dev, host, rel_max_err

pytestmark = pytest.mark.gpu

A_DT = 1.0 - 1.0 / np.sqrt(2.0)
SEED = inputs.DEFAULT_SEED


def _case(nx=3, ny=2, nz=2, r=2, L=1000.0):
    c = Case(nx, ny, nz, r, Lx=L, Ly=L, Lz=L, terrain=1, hc=300.0, ac=800.0, bc_lateral=2)
    rho, pk = c.random_coefficients(SEED + 11)
    c.set_coefficients(rho, pk, A_DT)
    c.rho, c.pk = rho, pk
    n = r + 1
    c.shape = (nz * n, ny * n, nx * n)
    c.perm = NL.dof_to_grid_index(nx, ny, nz, r)
    X = c.coords()
    c.hH = np.array([O.terrain_height(c.m, x, y) for x, y in zip(X[0], X[1])]) / L
    c.d = O.precond_diag(c.m, O.PC_HELMHOLTZ, A_DT, GAMMA, rho, pk)
    return c


def _random_params(layers, channels, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    params = []
    for l in range(layers):
        ci = 5 if l == 0 else channels
        co = 1 if l == layers - 1 else channels
        W = scale * np.sqrt(2.0 / (27 * ci)) * rng.standard_normal((co, ci, 3, 3, 3))
        params.append((W, 0.05 * rng.standard_normal(co)))
    return NL.pack(params).astype(np.float32)


def _oracle_params(p32, layers, channels):
    """The network the GPU evaluates: bfloat16 weights, FP32 biases."""
    return [(NL.bf16_round(W), b) for W, b in NL.unpack(p32.astype(np.float64), layers, channels)]


def _add_pair(c, v, e):
    vd, ed = dev(v), dev(e)
    dgx.dgx_learned_add_system(c.ctx, c._rho.data_ptr(), c._pk.data_ptr(), A_DT, GAMMA, vd.data_ptr(),
                               ed.data_ptr(), pairs=1)


def test_features_target_and_apply():
    c = _case()
    L, Ch = 3, 8
    dgx.dgx_learned_create(c.ctx, L, Ch, SEED)
    p = _random_params(L, Ch, 1)
    dgx.dgx_learned_set_params(c.ctx, p)
    v = inputs.random_field(c.N, SEED + 1)
    e = inputs.random_field(c.N, SEED + 2)
    _add_pair(c, v, e)
    G = c.N
    got = dgx.dgx_learned_sample(c.ctx, 0, G)
    f, s = NL.features(v, c.d, c.rho, c.pk, c.hH, c.perm, c.shape)
    assert np.abs(got[:5] - f.reshape(5, G)).max() <= 2e-6 * max(1.0, np.abs(f).max())
    t = NL.to_grid(e / s, c.shape, c.perm).ravel()
    assert rel_max_err(got[5], t) <= 1e-6
    # z = M(v) in FP64 and FP32
    params = _oracle_params(p, L, Ch)
    zo = NL.apply_preconditioner(params, v, c.d, c.rho, c.pk, c.hH, c.perm, c.shape)
    import torch
    vd = dev(v)
    z = torch.zeros_like(vd)
    dgx.dgx_learned_apply(c.ctx, dgx.DGX_F64, vd.data_ptr(), z.data_ptr())
    assert rel_max_err(host(z), zo) <= 1e-5
    v32 = vd.float()
    z32 = torch.zeros_like(v32)
    dgx.dgx_learned_apply(c.ctx, dgx.DGX_F32, v32.data_ptr(), z32.data_ptr())
    assert rel_max_err(host(z32), zo) <= 1e-5
    # the preconditioner entry point routes DGX_PC_LEARNED to the same call
    z2 = torch.zeros_like(vd)
    dgx.dgx_apply_preconditioner(c.ctx, dgx.DGX_PC_LEARNED, dgx.DGX_F64, vd.data_ptr(), z2.data_ptr())
    assert torch.equal(z, z2)
    c.close()


def test_training_pairs_satisfy_the_operator():
    """Every stored pair (v, e) of a system satisfies S e = v: in normalised
    form S t = D_H ch0 (t = e/s, ch0 = D_H^-1 v / s), checked with the oracle's
    operator; the first pair is (b, x), the others the residual / error of
    restarted Jacobi FGMRES cycles."""
    c = _case(4, 4, 4, 2)
    dgx.dgx_learned_create(c.ctx, 3, 8, SEED)
    b = inputs.random_field(c.N, SEED + 7)
    x = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, tol=1e-12, maxit=3000)[0]
    bd, xd = dev(b), dev(x)
    dgx.dgx_learned_add_system(c.ctx, c._rho.data_ptr(), c._pk.data_ptr(), A_DT, GAMMA, bd.data_ptr(),
                               xd.data_ptr(), pairs=5, stride=3)
    ntr, nte = dgx.dgx_learned_num_samples(c.ctx)
    assert nte == 0 and 3 <= ntr <= 5
    for k in range(ntr):
        smp = dgx.dgx_learned_sample(c.ctx, k, c.N).astype(np.float64)
        ch0 = NL.to_dof(smp[0].reshape(c.shape), c.perm)
        t = NL.to_dof(smp[5].reshape(c.shape), c.perm)
        r = c.d * ch0
        St = O.apply_S(c.m, A_DT, GAMMA, c.rho, c.pk, t)
        assert np.linalg.norm(St - r) <= 1e-3 * np.linalg.norm(r), k
    c.close()


def test_zero_network_is_jacobi():
    c = _case()
    dgx.dgx_learned_create(c.ctx, 3, 8, SEED)  # last layer starts at zero
    import torch
    v = dev(inputs.random_field(c.N, SEED + 3))
    z, zj = torch.zeros_like(v), torch.zeros_like(v)
    dgx.dgx_learned_apply(c.ctx, dgx.DGX_F64, v.data_ptr(), z.data_ptr())
    dgx.dgx_apply_preconditioner(c.ctx, dgx.DGX_PC_HELMHOLTZ, dgx.DGX_F64, v.data_ptr(), zj.data_ptr())
    assert torch.equal(z, zj)
    c.close()


@pytest.mark.parametrize("mesh,L,Ch,B", [((3, 2, 2, 2), 3, 8, 3), ((4, 4, 4, 2), 9, 32, 2),
                                         ((4, 4, 4, 2), 9, 32, 8), ((3, 5, 2, 2), 4, 32, 9)],
                         ids=["ragged_3layers_8ch", "box12_9layers_32ch", "box12_9layers_32ch_batch8_tensor_cores",
                              "ragged_4layers_32ch_batch9_tensor_cores"])
def test_loss_and_gradients(mesh, L, Ch, B):
    """Loss and gradients against the oracle.  From batch 8 on, the 32-channel
    hidden layers' forward and backward-data convolutions run on the tensor
    cores (bf16 high parts and remainders of the activations against the bf16
    weights, FP32 accumulation): the same 1e-4 bar."""
    c = _case(*mesh)
    dgx.dgx_learned_create(c.ctx, L, Ch, SEED)
    p = _random_params(L, Ch, 7)
    dgx.dgx_learned_set_params(c.ctx, p)
    for k in range(B):
        _add_pair(c, inputs.random_field(c.N, SEED + 20 + k), inputs.random_field(c.N, SEED + 40 + k))
    loss, g = dgx.dgx_learned_loss(c.ctx, 0, B)
    G = c.N
    samples = np.stack([dgx.dgx_learned_sample(c.ctx, k, G) for k in range(B)]).astype(np.float64)
    feats = samples[:, :5].reshape((B, 5) + c.shape)
    ch0 = feats[:, 0]
    t = samples[:, 5].reshape((B,) + c.shape)
    params = _oracle_params(p, L, Ch)
    lo, go = NL.loss_and_grad(params, feats, ch0, np.ones(B), t)
    assert abs(loss - lo) <= 1e-5 * lo
    gl = NL.unpack(g.astype(np.float64), L, Ch)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(gl, go)):
        assert rel_max_err(gW, oW) <= 1e-4, l
        assert rel_max_err(gb, ob) <= 1e-4, l
    c.close()


def test_adam_steps():
    """Two Adam steps on a fixed batch equal the oracle's Adam applied to the
    GPU's own gradients (gradient parity is tested above)."""
    c = _case()
    L, Ch, B = 3, 8, 4
    dgx.dgx_learned_create(c.ctx, L, Ch, SEED)
    p0 = _random_params(L, Ch, 9)
    dgx.dgx_learned_set_params(c.ctx, p0)
    for k in range(B):
        _add_pair(c, inputs.random_field(c.N, SEED + 60 + k), inputs.random_field(c.N, SEED + 80 + k))
    o = dgx.dgx_default_train_opts()
    o.epochs, o.batch, o.shuffle, o.lr, o.lr_final = 1, B, 0, 1e-3, 1e-3
    th = p0.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in (1, 2):
        _, g = dgx.dgx_learned_loss(c.ctx, 0, B)
        info = dgx.dgx_learned_train(c.ctx, o)
        assert info.steps == 1
        th, m, v = NL.adam_step(th, g.astype(np.float64), m, v, t, 1e-3)
        got = dgx.dgx_learned_get_params(c.ctx)
        assert np.abs(got - th).max() <= 1e-6 * np.abs(th).max() + 1e-3 * 1e-3, t
        th = got.astype(np.float64)
    c.close()


def _solve(c, b, pc, tol=1e-10, restart=30, maxit=600):
    import torch
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.restart, o.maxit = dgx.DGX_SOLVER_FGMRES, pc, tol, restart, maxit
    x = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    bd = dev(b)
    st, info = dgx.dgx_solve_pressure(c.ctx, bd.data_ptr(), x.data_ptr(), o)
    return st, info, host(x)


def test_fgmres_with_learned_preconditioner():
    """FGMRES accepts the (untrained, random) network as a variable
    preconditioner and reaches the oracle's solution; the FP64 residual
    decides convergence."""
    c = _case(4, 4, 4, 2)
    dgx.dgx_learned_create(c.ctx, 4, 8, SEED)
    dgx.dgx_learned_set_params(c.ctx, _random_params(4, 8, 13, scale=0.5))
    b = inputs.random_field(c.N, SEED + 5)
    st, info, x = _solve(c, b, dgx.DGX_PC_LEARNED)
    assert st in (dgx.DGX_OK, dgx.DGX_FALLBACK_USED) and info.relres <= 1e-10
    xo = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, tol=1e-12, maxit=3000)[0]
    assert rel_max_err(x, xo) <= 1e-7
    c.close()


def test_fallback_on_non_finite_network():
    """A network that returns NaN hands the solve to the Jacobi
    preconditioner: DGX_FALLBACK_USED, converged, the oracle's solution."""
    c = _case(4, 4, 4, 2)
    L, Ch = 3, 8
    dgx.dgx_learned_create(c.ctx, L, Ch, SEED)
    p = _random_params(L, Ch, 17)
    p[-1] = np.nan  # bias of the output layer
    dgx.dgx_learned_set_params(c.ctx, p)
    b = inputs.random_field(c.N, SEED + 6)
    st, info, x = _solve(c, b, dgx.DGX_PC_LEARNED)
    assert st == dgx.DGX_FALLBACK_USED and info.fallback == 1 and info.relres <= 1e-10
    xo = O.solve(c.m, A_DT, GAMMA, c.rho, c.pk, b, tol=1e-12, maxit=3000)[0]
    assert rel_max_err(x, xo) <= 1e-7
    c.close()


def test_learned_needs_network_and_fgmres():
    c = _case()
    import torch
    o = dgx.dgx_default_solve_opts()
    o.pc = dgx.DGX_PC_LEARNED
    b = dev(np.ones(c.N))
    x = torch.zeros_like(b)
    with pytest.raises(dgx.DgxError):
        dgx.dgx_solve_pressure(c.ctx, b.data_ptr(), x.data_ptr(), o)
    dgx.dgx_learned_create(c.ctx, 3, 8, SEED)
    o.method = dgx.DGX_SOLVER_MIXED
    with pytest.raises(dgx.DgxError):
        dgx.dgx_solve_pressure(c.ctx, b.data_ptr(), x.data_ptr(), o)
    with pytest.raises(dgx.DgxError):
        dgx.dgx_learned_create(c.ctx, 3, 12, SEED)
    with pytest.raises(dgx.DgxError):
        dgx.dgx_learned_loss(c.ctx, 0, 1)  # no samples yet
    c.close()


def test_recorded_systems_solve_the_oracle_operator():
    """Systems recorded inside the IMEX step: x solves S(rho, p_k) x = b of
    the oracle's operator on the same hill mesh."""
    import torch
    ctx = dgx.dgx_create(0, torch.cuda.current_stream().cuda_stream)
    N = LP.setup_hill(ctx, 500.0)
    recs, _ = LP.record_trajectory(ctx, 2, 2)
    assert recs.shape == (4, 4 * N + 2)
    m = O.make_mesh(4, 4, 4, 2, terrain=1, hc=500.0, ac=1000.0, xc=500.0, yc=500.0, bc_lateral=2)
    for k in (0, 3):
        rho, pk, b, x, a_dt, gamma = (t if isinstance(t, float) else host(t)
                                      for t in LP.split_record(recs[k], N))
        assert abs(a_dt - A_DT) <= 1e-15 and gamma == 1.4
        r = O.apply_S(m, a_dt, gamma, rho, pk, x) - b
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    dgx.dgx_destroy(ctx)


def test_training_gains_on_held_out_hill():
    """The learned-preconditioner workload (400 pressure systems recorded along
    trajectories over 16 seeded hills, 14 train, 2 held out; white-noise
    systems with the same coefficients): the trained network lowers the
    held-out loss and the FGMRES iterations to 1e-8 on held-out systems,
    against the Jacobi preconditioner on the same systems, and every solve
    reaches the recorded solution."""
    import torch
    ctx = dgx.dgx_create(0, torch.cuda.current_stream().cuda_stream)
    dgx.dgx_learned_create(ctx, 9, 32, SEED)
    heights = LP.hill_heights(16, SEED)
    held = LP.collect(ctx, heights, steps=25, record_stride=4, pairs=8, pair_stride=3, test_hills=(14, 15),
                      random_per_record=1)
    o = dgx.dgx_default_train_opts()
    o.epochs = 30
    info = dgx.dgx_learned_train(ctx, o)
    assert info.loss_test < 0.2 * info.loss_test0, (info.loss_test0, info.loss_test)
    N = dgx.dgx_num_dofs(ctx)
    its = {dgx.DGX_PC_HELMHOLTZ: [], dgx.DGX_PC_LEARNED: []}
    for hi, recs in held.items():
        LP.setup_hill(ctx, heights[hi])
        for rec in recs[::5]:
            rho, pk, b, xs, a_dt, gamma = LP.split_record(rec, N)
            dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), a_dt, gamma)
            for pc in its:
                o = dgx.dgx_default_solve_opts()
                o.pc, o.tol, o.restart, o.maxit = pc, 1e-8, 30, 1000
                x = torch.zeros(N, dtype=torch.float64, device="cuda")
                st, si = dgx.dgx_solve_pressure(ctx, b.data_ptr(), x.data_ptr(), o)
                assert st == dgx.DGX_OK and si.relres <= 1e-8, (pc, st, si.iterations, si.relres)
                assert float((x - xs).norm() / xs.norm()) <= 1e-6
                its[pc].append(si.iterations)
    plain, learned = np.mean(its[dgx.DGX_PC_HELMHOLTZ]), np.mean(its[dgx.DGX_PC_LEARNED])
    assert learned < 0.8 * plain, (plain, learned)
    dgx.dgx_destroy(ctx)
