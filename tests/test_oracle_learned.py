"""Pins of the learned-preconditioner oracle (oracle/learned.py).

The convolution is checked against its definition written as explicit loops
(independent of the vectorised form), against special cases (a centred delta
kernel is the identity, an off-centre delta is a shift with zero fill), the
backward pass against central finite differences of the loss, and the
DoF-to-grid map against the physical node coordinates.
"""
import numpy as np
import pytest

import oracle as O
import oracle.learned as NL


def _conv_loops(x, W, b):
    Ci, Z, Y, X = x.shape
    Co = W.shape[0]
    y = np.zeros((Co, Z, Y, X))
    for o in range(Co):
        for z in range(Z):
            for yy in range(Y):
                for xx in range(X):
                    s = b[o]
                    for i in range(Ci):
                        for dz in (-1, 0, 1):
                            for dy in (-1, 0, 1):
                                for dx in (-1, 0, 1):
                                    zz, y2, x2 = z + dz, yy + dy, xx + dx
                                    if 0 <= zz < Z and 0 <= y2 < Y and 0 <= x2 < X:
                                        s += W[o, i, dz + 1, dy + 1, dx + 1] * x[i, zz, y2, x2]
                    y[o, z, yy, xx] = s
    return y


def test_conv_matches_loop_definition():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    assert np.abs(NL.conv3d(x, W, b) - _conv_loops(x, W, b)).max() <= 1e-12


def test_conv_delta_kernels():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 5, 6))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 1] = 1.0
    assert np.array_equal(NL.conv3d(x, W, np.zeros(1)), x)
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 2] = 1.0  # y[x] = in[x+1]
    y = NL.conv3d(x, W, np.zeros(1))
    assert np.array_equal(y[..., :-1], x[..., 1:]) and np.all(y[..., -1] == 0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    shape = (3, 4, 5)
    params = [(0.3 * rng.standard_normal((4, 2, 3, 3, 3)), 0.1 * rng.standard_normal(4)),
              (0.3 * rng.standard_normal((3, 4, 3, 3, 3)), 0.1 * rng.standard_normal(3)),
              (0.3 * rng.standard_normal((1, 3, 3, 3, 3)), 0.1 * rng.standard_normal(1))]
    B = 2
    feats = rng.standard_normal((B, 2) + shape)
    j = rng.standard_normal((B,) + shape)
    x = rng.standard_normal((B,) + shape)
    s = np.array([0.7, 1.3])
    L, grads = NL.loss_and_grad(params, feats, j, s, x)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for idx in [(0, 0, 1, 1, 1), (1, 1, 0, 2, 1), (0, 1, 2, 0, 0)]:
            if any(k >= d for k, d in zip(idx, W.shape)):
                continue
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[li][0][idx] += h
            Wm[li][0][idx] -= h
            fd = (NL.loss_and_grad(Wp, feats, j, s, x)[0] - NL.loss_and_grad(Wm, feats, j, s, x)[0]) / (2 * h)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
        Bp = [(w.copy(), bb.copy()) for w, bb in params]
        Bm = [(w.copy(), bb.copy()) for w, bb in params]
        Bp[li][1][0] += h
        Bm[li][1][0] -= h
        fd = (NL.loss_and_grad(Bp, feats, j, s, x)[0] - NL.loss_and_grad(Bm, feats, j, s, x)[0]) / (2 * h)
        assert abs(fd - grads[li][1][0]) <= 1e-6 * max(1.0, abs(fd))


def test_grid_map_follows_the_mesh():
    """Grid point (k, j, i) holds the node at x_i, y_j, z_k of the lattice of
    every cell's GLL nodes (nodes shared by neighbouring cells appear twice),
    and the map is a permutation."""
    m = O.make_mesh(3, 2, 2, 2, Lx=3000.0, Ly=2000.0, Lz=1500.0)
    perm = NL.dof_to_grid_index(3, 2, 2, 2)
    assert np.array_equal(np.sort(perm), np.arange(O.ndofs(m)))
    X = O.node_coords(m)
    shape = (2 * 3, 2 * 3, 3 * 3)
    gx = NL.to_grid(X[0], shape, perm)
    gy = NL.to_grid(X[1], shape, perm)
    gz = NL.to_grid(X[2], shape, perm)
    xn, _ = O.gll(3)
    lat = lambda nc, L: ((np.arange(nc)[:, None] + xn[None, :]) * L / nc).ravel()
    assert np.allclose(gx, lat(3, 3000.0)[None, None, :], rtol=0, atol=1e-12)
    assert np.allclose(gy, lat(2, 2000.0)[None, :, None], rtol=0, atol=1e-12)
    assert np.allclose(gz, lat(2, 1500.0)[:, None, None], rtol=0, atol=1e-12)
    v = np.random.default_rng(4).standard_normal(O.ndofs(m))
    assert np.array_equal(NL.to_dof(NL.to_grid(v, shape, perm), perm), v)


def test_bf16_rounding():
    # bf16 keeps 7 fraction bits: ties go to the even neighbour.
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 3.14159, -2.5e-3])
    r = NL.bf16_round(a)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.015625 and r[3] == 1.0
    assert np.all(np.abs(r - a) <= np.abs(a) * 2 ** -8)


def test_features_normalisation():
    """Channel 0 has unit rms and is invariant to positive scaling of v;
    uniform coefficients give zero coefficient channels."""
    rng = np.random.default_rng(5)
    perm = NL.dof_to_grid_index(2, 2, 1, 1)
    shape = (2, 4, 4)
    n = perm.size
    v = rng.standard_normal(n)
    d = rng.uniform(1.0, 3.0, n)
    f, s = NL.features(v, d, np.full(n, 1.2), np.full(n, 9e4), np.zeros(n), perm, shape)
    assert abs(np.sqrt(np.mean(f[0] ** 2)) - 1.0) < 1e-14
    assert np.all(f[2] == 0) and np.all(f[3] == 0)
    f2, s2 = NL.features(7.5 * v, d, np.full(n, 1.2), np.full(n, 9e4), np.zeros(n), perm, shape)
    assert np.allclose(f2[0], f[0], rtol=1e-14, atol=1e-14) and abs(s2 / s - 7.5) < 1e-13
    # the diagonal and coefficient channels are invariant to uniform scaling
    rho, pk = rng.uniform(1.0, 1.3, n), rng.uniform(8e4, 1e5, n)
    f, _ = NL.features(v, d, rho, pk, np.zeros(n), perm, shape)
    f3, _ = NL.features(v, 4.0 * d, 2.0 * rho, 0.5 * pk, np.zeros(n), perm, shape)
    for ch in range(4):
        assert np.allclose(f3[ch], f[ch], rtol=1e-13, atol=1e-13)
    assert np.abs(f[1]).max() > 0.1 and np.abs(f[2]).max() > 0.01 and np.abs(f[3]).max() > 0.01
    # a zero network gives the Jacobi preconditioner
    params = [(np.zeros((4, 5, 3, 3, 3)), np.zeros(4)), (np.zeros((1, 4, 3, 3, 3)), np.zeros(1))]
    z = NL.apply_preconditioner(params, v, d, np.full(n, 1.2), np.full(n, 9e4), np.zeros(n), perm, shape)
    assert np.allclose(z, v / d, rtol=1e-15, atol=0)


def test_adam_closed_form():
    """First Adam step: m_hat = g, v_hat = g^2, so theta moves by
    -lr g / (|g| + eps); repeating the same gradient keeps that step."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    t1, m, v = NL.adam_step(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(t1 - th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    t2, m, v = NL.adam_step(t1, g, m, v, 2, lr=0.01)
    assert np.allclose(t2 - t1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_pack_roundtrip():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(5 * 8 * 27 + 8 + 8 * 8 * 27 + 8 + 8 * 27 + 1)
    params = NL.unpack(p, 3, 8)
    assert [W.shape for W, _ in params] == [(8, 5, 3, 3, 3), (8, 8, 3, 3, 3), (1, 8, 3, 3, 3)]
    assert np.array_equal(NL.pack(params), p)


def test_network_matches_torch_autograd():
    """Forward, loss and parameter gradients of the oracle network equal
    PyTorch's conv3d (zero padding 1, cross-correlation) with autograd in FP64."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    shape = (4, 3, 5)
    params = [(0.3 * rng.standard_normal((4, 5, 3, 3, 3)), 0.1 * rng.standard_normal(4)),
              (0.3 * rng.standard_normal((4, 4, 3, 3, 3)), 0.1 * rng.standard_normal(4)),
              (0.3 * rng.standard_normal((1, 4, 3, 3, 3)), 0.1 * rng.standard_normal(1))]
    B = 2
    feats = rng.standard_normal((B, 5) + shape)
    j = rng.standard_normal((B,) + shape)
    x = rng.standard_normal((B,) + shape)
    s = np.array([0.8, 1.7])
    L, grads = NL.loss_and_grad(params, feats, j, s, x)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    h = torch.tensor(feats)
    for l, (W, b) in enumerate(tp):
        h = torch.nn.functional.conv3d(h, W, b, padding=1)
        if l + 1 < len(tp):
            h = torch.relu(h)
    c = h[:, 0]
    e = torch.tensor(j) + torch.tensor(s)[:, None, None, None] * c - torch.tensor(x)
    Lt = ((e ** 2).sum(dim=(1, 2, 3)) / (torch.tensor(x) ** 2).sum(dim=(1, 2, 3))).mean()
    Lt.backward()
    assert abs(float(Lt.detach()) - L) <= 1e-12 * L
    for (gW, gb), (W, b) in zip(grads, tp):
        assert np.abs(gW - W.grad.numpy()).max() <= 1e-11 * max(1.0, np.abs(gW).max())
        assert np.abs(gb - b.grad.numpy()).max() <= 1e-11 * max(1.0, np.abs(gb).max())
