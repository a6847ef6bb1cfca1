"""FP64 oracle of the learned preconditioner network (TEST INFRASTRUCTURE).

The network is a stack of 3x3x3 convolutions (zero padding, stride 1) with
ReLU between layers, on the cell-DoF tensor: the nodal values of a DG field of
degree r on an nx x ny x nz mesh laid out as a grid of (nz (r+1)) x (ny (r+1)) x
(nx (r+1)) points (the (r+1)^3 nodes of each cell in their own block, x
fastest).  Plain numpy definitions in FP64, written for reading, used only
to check the CUDA kernels: forward and backward of each convolution, the
network, and the training loss

    L = (1/B) sum_b || j_b + s_b c_b - x_b ||^2 / || x_b ||^2,

where c_b is the network output for sample b, j_b = D^-1 v_b the Jacobi
guess, s_b = rms(j_b) and x_b the solver's solution.
"""
import numpy as np


def dof_to_grid_index(nx, ny, nz, r):
    """perm[g] = DoF index of grid point g (grid x fastest, shape (Z, Y, X))."""
    n = r + 1
    X, Y, Z = nx * n, ny * n, nz * n
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    cx, a = gx // n, gx % n
    cy, b = gy // n, gy % n
    cz, c = gz // n, gz % n
    cell = cx + nx * (cy + ny * cz)
    return (cell * n ** 3 + a + n * b + n * n * c).ravel()


def to_grid(v, shape, perm):
    return np.asarray(v)[..., perm].reshape(v.shape[:-1] + tuple(shape))


def to_dof(g, perm):
    out = np.empty(g.shape[:-3] + (perm.size,))
    out[..., perm] = g.reshape(g.shape[:-3] + (-1,))
    return out


def conv3d(x, W, b):
    """x: (Ci, Z, Y, X); W: (Co, Ci, 3, 3, 3); b: (Co,).  Zero padding 1."""
    Ci, Z, Y, X = x.shape
    xp = np.zeros((Ci, Z + 2, Y + 2, X + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((W.shape[0], Z, Y, X))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                y += np.einsum("oi,izyx->ozyx", W[:, :, dz, dy, dx], patch)
    return y + b[:, None, None, None]


def conv3d_backward(x, W, gy):
    """Gradients of sum(gy * conv3d(x, W, b)) w.r.t. x, W and b."""
    Ci, Z, Y, X = x.shape
    xp = np.zeros((Ci, Z + 2, Y + 2, X + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                gW[:, :, dz, dy, dx] = np.einsum("ozyx,izyx->oi", gy, patch)
                gxp[:, dz:dz + Z, dy:dy + Y, dx:dx + X] += np.einsum("oi,ozyx->izyx", W[:, :, dz, dy, dx], gy)
    return gxp[:, 1:-1, 1:-1, 1:-1], gW, gy.sum(axis=(1, 2, 3))


def forward(params, x):
    """params: list of (W, b); ReLU after every layer but the last.
    Returns the output and the list of layer inputs / pre-activations."""
    cache = []
    h = x
    for i, (W, b) in enumerate(params):
        z = conv3d(h, W, b)
        cache.append((h, z))
        h = np.maximum(z, 0.0) if i + 1 < len(params) else z
    return h, cache


def backward(params, cache, gout):
    grads = [None] * len(params)
    g = gout
    for i in range(len(params) - 1, -1, -1):
        h, z = cache[i]
        if i + 1 < len(params):
            g = g * (z > 0.0)
        gx, gW, gb = conv3d_backward(h, params[i][0], g)
        grads[i] = (gW, gb)
        g = gx
    return grads


def loss_and_grad(params, feats, j, s, x):
    """Mean relative squared error of j + s c against x over the batch, and its
    gradient w.r.t. the parameters.  feats: (B, Ci, Z, Y, X); j, x: (B, Z, Y, X);
    s: (B,)."""
    B = feats.shape[0]
    L = 0.0
    acc = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    for k in range(B):
        c, cache = forward(params, feats[k])
        e = j[k] + s[k] * c[0] - x[k]
        nx2 = float((x[k] ** 2).sum())
        L += float((e ** 2).sum()) / nx2 / B
        gout = (2.0 * s[k] / nx2 / B * e)[None]
        gr = backward(params, cache, gout)
        acc = [(a[0] + g[0], a[1] + g[1]) for a, g in zip(acc, gr)]
    return L, acc


def bf16_round(a):
    """Round FP64 values to the nearest bfloat16 (round to nearest even),
    returned as FP64: the weights the CUDA kernels store."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rnd = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rnd) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(v, d, rho, pk, h_over_H, perm, shape):
    """Input channels (5, Z, Y, X) of the network and the scale s for the
    vector v: j = v / d (Helmholtz Jacobi guess), s = rms(j) (1 if j = 0);
    channels j / s, log(d / mean d), p_k / mean p_k - 1, rho / mean rho - 1,
    and the terrain height over the domain height."""
    v, d = np.asarray(v, float), np.asarray(d, float)
    j = v / d
    s = float(np.sqrt(np.mean(j * j)))
    s = s if s > 0.0 else 1.0
    chans = [j / s, np.log(d / d.mean()), pk / np.mean(pk) - 1.0, rho / np.mean(rho) - 1.0,
             np.asarray(h_over_H, float)]
    return np.stack([to_grid(c, shape, perm) for c in chans]), s


def apply_preconditioner(params, v, d, rho, pk, h_over_H, perm, shape):
    """z = D^-1 v + s c(features(v)) in DoF order."""
    f, s = features(v, d, rho, pk, h_over_H, perm, shape)
    c, _ = forward(params, f)
    return np.asarray(v, float) / d + s * to_dof(c[0], perm)


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1; returns
    the new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def unpack(p, layers, channels, cin=5):
    """Split a flat parameter vector (per layer W[co][ci][3][3][3] then b[co])
    into [(W, b)]."""
    out, o = [], 0
    for l in range(layers):
        ci = cin if l == 0 else channels
        co = 1 if l == layers - 1 else channels
        W = np.asarray(p[o:o + co * ci * 27], float).reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = np.asarray(p[o:o + co], float)
        o += co
        out.append((W, b))
    assert o == len(p)
    return out


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])
