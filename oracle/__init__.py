"""FP64 CPU oracle of the IMEX-DG pressure operator and IMEX step.

TEST INFRASTRUCTURE.  The oracle is the independent, plain and slow checker
of the CUDA library (arXiv:2505.00384, Sec. 2 and Sec. 3).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path and
the CUDA path never imports it.

This module is argument marshalling only (ctypes over ``liboracle.so``, built
from ``orc.c`` / ``orc_imex.c`` on first use) plus small dense-algebra helpers
used by the pinning tests.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcMesh(C.Structure):
    """Mirror of ``orc_mesh`` in orc.c."""

    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("r", C.c_int), ("q", C.c_int), ("terrain", C.c_int), ("bc_lateral", C.c_int), ("pad", C.c_int),
        ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
        ("hc", C.c_double), ("ac", C.c_double), ("xc", C.c_double), ("yc", C.c_double),
        ("ref", C.c_int * 6),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_mesh(nx, ny, nz, r, Lx=1000.0, Ly=1000.0, Lz=1000.0, q=None, terrain=0, hc=0.0, ac=1000.0,
              xc=None, yc=None, bc_lateral=0, refine=None):
    """Structured hexahedral mesh on [0,Lx]x[0,Ly]x[0,Lz] (terrain-following
    in z when ``terrain`` > 0).  ``q`` defaults to the consistent rule 2r+1.
    ``refine`` = (x0, x1, y0, y1, z0, z1): the base cells of that box are split
    2 x 2 x 2 (a non-conforming mesh with 2:1 hanging faces; the base cells
    first, those in the box without unknowns, then the children)."""
    m = OrcMesh()
    m.nx, m.ny, m.nz, m.r = nx, ny, nz, r
    m.q = 2 * r + 1 if q is None else q
    m.terrain, m.bc_lateral = terrain, bc_lateral
    m.Lx, m.Ly, m.Lz = Lx, Ly, Lz
    m.hc, m.ac = hc, ac
    m.xc = Lx / 2 if xc is None else xc
    m.yc = Ly / 2 if yc is None else yc
    if refine is not None:
        for i, v in enumerate(refine):
            m.ref[i] = int(v)
    return m


def is_refined(m):
    return m.ref[1] > m.ref[0] and m.ref[3] > m.ref[2] and m.ref[5] > m.ref[4]


def num_cells(m):
    n = m.nx * m.ny * m.nz
    if is_refined(m):
        n += 8 * (m.ref[1] - m.ref[0]) * (m.ref[3] - m.ref[2]) * (m.ref[5] - m.ref[4])
    return n


def dead_cells(m):
    """Indices of the base cells replaced by their children (no unknowns)."""
    if not is_refined(m):
        return np.zeros(0, dtype=np.int64)
    z, y, x = np.meshgrid(np.arange(m.ref[4], m.ref[5]), np.arange(m.ref[2], m.ref[3]),
                          np.arange(m.ref[0], m.ref[1]), indexing="ij")
    return (x + m.nx * (y + m.ny * z)).reshape(-1)


def active_mask(m):
    """Per-DoF flag: 1 where the mesh has unknowns."""
    a = np.ones(num_cells(m), dtype=bool)
    a[dead_cells(m)] = False
    return np.repeat(a, (m.r + 1) ** 3)


def face_info(m, cell, f):
    """(relation, neighbours) of face f of a cell: -1 boundary, 0 conforming,
    1 base cell's hanging face (four children), 2 child's hanging face (base
    cell, child position), 3 dead cell."""
    nb = (C.c_long * 4)()
    rel = lib().orc_face_info(C.byref(m), C.c_long(cell), f, nb)
    return rel, list(nb)


def ndofs(m):
    return num_cells(m) * (m.r + 1) ** 3


def gauss(q):
    x = np.zeros(q); w = np.zeros(q)
    assert lib().orc_gauss(q, _dp(x), _dp(w)) == 0
    return x, w


def gll(n):
    x = np.zeros(n); w = np.zeros(n)
    assert lib().orc_gll(n, _dp(x), _dp(w)) == 0
    return x, w


def lagrange(nodes, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    n = len(nodes)
    l = np.zeros(n); dl = np.zeros(n)
    lib().orc_lagrange(n, _dp(nodes), C.c_double(x), _dp(l), _dp(dl))
    return l, dl


def terrain_height(m, x, y):
    f = lib().orc_terrain_height
    f.restype = C.c_double
    return f(C.byref(m), C.c_double(x), C.c_double(y))


def node_coords(m):
    X = np.zeros(3 * ndofs(m))
    assert lib().orc_node_coords(C.byref(m), _dp(X)) == 0
    return X.reshape(3, -1)


def apply_B(m, alpha, p):
    out = np.zeros(3 * ndofs(m))
    assert lib().orc_apply_B(C.byref(m), C.c_double(alpha), _dp(np.ascontiguousarray(p, dtype=np.float64)), _dp(out)) == 0
    return out


def _mass(m, rho, V, inverse, consistent):
    out = np.zeros(3 * ndofs(m))
    assert lib().orc_apply_mass(C.byref(m), int(bool(consistent)), int(inverse),
                                _dp(np.ascontiguousarray(rho, dtype=np.float64)),
                                _dp(np.ascontiguousarray(V, dtype=np.float64)), _dp(out)) == 0
    return out


def apply_A(m, rho, V, consistent=False):
    """Density-weighted mass A_rho V (3 components); the r+1 point rule of the
    fast inverse, or the consistent 2r+1 point rule with ``consistent``."""
    return _mass(m, rho, V, 0, consistent)


def apply_Ainv(m, rho, V, consistent=False):
    """A_rho^-1 V with the same choice of rule as apply_A."""
    return _mass(m, rho, V, 1, consistent)


def apply_C(m, alpha, gamma, pk, V):
    out = np.zeros(ndofs(m))
    assert lib().orc_apply_C(C.byref(m), C.c_double(alpha), C.c_double(gamma),
                             _dp(np.ascontiguousarray(pk, dtype=np.float64)),
                             _dp(np.ascontiguousarray(V, dtype=np.float64)), _dp(out)) == 0
    return out


def apply_M(m, f, scale=1.0):
    out = np.zeros(ndofs(m))
    assert lib().orc_apply_M(C.byref(m), C.c_double(scale), _dp(np.ascontiguousarray(f, dtype=np.float64)), _dp(out)) == 0
    return out


def apply_D(m, gamma, p):
    return apply_M(m, p, 1.0 / (gamma - 1.0))


def apply_S(m, alpha, gamma, rho, pk, p, cells=None, consistent=False):
    """y = S p = D p - C A^-1 B p.  With ``cells`` (indices), only those
    cells' entries are computed; the rest of y is NaN.  ``consistent``: A with
    the 2r+1 point rule instead of the fast inverse's r+1 points."""
    N = ndofs(m)
    y = np.zeros(N)
    args = [C.byref(m), int(bool(consistent)), C.c_double(alpha), C.c_double(gamma),
            _dp(np.ascontiguousarray(rho, dtype=np.float64)), _dp(np.ascontiguousarray(pk, dtype=np.float64)),
            _dp(np.ascontiguousarray(p, dtype=np.float64))]
    if cells is None:
        assert lib().orc_apply_S_rule(*args, None, _dp(y)) == 0
        return y
    y[:] = np.nan
    mask = np.zeros(num_cells(m), dtype=np.uint8)
    mask[np.asarray(cells)] = 1
    assert lib().orc_apply_S_rule(*args, mask.ctypes.data_as(C.c_void_p), _dp(y)) == 0
    return y


PC_NONE, PC_HELMHOLTZ, PC_INTERNAL_ENERGY = 0, 1, 2


def precond_diag(m, kind, alpha, gamma, rho, pk):
    d = np.zeros(ndofs(m))
    assert lib().orc_precond_diag(C.byref(m), kind, C.c_double(alpha), C.c_double(gamma),
                                  _dp(np.ascontiguousarray(rho, dtype=np.float64)),
                                  _dp(np.ascontiguousarray(pk, dtype=np.float64)), _dp(d)) == 0
    return d


def solve(m, alpha, gamma, rho, pk, b, method="fgmres", pc=PC_HELMHOLTZ, tol=1e-10, restart=30, maxit=1000, x0=None,
          consistent=False):
    """Solve S x = b.  Returns (x, status, iterations, relative residual).
    ``consistent`` (FGMRES only): S with the 2r+1 point rule for A."""
    N = ndofs(m)
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    pk = np.ascontiguousarray(pk, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    dinv = None
    if pc != PC_NONE:
        dinv = 1.0 / precond_diag(m, pc, alpha, gamma, rho, pk)
    its = C.c_int(0)
    rel = C.c_double(0.0)
    dptr = _dp(dinv) if dinv is not None else None
    if method == "fgmres":
        st = lib().orc_fgmres_rule(C.byref(m), int(bool(consistent)), C.c_double(alpha), C.c_double(gamma),
                                   _dp(rho), _dp(pk), dptr, _dp(b), _dp(x), C.c_double(tol), restart, maxit,
                                   C.byref(its), C.byref(rel))
    elif method == "cg":
        if consistent:
            raise ValueError("CG runs with the fast inverse only")
        st = lib().orc_cg(C.byref(m), C.c_double(alpha), C.c_double(gamma), _dp(rho), _dp(pk), dptr, _dp(b),
                          _dp(x), C.c_double(tol), maxit, C.byref(its), C.byref(rel))
    else:
        raise ValueError(method)
    return x, st, its.value, rel.value


def max_threads():
    return lib().orc_max_threads()


def set_threads(n):
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------- dense helpers
def assemble(apply, n_in, n_out):
    """Dense matrix of a linear map by applying it to unit vectors (the
    unit-vector construction of Sec. 3.1).  For tiny meshes only."""
    Mx = np.zeros((n_out, n_in))
    e = np.zeros(n_in)
    for j in range(n_in):
        e[j] = 1.0
        Mx[:, j] = apply(e)
        e[j] = 0.0
    return Mx


# ---------------------------------------------------------------- IMEX step
class OrcBg(C.Structure):
    """Mirror of ``orc_bg`` in orc_imex.c."""

    _fields_ = [("kind", C.c_int), ("pad", C.c_int), ("T", C.c_double), ("p0", C.c_double), ("Nbv", C.c_double),
                ("R", C.c_double), ("gamma", C.c_double), ("g", C.c_double), ("ubar", C.c_double)]


def make_bg(kind=0, T=250.0, p0=1e5, Nbv=0.01, R=287.0, gamma=1.4, g=9.81, ubar=10.0):
    b = OrcBg()
    b.kind, b.T, b.p0, b.Nbv, b.R, b.gamma, b.g, b.ubar = kind, T, p0, Nbv, R, gamma, g, ubar
    return b


def background(m, bg):
    N = ndofs(m)
    rb, pb = np.zeros(N), np.zeros(N)
    assert lib().orc_background(C.byref(m), C.byref(bg), _dp(rb), _dp(pb)) == 0
    return rb, pb


def explicit(m, bg, rho, u, rho_bar, cells=None):
    """Explicit tendencies (Erho, Em (3N), Ee) as dual vectors; with ``cells``
    only those cells are computed (the rest is NaN)."""
    N = ndofs(m)
    Er, Em, Ee = np.zeros(N), np.zeros(3 * N), np.zeros(N)
    mask = None
    if cells is not None:
        for a in (Er, Em, Ee):
            a[:] = np.nan
        mk = np.zeros(num_cells(m), dtype=np.uint8)
        mk[np.asarray(cells)] = 1
        mask = mk.ctypes.data_as(C.c_void_p)
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    assert lib().orc_explicit_masked(C.byref(m), C.byref(bg), _dp(c(rho)), _dp(c(u)), _dp(c(rho_bar)), mask,
                                     _dp(Er), _dp(Em), _dp(Ee)) == 0
    return Er, Em, Ee


def kinetic_mass(m, rho, u):
    out = np.zeros(ndofs(m))
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    assert lib().orc_kinetic_mass(C.byref(m), _dp(c(rho)), _dp(c(u)), _dp(out)) == 0
    return out


def ars222():
    """ARS(2,2,2) tableaux (explicit A, implicit At), gamma = 1 - 1/sqrt(2)."""
    g = 1.0 - 1.0 / np.sqrt(2.0)
    d = 1.0 - 1.0 / (2.0 * g)
    A = np.array([[0, 0, 0], [g, 0, 0], [d, 1 - d, 0]], dtype=np.float64)
    At = np.array([[0, 0, 0], [0, g, 0], [0, 1 - g, g]], dtype=np.float64)
    return A, At


def imex_step(m, bg, rho, u, p, dt, A=None, At=None, K=2, tol=1e-12, consistent=False):
    """One IMEX step; returns (rho, u, p, status, Krylov iterations).
    ``consistent``: every density-weighted mass and inverse with the 2r+1
    point rule instead of the fast inverse's r+1 points (Sec. 3.3)."""
    if A is None:
        A, At = ars222()
    A = np.ascontiguousarray(A, dtype=np.float64)
    At = np.ascontiguousarray(At, dtype=np.float64)
    r = np.array(rho, dtype=np.float64)
    v = np.array(u, dtype=np.float64)
    q = np.array(p, dtype=np.float64)
    its = C.c_int(0)
    st = lib().orc_imex_step_rule(C.byref(m), int(bool(consistent)), C.byref(bg), A.shape[0], _dp(A), _dp(At),
                                  C.c_double(dt), int(K), C.c_double(tol), _dp(r), _dp(v), _dp(q), C.byref(its))
    return r, v, q, st, its.value
