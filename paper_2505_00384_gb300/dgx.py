"""Python binding of the dgx C ABI (``include/dgx.h``): argument marshalling only.

Every function has the name of the C entry point it wraps and takes plain
integers (device pointers, e.g. ``tensor.data_ptr()``) or ctypes structures.
All arithmetic of the solver runs in the CUDA kernels of ``libdgx.so``; there
is no CPU fallback: loading fails loudly if the library is missing.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgx.so")

DGX_OK = 0
DGX_NOT_CONVERGED = 1
DGX_FALLBACK_USED = 2
DGX_ERR_ARG = -1
DGX_ERR_OOM = -2
DGX_ERR_CUDA = -3
DGX_ERR_BREAKDOWN = -4
DGX_ERR_DEVICE_TIMEOUT = -5
DGX_ERR_STATE = -6

DGX_F64, DGX_F32 = 0, 1
DGX_PC_NONE, DGX_PC_HELMHOLTZ, DGX_PC_INTERNAL_ENERGY, DGX_PC_LEARNED, DGX_PC_MULTIGRID = 0, 1, 2, 3, 4
DGX_SOLVER_FGMRES, DGX_SOLVER_CG, DGX_SOLVER_MIXED = 0, 1, 2
DGX_MASS_FAST, DGX_MASS_CONSISTENT = 0, 1


class dgx_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("degree", C.c_int), ("n_q", C.c_int),
                ("terrain", C.c_int), ("bc_lateral", C.c_int), ("reserved", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("h_c", C.c_double), ("a_c", C.c_double), ("x_c", C.c_double), ("y_c", C.c_double),
                ("refine", C.c_int * 6)]


class dgx_background(C.Structure):
    _fields_ = [("kind", C.c_int), ("reserved", C.c_int), ("T", C.c_double), ("p0", C.c_double),
                ("N_bv", C.c_double), ("R", C.c_double), ("gamma", C.c_double), ("g", C.c_double),
                ("u_bar", C.c_double)]


class dgx_solve_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("pc", C.c_int), ("restart", C.c_int), ("maxit", C.c_int),
                ("tol", C.c_double), ("inner_restart", C.c_int), ("inner_maxit", C.c_int),
                ("inner_tol", C.c_double), ("use_x0", C.c_int), ("reserved", C.c_int)]


class dgx_mg_opts(C.Structure):
    _fields_ = [("levels", C.c_int), ("degree", C.c_int), ("power_its", C.c_int), ("coarse_maxit", C.c_int),
                ("coarse_solver", C.c_int), ("reserved", C.c_int), ("smooth_range", C.c_double),
                ("coarse_tol", C.c_double)]


class dgx_step_info(C.Structure):
    _fields_ = [("steps", C.c_int), ("solves", C.c_int), ("krylov_iterations", C.c_int),
                ("inner_iterations", C.c_int), ("operator_f64", C.c_int), ("operator_f32", C.c_int),
                ("status", C.c_int), ("reserved", C.c_int), ("max_relres", C.c_double), ("seconds", C.c_double),
                ("seconds_solve", C.c_double)]


class dgx_solve_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("inner_iterations", C.c_int),
                ("operator_f64", C.c_int), ("operator_f32", C.c_int), ("fallback", C.c_int),
                ("relres", C.c_double), ("seconds", C.c_double)]


class dgx_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("lr_final", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double), ("seed", C.c_ulonglong),
                ("shuffle", C.c_int), ("reserved", C.c_int)]


class dgx_train_info(C.Structure):
    _fields_ = [("steps", C.c_int), ("train_samples", C.c_int), ("test_samples", C.c_int), ("reserved", C.c_int),
                ("loss_train0", C.c_double), ("loss_test0", C.c_double), ("loss_train", C.c_double),
                ("loss_test", C.c_double), ("seconds", C.c_double)]


# (name, restype, argtypes) of every entry point declared in include/dgx.h
_P = C.c_void_p
SIGNATURES = [
    ("dgx_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int, _P]),
    ("dgx_destroy", None, [_P]),
    ("dgx_last_error", C.c_char_p, [_P]),
    ("dgx_mesh_build", C.c_int, [_P, C.POINTER(dgx_mesh_desc)]),
    ("dgx_num_dofs", C.c_longlong, [_P]),
    ("dgx_node_coords", C.c_int, [_P, _P]),
    ("dgx_set_background", C.c_int, [_P, C.POINTER(dgx_background)]),
    ("dgx_background_fields", C.c_int, [_P, _P, _P]),
    ("dgx_set_coefficients", C.c_int, [_P, _P, _P, C.c_double, C.c_double]),
    ("dgx_apply_operator", C.c_int, [_P, C.c_int, _P, _P]),
    ("dgx_apply_grad", C.c_int, [_P, C.c_int, _P, _P]),
    ("dgx_apply_div", C.c_int, [_P, C.c_int, _P, _P, _P]),
    ("dgx_apply_mass_inverse", C.c_int, [_P, C.c_int, _P, _P]),
    ("dgx_apply_preconditioner", C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    ("dgx_preconditioner_diagonal", C.c_int, [_P, C.c_int, _P]),
    ("dgx_solve_pressure", C.c_int, [_P, _P, _P, C.POINTER(dgx_solve_opts), C.POINTER(dgx_solve_info)]),
    ("dgx_default_solve_opts", None, [C.POINTER(dgx_solve_opts)]),
    ("dgx_operator_cost", C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("dgx_kernel_launches", C.c_longlong, []),
    ("dgx_operator_threads", C.c_int, [_P, C.c_int]),
    ("dgx_default_mg_opts", None, [C.POINTER(dgx_mg_opts)]),
    ("dgx_mg_setup", C.c_int, [_P, C.POINTER(dgx_mg_opts)]),
    ("dgx_mg_vcycle", C.c_int, [_P, _P, _P]),
    ("dgx_mg_levels", C.c_int, [_P, C.POINTER(C.c_int), _P, C.c_int]),
    ("dgx_operator_variant", C.c_int, [_P, C.c_int]),
    ("dgx_set_operator_variant", C.c_int, [_P, C.c_int, C.c_int]),
    ("dgx_set_explicit_variant", C.c_int, [_P, C.c_int]),
    ("dgx_explicit_variant", C.c_int, [_P]),
    ("dgx_basis_tables", C.c_int, [C.c_int, _P, C.c_int]),
    ("dgx_set_mass_rule", C.c_int, [_P, C.c_int, C.c_double, C.c_int]),
    ("dgx_mass_cg_stats", C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("dgx_apply_operator_noalloc", C.c_int, [_P, C.c_int, _P, _P]),
    ("dgx_set_imex", C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int]),
    ("dgx_explicit_tendencies", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("dgx_apply_mass", C.c_int, [_P, _P, _P, _P]),
    ("dgx_kinetic_mass", C.c_int, [_P, _P, _P, _P]),
    ("dgx_imex_step", C.c_int, [_P, _P, _P, _P, C.c_int, C.POINTER(dgx_solve_opts), C.POINTER(dgx_step_info)]),
    ("dgx_ensemble_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int, _P, C.c_int, C.POINTER(dgx_mesh_desc)]),
    ("dgx_ensemble_destroy", None, [_P]),
    ("dgx_ensemble_last_error", C.c_char_p, [_P]),
    ("dgx_ensemble_num_dofs", C.c_longlong, [_P, C.c_int]),
    ("dgx_ensemble_offset", C.c_longlong, [_P, C.c_int]),
    ("dgx_ensemble_member", C.c_int, [_P, C.c_int, C.POINTER(C.c_void_p)]),
    ("dgx_ensemble_set_coefficients", C.c_int, [_P, _P, _P, C.c_double, C.c_double]),
    ("dgx_ensemble_apply_operator", C.c_int, [_P, C.c_int, _P, _P]),
    ("dgx_ensemble_autotune", C.c_int, [_P]),
    ("dgx_ensemble_tile", C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("dgx_ensemble_tuning", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
    ("dgx_ensemble_solve", C.c_int, [_P, _P, _P, C.POINTER(dgx_solve_opts), C.POINTER(dgx_solve_info)]),
    ("dgx_imex_record", C.c_int, [_P, _P, C.c_int, C.c_int]),
    ("dgx_imex_recorded", C.c_int, [_P]),
    ("dgx_learned_create", C.c_int, [_P, C.c_int, C.c_int, C.c_ulonglong]),
    ("dgx_learned_num_params", C.c_longlong, [_P]),
    ("dgx_learned_get_params", C.c_int, [_P, _P]),
    ("dgx_learned_set_params", C.c_int, [_P, _P]),
    ("dgx_learned_apply", C.c_int, [_P, C.c_int, _P, _P]),
    ("dgx_learned_add_system", C.c_int, [_P, _P, _P, C.c_double, C.c_double, _P, _P, C.c_int, C.c_int, C.c_int]),
    ("dgx_learned_num_samples", C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("dgx_learned_sample", C.c_int, [_P, C.c_int, _P]),
    ("dgx_learned_clear_samples", C.c_int, [_P]),
    ("dgx_learned_loss", C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_double), _P]),
    ("dgx_learned_train", C.c_int, [_P, C.POINTER(dgx_train_opts), C.POINTER(dgx_train_info)]),
    ("dgx_default_train_opts", None, [C.POINTER(dgx_train_opts)]),
]

_lib = None


def load(build_if_missing=True):
    """Load libdgx.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdgx.so not found at %s: build it with __graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class DgxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dgx error %d: %s" % (code, msg))
        self.code = code


def _check(ctx, rc, allow=(DGX_OK,)):
    if rc in allow:
        return rc
    msg = load().dgx_last_error(ctx).decode() if ctx else ""
    raise DgxError(rc, msg)


# ---------------------------------------------------------------- same-name wrappers
def dgx_create(device=0, stream=0):
    h = C.c_void_p()
    rc = load().dgx_create(C.byref(h), int(device), C.c_void_p(int(stream) or None))
    if rc != DGX_OK:
        raise DgxError(rc, "dgx_create failed (device %d)" % device)
    return h


def dgx_destroy(ctx):
    load().dgx_destroy(ctx)


def dgx_last_error(ctx):
    return load().dgx_last_error(ctx).decode()


def dgx_mesh_build(ctx, desc):
    return _check(ctx, load().dgx_mesh_build(ctx, C.byref(desc)))


def dgx_num_dofs(ctx):
    return int(load().dgx_num_dofs(ctx))


def dgx_node_coords(ctx, X_ptr):
    return _check(ctx, load().dgx_node_coords(ctx, C.c_void_p(X_ptr)))


def dgx_set_background(ctx, bg):
    return _check(ctx, load().dgx_set_background(ctx, C.byref(bg)))


def dgx_background_fields(ctx, rho_ptr, p_ptr):
    return _check(ctx, load().dgx_background_fields(ctx, C.c_void_p(rho_ptr), C.c_void_p(p_ptr)))


def dgx_set_coefficients(ctx, rho_ptr, pk_ptr, a_dt, gamma=1.4):
    return _check(ctx, load().dgx_set_coefficients(ctx, C.c_void_p(rho_ptr), C.c_void_p(pk_ptr), float(a_dt),
                                                   float(gamma)))


def dgx_apply_operator(ctx, prec, x_ptr, y_ptr):
    return _check(ctx, load().dgx_apply_operator(ctx, prec, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def dgx_apply_grad(ctx, prec, p_ptr, V_ptr):
    return _check(ctx, load().dgx_apply_grad(ctx, prec, C.c_void_p(p_ptr), C.c_void_p(V_ptr)))


def dgx_apply_div(ctx, prec, V_ptr, p_ptr, y_ptr):
    return _check(ctx, load().dgx_apply_div(ctx, prec, C.c_void_p(V_ptr), C.c_void_p(p_ptr), C.c_void_p(y_ptr)))


def dgx_apply_mass_inverse(ctx, prec, in_ptr, out_ptr):
    return _check(ctx, load().dgx_apply_mass_inverse(ctx, prec, C.c_void_p(in_ptr), C.c_void_p(out_ptr)))


def dgx_apply_preconditioner(ctx, pc, prec, x_ptr, y_ptr):
    return _check(ctx, load().dgx_apply_preconditioner(ctx, pc, prec, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def dgx_preconditioner_diagonal(ctx, pc, d_ptr):
    return _check(ctx, load().dgx_preconditioner_diagonal(ctx, pc, C.c_void_p(d_ptr)))


def dgx_default_mg_opts():
    o = dgx_mg_opts()
    load().dgx_default_mg_opts(C.byref(o))
    return o


def dgx_mg_setup(ctx, opts=None):
    """Build the geometric-multigrid hierarchy for the current mesh and coefficients."""
    return _check(ctx, load().dgx_mg_setup(ctx, C.byref(opts) if opts is not None else None))


def dgx_mg_vcycle(ctx, r_ptr, z_ptr):
    """z = one V-cycle applied to r (device FP64)."""
    return _check(ctx, load().dgx_mg_vcycle(ctx, C.c_void_p(r_ptr), C.c_void_p(z_ptr)))


def dgx_mg_levels(ctx, capacity=12):
    """(levels, [lambda_max of each level])."""
    n = C.c_int()
    lam = (C.c_double * capacity)()
    _check(ctx, load().dgx_mg_levels(ctx, C.byref(n), lam, capacity))
    return n.value, [lam[i] for i in range(min(n.value, capacity))]


def dgx_default_solve_opts():
    o = dgx_solve_opts()
    load().dgx_default_solve_opts(C.byref(o))
    return o


def dgx_solve_pressure(ctx, b_ptr, x_ptr, opts=None):
    """Returns (status, dgx_solve_info); raises DgxError on errors (< 0)."""
    o = opts if opts is not None else dgx_default_solve_opts()
    info = dgx_solve_info()
    rc = load().dgx_solve_pressure(ctx, C.c_void_p(b_ptr), C.c_void_p(x_ptr), C.byref(o), C.byref(info))
    _check(ctx, rc, allow=(DGX_OK, DGX_NOT_CONVERGED, DGX_FALLBACK_USED))
    return rc, info


def dgx_operator_cost(ctx):
    """(flops of the gradient kernel, flops of the divergence kernel, HBM floor bytes in FP64)."""
    f1, f2, b64 = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, load().dgx_operator_cost(ctx, C.byref(f1), C.byref(f2), C.byref(b64)))
    return f1.value, f2.value, b64.value


def dgx_apply_operator_noalloc(ctx, prec, x_ptr, y_ptr):
    """y = S x with the scratch in the library's fixed static device array
    (no allocation; N limited by DGX_NOALLOC_SCRATCH_BYTES)."""
    return _check(ctx, load().dgx_apply_operator_noalloc(ctx, prec, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


DGX_NOALLOC_SCRATCH_BYTES = 16 << 20


def dgx_set_imex(ctx, A, At, dt, K=2):
    """A, At: host (s, s) float64 arrays (numpy)."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float64)
    At = np.ascontiguousarray(At, dtype=np.float64)
    s = A.shape[0]
    return _check(ctx, load().dgx_set_imex(ctx, s, A.ctypes.data_as(C.c_void_p), At.ctypes.data_as(C.c_void_p),
                                           float(dt), int(K)))


def dgx_explicit_tendencies(ctx, rho_ptr, u_ptr, Erho_ptr, Em_ptr, Ee_ptr):
    return _check(ctx, load().dgx_explicit_tendencies(ctx, C.c_void_p(rho_ptr), C.c_void_p(u_ptr),
                                                      C.c_void_p(Erho_ptr), C.c_void_p(Em_ptr), C.c_void_p(Ee_ptr)))


def dgx_apply_mass(ctx, rho_ptr, in_ptr, out_ptr):
    return _check(ctx, load().dgx_apply_mass(ctx, C.c_void_p(rho_ptr), C.c_void_p(in_ptr), C.c_void_p(out_ptr)))


def dgx_kinetic_mass(ctx, rho_ptr, u_ptr, out_ptr):
    return _check(ctx, load().dgx_kinetic_mass(ctx, C.c_void_p(rho_ptr), C.c_void_p(u_ptr), C.c_void_p(out_ptr)))


def dgx_imex_step(ctx, rho_ptr, u_ptr, p_ptr, nsteps=1, opts=None):
    """Returns (status, dgx_step_info); raises DgxError on errors (< 0)."""
    o = opts if opts is not None else dgx_default_solve_opts()
    info = dgx_step_info()
    rc = load().dgx_imex_step(ctx, C.c_void_p(rho_ptr), C.c_void_p(u_ptr), C.c_void_p(p_ptr), int(nsteps),
                              C.byref(o), C.byref(info))
    _check(ctx, rc, allow=(DGX_OK, DGX_NOT_CONVERGED))
    return rc, info


def dgx_imex_record(ctx, store_ptr, capacity, stride=1):
    """Record every stride-th pressure system of dgx_imex_step into a device
    buffer of capacity x (4 N + 2) float64: rho, p_k, b, x, a_dt, gamma."""
    return _check(ctx, load().dgx_imex_record(ctx, C.c_void_p(store_ptr), int(capacity), int(stride)))


def dgx_imex_recorded(ctx):
    return load().dgx_imex_recorded(ctx)


# ---------------------------------------------------------------- learned preconditioner
DGX_LEARNED_CHANNELS = 5  # input channels; a stored sample holds these plus the target


def dgx_learned_create(ctx, layers, channels, seed=20250501):
    return _check(ctx, load().dgx_learned_create(ctx, int(layers), int(channels), C.c_ulonglong(seed)))


def dgx_learned_num_params(ctx):
    return load().dgx_learned_num_params(ctx)


def dgx_learned_get_params(ctx):
    """FP32 master parameters as a numpy array (host)."""
    import numpy as np
    out = np.empty(dgx_learned_num_params(ctx), dtype=np.float32)
    _check(ctx, load().dgx_learned_get_params(ctx, out.ctypes.data_as(C.c_void_p)))
    return out


def dgx_learned_set_params(ctx, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != dgx_learned_num_params(ctx):
        raise ValueError("expected %d parameters, got %d" % (dgx_learned_num_params(ctx), p.size))
    return _check(ctx, load().dgx_learned_set_params(ctx, p.ctypes.data_as(C.c_void_p)))


def dgx_learned_apply(ctx, prec, v_ptr, z_ptr):
    return _check(ctx, load().dgx_learned_apply(ctx, prec, C.c_void_p(v_ptr), C.c_void_p(z_ptr)))


def dgx_learned_add_system(ctx, rho_ptr, pk_ptr, a_dt, gamma, b_ptr, x_ptr, pairs=1, stride=4, test=False):
    return _check(ctx, load().dgx_learned_add_system(ctx, C.c_void_p(rho_ptr), C.c_void_p(pk_ptr), float(a_dt),
                                                     float(gamma), C.c_void_p(b_ptr), C.c_void_p(x_ptr), int(pairs),
                                                     int(stride), int(bool(test))))


def dgx_learned_num_samples(ctx):
    tr, te = C.c_int(), C.c_int()
    _check(ctx, load().dgx_learned_num_samples(ctx, C.byref(tr), C.byref(te)))
    return tr.value, te.value


def dgx_learned_sample(ctx, i, grid_points):
    """Sample i as a (6, G) float32 numpy array: channels 0..4, then the target."""
    import numpy as np
    out = np.empty((DGX_LEARNED_CHANNELS + 1, grid_points), dtype=np.float32)
    _check(ctx, load().dgx_learned_sample(ctx, int(i), out.ctypes.data_as(C.c_void_p)))
    return out


def dgx_learned_clear_samples(ctx):
    return _check(ctx, load().dgx_learned_clear_samples(ctx))


def dgx_learned_loss(ctx, first, count, want_grad=True):
    """(mean loss, gradient as float32 numpy array or None) over samples first..first+count-1."""
    import numpy as np
    loss = C.c_double()
    g = np.empty(dgx_learned_num_params(ctx), dtype=np.float32) if want_grad else None
    _check(ctx, load().dgx_learned_loss(ctx, int(first), int(count), C.byref(loss),
                                        g.ctypes.data_as(C.c_void_p) if g is not None else None))
    return loss.value, g


def dgx_default_train_opts():
    o = dgx_train_opts()
    load().dgx_default_train_opts(C.byref(o))
    return o


def dgx_learned_train(ctx, opts=None):
    o = opts if opts is not None else dgx_default_train_opts()
    info = dgx_train_info()
    _check(ctx, load().dgx_learned_train(ctx, C.byref(o), C.byref(info)))
    return info


def _echeck(e, rc, allow=(DGX_OK,)):
    if rc in allow:
        return rc
    raise DgxError(rc, load().dgx_ensemble_last_error(e).decode() if e else "")


def dgx_ensemble_create(device, stream, descs):
    """descs: list of dgx_mesh_desc.  Returns the ensemble handle."""
    arr = (dgx_mesh_desc * len(descs))(*descs)
    h = C.c_void_p()
    rc = load().dgx_ensemble_create(C.byref(h), int(device), C.c_void_p(int(stream) or None), len(descs), arr)
    if rc != DGX_OK:
        msg = load().dgx_ensemble_last_error(h).decode() if h else ""
        if h:
            load().dgx_ensemble_destroy(h)
        raise DgxError(rc, "dgx_ensemble_create: " + msg)
    return h


def dgx_ensemble_destroy(e):
    load().dgx_ensemble_destroy(e)


def dgx_ensemble_num_dofs(e, m=-1):
    return int(load().dgx_ensemble_num_dofs(e, m))


def dgx_ensemble_offset(e, m):
    return int(load().dgx_ensemble_offset(e, m))


def dgx_ensemble_member(e, m):
    h = C.c_void_p()
    _echeck(e, load().dgx_ensemble_member(e, m, C.byref(h)))
    return h


def dgx_ensemble_set_coefficients(e, rho_ptr, pk_ptr, a_dt, gamma=1.4):
    return _echeck(e, load().dgx_ensemble_set_coefficients(e, C.c_void_p(rho_ptr), C.c_void_p(pk_ptr), float(a_dt),
                                                           float(gamma)))


def dgx_ensemble_apply_operator(e, prec, x_ptr, y_ptr):
    return _echeck(e, load().dgx_ensemble_apply_operator(e, prec, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def dgx_ensemble_autotune(e):
    return _echeck(e, load().dgx_ensemble_autotune(e))


def dgx_ensemble_tuning(e, g):
    v = [C.c_int() for _ in range(4)]
    _echeck(e, load().dgx_ensemble_tuning(e, g, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def dgx_ensemble_tile(e, g, prec=DGX_F32):
    """(fused, cells per CTA) of the kernels the autotuner chose for degree group g and prec."""
    f, v = C.c_int(), C.c_int()
    _echeck(e, load().dgx_ensemble_tile(e, g, int(prec), C.byref(f), C.byref(v)))
    return f.value, v.value


def dgx_ensemble_solve(e, b_ptr, x_ptr, n_members, opts=None):
    """Returns (status, [dgx_solve_info per member])."""
    o = opts if opts is not None else dgx_default_solve_opts()
    infos = (dgx_solve_info * n_members)()
    rc = load().dgx_ensemble_solve(e, C.c_void_p(b_ptr), C.c_void_p(x_ptr), C.byref(o), infos)
    _echeck(e, rc, allow=(DGX_OK, DGX_NOT_CONVERGED))
    return rc, list(infos)


def ars222():
    """ARS(2,2,2) companion tableaux (A explicit, At implicit), gamma = 1 - 1/sqrt(2)."""
    import numpy as np
    g = 1.0 - 1.0 / np.sqrt(2.0)
    d = 1.0 - 1.0 / (2.0 * g)
    A = np.array([[0, 0, 0], [g, 0, 0], [d, 1 - d, 0]], dtype=np.float64)
    At = np.array([[0, 0, 0], [0, g, 0], [0, 1 - g, g]], dtype=np.float64)
    return A, At


def dgx_basis_tables(degree):
    """The host-built 1D tables of a degree (host only, no GPU): a dict of
    numpy arrays I, D, IT, DT, Ia, P, PT, IIT, DDT, IDT, wq, wa, gq."""
    import numpy as np
    n = load().dgx_basis_tables(int(degree), None, 0)
    if n < 0:
        raise DgxError(n, "unsupported degree %d" % degree)
    buf = np.zeros(n)
    load().dgx_basis_tables(int(degree), buf.ctypes.data_as(C.c_void_p), n)
    N, Q = degree + 1, 2 * degree + 1
    out, o = {}, 0
    for name, shape in [("I", (Q, N)), ("D", (Q, N)), ("IT", (N, Q)), ("DT", (N, Q)), ("Ia", (N, N)), ("P", (N, N)),
                        ("PT", (N, N)), ("IIT", (N, Q)), ("DDT", (N, Q)), ("IDT", (N, Q)), ("wq", (Q,)),
                        ("wa", (N,)), ("gq", (Q,))]:
        k = int(np.prod(shape))
        out[name] = buf[o:o + k].reshape(shape)
        o += k
    assert o == n
    return out


def dgx_set_mass_rule(ctx, rule, cg_tol=1e-13, cg_maxit=50):
    """Quadrature of the density-weighted mass for every use in ctx: DGX_MASS_FAST
    (r+1 points, fast inverse) or DGX_MASS_CONSISTENT (2r+1 points, per-cell PCG)."""
    return _check(ctx, load().dgx_set_mass_rule(ctx, int(rule), float(cg_tol), int(cg_maxit)))


def dgx_mass_cg_stats(ctx):
    """(largest PCG iteration count, unconverged cell solves) since the previous call."""
    it, bad = C.c_int(), C.c_int()
    _check(ctx, load().dgx_mass_cg_stats(ctx, C.byref(it), C.byref(bad)))
    return it.value, bad.value


DGX_OP_VARIANTS = 7


def dgx_operator_variant(ctx, prec):
    """Launch variant of the operator kernels in use for prec (-1: the default)."""
    return load().dgx_operator_variant(ctx, prec)


def dgx_set_explicit_variant(ctx, variant):
    """Explicit fluxes in double-words (1, default) or on the FP64 pipe (0)."""
    return _check(ctx, load().dgx_set_explicit_variant(ctx, int(variant)))


def dgx_explicit_variant(ctx):
    return load().dgx_explicit_variant(ctx)


def dgx_set_operator_variant(ctx, prec, variant):
    """Pin launch variant 0..6 for prec on the current mesh, or -1 for the autotuner."""
    return _check(ctx, load().dgx_set_operator_variant(ctx, int(prec), int(variant)))


def dgx_operator_threads(ctx, prec):
    """Threads per CTA of the operator kernels chosen by the autotuner (0 = default)."""
    return load().dgx_operator_threads(ctx, prec)


def dgx_kernel_launches():
    return int(load().dgx_kernel_launches())


def mesh_desc(nx, ny, nz, degree, Lx, Ly, Lz, terrain=0, h_c=0.0, a_c=1000.0, x_c=None, y_c=None, bc_lateral=0,
              refine=None):
    d = dgx_mesh_desc()
    d.nx, d.ny, d.nz, d.degree, d.n_q = nx, ny, nz, degree, 0
    d.terrain, d.bc_lateral = terrain, bc_lateral
    d.Lx, d.Ly, d.Lz = Lx, Ly, Lz
    d.h_c, d.a_c = h_c, a_c
    d.x_c = Lx / 2 if x_c is None else x_c
    d.y_c = Ly / 2 if y_c is None else y_c
    if refine is not None:
        for i, v in enumerate(refine):
            d.refine[i] = int(v)
    return d


def background(kind=0, T=250.0, p0=1e5, N_bv=0.01, R=287.0, gamma=1.4, g=9.81, u_bar=10.0):
    b = dgx_background()
    b.kind, b.T, b.p0, b.N_bv, b.R, b.gamma, b.g, b.u_bar = kind, T, p0, N_bv, R, gamma, g, u_bar
    return b
