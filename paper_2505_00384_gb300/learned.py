"""Training data for the learned preconditioner: pressure systems produced by
the solver itself along IMEX trajectories over terrain.

Host orchestration of library calls only (mesh set-up, trajectories with the
system recorder of ``dgx_imex_step``, ``dgx_learned_add_system``); every
arithmetic step runs in ``libdgx.so``.

Workload (small-box hill flow): a [0, L]^3 box of nx x ny x nz cells of
degree r with periodic lateral faces and slip walls at bottom and top, a
Gal-Chen bell hill h(x, y) = h_c / (1 + ((x - L/2)^2 + (y - L/2)^2) / a_c^2)
centred in the box (the terrain test of Sec. 3, scaled down), isothermal background
at 250 K, initial state background plus a uniform wind u_bar along x,
ARS(2,2,2) steps of dt with K = 2 fixed-point iterations.
"""
from . import dgx
from .inputs import DEFAULT_SEED, uniform

BOX = dict(nx=4, ny=4, nz=4, degree=2, L=1000.0, a_c=1000.0, T=250.0, u_bar=10.0, dt=1.0, K=2)


def hill_heights(count, seed=DEFAULT_SEED, lo=200.0, hi=800.0):
    """Seeded hill heights h_c ~ U[lo, hi] (metres)."""
    return lo + (hi - lo) * uniform(seed, count)


def box_mesh(h_c, box=BOX):
    L = box["L"]
    return dgx.mesh_desc(box["nx"], box["ny"], box["nz"], box["degree"], L, L, L, terrain=1, h_c=float(h_c),
                         a_c=box["a_c"], x_c=L / 2, y_c=L / 2, bc_lateral=2)


def setup_hill(ctx, h_c, box=BOX):
    """Build the hill mesh on ctx with its background and tableau; returns N."""
    dgx.dgx_mesh_build(ctx, box_mesh(h_c, box))
    dgx.dgx_set_background(ctx, dgx.background(kind=0, T=box["T"], u_bar=box["u_bar"]))
    A, At = dgx.ars222()
    dgx.dgx_set_imex(ctx, A, At, box["dt"], box["K"])
    return dgx.dgx_num_dofs(ctx)


def record_trajectory(ctx, steps, stride, box=BOX, tol=1e-11):
    """Run `steps` IMEX steps from the wind-over-hill initial state on the
    current mesh, recording every stride-th pressure system.  Returns a device
    float64 tensor of records (rho, p_k, b, x, a_dt, gamma) and the final state."""
    import torch
    N = dgx.dgx_num_dofs(ctx)
    f64 = torch.float64
    rho = torch.zeros(N, dtype=f64, device="cuda")
    p = torch.zeros(N, dtype=f64, device="cuda")
    dgx.dgx_background_fields(ctx, rho.data_ptr(), p.data_ptr())
    u = torch.zeros(3 * N, dtype=f64, device="cuda")
    u[:N] = box["u_bar"]
    cap = (steps * 2 * box["K"]) // stride + 1
    store = torch.zeros((cap, 4 * N + 2), dtype=f64, device="cuda")
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.restart, o.maxit = dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_HELMHOLTZ, tol, 40, 4000
    dgx.dgx_imex_record(ctx, store.data_ptr(), cap, stride)
    try:
        st, info = dgx.dgx_imex_step(ctx, rho.data_ptr(), u.data_ptr(), p.data_ptr(), steps, o)
        if st != dgx.DGX_OK:
            raise RuntimeError("trajectory: a pressure solve did not converge (relres %g)" % info.max_relres)
        n = dgx.dgx_imex_recorded(ctx)
    finally:
        dgx.dgx_imex_record(ctx, 0, 0, 1)
    return store[:n].clone(), (rho, u, p)


def split_record(rec, N):
    """Views (rho, p_k, b, x) and scalars (a_dt, gamma) of one record."""
    return rec[:N], rec[N:2 * N], rec[2 * N:3 * N], rec[3 * N:4 * N], float(rec[4 * N]), float(rec[4 * N + 1])


def add_records(ctx, records, pairs, stride, test=False):
    """Turn recorded systems of the current mesh into training pairs."""
    N = dgx.dgx_num_dofs(ctx)
    for k in range(records.shape[0]):
        rho, pk, b, x, a_dt, gamma = split_record(records[k], N)
        dgx.dgx_learned_add_system(ctx, rho.data_ptr(), pk.data_ptr(), a_dt, gamma, b.data_ptr(), x.data_ptr(),
                                   pairs=pairs, stride=stride, test=test)


def add_random_systems(ctx, records, per_record, pairs, stride, seed, test=False):
    """For the coefficients of each recorded system, systems S y = b with a
    known solution y of seeded white noise (b = S y by the library's
    operator), turned into pairs like add_records: (S y, y) and the residual /
    error pairs of Jacobi FGMRES cycles on it.  They show the network inputs
    of every roughness, from white noise to the smooth late residuals."""
    import torch
    from .inputs import normal
    N = dgx.dgx_num_dofs(ctx)
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    b = torch.empty_like(y)
    for k in range(records.shape[0]):
        rho, pk, _, _, a_dt, gamma = split_record(records[k], N)
        dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), a_dt, gamma)
        for j in range(per_record):
            y.copy_(torch.from_numpy(normal(seed + 1000 * k + j, N)))
            dgx.dgx_apply_operator(ctx, dgx.DGX_F64, y.data_ptr(), b.data_ptr())
            dgx.dgx_learned_add_system(ctx, rho.data_ptr(), pk.data_ptr(), a_dt, gamma, b.data_ptr(), y.data_ptr(),
                                       pairs=pairs, stride=stride, test=test)


def collect(ctx, heights, steps, record_stride, pairs, pair_stride, test_hills=(), random_per_record=0,
            seed=DEFAULT_SEED, box=BOX):
    """For each hill height: build its mesh, run a trajectory and add its
    systems as pairs (held out when its index is in test_hills), plus
    random_per_record white-noise systems per recorded system.  Returns
    {hill index: records tensor} of the held-out hills (for solve timing)."""
    held = {}
    for i, h in enumerate(heights):
        setup_hill(ctx, h, box)
        recs, _ = record_trajectory(ctx, steps, record_stride, box)
        add_records(ctx, recs, pairs, pair_stride, test=i in test_hills)
        if random_per_record:
            add_random_systems(ctx, recs, random_per_record, pairs, pair_stride, seed + 7919 * i,
                               test=i in test_hills)
        if i in test_hills:
            held[i] = recs
    return held
