#!/usr/bin/env python3
"""Benchmark of the GB300 IMEX-DG hot path (one JSON line on rank 0).

Workload: flow over a bell-shaped hill (h = 400 m / (1 + r^2/(1 km)^2) at the
domain centre) on a terrain-following 60 x 60 x 20 km mesh of 64 x 64 x 32
cells at degree 4 (16 384 000 DoFs per scalar field), far-field lateral
boundaries (uniform 10 m/s inflow: the ghost state is the background plus the
wind), slip walls at bottom and top, isothermal background at 250 K, initial
state = background plus a uniform 10 m/s wind, dt = 1 s, ARS(2,2,2) with two
fixed-point iterations per implicit stage.  Synthetic inputs.

One step = one IMEX step through the public API (dgx_imex_step): explicit
fluxes, stage assembly, four Helmholtz pressure solves to 1e-8 FP64 relative
residual with the mixed-precision solver (FP32 GMRES inside FP64 flexible
GMRES), velocity recovery.  The metric is seconds per step (lower is better);
the same step with plain FP64 FGMRES solves and the operator throughput
(vmult GDoF/s) are reported beside it.  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pressure solve s/step @1e-8 rel residual (mixed/learned vs plain FP64); vmult GDoF/s"

FULL = dict(name="hill_64x64x32_r4_16.4M_dofs_imex", nx=64, ny=64, nz=32, r=4, Lx=60000.0, Ly=60000.0, Lz=20000.0)
SMALL = dict(name="hill_16x16x8_r4_256k_dofs_imex", nx=16, ny=16, nz=8, r=4, Lx=15000.0, Ly=15000.0, Lz=5000.0)
COMMON = dict(terrain=1, hc=400.0, ac=1000.0, bc_lateral=1, T=250.0, p0=1e5, R=287.0, g=9.81, gamma=1.4, dt=1.0,
              ubar=10.0, K=2)
A_LL = 1.0 - 1.0 / 2.0 ** 0.5
# FP64 operator applications of one IMEX step of this workload with plain FP64 FGMRES(30) solves to 1e-8
# (four solves), and the other operator-type kernel calls of a step (velocity recovery, -C A^-1 F, stage
# terms, counted as half applications); used only to scale the oracle's sampled cost to a step.
PLAIN_STEP_APPLIES = 138
STEP_EXTRA_HALF_APPLIES = 12
# DRAM bytes per DoF of one launch of the operator kernels, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum) on the 48x48x24 r=4 hill mesh
# (6 912 000 DoFs, inputs larger than L2); one launch reads each cell's data once,
# so the traffic scales with the DoFs.  k_div / kf_div<df64> as applied inside the
# solver (with the per-coefficient-set kappa at the Gauss points); the fused kernels
# in the configuration the autotuner picks on the 64x64x32 mesh.  Valid for the
# kernels as captured.
DRAM_BYTES_PER_DOF_F64 = {"k_div<double>": 696.2e6 / 6912000, "k_grad<double>": 252.9e6 / 6912000,
                          "kf_div<df64>": 688.5e6 / 6912000, "kf_grad<df64>": 245.5e6 / 6912000,
                          "kf_div<float>": 162.2e6 / 6912000, "kf_grad<float>": 94.1e6 / 6912000}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="small mesh")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vmult-reps", type=int, default=10)
    ap.add_argument("--mesh", default=None, help="NXxNYxNZ cells at the same cell size as the 64x64x32 workload")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed steps (for profiler launch lists); no side measurements")
    ap.add_argument("--variant-f64", type=int, default=None, help="vmult workload: pin this FP64 launch variant")
    ap.add_argument("--variant-f32", type=int, default=None, help="vmult workload: pin this FP32 launch variant")
    ap.add_argument("--workload", default="hill",
                    choices=["hill", "ensemble", "learned", "mixed", "paper", "consistent", "vmult", "mg", "nonconf"],
                    help="hill: one IMEX step of the 64x64x32 hill (default); ensemble: 16-member batched solve; "
                         "learned: pressure solves of held-out hill systems with the trained network; "
                         "mixed: mixed-precision solves on the 4x4x4 box at degrees 2, 3, 5 against the oracle; "
                         "paper: the Sec. 3 test case (120x80x32 cells, r = 4, stratified), Helmholtz vs "
                         "internal-energy Jacobi; consistent: fast vs consistent density-weighted mass "
                         "(Sec. 3.3) on the 60x40x16 r = 4 mesh; nonconf: the Sec. 3 domain on a non-conforming "
                         "mesh (2:1 refined box around the hill), Helmholtz vs internal-energy Jacobi")
    ap.add_argument("--epochs", type=int, default=100, help="learned workload: training epochs (batch 32)")
    ap.add_argument("--members", type=int, default=16, help="ensemble members (first k of the 16)")
    ap.add_argument("--inner-maxit", type=int, default=None, help="override the FP32 GMRES cycle length")
    ap.add_argument("--inner-tol", type=float, default=None, help="override the FP32 GMRES tolerance")
    ap.add_argument("--plain-steps", type=int, default=3, help="hill workload: timed steps with plain FP64 solves")
    ap.add_argument("--paper-steps", type=int, default=0,
                    help="paper / nonconf workloads: after the solver comparison, this many consecutive mixed-solver "
                         "IMEX steps from the initial state (simulated time = steps x 1 s)")
    ap.add_argument("--no-extras", action="store_true",
                    help="hill workload: skip the compact mixed and learned results (run as subprocesses)")
    return ap.parse_args()


def dist_env():
    from paper_2505_00384_gb300 import replicas
    return replicas.env()


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.proc, self.lines = gpu, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload(args):
    work = dict(SMALL if args.small else FULL)
    if args.mesh:
        nx, ny, nz = (int(v) for v in args.mesh.lower().split("x"))
        work.update(name="hill_%dx%dx%d_r4_imex" % (nx, ny, nz), nx=nx, ny=ny, nz=nz, Lx=937.5 * nx, Ly=937.5 * ny,
                    Lz=625.0 * nz)
    work.update(COMMON)
    return work


def measured_hbm_gbs():
    """(HBM copy bandwidth in GB/s, source): the measured figure of this machine's
    GB300s when MEASURED_PEAKS.json is present, else the earlier measurement
    used as the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback (earlier GB300 copy measurement)"


def hbm_fractions(bytes_moved, seconds, hbm_gbs):
    """Achieved GB/s of `bytes_moved` in `seconds` and its fraction of hbm_gbs
    (None where the bytes are unknown)."""
    if bytes_moved is None or not seconds > 0:
        return None, None
    gbs = bytes_moved / seconds / 1e9
    return gbs, gbs / hbm_gbs


def oracle_step_cost(work, budget_s=15.0, threads=None):
    """FP64 CPU oracle on a bounded sample of cells of this workload: seconds
    per full-mesh operator application and per explicit-tendency evaluation,
    scaled by cells; returns (seconds per IMEX step, sample text, threads).
    threads: OpenMP threads for this measurement (all cores when None)."""
    import numpy as np
    import oracle as O
    prev = O.max_threads()
    if threads:
        O.set_threads(threads)
    try:
        return _oracle_step_cost(O, np, work, budget_s)
    finally:
        O.set_threads(prev)


def _oracle_step_cost(O, np, work, budget_s):
    m = O.make_mesh(work["nx"], work["ny"], work["nz"], work["r"], Lx=work["Lx"], Ly=work["Ly"], Lz=work["Lz"],
                    terrain=work["terrain"], hc=work["hc"], ac=work["ac"], bc_lateral=work["bc_lateral"])
    bg = O.make_bg(kind=0, T=work["T"], p0=work["p0"], R=work["R"], gamma=work["gamma"], g=work["g"],
                   ubar=work["ubar"])
    ncell = work["nx"] * work["ny"] * work["nz"]
    N = ncell * (work["r"] + 1) ** 3
    X = O.node_coords(m)
    rb, pb = O.background(m, bg)
    u = np.concatenate([np.full(N, work["ubar"]), np.zeros(N), np.zeros(N)])
    pprime = 50.0 * np.exp(-((X[0] - work["Lx"] / 2) ** 2 + (X[2] - 3000.0) ** 2) / (2 * 3000.0 ** 2))
    rng = np.random.default_rng(5)
    t_s = t_e = 0.0
    done = 0
    ncs = 8
    while True:
        cells = rng.choice(ncell, size=min(ncs, ncell - done), replace=False)
        t0 = time.perf_counter()
        O.apply_S(m, A_LL * work["dt"], work["gamma"], rb, pb, pprime, cells=cells)
        t1 = time.perf_counter()
        O.explicit(m, bg, rb, u, rb, cells=cells)
        t2 = time.perf_counter()
        t_s += t1 - t0
        t_e += t2 - t1
        done += len(cells)
        if t_s + t_e > budget_s or done >= ncell:
            break
        ncs = min(ncell - done, max(ncs, int(ncs * budget_s / max(t_s + t_e, 1e-3) / 4)))
    per_apply = t_s / done * ncell
    per_explicit = t_e / done * ncell
    step = per_apply * (PLAIN_STEP_APPLIES + STEP_EXTRA_HALF_APPLIES / 2.0) + 2 * per_explicit
    sample = ("oracle operator S and explicit tendencies on %d random cells of %d (with face neighbours), %.1f s, "
              "scaled by cells; step = %d FP64 operator applications (plain FGMRES solves) + %d half applications "
              "+ 2 explicit evaluations" % (done, ncell, t_s + t_e, PLAIN_STEP_APPLIES, STEP_EXTRA_HALF_APPLIES))
    return step, sample, O.max_threads()


def fp64_peak(torch):
    """Measured FP64 throughput: cuBLAS DGEMM (torch.matmul float64, 4096^3)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def run_reference(args, work):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    sample, threads = "", 0
    for _ in range(args.warmup + args.steps):
        v, sample, threads = oracle_step_cost(work, budget_s=max(2.0, 40.0 / (args.warmup + args.steps)))
        vals.append(v)
    v = statistics.median(vals[args.warmup:])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/step", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": work["name"]},
            "cpu_baseline": {"value": v, "unit": "s/step", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


ENSEMBLE = [(32, 32, 32), (40, 40, 32), (48, 48, 32), (48, 48, 40), (56, 56, 32), (64, 64, 32), (64, 64, 40),
            (64, 64, 48), (72, 72, 36), (80, 80, 40), (80, 80, 48), (88, 88, 44), (96, 96, 32), (96, 96, 40),
            (96, 96, 48), (32, 64, 32)]


def run_mixed(args):
    """Mixed precision on the 4 x 4 x 4-cell (1 km)^3 box with slip walls at
    degrees 2, 3 and 5 (1728, 4096, 13 824 DoFs): isothermal 250 K background as
    rho^(l) and p_k, a~_ll dt = 1 - 1/sqrt(2), right-hand side = Gaussian bump
    (sigma 200 m, box centre) + N(0, 1e-3^2) noise.  FP32 GMRES(30) inside FP64
    FGMRES(20) against plain FP64 FGMRES(30), both to 1e-8 from zero, each
    solution's error against the oracle's FP64 solution (to 1e-12); then one
    IMEX step with mixed solves on the degree-2 box with a centred 400 m hill
    (periodic lateral faces, background + 10 m/s wind + a pressure bump)
    against the oracle's step, error per field.  One step = the three mixed
    solves; L2 is flushed before every timed solve.  The oracle runs only in the
    CPU-baseline leg (skipped with --no-cpu-baseline): its solves and step are
    the timed baseline, and their results give the errors against the oracle."""
    import numpy as np
    import torch
    from paper_2505_00384_gb300 import dgx, inputs
    from paper_2505_00384_gb300 import learned as LP
    torch.cuda.set_device(0)
    dgx.load()
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    f64 = torch.float64
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def sopts(method, restart):
        so = dgx.dgx_default_solve_opts()
        so.method, so.pc, so.restart, so.tol, so.maxit = method, dgx.DGX_PC_HELMHOLTZ, restart, 1e-8, 3000
        so.inner_maxit, so.inner_tol = 30, 1e-5
        return so

    solvers = {"mixed": sopts(dgx.DGX_SOLVER_MIXED, 20), "plain_fp64": sopts(dgx.DGX_SOLVER_FGMRES, 30)}
    degrees, ts_mixed, launches, cpu = [], [], 0, None
    systems, solutions = [], {}
    for r in (2, 3, 5):
        dgx.dgx_mesh_build(ctx, dgx.mesh_desc(4, 4, 4, r, 1000.0, 1000.0, 1000.0))
        N = dgx.dgx_num_dofs(ctx)
        dgx.dgx_set_background(ctx, dgx.background(kind=0, T=250.0, u_bar=0.0))
        rho = torch.zeros(N, dtype=f64, device="cuda")
        pk = torch.zeros_like(rho)
        dgx.dgx_background_fields(ctx, rho.data_ptr(), pk.data_ptr())
        dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), A_LL, 1.4)
        X = torch.zeros(3 * N, dtype=f64, device="cuda")
        dgx.dgx_node_coords(ctx, X.data_ptr())
        Xh = X.cpu().numpy().reshape(3, N)
        b = inputs.gaussian_bump_rhs(Xh, [500.0, 500.0, 500.0], 200.0, 1e-3, inputs.DEFAULT_SEED)
        systems.append((r, rho.cpu().numpy(), pk.cpu().numpy(), b))
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        row = {"degree": r, "dofs": N}
        for name, so in solvers.items():
            for _ in range(max(args.warmup, 3)):
                x.zero_()
                dgx.dgx_solve_pressure(ctx, bd.data_ptr(), x.data_ptr(), so)
            ts = []
            for _ in range(args.steps):
                x.zero_()
                flush.zero_()
                torch.cuda.synchronize()
                l0 = dgx.dgx_kernel_launches()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st, si = dgx.dgx_solve_pressure(ctx, bd.data_ptr(), x.data_ptr(), so)
                e1.record(stream)
                torch.cuda.synchronize()
                if name == "mixed":
                    launches += dgx.dgx_kernel_launches() - l0
                if st != dgx.DGX_OK:
                    raise RuntimeError("%s solve at degree %d did not converge" % (name, r))
                ts.append(e0.elapsed_time(e1) / 1e3)
            solutions[(r, name)] = x.cpu().numpy()
            row[name] = {"s_per_solve": statistics.median(ts), "iterations": si.iterations,
                         "inner_iterations": si.inner_iterations, "relres": si.relres}
            if name == "mixed":
                ts_mixed.append(statistics.median(ts))
        degrees.append(row)
    # e2e at degree 5 (the last mesh): host right-hand side in, host solution out
    bh = bd.cpu().pin_memory()
    xhost = torch.empty_like(bh).pin_memory()
    te = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bd.copy_(bh, non_blocking=True)
        x.zero_()
        dgx.dgx_solve_pressure(ctx, bd.data_ptr(), x.data_ptr(), solvers["mixed"])
        xhost.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        te.append(e0.elapsed_time(e1) / 1e3)
    # one IMEX step with mixed solves on the hill box: background + wind + a 100 Pa bump
    N = LP.setup_hill(ctx, 400.0)
    rbd = torch.zeros(N, dtype=f64, device="cuda")
    pbd = torch.zeros_like(rbd)
    dgx.dgx_background_fields(ctx, rbd.data_ptr(), pbd.data_ptr())
    X = torch.zeros(3 * N, dtype=f64, device="cuda")
    dgx.dgx_node_coords(ctx, X.data_ptr())
    Xh = X.cpu().numpy().reshape(3, N)
    bump = np.exp(-((Xh[0] - 500.0) ** 2 + (Xh[1] - 500.0) ** 2 + (Xh[2] - 500.0) ** 2) / (2 * 150.0 ** 2))
    r0, p0 = rbd.cpu().numpy(), pbd.cpu().numpy() + 100.0 * bump
    u0 = np.concatenate([np.full(N, LP.BOX["u_bar"]), np.zeros(N), np.zeros(N)])
    rd, ud, pd = (torch.from_numpy(a.copy()).cuda() for a in (r0, u0, p0))
    so = sopts(dgx.DGX_SOLVER_MIXED, 20)
    st, sinfo = dgx.dgx_imex_step(ctx, rd.data_ptr(), ud.data_ptr(), pd.data_ptr(), 1, so)
    rg, ug, pg = rd.cpu().numpy(), ud.cpu().numpy(), pd.cpu().numpy()

    # CPU-baseline leg: the oracle's solves and step (timed), and the errors against them
    fields = None
    if not args.no_cpu_baseline:
        import oracle as O
        for r, rho_h, pk_h, b in systems:
            m = O.make_mesh(4, 4, 4, r)
            if r == 2:
                tc = time.time()
                _, _, its_o, _ = O.solve(m, A_LL, 1.4, rho_h, pk_h, b, tol=1e-8, maxit=3000)
                cpu = {"value": time.time() - tc, "unit": "s/solve", "cores": O.max_threads(), "kind": "oracle",
                       "sample": "degree-2 box, FP64 FGMRES(30) + Helmholtz Jacobi to 1e-8 (%d iterations)" % its_o}
            xo = O.solve(m, A_LL, 1.4, rho_h, pk_h, b, tol=1e-12, maxit=6000)[0]
            row = next(d for d in degrees if d["degree"] == r)
            for name in solvers:
                xh = solutions[(r, name)]
                row[name]["max_rel_err_vs_oracle"] = float(np.abs(xh - xo).max() / np.abs(xo).max())
                row[name]["l2_rel_err_vs_oracle"] = float(np.linalg.norm(xh - xo) / np.linalg.norm(xo))
        L = LP.BOX["L"]
        m = O.make_mesh(4, 4, 4, 2, Lx=L, Ly=L, Lz=L, terrain=1, hc=400.0, ac=LP.BOX["a_c"], xc=L / 2, yc=L / 2,
                        bc_lateral=2)
        obg = O.make_bg(kind=0, T=250.0, ubar=LP.BOX["u_bar"])
        rb, pb = O.background(m, obg)
        ro, uo, po, sto, _ = O.imex_step(m, obg, r0, u0, p0, LP.BOX["dt"], K=LP.BOX["K"], tol=1e-11)

        def rel(a, b, ref):
            return float(np.abs(a - b).max() / max(np.abs(ref).max(), 1e-300))

        fields = {"rho'": rel(rg, ro, ro - rb), "u": rel(ug[:N], uo[:N], uo[:N]),
                  "v": rel(ug[N:2 * N], uo[N:2 * N], uo), "w": rel(ug[2 * N:], uo[2 * N:], uo),
                  "p'": rel(pg, po, po - pb)}
    v = ts_mixed[0]
    line = {"metric": "mixed-precision pressure solve s/solve @1e-8 rel residual (4x4x4 box, degree 2)",
            "value": v, "unit": "s/solve", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": sum(ts_mixed) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "mixed_box_4x4x4_degrees_2_3_5", "step": "mixed solves at degrees 2, 3, 5",
                       "l2": "flushed before every timed solve"},
            "degrees": degrees,
            "imex_step_vs_oracle": {"mesh": "4x4x4 r=2 box, 400 m hill, periodic", "status": st,
                                    "solves": sinfo.solves, "max_rel_err_per_field": fields},
            "e2e": {"value": statistics.median(te), "unit": "s/solve (degree 5)", "h2d_bytes_per_step": bd.numel() * 8,
                    "d2h_bytes_per_step": bd.numel() * 8},
            "gpu_launches": launches / args.steps,
            "roofline": None, "roofline_note": "latency-bound meshes of 1728-13824 DoFs: see the hill workload",
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    dgx.dgx_destroy(ctx)
    return 0


def run_paper(args, dims=(120, 80, 32), refine=None, name="paper_sec3_120x80x32_r4_38.4M_dofs_stratified"):
    """The test case of Sec. 3 on its uniform mesh: (0, 60) x (0, 40) x (0, 16) km,
    120 x 80 x 32 cells at degree 4 (38 400 000 DoFs per scalar, 125 m), the -3/2
    bell hill h_c = 400 m, a_c = 1 km at (30, 20) km, the constant-N background
    (N = 0.01 1/s, T_ref = 293.15 K, p_ref = 1e5 Pa), u_bar = 10 m/s, far-field
    lateral faces, slip walls at bottom and top; ARS(2,2,2) with two fixed-point
    iterations, dt = 1 s.  From the initial state, one IMEX step with plain FP64
    FGMRES(30) solves to 1e-8 preconditioned by the Helmholtz Jacobi diagonal, the
    step with the mixed-precision solver, then the step with FP64 FGMRES(30) and the
    internal-energy (D) diagonal (the comparison of Sec. 3.1).  One line per solver
    is printed as soon as it is measured, then the summary line."""
    import torch
    from paper_2505_00384_gb300 import dgx
    torch.cuda.set_device(0)
    dgx.load()
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    desc = dgx.mesh_desc(dims[0], dims[1], dims[2], 4, 60000.0, 40000.0, 16000.0, terrain=2, h_c=400.0, a_c=1000.0,
                         x_c=30000.0, y_c=20000.0, bc_lateral=1, refine=refine)
    t0 = time.perf_counter()
    dgx.dgx_mesh_build(ctx, desc)
    N = dgx.dgx_num_dofs(ctx)
    dgx.dgx_set_background(ctx, dgx.background(kind=1, T=293.15, p0=1e5, N_bv=0.01, R=287.0, gamma=1.4, g=9.81,
                                               u_bar=10.0))
    A, At = dgx.ars222()
    dgx.dgx_set_imex(ctx, A, At, 1.0, 2)
    f64 = torch.float64
    rho0 = torch.zeros(N, dtype=f64, device="cuda")
    p0 = torch.zeros(N, dtype=f64, device="cuda")
    dgx.dgx_background_fields(ctx, rho0.data_ptr(), p0.data_ptr())
    u0 = torch.zeros(3 * N, dtype=f64, device="cuda")
    u0[:N] = 10.0
    # first applications in each precision (the per-context choice of threads per
    # CTA runs there), outside the measured steps
    dgx.dgx_set_coefficients(ctx, rho0.data_ptr(), p0.data_ptr(), A_LL, 1.4)
    y = torch.empty(N, dtype=f64, device="cuda")
    dgx.dgx_apply_operator(ctx, dgx.DGX_F64, p0.data_ptr(), y.data_ptr())
    x32, y32 = p0.float(), torch.empty(N, dtype=torch.float32, device="cuda")
    dgx.dgx_apply_operator(ctx, dgx.DGX_F32, x32.data_ptr(), y32.data_ptr())
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    op_ms = {}
    for prec, xx, yy in ((dgx.DGX_F64, p0, y), (dgx.DGX_F32, x32, y32)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            dgx.dgx_apply_operator(ctx, prec, xx.data_ptr(), yy.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        op_ms["f64" if prec == dgx.DGX_F64 else "f32"] = e0.elapsed_time(e1) / 5
    del y, x32, y32

    def opts(method, pc, maxit=3000):
        o = dgx.dgx_default_solve_opts()
        o.method, o.pc, o.tol, o.maxit = method, pc, 1e-8, maxit
        o.restart = 20 if method == dgx.DGX_SOLVER_MIXED else 30
        o.inner_maxit, o.inner_tol = 25, 3e-6
        return o

    # the internal-energy solves are capped at 150 iterations each (about 4.5x the
    # Helmholtz count of the hill workload) to bound the run; a capped solve is
    # reported as not converged and the saving is then a lower bound
    runs = [("fgmres_helmholtz", opts(dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_HELMHOLTZ)),
            ("mixed_helmholtz", opts(dgx.DGX_SOLVER_MIXED, dgx.DGX_PC_HELMHOLTZ)),
            ("fgmres_internal_energy", opts(dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_INTERNAL_ENERGY, 150))]
    res, pres = {}, {}
    for name, o in runs:
        r, u, p = rho0.clone(), u0.clone(), p0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = dgx.dgx_imex_step(ctx, r.data_ptr(), u.data_ptr(), p.data_ptr(), 1, o)
        e1.record(stream)
        torch.cuda.synchronize()
        if st != dgx.DGX_OK and name != "fgmres_internal_energy":
            raise RuntimeError("%s: a pressure solve did not converge (relres %g)" % (name, info.max_relres))
        pres[name] = p - p0
        res[name] = {"converged": st == dgx.DGX_OK, "s_per_step": e0.elapsed_time(e1) / 1e3,
                     "pressure_solve_s": info.seconds_solve,
                     "solves": info.solves, "krylov_iterations": info.krylov_iterations,
                     "inner_iterations": info.inner_iterations, "operator_f64": info.operator_f64,
                     "operator_f32": info.operator_f32, "max_relres": info.max_relres}
        print(json.dumps({"paper_case_solver": name, **res[name]}), flush=True)
        del r, u, p
    ref = pres["fgmres_helmholtz"]
    sc = float(ref.abs().max().clamp_min(1e-30))
    for name in pres:
        res[name]["p_prime_max_rel_diff_vs_fgmres_helmholtz"] = float((pres[name] - ref).abs().max()) / sc
    run = None
    if args.paper_steps > 0:  # a longer run with the mixed solver: per-step times and the flow's growth
        o = opts(dgx.DGX_SOLVER_MIXED, dgx.DGX_PC_HELMHOLTZ)
        r, u, p = rho0.clone(), u0.clone(), p0.clone()
        per, wmax, pmax, its = [], [], [], 0
        for k in range(args.paper_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, info = dgx.dgx_imex_step(ctx, r.data_ptr(), u.data_ptr(), p.data_ptr(), 1, o)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != dgx.DGX_OK:
                raise RuntimeError("step %d: a pressure solve did not converge (relres %g)" % (k, info.max_relres))
            per.append(e0.elapsed_time(e1) / 1e3)
            its += info.krylov_iterations
            wmax.append(float(u[2 * N:].abs().max()))
            pmax.append(float((p - p0).abs().max()))
        run = {"steps": args.paper_steps, "simulated_s": args.paper_steps * 1.0, "s_per_step_mean": sum(per) / len(per),
               "s_per_step_first_last": [per[0], per[-1]], "krylov_iterations_per_step": its / args.paper_steps,
               "w_max_m_s": wmax[:: max(1, args.paper_steps // 10)] + [wmax[-1]],
               "p_prime_max_pa": pmax[:: max(1, args.paper_steps // 10)] + [pmax[-1]],
               "finite": bool(torch.isfinite(p).all() and torch.isfinite(u).all())}
        print(json.dumps({"paper_case_run": run}), flush=True)
        del r, u, p
    h, ie = res["fgmres_helmholtz"], res["fgmres_internal_energy"]
    out = {"metric": "pressure solve s/step @1e-8 rel residual, Helmholtz vs internal-energy Jacobi",
           "value": h["pressure_solve_s"], "unit": "s/step", "n_gpus": 1, "steps": 1, "warmup": 0,
           "higher_is_better": False, "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "dofs_per_scalar": N, "cells": dims[0] * dims[1] * dims[2] if refine is None
                      else dims[0] * dims[1] * dims[2] + 7 * (refine[1] - refine[0]) * (refine[3] - refine[2])
                      * (refine[5] - refine[4]), "refine_box_base_cells": refine,
                      "terrain": "-3/2 bell h_c=400 m a_c=1 km at (30, 20) km, Gal-Chen",
                      "background": "constant N = 0.01 1/s, T_ref = 293.15 K", "lateral": "far field",
                      "dt_s": 1.0, "setup_s": t_setup},
           "operator_ms": op_ms, "solvers": res, "run": run,
           "helmholtz_time_saving_vs_internal_energy": 1.0 - h["pressure_solve_s"] / ie["pressure_solve_s"],
           "helmholtz_iteration_ratio_vs_internal_energy": h["krylov_iterations"] / ie["krylov_iterations"],
           "mixed_speedup_vs_fgmres_helmholtz": h["pressure_solve_s"] / res["mixed_helmholtz"]["pressure_solve_s"]}
    print(json.dumps(out), flush=True)
    dgx.dgx_destroy(ctx)
    return 0


def run_nonconf(args):
    """The test case of Sec. 3 on a non-conforming mesh (Sec. 3: cells of
    different resolution horizontally and vertically): base cells of 500 m x
    500 m x 1 km (120 x 80 x 16), the box of base cells [48, 72) x [28, 52) x [0, 8)
    around the hill split 2 x 2 x 2 (250 m x 250 m x 500 m near the ground), degree
    4: 190 464 cells (185 856 with unknowns), 23.2 M DoFs per scalar (the paper's
    non-conforming mesh: 204 816 cells, 25.6 M).  The rest as `--workload paper`:
    one IMEX step from the initial state per solver (FP64 FGMRES(30) with the
    Helmholtz and with the internal-energy Jacobi diagonal, the mixed solver), the
    comparison of Sec. 3.1 on the non-conforming mesh; plus the operator
    application times on this mesh."""
    return run_paper(args, dims=(120, 80, 16), refine=(48, 72, 28, 52, 0, 8),
                     name="sec3_nonconforming_120x80x16_box2to1_r4_23.2M_dofs_stratified")


def run_consistent(args):
    """Fast against consistent density-weighted mass (Sec. 3.3) on the Sec. 3
    domain at 250 m resolution: 60 x 40 x 16 cells at degree 4 (4 800 000 DoFs
    per scalar), -3/2 bell hill, constant-N background, u_bar = 10 m/s, far-field
    lateral faces, dt = 1 s, mixed-precision solves to 1e-8.  For each rule, from
    the same initial state: --warmup + --steps IMEX steps, the last --steps timed;
    then the relative difference of the final vertical velocity and pressure
    perturbation, and the consistent rule's PCG iteration counts."""
    import torch
    from paper_2505_00384_gb300 import dgx
    torch.cuda.set_device(0)
    dgx.load()
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    desc = dgx.mesh_desc(60, 40, 16, 4, 60000.0, 40000.0, 16000.0, terrain=2, h_c=400.0, a_c=1000.0,
                         x_c=30000.0, y_c=20000.0, bc_lateral=1)
    dgx.dgx_mesh_build(ctx, desc)
    N = dgx.dgx_num_dofs(ctx)
    dgx.dgx_set_background(ctx, dgx.background(kind=1, T=293.15, p0=1e5, N_bv=0.01, R=287.0, gamma=1.4, g=9.81,
                                               u_bar=10.0))
    A, At = dgx.ars222()
    dgx.dgx_set_imex(ctx, A, At, 1.0, 2)
    f64 = torch.float64
    rho0 = torch.zeros(N, dtype=f64, device="cuda")
    p0 = torch.zeros(N, dtype=f64, device="cuda")
    dgx.dgx_background_fields(ctx, rho0.data_ptr(), p0.data_ptr())
    u0 = torch.zeros(3 * N, dtype=f64, device="cuda")
    u0[:N] = 10.0
    o = dgx.dgx_default_solve_opts()
    o.method, o.pc, o.tol, o.maxit, o.restart = dgx.DGX_SOLVER_MIXED, dgx.DGX_PC_HELMHOLTZ, 1e-8, 2000, 20
    o.inner_maxit, o.inner_tol = 25, 3e-6
    res, final = {}, {}
    for name, rule in (("fast", dgx.DGX_MASS_FAST), ("consistent", dgx.DGX_MASS_CONSISTENT)):
        dgx.dgx_set_mass_rule(ctx, rule, 1e-13, 50)
        r, u, p = rho0.clone(), u0.clone(), p0.clone()
        for _ in range(args.warmup):
            dgx.dgx_imex_step(ctx, r.data_ptr(), u.data_ptr(), p.data_ptr(), 1, o)
        dgx.dgx_mass_cg_stats(ctx)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = dgx.dgx_imex_step(ctx, r.data_ptr(), u.data_ptr(), p.data_ptr(), args.steps, o)
        e1.record(stream)
        torch.cuda.synchronize()
        its, bad = dgx.dgx_mass_cg_stats(ctx)
        if st != dgx.DGX_OK or bad:
            raise RuntimeError("%s: status %d, %d unconverged cell solves" % (name, st, bad))
        res[name] = {"s_per_step": e0.elapsed_time(e1) / 1e3 / args.steps,
                     "pressure_solve_s_per_step": info.seconds_solve / args.steps,
                     "krylov_iterations_per_step": info.krylov_iterations / args.steps,
                     "max_relres": info.max_relres, "mass_cg_max_iterations": its}
        final[name] = (u[2 * N:].clone(), p - p0)
        del r, u, p
    wf, wc = final["fast"][0], final["consistent"][0]
    pf, pc = final["fast"][1], final["consistent"][1]
    out = {"metric": "IMEX s/step, fast vs consistent density-weighted mass", "value": res["consistent"]["s_per_step"],
           "unit": "s/step", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "f64 (FP32 inner solves)", "data": "synthetic",
           "config": {"workload": "paper_sec3_60x40x16_r4_4.8M_dofs_stratified", "dofs_per_scalar": N, "dt_s": 1.0},
           "rules": res, "consistent_over_fast_time": res["consistent"]["s_per_step"] / res["fast"]["s_per_step"],
           "w_max_rel_diff": float((wf - wc).abs().max() / wc.abs().max().clamp_min(1e-30)),
           "p_prime_max_rel_diff": float((pf - pc).abs().max() / pc.abs().max().clamp_min(1e-30))}
    print(json.dumps(out), flush=True)
    dgx.dgx_destroy(ctx)
    return 0


def run_vmult(args):
    """Operator application y = S x (the vmult of the metric) on the hill mesh
    (64x64x32 r=4 unless --mesh): every launch variant in FP64 and FP32,
    --warmup untimed and --steps timed applications each (CUDA events, inputs
    larger than L2), GDoF/s and the agreement of each variant with variant 0.
    Coefficients: isothermal hydrostatic profiles with 5 % seeded noise;
    x: seeded N(0, 100^2).  With --profile and --variant-f64 / --variant-f32:
    only those variants, --warmup + --steps applications each (profiler driver)."""
    import torch
    from paper_2505_00384_gb300 import dgx, inputs
    torch.cuda.set_device(0)
    dgx.load()
    work = workload(args)
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    desc = dgx.mesh_desc(work["nx"], work["ny"], work["nz"], work["r"], work["Lx"], work["Ly"], work["Lz"],
                         terrain=work["terrain"], h_c=work["hc"], a_c=work["ac"], bc_lateral=work["bc_lateral"])
    dgx.dgx_mesh_build(ctx, desc)
    N = dgx.dgx_num_dofs(ctx)
    X = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    dgx.dgx_node_coords(ctx, X.data_ptr())
    z = X[2 * N:].cpu().numpy()
    del X
    rho = torch.from_numpy(inputs.perturbed_profile(z, 1.2, 7314.0, 0.05, 1)).cuda()
    pk = torch.from_numpy(inputs.perturbed_profile(z, 1e5, 7314.0, 0.05, 2)).cuda()
    dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), A_LL, work["gamma"])
    x64 = torch.from_numpy(inputs.random_field(N, 3, 100.0)).cuda()
    fl_grad, fl_div, bytes64 = dgx.dgx_operator_cost(ctx)
    out, ref = {}, {}
    pins = {dgx.DGX_F64: args.variant_f64, dgx.DGX_F32: args.variant_f32}
    for prec, dt in ((dgx.DGX_F64, torch.float64), (dgx.DGX_F32, torch.float32)):
        x = x64.to(dt)
        y = torch.zeros(N, dtype=dt, device="cuda")
        variants = [pins[prec]] if pins[prec] is not None else list(range(dgx.DGX_OP_VARIANTS))
        if args.profile and pins[prec] is None:
            continue
        for v in variants:
            try:
                dgx.dgx_set_operator_variant(ctx, prec, v)
            except dgx.DgxError:
                continue
            for _ in range(args.warmup):
                dgx.dgx_apply_operator(ctx, prec, x.data_ptr(), y.data_ptr())
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                dgx.dgx_apply_operator(ctx, prec, x.data_ptr(), y.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            if args.profile:
                continue
            ms = e0.elapsed_time(e1) / args.steps
            yy = y.double()
            if prec not in ref:
                ref[prec] = yy.clone()
            out["%s_v%d" % ("f64" if prec == dgx.DGX_F64 else "f32", v)] = {
                "ms": ms, "gdofs": N / ms / 1e6, "tflops_counted": (fl_grad + fl_div) / ms / 1e9,
                "threads_per_cta": dgx.dgx_operator_threads(ctx, prec),
                "max_rel_diff_vs_first": float((yy - ref[prec]).abs().max() / ref[prec].abs().max())}
    dgx.dgx_destroy(ctx)
    if args.profile:
        print(json.dumps({"profile_run": True, "workload": "vmult_" + work["name"], "N": N}), flush=True)
        return 0
    best = {p_: min((v for k, v in out.items() if k.startswith(p_)), key=lambda d: d["ms"]) for p_ in ("f64", "f32")}
    line = {"metric": "vmult GDoF/s (operator application y = S x)", "value": best["f64"]["gdofs"], "unit": "GDoF/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (and f32)", "data": "synthetic",
            "config": {"workload": "vmult_" + work["name"], "dofs": N, "l2": "inputs larger than L2"},
            "best": best, "variants": out, "flops_per_apply": fl_grad + fl_div, "hbm_floor_bytes_f64": bytes64}
    print(json.dumps(line), flush=True)
    return 0


def run_mg(args):
    """Geometric multigrid (Sec. 3.1): (1) the SPD case -- a 64 x 64 x 32-cell box
    of 64 x 64 x 20 km at degree 3 (8 388 608 DoFs), slip walls, uniform
    coefficients (rho = 1.2, p_k = 1e5: S symmetric positive definite), seeded
    N(0, 1) right-hand side -- solved to 1e-8 from zero by CG with the Helmholtz
    Jacobi and by CG with one V-cycle per iteration (4 levels, Chebyshev degree
    3, coarsest CG to 1e-10); (2) the experiment on the non-symmetric Schur
    system of the hill workload (64 x 64 x 32 cells, r = 4, far-field faces,
    background coefficients with 5 % seeded noise): FGMRES(30) with the
    Helmholtz Jacobi against FGMRES with the V-cycle (3 levels, coarsest FGMRES).
    --warmup untimed and --steps timed solves each (CUDA events)."""
    import torch
    from paper_2505_00384_gb300 import dgx, inputs
    torch.cuda.set_device(0)
    dgx.load()
    stream = torch.cuda.current_stream()
    f64 = torch.float64
    out = {}

    def timed(ctx, b, o):
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            dgx.dgx_solve_pressure(ctx, b.data_ptr(), x.data_ptr(), o)
        ts, info = [], None
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, info = dgx.dgx_solve_pressure(ctx, b.data_ptr(), x.data_ptr(), o)
            e1.record(stream)
            torch.cuda.synchronize()
            if st != dgx.DGX_OK:
                raise RuntimeError("solve did not converge (relres %g)" % info.relres)
            ts.append(e0.elapsed_time(e1) / 1e3)
        return {"s_per_solve": statistics.median(ts), "iterations": info.iterations, "relres": info.relres,
                "operator_f64": info.operator_f64}

    # (1) SPD box
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    dgx.dgx_mesh_build(ctx, dgx.mesh_desc(64, 64, 32, 3, 64000.0, 64000.0, 20000.0))
    N = dgx.dgx_num_dofs(ctx)
    rho = torch.full((N,), 1.2, dtype=f64, device="cuda")
    pk = torch.full((N,), 1e5, dtype=f64, device="cuda")
    dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), A_LL, 1.4)
    mo = dgx.dgx_default_mg_opts()
    mo.levels, mo.coarse_tol = 4, 1e-10
    t0 = time.perf_counter()
    dgx.dgx_mg_setup(ctx, mo)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    b = torch.from_numpy(inputs.normal(inputs.DEFAULT_SEED + 11, N)).cuda()
    o = dgx.dgx_default_solve_opts()
    o.method, o.tol, o.maxit = dgx.DGX_SOLVER_CG, 1e-8, 5000
    o.pc = dgx.DGX_PC_HELMHOLTZ
    jac = timed(ctx, b, o)
    o.pc = dgx.DGX_PC_MULTIGRID
    mgr = timed(ctx, b, o)
    out["spd_box"] = {"mesh": "64x64x32 cells, r=3, %d DoFs, slip walls, uniform coefficients" % N,
                      "cg_jacobi": jac, "cg_multigrid": mgr, "multigrid_setup_s": t_setup,
                      "levels": dgx.dgx_mg_levels(ctx)[0], "speedup": jac["s_per_solve"] / mgr["s_per_solve"]}
    dgx.dgx_destroy(ctx)
    del rho, pk, b
    # (2) the hill Schur system
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    work = dict(FULL)
    work.update(COMMON)
    dgx.dgx_mesh_build(ctx, dgx.mesh_desc(64, 64, 32, 4, work["Lx"], work["Ly"], work["Lz"], terrain=1, h_c=400.0,
                                          a_c=1000.0, bc_lateral=1))
    N = dgx.dgx_num_dofs(ctx)
    dgx.dgx_set_background(ctx, dgx.background(kind=0, T=250.0))
    rho = torch.zeros(N, dtype=f64, device="cuda")
    pk = torch.zeros_like(rho)
    dgx.dgx_background_fields(ctx, rho.data_ptr(), pk.data_ptr())
    noise = torch.from_numpy(inputs.normal(inputs.DEFAULT_SEED + 12, N)).cuda()
    rho *= 1.0 + 0.05 * noise
    pk *= 1.0 - 0.05 * noise
    del noise
    dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), A_LL, 1.4)
    mo = dgx.dgx_default_mg_opts()
    mo.levels, mo.coarse_solver, mo.coarse_tol = 3, 1, 1e-6
    dgx.dgx_mg_setup(ctx, mo)
    b = torch.from_numpy(inputs.normal(inputs.DEFAULT_SEED + 13, N)).cuda()
    o = dgx.dgx_default_solve_opts()
    o.method, o.tol, o.maxit, o.restart = dgx.DGX_SOLVER_FGMRES, 1e-8, 2000, 30
    o.pc = dgx.DGX_PC_HELMHOLTZ
    jac = timed(ctx, b, o)
    o.pc = dgx.DGX_PC_MULTIGRID
    mgr = timed(ctx, b, o)
    out["schur_hill_experiment"] = {"mesh": "64x64x32 cells, r=4, %d DoFs, hill, far-field faces" % N,
                                    "fgmres_helmholtz_jacobi": jac, "fgmres_multigrid": mgr,
                                    "speedup": jac["s_per_solve"] / mgr["s_per_solve"]}
    dgx.dgx_destroy(ctx)
    line = {"metric": "pressure solve s/solve @1e-8 rel residual, CG + geometric multigrid (SPD case)",
            "value": out["spd_box"]["cg_multigrid"]["s_per_solve"], "unit": "s/solve", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "mg_spd_box_64x64x32_r3_and_hill_schur_64x64x32_r4"}, **out}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """Learned preconditioner: 400 pressure systems recorded along IMEX
    trajectories over 16 seeded hills (h_c ~ U[200, 800] m, 25 steps each, the
    last solve of every step) on the 4 x 4 x 4-cell degree-2 box of 1 km
    (1728 DoFs, periodic lateral faces); 14 hills train a 9-layer 32-channel
    network (198 977 parameters) on the GPU, the 50 systems of the other two
    are solved to 1e-8 from x = 0 with FP64 FGMRES(30) + Helmholtz Jacobi
    (plain), the same with the learned preconditioner, and the mixed-precision
    solver.  One step = the 50 held-out solves with the learned
    preconditioner; L2 is flushed before every timed solve."""
    import numpy as np
    import torch
    from paper_2505_00384_gb300 import dgx, inputs
    from paper_2505_00384_gb300 import learned as LP
    torch.cuda.set_device(0)
    dgx.load()
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(0, stream.cuda_stream)
    layers, channels = 9, 32
    dgx.dgx_learned_create(ctx, layers, channels, inputs.DEFAULT_SEED)
    nparams = dgx.dgx_learned_num_params(ctx)
    if args.profile:
        # for profiler launch lists: --warmup + --steps applies of the (untrained)
        # network on the 500 m hill box with the background as coefficients
        N = LP.setup_hill(ctx, 500.0)
        rho = torch.zeros(N, dtype=torch.float64, device="cuda")
        pk = torch.zeros_like(rho)
        dgx.dgx_background_fields(ctx, rho.data_ptr(), pk.data_ptr())
        dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), A_LL, 1.4)
        v = torch.from_numpy(inputs.normal(inputs.DEFAULT_SEED + 9, N)).cuda()
        z = torch.zeros_like(v)
        for _ in range(args.warmup + args.steps):
            dgx.dgx_learned_apply(ctx, dgx.DGX_F64, v.data_ptr(), z.data_ptr())
        torch.cuda.synchronize()
        dgx.dgx_destroy(ctx)
        return 0
    nh, steps, test_hills = 16, 25, (14, 15)
    heights = LP.hill_heights(nh)
    t0 = time.time()
    held = LP.collect(ctx, heights, steps=steps, record_stride=4, pairs=8, pair_stride=3, test_hills=test_hills,
                      random_per_record=1)
    t_collect = time.time() - t0
    ntr, nte = dgx.dgx_learned_num_samples(ctx)
    o = dgx.dgx_default_train_opts()
    o.epochs, o.batch = args.epochs, 32  # from a sweep of epochs, batch and rate on this workload
    tinfo = dgx.dgx_learned_train(ctx, o)
    N = dgx.dgx_num_dofs(ctx)
    f64 = torch.float64

    def sopts(method, pc, restart):
        so = dgx.dgx_default_solve_opts()
        so.method, so.pc, so.restart, so.tol, so.maxit = method, pc, restart, 1e-8, 3000
        so.inner_maxit, so.inner_tol = 30, 1e-5
        return so

    solvers = {"learned": sopts(dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_LEARNED, 30),
               "plain_fp64": sopts(dgx.DGX_SOLVER_FGMRES, dgx.DGX_PC_HELMHOLTZ, 30),
               "mixed": sopts(dgx.DGX_SOLVER_MIXED, dgx.DGX_PC_HELMHOLTZ, 20)}
    systems = [(hi, rec) for hi in sorted(held) for rec in held[hi]]
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2
    x = torch.zeros(N, dtype=f64, device="cuda")
    cur = [None]

    def solve(name, hi, rec, timed):
        if cur[0] != hi:
            LP.setup_hill(ctx, heights[hi])
            cur[0] = hi
        rho, pk, b, _, a_dt, gamma = LP.split_record(rec, N)
        dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), a_dt, gamma)
        x.zero_()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, si = dgx.dgx_solve_pressure(ctx, b.data_ptr(), x.data_ptr(), solvers[name])
        e1.record(stream)
        torch.cuda.synchronize()
        if st not in (dgx.DGX_OK, dgx.DGX_FALLBACK_USED) or si.relres > 1e-8:
            raise RuntimeError("%s solve did not converge (relres %g)" % (name, si.relres))
        return e0.elapsed_time(e1) / 1e3, si

    for _ in range(max(args.warmup, 3)):
        for name in solvers:
            solve(name, *systems[0], False)
    res = {k: [] for k in solvers}
    launches0 = dgx.dgx_kernel_launches()
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            for hi, rec in systems:
                res["learned"].append(solve("learned", hi, rec, True))
    launches = (dgx.dgx_kernel_launches() - launches0) / args.steps
    for name in ("plain_fp64", "mixed"):
        for hi, rec in systems:
            res[name].append(solve(name, hi, rec, True))

    def summary(rs):
        return {"s_per_solve": float(np.mean([t for t, _ in rs])),
                "iterations": float(np.mean([si.iterations for _, si in rs])),
                "max_relres": float(max(si.relres for _, si in rs)),
                "fallbacks": int(sum(si.fallback for _, si in rs))}

    stats = {k: summary(v) for k, v in res.items()}
    # e2e: host coefficients and right-hand side in, host solution out, per system
    hosts = [(hi, [t.cpu().pin_memory() for t in LP.split_record(rec, N)[:3]], LP.split_record(rec, N)[4:])
             for hi, rec in systems]
    dev_in = [torch.empty(N, dtype=f64, device="cuda") for _ in range(3)]
    xh = torch.empty(N, dtype=f64).pin_memory()
    te = []
    for hi, (rh, pkh, bh), (a_dt, gamma) in hosts:
        if cur[0] != hi:
            LP.setup_hill(ctx, heights[hi])
            cur[0] = hi
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d, h in zip(dev_in, (rh, pkh, bh)):
            d.copy_(h, non_blocking=True)
        dgx.dgx_set_coefficients(ctx, dev_in[0].data_ptr(), dev_in[1].data_ptr(), a_dt, gamma)
        x.zero_()
        dgx.dgx_solve_pressure(ctx, dev_in[2].data_ptr(), x.data_ptr(), solvers["learned"])
        xh.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        te.append(e0.elapsed_time(e1) / 1e3)
    # roofline of the learned apply (graph of the network's kernels): FP32 FMA work
    conv_flops = 2.0 * 27 * N * sum(ci * co for ci, co in
                                     zip([5] + [channels] * (layers - 1), [channels] * (layers - 1) + [1]))
    v = torch.from_numpy(inputs.normal(inputs.DEFAULT_SEED + 9, N)).cuda()
    z = torch.zeros_like(v)
    dgx.dgx_learned_apply(ctx, dgx.DGX_F64, v.data_ptr(), z.data_ptr())
    dgx.dgx_learned_apply(ctx, dgx.DGX_F64, v.data_ptr(), z.data_ptr())
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(200):
        dgx.dgx_learned_apply(ctx, dgx.DGX_F64, v.data_ptr(), z.data_ptr())
    a1.record(stream)
    torch.cuda.synchronize()
    t_apply = a0.elapsed_time(a1) / 1e3 / 200
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # FMA lanes x 2 flops x max SM clock
    # CPU baseline: the oracle's plain FGMRES on one held-out system
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        hi, rec = systems[0]
        rho, pk, b, _, a_dt, gamma = (t if isinstance(t, float) else t.cpu().numpy() for t in LP.split_record(rec, N))
        L = LP.BOX["L"]
        m = O.make_mesh(4, 4, 4, 2, Lx=L, Ly=L, Lz=L, terrain=1, hc=float(heights[hi]), ac=LP.BOX["a_c"],
                        xc=L / 2, yc=L / 2, bc_lateral=2)
        tc = time.time()
        _, st, its, rel = O.solve(m, a_dt, gamma, rho, pk, b, tol=1e-8, restart=30, maxit=3000)
        cpu = {"value": time.time() - tc, "unit": "s/solve", "cores": O.max_threads(), "kind": "oracle",
               "sample": "1 held-out system, FP64 FGMRES(30) + Helmholtz Jacobi to 1e-8 (%d iterations)" % its}
    lv = stats["learned"]["s_per_solve"]
    line = {"metric": "pressure solve s/solve @1e-8 rel residual (learned preconditioner, held-out hills)",
            "value": lv, "unit": "s/solve", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": lv * len(systems) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (network f32, bf16 weights)", "data": "synthetic",
            "config": {"workload": "learned_box_4x4x4_r2_1728_dofs_16_hills", "systems_recorded": 400,
                       "train_hills": nh - len(test_hills), "held_out_systems": len(systems),
                       "network": "%d conv3d layers, %d channels, %d params" % (layers, channels, nparams),
                       "l2": "flushed before every timed solve"},
            "solvers": stats,
            "speedup_vs_plain_fp64": stats["plain_fp64"]["s_per_solve"] / lv,
            "iterations_ratio_vs_plain": stats["learned"]["iterations"] / stats["plain_fp64"]["iterations"],
            "training": {"samples_train": ntr, "samples_test": nte, "epochs": args.epochs, "steps": tinfo.steps,
                         "seconds": tinfo.seconds, "collect_seconds": t_collect,
                         "loss_train": [tinfo.loss_train0, tinfo.loss_train],
                         "loss_test": [tinfo.loss_test0, tinfo.loss_test]},
            "e2e": {"value": float(np.mean(te)), "unit": "s/solve", "h2d_bytes_per_step": 3 * N * 8 * len(systems),
                    "d2h_bytes_per_step": N * 8 * len(systems)},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "kernel": "learned apply (k_conv graph)", "achieved": conv_flops / t_apply / 1e12,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": conv_flops / t_apply / 1e12 / fp32_peak,
                         "traffic": None, "apply_us": t_apply * 1e6},
            "cpu_baseline": cpu, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    dgx.dgx_destroy(ctx)
    return 0


def run_ensemble(args):
    """16 members (meshes 32^3 .. 96x96x48, degrees 3 + i mod 3, seeded hill
    heights 200-800 m and widths 0.5-2 km, 60 x 60 x 20 km, periodic lateral
    faces): all pressure solves to 1e-8 in one call, the whole FP64 refinement
    loop around FP32 GMRES cycles of all members one CUDA-graph launch (a WHILE
    conditional node), tile shapes (cells and threads per CTA) autotuned per
    degree."""
    import numpy as np
    import torch
    from paper_2505_00384_gb300 import dgx, inputs
    torch.cuda.set_device(0)
    dgx.load()
    nm = max(1, min(args.members, len(ENSEMBLE)))
    u = inputs.uniform(inputs.DEFAULT_SEED + 5, 2 * nm)
    descs = []
    for i in range(nm):
        nx, ny, nz = ENSEMBLE[i]
        descs.append(dgx.mesh_desc(nx, ny, nz, 3 + i % 3, 60000.0, 60000.0, 20000.0, terrain=1,
                                   h_c=200.0 + 600.0 * u[2 * i], a_c=500.0 + 1500.0 * u[2 * i + 1], bc_lateral=2))
    stream = torch.cuda.current_stream()
    e = dgx.dgx_ensemble_create(0, stream.cuda_stream, descs)
    Nt = dgx.dgx_ensemble_num_dofs(e)
    f64 = torch.float64
    rho = torch.zeros(Nt, dtype=f64, device="cuda")
    pk = torch.zeros(Nt, dtype=f64, device="cuda")
    ptrue = torch.zeros(Nt, dtype=f64, device="cuda")
    for i in range(nm):
        c = dgx.dgx_ensemble_member(e, i)
        dgx.dgx_set_background(c, dgx.background(kind=0, T=250.0))
        o, n = dgx.dgx_ensemble_offset(e, i), dgx.dgx_ensemble_num_dofs(e, i)
        dgx.dgx_background_fields(c, rho[o:o + n].data_ptr(), pk[o:o + n].data_ptr())
        X = torch.zeros(3 * n, dtype=f64, device="cuda")
        dgx.dgx_node_coords(c, X.data_ptr())
        # the member contexts work on the ensemble's own stream: wait for the
        # coordinates (and fields) before torch reads them on its stream
        torch.cuda.synchronize()
        x, y, z = X[:n], X[n:2 * n], X[2 * n:]
        ptrue[o:o + n] = 100.0 * torch.exp(-((x - 30000.0) ** 2 + (y - 30000.0) ** 2 + (z - 5000.0) ** 2)
                                           / (2 * 2000.0 ** 2))
        del X, x, y, z
    torch.cuda.synchronize()
    noise = torch.from_numpy(inputs.normal(inputs.DEFAULT_SEED + 6, Nt)).cuda()
    rho *= 1.0 + 1e-3 * noise
    pk *= 1.0 - 1e-3 * noise
    ptrue += noise
    del noise
    dgx.dgx_ensemble_set_coefficients(e, rho.data_ptr(), pk.data_ptr(), A_LL, 1.4)
    b = torch.zeros_like(ptrue)
    dgx.dgx_ensemble_apply_operator(e, dgx.DGX_F64, ptrue.data_ptr(), b.data_ptr())
    dgx.dgx_ensemble_autotune(e)
    o = dgx.dgx_default_solve_opts()
    o.tol, o.maxit, o.inner_maxit, o.inner_tol = 1e-8, 50, 30, 1e-5
    if args.inner_maxit:
        o.inner_maxit = args.inner_maxit
    if args.inner_tol:
        o.inner_tol = args.inner_tol
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        x.zero_()
        st, infos = dgx.dgx_ensemble_solve(e, b.data_ptr(), x.data_ptr(), nm, o)
    ts = []
    launches0 = dgx.dgx_kernel_launches()
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, infos = dgx.dgx_ensemble_solve(e, b.data_ptr(), x.data_ptr(), nm, o)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
            if st != dgx.DGX_OK:
                raise RuntimeError("ensemble solve did not converge")
    launches = (dgx.dgx_kernel_launches() - launches0) / args.steps
    err = float((x - ptrue).abs().max() / ptrue.abs().max())
    # operator throughput of all members at once
    x32 = ptrue.float()
    y32 = torch.zeros_like(x32)
    y64 = torch.zeros_like(ptrue)

    def tcall(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        bb.record(stream)
        bb.synchronize()
        return a.elapsed_time(bb) / 1e3 / reps

    t32 = tcall(lambda: dgx.dgx_ensemble_apply_operator(e, dgx.DGX_F32, x32.data_ptr(), y32.data_ptr()), 3)
    t64 = tcall(lambda: dgx.dgx_ensemble_apply_operator(e, dgx.DGX_F64, ptrue.data_ptr(), y64.data_ptr()), 1)
    tuning = []
    g = 0
    while True:
        try:
            deg, nmem, th64, th32 = dgx.dgx_ensemble_tuning(e, g)
        except dgx.DgxError:
            break
        f64k, c64 = dgx.dgx_ensemble_tile(e, g, dgx.DGX_F64)
        f32k, c32 = dgx.dgx_ensemble_tile(e, g, dgx.DGX_F32)
        tuning.append({"degree": deg, "members": nmem, "threads_f64": th64, "threads_f32": th32,
                       "f64_kernels": "fused, double-word" if f64k else "one cell per CTA", "cells_per_cta_f64": c64,
                       "f32_kernels": "fused" if f32k else "one cell per CTA", "cells_per_cta_f32": c32})
        g += 1
    v = statistics.median(ts)
    line = {"metric": "ensemble pressure solves s/solve @1e-8 rel residual (all members)", "value": v,
            "unit": "s/solve", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": "ensemble_%d_members_%.1fM_dofs" % (nm, Nt / 1e6), "members": nm,
                       "degrees": "3 + i mod 3",
                       "solver": "FP64 refinement around FP32 GMRES(30) cycles, one CUDA-graph launch per solve"},
            "gdofs_solved_per_s": Nt / v / 1e9, "gpu_launches_host_side": launches,
            "sweeps": [i.iterations for i in infos], "max_relres": max(i.relres for i in infos),
            "max_rel_err_vs_p_true": err, "autotune": tuning,
            "operator_all_members": {"f32_ms": t32 * 1e3, "f64_ms": t64 * 1e3, "f32_gdofs": Nt / t32 / 1e9,
                                     "f64_gdofs": Nt / t64 / 1e9},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    dgx.dgx_ensemble_destroy(e)
    return 0


def main():
    args = parse()
    work = workload(args)
    if args.impl == "reference":
        return run_reference(args, work)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "vmult":
        return run_vmult(args)
    if args.workload == "mg":
        return run_mg(args)
    if args.workload == "nonconf":
        return run_nonconf(args)
    if args.workload == "consistent":
        return run_consistent(args)

    import torch
    from paper_2505_00384_gb300 import dgx

    from paper_2505_00384_gb300 import replicas
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = replicas.init("nccl")
    dgx.load()
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(local, stream.cuda_stream)
    desc = dgx.mesh_desc(work["nx"], work["ny"], work["nz"], work["r"], work["Lx"], work["Ly"], work["Lz"],
                         terrain=work["terrain"], h_c=work["hc"], a_c=work["ac"], bc_lateral=work["bc_lateral"])
    dgx.dgx_mesh_build(ctx, desc)
    N = dgx.dgx_num_dofs(ctx)
    dgx.dgx_set_background(ctx, dgx.background(kind=0, T=work["T"], p0=work["p0"], R=work["R"], gamma=work["gamma"],
                                               g=work["g"], u_bar=work["ubar"]))
    A, At = dgx.ars222()
    dgx.dgx_set_imex(ctx, A, At, work["dt"], work["K"])
    f64 = torch.float64
    rho0 = torch.zeros(N, dtype=f64, device="cuda")
    p0 = torch.zeros(N, dtype=f64, device="cuda")
    dgx.dgx_background_fields(ctx, rho0.data_ptr(), p0.data_ptr())
    u0 = torch.zeros(3 * N, dtype=f64, device="cuda")
    u0[:N] = work["ubar"]
    rho, u, p = rho0.clone(), u0.clone(), p0.clone()

    def opts(method):
        # inner FP32 GMRES(25) to 3e-6: the fastest of a sweep of (inner_maxit, inner_tol) on this
        # workload; the outer FP64 FGMRES tolerance 1e-8 is the method's and does not change
        o = dgx.dgx_default_solve_opts()
        o.method, o.pc, o.tol, o.maxit = method, dgx.DGX_PC_HELMHOLTZ, 1e-8, 2000
        o.restart = 20 if method == dgx.DGX_SOLVER_MIXED else 30
        o.inner_maxit, o.inner_tol = 25, 3e-6
        return o

    o_mixed, o_plain = opts(dgx.DGX_SOLVER_MIXED), opts(dgx.DGX_SOLVER_FGMRES)
    infos = []

    def step(r_, u_, p_, o=o_mixed):
        st, info = dgx.dgx_imex_step(ctx, r_.data_ptr(), u_.data_ptr(), p_.data_ptr(), 1, o)
        if st != dgx.DGX_OK:
            raise RuntimeError("IMEX step: a pressure solve did not converge (relres %g)" % info.max_relres)
        infos.append(info)

    # ---- warm-up (advances the flow from the initial state), then the timed steps
    for _ in range(args.warmup):
        step(rho, u, p)
    torch.cuda.synchronize()
    infos.clear()
    if pg:
        pg.barrier()
    launches0 = dgx.dgx_kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(rho, u, p)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = dgx.dgx_kernel_launches() - launches0
    t_dev = e0.elapsed_time(e1) / 1e3
    t_dev = replicas.max_over_ranks(pg, t_dev, "cuda")
    replicas.barrier(pg)
    step_infos = list(infos)
    finite = bool(torch.isfinite(p).all() and torch.isfinite(u).all())
    if args.profile:
        print(json.dumps({"profile_run": True, "workload": work["name"], "N": N, "steps": args.steps,
                          "s_per_step": t_dev / args.steps, "launches": launches, "finite": finite}), flush=True)
        dgx.dgx_destroy(ctx)
        return 0

    # ---- the same step with plain FP64 FGMRES solves (from the same state), --plain-steps
    # steps timed with CUDA events; the first one is kept for the comparison below
    rp, up, pp = rho.clone(), u.clone(), p.clone()
    infos.clear()
    torch.cuda.synchronize()
    ep = [torch.cuda.Event(enable_timing=True) for _ in range(args.plain_steps + 1)]
    p_first = None
    ep[0].record(stream)
    for k in range(args.plain_steps):
        step(rp, up, pp, o_plain)
        ep[k + 1].record(stream)
        if k == 0:
            p_first = pp.clone()
    torch.cuda.synchronize()
    t_plain = [ep[k].elapsed_time(ep[k + 1]) / 1e3 for k in range(args.plain_steps)]
    plain = {"s_per_step": statistics.mean(t_plain), "s_per_step_each": t_plain, "steps": args.plain_steps,
             "timing": "CUDA events on the library's stream, per step",
             "pressure_solve_s": statistics.mean(i.seconds_solve for i in infos),
             "krylov_iterations": statistics.mean(i.krylov_iterations for i in infos),
             "operator_f64": statistics.mean(i.operator_f64 for i in infos),
             "max_relres": max(i.max_relres for i in infos)}
    infos.clear()
    del rp, up, pp
    # mixed step from the same state: the difference of the results, and the true
    # FP64 residual b - S x of its four solves (recorded systems, S applied afresh)
    rm, um, pm = rho.clone(), u.clone(), p.clone()
    rec = torch.zeros(4 * (4 * N + 2), dtype=f64, device="cuda")
    dgx.dgx_imex_record(ctx, rec.data_ptr(), 4, 1)
    step(rm, um, pm)
    nrec = dgx.dgx_imex_recorded(ctx)
    dgx.dgx_imex_record(ctx, 0, 0, 1)
    diff = float((p_first - pm).abs().max() / (pm - p0).abs().max().clamp_min(1e-30))
    true_res = []
    yv = torch.zeros(N, dtype=f64, device="cuda")
    # native FP64 arithmetic for this check (variant 1: one cell per CTA, FP64 pipe),
    # whatever variant the autotuner chose for the solves; restored afterwards
    v_tuned = dgx.dgx_operator_variant(ctx, dgx.DGX_F64)
    dgx.dgx_set_operator_variant(ctx, dgx.DGX_F64, 1)
    for k in range(nrec):
        r_ = rec[k * (4 * N + 2):(k + 1) * (4 * N + 2)]
        rr, pk_, b_, x_ = r_[:N], r_[N:2 * N], r_[2 * N:3 * N], r_[3 * N:4 * N]
        dgx.dgx_set_coefficients(ctx, rr.data_ptr(), pk_.data_ptr(), float(r_[4 * N]), float(r_[4 * N + 1]))
        dgx.dgx_apply_operator(ctx, dgx.DGX_F64, x_.data_ptr(), yv.data_ptr())
        true_res.append(float((b_ - yv).norm() / b_.norm()))
    dgx.dgx_set_operator_variant(ctx, dgx.DGX_F64, v_tuned)
    del rm, um, pm, rec, p_first

    # ---- end to end through the C ABI with host buffers: state in from pinned host memory, step, state out
    h_state = [t.cpu().pin_memory() for t in (rho, u, p)]
    d_state = [t.clone() for t in (rho, u, p)]
    out_h = [torch.empty_like(t).pin_memory() for t in h_state]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        for d_, h_ in zip(d_state, h_state):
            d_.copy_(h_, non_blocking=True)
        step(*d_state)
        for h_, d_ in zip(out_h, d_state):
            h_.copy_(d_, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    t_e2e = e2.elapsed_time(e3) / 1e3
    t_e2e = replicas.max_over_ranks(pg, t_e2e, "cuda")
    io_bytes = sum(t.numel() * t.element_size() for t in h_state)
    del d_state

    if rank != 0:
        dgx.dgx_destroy(ctx)
        if pg:
            pg.destroy_process_group()
        return 0

    # ---- per-kernel durations (CUDA events on the library's stream) at the current coefficients
    def time_calls(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    R = args.vmult_reps
    x64 = (p - p0).contiguous()
    x32 = x64.float()
    y64 = torch.zeros(N, dtype=f64, device="cuda")
    y32 = torch.zeros(N, dtype=torch.float32, device="cuda")
    V64 = torch.zeros(3 * N, dtype=f64, device="cuda")
    V32 = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    Er, Em, Ee = (torch.zeros(N, dtype=f64, device="cuda"), torch.zeros(3 * N, dtype=f64, device="cuda"),
                  torch.zeros(N, dtype=f64, device="cuda"))
    t_app64 = time_calls(lambda: dgx.dgx_apply_operator(ctx, dgx.DGX_F64, x64.data_ptr(), y64.data_ptr()), R)
    t_app32 = time_calls(lambda: dgx.dgx_apply_operator(ctx, dgx.DGX_F32, x32.data_ptr(), y32.data_ptr()), 3 * R)
    t_grad64 = time_calls(lambda: dgx.dgx_apply_grad(ctx, dgx.DGX_F64, x64.data_ptr(), V64.data_ptr()), R)
    t_div64 = time_calls(lambda: dgx.dgx_apply_div(ctx, dgx.DGX_F64, V64.data_ptr(), x64.data_ptr(),
                                                   y64.data_ptr()), R)
    t_grad32 = time_calls(lambda: dgx.dgx_apply_grad(ctx, dgx.DGX_F32, x32.data_ptr(), V32.data_ptr()), 3 * R)
    t_div32 = time_calls(lambda: dgx.dgx_apply_div(ctx, dgx.DGX_F32, V32.data_ptr(), x32.data_ptr(),
                                                   y32.data_ptr()), 3 * R)
    t_expl = time_calls(lambda: dgx.dgx_explicit_tendencies(ctx, rho.data_ptr(), u.data_ptr(), Er.data_ptr(),
                                                            Em.data_ptr(), Ee.data_ptr()), max(2, R // 3))
    expl_variant = dgx.dgx_explicit_variant(ctx)
    dgx.dgx_set_explicit_variant(ctx, 1 - expl_variant)  # the other arithmetic, for comparison
    t_expl_other = time_calls(lambda: dgx.dgx_explicit_tendencies(ctx, rho.data_ptr(), u.data_ptr(), Er.data_ptr(),
                                                                  Em.data_ptr(), Ee.data_ptr()), max(2, R // 3))
    dgx.dgx_set_explicit_variant(ctx, expl_variant)
    fl_grad, fl_div, bytes64 = dgx.dgx_operator_cost(ctx)

    f64_applies = statistics.mean(i.operator_f64 for i in step_infos)
    f32_applies = statistics.mean(i.operator_f32 for i in step_infos)
    share = {"f64_operator": f64_applies * t_app64 + STEP_EXTRA_HALF_APPLIES * t_app64 / 2,
             "f32_operator": f32_applies * t_app32, "explicit": 2 * t_expl}
    peak64 = fp64_peak(torch)
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = clocks.get("sm_max_mhz") or 2070.0
    fp32_nominal = n_sm * 128 * 2 * sm_max_mhz * 1e6 / 1e12
    dom = max(share, key=share.get)
    # kernel names of the launch variant the autotuner chose (0-2: k_grad / k_div, 3-4: fused kf_grad / kf_div,
    # 5-6: the fused kernels in double-word arithmetic, kf_grad<df64> / kf_div<df64>)
    v64, v32 = dgx.dgx_operator_variant(ctx, dgx.DGX_F64), dgx.dgx_operator_variant(ctx, dgx.DGX_F32)
    pre32 = "kf_" if v32 >= 3 else "k_"
    pre64, t64 = ("kf_", "df64") if v64 >= 5 else (("kf_" if v64 >= 3 else "k_"), "double")
    fp32_src = ("derived: %d SMs (device properties) x 128 FP32 lanes x 2 flop x %.0f MHz (maximum SM clock)"
                % (n_sm, sm_max_mhz))
    extra = {}
    if dom == "f32_operator":
        kname, t_k, fl_k = ((pre32 + "div<float>", t_div32, fl_div) if t_div32 >= t_grad32
                            else (pre32 + "grad<float>", t_grad32, fl_grad))
        peak, peak_src = fp32_nominal, fp32_src
    else:
        kname, t_k, fl_k = ((pre64 + "div<%s>" % t64, t_div64, fl_div) if t_div64 >= t_grad64
                            else (pre64 + "grad<%s>" % t64, t_grad64, fl_grad))
        if t64 == "df64":
            # FP64-accuracy arithmetic on the FP32 pipes: one multiply-add of the line products (2 flops)
            # is a compensated dot-product term of 12 FP32 operations, so the roof in FP64-equivalent
            # flops is the FP32 peak / 6
            peak, peak_src = fp32_nominal / 6.0, ("derived: FP32 peak (%s) / 6 FP32 operations per FP64-"
                                                  "equivalent flop of the double-word multiply-add" % fp32_src)
            extra = {"fp64_dgemm_peak": peak64, "vs_fp64_dgemm_peak": fl_k / t_k / 1e12 / peak64}
        else:
            peak, peak_src = peak64, "measured cuBLAS DGEMM (torch.matmul float64 4096^3) on this GPU"
    achieved = fl_k / t_k / 1e12
    traffic = DRAM_BYTES_PER_DOF_F64[kname] * N if kname in DRAM_BYTES_PER_DOF_F64 else None
    hbm_gbs, hbm_src = measured_hbm_gbs()
    k_gbs, k_hbm_frac = hbm_fractions(traffic, t_k, hbm_gbs)
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": "ncu DRAM bytes per DoF on the 48x48x24 r=4 mesh, scaled by DoFs" if traffic else None,
                "peak_source": peak_src, "flops_per_launch": fl_k, "launch_s": t_k, "step_share_estimate_s": share,
                **extra,
                "hbm": {"achieved_gbs": k_gbs, "frac": k_hbm_frac, "peak_gbs": hbm_gbs, "peak_source": hbm_src,
                        "note": "the kernel's DRAM traffic per launch over its launch time: far below the copy "
                                "bandwidth, the arithmetic pipes bind"}}

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        v, sample, threads = oracle_step_cost(work, budget_s=15.0)
        cpu = {"value": v, "unit": "s/step", "cores": threads, "kind": "oracle", "sample": sample}
        v1, sample1, _ = oracle_step_cost(work, budget_s=8.0, threads=1)
        cpu["single_core"] = {"value": v1, "unit": "s/step", "cores": 1, "sample": sample1}

    value = t_dev / (args.steps * ws)
    mean = lambda k: statistics.mean(getattr(i, k) for i in step_infos)
    line = {
        "metric": METRIC, "value": value, "unit": "s/step", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": work["name"],
                   "mesh": "%dx%dx%d cells, r=%d, N=%d per field" % (work["nx"], work["ny"], work["nz"], work["r"], N),
                   "terrain": "bell h_c=400 m a_c=1 km centred, Gal-Chen", "background": "isothermal 250 K",
                   "boundaries": "far-field lateral (uniform 10 m/s inflow), slip walls bottom/top",
                   "initial": "background + 10 m/s wind",
                   "step": "dgx_imex_step: ARS(2,2,2), 2 fixed-point its, 4 mixed FGMRES(20)/FP32 GMRES(25) "
                           "solves to 1e-8",
                   "l2": "state and Krylov bases larger than L2 (no flush needed)", "parallelism": "replicas"},
        "e2e": {"value": t_e2e / (args.steps * ws), "unit": "s/step", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes},
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "pressure_solve_s_per_step": mean("seconds_solve"),
        "plain_fp64": plain,
        "mixed_vs_plain_max_rel_diff_p_prime": diff,
        "true_fp64_relres": {"values": true_res, "max": max(true_res) if true_res else None,
                             "how": "one more mixed step from the final state with its 4 systems recorded; "
                                    "||b - S x|| / ||b|| with S applied afresh by the native FP64 kernels "
                                    "(variant 1; outside the timed region)"},
        "device": {"name": torch.cuda.get_device_name(local), "multi_processor_count": n_sm},
        "step": {"solves": mean("solves"), "krylov_iterations": mean("krylov_iterations"),
                 "inner_iterations": mean("inner_iterations"), "operator_f64": f64_applies,
                 "operator_f32": f32_applies, "max_relres": max(i.max_relres for i in step_infos), "finite": finite},
        "vmult": {"f64_gdofs": N / t_app64 / 1e9, "f32_gdofs": N / t_app32 / 1e9, "f64_ms": t_app64 * 1e3,
                  "f32_ms": t_app32 * 1e3, "k_grad_f64_ms": t_grad64 * 1e3, "k_div_f64_ms": t_div64 * 1e3,
                  "k_grad_f32_ms": t_grad32 * 1e3, "k_div_f32_ms": t_div32 * 1e3, "k_explicit_ms": t_expl * 1e3,
                  "k_explicit_variant": expl_variant, "k_explicit_other_variant_ms": t_expl_other * 1e3,
                  "flops_per_apply": fl_grad + fl_div, "hbm_floor_bytes_f64": bytes64,
                  "f64_tflops": (fl_grad + fl_div) / t_app64 / 1e12, "f32_tflops": (fl_grad + fl_div) / t_app32 / 1e12,
                  "fp64_peak_measured_tflops": peak64,
                  "f64_hbm_floor_frac": hbm_fractions(bytes64, t_app64, hbm_gbs)[1],
                  "threads_per_cta_autotuned": {"f64": dgx.dgx_operator_threads(ctx, dgx.DGX_F64),
                                                "f32": dgx.dgx_operator_threads(ctx, dgx.DGX_F32)},
                  "variant_autotuned": {"f64": dgx.dgx_operator_variant(ctx, dgx.DGX_F64),
                                        "f32": dgx.dgx_operator_variant(ctx, dgx.DGX_F32)}},
    }
    dgx.dgx_destroy(ctx)
    if ws == 1 and not args.no_extras:
        line["extras"] = extras()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def extras():
    """Compact results of the mixed-precision (box at degrees 2, 3, 5) and
    learned-preconditioner workloads, each run by this script as a subprocess
    with its own defaults, so that a default run reports them as well."""
    out = {}
    for name, argv in (("mixed", ["--workload", "mixed", "--steps", "3", "--warmup", "3"]),
                       ("learned", ["--workload", "learned", "--steps", "1", "--warmup", "3"])):
        t0 = time.time()
        r = subprocess.run([sys.executable, os.path.abspath(__file__)] + argv, capture_output=True, text=True)
        js = [l for l in r.stdout.splitlines() if l.startswith("{")]
        if r.returncode != 0 or not js:
            out[name] = {"error": "rc %d: %s" % (r.returncode, (r.stderr or r.stdout)[-300:])}
            continue
        d = json.loads(js[-1])
        if name == "mixed":
            out[name] = {"unit": "s/solve", "wall_s": round(time.time() - t0, 1), "degrees": [
                {"degree": g["degree"], "dofs": g["dofs"], "mixed": g["mixed"]["s_per_solve"],
                 "plain_fp64": g["plain_fp64"]["s_per_solve"],
                 "mixed_max_rel_err_vs_oracle": g["mixed"]["max_rel_err_vs_oracle"],
                 "plain_max_rel_err_vs_oracle": g["plain_fp64"]["max_rel_err_vs_oracle"]} for g in d["degrees"]],
                "imex_step_vs_oracle": d.get("imex_step_vs_oracle")}
        else:
            keep = ("value", "unit", "solvers", "speedup_vs_plain_fp64", "iterations_ratio_vs_plain", "training")
            out[name] = {k: d[k] for k in keep if k in d}
            out[name]["wall_s"] = round(time.time() - t0, 1)
    return out


if __name__ == "__main__":
    sys.exit(main())
