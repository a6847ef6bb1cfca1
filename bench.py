#!/usr/bin/env python3
"""Benchmark of the GB300 pressure-solve hot path (one JSON line on rank 0).

Workload: terrain-following bell-shaped hill (h = 400 m / (1 + r^2 / (1 km)^2)
at the domain centre), 60 x 60 x 20 km, 64 x 64 x 32 cells at degree 4
(16 384 000 pressure DoFs), far-field lateral faces, isothermal background at
250 K, dt = 1 s, a~_ll = 1 - 1/sqrt(2) (ARS(2,2,2)).  Synthetic, seeded inputs.

One step = the implicit part of one IMEX stage with resident inputs:
  set_coefficients(rho^(l), p_k)   (copies + Helmholtz diagonal)
  solve S p' = b to 1e-8 FP64 relative residual (mixed: FP32 GMRES inside FP64 FGMRES)
  velocity recovery U = A^-1 F - A^-1 B p'.
The metric is seconds per step (lower is better); the plain FP64 FGMRES solve of
the same system and the operator throughput (vmult GDoF/s) are reported next
to it.  `--impl reference` times the FP64 CPU oracle on a bounded sample of the
same workload.
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

FULL = dict(name="hill_64x64x32_r4_16.4M_dofs", nx=64, ny=64, nz=32, r=4, Lx=60000.0, Ly=60000.0, Lz=20000.0)
SMALL = dict(name="hill_16x16x8_r4_256k_dofs", nx=16, ny=16, nz=8, r=4, Lx=15000.0, Ly=15000.0, Lz=5000.0)
COMMON = dict(terrain=1, hc=400.0, ac=1000.0, bc_lateral=1, T=250.0, p0=1e5, R=287.0, g=9.81, gamma=1.4, dt=1.0)
A_LL = 1.0 - 1.0 / 2.0 ** 0.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="small mesh (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vmult-reps", type=int, default=10)
    ap.add_argument("--mesh", default=None, help="NXxNYxNZ cells (keeps the 60x60x20 km domain scaled per cell)")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed steps (for profiler launch lists); no side measurements")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def oracle_sample(work, rho, pk, p, budget_s=12.0):
    """Time the FP64 oracle's operator on a bounded sample of cells; returns
    (seconds per full-mesh operator application, sample description, threads)."""
    import numpy as np
    import oracle as O
    m = O.make_mesh(work["nx"], work["ny"], work["nz"], work["r"], Lx=work["Lx"], Ly=work["Ly"], Lz=work["Lz"],
                    terrain=work["terrain"], hc=work["hc"], ac=work["ac"], bc_lateral=work["bc_lateral"])
    ncell = work["nx"] * work["ny"] * work["nz"]
    rng = np.random.default_rng(5)
    ncs = 8
    t = 0.0
    done = 0
    threads = O.max_threads()
    while True:
        cells = rng.choice(ncell, size=ncs, replace=False)
        t0 = time.perf_counter()
        O.apply_S(m, A_LL * work["dt"], work["gamma"], rho, pk, p, cells=cells)
        t += time.perf_counter() - t0
        done += ncs
        if t > budget_s or done >= ncell:
            break
        ncs = min(ncell - done, max(ncs, int(ncs * budget_s / max(t, 1e-3) / 4)))
    per_apply = t / done * ncell
    return per_apply, "operator S on %d random cells of %d (with face neighbours), %.1f s, scaled by cells" % (
        done, ncell, t), threads


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
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def run_reference(args, work):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from paper_2505_00384_gb300 import inputs
    import oracle as O
    N = work["nx"] * work["ny"] * work["nz"] * (work["r"] + 1) ** 3
    # coefficient fields on the oracle's own nodes (the GPU is not used)
    m = O.make_mesh(work["nx"], work["ny"], work["nz"], work["r"], Lx=work["Lx"], Ly=work["Ly"], Lz=work["Lz"],
                    terrain=work["terrain"], hc=work["hc"], ac=work["ac"], bc_lateral=work["bc_lateral"])
    X = O.node_coords(m)
    rho = inputs.perturbed_profile(X[2], 1.2, 7314.0, 0.01, 11)
    pk = inputs.perturbed_profile(X[2], 1e5, 7314.0, 0.01, 12)
    p = inputs.random_field(N, 13, 100.0)
    applies = 84  # FP64 operator applications of one plain FP64 FGMRES(30) solve of this system to 1e-8
    vals = []
    for _ in range(args.warmup + args.steps):
        per_apply, sample, threads = oracle_sample(work, rho, pk, p, budget_s=max(2.0, 20.0 / (args.steps + 1)))
        vals.append(per_apply * applies)
    v = statistics.median(vals[args.warmup:])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/step", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": work["name"]},
            "cpu_baseline": {"value": v, "unit": "s/step", "cores": threads, "kind": "oracle",
                             "sample": sample + "; x %d FP64 operator applications per solve" % applies},
            "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    work = dict(SMALL if args.small else FULL)
    if args.mesh:
        nx, ny, nz = (int(v) for v in args.mesh.lower().split("x"))
        # same cell size as the 64 x 64 x 32 workload (937.5 m x 937.5 m x 625 m)
        work.update(name="hill_%dx%dx%d_r4" % (nx, ny, nz), nx=nx, ny=ny, nz=nz, Lx=937.5 * nx, Ly=937.5 * ny,
                    Lz=625.0 * nz)
    work.update(COMMON)
    if args.impl == "reference":
        return run_reference(args, work)

    import numpy as np
    import torch
    from paper_2505_00384_gb300 import dgx, inputs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    dgx.load()
    stream = torch.cuda.current_stream()
    ctx = dgx.dgx_create(local, stream.cuda_stream)
    desc = dgx.mesh_desc(work["nx"], work["ny"], work["nz"], work["r"], work["Lx"], work["Ly"], work["Lz"],
                         terrain=work["terrain"], h_c=work["hc"], a_c=work["ac"], bc_lateral=work["bc_lateral"])
    dgx.dgx_mesh_build(ctx, desc)
    N = dgx.dgx_num_dofs(ctx)
    bg = dgx.background(kind=0, T=work["T"], p0=work["p0"], R=work["R"], gamma=work["gamma"], g=work["g"])
    dgx.dgx_set_background(ctx, bg)
    f64 = torch.float64
    X = torch.zeros(3 * N, dtype=f64, device="cuda")
    dgx.dgx_node_coords(ctx, X.data_ptr())
    rho_bar = torch.zeros(N, dtype=f64, device="cuda")
    p_bar = torch.zeros(N, dtype=f64, device="cuda")
    dgx.dgx_background_fields(ctx, rho_bar.data_ptr(), p_bar.data_ptr())
    # synthetic stage state: background times (1 + 1e-3 seeded noise)
    seed = inputs.DEFAULT_SEED + 97 * rank
    rho = rho_bar * torch.from_numpy(1.0 + 1e-3 * inputs.normal(seed, N)).cuda()
    pk = p_bar * torch.from_numpy(1.0 + 1e-3 * inputs.normal(seed + 1, N)).cuda()
    a_dt = A_LL * work["dt"]
    dgx.dgx_set_coefficients(ctx, rho.data_ptr(), pk.data_ptr(), a_dt, work["gamma"])
    # right-hand side b = S p_true, p_true a 100 Pa Gaussian bubble (sigma 2 km) plus noise
    Xh = X.cpu().numpy().reshape(3, -1)
    ptrue = 100.0 * np.exp(-(((Xh[0] - 30000.0) ** 2 + (Xh[1] - 30000.0) ** 2 + (Xh[2] - 5000.0) ** 2)
                             / (2 * 2000.0 ** 2))) + inputs.normal(seed + 2, N)
    ptrue_d = torch.from_numpy(ptrue).cuda()
    b = torch.zeros(N, dtype=f64, device="cuda")
    dgx.dgx_apply_operator(ctx, dgx.DGX_F64, ptrue_d.data_ptr(), b.data_ptr())
    F = torch.from_numpy(inputs.random_field(3 * N, seed + 3, 1e3)).cuda()
    x = torch.zeros(N, dtype=f64, device="cuda")
    U = torch.zeros(3 * N, dtype=f64, device="cuda")
    AF = torch.zeros(3 * N, dtype=f64, device="cuda")
    torch.cuda.synchronize()

    def opts(method):
        o = dgx.dgx_default_solve_opts()
        o.method, o.pc, o.tol, o.maxit = method, dgx.DGX_PC_HELMHOLTZ, 1e-8, 2000
        o.restart = 20 if method == dgx.DGX_SOLVER_MIXED else 30
        o.inner_maxit, o.inner_tol = 30, 1e-5
        return o

    o_mixed = opts(dgx.DGX_SOLVER_MIXED)
    infos = []

    def step(rho_d, pk_d, b_d, F_d, x_d, U_d):
        dgx.dgx_set_coefficients(ctx, rho_d.data_ptr(), pk_d.data_ptr(), a_dt, work["gamma"])
        st, info = dgx.dgx_solve_pressure(ctx, b_d.data_ptr(), x_d.data_ptr(), o_mixed)
        if st != dgx.DGX_OK:
            raise RuntimeError("pressure solve did not converge: relres %g" % info.relres)
        dgx.dgx_apply_mass_inverse(ctx, dgx.DGX_F64, F_d.data_ptr(), AF.data_ptr())
        dgx.dgx_apply_grad(ctx, dgx.DGX_F64, x_d.data_ptr(), U_d.data_ptr())
        torch.sub(AF, U_d, out=U_d)
        infos.append(info)

    # ---- operator throughput (vmult) and per-kernel durations, CUDA events on the library's stream
    def time_calls(fn, reps):
        if reps == 0:
            return float("nan")
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    y64 = torch.zeros(N, dtype=f64, device="cuda")
    x32 = ptrue_d.float()
    if args.profile:
        args.vmult_reps = 0
    y32 = torch.zeros(N, dtype=torch.float32, device="cuda")
    V64 = torch.zeros(3 * N, dtype=f64, device="cuda")
    V32 = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    R = args.vmult_reps
    t_app64 = time_calls(lambda: dgx.dgx_apply_operator(ctx, dgx.DGX_F64, ptrue_d.data_ptr(), y64.data_ptr()), R)
    t_app32 = time_calls(lambda: dgx.dgx_apply_operator(ctx, dgx.DGX_F32, x32.data_ptr(), y32.data_ptr()), 3 * R)
    t_grad64 = time_calls(lambda: dgx.dgx_apply_grad(ctx, dgx.DGX_F64, ptrue_d.data_ptr(), V64.data_ptr()), R)
    t_div64 = time_calls(lambda: dgx.dgx_apply_div(ctx, dgx.DGX_F64, V64.data_ptr(), ptrue_d.data_ptr(),
                                                   y64.data_ptr()), R)
    t_grad32 = time_calls(lambda: dgx.dgx_apply_grad(ctx, dgx.DGX_F32, x32.data_ptr(), V32.data_ptr()), 3 * R)
    t_div32 = time_calls(lambda: dgx.dgx_apply_div(ctx, dgx.DGX_F32, V32.data_ptr(), x32.data_ptr(),
                                                   y32.data_ptr()), 3 * R)
    fl_grad, fl_div, bytes64 = dgx.dgx_operator_cost(ctx)

    # ---- plain FP64 solve of the same system (reference point of the metric)
    plain = None
    if not args.profile:
        xp = torch.zeros(N, dtype=f64, device="cuda")
        st, info_plain = dgx.dgx_solve_pressure(ctx, b.data_ptr(), xp.data_ptr(), opts(dgx.DGX_SOLVER_FGMRES))
        plain = {"s_per_solve": info_plain.seconds, "iterations": info_plain.iterations,
                 "operator_f64": info_plain.operator_f64, "relres": info_plain.relres, "status": st}
        del xp

    # ---- timed steps (inputs resident in HBM; the Krylov basis, 4+ GB, exceeds L2)
    for _ in range(args.warmup):
        step(rho, pk, b, F, x, U)
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
            step(rho, pk, b, F, x, U)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = dgx.dgx_kernel_launches() - launches0
    t_dev = e0.elapsed_time(e1) / 1e3
    if pg:
        tt = torch.tensor([t_dev], dtype=f64, device="cuda")
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_dev = float(tt.item())
        pg.barrier()
    err_true = float((x - ptrue_d).abs().max() / ptrue_d.abs().max())

    if args.profile:
        print(json.dumps({"profile_run": True, "workload": work["name"], "N": N, "steps": args.steps,
                          "s_per_step": t_dev / args.steps, "launches": launches}), flush=True)
        dgx.dgx_destroy(ctx)
        return 0

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    h_in = [t.cpu().pin_memory() for t in (rho, pk, b, F)]
    h_x = torch.zeros(N, dtype=f64).pin_memory()
    h_U = torch.zeros(3 * N, dtype=f64).pin_memory()
    d_in = [torch.empty_like(t) for t in (rho, pk, b, F)]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        for d_, h_ in zip(d_in, h_in):
            d_.copy_(h_, non_blocking=True)
        step(d_in[0], d_in[1], d_in[2], d_in[3], x, U)
        h_x.copy_(x, non_blocking=True)
        h_U.copy_(U, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    t_e2e = e2.elapsed_time(e3) / 1e3
    if pg:
        tt = torch.tensor([t_e2e], dtype=f64, device="cuda")
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_e2e = float(tt.item())
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = (h_x.numel() + h_U.numel()) * 8

    if rank != 0:
        dgx.dgx_destroy(ctx)
        if pg:
            pg.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel of the timed step
    f64_applies = statistics.mean(i.operator_f64 for i in infos)
    f32_applies = statistics.mean(i.operator_f32 for i in infos)
    share64 = f64_applies * t_app64
    share32 = f32_applies * t_app32
    peak64 = fp64_peak(torch)
    clocks = clk.summary()
    fp32_nominal = 152 * 128 * 2 * 2.07e9 / 1e12
    if share64 >= share32:
        kname, t_k, fl_k = ("k_div<double>", t_div64, fl_div) if t_div64 >= t_grad64 else ("k_grad<double>", t_grad64,
                                                                                          fl_grad)
        peak, peak_src = peak64, "measured cuBLAS DGEMM (torch.matmul float64 4096^3) on this GPU"
    else:
        kname, t_k, fl_k = ("k_div<float>", t_div32, fl_div) if t_div32 >= t_grad32 else ("k_grad<float>", t_grad32,
                                                                                         fl_grad)
        peak, peak_src = fp32_nominal, "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    achieved = fl_k / t_k / 1e12
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                "flops_per_launch": fl_k, "launch_s": t_k}

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        rho_h, pk_h, p_h = rho.cpu().numpy(), pk.cpu().numpy(), ptrue
        per_apply, sample, threads = oracle_sample(work, rho_h, pk_h, p_h, budget_s=15.0)
        v = per_apply * plain["operator_f64"]
        cpu = {"value": v, "unit": "s/step", "cores": threads, "kind": "oracle",
               "sample": sample + "; x %d FP64 operator applications of the plain FGMRES solve" % plain["operator_f64"]}

    value = t_dev / (args.steps * ws)
    line = {
        "metric": METRIC, "value": value, "unit": "s/step", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": work["name"], "mesh": "%dx%dx%d cells, r=%d, N=%d" % (work["nx"], work["ny"], work["nz"],
                                                                                   work["r"], N),
                   "terrain": "bell h_c=400 m a_c=1 km, Gal-Chen", "background": "isothermal 250 K",
                   "step": "set_coefficients + mixed FGMRES(20)/FP32 GMRES(30) to 1e-8 + velocity recovery",
                   "l2": "inputs and Krylov basis larger than L2 (no flush needed)", "parallelism": "replicas"},
        "e2e": {"value": t_e2e / (args.steps * ws), "unit": "s/step", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "plain_fp64": plain,
        "solve": {"outer_iterations": statistics.mean(i.iterations for i in infos),
                  "inner_iterations": statistics.mean(i.inner_iterations for i in infos),
                  "operator_f64": f64_applies, "operator_f32": f32_applies,
                  "relres": max(i.relres for i in infos), "max_rel_err_vs_p_true": err_true},
        "vmult": {"f64_gdofs": N / t_app64 / 1e9, "f32_gdofs": N / t_app32 / 1e9,
                  "f64_ms": t_app64 * 1e3, "f32_ms": t_app32 * 1e3,
                  "k_grad_f64_ms": t_grad64 * 1e3, "k_div_f64_ms": t_div64 * 1e3,
                  "k_grad_f32_ms": t_grad32 * 1e3, "k_div_f32_ms": t_div32 * 1e3,
                  "flops_per_apply": fl_grad + fl_div, "hbm_floor_bytes_f64": bytes64,
                  "f64_tflops": (fl_grad + fl_div) / t_app64 / 1e12,
                  "f32_tflops": (fl_grad + fl_div) / t_app32 / 1e12,
                  "fp64_peak_measured_tflops": peak64},
    }
    print(json.dumps(line), flush=True)
    dgx.dgx_destroy(ctx)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
