#!/usr/bin/env python
"""Benchmark of the B300 monolithic ALE cylinder solver.

One step = one BDF2 time step of the cylinder case, Newton-converged to
||NL||_2 <= 1e-10 (residual, Jacobian, multifrontal factorisation, refined
solve, update - every phase on the GPU through the C ABI).  The default
workload is the 38,800-quad O-grid cylinder (Re 200, U* 10, dt 0.02) on the
mixed path (FP32 fronts, FP64 residual / refinement / state); the plain FP64
path on the same workload is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica of the case (the case
does not shard; replicas only) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time steps/s at ||r||<=1e-10 (BDF2 + Newton, cylinder VIV, mixed path)"
WORKLOADS = {
    # name: O-grid refinement m (quads = 1552 (m/12)^2 -> m=60: 38,800), Re, U*, dt
    "viv_re200_m60": dict(m=60, Re=200.0, Ustar=10.0, dt=0.02),
    "viv_re100_m12": dict(m=12, Re=100.0, Ustar=8.0, dt=0.1),
    "viv_re100_m24": dict(m=24, Re=100.0, Ustar=8.0, dt=0.05),
    "viv_re200_m40": dict(m=40, Re=200.0, Ustar=10.0, dt=0.02),   # (profiling: top fronts of ~2,500)
    # 3-D: the m = 7 section (555 quads) extruded into 24 periodic layers over a 2 pi span
    # (13,320 Q2-Q1 hexahedra, 662,114 unknowns), Re 300, U* 8 (L = span), dt 0.05
    "viv3d_re300_m7_z24": dict(m=7, layers=24, span=2.0 * math.pi, Re=300.0, Ustar=8.0, dt=0.05),
    # the paper's own spaces (P2-P1 triangles, P1 position) on the headline mesh split into
    # 77,600 triangles with straight edges
    "viv_tri_re200_m60": dict(m=60, tri=True, Re=200.0, Ustar=10.0, dt=0.02),
    # (profiling: the m = 4 section, 188 quads, in 8 layers of the same thickness: 1,504 hexahedra, 5.5 GB)
    "viv3d_re300_m4_z8": dict(m=4, layers=8, span=2.0 * math.pi / 3.0, Re=300.0, Ustar=8.0, dt=0.05),
    # (profiling: the m = 5 section, 251 quads, in 12 layers of the same thickness: 3,012 hexahedra)
    "viv3d_re300_m5_z12": dict(m=5, layers=12, span=math.pi, Re=300.0, Ustar=8.0, dt=0.05),
}
FP32_SIMT_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12      # 148 SMs x 128 FP32 lanes x FMA x 2.032 GHz
FP64_TFLOPS = 1.25                                       # B300 FP64, nominal
# DRAM bytes (read + write) per 128 x 128 tile of the tensor-core Schur update (tc_pipe_kernel), from one
# ncu capture of that kernel; None until a capture of the current kernel exists (the line's traffic is null)
TC_DRAM_BYTES_PER_TILE = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="viv_re200_m60", choices=sorted(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--oracle-full-steps", type=int, default=10,
                    help="steps of the fully timed oracle run on the 1,552-quad case (0: skip)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip viv_autotune (large-front threshold and per-level block LU choice) before "
                         "the warm-up steps")
    ap.add_argument("--big-front", type=int, default=0,
                    help="with --block-levels: set this schedule instead of autotuning (reproducible profiles)")
    ap.add_argument("--block-levels", type=int, default=None,
                    help="tree levels allowed the block LU (bit mask), with --big-front")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-cases", type=int, default=16)
    ap.add_argument("--sweep-steps", type=int, default=10)
    ap.add_argument("--pivoting", default="window", choices=["window", "threshold"],
                    help="front pivoting: partial pivoting inside each 32-row diagonal block (window) or "
                         "threshold pivoting over all fully summed rows")
    ap.add_argument("--no-threshold-path", action="store_true")
    ap.add_argument("--no-reuse-path", action="store_true",
                    help="skip the line of the mixed path with factor_reuse (factors of a step's first Newton "
                         "iterate preconditioning the later iterates' refined solves)")
    ap.add_argument("--predictor", default="extrapolate", choices=["extrapolate", "previous"],
                    help="Newton starting point of a BDF2 step: 2 U^n - U^(n-1) or U^n")
    ap.add_argument("--jacobian", default="fp32", choices=["fp32", "fp64"],
                    help="mixed path: volume element Jacobians in FP32 (faces, border rows, residual and "
                         "refinement stay FP64) or everything in FP64")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_throughput(ms_local, steps, world, device=None):
    """Whole-job throughput of `world` independent replicas that each ran
    `steps` steps in `ms_local` ms: the job time is the slowest rank's (a MAX
    all-reduce over the process group); returns (job ms, steps/s)."""
    t_max = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * steps / (t_max / 1e3)


# ---------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        # raw samples: $VIV_BENCH_CLOCKS_DIR if set (to keep them), else the temp directory
        out_dir = os.environ.get("VIV_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"viv_clocks_{os.getpid()}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        self.f = open(self.path, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_id)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# ---------------------------------------------------------------------------------
def oracle_sample(wl, newton_iters):
    """Time the FP64 oracle on a bounded sample of the workload and scale it to
    one time step: residual on the full mesh, complex-step Jacobian on 1/32 of
    the elements (x32), sparse LU (SuperLU) of the 6,208-quad member of the same
    mesh family (x (N/N_6208)^1.5, the 2-D nested-dissection cost law).
    Returns (steps/s, description, seconds of CPU work)."""
    import numpy as np
    from paper_2609_31477_b300 import inputs as I
    from oracle.solver import sparse_lu, viv_oracle_case
    from oracle.solver_tri import viv_oracle_case_tri
    tri = bool(wl.get("tri"))
    make_mesh = (lambda m: I.triangulate_q2(I.viv_cylinder_mesh(m))) if tri else I.viv_cylinder_mesh
    make_case = viv_oracle_case_tri if tri else viv_oracle_case
    t_all = time.perf_counter()
    mesh = make_mesh(wl["m"])
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    oc = make_case(mesh, wl["Re"], wl["Ustar"], wl["dt"], u0)
    oc.u_n, oc.x_n = oc.u.copy(), oc.x.copy()
    c0, hu, hx = oc.bdf_coefficients()
    t0 = time.perf_counter()
    oc.residual(c0, hu, hx, wl["dt"])
    t_res = time.perf_counter() - t0
    # Jacobian on an element subset
    E = len(mesh["conn"])
    sub_e = np.arange(0, E, 32)
    conn = mesh["conn"][sub_e]
    used, inv = np.unique(conn, return_inverse=True)
    sub = dict(X=mesh["X"][used], conn=inv.reshape(conn.shape), tags=mesh["tags"][used] & ~I.CYL,
               gamma_faces=np.zeros((0, 2), np.int64))
    sc = make_case(sub, wl["Re"], wl["Ustar"], wl["dt"], u0[used])
    sc.u_n, sc.x_n = sc.u.copy(), sc.x.copy()
    c0s, hus, hxs = sc.bdf_coefficients()
    t0 = time.perf_counter()
    sc.jacobian(c0s, hus, hxs, wl["dt"])
    t_jac = (time.perf_counter() - t0) * E / len(sub_e)
    # LU on the 6,208-quad member of the family
    m24 = make_mesh(24)
    lc = make_case(m24, wl["Re"], wl["Ustar"], wl["dt"], I.viv_initial_velocity(m24, 1.0, 1e-3, 1))
    lc.u_n, lc.x_n = lc.u.copy(), lc.x.copy()
    c0l, hul, hxl = lc.bdf_coefficients()
    J24 = lc.jacobian(c0l, hul, hxl, wl["dt"]).tocsc()
    t0 = time.perf_counter()
    sparse_lu(J24)
    t_lu24 = time.perf_counter() - t0
    t_lu = t_lu24 * (oc.ndof / lc.ndof) ** 1.5
    per_step = newton_iters * (t_res + t_jac + t_lu) + t_res
    kind = "triangle" if tri else "quad"
    desc = (f"oracle on {E}-{kind} mesh: residual full ({t_res:.2f}s), complex-step Jacobian on 1/32 of the "
            f"elements x32 ({t_jac:.1f}s), SuperLU of the {len(m24['conn'])}-{kind} mesh scaled by (N ratio)^1.5 "
            f"({t_lu24:.1f}s -> {t_lu:.0f}s); {newton_iters:.2f} Newton iterations per step; extrapolated")
    return 1.0 / per_step, desc, time.perf_counter() - t_all


def oracle_sample3d(wl, newton_iters):
    """The 3-D form of `oracle_sample`: residual on the full hexahedral mesh,
    complex-step Jacobian on 1/64 of the elements (x64), sparse LU (SuperLU)
    of the 194-hexahedron member (the m = 3 section in 2 layers) scaled by
    (N ratio)^2, the 3-D nested-dissection cost law."""
    import numpy as np
    from paper_2609_31477_b300 import inputs as I
    from oracle.solver import sparse_lu
    from oracle.solver3d import viv_oracle_case3d
    t_all = time.perf_counter()
    mesh = I.viv_cylinder_mesh3d(wl["m"], wl["layers"], wl["span"])
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    oc = viv_oracle_case3d(mesh, wl["Re"], wl["Ustar"], wl["dt"], u0)
    oc.u_n, oc.x_n = oc.u.copy(), oc.x.copy()
    c0, hu, hx = oc.bdf_coefficients()
    t0 = time.perf_counter()
    oc.residual(c0, hu, hx, wl["dt"])
    t_res = time.perf_counter() - t0
    E = len(mesh["conn"])
    sub_e = np.arange(0, E, 64)
    conn = mesh["conn"][sub_e]
    used, inv = np.unique(conn, return_inverse=True)
    sub = dict(X=mesh["X"][used], conn=inv.reshape(conn.shape), tags=mesh["tags"][used] & ~I.CYL,
               gamma_faces=np.zeros((0, 2), np.int64), wrap=mesh["wrap"][sub_e], span=mesh["span"])
    sc = viv_oracle_case3d(sub, wl["Re"], wl["Ustar"], wl["dt"], u0[used])
    sc.u_n, sc.x_n = sc.u.copy(), sc.x.copy()
    c0s, hus, hxs = sc.bdf_coefficients()
    t0 = time.perf_counter()
    sc.jacobian(c0s, hus, hxs, wl["dt"])
    t_jac = (time.perf_counter() - t0) * E / len(sub_e)
    small = I.viv_cylinder_mesh3d(3, 2, wl["span"] * 2 / wl["layers"])
    lc = viv_oracle_case3d(small, wl["Re"], wl["Ustar"], wl["dt"], I.viv_initial_velocity(small, 1.0, 1e-3, 1))
    lc.u_n, lc.x_n = lc.u.copy(), lc.x.copy()
    c0l, hul, hxl = lc.bdf_coefficients()
    Js = lc.jacobian(c0l, hul, hxl, wl["dt"]).tocsc()
    t0 = time.perf_counter()
    sparse_lu(Js)
    t_lus = time.perf_counter() - t0
    t_lu = t_lus * (oc.ndof / lc.ndof) ** 2
    per_step = newton_iters * (t_res + t_jac + t_lu) + t_res
    desc = (f"oracle on {E}-hexahedron mesh: residual full ({t_res:.1f}s), complex-step Jacobian on 1/64 of the "
            f"elements x64 ({t_jac:.0f}s), SuperLU of the {len(small['conn'])}-hexahedron mesh scaled by "
            f"(N ratio)^2 ({t_lus:.1f}s -> {t_lu:.0f}s); {newton_iters:.2f} Newton iterations per step; extrapolated")
    return 1.0 / per_step, desc, time.perf_counter() - t_all


def host_info():
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model,
            "threads_used": 1, "note": "the oracle's element loops and SuperLU run on one core"}


def oracle_full_run(steps):
    """The oracle as it stands, fully timed (no extrapolation) on the 1,552-quad
    cylinder case (Re 100, U* 8, dt 0.1, seed 1): `steps` BDF steps, each
    Newton-converged to ||NL|| <= 1e-10.  Returns steps/s and the seconds."""
    from paper_2609_31477_b300 import inputs as I
    from oracle.solver import viv_oracle_case
    mesh = I.viv_cylinder_mesh(12)
    oc = viv_oracle_case(mesh, 100.0, 8.0, 0.1, I.viv_initial_velocity(mesh, 1.0, 1e-3, 1))
    t0 = time.perf_counter()
    newton = 0
    for _ in range(steps):
        newton += len(oc.step()) - 1
    el = time.perf_counter() - t0
    return {"value": steps / el, "unit": "time steps/s", "steps": steps, "seconds": round(el, 2),
            "newton_iters_per_step": newton / steps, "workload": "viv_re100_m12 (1,552 quads, 26,554 unknowns)",
            "kind": "oracle, fully timed"}


# ---------------------------------------------------------------------------------
def run_sweep(viv, I, n_cases, n_steps, pivoting, jacobian_fp32, predictor, seed=7):
    """Served parameter sweep (a sample of the 64-case, 200-step sweep): cases
    with 2k-20k quads, Re ~ U[100, 300], U* log-uniform in [4, 20], Poisson
    arrivals, a 24 GB device budget; every case runs n_steps BDF steps."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ms_set = (14, 22, 30, 38, 43)                      # O-grid refinements: 2.1k .. 19.9k quads
    meshes, dev = {}, {}
    cases = []
    for k in range(n_cases):
        quads = rng.uniform(2000, 20000)
        m = min(ms_set, key=lambda v: abs(1552 * (v / 12) ** 2 - quads))
        Re = rng.uniform(100, 300)
        Us = float(np.exp(rng.uniform(np.log(4), np.log(20))))
        cases.append((m, Re, Us))
    for m, _, _ in cases:
        if m not in meshes:
            meshes[m] = I.viv_cylinder_mesh(m)
            dev[m] = viv.Mesh(meshes[m])
    arrivals = np.cumsum(rng.exponential(0.05, size=n_cases))
    srv = viv.Server(24 << 30, max_active=16)
    for k, (m, Re, Us) in enumerate(cases):
        srv.submit(dev[m], I.viv_initial_velocity(meshes[m], 1.0, 1e-3, 100 + k), Re=Re, Ustar=Us, dt=0.02,
                   n_steps=n_steps, arrival_time=float(arrivals[k]), pivoting=pivoting,
                   jacobian_fp32=jacobian_fp32, predictor=predictor)
    res = srv.wait_all(n_cases, timeout_s=900)
    st = srv.stats()
    srv.close()
    ok = sum(r["status"] == "OK" for r in res)
    last = max(r["finish_s"] for r in res) if res else 0.0
    return {"cases": n_cases, "ok": ok, "steps_per_case": n_steps, "step_ms_p50": st["step_ms_p50"],
            "step_ms_p99": st["step_ms_p99"], "steady_step_ms_p50": st["steady_ms_p50"],
            "steady_step_ms_p99": st["steady_ms_p99"],
            "steady_note": "without each case's first two steps (they capture its CUDA graphs)",
            "steps": st["steps"], "elapsed_s": last,
            "steps_per_s": st["steps"] / last if last else None,
            "cases_per_hour_at_200_steps": 3600.0 * ok / last * n_steps / 200.0 if last else None,
            "peak_active": st["peak_active"], "peak_gb": st["peak_bytes"] / 1e9,
            "quads": sorted({int(1552 * (m / 12) ** 2) for m, _, _ in cases}),
            "sample": ("the full sweep: 64 cases x 200 steps" if (n_cases, n_steps) == (64, 200) else
                       f"{n_cases} of 64 cases, {n_steps} of 200 steps each; cases/hour extrapolated")}


def run_reference(args, wl, rank):
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        v, desc, secs = (oracle_sample3d if "layers" in wl else oracle_sample)(wl, 3.0)
        if i >= args.warmup:
            steps.append(v)
    value = sum(steps) / len(steps)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "time steps/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, **wl},
           "cpu_baseline": {"value": value, "unit": "time steps/s", "cores": 1, "kind": "oracle", "sample": desc,
                            "host": host_info()},
           "e2e": {"value": value, "unit": "time steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, wl, rank, world, local):
    import numpy as np
    import torch
    from paper_2609_31477_b300 import build, inputs as I, viv

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    viv.load()
    three_d, tri = "layers" in wl, bool(wl.get("tri"))
    if three_d:
        mesh = I.viv_cylinder_mesh3d(wl["m"], wl["layers"], wl["span"])
    elif tri:
        mesh = I.triangulate_q2(I.viv_cylinder_mesh(wl["m"]))
    else:
        mesh = I.viv_cylinder_mesh(wl["m"])
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1 + rank)
    M = viv.Mesh(mesh)
    info = M.info
    piv = viv.VIV_PIVOT_WINDOW if args.pivoting == "window" else viv.VIV_PIVOT_THRESHOLD
    j32 = 1 if args.jacobian == "fp32" else 0
    pred = 1 if args.predictor == "extrapolate" else 0
    case = viv.viv_case(M, wl["Re"], wl["Ustar"], wl["dt"], u0, precision=viv.VIV_MIXED, pivoting=piv,
                        jacobian_fp32=j32, predictor=pred)
    stream = case.stream           # every kernel of the case runs on its own stream
    if args.block_levels is not None or args.big_front:
        args.autotune = False
        if args.big_front:
            case.set_big_front(args.big_front)
        if args.block_levels is not None:
            case.set_block_levels(args.block_levels)
        info = M.refresh_info()
    if args.autotune:
        tuned = case.autotune()
        info = M.refresh_info()
    for _ in range(args.warmup):
        case.step()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gpu_id = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(gpu_id)
    l0 = viv.kernel_launches()
    # (for an ncu launch list of the timed steps: this library's launches before them,
    # to pass as ncu --kernel-name-base mangled -k regex:_ZN3viv -s <count>)
    print(f"# library kernel launches before the timed steps: {l0}", file=sys.stderr, flush=True)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [case.step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = viv.kernel_launches() - l0
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    # per-kernel-kind CUDA events on the case stream, over K more steps
    case.profile(True)
    torch.cuda.synchronize()
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    pinfos = [case.step() for _ in range(args.steps)]
    ep1.record(stream)
    torch.cuda.synchronize()
    kern = case.profile_read()
    case.profile(False)
    prof_ms = ep0.elapsed_time(ep1)
    t_max, value = replica_throughput(ms, args.steps, world, torch.device("cuda", local))
    newton = sum(i["newton_iters"] for i in infos) / len(infos)
    sweeps = sum(i["refine_sweeps"] for i in infos) / len(infos)
    n_fact = sum(i["newton_iters"] for i in pinfos)
    sweeps_p = sum(i["refine_sweeps"] for i in pinfos)

    # roofline of every kernel class from the events of the profiled pass;
    # the dominant class (most time) is the headline
    peaks, src = measured_peaks()
    bf16_key = "bf16_tflops_sustained" if "bf16_tflops_sustained" in peaks else "bf16_tflops"
    tc_peak = peaks[bf16_key] / 2.0 / 3.0
    fbytes = 4 * info["front_entries"]
    # factor entries p (2m - p) per front (L and U with the pivot block; a front's contribution
    # block is not factor data): a forward or backward sweep reads about half of them
    fr = M.fronts()
    factor_bytes = 4 * float(np.sum(fr["p"].astype(np.float64) * (2.0 * fr["m"] - fr["p"])))
    window = args.pivoting == "window"
    tc_flops = info["window_tc_flops"] if window else info["outer_flops"]

    def roofline_of(kind):
        k_ms, k_n = kern[kind]
        if k_ms <= 0:
            return None
        sec = k_ms / 1e3
        if kind == "tc_schur_gemm":
            # kind::tf32 with three products per FP32 multiply-add (3xTF32): algorithmic
            # FP32 flops / time against TF32 dense (BF16 measured / 2, nominal) / 3
            a = tc_flops * n_fact / sec / 1e12
            return {"bound": "tensor", "achieved": a, "peak": tc_peak, "unit": "TFLOP/s", "frac": a / tc_peak,
                    "peak_source": f"{src} {bf16_key} / 2 (TF32:BF16 nominal) / 3 (3xTF32 products)"}
        if kind in ("schur_gemm", "panel_lu", "trsm"):
            if window:
                fl = {"schur_gemm": info["window_gemm_flops"], "panel_lu": info["window_lu_flops"]}.get(kind)
                if fl is None:   # (windowed: row moves and window solves, no flop count)
                    return None
            else:
                fl = {"schur_gemm": info["gemm_flops"] - info["outer_flops"],
                      "panel_lu": info["panel_flops"], "trsm": info["trsm_flops"]}[kind]
            a = fl * n_fact / sec / 1e12
            return {"bound": "alu", "achieved": a, "peak": FP32_SIMT_TFLOPS, "unit": "TFLOP/s",
                    "frac": a / FP32_SIMT_TFLOPS,
                    "peak_source": "FP32 SIMT: 148 SMs x 128 lanes x 2 flop x 2.032 GHz (derived)"}
        if kind == "residual":
            # FP64 ALU: about 4k double FMAs per quad (2-D), 1.5k per triangle or 75k per hexahedron (3-D)
            # (quadrature of the Q2-Q1-Q2 element residual, counted from the kernels' loops), against
            # the nominal FP64 rate
            evals = n_fact + args.steps          # one per Newton iteration, one for the converged state
            a = (1.5e5 if three_d else (3.0e3 if tri else 8.0e3)) * len(mesh["conn"]) * evals / sec / 1e12
            return {"bound": "alu", "achieved": a, "peak": FP64_TFLOPS, "unit": "TFLOP/s", "frac": a / FP64_TFLOPS,
                    "peak_source": "FP64 nominal 1.25 TFLOP/s (no FP64 measurement); flops approximate"}
        per = {"fwd_solve": factor_bytes / 2, "bwd_solve": factor_bytes / 2, "front_assemble": 2 * fbytes,
               "spmv": 12 * info["nnz"] + 24 * info["n_dofs"], "jacobian": 12 * info["nnz"]}.get(kind)
        if per is None:
            return None
        calls = sweeps_p if kind in ("fwd_solve", "bwd_solve", "spmv") else n_fact
        a = per * calls / sec / 1e9
        return {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                "peak_source": src}

    rooflines = {}
    for kind in kern:
        r = roofline_of(kind)
        if r is not None:
            rooflines[kind] = {"achieved": round(r["achieved"], 3), "unit": r["unit"], "frac": round(r["frac"], 4)}
    dom = max((k for k in kern if roofline_of(k) is not None), key=lambda k: kern[k][0])
    roof = roofline_of(dom)
    traffic = None
    if dom == "tc_schur_gemm" and kern[dom][1] and TC_DRAM_BYTES_PER_TILE:
        # tiles per launch from the tensor-core flops (K = 128 per tile)
        tiles = tc_flops * n_fact / (2.0 * 128 * 128 * 128) / kern[dom][1]
        traffic = TC_DRAM_BYTES_PER_TILE * tiles
        roof["traffic_note"] = (f"ncu DRAM bytes per tile x {tiles:.0f} tiles per launch; algorithmic "
                                "operand + C bytes per tile without reuse: 393216")
    roof.update({"traffic": traffic, "kernel": dom, "launches": kern[dom][1], "ms_total": kern[dom][0]})

    out = {"metric": METRIC, "value": value, "unit": "time steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": ("f32 fronts and volume Jacobians + f64 residual/border/refinement" if j32 else
                     "f32 fronts + f64 residual/Jacobian/refinement"), "data": "synthetic",
           "config": {"workload": args.workload,
                      ("hexahedra" if three_d else ("triangles" if tri else "quads")): len(mesh["conn"]),
                      "dofs": info["n_dofs"],
                      "nnz": info["nnz"], "fronts": info["n_fronts"], "max_front": info["max_front"],
                      "factor_gflop": info["factor_flops"] / 1e9, **wl, "precision": "mixed",
                      "pivoting": args.pivoting, "jacobian": args.jacobian, "predictor": args.predictor,
                      "l2": f"inputs larger than L2 (front pool {4 * info['front_entries'] / 1e9:.1f} GB)",
                      "parallelism": "replicas" if world > 1 else "single"},
           "newton_iters_per_step": newton, "refine_sweeps_per_step": sweeps,
           "pivoting_record": {"threshold_misses": sum(i["threshold_misses"] for i in infos),
                               "perturbed_pivots": sum(i["perturbed_pivots"] for i in infos),
                               "note": "summed over the timed steps' factorisations; a miss is a multiplier "
                                       "above 1/u (u = 0.01), i.e. a pivot the threshold test would reject"},
           "kernels_ms": {k: round(v[0], 3) for k, v in kern.items()},
           "profiled": {"steps": args.steps, "ms_per_step": prof_ms / args.steps,
                        "note": "second pass with a CUDA event pair around every launch (kernels_ms, roofline)"},
           "roofline": roof, "rooflines_by_kind": rooflines, "gpu_launches": launches, "clocks": clk,
           "graphs": "residual, Jacobian, factorisation and refinement sweeps replayed as CUDA graphs"}
    out["schedule"] = {"block_lu_levels": [l for l in range(info["n_levels"]) if info["block_level_mask"] >> l & 1],
                       "set_by": "autotune" if args.autotune else ("flags" if args.big_front or args.block_levels
                                                                   is not None else "library defaults")}
    if args.autotune:
        out["autotune"] = {"big_front": tuned[0], "factor_ms": tuned[1],
                           "block_lu_levels": [l for l in range(info["n_levels"]) if info["block_level_mask"] >> l & 1]}

    if three_d:
        # the FP64 fronts of this case need ~245 GB; the threshold-pivoting path and the
        # 2-D serving sweep are measured on the 2-D workloads
        args.no_fp64 = args.no_threshold_path = args.no_sweep = True
    if tri:
        args.no_threshold_path = args.no_sweep = True   # (measured on the Q2 workloads)
    if not args.no_fp64 and rank == 0:
        c64 = viv.viv_case(M, wl["Re"], wl["Ustar"], wl["dt"], u0, precision=viv.VIV_FP64, pivoting=piv,
                           predictor=pred)
        for _ in range(max(2, args.warmup)):     # BDF1, then BDF2: both graph sets captured before timing
            c64.step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(c64.stream)
        i64 = [c64.step() for _ in range(args.fp64_steps)]
        e1.record(c64.stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        out["fp64_path"] = {"value": args.fp64_steps / (ms64 / 1e3), "unit": "time steps/s",
                            "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                            "warmup": max(2, args.warmup),
                            "newton_iters_per_step": sum(i["newton_iters"] for i in i64) / len(i64)}
        out["speedup_mixed_vs_fp64"] = value / world / out["fp64_path"]["value"]
        c64.close()

    if not args.no_threshold_path and args.pivoting == "window" and rank == 0:
        # the same mixed path with threshold pivoting over all fully summed rows
        ct = viv.viv_case(M, wl["Re"], wl["Ustar"], wl["dt"], u0, precision=viv.VIV_MIXED,
                          pivoting=viv.VIV_PIVOT_THRESHOLD, jacobian_fp32=j32, predictor=pred)
        for _ in range(max(2, args.warmup)):
            ct.step()
        torch.cuda.synchronize()
        nt = max(3, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ct.stream)
        it_ = [ct.step() for _ in range(nt)]
        e1.record(ct.stream)
        torch.cuda.synchronize()
        mst = e0.elapsed_time(e1)
        out["threshold_pivoting_path"] = {"value": nt / (mst / 1e3), "unit": "time steps/s", "ms_per_step": mst / nt,
                                          "steps": nt, "warmup": max(2, args.warmup),
                                          "newton_iters_per_step": sum(i["newton_iters"] for i in it_) / nt,
                                          "refine_sweeps_per_step": sum(i["refine_sweeps"] for i in it_) / nt,
                                          "threshold_misses": sum(i["threshold_misses"] for i in it_),
                                          "perturbed_pivots": sum(i["perturbed_pivots"] for i in it_)}
        ct.close()

    if not args.no_reuse_path and rank == 0:
        # the same mixed path, factoring only at each step's first Newton iterate (vivParams.factor_reuse)
        cr = viv.viv_case(M, wl["Re"], wl["Ustar"], wl["dt"], u0, precision=viv.VIV_MIXED, pivoting=piv,
                          jacobian_fp32=j32, predictor=pred, factor_reuse=1)   # (the mesh's tuned schedule)
        for _ in range(max(2, args.warmup)):
            cr.step()
        torch.cuda.synchronize()
        nr_ = max(3, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cr.stream)
        ir_ = [cr.step() for _ in range(nr_)]
        e1.record(cr.stream)
        torch.cuda.synchronize()
        msr = e0.elapsed_time(e1)
        out["factor_reuse_path"] = {"value": nr_ / (msr / 1e3), "unit": "time steps/s", "ms_per_step": msr / nr_,
                                    "steps": nr_, "warmup": max(2, args.warmup),
                                    "factorisations_per_step": sum(i["newton_iters"] for i in ir_) / nr_,
                                    "reused_factor_solves_per_step": sum(i["reused_factor_solves"] for i in ir_) / nr_,
                                    "refine_sweeps_per_step": sum(i["refine_sweeps"] for i in ir_) / nr_,
                                    "res_norm_max": max(i["res_norm"] for i in ir_),
                                    "note": "Newton iterates after a step's first assemble their Jacobian and solve "
                                            "with it by FP64 refinement preconditioned with the first iterate's "
                                            "factors (the paper factors at every iterate: the headline value does)"}
        cr.close()

    if not args.no_e2e:
        # end to end through viv_step_host: the packed state crosses the bus every step
        n_st = M.state_size()
        h_in = torch.empty(n_st, dtype=torch.float64, pin_memory=True)
        h_out = torch.empty(n_st, dtype=torch.float64, pin_memory=True)
        st = case.get_state()
        n = len(mesh["X"])
        packed = np.concatenate([st["u"].ravel(), st["p"], st["x"].ravel(), st["lam"].ravel(), st["delta"],
                                 st["u"].ravel(), st["x"].ravel(), [st["t"], 0.0]])
        h_in.numpy()[:] = packed
        case.step_host(h_in.numpy(), h_out.numpy())
        h_in.numpy()[:] = h_out.numpy()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            case.step_host(h_in.numpy(), h_out.numpy())
            h_in.numpy()[:] = h_out.numpy()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        barrier()
        out["e2e"] = {"value": world * args.steps / el, "unit": "time steps/s",
                      "h2d_bytes_per_step": 8 * n_st, "d2h_bytes_per_step": 8 * n_st}

    if rank == 0 and not args.no_sweep:
        out["sweep"] = run_sweep(viv, I, args.sweep_cases, args.sweep_steps, piv, j32, pred)

    if rank == 0 and not args.no_cpu_baseline:
        # the oracle starts Newton from U^n: 3 iterations per step on this case (the GPU path's
        # count with the same starting point)
        v, desc, secs = (oracle_sample3d if three_d else oracle_sample)(wl, 3.0)
        out["cpu_baseline"] = {"value": v, "unit": "time steps/s", "cores": 1, "kind": "oracle", "sample": desc,
                               "sample_seconds": round(secs, 1), "host": host_info()}
        if args.oracle_full_steps > 0 and not three_d and not tri:
            out["cpu_baseline"]["full_run_small_case"] = oracle_full_run(args.oracle_full_steps)
    if rank == 0:
        print(json.dumps(out), flush=True)
    case.close()
    M.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl, rank)
    else:
        run_ours(args, wl, rank, world, local)


if __name__ == "__main__":
    main()
