"""Benchmark of the ADG hot path on GB300: GDoF-RK-stages/s.

Workload (default): 2D isentropic vortex, periodic [-5,5]^2, 256^2 quads, degree 4
(5x5 Gauss points), 8x8 subdomains of 32x32 elements, communication-avoiding schedule with
L = 3 and the AT flux (N_p + 1 = 5 stored levels), CK4(5) low-storage RK, CFL 0.1, FP64.
One benchmark step is one full schedule cycle: L + N_p + 1 = 8 time steps (5 communication
steps, 3 delayed ones), i.e. 40 RK stages over 6,553,600 DoF.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--precision fp64|df64|fp32] [--no-cpu-baseline] [--no-variants]
                  [--no-batch] [--no-3d] [--no-learned]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an independent
replica on its own GPU ("replicas only": the path has no exchange between GPUs).
Besides the headline (value, e2e through the C ABI with pinned host buffers, roofline of
the volume kernel from live CUDA events, clocks sampled by nvidia-smi, the oracle's CPU
throughput, launch count) the line carries:
  variants         the same workload with the FP64, FP32-pair and FP32 operators, with
                   their L2 errors against the exact vortex;
  batched          64 uneven vortex instances in one CUDA graph per step vs separate handles;
  taylor_green_3d  the 3D Taylor-Green vortex (64^3, p = 3) in each operator arithmetic;
  learned_ghost    the learned ghost-trace predictor against plain AT on its 3D case.
`--impl reference` times the CPU oracle on the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF-RK-stages/s"
N_ELEM, DEGREE, P, L = 256, 4, 8, 3
CFL = 0.1


def workload_config(precision):
    return {"workload": f"2D isentropic vortex 256^2 quads p=4, 8x8 subdomains, CAA L=3, AT flux "
                        f"(5 levels), CK4(5), CFL 0.1, operator {precision}",
            "n_elem": [N_ELEM, N_ELEM], "degree": DEGREE, "subdomains": [P, P], "max_delay": L,
            "flux": "at", "rk": "ck45", "precision": precision,
            "time_steps_per_step": L + DEGREE + 1, "rk_stages": 5,
            "n_dof": 4 * N_ELEM * N_ELEM * (DEGREE + 1) ** 2,
            "l2_policy": "L2 flushed (256 MiB write) between timed steps",
            "parallelism": "replicas"}


# ---- algorithmic work per DoF and RK stage -------------------------------------------
def vol_flops_per_node(D=2, N=DEGREE + 1):
    """Flops of the volume/update kernel per node (FMA = 2): pointwise Euler flux,
    sum-factorised derivative along D directions, face lift, 2N RK update, next traces."""
    NV = D + 2
    pointwise = 1 + D + 2 * D + 3 + 1 + D * (D + 2)
    sweeps = 2 * D * N * NV
    lift = 4 * D * NV
    rk = 5 * NV
    traces = 4 * D * NV
    return pointwise + sweeps + lift + rk + traces


Q_BYTES = {"fp64": 8, "df64": 8, "fp32": 4}  # storage of the 2N register q per value


def vol_bytes_per_dof_stage(stage, stages=5, qbytes=8):
    """Algorithmic HBM bytes per DoF of one 2N stage: read and write the FP64 solution w,
    read q after the first stage, write q before the last stage (q in the operator's
    storage: FP64, FP32 pair or FP32)."""
    b = 16
    if stage > 0:
        b += qbytes
    if stage < stages - 1:
        b += qbytes
    return b


def kernel_source_hash(precision):
    """Hash of the sources the single-instance operator kernels of one arithmetic compile
    from (a profile taken on other sources no longer describes them)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_28710_gb300", "csrc")
    for name in ("adg_internal.h", "arith.cuh", "df64.cuh", "kernels.cuh", f"k_{precision}.cu"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(precision):
    """DRAM bytes per launch of the volume kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"vol_kernel_traffic_{precision}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != kernel_source_hash(precision):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


# ---- clocks sampled during the timed region -------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- oracle CPU baseline ---------------------------------------------------------------
def make_oracle():
    """The CPU oracle on the full-size workload with the CFL-0.1 time step."""
    import oracle
    o = oracle.Oracle(n_elem=(N_ELEM, N_ELEM), degree=DEGREE, P=(P, P), max_delay=L, flux="at",
                      rk="ck45", dt=1.0)
    u0 = o.init_vortex()
    dt = o.dt_from_cfl(u0, CFL, 0.0)
    o = oracle.Oracle(n_elem=(N_ELEM, N_ELEM), degree=DEGREE, P=(P, P), max_delay=L, flux="at",
                      rk="ck45", dt=dt)
    o.set_state(u0)
    return o


def oracle_sample(time_steps):
    """Times the CPU oracle on the full-size workload for a few time steps; returns
    (GDoF-RK-stages/s, seconds)."""
    o = make_oracle()
    t0 = time.perf_counter()
    o.step(time_steps)
    sec = time.perf_counter() - t0
    ndof = 4 * N_ELEM * N_ELEM * (DEGREE + 1) ** 2
    return ndof * 5 * time_steps / sec / 1e9, sec


def run_reference(args, rank, world):
    """The oracle as the reference arm, single-threaded on the host cores (rank 0 only).
    Each step is a bounded sample of the workload: one RK time step (5 stages), or one
    stage (one operator evaluation) when K time steps would take more than about two
    minutes."""
    if rank != 0:
        return
    o = make_oracle()
    o.step(args.warmup)
    ndof = 4 * N_ELEM * N_ELEM * (DEGREE + 1) ** 2
    t0 = time.perf_counter()
    o.step(1)
    t_step = time.perf_counter() - t0
    per_stage = args.steps * t_step > 120.0
    total, stages = (0.0, 0) if per_stage else (t_step, 5)
    u = o.get_state() if per_stage else None
    for _ in range(args.steps if per_stage else args.steps - 1):
        t0 = time.perf_counter()
        if per_stage:
            o.rhs(u)
            stages += 1
        else:
            o.step(1)
            stages += 5
        total += time.perf_counter() - t0
    value = ndof * stages / total / 1e9
    sample = ("one RK stage (operator evaluation)" if per_stage else "one RK time step (5 stages)")
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config("fp64"),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{sample} of the full 256^2 p=4 workload per step, "
                                       "single-threaded C oracle"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- multi-rank aggregation ---------------------------------------------------------------
def reduce_max(x, device=None):
    """Maximum of a float over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(work_per_rank_per_step, steps, seconds_max, world):
    """Whole-job throughput in G-units/s: every rank's work over the slowest rank's time."""
    return world * work_per_rank_per_step * steps / seconds_max / 1e9


def variant_run(adg, stream, precision, steps_per, k, warm, dt):
    """Throughput and L2 error vs the exact vortex of one operator arithmetic on the bench
    workload (fixed dt, same initial state)."""
    import torch
    s = adg.Solver(n_elem=(N_ELEM, N_ELEM), degree=DEGREE, P=(P, P), max_delay=L, flux="at",
                   rk="ck45", dt=dt, precision=precision, stream=stream.cuda_stream)
    s.init_vortex()
    s.step(steps_per * warm)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps_per * k)          # unprofiled: the throughput
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.set_profiling(True)          # second pass: per-kernel times
    s.step(steps_per * 2)
    prof = s.get_profile()
    s.set_profiling(False)
    ndof = 4 * N_ELEM * N_ELEM * (DEGREE + 1) ** 2
    info = s.info()
    err = s.l2_error_vortex(info["t"])  # after warm + k + 2 benchmark steps
    s.close()
    return {"value": ndof * 5 * steps_per * k / (ms * 1e-3) / 1e9, "l2_flush": False,
            "vol_ms_per_launch": prof["vol"][0] / max(prof["vol"][1], 1),
            "flux_ms_per_launch": prof["flux"][0] / max(prof["flux"][1], 1),
            "l2_error_vs_exact": [float(x) for x in err], "t": info["t"]}


def batched_run(adg, stream, k=6):
    """64 uneven vortex instances (meshes 32^2..256^2, degrees 2..5, L in {2,3,4}, 8x8
    subdomains, AT flux, CK4(5), FP32 operator with FP64 accumulation): batched graph steps
    against the same instances stepped one handle after another."""
    import torch
    from paper_2603_28710_gb300.inputs import vortex_instances
    specs = vortex_instances(64, seed=7)
    insts = [dict(n_elem=(q["n"], q["n"]), degree=q["degree"], P=(8, 8), max_delay=q["max_delay"])
             for q in specs]
    work = sum(4 * q["n"] ** 2 * (q["degree"] + 1) ** 2 for q in specs) * 5  # DoF-stages per step
    b = adg.Batch(insts, flux="at", rk="ck45", cfl=0.1, precision="fp32", stream=stream.cuda_stream)
    t0 = time.perf_counter()
    tiles = b.autotune(trials=3)
    tune_s = time.perf_counter() - t0
    for i, q in enumerate(specs):
        b.init_vortex(i, beta=q["beta"], x0=q["x0"], y0=q["y0"])
    b.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    b.close()
    singles = []
    for q in specs:
        s = adg.Solver(n_elem=(q["n"], q["n"]), degree=q["degree"], P=(8, 8), max_delay=q["max_delay"],
                       flux="at", rk="ck45", cfl=0.1, precision="fp32", stream=stream.cuda_stream)
        s.init_vortex(beta=q["beta"], x0=q["x0"], y0=q["y0"])
        s.step(2)
        singles.append(s)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        for s in singles:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for s in singles:
        s.close()
    return {"workload": "64 vortex instances, meshes 32^2..256^2, p 2..5, L 2..4, 8x8 subdomains, "
                        "AT flux, CK4(5), FP32 operator / FP64 accumulation, one CUDA graph per step",
            "value": work * k / (ms_batch * 1e-3) / 1e9, "unit": METRIC, "steps": k,
            "ms_per_step": ms_batch / k, "sequential_handles_value": work * k / (ms_seq * 1e-3) / 1e9,
            "speedup_vs_sequential": ms_seq / ms_batch, "tile_threads_per_degree_group": tiles,
            "autotune_s": tune_s}


def tgv_run(adg, stream, k=3, total_steps=100):
    """3D Taylor-Green vortex, 64^3 hexes, p = 3, 8x8x8 subdomains, L = 4, AT flux,
    CK4(5), CFL 0.1: throughput per operator arithmetic (one benchmark step = one schedule
    cycle of L + N_p + 1 = 8 time steps), and after total_steps RK steps from the initial
    condition each form's relative L2 difference from the FP64 form and its drift of the
    conserved totals (mass, momentum, energy; max over variables, relative)."""
    import torch
    out = {}
    ndof = 5 * 64 ** 3 * 4 ** 3
    u64 = None
    for prec in ("fp64", "df64", "fp32"):
        s = adg.Solver(dim=3, n_elem=(64, 64, 64), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3,
                       P=(8, 8, 8), max_delay=4, flux="at", rk="ck45", cfl=0.1, precision=prec,
                       stream=stream.cuda_stream)
        s.init_tgv(0.1)
        c0 = s.conservation()
        s.step(8)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(8 * k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s.set_profiling(True)
        s.step(8)
        prof = s.get_profile()
        s.set_profiling(False)
        s.step(total_steps - 8 * (k + 2))
        u = s.get_state()
        c1 = s.conservation()
        s.close()
        out[prec] = {"value": ndof * 5 * 8 * k / (ms * 1e-3) / 1e9,
                     "vol_ms_per_launch": prof["vol"][0] / max(prof["vol"][1], 1),
                     "flux_ms_per_launch": prof["flux"][0] / max(prof["flux"][1], 1),
                     f"conservation_drift_after_{total_steps}_steps":
                         float(np.max(np.abs(c1 - c0)) / np.max(np.abs(c0)))}
        if prec == "fp64":
            u64 = u
        else:
            out[prec][f"rel_l2_diff_vs_fp64_after_{total_steps}_steps"] = float(
                np.linalg.norm(u - u64) / np.linalg.norm(u64))
        del u
    out["workload"] = ("3D Taylor-Green vortex 64^3 hexes p=3 (83.9M DoF), 8x8x8 subdomains, "
                       "CAA L=4, AT flux, CK4(5), CFL 0.1")
    out["unit"] = METRIC
    return out


def learned_run(adg, stream, k=2, err_steps=24):
    """Learned ghost-trace predictor on its evaluation case (3D Taylor-Green vortex, 64^3
    hexes, p = 3, 8x8x8 subdomains, L = 4, N_p = 2, CK4(5), CFL 0.1, FP64 operator) against
    the plain AT extrapolation of the same stored traces: throughput (one benchmark step =
    8 time steps) and the relative delay error after err_steps time steps against the
    synchronous run (|w - w_sync| / |w_sync - w_0|)."""
    import torch
    from paper_2603_28710_gb300 import learned
    if not os.path.exists(learned.MODEL_PATH):
        return None
    model, _ = learned.load()
    kw = dict(dim=3, n_elem=(64, 64, 64), degree=3, lo=(0, 0, 0), hi=(2 * np.pi,) * 3,
              P=(8, 8, 8), rk="ck45", cfl=0.1, precision="fp64", stream=stream.cuda_stream)
    ndof = 5 * 64 ** 3 * 4 ** 3
    ref = adg.Solver(flux="sync", **kw)
    ref.init_tgv(0.1)
    u0 = ref.get_state()
    ref.step(err_steps)
    u_sync = ref.get_state()
    ref.close()
    out = {}
    for name, flux, trust in (("at_trace", "at_trace", None), ("learned", "learned", 1.0)):
        s = adg.Solver(flux=flux, max_delay=4, at_np=2, **kw)
        if trust is not None:
            s.set_learned_model(model, trust)
        s.init_tgv(0.1)
        s.step(err_steps)
        err = float(np.linalg.norm(s.get_state() - u_sync) / np.linalg.norm(u_sync - u0))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(8 * k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        out[name] = {"value": ndof * 5 * 8 * k / (ms * 1e-3) / 1e9,
                     "delay_error_vs_sync": err}
    out["learned"]["trust"] = 1.0
    out["speedup_vs_fp64_at"] = out["learned"]["value"] / out["at_trace"]["value"]
    out["delay_error_ratio_vs_at"] = (out["learned"]["delay_error_vs_sync"]
                                      / out["at_trace"]["delay_error_vs_sync"])
    out["workload"] = ("3D Taylor-Green vortex 64^3 hexes p=3, 8x8x8 subdomains, CAA L=4, "
                       "N_p=2, CK4(5), CFL 0.1, FP64 operator; delay error after "
                       f"{err_steps} steps against the synchronous run")
    out["unit"] = METRIC
    return out


# ---- GPU arm -----------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2603_28710_gb300 import adg, build

    if rank == 0 or not os.path.exists(adg.LIB_PATH):
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    steps_per = L + DEGREE + 1
    ndof = 4 * N_ELEM * N_ELEM * (DEGREE + 1) ** 2
    work = ndof * 5 * steps_per  # DoF-stages per benchmark step

    s = adg.Solver(n_elem=(N_ELEM, N_ELEM), degree=DEGREE, P=(P, P), max_delay=L, flux="at",
                   rk="ck45", cfl=CFL, precision=args.precision, stream=stream.cuda_stream)
    s.init_vortex()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        s.step(steps_per)
    torch.cuda.synchronize()

    # device-timed region: K steps, L2 flushed between them (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    gpu_idx = os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank] \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local_rank)
    barrier()
    torch.cuda.synchronize()
    s.set_profiling(True)
    with ClockSampler(gpu_idx) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            s.step(steps_per)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    prof = s.get_profile()
    s.set_profiling(False)
    ms_list = [a.elapsed_time(b) for a, b in ev]
    ms = reduce_max(sum(ms_list), dev)
    value = whole_job_value(work, args.steps, ms * 1e-3, world)

    # end to end through the public API: pinned host state in, 8 steps, state out
    host_in = torch.from_numpy(s.get_state()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dt = s.info()["dt"]
    s2 = adg.Solver(n_elem=(N_ELEM, N_ELEM), degree=DEGREE, P=(P, P), max_delay=L, flux="at",
                    rk="ck45", dt=dt, precision=args.precision, stream=stream.cuda_stream)
    for _ in range(2):
        s2.set_state(host_in)
        s2.step(steps_per)
        s2.get_state(host_out)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        s2.set_state(host_in)
        s2.step(steps_per)
        s2.get_state(host_out)
    torch.cuda.synchronize()
    e2e_sec = reduce_max(time.perf_counter() - t0, dev)
    e2e_value = whole_job_value(work, args.steps, e2e_sec, world)
    state_bytes = ndof * 8

    if rank != 0:
        return

    # roofline of the dominant kernel (volume/update kernel), timed live above
    vol_ms, vol_n = prof["vol"]
    flux_ms, flux_n = prof["flux"]
    vol_avg_s = vol_ms * 1e-3 / max(vol_n, 1)
    nodes = N_ELEM * N_ELEM * (DEGREE + 1) ** 2
    flops_launch = vol_flops_per_node() * nodes
    bytes_launch = np.mean([vol_bytes_per_dof_stage(m, 5, Q_BYTES[args.precision])
                            for m in range(5)]) * ndof
    pk = peaks()
    fp64_peak_tflops = 1.25  # nominal GB300 FP64 rate (no FP64 tensor advantage)
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": flops_launch / vol_avg_s / 1e12,
                "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table); 1.19 measured by an FMA probe"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_launch / vol_avg_s / 1e9,
                "peak": pk.get("hbm_gbs", 6800.0), "unit": "GB/s",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in pk else "fallback 6.8 TB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = "vol_kernel<2,5>"
    roof["traffic"] = ncu_traffic(args.precision)
    roof["algorithmic_bytes_per_launch"] = bytes_launch
    roof["algorithmic_flops_per_launch"] = flops_launch
    roof["hbm_view"] = {"achieved_gbs": bytes_launch / vol_avg_s / 1e9,
                        "peak_gbs": pk.get("hbm_gbs", 6800.0),
                        "frac": bytes_launch / vol_avg_s / 1e9 / pk.get("hbm_gbs", 6800.0)}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, sec = oracle_sample(args.cpu_steps)
        cpu = {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_steps} RK time steps (5 stages each) of the full 256^2 p=4 "
                         f"workload, single-threaded C oracle, {sec:.1f} s"}

    variants = None
    if world == 1 and not args.no_variants:
        variants = {}
        for prec in ("fp64", "df64", "fp32"):
            variants[prec] = variant_run(adg, stream, prec, steps_per, args.variant_steps, 2, dt)
        base = variants["fp64"]
        for prec, v in variants.items():
            v["speedup_vs_fp64"] = v["value"] / base["value"]
            v["l2_error_ratio_vs_fp64"] = [a / b for a, b in zip(v["l2_error_vs_exact"],
                                                                 base["l2_error_vs_exact"])]
        # the fastest operator form whose L2 errors match the plain FP64 form's (within
        # 0.1 % in density, momentum and energy)
        matched = [(v["value"], prec) for prec, v in variants.items()
                   if all(abs(r - 1.0) < 1e-3 for r in v["l2_error_ratio_vs_fp64"])]
        best_value, best_prec = max(matched)
        variants["matched_error_best"] = {
            "form": best_prec, "value": best_value, "unit": METRIC,
            "speedup_vs_fp64": variants[best_prec]["speedup_vs_fp64"],
            "l2_error_ratio_vs_fp64": variants[best_prec]["l2_error_ratio_vs_fp64"]}

    batched = None
    if world == 1 and not args.no_batch:
        batched = batched_run(adg, stream)
    tgv = None
    if world == 1 and not args.no_3d:
        tgv = tgv_run(adg, stream)
    learned_line = None
    if world == 1 and not args.no_learned:
        learned_line = learned_run(adg, stream)

    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "df64": "f32x2"}[args.precision],
            "data": "synthetic", "config": workload_config(args.precision),
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes},
            "roofline": roof, "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": int(vol_n + flux_n),
            "kernels": {"vol_kernel": {"ms_per_launch": vol_ms / max(vol_n, 1), "launches": vol_n},
                        "flux_kernel": {"ms_per_launch": flux_ms / max(flux_n, 1),
                                        "launches": flux_n}},
            "variants": variants, "batched": batched, "taylor_green_3d": tgv,
            "learned_ghost": learned_line}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df64"])
    ap.add_argument("--cpu-steps", type=int, default=4)  # about 12 s of oracle work
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP64 / FP32-pair / FP32 comparison runs")
    ap.add_argument("--variant-steps", type=int, default=10)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances run")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D Taylor-Green runs")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned ghost-trace predictor run")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
