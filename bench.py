"""Benchmark of the fused GB300 path on the headline workload.

Workload ("2D 1024^2, M = 16"): periodic [-pi,pi)^2 on 1024 x 1024 points,
Q(x, y) = seeded low-passed noise mapped to [5, 100], c0 = 1, omega0 = 2 pi,
Ricker source (f0 = 10) at the centre, u0 = u_t = 0, dt = 5e-4, 1000
leap-frog steps of Eq. (1.1) with both operators by Eq. (2.13), M = 16.

One bench "step" = one complete run of that workload (model precompute from
Q, state and source set-up, start step + 999 leap-frog steps).  The metric
is Mpoint-steps/s = 1024^2 * 1000 * runs / time.

  value  device-resident inputs (Q, u0, source samples already in HBM);
  e2e    the same run through the C ABI with host buffers: the H2D copies of
         Q, u0 and the samples and the D2H copy of the final wavefield are
         inside the timed region;
  plain  the cuFFT + elementwise baseline on the same run;
  batch  64 independent 2D simulations of uneven sizes {256, 512, 768,
         1024}^2 (M = 12, 300 steps each, dt a quarter of the leap-frog bound
         of each model) advanced together by one batch (vofl_batch_*), the
         transform schedule of each size and the launch layout autotuned
         (vofl_batch_tune_transform), timed over the whole 300-step run;
  configs  the 1D 256 FP64 (M = 8, 200 steps) and 3D 256^3 FP32 (M = 8,
         500 steps) runs, fused and plain; the general model of the
         paper's Tables 3 (leap-frog) and 2 (Crank-Nicolson) on the FP64
         path (timed reference runs, errors beside the printed ones) and
         the generic 2D operator apply;
  serve  continuous batching of a Poisson request stream (mean 200 per
         second, seed 5; 1D 4096 / 2D 512^2 / 2D 1024^2 / 3D 128^3 with equal
         probability, 100..2000 steps, M 8..16) served in real time:
         p50/p99 latency from arrival to the answer on the host, and
         point-steps/s; a bounded prefix of the 600-request stream by
         default (--serve-requests), with a few answers re-run alone and
         compared bit for bit.

L2 is flushed (256 MiB write) before every timed run.  Times are CUDA events
on the context stream.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead (the reference arm).
"""
from __future__ import annotations

import argparse
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

NX = NY = 1024
NSTEPS = 1000
M = 16
DT = 5e-4
# DRAM bytes (read + write) per launch of the dominant kernel come from an
# ncu capture summarised in a text file under profiles/, which also records
# a digest of the kernel sources it was taken on; a kernel changed since then
# reports traffic null (see _ncu_traffic).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic_2d_1024_M16.txt")
KERNEL_SOURCES = ["paper_2311_13049_gb300/csrc/kernels.cuh", "paper_2311_13049_gb300/csrc/fft_warp.cuh",
                  "paper_2311_13049_gb300/csrc/kernels_wide.cuh", "paper_2311_13049_gb300/csrc/fft_wide.cuh",
                  "paper_2311_13049_gb300/csrc/tma.cuh", "paper_2311_13049_gb300/csrc/internal.h"]
METRIC = "Mpoint-steps/s (2D 1024², M=16) fused vs plain at ≤1e-5 rel L2; serve p50/p99"
UNIT = "Mpoint-steps/s"
WORKLOAD = "2D periodic 1024x1024, FP32, M=16, Q low-passed noise in [5,100] (seed 2), Ricker f0=10 at centre, dt=5e-4, 1000 steps"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(ms, dist=None, device="cuda"):
    """The slowest rank's time: every rank's timed region ends when the
    last one does (the job's wall time)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, points_per_run, runs, ms_max):
    """Whole-job throughput in Mpoint-steps/s: every rank runs its own
    replica of the workload, so the job does world_size times the work in
    the slowest rank's time."""
    return world_size * points_per_run * runs / (ms_max * 1e-3) / 1e6


def _config(extra=None):
    c = {"workload": WORKLOAD, "grid": [NY, NX], "M": M, "steps_per_run": NSTEPS, "dt": DT,
         "parallelism": "replicas (one independent run per GPU)",
         "l2": "flushed between timed runs (256 MiB write)", "step_unit": "one full 1000-step run"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.p = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.p.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_sources_digest():
    """sha256 over the sources of the fused 2D kernels (file name + bytes)."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(rel.encode())
            h.update(f.read())
    return h.hexdigest()


def _ncu_traffic(kernel):
    """(bytes per launch, note) of `kernel` from the traffic summary, or
    (None, why) when there is none or the kernel sources changed since the
    capture.  File lines: 'key: value'."""
    try:
        with open(TRAFFIC_FILE) as f:
            kv = dict(ln.split(":", 1) for ln in f if ":" in ln and not ln.startswith((" ", "#")))
    except OSError:
        return None, "no ncu traffic summary"
    kv = {k.strip(): v.strip() for k, v in kv.items()}
    if kv.get("kernel") != kernel:
        return None, f"the ncu traffic summary covers {kv.get('kernel')}, not {kernel}"
    if kv.get("sources_sha256") != kernel_sources_digest():
        return None, "kernel sources changed since the ncu capture"
    return float(kv["dram_bytes_per_launch"]), "ncu capture of the same kernel sources"


def _sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle, as it stands
# ---------------------------------------------------------------------------
def _oracle_sample(w, gamma, nsteps):
    import oracle as O
    t0 = time.perf_counter()
    O.seismic_lffp(gamma, w["c0"], w["omega0"], w["u0"], None, w["dt"], nsteps, w["M"],
                   src_idx=w["src_idx"], src=w["src"])
    return time.perf_counter() - t0


def _oracle_worker(nsteps):
    """One independent copy of the bounded oracle sample (a spawned process:
    no CUDA in it); returns its wall time."""
    import oracle as O
    import synthetic as S
    w = S.workload_2d_1024(nsteps=NSTEPS)
    gamma = O.seismic_coefficients(w["Q"], w["c0"], w["omega0"])["gamma"]
    _oracle_sample(w, gamma, 1)  # warm the multiplier-table cache
    return _oracle_sample(w, gamma, nsteps)


def cpu_baseline(nsteps=10, par_steps=4):
    """The FP64 oracle as it stands on the host cores.  One simulation runs
    on one core (NumPy's FFT is single-threaded), so the all-core figure is
    the aggregate of os.cpu_count() independent copies of the same bounded
    sample, run as spawned processes at the same time."""
    import multiprocessing as mp
    import oracle as O
    import synthetic as S
    w = S.workload_2d_1024(nsteps=NSTEPS)
    gamma = O.seismic_coefficients(w["Q"], w["c0"], w["omega0"])["gamma"]
    _oracle_sample(w, gamma, 1)  # warm the multiplier-table cache
    t1 = _oracle_sample(w, gamma, nsteps)
    one = {"value": NX * NY * nsteps / t1 / 1e6, "unit": UNIT, "cores": 1,
           "sample": f"{nsteps} leap-frog steps of the 1024^2 M=16 workload (FP64 NumPy, pocketfft, 1 thread), "
                     f"{t1:.1f} s"}
    ncores = os.cpu_count() or 1
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            t0 = time.perf_counter()
            times = pool.map(_oracle_worker, [par_steps] * ncores)
            wall = time.perf_counter() - t0
        # aggregate over the stepping phases (each copy's set-up is outside its timed sample)
        agg = NX * NY * par_steps * ncores / max(times) / 1e6
    except Exception as e:  # noqa: BLE001 - report, do not fail the bench
        return dict(one, kind="oracle", box_cores=ncores, all_cores_error=str(e)[:200])
    return {"value": agg, "unit": UNIT, "cores": ncores, "kind": "oracle", "box_cores": ncores,
            "sample": f"{ncores} independent copies (spawned processes, one per host core) of {par_steps} leap-frog "
                      f"steps of the 1024^2 M=16 workload each (FP64 NumPy, pocketfft); aggregate point-steps over the "
                      f"slowest copy's stepping time {max(times):.1f} s (wall {wall:.1f} s with set-up)",
            "single_thread": one}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    import oracle as O
    import synthetic as S
    w = S.workload_2d_1024(nsteps=NSTEPS)
    gamma = O.seismic_coefficients(w["Q"], w["c0"], w["omega0"])["gamma"]
    per = 2  # oracle leap-frog steps per bench step (bounded sample)
    for _ in range(args.warmup):
        _oracle_sample(w, gamma, 1)
    times = [_oracle_sample(w, gamma, per) for _ in range(args.steps)]
    tot = sum(times)
    value = NX * NY * per * args.steps / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": _config({"reference": "FP64 NumPy oracle (oracle/), each bench step = "
                                             f"{per} leap-frog steps of the workload on the host"}),
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": UNIT,
                             "sample": f"{per} oracle leap-frog steps per bench step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# batched workload: 64 uneven 2D simulations
# ---------------------------------------------------------------------------
def batch_bench(V, torch, stream, flush):
    import synthetic as S
    sims = S.workload_batch()
    nsteps = sims[0]["nsteps"]
    solvers = []
    t_setup = time.perf_counter()
    b = V.Batch(stream=stream.cuda_stream)
    pts = 0
    for sp in sims:
        s = V.Solver(sp["shape"], stream=stream.cuda_stream)
        s.set_q(sp["Q"], sp["c0"], sp["omega0"])
        s.set_M(sp["M"])
        dt = s.suggest_dt(0.25)
        s.set_state(np.zeros(sp["shape"], np.float32))
        s.set_source(sp["src_idx"], S.ricker_samples(nsteps, dt, sp["f0"]))
        b.add(s, dt)
        solvers.append(s)
        pts += sp["shape"][0] * sp["shape"][1]
    t_setup = time.perf_counter() - t_setup
    ms_default = b.time(reps=2)
    sizes = sorted({sp["shape"][0] for sp in sims})
    b.set_schedule(False, {n: 1 for n in sizes})
    ms_serial = b.time(reps=2)
    b.set_schedule(True, {})
    ms_layout = b.tune(reps=2)  # launch layout only (bit-preserving)
    ms_tuned = b.tune_transform(reps=2)  # transform schedule per size, then the layout
    par, chunks = b.schedule()
    transforms = {str(n): b.transform(n) for n in sorted({sp["shape"][0] for sp in sims})}
    kps = b.kernels_per_step()
    with torch.cuda.stream(stream):
        flush.zero_()
        stream.synchronize()
        l0 = V.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(nsteps)
        e1.record(stream)
        e1.synchronize()
        launches = V.kernel_launches() - l0
    b.sync()
    ms = e0.elapsed_time(e1)
    b.close()
    for s in solvers:
        s.close()
    counts = {}
    for sp in sims:
        counts[sp["shape"][0]] = counts.get(sp["shape"][0], 0) + 1
    return {"value": pts * nsteps / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_run": ms,
            "workload": f"64 independent 2D runs, edges drawn from {sizes} (seed 4): "
                        + ", ".join(f"{counts[n]}x{n}^2" for n in sizes)
                        + f"; M=12, {nsteps} steps each, dt = 0.25 * 2/omega_max per model",
            "points": pts, "steps": nsteps, "kernels_per_step": kps, "gpu_launches": launches,
            "ms_per_batch_step": {"tuned": ms_tuned, "default_all_per_launch": ms_default,
                                  "layout_tuned_default_transforms": ms_layout,
                                  "one_sim_per_launch_serial": ms_serial,
                                  "tuned_over_default": ms_default / ms_tuned},
            "schedule": {"parallel_branches": par, "sims_per_launch": {str(k): v for k, v in chunks.items()},
                         "transforms": transforms},
            "setup_s": t_setup}


# ---------------------------------------------------------------------------
# the other two single-run workloads: 1D 256 FP64 and 3D 256^3 FP32
# ---------------------------------------------------------------------------
def configs_bench(V, torch, stream, flush, reps=3):
    import synthetic as S

    def run(w, prec, impl):
        ty = torch.float32 if prec == V.F32 else torch.float64
        Q = torch.from_numpy(w["Q"]).cuda()
        u0 = torch.from_numpy(w["u0"]).to(ty).cuda()
        s = V.Solver(w["shape"], prec=prec, impl=impl, stream=stream.cuda_stream)
        s.set_M(w["M"])
        times = []
        with torch.cuda.stream(stream):
            for i in range(reps + 1):  # the first run warms up (tables, graphs)
                flush.zero_()
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.set_q(Q, w["c0"], w["omega0"])
                s.set_state(u0)
                s.step(w["nsteps"], w["dt"])
                e1.record(stream)
                e1.synchronize()
                if i:
                    times.append(e0.elapsed_time(e1))
        s.close()
        ms = statistics.median(times)
        pts = int(np.prod(w["shape"])) * w["nsteps"]
        return {"value": pts / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_run": ms}

    out = {}
    w1 = S.workload_1d_256()
    f, p = run(w1, V.F64, V.IMPL_FUSED), run(w1, V.F64, V.IMPL_PLAIN)
    out["1d_256_f64"] = {"workload": "1D 256, FP64, M=8, Q = 20 + 15 sin x, u0 = exp(-20 x^2), dt = 1e-3, "
                                     "200 steps (one run incl. model set-up)",
                         "fused": f, "plain": p, "fused_over_plain": f["value"] / p["value"]}
    out["general_table3_s1_1d_4096_f64"] = table3_bench(V, S, stream)
    out["cnfp_table2_s1_1d_4096_f64"] = cnfp_bench(V, S, stream)
    out["generic_apply_2d_512_M20_f32"] = generic_apply_bench(V, S, torch, stream)
    out["tsfp2_2d_1024_M16_f32"] = tsfp2_2d_bench(V, S, torch, stream)
    out["small_grids_2d_f32"] = small_grids_bench(V, S, torch, stream)
    w3 = S.workload_3d_256()
    f, p = run(w3, V.F32, V.IMPL_FUSED), run(w3, V.F32, V.IMPL_PLAIN)
    out["3d_256_f32"] = {"workload": "3D 256^3, FP32, M=8, two-layer Q (10/80), Gaussian pulse sigma = 4 cells, "
                                     "dt = 2e-3, 500 steps (one run incl. model set-up)",
                         "fused": f, "plain": p, "fused_over_plain": f["value"] / p["value"]}
    return out


# Table 3 of the paper (Sec. 3.2), column s1(x) = 1 + 0.3 sin(pi x/8):
# printed LFFP temporal errors at t = 1 for dt = 2^-p
TABLE3_S1 = {9: 3.531e-7, 10: 8.758e-8, 11: 2.120e-8}


def table3_bench(V, S, stream):
    """The general model of the paper's Table 3 (Eq. (4.1): [-32, 32],
    h = 1/64, M = 15, f(u) = u^3, u0 = exp(-x^2)) on the GPU's FP64 path:
    the dt = 1e-4 reference run to t = 1 is timed; the errors of the
    dt = 2^-p runs against it are reported beside the printed ones."""
    import torch
    J = 4096
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s1 = 1.0 + 0.3 * np.sin(np.pi * x / 8)

    def run(dt, n, timed=False):
        with V.Solver((J,), [-32.0], [32.0], V.F64, V.IMPL_PLAIN, stream=stream.cuda_stream) as sv:
            sv.set_order(s1, kappa=1.0, f3=1.0)
            sv.set_M(15)
            sv.set_state(phi)
            ms = None
            with torch.cuda.stream(stream):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sv.step(n, dt)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
            u = sv.get_state()
            sv.sync()
        return u, ms

    run(2.0 ** -9, 16)  # warm-up (plans, graphs)
    ref, ms = run(1e-4, 10000, timed=True)
    errs = {}
    for p, printed in TABLE3_S1.items():
        u, _ = run(2.0 ** -p, 2 ** p)
        errs[str(p)] = {"gpu": float(np.sqrt((1.0 / 64) * np.sum((u - ref) ** 2))), "printed": printed}
    return {"workload": "1D 4096 on [-32,32], FP64 plain path, M=15, s1 = 1 + 0.3 sin(pi x/8), f = u^3, "
                        "reference run dt = 1e-4 to t = 1 (10000 steps, timed)",
            "value": J * 10000 / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_run": ms, "l2_error_vs_reference": errs}


# Table 2 of the paper (Sec. 3.1), column s1(x): printed CNFP temporal
# errors at t = 1 for dt = 2^-p (their reference is the dt = 2^-12 run)
TABLE2_S1 = {9: 1.739e-6, 10: 4.143e-7, 11: 8.281e-8}


def cnfp_bench(V, S, stream):
    """The Crank-Nicolson scheme (Sec. 3.1) on the problem of Table 2 (as in
    Table 3, FP64 plain path, CG on the normal equations to the default
    relative residual 1e-15): the dt = 2^-12 reference run to t = 1 is
    timed; the errors of the dt = 2^-p runs against it are reported beside
    the printed ones, with the solver's iteration counts."""
    import torch
    J = 4096
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s1 = 1.0 + 0.3 * np.sin(np.pi * x / 8)

    def run(dt, n):
        with V.Solver((J,), [-32.0], [32.0], V.F64, V.IMPL_PLAIN, stream=stream.cuda_stream) as sv:
            sv.set_order(s1, kappa=1.0, f3=1.0)
            sv.set_M(15)
            sv.set_scheme(V.SCHEME_CNFP)
            sv.set_state(phi)
            with torch.cuda.stream(stream):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sv.step(n, dt)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
            u = sv.get_state()
            sv.sync()
            return u, ms, sv.solver_stats()

    run(2.0 ** -9, 16)  # warm-up (plans, graphs)
    ref, ms, (iters, solves) = run(2.0 ** -12, 4096)
    errs = {}
    for p, printed in TABLE2_S1.items():
        u, ms_p, (it_p, so_p) = run(2.0 ** -p, 2 ** p)
        errs[str(p)] = {"gpu": float(np.sqrt((1.0 / 64) * np.sum((u - ref) ** 2))), "printed": printed,
                        "cg_iterations": it_p, "ms_run": ms_p}
    return {"workload": "1D 4096 on [-32,32], FP64 plain path, CNFP (CG on the normal equations, rel. residual "
                        "1e-15), M=15, s1 = 1 + 0.3 sin(pi x/8), f = u^3, reference run dt = 2^-12 to t = 1 "
                        "(4096 steps, timed)",
            "value": J * 4096 / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_run": ms, "cg_iterations": iters,
            "linear_solves": solves, "l2_error_vs_reference": errs}


def generic_apply_bench(V, S, torch, stream, reps=20):
    """(-Delta)^{s(x)} u at 512^2 on [-8,8]^2, s = 1 - 0.4 cos(pi x/4)
    cos(pi y/4), M = 20 (the shape of the paper's 2D example): one apply,
    fused FP32 and plain FP32, CUDA events over `reps` applies."""
    shape, lo, hi = (512, 512), [-8.0, -8.0], [8.0, 8.0]
    xg, yg = S.mesh(shape, lo, hi)
    so = 1.0 - 0.4 * np.cos(np.pi * xg / 4) * np.cos(np.pi * yg / 4)
    u = torch.from_numpy(S.random_field(shape, 3).astype(np.float32)).cuda()
    res = {}
    for nm, im in (("fused", V.IMPL_FUSED), ("plain", V.IMPL_PLAIN)):
        with V.Solver(shape, lo, hi, V.F32, im, stream=stream.cuda_stream) as sv:
            sv.set_order(so)
            sv.set_M(20)
            out = torch.empty_like(u)
            with torch.cuda.stream(stream):
                sv.apply(V.OP_S, u, out)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    sv.apply(V.OP_S, u, out)
                e1.record(stream)
                e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
        res[nm] = {"ms_per_apply": ms, "value": 512 * 512 / (ms * 1e-3) / 1e6, "unit": "Mpoint/s"}
    res["fused_over_plain"] = res["plain"]["ms_per_apply"] / res["fused"]["ms_per_apply"]
    return res


def tsfp2_2d_bench(V, S, torch, stream, nsteps=100):
    """The time splitting (Sec. 3.3) of the general model in 2D: 1024^2 on
    [-8,8]^2, s = 1 - 0.4 cos(pi x/4) cos(pi y/4), kappa = 1, f(u) = u^3,
    M = 16, dt = 0.25 x the explicit limit 2 / omega_max (vofl_suggest_dt;
    the kick is explicit), u0 a Gaussian (sigma = 1), v0 = 0; fused FP32 and
    plain FP32 (cuFFT), CUDA events over `nsteps` steps after a warm-up run;
    accuracy of both against the plain FP64 run (vofl_rel_l2)."""
    shape, lo, hi = (1024, 1024), [-8.0, -8.0], [8.0, 8.0]
    xg, yg = S.mesh(shape, lo, hi)
    so = 1.0 - 0.4 * np.cos(np.pi * xg / 4) * np.cos(np.pi * yg / 4)
    u0 = np.exp(-(xg ** 2 + yg ** 2) / 2.0)
    M = 16
    with V.Solver(shape, lo, hi) as sv:
        sv.set_order(so, kappa=1.0, f3=1.0)
        dt = sv.suggest_dt(0.25)
    res, finals = {}, {}
    for nm, im, prec in (("fused", V.IMPL_FUSED, V.F32), ("plain", V.IMPL_PLAIN, V.F32),
                         ("plain_f64", V.IMPL_PLAIN, V.F64)):
        ty = torch.float32 if prec == V.F32 else torch.float64
        u0t = torch.from_numpy(u0).to(ty).cuda()
        sv = V.Solver(shape, lo, hi, prec, im, stream=stream.cuda_stream)
        sv.set_order(so, kappa=1.0, f3=1.0)
        sv.set_M(M)
        sv.set_scheme(V.SCHEME_TSFP2)
        with torch.cuda.stream(stream):
            sv.set_state(u0t)
            sv.step(3, dt)  # warm-up (tables, graphs)
            sv.set_state(u0t)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.step(nsteps, dt)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        finals[nm] = (sv, torch.empty_like(u0t))
        sv.get_state(finals[nm][1])
        sv.sync()
        res[nm] = {"ms_per_step": ms, "value": shape[0] * shape[1] / (ms * 1e-3) / 1e6, "unit": UNIT}
    ref_sv, ref = finals["plain_f64"]
    for nm in ("fused", "plain"):
        res[nm]["rel_l2_vs_plain_f64"] = ref_sv.rel_l2(finals[nm][1], ref)[0]
    for sv, _ in finals.values():
        sv.close()
    res["fused_over_plain"] = res["plain"]["ms_per_step"] / res["fused"]["ms_per_step"]
    res["workload"] = ("1024^2 on [-8,8]^2, s = 1 - 0.4 cos(pi x/4) cos(pi y/4), kappa = 1, f(u) = u^3, M = 16, "
                       f"dt = {dt:.4g} (0.25 x 2/omega_max), Gaussian u0, v0 = 0, {nsteps} splitting steps")
    return res


def small_grids_bench(V, S, torch, stream, nsteps=200, reps=3):
    """The seismic leap-frog step on the smaller grids of the batch and
    serve workloads: the headline's model and source (Q low-passed noise,
    Ricker f0 = 10 at the centre, dt = 5e-4) at 256^2 and 512^2, M = 12 and
    16, fused FP32 against the plain (cuFFT) FP32 path; per step, CUDA events
    over `nsteps` graph-replayed steps after 10, best of `reps`."""
    res = {}
    for n in (256, 512):
        for M in (12, 16):
            w = S.workload_2d_1024(nsteps=nsteps + 10, n=n, M=M)
            row = {}
            for nm, im in (("fused", V.IMPL_FUSED), ("plain", V.IMPL_PLAIN)):
                best = 1e9
                with V.Solver(w["shape"], prec=V.F32, impl=im, stream=stream.cuda_stream) as sv:
                    sv.set_q(w["Q"], w["c0"], w["omega0"])
                    sv.set_M(M)
                    for _ in range(reps):
                        with torch.cuda.stream(stream):
                            sv.set_state(np.zeros(w["shape"], np.float32))
                            sv.set_source(w["src_idx"], w["src"])
                            sv.step(10, w["dt"])
                            stream.synchronize()
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            e0.record(stream)
                            sv.step(nsteps, w["dt"])
                            e1.record(stream)
                            e1.synchronize()
                        best = min(best, e0.elapsed_time(e1) / nsteps)
                row[nm + "_ms_per_step"] = best
            row["fused_over_plain"] = row["plain_ms_per_step"] / row["fused_ms_per_step"]
            res[f"{n}x{n}_M{M}"] = row
    res["workload"] = ("seismic model of the headline (Q low-passed noise seed 2, Ricker f0 = 10 at the centre, "
                       "dt = 5e-4) at 256^2 and 512^2, M = 12 and 16; per leap-frog step")
    return res


# ---------------------------------------------------------------------------
# serving: a Poisson request stream through the continuous-batching server
# ---------------------------------------------------------------------------
def serve_bench(nreq, check=3):
    import synthetic as S
    from paper_2311_13049_gb300 import serve as SV

    def source(sp, dt):
        return S.ricker_samples(sp["nsteps"], dt, sp["f0"])

    reqs = S.serve_requests(600)[:nreq]
    per_kind = min(12, nreq)  # contexts allocated at server start-up, per request kind
    srv = SV.Server(budget_bytes=64 << 30, max_active=48, quantum=50, realtime=True,
                    prewarm={k: per_kind for k in S.SERVE_KINDS})
    try:
        recs, span = srv.run(reqs, S.serve_inputs, source)
    finally:
        srv.close()
    out = SV.summarize(recs, span)
    # a few answers against the same request run alone (first of each kind)
    seen, same = set(), []
    for r, sp in zip(recs, sorted(reqs, key=lambda d: d["arrival"])):
        if sp["shape"] in seen or len(same) >= check:
            continue
        seen.add(sp["shape"])
        Q, idx = S.serve_inputs(sp)
        same.append(bool(np.array_equal(r["result"], SV.solo(sp, Q, idx, source))))
    kinds = {}
    for sp in reqs:
        k = "x".join(str(v) for v in sp["shape"])
        kinds[k] = kinds.get(k, 0) + 1
    out.update({"sample": f"first {nreq} of the 600-request stream (arrivals over "
                          f"{reqs[-1]['arrival']:.2f} s)", "mix": kinds,
                "point_steps": int(sum(r["point_steps"] for r in recs)),
                "solo_equal": same, "policy": "FIFO admission by free slot (48) and footprint (64 GiB); "
                                              "square 2D requests batched, 50-step quanta; "
                                              f"{per_kind} contexts per kind allocated at start-up"})
    return out


def profile_run(V, S, stream, args):
    """Short runs for profilers (print nothing): set-up, then ncu_steps steps
    of the 3D 256^3 workload, of the 64-simulation batch, of the Table 2
    CNFP problem (1D 4096 FP64, dt = 2^-9), of the 1D 256 FP64 run, of the
    fused 2D time splitting (1024^2, M = 16), or ncu_steps applies of the
    generic 512^2 operator (M = 20)."""
    if args.ncu_workload == "cnfp":
        J = 4096
        x = S.axis(J, -32.0, 32.0)
        with V.Solver((J,), [-32.0], [32.0], V.F64, V.IMPL_PLAIN, stream=stream.cuda_stream) as sv:
            sv.set_order(1.0 + 0.3 * np.sin(np.pi * x / 8), kappa=1.0, f3=1.0)
            sv.set_M(15)
            sv.set_scheme(V.SCHEME_CNFP)
            sv.set_state(np.exp(-x * x))
            sv.step(args.ncu_steps, 2.0 ** -9)
            sv.sync()
        return 0
    if args.ncu_workload == "1d":
        w = S.workload_1d_256()
        with V.Solver(w["shape"], prec=V.F64, stream=stream.cuda_stream) as sv:
            sv.set_M(w["M"])
            sv.set_q(w["Q"], w["c0"], w["omega0"])
            sv.set_state(w["u0"])
            sv.step(args.ncu_steps, w["dt"])
            sv.sync()
        return 0
    if args.ncu_workload == "tsfp2":
        shape, lo, hi = (1024, 1024), [-8.0, -8.0], [8.0, 8.0]
        xg, yg = S.mesh(shape, lo, hi)
        with V.Solver(shape, lo, hi, V.F32, V.IMPL_FUSED, stream=stream.cuda_stream) as sv:
            sv.set_order(1.0 - 0.4 * np.cos(np.pi * xg / 4) * np.cos(np.pi * yg / 4), kappa=1.0, f3=1.0)
            sv.set_M(16)
            sv.set_scheme(V.SCHEME_TSFP2)
            sv.set_state(np.exp(-(xg ** 2 + yg ** 2) / 2.0).astype(np.float32))
            sv.step(args.ncu_steps, sv.suggest_dt(0.25))
            sv.sync()
        return 0
    if args.ncu_workload == "generic":
        import torch
        shape, lo, hi = (512, 512), [-8.0, -8.0], [8.0, 8.0]
        xg, yg = S.mesh(shape, lo, hi)
        with V.Solver(shape, lo, hi, V.F32, V.IMPL_FUSED, stream=stream.cuda_stream) as sv:
            sv.set_order(1.0 - 0.4 * np.cos(np.pi * xg / 4) * np.cos(np.pi * yg / 4))
            sv.set_M(20)
            ut = torch.from_numpy(S.gaussian_pulse(shape, 8.0).astype(np.float32)).cuda()
            out = torch.empty_like(ut)
            for _ in range(args.ncu_steps):
                sv.apply(V.OP_S, ut, out)
            sv.sync()
        return 0
    if args.ncu_workload == "3d":
        w = S.workload_3d_256()
        with V.Solver(w["shape"], stream=stream.cuda_stream) as s:
            s.set_M(w["M"])
            s.set_q(w["Q"], w["c0"], w["omega0"])
            s.set_state(w["u0"].astype(np.float32))
            s.step(args.ncu_steps, w["dt"])
            s.sync()
        return 0
    sims = S.workload_batch()
    solvers = []
    with V.Batch(stream=stream.cuda_stream) as b:
        for sp in sims:
            s = V.Solver(sp["shape"], stream=stream.cuda_stream)
            s.set_q(sp["Q"], sp["c0"], sp["omega0"])
            s.set_M(sp["M"])
            dt = s.suggest_dt(0.25)
            s.set_state(np.zeros(sp["shape"], np.float32))
            s.set_source(sp["src_idx"], S.ricker_samples(sp["nsteps"], dt, sp["f0"]))
            b.add(s, dt)
            solvers.append(s)
        b.step(args.ncu_steps)
        b.sync()
    for s in solvers:
        s.close()
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch

    import paper_2311_13049_gb300 as V
    import synthetic as S
    from paper_2311_13049_gb300 import build as B

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()

    w = S.workload_2d_1024(nsteps=NSTEPS)
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    Q_host = torch.from_numpy(w["Q"]).pin_memory()
    u0_host = torch.zeros((NY, NX), dtype=torch.float32).pin_memory()
    src_host = torch.from_numpy(w["src"]).pin_memory()
    out_host = torch.empty((NY, NX), dtype=torch.float32).pin_memory()
    Q_dev = Q_host.cuda()
    u0_dev = u0_host.cuda()
    src_dev = src_host.cuda()
    idx = w["src_idx"]

    def make(impl):
        s = V.Solver((NY, NX), prec=V.F32, impl=impl, stream=stream.cuda_stream)
        s.set_M(M)
        return s

    def run_once(s, host):
        if host:
            s.set_q(Q_host, w["c0"], w["omega0"])
            s.set_state(u0_host)
            s.set_source(idx, src_host)
            s.step(NSTEPS, DT)
            s.get_state(out_host)
        else:
            s.set_q(Q_dev, w["c0"], w["omega0"])
            s.set_state(u0_dev)
            s.set_source(idx, src_dev)
            s.step(NSTEPS, DT)

    def run_once_steps(s, n):
        s.set_q(Q_dev, w["c0"], w["omega0"])
        s.set_state(u0_dev)
        s.set_source(idx, src_dev)
        s.step(n, DT)

    def steady_step_ms(s, n=200):
        """Average time of one leap-frog step inside a run (graph replays)."""
        with torch.cuda.stream(stream):
            run_once_steps(s, 10)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(n, DT)
            e1.record(stream)
            e1.synchronize()
        return e0.elapsed_time(e1) / n

    def timed(s, host, k, wu):
        with torch.cuda.stream(stream):
            for _ in range(wu):
                run_once(s, host)
            stream.synchronize()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            tot = 0.0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(k):
                flush.zero_()
                stream.synchronize()
                e0.record(stream)
                run_once(s, host)
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            torch.cuda.synchronize()
        return max_over_ranks(tot, dist)

    if args.serve_only:
        res = serve_bench(args.serve_requests)
        if rank == 0:
            print(json.dumps({"metric": "serve p50/p99 latency and Mpoint-steps/s", "serve": res}))
        return 0
    if args.ncu_steps and args.ncu_workload != "2d":
        return profile_run(V, S, stream, args)
    fused = make(V.IMPL_FUSED)
    if args.ncu_steps:
        # short run for profilers: set-up, then ncu_steps leap-frog steps
        with torch.cuda.stream(stream):
            run_once_steps(fused, args.ncu_steps)
        stream.synchronize()
        fused.close()
        return 0
    clocks = ClockSampler(local)
    launches0 = V.kernel_launches()
    clocks.start()
    ms_dev = timed(fused, False, args.steps, args.warmup)
    clk = clocks.stop()
    launches = V.kernel_launches() - launches0
    # launches in the timed region only: subtract the warm-up runs' share
    per_run = launches / (args.steps + args.warmup)
    gpu_launches = int(round(per_run * args.steps))
    ms_e2e = timed(fused, True, args.steps, 1)
    final = fused.get_state()  # wavefield after the last run (host)

    lffp_fused = steady_step_ms(fused)
    # adaptive M: the Taylor power the remainder rule picks for this model
    # at 1e-8, its step time, and its apply against M = 16 (same FP32 path)
    adaptive = None
    if rank == 0:
        M_ad = fused.suggest_M(1e-8)
        fused.set_M(M_ad)
        ms_ad = steady_step_ms(fused)
        ut = torch.from_numpy(final).cuda()
        o_ad = [torch.empty_like(ut), torch.empty_like(ut)]
        fused.apply_pair(ut, *o_ad)
        fused.set_M(M)
        o16 = [torch.empty_like(ut), torch.empty_like(ut)]
        fused.apply_pair(ut, *o16)
        fused.sync()
        adaptive = {"tol": 1e-8, "M": M_ad, "ms_per_lffp_step": ms_ad, "speedup_vs_M16": lffp_fused / ms_ad,
                    "apply_rel_l2_vs_M16": [float(torch.linalg.norm(a.double() - b.double()) /
                                                  torch.linalg.norm(b.double())) for a, b in zip(o_ad, o16)]}
    plain = make(V.IMPL_PLAIN)
    kp = max(1, min(args.steps, 3))
    ms_plain = timed(plain, False, kp, 1)
    lffp_plain = steady_step_ms(plain, 50)

    pts = NX * NY * NSTEPS
    value = job_value(ws, pts, args.steps, ms_dev)
    e2e = job_value(ws, pts, args.steps, ms_e2e)
    plain_value = job_value(ws, pts, kp, ms_plain)

    # --- roofline of the dominant kernel (isolated launches, CUDA events on the context stream)
    prof = fused.profile_kernels(reps=20)
    sched = fused.schedule()
    groups = -(-(M + 1) // sched["group"])
    launches_per_step = {nm: (groups if nm.startswith("k2d_inv") else 1) for nm, _, _ in prof}
    share = {nm: ms * launches_per_step.get(nm, 1) for nm, ms, _ in prof}
    dom = max(share, key=share.get)
    dom_ms, dom_units = [(ms, u) for nm, ms, u in prof if nm == dom][0]
    # algorithmic flops of a complex line FFT of length L: 5 L log2 L
    flops = dom_units * 5.0 * 1024 * 10
    peaks = _peaks()
    # the SM clock ceiling: nvidia-smi's clocks.max.sm seen during the timed
    # region, else the measured-peaks file, else GB300's 2070 MHz
    sm_max = float((clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0)
    n_sm = _sm_count()
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    achieved = flops / (dom_ms * 1e-3) / 1e12
    traffic, traffic_note = _ncu_traffic(dom)
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic, "traffic_note": traffic_note,
            "peak_note": f"derived FP32 FMA peak: {n_sm} SMs (read from the device) x 128 lanes x 2 flop x "
                         f"sm_max_mhz {sm_max:.0f}",
            "schedule": sched,
            "flops_per_launch": flops, "ms_per_launch": dom_ms,
            "kernels": {nm: {"ms": ms, "units": u, "launches_per_step": launches_per_step.get(nm, 1)}
                        for nm, ms, u in prof}}

    # --- precision (outside the timed region): one operator-pair apply on the
    # final wavefield by the fused FP32 path and the plain FP32 path, against
    # the plain FP64 path (cuFFT in double) on the same input
    acc = None
    if rank == 0 and not args.skip_accuracy:
        ut = torch.from_numpy(final).cuda()
        ref = V.Solver((NY, NX), prec=V.F64, impl=V.IMPL_PLAIN, stream=stream.cuda_stream)
        ref.set_M(M)
        ref.set_q(Q_dev, w["c0"], w["omega0"])
        u64 = ut.double()
        r1, r2 = torch.empty_like(u64), torch.empty_like(u64)
        ref.apply_pair(u64, r1, r2)
        ref.sync()
        ref.close()
        acc = {}
        for nm, s in (("fused_f32", fused), ("plain_f32", plain)):
            o1, o2 = torch.empty_like(ut), torch.empty_like(ut)
            s.apply_pair(ut, o1, o2)
            s.sync()
            # the library's FP64-accumulating diagnostic (vofl_rel_l2) on the GPU
            d = [fused.rel_l2(o, r) for o, r in ((o1, r1), (o2, r2))]
            acc[nm + "_rel_l2_vs_f64"] = [x[0] for x in d]
            acc[nm + "_max_abs_over_max_vs_f64"] = [x[1] for x in d]
        acc["input"] = ("final wavefield of the timed run (FP32); reference: the plain path in FP64 on the GPU "
                        "(same operators, cuFFT in double); measured by vofl_rel_l2")

    batch = None if args.skip_batch else batch_bench(V, torch, stream, flush)
    configs = None if args.skip_configs else configs_bench(V, torch, stream, flush)
    serve_res = None if args.serve_requests <= 0 else serve_bench(args.serve_requests)
    cpu = cpu_baseline() if (rank == 0 and not args.skip_cpu) else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_dev / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _config(), "impl": "fused",
                "e2e": {"value": e2e, "unit": UNIT, "ms_per_step": ms_e2e / args.steps,
                        "h2d_bytes_per_step": int(Q_host.numel() * 8 + u0_host.numel() * 4 + src_host.numel() * 8),
                        "d2h_bytes_per_step": int(out_host.numel() * 4)},
                "plain": {"value": plain_value, "unit": UNIT, "ms_per_step": ms_plain / kp, "steps": kp,
                          "ms_per_lffp_step": lffp_plain},
                "ms_per_lffp_step": lffp_fused, "adaptive_M": adaptive,
                "fused_over_plain": value / plain_value,
                "accuracy": acc, "gpu_launches": gpu_launches, "roofline": roof,
                "cpu_baseline": cpu, "clocks": clk, "batch": batch, "configs": configs, "serve": serve_res}
        print(json.dumps(line))
    fused.close()
    plain.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--skip-cpu", action="store_true", help="omit the oracle CPU baseline")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-batch", action="store_true", help="omit the 64-simulation batch measurement")
    ap.add_argument("--skip-configs", action="store_true", help="omit the 1D 256 and 3D 256^3 runs")
    ap.add_argument("--serve-requests", type=int, default=40,
                    help="requests of the 600-request serving stream to serve (0: skip)")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving measurement")
    ap.add_argument("--ncu-workload", default="2d", choices=["2d", "3d", "batch", "cnfp", "generic", "1d", "tsfp2"],
                    help="workload of the --ncu-steps profiling mode")
    ap.add_argument("--ncu-steps", type=int, default=0,
                    help="profiling mode: set up the workload, run this many leap-frog steps, print nothing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
