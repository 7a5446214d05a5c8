"""Benchmark of the GB300 acoustic finite-difference hot path.

Default workload (one "step" = one complete forward modelling run): 3D acoustic
forward on a 256^3 physical grid (336^3 computational with the 40-point layer),
12.5 m spacing, space order 8, 1000 time samples (999 stencil updates per
point), one off-grid 15 Hz Ricker source, 128 x 128 receivers at 20 m depth,
FP32 arithmetic, FP32 model.  Inputs are synthetic (seeded two-layer model with
a smoothed +-5% perturbation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload forward|so16|precision|diffusion|fwi|decomp|tblock]

Prints one JSON line (rank 0).  `value` is device-timed throughput in grid-point
updates per second (GPts/s) with inputs resident in HBM; `e2e` is the same
metric through the public API with pinned host buffers (model and wavelet
copied in, traces copied out, every step).  Under torchrun each rank runs its
own shot (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GPts/s & % HBM roofline (SO-8 3D FP32); FWI gradient s/shot, batched vs plain"
B_ALG = 16  # algorithmic bytes per point update: read u^n, u^{n-1}, m; write u^{n+1}
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
KERNEL_SOURCES = ["paper_1609_03361_gb300/csrc/fdw_step.cuh",
                  "paper_1609_03361_gb300/csrc/fdw_device.cuh",
                  "paper_1609_03361_gb300/csrc/fdw_types.h",
                  "paper_1609_03361_gb300/csrc/fdw_internal.h"]


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- distributed

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- workloads

def cfg2_workload(nt=1000, dt_max=None):
    """The 256^3 SO8 workload; `dt_max(ndim, spacing, order, vmax)` gives the
    stability limit (the library's by default; the oracle arm passes the
    oracle's own, so it never loads the library)."""
    from paper_1609_03361_gb300 import workloads as W
    if dt_max is None:
        from paper_1609_03361_gb300 import fdwave as fw
        dt_max = fw.fdw_dt_max
    w = W.config_3d(256, 12.5, 8, nt)
    w.dt = W.choose_dt(dt_max(3, 12.5, 8, w.vmax))
    return w


def cpu_model():
    """Host CPU description for the baseline records (best effort)."""
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for key in ("model name", "Model name", "CPU part"):
            for line in txt.splitlines():
                if line.startswith(key):
                    return f"{key}: {line.split(':', 1)[1].strip()}"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(w, target_s=15.0):
    """FP64 oracle on the host cores: the full computational grid for a few
    time steps, GPts/s (test infrastructure, timed as it stands)."""
    import oracle
    pts = int(np.prod(w.comp_shape))

    def run(nts):
        s = oracle.Setup(w.shape, w.spacing, w.space_order, w.nbl, w.dt, nts)
        M = oracle.extend_model(s, w.m.astype(np.float32).astype(np.float64))
        eta = oracle.damping(s, w.vmax)
        q = w.wavelet()[:nts, None]
        t = time.perf_counter()
        oracle.forward(s, M, eta, w.src, q, w.rec)
        return time.perf_counter() - t

    t2 = run(2)  # one update: calibration
    nts = int(max(2, min(200, target_s / max(t2, 1e-3)))) + 1
    el = run(nts)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if os.environ.get("OMP_NUM_THREADS"):
        cores = min(cores, int(os.environ["OMP_NUM_THREADS"]))
    return {"value": pts * (nts - 1) / el / 1e9, "unit": "GPts/s", "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{w.comp_shape[0]}^3 computational grid, {nts - 1} FP64 time steps "
                      f"({el:.1f} s), same model/source/receivers"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    w = cfg2_workload(dt_max=oracle.dt_max)
    pts = int(np.prod(w.comp_shape))
    s2 = oracle.Setup(w.shape, w.spacing, w.space_order, w.nbl, w.dt, 2)
    M = oracle.extend_model(s2, w.m.astype(np.float32).astype(np.float64))
    eta = oracle.damping(s2, w.vmax)
    q = w.wavelet()[:, None]

    def sample(nts):
        s = oracle.Setup(w.shape, w.spacing, w.space_order, w.nbl, w.dt, nts)
        t = time.perf_counter()
        oracle.forward(s, M, eta, w.src, q[:nts], w.rec)
        return time.perf_counter() - t

    t2 = sample(2)
    per_step_budget = args.ref_seconds / max(1, args.steps + args.warmup)
    nts = int(max(2, min(50, per_step_budget / max(t2, 1e-3)))) + 1
    for _ in range(args.warmup):
        sample(2)
    times = [sample(nts) for _ in range(args.steps)]
    el = sum(times)
    value = pts * (nts - 1) * args.steps / el / 1e9
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GPts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "3D acoustic forward 256^3 (336^3 computational), SO8, FP64 "
                                   f"oracle sample of {nts - 1} time steps per step"},
            "cpu_baseline": {"value": value, "unit": "GPts/s", "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"{nts - 1} time steps of the full 336^3 grid per step"},
            "e2e": {"value": value, "unit": "GPts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_forward(args, world, rank, local):
    import torch
    from paper_1609_03361_gb300 import fdwave as fw
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = cfg2_workload(args.nt)
    pts = int(np.prod(w.comp_shape))
    s = fw.Solver(w.shape, w.spacing, w.space_order, w.nbl, w.dt, w.nt, w.vmax, device=local)
    m32 = w.m.astype(np.float32)
    m_dev = torch.from_numpy(m32).to(dev)
    s.set_model(m_dev)
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    q_dev = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev)
    rec_dev = torch.empty((w.nt, w.rec.shape[0]), dtype=torch.float32, device=dev)
    if args.tiling:
        t, lx, st = (int(v) for v in args.tiling.split(","))
        s.set_tiling(t, lx, st)
        s.set_model(m_dev)
        s.set_sources(w.src)
        s.set_receivers(w.rec)
    elif not args.no_autotune:
        s.autotune(20)
    tiling = s.tiling()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        s.forward(q_dev, rec_dev)
    torch.cuda.synchronize(dev)
    s.sync()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.forward(q_dev, rec_dev)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    ms = max_over_ranks(ms_local, world)
    s.sync()
    updates = pts * (w.nt - 1)
    value = world * updates * args.steps / (ms * 1e-3) / 1e9
    # one persistent step-kernel launch over the nt-1 steps and one sampling
    # launch for the last time sample, per forward run
    launches = args.steps * 2

    # roofline of the step kernel (its launches fill the timed region),
    # per time step of the persistent launch: 16 B x points per step over
    # the launch's time per step
    avg_step_s = (ms_local * 1e-3) / (args.steps * (w.nt - 1))
    achieved = B_ALG * pts / avg_step_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    try:
        with open(PROFILE_TRAFFIC) as f:
            tr = json.load(f)
        if tr.get("kernel_hash") == kernel_hash() and tr.get("points") == pts:
            traffic = tr["dram_bytes_per_step"]
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "frac_of_nominal_7900": achieved / 7900.0,
                "bytes_per_point": B_ALG, "points_per_step": pts,
                "per": "time step of the persistent step-kernel launch (nt - 1 steps a launch)"}

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        m_h = torch.from_numpy(m32).pin_memory()
        q_h = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).pin_memory()
        rec_h = torch.empty((w.nt, w.rec.shape[0]), dtype=torch.float32).pin_memory()
        s.set_model(m_h)
        s.forward(q_h, rec_h)
        torch.cuda.synchronize(dev)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.set_model(m_h)
            s.forward(q_h, rec_h)
            torch.cuda.synchronize(dev)
            float(rec_h[-1, 0])   # the host reads the result of the step
        el = max_over_ranks(time.perf_counter() - t0, world)
        assert torch.allclose(rec_h.to(dev), rec_dev), "host-buffer path disagrees"
        e2e = {"value": world * updates * args.steps / el / 1e9, "unit": "GPts/s",
               "h2d_bytes_per_step": int(m32.nbytes + q_h.numel() * 4),
               "d2h_bytes_per_step": int(rec_h.numel() * 4)}
    s.sync()

    # the adjoint propagator on the same shot (receivers inject the data,
    # the source samples), graph launched like the forward
    adjoint = None
    if not args.no_extras and world == 1:
        d_dev = rec_dev.clone()
        s.set_model(m_dev)
        s.adjoint(d_dev)
        torch.cuda.synchronize(dev)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(3):
            s.adjoint(d_dev)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ms_a = a0.elapsed_time(a1) / 3
        adjoint = {"workload": "the same shot backwards: 16384 receivers inject, the source samples",
                   "gpts": updates / (ms_a * 1e-3) / 1e9, "ms_per_run": ms_a}
        s.sync()

    base = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(w)

    extras = {}
    if not args.no_extras and world == 1:   # single-GPU measurements: once, at N = 1
        extras["adjoint"] = adjoint
        extras["batched"] = run_batched(args.batch_shots, 800, dev)
        extras["fwi"] = run_fwi(args.fwi_shots, args.fwi_nt, 10, dev)
        extras["diffusion"] = run_diffusion(dev)
        extras["decomposition"] = run_decomp(dev)
        extras["two_step"] = run_tblock(dev)
        extras["so16"] = so16_measure(dev)
        extras["precision"] = precision_measure(dev)
        snap = extras["precision"]["snapshot_storage_vs_fp64_oracle_gradient"]
        extras["fwi"]["reduced_case_vs_fp64_oracle"] = {
            "workload": snap["workload"],
            "grad_rel_l2_fp16_vs_fp64": snap["rel_l2_gradient"]["f16"],
            "grad_rel_l2_bf16_vs_fp64": snap["rel_l2_gradient"]["bf16"],
            "grad_rel_l2_fp32_vs_fp64": snap["rel_l2_gradient"]["f32"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GPts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "3D acoustic forward, 256^3 physical (336^3 computational, "
                                       "40-point layer), h=12.5 m, SO8, 1000 time samples, 1 "
                                       "Ricker 15 Hz source, 128x128 receivers, FP32 model",
                           "updates_per_step": updates, "parallelism": f"shots x{world}",
                           "l2": "inputs larger than L2 (3 fields x 159 MB resident)",
                           "tiling": tiling},
                "roofline": roofline, "cpu_baseline": base, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk}
        line.update(extras)
        print(json.dumps(line), flush=True)
    s.close()


def run_diffusion(dev):
    """2D diffusion of Sec. 4: the 1000^2, 500-step example (L2-resident) and a
    16384^2 grid (1 GiB per field, HBM-bound), GPts/s = point updates per
    second from CUDA events; the example is checked against the FP64 oracle,
    which is also timed on it (test infrastructure, as it stands)."""
    import torch
    import oracle
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300 import workloads as W
    out = {"workload": "2D diffusion, forward Euler, 5-point, dt at the Eq. 2 limit"}
    stream = torch.cuda.current_stream(dev)

    def timed(u0, dx, steps, spp, reps):
        u = u0.clone()
        tmp = torch.empty_like(u)
        dt = W.diffusion_dt(dx, dx)
        fw.fdw_diffusion2d(u, tmp, dx, dx, 1.0, dt, steps, spp)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(reps):
            u.copy_(u0)
            e0.record(stream)
            fw.fdw_diffusion2d(u, tmp, dx, dx, 1.0, dt, steps, spp)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1))
        return u, best

    u0h = W.diffusion_field(1000, 1000, seed=0).astype(np.float32)
    u0 = torch.from_numpy(u0h).to(dev)
    u, ms = timed(u0, 0.001, 500, 0, 5)
    t = time.perf_counter()
    ref = oracle.diffusion(u0h.astype(np.float64), 0.001, 0.001, 1.0, W.diffusion_dt(0.001, 0.001), 500)
    el = time.perf_counter() - t
    out["example_1000sq_500_steps"] = {
        "gpts": 1e6 * 500 / (ms * 1e-3) / 1e9, "ms": ms, "steps_per_pass": 4,
        "max_abs_err_vs_oracle": float(np.abs(u.cpu().numpy() - ref).max()),
        "oracle_gpts": 1e6 * 500 / el / 1e9, "oracle_cores": 1}
    del u, u0
    big = torch.from_numpy(W.diffusion_field(4096, 4096, seed=1).astype(np.float32)).to(dev)
    u0 = big.repeat(4, 4)   # 16384^2, 1 GiB per field
    del big
    peak, kind = measured_peaks()
    res = {}
    for spp in (1, 2, 4, 8):
        _, ms = timed(u0, 1e-3, 32, spp, 3)
        g = 16384 * 16384 * 32 / (ms * 1e-3) / 1e9
        res[f"spp{spp}"] = {"gpts": g, "hbm_gbs_algorithmic": 8.0 * g / spp}
    one = res["spp1"]["hbm_gbs_algorithmic"]
    out["grid_16384sq_32_steps"] = res
    out["roofline_1step"] = {"bound": "hbm", "bytes_per_point": 8, "achieved": one, "peak": peak,
                             "unit": "GB/s", "frac": one / peak, "peak_kind": kind,
                             "ceiling_gpts": peak / 8.0}
    del u0
    torch.cuda.empty_cache()
    return out


def run_decomp(dev, nt=200, nparts=2):
    """Single-shot domain decomposition on this one GPU: the 256^3 SO8 shot cut
    into x slabs held by one process (ghost planes exchanged by device copies
    after every step), against the whole grid stepped the same way (one host
    call per step, no CUDA graph).  On one GPU the slabs share the device, so
    this measures the cost of the decomposition (exchange, smaller launches),
    not a speed-up."""
    import torch
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300.decomp import SlabForward
    w = cfg2_workload(nt)
    pts = int(np.prod(w.comp_shape))
    q = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev)
    m = torch.from_numpy(w.m.astype(np.float32)).to(dev)
    nrec = w.rec.shape[0]
    stream = torch.cuda.current_stream(dev)

    def timed(run):
        run()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    s = fw.Solver(w.shape, w.spacing, w.space_order, w.nbl, w.dt, nt, w.vmax,
                  device=dev.index or 0)
    s.set_model(m)
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    rec = torch.zeros((nt, nrec), device=dev)

    def whole():
        for n in range(nt):
            s.step(n, q, rec)
    ms_whole = timed(whole)
    sf = SlabForward(w.shape, w.spacing, w.space_order, w.nbl, w.dt, nt, w.vmax, nparts,
                     devices=[dev.index or 0] * nparts)
    sf.set_model(m)
    sf.set_sources(w.src)
    sf.set_receivers(w.rec)
    recs = [torch.zeros((nt, nrec), device=dev) for _ in range(nparts)]
    ms_slabs = timed(lambda: sf.forward([q] * nparts, recs))
    same = bool(torch.equal(sum(recs), rec))
    halo = fw.fdw_halo_planes(sf.slabs[0].ctx, 0)[4] * 4
    sf.close()
    s.close()
    return {"workload": f"256^3 SO8 shot, {nt} steps, {nparts} x slabs on one GPU",
            "gpts_whole_stepwise": pts * (nt - 1) / (ms_whole * 1e-3) / 1e9,
            "gpts_slabs": pts * (nt - 1) / (ms_slabs * 1e-3) / 1e9,
            "exchange_bytes_per_step": 2 * (nparts - 1) * halo,
            "traces_identical": same}


def run_batched(nshots, nt, dev, timed_reps=1):
    """Batched forward: nshots uneven cubes (96^3..192^3 physical, +40-point
    layer), SO8, nt steps, one launch per time step over all shots, against
    the same shots run one after the other.  Returns a dict."""
    import torch
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300 import workloads as W
    shots = W.batched_shots(nshots=nshots, nt=nt)
    vmax = max(w.vmax for w in shots)
    dt = W.choose_dt(fw.fdw_dt_max(3, shots[0].spacing, 8, vmax))
    solvers, qs, recs = [], [], []
    for w in shots:
        w.dt = dt
        s = fw.Solver(w.shape, w.spacing, 8, w.nbl, dt, nt, vmax, device=dev.index or 0)
        s.set_model(torch.from_numpy(w.m.astype(np.float32)).to(dev))
        s.set_sources(w.src)
        s.set_receivers(w.rec)
        solvers.append(s)
        qs.append(torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev))
        recs.append(torch.empty((nt, w.rec.shape[0]), device=dev))
    updates = sum(int(np.prod(w.comp_shape)) for w in shots) * (nt - 1)
    b = fw.Batch(solvers)
    b.autotune(10)
    b.forward(qs, recs)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(timed_reps):
        b.forward(qs, recs)
    e1.record()
    torch.cuda.synchronize(dev)
    t_batch = e0.elapsed_time(e1) / 1e3 / timed_reps
    ref = [r.clone() for r in recs]
    b.close()
    for s, q, r in zip(solvers, qs, recs):   # warm each plain path once
        s.forward(q, r)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(timed_reps):
        for s, q, r in zip(solvers, qs, recs):
            s.forward(q, r)
    e1.record()
    torch.cuda.synchronize(dev)
    t_plain = e0.elapsed_time(e1) / 1e3 / timed_reps
    same = all(bool(torch.equal(a, c)) for a, c in zip(ref, recs))
    for s in solvers:
        s.close()
    return {"workload": f"{nshots} shots, cubes of {min(w.shape[0] for w in shots)}^3.."
                        f"{max(w.shape[0] for w in shots)}^3 (+40-point layer), SO8, {nt} steps",
            "gpts_batched": updates / t_batch / 1e9, "gpts_plain": updates / t_plain / 1e9,
            "s_batched": t_batch, "s_plain": t_plain, "traces_identical": same}


def run_fwi(nshots, nt, k, dev, group=4):
    """FWI gradient of J = 1/2 sum |P_r u - d_obs|^2 over nshots shots on the
    256^3 SO8 model (observed data from the model with a +5% Gaussian anomaly):
    plain = shots one by one with FP32 checkpoints; batched = all shots per
    launch with FP16 snapshots (one float32 scale each).  Returns s/shot for
    both and the relative L2 difference of the summed gradients."""
    import torch
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300 import workloads as W
    shots, v_true = W.fwi_shots(nt=nt, nshots=nshots)
    base = shots[0]
    vmax = float(max(base.velocity.max(), v_true.max()))
    dt = W.choose_dt(fw.fdw_dt_max(3, base.spacing, base.space_order, vmax))
    m0 = torch.from_numpy(base.m.astype(np.float32)).to(dev)
    mt = torch.from_numpy((1.0 / v_true ** 2).astype(np.float32)).to(dev)
    for w in shots:
        w.dt = dt
    qs = [torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev) for w in shots]
    nrec = base.rec.shape[0]
    # observed data and the plain per-shot gradient with one reused solver
    s = fw.Solver(base.shape, base.spacing, base.space_order, base.nbl, dt, nt, vmax,
                  device=dev.index or 0)
    s.set_receivers(base.rec)
    dobs = []
    s.set_model(mt)
    for w, q in zip(shots, qs):
        s.set_sources(w.src)
        dobs.append(s.forward(q))
    s.set_model(m0)
    rec = torch.empty((nt, nrec), device=dev)
    g_plain = torch.zeros(base.comp_shape, device=dev, dtype=torch.float64)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g_first = None
    for w, q, d in zip(shots, qs, dobs):
        s.set_sources(w.src)
        s.forward_ckpt(q, k, "f32", rec=rec)
        g = s.gradient(rec, d)
        if g_first is None:
            g_first = g.clone()
        g_plain += g.double()
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    # the first shot again under a budget of `budget` FP16 checkpoint pairs
    # (binomial schedule) instead of one pair per k steps
    budget = 10
    s.set_sources(shots[0].src)
    s.set_checkpoint_budget(budget)
    s.forward_ckpt(qs[0], k, "f16", rec=rec)
    s.gradient(rec, dobs[0])   # schedule set-up and graph capture, untimed
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s.forward_ckpt(qs[0], k, "f16", rec=rec)
    g_budget = s.gradient(rec, dobs[0])
    torch.cuda.synchronize(dev)
    t_budget = time.perf_counter() - t0
    gn1 = float(torch.linalg.vector_norm(g_first.double()))
    budget_diff = (float(torch.linalg.vector_norm(g_budget.double() - g_first.double())) / gn1
                   if gn1 > 0 else None)   # None: the residual is zero (too few steps)
    pair_bytes = 2 * 2 * base.comp_shape[0] * base.comp_shape[1] * ((base.comp_shape[2] + 31) // 32 * 32)
    s.close()
    # batched with FP16 snapshots
    solvers = []
    for w in shots:
        sv = fw.Solver(base.shape, base.spacing, base.space_order, base.nbl, dt, nt, vmax,
                       device=dev.index or 0)
        sv.set_model(m0)
        sv.set_sources(w.src)
        sv.set_receivers(base.rec)
        solvers.append(sv)
    # groups of `group` shots per batch keep the FP16 snapshots within HBM
    groups = [list(range(i, min(i + group, nshots))) for i in range(0, nshots, group)]
    batches = [fw.Batch([solvers[i] for i in g]) for g in groups]
    recs = [torch.empty((nt, nrec), device=dev) for _ in shots]
    g_batch = torch.zeros_like(g_plain)
    b0 = batches[0]
    b0.forward_ckpt([qs[i] for i in groups[0]], k, "f16", recs=[recs[i] for i in groups[0]])
    torch.cuda.synchronize(dev)   # allocation and graph capture of one group, untimed
    t0 = time.perf_counter()
    for g, b in zip(groups, batches):
        b.forward_ckpt([qs[i] for i in g], k, "f16", recs=[recs[i] for i in g])
        grads = b.gradient([recs[i] for i in g], [dobs[i] for i in g])
        for gr in grads:
            g_batch += gr.double()
        if len(groups) > 1:   # release this group's checkpoints before the next group
            b.close()
            for i in g:
                solvers[i].close()
    torch.cuda.synchronize(dev)
    t_batch = time.perf_counter() - t0
    gn = float(torch.linalg.vector_norm(g_plain))
    diff = float(torch.linalg.vector_norm(g_batch - g_plain)) / gn if gn > 0 else None
    for b in batches:
        b.close()
    for sv in solvers:
        sv.close()
    # the FP64 oracle's gradient (full forward history kept in host memory) on
    # a bounded sample: the first shot over the first few time steps, scaled to
    # nt steps (test infrastructure, timed as it stands)
    import oracle
    nts = 12
    st = oracle.Setup(base.shape, base.spacing, base.space_order, base.nbl, dt, nts)
    M = oracle.extend_model(st, base.m.astype(np.float32).astype(np.float64))
    eta = oracle.damping(st, vmax)
    q0 = shots[0].wavelet()[:nts, None].astype(np.float64)
    r0 = np.random.default_rng(0).standard_normal((nts, nrec))
    t0 = time.perf_counter()
    oracle.forward(st, M, eta, shots[0].src, q0, base.rec)
    oracle.gradient(st, M, eta, shots[0].src, q0, base.rec, r0)
    t_oracle = (time.perf_counter() - t0) * (nt - 1) / (nts - 1)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"workload": f"{nshots} shots, 256^3 (336^3 computational), SO8, {nt} steps, "
                        f"checkpoints every {k} steps",
            "oracle_s_per_shot": t_oracle,
            "oracle_sample": f"first shot, {nts} time steps of forward + gradient on the full "
                             f"grid, FP64, {cores} host cores, scaled to {nt} steps",
            "s_per_shot_plain_fp32": t_plain / nshots, "s_per_shot_batched_fp16": t_batch / nshots,
            "grad_rel_l2_batched_fp16_vs_plain_fp32": diff,
            "budget": {"pairs": budget, "checkpoint_gb": budget * pair_bytes / 1e9,
                       "unlimited_pairs": (nt - 1) // k,
                       "unlimited_checkpoint_gb": ((nt - 1) // k) * pair_bytes / 1e9,
                       "s_per_shot_fp16": t_budget,
                       "grad_rel_l2_vs_plain_fp32": budget_diff}}


def so16_measure(dev, steps=3, warmup=1, nt=2000, tiling=None):
    """512^3 SO16 forward (592^3 computational), nt steps, FP32: GPts/s from
    CUDA events over `steps` whole runs after `warmup` runs, autotuned tiles,
    and the step kernel's HBM roofline fraction (16 B per point update)."""
    import torch
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300 import workloads as W
    w = W.config_3d(512, 12.5, 16, nt)
    w.dt = W.choose_dt(fw.fdw_dt_max(3, w.spacing, 16, w.vmax))
    pts = int(np.prod(w.comp_shape))
    s = fw.Solver(w.shape, w.spacing, 16, w.nbl, w.dt, w.nt, w.vmax, device=dev.index or 0)
    s.set_model(torch.from_numpy(w.m.astype(np.float32)).to(dev))
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    q = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev)
    rec = torch.empty((w.nt, w.rec.shape[0]), device=dev)
    if tiling:
        s.set_tiling(*tiling)
        s.set_model(torch.from_numpy(w.m.astype(np.float32)).to(dev))
        s.set_sources(w.src)
        s.set_receivers(w.rec)
    else:
        s.autotune(3)
    for _ in range(warmup):
        s.forward(q, rec)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        s.forward(q, rec)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    s.sync()
    tiling = s.tiling()
    s.close()
    g = pts * (w.nt - 1) / (ms * 1e-3) / 1e9
    peak, kind = measured_peaks()
    return {"workload": f"3D acoustic forward 512^3 (592^3 computational), SO16, {w.nt} time "
                        "samples, FP32 model, 16384 receivers",
            "gpts": g, "ms_per_run": ms, "runs_timed": steps, "tiling": tiling,
            "roofline": {"bound": "hbm", "achieved": g * B_ALG, "peak": peak, "unit": "GB/s",
                         "frac": g * B_ALG / peak, "peak_kind": kind,
                         "bytes_per_point": B_ALG, "points_per_launch": pts}}


def run_so16(args, dev):
    tiling = tuple(int(v) for v in args.tiling.split(",")) if args.tiling else None
    r = so16_measure(dev, args.steps, args.warmup, args.nt if args.nt != 1000 else 2000, tiling)
    line = {"metric": "GPts/s (SO-16 3D FP32 forward)", "value": r["gpts"], "unit": "GPts/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_run"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": r["workload"], "tiling": r["tiling"]},
            "roofline": r["roofline"]}
    print(json.dumps(line), flush=True)


def run_tblock(dev, nt=101, orders=(2, 4), variants=(0, 1), baseline=True, reps=5):
    """Forward on the 256^3 recipe (336^3 computational) at space orders
    2 and 4: one step per launch (autotuned) against two steps per launch
    (both row variants), GPts/s, the algorithmic-HBM fraction of each (16 B
    per point-step for one step; 20 B per point per pass = 10 B per
    point-step for two) and the traces' difference."""
    import torch
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300 import workloads as W
    peak, _ = measured_peaks()
    out = {"workload": f"3D acoustic forward 256^3 (336^3 computational), {nt} steps, FP32",
           "orders": {}}
    for p in orders:
        w = W.config_3d(256, 12.5, p, nt)
        w.dt = W.choose_dt(fw.fdw_dt_max(3, w.spacing, p, w.vmax))
        pts = int(np.prod(w.comp_shape))
        m = torch.from_numpy(w.m.astype(np.float32)).to(dev)
        q = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev)
        res, recs = {}, {}
        runs = ([("one_step", 1, -1)] if baseline else []) + \
            [(f"two_step_v{v}", 2, v) for v in variants]
        for name, steps, variant in runs:
            s = fw.Solver(w.shape, w.spacing, p, w.nbl, w.dt, w.nt, w.vmax, device=dev.index or 0)
            s.set_model(m)
            s.set_sources(w.src)
            s.set_receivers(w.rec)
            if steps == 2:
                s.set_time_blocking(2, variant)
            else:
                s.autotune(10)
            rec = torch.empty((w.nt, w.rec.shape[0]), device=dev)
            for _ in range(3):
                s.forward(q, rec)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                s.forward(q, rec)
            e1.record()
            torch.cuda.synchronize(dev)
            s.sync()
            ms = e0.elapsed_time(e1) / reps
            g = pts * (w.nt - 1) / (ms * 1e-3) / 1e9
            b = 16.0 if steps == 1 else 10.0
            res[name] = {"gpts": g, "ms_per_run": ms, "hbm_frac_alg": g * b / peak,
                         "config": s.tiling() if steps == 1 else s.time_blocking()}
            recs[name] = rec.cpu().numpy().astype(np.float64)
            s.close()
        if baseline:
            ref = recs["one_step"]
            for name in recs:
                if name != "one_step":
                    res[name]["rec_rel_l2_vs_one_step"] = float(
                        np.linalg.norm(recs[name] - ref) / np.linalg.norm(ref))
        out["orders"][f"so{p}"] = res
    return out


def precision_measure(dev):
    """Errors of the 16-bit model and snapshot storage.  Model: SO16 with the
    512^3 recipe, traces of FP32 / FP16 / BF16 model storage against the FP64
    oracle on a 128^3 grid (all steps) and against each other on the full
    512^3 grid.  Snapshots: SO8 gradients with FP32 / FP16 / BF16 checkpoints
    against the FP64 oracle gradient on a 64^3 grid, 400 steps (the oracle is
    test infrastructure, run as it stands)."""
    import torch
    import oracle
    from paper_1609_03361_gb300 import fdwave as fw
    from paper_1609_03361_gb300 import workloads as W

    def rel(a, b):
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    out = {}
    # (1) model storage vs FP64 oracle, reduced grid, SO16
    n, nt = 128, 600
    w = W.config_3d(n, 12.5, 16, nt, nrec_side=32)
    w.dt = W.choose_dt(fw.fdw_dt_max(3, w.spacing, 16, w.vmax))
    st = oracle.Setup(w.shape, w.spacing, 16, w.nbl, w.dt, nt)
    q = w.wavelet().astype(np.float32)[:, None]
    ref = oracle.forward(st, oracle.extend_model(st, w.m.astype(np.float32).astype(np.float64)),
                         oracle.damping(st, w.vmax), w.src, q.astype(np.float64), w.rec)
    s = fw.Solver(w.shape, w.spacing, 16, w.nbl, w.dt, nt, w.vmax, device=dev.index or 0)
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    res = {}
    for mt in ("f32", "f16", "bf16"):
        s.set_model(w.m.astype(np.float32), "physical", mt)
        res[mt] = rel(s.forward(q), ref)
    s.close()
    out["model_storage_vs_fp64_oracle"] = {"workload": f"{n}^3 SO16, {nt} steps, 1024 receivers",
                                           "rel_l2_traces": res}
    # (2) model storage on the full 512^3 grid, against FP32 storage
    w = W.config_3d(512, 12.5, 16, 2000)
    w.dt = W.choose_dt(fw.fdw_dt_max(3, w.spacing, 16, w.vmax))
    s = fw.Solver(w.shape, w.spacing, 16, w.nbl, w.dt, w.nt, w.vmax, device=dev.index or 0)
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    qd = torch.from_numpy(w.wavelet().astype(np.float32)[:, None]).to(dev)
    md = torch.from_numpy(w.m.astype(np.float32)).to(dev)
    tr, gp = {}, {}
    pts = int(np.prod(w.comp_shape))
    for mt in ("f32", "f16", "bf16"):
        s.set_model(md, "physical", mt)
        tr[mt] = s.forward(qd).cpu().numpy()
        # the same run again, timed (16 B of algorithmic traffic per point
        # with the FP32 model, 14 B with a 16-bit one)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.forward(qd)
        e1.record()
        torch.cuda.synchronize(dev)
        gp[mt] = pts * (w.nt - 1) / (e0.elapsed_time(e1) * 1e-3) / 1e9
    tiling = s.tiling()
    s.close()
    out["model_storage_full_grid_vs_fp32"] = {
        "workload": "512^3 (592^3 computational) SO16, 2000 steps, 16384 receivers",
        "rel_l2_traces": {mt: rel(tr[mt], tr["f32"]) for mt in ("f16", "bf16")},
        "gpts": gp, "tiling": tiling}
    # (3) snapshot storage vs the FP64 oracle gradient
    n, nt = 64, 400
    w = W.config_3d(n, 12.5, 8, nt, nrec_side=32)
    w.dt = W.choose_dt(fw.fdw_dt_max(3, w.spacing, 8, w.vmax))
    st = oracle.Setup(w.shape, w.spacing, 8, w.nbl, w.dt, nt)
    M = oracle.extend_model(st, w.m.astype(np.float32).astype(np.float64))
    eta = oracle.damping(st, w.vmax)
    q = w.wavelet().astype(np.float32)[:, None]
    d = oracle.forward(st, oracle.extend_model(st, (1 / W.anomaly(w.velocity) ** 2)),
                       eta, w.src, q.astype(np.float64), w.rec)
    s = fw.Solver(w.shape, w.spacing, 8, w.nbl, w.dt, nt, w.vmax, device=dev.index or 0)
    s.set_model(w.m.astype(np.float32))
    s.set_sources(w.src)
    s.set_receivers(w.rec)
    d32 = d.astype(np.float32)
    gres = {}
    for stype in ("f32", "f16", "bf16"):
        rec = s.forward_ckpt(q, 10, stype)
        g = s.gradient(rec, d32)
        if stype == "f32":
            gref = oracle.gradient(st, M, eta, w.src, q.astype(np.float64), w.rec,
                                   rec.astype(np.float64) - d)
        gres[stype] = rel(g, gref)
    s.close()
    out["snapshot_storage_vs_fp64_oracle_gradient"] = {
        "workload": f"{n}^3 SO8, {nt} steps, checkpoints every 10 steps, +5% anomaly data",
        "rel_l2_gradient": gres,
        "bound": 1e-3, "within_bound": {k: v <= 1e-3 for k, v in gres.items()}}
    return out


def run_precision(args, dev):
    print(json.dumps(precision_measure(dev)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="forward",
                    choices=["forward", "so16", "precision", "diffusion", "fwi", "decomp",
                             "tblock"])
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="host-time budget of the --impl reference run (oracle steps per step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiling", default="", help="tile,xchunk,stages instead of autotuning")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and FWI parts")
    ap.add_argument("--batch-shots", type=int, default=64)
    ap.add_argument("--fwi-shots", type=int, default=16)
    ap.add_argument("--fwi-nt", type=int, default=2000)
    ap.add_argument("--tb-orders", default="2,4", help="space orders of --workload tblock")
    ap.add_argument("--tb-variants", default="0,1", help="two-step row variants to time")
    ap.add_argument("--tb-no-baseline", action="store_true",
                    help="skip the one-step runs of --workload tblock")
    ap.add_argument("--tb-reps", type=int, default=5, help="timed runs per tblock config")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mine":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    world, rank, local = dist_init()
    if args.workload != "forward":
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        if rank == 0:
            if args.workload == "diffusion":
                print(json.dumps(run_diffusion(dev)), flush=True)
            elif args.workload == "decomp":
                print(json.dumps(run_decomp(dev)), flush=True)
            elif args.workload == "tblock":
                print(json.dumps(run_tblock(
                    dev, args.nt if args.nt != 1000 else 101,
                    tuple(int(v) for v in args.tb_orders.split(",")),
                    tuple(int(v) for v in args.tb_variants.split(",")),
                    not args.tb_no_baseline, args.tb_reps)), flush=True)
            elif args.workload == "fwi":
                print(json.dumps(run_fwi(args.fwi_shots, args.fwi_nt, 10, dev)), flush=True)
            else:
                (run_so16 if args.workload == "so16" else run_precision)(args, dev)
        return
    run_forward(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
