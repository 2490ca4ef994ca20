#!/usr/bin/env python
"""Throughput benchmark of the GB300 PIC hot path.

One benchmark "step" is one pass of the whole hot path over the resident
particle store: re-binning when due, CIC deposit, FFT field solve, fused
gather + push, and the FP64 diagnostic reductions.  The default workload is
Landau damping on a 128^3 grid with 64 particles per cell (134,217,728
particles, L = 4 pi, alpha = 0.05, dt = 0.05), synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Rank 0 prints one JSON line.  With N > 1 (launched by torchrun) every rank
runs an independent replica of the workload on its own GPU (replicas only:
no data-path collective); the value is the particle-steps of all ranks over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (deposit+gather+push) & % HBM roofline; adjoint/forward time"

# launch configuration of the timed step (also used by the full-size parity test)
LAUNCH = dict(sort_period=4, options=1)
UNIT = "particle-steps/s"
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 20; 100 for the ensemble, as configured)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--grid", type=int, default=None,
                    help="grid nodes per axis (default 128; 256 for the Penning bunch)")
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--sort-period", type=int, default=None,
                    help="steps between re-binnings (default 4; 2 for the Penning bunch, whose "
                         "particles cross cells faster on its 256^3 mesh)")
    ap.add_argument("--options", type=int, default=LAUNCH["options"])
    ap.add_argument("--stray-rebin", type=float, default=0.0,
                    help="re-bin on the device when the last push left more than this fraction "
                         "of the particles outside their tile's guard (0: period only)")
    ap.add_argument("--diag-every", type=int, default=1)
    ap.add_argument("--dt", type=float, default=0.05,
                    help="time step (0.05: the Landau benchmark; the paper's scaling runs use "
                         "0.5 h_min, i.e. 0.005 for its finest mesh)")
    ap.add_argument("--guard", type=int, default=None,
                    help="deposit tile guard layers (default 2; 3 for the Penning bunch)")
    ap.add_argument("--tile", type=int, default=0,
                    help="deposit / binning tile edge in cells (default 8)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=1 << 21,
                    help="particles in the oracle's bounded sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cpu-configs", dest="cpu_configs", action="store_false",
                    help="skip the oracle timings of the other configurations")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the side measurements of the default run (split-call deposit "
                         "roofline, FP32-deposit line, Penning line, 512-instance ensemble)")
    ap.add_argument("--no-side-lines", action="store_true",
                    help="skip the FP32-deposit, Penning and ensemble lines but keep the "
                         "split-call deposit roofline")
    ap.add_argument("--side-steps", type=int, default=10,
                    help="timed steps of each side measurement")
    ap.add_argument("--workload", default="landau",
                    choices=["landau", "uniform", "penning", "ensemble", "adjoint"],
                    help="landau: the benchmark step; uniform: the uniform plasma test (random "
                         "moves instead of the push) on the same grid; penning: the Penning-trap "
                         "bunch (256^3, 1.3e8 particles, Boris + quadrupole); ensemble: batched "
                         "instances vs per-instance launches; adjoint: only the adjoint cost")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--shard", default="replicas", choices=["replicas", "particles"],
                    help="with N > 1 GPUs: replicas (independent runs, the default) or "
                         "particles (one run, particles split over the ranks, rho summed by an "
                         "all-reduce each step, the field solved on every rank)")
    ap.add_argument("--ens-count", type=int, default=512, help="ensemble instances")
    ap.add_argument("--record-traffic", metavar="NCU_CSV",
                    help="write profiles/traffic.json from an ncu --csv capture of "
                         "k_push_deposit on the 64^3 x 64 case (dram__bytes_read/write.sum), "
                         "then exit")
    args = ap.parse_args()
    penning = args.workload == "penning"
    if args.steps is None:
        args.steps = 100 if args.workload == "ensemble" else 20
    if args.grid is None:
        args.grid = 256 if penning else 128
    if args.sort_period is None:
        args.sort_period = 2 if penning else LAUNCH["sort_period"]
    if args.guard is None:
        args.guard = 3 if penning else 0
    return args


def workload_name(args):
    n = args.grid
    if args.workload == "penning":
        return (f"penning_trap_3d: {n}^3 grid on [0,20)^3, 130,000,000 particles in a Gaussian "
                f"bunch sigma=(1,1,2), Bz=5, axial frequency 1, Q=-1562.5, dt={args.dt:g}")
    if args.workload == "uniform":
        return (f"uniform_plasma_3d (random moves in [-h, h)): {n}^3 grid, {args.ppc} "
                f"particles/cell ({n ** 3 * args.ppc:,} particles), L=4pi, dt={args.dt:g}")
    return (f"landau_damping_3d: {n}^3 grid, {args.ppc} particles/cell "
            f"({n ** 3 * args.ppc:,} particles), L=4pi, alpha=0.05, k=0.5, dt={args.dt:g}")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- ranks

def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's figure (replicas report the job's time as the max)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas: all ranks' units over the max time."""
    return units_per_rank * world * steps / seconds


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        mhz, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxes),
                "reasons": sorted(reasons), "samples": len(mhz)}


# ---------------------------------------------------------------- oracle arm

def oracle_sample(args, n_particles):
    """A bounded sample of the benchmark workload: the same grid and physics,
    n_particles drawn from the same distribution."""
    import pic_inputs as pi

    ppc = max(1, -(-n_particles // args.grid ** 3))
    if args.workload == "uniform":
        w = pi.uniform_plasma(n=args.grid, ppc=ppc, seed=1004, dt=args.dt)
    elif args.workload == "penning":
        w = pi.penning(n=args.grid, n_particles=n_particles, seed=1002, dt=args.dt)
    else:
        w = pi.landau(n=args.grid, ppc=ppc, seed=1001, dt=args.dt)
    if w.n_particles > n_particles:
        w.x = w.x[:n_particles].copy()
        w.v = w.v[:n_particles].copy()
    return w


def time_oracle(w, steps, warmup=0, uniform=False):
    from oracle import pic_oracle as po

    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q, B=w.B, wz2=w.wz2)

    def one(x, v, n, diag):
        if uniform:
            out = po.step_uniform(x, v, g, p, n, 2022, with_diag=diag)
        else:
            out = po.step(x, v, g, p, with_diag=diag)
        return out[0], out[1]

    x, v = w.x, w.v
    for n in range(warmup):
        x, v = one(x, v, n, False)
    t0 = time.perf_counter()
    for n in range(steps):
        x, v = one(x, v, warmup + n, True)
    dt = time.perf_counter() - t0
    return w.n_particles * steps / dt, dt


# The all-core oracle figure: the oracle's own functions (deposit, solve_field,
# gather, boris_kick, wrap, in the order of its step) driven over particle
# chunks by a process pool; the chunks' density grids are summed in a fixed
# order and the field solve runs once per step in the parent process.
_ORC = {}


def _orc_init(shm_names, shapes, grid_n, grid_L, params):
    from multiprocessing import shared_memory

    import numpy as np

    from oracle import pic_oracle as po

    _ORC["shm"] = [shared_memory.SharedMemory(name=nm) for nm in shm_names]
    _ORC["arr"] = [np.ndarray(sh, dtype=np.float64, buffer=s.buf)
                   for s, sh in zip(_ORC["shm"], shapes)]
    _ORC["grid"] = po.Grid(grid_n, grid_L)
    _ORC["params"] = po.Params(**params)


def _orc_deposit(job):
    from oracle import pic_oracle as po

    i, s, e, N = job
    x, v, xh, rho_parts, _ = _ORC["arr"]
    g, p = _ORC["grid"], _ORC["params"]
    xh[s:e] = po.wrap(x[s:e] + 0.5 * p.dt * v[s:e], g)
    rho_parts[i] = po.deposit(xh[s:e], g, p.Q / N).ravel()
    return i


def _orc_push(job):
    import numpy as np

    from oracle import pic_oracle as po

    i, s, e, N = job
    x, v, xh, _, E = _ORC["arr"]
    g, p = _ORC["grid"], _ORC["params"]
    e_p = po.gather(xh[s:e], E.reshape((3,) + g.shape), g)
    if p.wz2 != 0.0:
        e_p = e_p + po.external_field(xh[s:e], g, p.wz2)
    v1 = po.boris_kick(v[s:e], e_p, p.q_over_m, p.B, p.dt)
    x[s:e] = po.wrap(xh[s:e] + 0.5 * p.dt * v1, g)
    v[s:e] = v1
    return np.concatenate([v1.sum(axis=0), [float(np.sum(v1 * v1))]])


def time_oracle_parallel(w, steps, workers, return_state=False):
    """Particle-steps/s of the oracle over `workers` processes (spawned);
    with return_state, also the final (x, v)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np

    from oracle import pic_oracle as po

    N = w.n_particles
    g = po.Grid(w.n, w.L)
    chunks = max(1, workers)
    shapes = [(N, 3), (N, 3), (N, 3), (chunks, g.n_nodes), (3 * g.n_nodes,)]
    shms, arrs = [], []
    try:
        for sh in shapes:
            s = shared_memory.SharedMemory(create=True, size=int(np.prod(sh)) * 8)
            shms.append(s)
            arrs.append(np.ndarray(sh, dtype=np.float64, buffer=s.buf))
        arrs[0][:] = w.x
        arrs[1][:] = w.v
        params = dict(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q, B=tuple(w.B), wz2=w.wz2)
        bounds = np.linspace(0, N, chunks + 1).astype(np.int64)
        jobs = [(i, int(bounds[i]), int(bounds[i + 1]), N) for i in range(chunks)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_orc_init,
                      initargs=([s.name for s in shms], shapes, w.n, w.L, params)) as pool:
            pool.map(_orc_deposit, jobs[:1])          # workers up (imports done)
            t0 = time.perf_counter()
            for _ in range(steps):
                list(pool.map(_orc_deposit, jobs))
                rho = np.zeros(g.n_nodes)
                for i in range(chunks):               # fixed-order sum of the chunk grids
                    rho += arrs[3][i]
                arrs[4][:] = po.solve_field(rho.reshape(g.shape), g).ravel()
                moments = pool.map(_orc_push, jobs)
                _ = np.sum(moments, axis=0)
            secs = time.perf_counter() - t0
        state = (arrs[0].copy(), arrs[1].copy()) if return_state else None
    finally:
        del arrs
        for s in shms:
            s.close()
            s.unlink()
    if return_state:
        return N * steps / secs, secs, state
    return N * steps / secs, secs


def cpu_baseline_figures(args, steps=2):
    """Single-thread and all-core oracle throughput on a bounded sample of the
    workload, with the core count of this host."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ws = oracle_sample(args, args.cpu_sample)
    one, secs1 = time_oracle(ws, steps, uniform=args.workload == "uniform")
    out = {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{ws.n_particles:,} particles of the workload on the full {args.grid}^3 "
                     f"grid, {steps} oracle steps ({secs1:.1f} s, numpy FP64, single thread)",
           "host_cores": cores}
    if cores > 1 and args.workload != "uniform":
        try:
            allc, secs_a = time_oracle_parallel(ws, steps, cores)
            out["all_cores"] = {"value": allc, "unit": UNIT, "cores": cores,
                                "sample": f"the same sample and steps ({secs_a:.1f} s) over "
                                          f"{cores} spawned processes, one particle chunk each; "
                                          f"chunk grids summed in a fixed order, the FFT solve "
                                          f"in the parent"}
        except Exception as e:   # pragma: no cover - hosts without shared memory
            out["all_cores"] = {"unavailable": str(e)[:200]}
    if getattr(args, "cpu_configs", True):
        out["configs"] = cpu_config_figures(cores)
        out["configs_unit"] = UNIT
    return out


# The survey's configurations for the CPU oracle: the small Landau case, the
# Landau and Penning cases reduced to a 2M-particle sample, and the adjoint's
# bump-on-tail case at full size (name, workload factory, timed steps).
CPU_CONFIGS = [
    ("landau 16^3 x 8 particles/cell (32,768 particles)",
     lambda pi: pi.landau(n=16, ppc=8, seed=1000), 5),
    ("landau 32^3 x 64 particles/cell (2,097,152 particles)",
     lambda pi: pi.landau(n=32, ppc=64, seed=1001), 1),
    ("penning 64^3, 2,097,152 particles",
     lambda pi: pi.penning(n=64, n_particles=1 << 21, seed=1002), 1),
    ("bump-on-tail 64^3 x 16 particles/cell (4,194,304 particles)",
     lambda pi: pi.bump_on_tail(n=64, ppc=16, seed=1003), 1),
]


def cpu_config_figures(cores, configs=None):
    """Single-thread and all-core oracle throughput (particle-steps/s) on each
    configuration of `configs` (default CPU_CONFIGS)."""
    import pic_inputs as pi

    out = []
    for name, make, steps in (configs or CPU_CONFIGS):
        w = make(pi)
        one, secs1 = time_oracle(w, steps)
        ent = {"config": name, "steps": steps, "single": one, "single_s": round(secs1, 2)}
        if cores > 1:
            try:
                allc, secs_a = time_oracle_parallel(w, steps, cores)
                ent.update({"all_cores": allc, "all_cores_s": round(secs_a, 2)})
            except Exception as e:   # pragma: no cover - hosts without shared memory
                ent["all_cores"] = None
                ent["all_cores_unavailable"] = str(e)[:200]
        out.append(ent)
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    w = oracle_sample(args, args.cpu_sample)
    val, secs = time_oracle(w, args.steps, args.warmup, uniform=args.workload == "uniform")
    sample = (f"{w.n_particles:,} particles of the workload on the full {args.grid}^3 grid, "
              f"{args.steps} oracle steps (numpy FP64, single thread)")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(args)},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample,
                         "host_cores": len(os.sched_getaffinity(0))
                         if hasattr(os, "sched_getaffinity") else os.cpu_count()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- adjoint

def measure_adjoint(n_steps=200, K=20, launch=None):
    """Cost of the discrete adjoint against the forward step on the
    bump-on-tail workload (64^3 grid, 16 particles per cell, 200 steps).

    Device time of pic_step (the forward step), and of pic_adjoint_forward /
    pic_adjoint_backward twice: with checkpoints every K steps (the backward
    pass recomputes each segment, then reverses it) and with the whole
    trajectory kept in device memory (K = n_steps - 1: the backward pass is
    the reverse sweep alone, so its cost per step is the adjoint step)."""
    import torch

    import pic_inputs as pi
    from paper_2205_11052_gb300.sim import Simulation

    launch = dict(LAUNCH if launch is None else launch)
    w = pi.by_name("bump_on_tail_64")
    sim = Simulation.from_workload(w, **launch)
    st = sim.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    sim.step(5)                              # warm-up, then back to the loaded state
    sim.load(w.x, w.v)
    torch.cuda.synchronize()
    ev[0].record(st)
    sim.step(n_steps)
    ev[1].record(st)
    torch.cuda.synchronize()
    fwd_ms = ev[0].elapsed_time(ev[1]) / n_steps
    out = {"workload": f"bump-on-tail 64^3 x 16 particles/cell ({w.n_particles:,} particles), "
                       f"{n_steps} steps, objective W_z of the last field",
           "forward_ms_per_step": fwd_ms}
    for key, kk in (("checkpoints", K), ("kept_trajectory", n_steps - 1)):
        sim.load(w.x, w.v)
        sim.adjoint_forward(n_steps, (0.0, 0.0, 1.0), checkpoint_every=kk)     # warm-up
        sim.adjoint_backward(device=True)
        torch.cuda.synchronize()
        ev[0].record(st)
        J = sim.adjoint_forward(n_steps, (0.0, 0.0, 1.0), checkpoint_every=kk)
        ev[1].record(st)
        ev[2].record(st)
        gx, gv = sim.adjoint_backward(device=True)
        ev[3].record(st)
        torch.cuda.synchronize()
        af_ms = ev[0].elapsed_time(ev[1]) / n_steps
        ab_ms = ev[2].elapsed_time(ev[3]) / n_steps
        out[key] = {"checkpoint_every": kk,
                    "buffer_gb": round(sim._adj_buf.numel() / 1e9, 2),
                    "adjoint_forward_ms_per_step": af_ms,
                    "adjoint_backward_ms_per_step": ab_ms,
                    "backward_over_forward": ab_ms / fwd_ms,
                    "gradient_over_forward": (af_ms + ab_ms) / fwd_ms,
                    "J": J,
                    "finite": bool(torch.isfinite(gx).all().item() and
                                   torch.isfinite(gv).all().item())}
        sim._adj_buf = None
        torch.cuda.empty_cache()
    # headline: the backward pass with checkpoints every K steps (segment
    # recomputation included) against the forward step
    out["adjoint_step_over_forward"] = out["checkpoints"]["backward_over_forward"]
    out["adjoint_step_over_forward_kept_trajectory"] = out["kept_trajectory"]["backward_over_forward"]
    # dJ/dalpha = <dJ/dx0, dx0/dalpha> (FP64 dot on the device); the sample
    # map's Jacobian comes from the input generator
    sim.load(w.x, w.v)
    sim.adjoint_forward(n_steps, (0.0, 0.0, 1.0), checkpoint_every=K)
    gx, _ = sim.adjoint_backward(device=True)
    dxa = torch.zeros_like(gx)
    dxa[:, 2] = torch.from_numpy(pi.sample_cosine_density_dalpha(
        w.x[:, 2], w.meta["alpha"], w.meta["k"])).to(gx.device)
    out["dJ_dalpha"] = sim.dot(gx, dxa)
    sim._adj_buf = None
    sim.close()
    return out


# ---------------------------------------------------------------- ensemble

def ensemble_members(count, seed=1_000_000):
    """Landau-damping instances: grids U{16,24,32,48}^3, 8..64 particles per
    cell, alpha U[0.01, 0.1], independent seeds (seed + i)."""
    import numpy as np

    import pic_inputs as pi

    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([16, 24, 32, 48]))
        ppc = int(rng.integers(8, 65))
        alpha = float(rng.uniform(0.01, 0.1))
        out.append((n, ppc, alpha, seed + i))
    # instances are independent (each from its own seed): draw them in parallel
    import concurrent.futures as cf

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        members = list(ex.map(lambda a: pi.landau(n=a[0], ppc=a[1], alpha=a[2], seed=a[3],
                                                  chunk=1 << 18), out))
    return members


# the autotuner's choice for the 512-instance ensemble on a GB300
# (profiles/ensemble512_bench.md), used when the default run times it
ENSEMBLE_TUNED = dict(tile=(8, 8, 8), block=256, sort_period=4, options=1)


def measure_ensemble(count, steps, warmup, tune=True, sort_period=4, options=1):
    """Batched ensemble vs the same instances stepped (a) one launch sequence
    per instance and (b) one CUDA graph per instance, all timed on the device
    over the same steps.  Returns the measurement as a dict."""
    import torch

    from paper_2205_11052_gb300 import capi
    from paper_2205_11052_gb300.batch import Ensemble
    from paper_2205_11052_gb300.sim import Simulation

    t0 = time.perf_counter()
    ws = ensemble_members(count)
    gen_s = time.perf_counter() - t0
    N = sum(w.n_particles for w in ws)
    opts = dict(sort_period=sort_period, options=options)
    members = [(w.n, w.L, w.x, w.v, w.Q) for w in ws]
    tuned = None
    if tune:
        from paper_2205_11052_gb300.autotune import tune_ensemble

        t1 = time.perf_counter()
        best, table = tune_ensemble(members, 0.05, space={"tile": [(8, 8, 8), (4, 4, 4)],
                                                          "block": [128, 256],
                                                          "sort_period": [2, 4], "options": [1]})
        opts = {k: tuple(v) if isinstance(v, list) else v for k, v in best.items()}
        tuned = {"best": best, "table": table, "seconds": round(time.perf_counter() - t1, 1)}
    else:
        opts = dict(ENSEMBLE_TUNED)
    ens = Ensemble(members, dt=0.05, **opts)
    # all instances, all K steps: one CUDA graph, replayed once per timing
    graph = ens.capture(steps)
    for _ in range(max(1, warmup // max(1, steps))):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    rs = torch.cuda.current_stream()
    e0.record(rs)
    graph.replay()
    e1.record(rs)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_batch = e0.elapsed_time(e1)
    del graph
    ens.close()
    del ens
    torch.cuda.empty_cache()
    single_opts = {k: v for k, v in opts.items() if k != "block"}
    sims = [Simulation.from_workload(w, **single_opts) for w in ws]
    for s in sims:
        s.step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(steps):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    # (b) one CUDA graph of all the steps per instance, replayed one after the other
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    graphs = []
    for s in sims:
        capi.pic_set_stream(s.handle, gs.cuda_stream)
        with torch.cuda.stream(gs):
            s.step(1)
        gs.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            s.step(steps)
        graphs.append(g)
    torch.cuda.synchronize()
    e0.record(stream)
    for g in graphs:
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graphs = e0.elapsed_time(e1)
    del graphs
    for s in sims:
        s.close()
    torch.cuda.empty_cache()
    return {
        "workload": f"ensemble of {len(ws)} Landau instances, grids U{{16,24,32,48}}^3, "
                    f"8-64 particles/cell, alpha U[0.01,0.1], {N:,} particles; {steps} batched "
                    f"steps captured in one CUDA graph",
        "value": N * steps / (ms_batch * 1e-3), "unit": UNIT, "ms_per_step": ms_batch / steps,
        "steps": steps, "warmup": warmup, "generation_s": round(gen_s, 1),
        "config": {k: list(v) if isinstance(v, tuple) else v for k, v in opts.items()},
        "per_instance_launches": {"value": N * steps / (ms_single * 1e-3),
                                  "ms_per_step": ms_single / steps},
        "per_instance_graphs": {"value": N * steps / (ms_graphs * 1e-3),
                                "ms_per_step": ms_graphs / steps,
                                "what": f"one CUDA graph of {steps} steps per instance, the "
                                        f"{len(ws)} graphs replayed in turn"},
        "autotune": tuned,
        "speedup": ms_single / ms_batch,
        "speedup_vs_graphs": ms_graphs / ms_batch,
        "clocks": clk,
    }


def run_ensemble(args):
    """The batched-ensemble line (`--workload ensemble`)."""
    from paper_2205_11052_gb300.build import build

    build()
    m = measure_ensemble(args.ens_count, args.steps, args.warmup, tune=not args.no_tune,
                         sort_period=args.sort_period, options=args.options)
    line = {
        "metric": "ensemble particle-steps/s (batched launch vs one launch sequence per instance)",
        "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload=m["workload"], generation_s=m["generation_s"], **m["config"]),
        **{k: m[k] for k in ("per_instance_launches", "per_instance_graphs", "autotune",
                             "speedup", "speedup_vs_graphs", "clocks")},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- side lines

def timed_steps(sim, steps, gpu_index=0):
    """Device time of `steps` pic_step calls with the phase timers on and the
    SM clocks sampled; returns (ms, phases, launches, clocks)."""
    import torch

    from paper_2205_11052_gb300 import capi

    capi.pic_enable_timers(sim.handle, True)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    for _ in range(steps):
        sim.step(1)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    phases, launches = capi.pic_read_timers(sim.handle)
    capi.pic_enable_timers(sim.handle, False)
    return ev0.elapsed_time(ev1), phases, launches, clk


def push_roofline(phases, N, ng, peak, peak_kind):
    """The fused push + deposit kernel against HBM: 56 B per particle (state
    read and written once) + 20 B per node (E read, rho written)."""
    avg_ms = phases["push"][0] / max(1, phases["push"][1])
    achieved = (56.0 * N + 20.0 * ng) / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "k_push_deposit", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
            "ms_per_launch": avg_ms}


def deposit_roofline(sim, N, ng, peak, peak_kind, launches=3):
    """The split-call deposit kernel (k_deposit_tiles) at full size, right
    after a re-binning: 16 B per particle (cell + offsets read) + 4 B per node."""
    import torch

    from paper_2205_11052_gb300 import capi

    sim.sort()
    sim.deposit()                       # warm-up
    torch.cuda.synchronize()
    capi.pic_enable_timers(sim.handle, True)
    for _ in range(launches):
        sim.deposit()
    torch.cuda.synchronize()
    phases, _ = capi.pic_read_timers(sim.handle)
    capi.pic_enable_timers(sim.handle, False)
    avg_ms = phases["deposit"][0] / max(1, phases["deposit"][1])
    achieved = (16.0 * N + 4.0 * ng) / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "k_deposit_tiles", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
            "ms_per_launch": avg_ms, "particles_per_s": N / (avg_ms * 1e-3),
            "what": f"pic_deposit (split call, fixed point) right after a re-binning, mean of "
                    f"{launches} launches; 16 B per particle + 4 B per node"}


def side_line(x, v, w_like, opts, warmup, steps, peak, peak_kind, ng, what):
    """One more configuration on the same GPU: load, warm up, time `steps`."""
    import torch

    from paper_2205_11052_gb300.sim import Simulation

    sim = Simulation(n=w_like.n, L=w_like.L, n_particles=x.shape[0], dt=w_like.dt,
                     q_over_m=w_like.q_over_m, Q=w_like.Q, B=w_like.B, wz2=w_like.wz2,
                     mode=w_like.mode, mode_comp=w_like.mode_comp, **opts)
    sim.load(x, v)
    sim.step(warmup)
    torch.cuda.synchronize()
    r0, _ = sim.rebin_stats()
    ms, phases, launches, clk = timed_steps(sim, steps)
    r1, _ = sim.rebin_stats()
    hist = sim.diagnostics()
    flags = sim.flags()
    N = x.shape[0]
    out = {"workload": what, "value": N * steps / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
           "config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in opts.items()},
           "phases_ms": {k: round(p[0] / max(1, p[1]), 4) for k, p in phases.items()},
           "roofline": push_roofline(phases, N, ng, peak, peak_kind),
           "rebins": r1 - r0, "gpu_launches": launches, "clocks": clk, "device_flags": flags,
           "diag_last": {k: hist[-1][k] for k in ("step", "Wx", "Wz", "Q", "K")} if hist else None}
    sim.close()
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- particle sharding

def run_sharded(args, dist, rank, world):
    """One Landau run with its particles split over the ranks: per step each
    rank deposits its share (pic_deposit), an all-reduce sums rho, and each
    rank solves and pushes (pic_field_solve, pic_gather_push).  Total work is
    fixed, so this is strong scaling."""
    import torch

    import pic_inputs as pi
    from paper_2205_11052_gb300.shard import sharded_simulation

    w = pi.landau(n=args.grid, ppc=args.ppc, seed=1001, n_steps=args.steps, dt=args.dt)
    N = w.n_particles
    sim, stepper, (s0, s1) = sharded_simulation(
        w, rank, world, dist if world > 1 else None, sort_period=args.sort_period,
        options=args.options, guard=args.guard, diag_every=0)
    del w
    stepper.step(args.warmup)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    stepper.step(args.steps)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    flags = sim.flags()
    sim.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": N * args.steps / (ms * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), "n_particles": N,
                       "parallelism": f"particles split over {world} rank(s); rho summed by an "
                                      f"all-reduce every step; field solved on every rank",
                       "path": "split calls: pic_deposit, all-reduce, pic_set_rho, "
                               "pic_field_solve, pic_gather_push",
                       "l2": "inputs larger than L2, no flush"},
            "clocks": clk, "device_flags": flags}), flush=True)


# ---------------------------------------------------------------- native arm

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.record_traffic:
        record_traffic(args.record_traffic)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "ensemble":
        run_ensemble(args)
        return
    if args.workload == "adjoint":
        from paper_2205_11052_gb300.build import build

        build()
        print(json.dumps(measure_adjoint(n_steps=args.adjoint_steps)), flush=True)
        return

    import numpy as np
    import torch

    import pic_inputs as pi
    from paper_2205_11052_gb300 import capi
    from paper_2205_11052_gb300.build import build
    from paper_2205_11052_gb300.sim import Simulation

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build()
    if args.shard == "particles":
        run_sharded(args, dist, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- inputs: seeded synthetic Landau damping (per-rank seed offset)
    options = args.options
    if args.workload == "penning":
        w = pi.penning(n=args.grid, seed=1002 + rank, dt=args.dt)
    elif args.workload == "uniform":
        w = pi.uniform_plasma(n=args.grid, ppc=args.ppc, seed=1004 + rank, n_steps=args.steps,
                              dt=args.dt)
        options |= capi.PIC_OPT_UNIFORM_MOVE
    else:
        w = pi.landau(n=args.grid, ppc=args.ppc, seed=1001 + rank, n_steps=args.steps, dt=args.dt)
    N = w.n_particles
    ng = args.grid ** 3
    sim = Simulation.from_workload(w, sort_period=args.sort_period, options=options,
                                   diag_every=args.diag_every, guard=args.guard, seed=2022 + rank,
                                   stray_rebin=args.stray_rebin, tile=(args.tile,) * 3)
    stream = sim.stream

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- warm-up
    sim.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K steps, timers on, clocks sampled
    rebins0, _ = sim.rebin_stats()
    capi.pic_enable_timers(sim.handle, True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    phases, launches = capi.pic_read_timers(sim.handle)
    capi.pic_enable_timers(sim.handle, False)
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(N, world, args.steps, ms * 1e-3)

    hist = sim.diagnostics()
    flags = sim.flags()
    rebins = sim.rebin_stats()[0] - rebins0

    # ---- roofline of the dominant kernel (CUDA events inside the timed region)
    peak, peak_kind = load_peaks()
    # fused gather + push + deposit: particle store read and written once (56 B
    # per particle), E read once (16 B per node), rho written once (4 B per node)
    algo = {"push": 56.0 * N + 20.0 * ng, "deposit": 16.0 * N + 4.0 * ng}
    kernel_names = {"push": "k_push_deposit", "deposit": "k_deposit_tiles"}
    if args.workload == "uniform":
        # random move + deposit: cell, offsets and pid read, cell and offsets
        # written (36 B), velocities read for the moments when diagnostics run
        algo["push"] = (48.0 if args.diag_every > 0 else 36.0) * N + 4.0 * ng
        kernel_names["push"] = "k_move_deposit"
    dom = max(algo, key=lambda k: phases[k][0])
    avg_ms = phases[dom][0] / max(1, phases[dom][1])
    achieved = algo[dom] / (avg_ms * 1e-3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        try:
            with open(tp) as f:
                tj = json.load(f)
            ent = tj.get(kernel_names[dom])
            # the record is for the 128^3 x 64 workload in the default launch configuration
            same = (args.workload, args.grid, args.ppc, args.sort_period, args.options, args.guard,
                    args.dt, args.tile) == ("landau", 128, 64, LAUNCH["sort_period"],
                                            LAUNCH["options"], 0, 0.05, 0)
            if same and ent and ent.get("source_sha") == _source_sha(ent.get("source")):
                traffic = ent["bytes_per_launch_full_size"]
        except Exception:
            traffic = None
    roof = {"bound": "hbm", "kernel": kernel_names[dom], "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{peak_kind} hbm_gbs"}
    phase_ms = {k: (v[0] / max(1, v[1]), v[1]) for k, v in phases.items()}

    # ---- the split-call deposit kernel at full size (its own roofline line)
    roof_dep = None
    if rank == 0 and not args.no_extras and args.workload == "landau":
        roof_dep = deposit_roofline(sim, N, ng, peak, peak_kind)

    # ---- end-to-end through the C ABI with pinned host buffers
    e2e = None
    xh = vh = None
    if not args.no_e2e and args.e2e_steps > 0:
        xh = torch.from_numpy(w.x).pin_memory()
        vh = torch.from_numpy(w.v).pin_memory()
        diag_buf = (capi.pic_diag_t * 1)()
        import ctypes as C
        lib = capi.load_library()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            capi.pic_load_particles(sim.handle, xh.data_ptr(), vh.data_ptr(), N, False)
            sim.step(1)
            n_out = C.c_int()
            rc = lib.pic_diagnostics(sim.handle, diag_buf, 1, C.byref(n_out))
            capi.check(rc, "pic_diagnostics")
        torch.cuda.synchronize()
        barrier()
        secs = time.perf_counter() - t0
        secs = max_over_ranks(secs, dist, "cuda")
        e2e = {"value": job_throughput(N, world, args.e2e_steps, secs), "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * 8 + vh.numel() * 8),
               "d2h_bytes_per_step": C.sizeof(capi.pic_diag_t),
               "what": "per step: pic_load_particles from pinned host FP64 (x, v), "
                       "pic_step(1), pic_diagnostics readback"}

    # ---- side lines on the same GPU: the FP32 tile-accumulation deposit on
    # this workload, the Penning-trap bunch (256^3, 1.3e8 particles) and the
    # 512-instance batched ensemble
    fp32_line = penning_line = ens_line = None
    if (rank == 0 and world == 1 and not args.no_extras and not args.no_side_lines
            and args.workload == "landau"):
        sim.close()
        sim = None
        torch.cuda.empty_cache()
        if xh is None:
            xh, vh = w.x, w.v
        opts = dict(sort_period=args.sort_period, options=args.options & ~capi.PIC_OPT_FIXED_DEPOSIT,
                    diag_every=args.diag_every, guard=args.guard)
        fp32_line = side_line(xh, vh, w, opts, 3, args.side_steps, peak, peak_kind, ng,
                              workload_name(args) + "; FP32 tile accumulation (float shared "
                              "atomics, float grid atomics)")
        del xh, vh, w
        wp = pi.penning(n=256, seed=1002, dt=0.05)
        popts = dict(sort_period=2, guard=3, options=capi.PIC_OPT_FIXED_DEPOSIT,
                     diag_every=args.diag_every)
        penning_line = side_line(wp.x, wp.v, wp, popts, 3, args.side_steps, peak, peak_kind,
                                 256 ** 3,
                                 "penning_trap_3d: 256^3 grid on [0,20)^3, 130,000,000 particles "
                                 "in a Gaussian bunch sigma=(1,1,2), Bz=5, axial frequency 1, "
                                 f"Q=-1562.5, dt=0.05; {args.side_steps} of its 100 steps")
        del wp
        # the 512-instance batched ensemble, its configured 100 steps in one graph
        # (the autotuner's setting, fixed), against per-instance launches and graphs
        ens_line = measure_ensemble(args.ens_count, 100, 3, tune=False)

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_figures(args)

    # ---- adjoint step cost against the forward step (bump-on-tail, 64^3)
    adj = None
    if rank == 0 and not args.no_adjoint:
        if sim is not None:
            sim.close()
            sim = None
        torch.cuda.empty_cache()
        adj = measure_adjoint()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "n_particles": N,
                       "grid": [args.grid] * 3, "sort_period": args.sort_period,
                       "tile": [args.tile or 8] * 3, "guard": args.guard or 2,
                       "deposit": "fixed-point" if args.options & 1 else "fp32",
                       "diag_every": args.diag_every,
                       "l2": f"inputs larger than L2 ({32 * N / 1e9:.2f} GB particle store "
                             f"vs {L2_BYTES / 2**20:.0f} MiB L2), no flush",
                       "parallelism": "replicas" if world > 1 else "single-gpu"},
            "roofline": roof,
            "roofline_deposit": roof_dep,
            "phases_ms": {k: round(v[0], 4) for k, v in phase_ms.items()},
            "rebins": rebins,
            "fp32_deposit": fp32_line,
            "penning": penning_line,
            "ensemble": ens_line,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "adjoint": adj,
            "gpu_launches": launches,
            "clocks": clk,
            "device_flags": flags,
            "diag_last": {k: hist[-1][k] for k in ("step", "Wx", "Q", "K")} if hist else None,
        }
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if dist is not None:
        dist.destroy_process_group()


TRAFFIC_SOURCES = ["paper_2205_11052_gb300/csrc/k_particles.cu",
                   "paper_2205_11052_gb300/csrc/push.cuh",
                   "paper_2205_11052_gb300/csrc/cic.cuh",
                   "paper_2205_11052_gb300/csrc/pic_internal.cuh"]


def record_traffic(csv_path, small_particles=64 ** 3 * 64, small_nodes=64 ** 3,
                   full_particles=128 ** 3 * 64, full_nodes=128 ** 3):
    """DRAM bytes of one k_push_deposit launch from an ncu CSV of the 64^3 x 64
    case, scaled to the 128^3 x 64 launch by the particle ratio (the kernel's
    traffic is proportional to particles and nodes, both x8), into
    profiles/traffic.json with the hash of the kernel's sources."""
    import csv

    with open(csv_path) as f:
        rows = [r for r in csv.reader(f)]
    hi = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    h = rows[hi]
    ki, mi, ui, vi = (h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Unit"),
                      h.index("Metric Value"))
    unit = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    for r in rows[hi + 1:]:
        if len(r) > vi and "k_push_deposit" in r[ki] and r[mi].startswith("dram__bytes_"):
            per.setdefault(r[mi], []).append(float(r[vi].replace(",", "")) * unit[r[ui]])
    small = sum(v[0] for v in per.values())
    scale = full_particles / small_particles
    assert abs(full_nodes / small_nodes - scale) < 1e-12
    out = {"k_push_deposit": {
        "source": TRAFFIC_SOURCES, "source_sha": _source_sha(TRAFFIC_SOURCES),
        "bytes_per_launch_small": small,
        "small_case": "landau 64^3 x 64 ppc (16,777,216 particles), sort period 4, fixed-point deposit",
        "scale": scale, "bytes_per_launch_full_size": small * scale,
        "note": "dram__bytes_read.sum + dram__bytes_write.sum of one launch, scaled by the "
                "particle (and node) ratio to the 128^3 x 64 workload"}}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


def _source_sha(rels):
    """Hash of the kernel's source files: the traffic figure is void once they change."""
    import hashlib

    if not rels:
        return None
    h = hashlib.sha256()
    for rel in ([rels] if isinstance(rels, str) else rels):
        p = os.path.join(ROOT, rel)
        if not os.path.exists(p):
            return None
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
