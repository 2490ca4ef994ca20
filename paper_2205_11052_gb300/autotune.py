"""Autotuner for the launch configuration of the PIC step.

Times a few candidate settings of the tuning knobs of ``pic_params_t`` --
deposit tile, guard layers, re-binning period, deposit accumulator, and for
ensembles the thread-block size of the batched push -- on the
caller's own particles with CUDA events (a few warm-up steps, then a few
timed steps each) and returns the fastest.  Results are cached by the shape
of the workload (grid, particles per cell, external fields), in memory and
optionally in a JSON file.  ``tune_ensemble`` does the same for a batched
ensemble, timing the whole ensemble per candidate.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np

DEFAULT_SPACE = {
    "tile": [(8, 8, 8), (4, 4, 4)],
    "guard": [2, 1],
    "sort_period": [2, 4, 8],
    "options": [1, 0],
}


def workload_key(n, n_particles, B=(0.0, 0.0, 0.0), wz2=0.0) -> str:
    n = tuple(int(a) for a in n)
    ppc = n_particles / float(np.prod(n))
    bucket = int(2 ** round(np.log2(max(ppc, 1.0))))
    return f"{n[0]}x{n[1]}x{n[2]}|ppc~{bucket}|B{int(any(B))}|E{int(wz2 != 0.0)}"


class Autotuner:
    def __init__(self, space=None, warmup=2, steps=4, cache_path=None):
        self.space = dict(DEFAULT_SPACE if space is None else space)
        self.warmup = int(warmup)
        self.steps = int(steps)
        self.cache_path = cache_path
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def candidates(self, n):
        keys = sorted(self.space)
        for combo in itertools.product(*(self.space[k] for k in keys)):
            cfg = dict(zip(keys, combo))
            if "tile" in cfg:
                cfg["tile"] = tuple(min(int(t), int(m)) for t, m in zip(cfg["tile"], n))
            yield cfg

    def time_config(self, w, cfg) -> float:
        """Milliseconds per step of `cfg` on workload `w` (device-timed)."""
        import torch

        from .sim import Simulation

        sim = Simulation.from_workload(w, **cfg)
        try:
            sim.step(self.warmup)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sim.stream)
            sim.step(self.steps)
            e1.record(sim.stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / self.steps
        finally:
            sim.close()

    def tune(self, w, force=False):
        """Best configuration for workload `w` (a pic_inputs.Workload-like object)."""
        key = workload_key(w.n, w.n_particles, w.B, w.wz2)
        if key in self.cache and not force:
            return self.cache[key]["best"]
        table = []
        for cfg in self.candidates(w.n):
            ms = self.time_config(w, cfg)
            table.append({"cfg": {k: list(v) if isinstance(v, tuple) else v for k, v in cfg.items()},
                          "ms_per_step": ms})
        table.sort(key=lambda r: r["ms_per_step"])
        best = table[0]["cfg"]
        self.cache[key] = {"best": best, "table": table}
        if self.cache_path:
            os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1)
        return best


ENSEMBLE_SPACE = {
    "tile": [(8, 8, 8), (4, 4, 4), (8, 8, 4)],
    "block": [128, 256],
    "sort_period": [2, 4],
    "options": [1, 0],
}


def ensemble_key(members) -> str:
    """Cache key of an ensemble: its sorted (grid, particles-per-cell bucket) mix."""
    parts = sorted(workload_key(n, np.asarray(x).shape[0]) for n, L, x, v, Q in members)
    return "ens|" + ";".join(f"{p}x{parts.count(p)}" for p in sorted(set(parts)))


def tune_ensemble(members, dt, space=None, warmup=2, steps=4, cache=None, **fixed):
    """Fastest ensemble setting among the candidates of `space` (a dict of
    lists over tile / block / sort_period / options / guard), each timed on the
    device over `steps` steps of the whole ensemble after `warmup` steps.
    Returns (best setting, table of (setting, ms per step))."""
    import torch

    from .batch import Ensemble

    space = dict(ENSEMBLE_SPACE if space is None else space)
    key = ensemble_key(members)
    if cache is not None and key in cache:
        return cache[key]["best"], cache[key]["table"]
    nmin = min(min(int(a) for a in (n if np.ndim(n) else (n, n, n))) for n, *_ in members)
    keys = sorted(space)
    table = []
    for combo in itertools.product(*(space[k] for k in keys)):
        cfg = dict(zip(keys, combo))
        if "tile" in cfg:
            cfg["tile"] = tuple(min(int(t), nmin) for t in cfg["tile"])
        ens = Ensemble(members, dt=dt, **fixed, **cfg)
        try:
            ens.step(warmup)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ens.stream)
            ens.step(steps)
            e1.record(ens.stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
        finally:
            ens.close()
            del ens
            torch.cuda.empty_cache()
        table.append(({k: list(v) if isinstance(v, tuple) else v for k, v in cfg.items()}, ms))
    table.sort(key=lambda r: r[1])
    best = table[0][0]
    if cache is not None:
        cache[key] = {"best": best, "table": table}
    return best, table
