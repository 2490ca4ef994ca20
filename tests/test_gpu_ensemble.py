"""Batched ensembles vs independent oracle runs of every instance (GPU).

Instances differ in grid (including non-cubic and tile-ragged ones),
particle count, perturbation and charge; each must follow its own oracle
trajectory to the tolerances of the single-run parity tests.
"""
import numpy as np
import pytest

import pic_inputs as pi
from oracle import pic_oracle as po

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2205_11052_gb300 import capi  # noqa: E402
from paper_2205_11052_gb300.batch import Ensemble  # noqa: E402
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()


def _members():
    ws = [pi.landau(n=8, ppc=4, seed=41, alpha=0.1),
          pi.landau(n=12, ppc=3, seed=42, alpha=0.05),
          pi.landau(n=16, ppc=2, seed=43, alpha=0.08),
          pi.landau(n=16, ppc=5, seed=44, alpha=0.02),
          pi.uniform_plasma(n=(10, 8, 6), ppc=3, L=(2.0, 1.5, 1.0), seed=45)]
    return ws


def _pos_err(x, xo, w):
    L = np.asarray(w.L)
    d = x - xo
    d -= L * np.round(d / L)
    return np.max(np.abs(d) / (L / np.asarray(w.n)))


@pytest.mark.parametrize("options", [0, capi.PIC_OPT_FIXED_DEPOSIT], ids=["fp32", "fixed"])
def test_every_instance_follows_its_oracle(options):
    ws = _members()
    ens = Ensemble([(w.n, w.L, w.x, w.v, w.Q) for w in ws], dt=0.05, diag_every=1,
                   sort_period=2, options=options)
    ens.step(6)
    xs, vs = ens.particles()
    hist = ens.diagnostics()
    assert len(hist) == 6
    for i, w in enumerate(ws):
        g = po.Grid(w.n, w.L)
        p = po.Params(dt=0.05, Q=w.Q, q_over_m=w.q_over_m)
        xo, vo, ho = po.run(w.x, w.v, g, p, 6)
        assert _pos_err(xs[i], xo, w) <= 1e-4, i
        assert np.max(np.abs(vs[i] - vo)) <= 1e-4 * np.max(np.abs(vo)), i
        for r, ro in zip(hist, ho):
            assert r[i]["step"] == ro["step"]
            assert r[i]["Wx"] == pytest.approx(ro["Wx"], rel=1e-4)
            assert r[i]["K"] == pytest.approx(ro["K"], rel=1e-4)
            assert r[i]["Q"] == pytest.approx(ro["Q"], rel=1e-6)
    ens.close()


def test_ensemble_equals_single_runs_of_its_members():
    ws = _members()[:3]
    ens = Ensemble([(w.n, w.L, w.x, w.v, w.Q) for w in ws], dt=0.05, sort_period=1,
                   options=capi.PIC_OPT_FIXED_DEPOSIT)
    ens.step(4)
    xs, vs = ens.particles()
    for i, w in enumerate(ws):
        sim = Simulation.from_workload(w, sort_period=1, options=capi.PIC_OPT_FIXED_DEPOSIT)
        sim.step(4)
        x, v = sim.particles()
        assert _pos_err(xs[i], x, w) <= 1e-5
        assert np.max(np.abs(vs[i] - v)) <= 1e-5 * np.max(np.abs(v))
        sim.close()
    ens.close()


def test_ensemble_step_replays_from_a_cuda_graph():
    ws = _members()
    ens = Ensemble([(w.n, w.L, w.x, w.v, w.Q) for w in ws], dt=0.05, sort_period=2,
                   options=capi.PIC_OPT_FIXED_DEPOSIT)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    ens.set_stream(s)
    with torch.cuda.stream(s):
        ens.step(2)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ens.step(2)
    for _ in range(2):
        g.replay()               # on the current stream
    torch.cuda.synchronize()
    xs, vs = ens.particles()
    for i, w in enumerate(ws):
        xo, vo, _ = po.run(w.x, w.v, po.Grid(w.n, w.L), po.Params(dt=0.05, Q=w.Q), 6)
        assert _pos_err(xs[i], xo, w) <= 1e-4
        assert np.max(np.abs(vs[i] - vo)) <= 1e-4 * np.max(np.abs(vo))
    ens.close()


def test_autotuner_picks_the_fastest_measured_setting():
    from paper_2205_11052_gb300.autotune import Autotuner, tune_ensemble

    ws = _members()
    members = [(w.n, w.L, w.x, w.v, w.Q) for w in ws]
    cache = {}
    best, table = tune_ensemble(members, 0.05, space={"tile": [(8, 8, 8), (4, 4, 4)],
                                                      "sort_period": [2], "options": [1]},
                                warmup=1, steps=2, cache=cache)
    assert len(table) == 2 and best == table[0][0]
    assert table[0][1] <= table[1][1] and all(ms > 0 for _, ms in table)
    assert tune_ensemble(members, 0.05, cache=cache)[0] == best      # served from the cache
    tuner = Autotuner(space={"tile": [(8, 8, 8), (4, 4, 4)], "sort_period": [2], "options": [1]},
                      warmup=1, steps=2)
    cfg = tuner.tune(ws[0])
    assert cfg in [r["cfg"] for r in next(iter(tuner.cache.values()))["table"]]


@pytest.mark.parametrize("block", [128, 256])
def test_block_size_does_not_change_the_result(block):
    """The batched push's thread-block size is a tuning knob only: with the
    fixed-point deposit every block size gives the same bits."""
    ws = _members()
    out = []
    for blk in (block, 256):
        ens = Ensemble([(w.n, w.L, w.x, w.v, w.Q) for w in ws], dt=0.05, sort_period=2,
                       options=capi.PIC_OPT_FIXED_DEPOSIT, block=blk)
        ens.step(3)
        out.append(ens.particles())
        ens.close()
    for a, b in zip(out[0][0] + out[0][1], out[1][0] + out[1][1]):
        assert np.array_equal(a, b)


def test_sample_of_the_512_instance_ensemble_follows_the_oracle():
    """The 512-instance Landau ensemble of the benchmark (grids U{16,24,32,48}^3,
    8-64 particles per cell, alpha U[0.01, 0.1], seeds 10^6 + i) advanced
    by a captured CUDA graph with 128-thread blocks, 4^3 tiles and re-binning
    every 2 steps: one instance of each grid size, drawn with a fixed seed
    among the lighter ones, against its own oracle run."""
    import bench

    ws = bench.ensemble_members(512)
    ens = Ensemble([(w.n, w.L, w.x, w.v, w.Q) for w in ws], dt=0.05, diag_every=1,
                   tile=(4, 4, 4), sort_period=2, block=128,
                   options=capi.PIC_OPT_FIXED_DEPOSIT)
    g = ens.capture(3)            # one eager step, then the captured three
    g.replay()
    torch.cuda.synchronize()
    xs, vs = ens.particles()
    hist = ens.diagnostics()
    ens.close()
    rng = np.random.default_rng(2024)
    picks = []
    for n in (16, 24, 32, 48):
        cand = [i for i, w in enumerate(ws) if w.n[0] == n and w.n_particles <= 16 * n ** 3]
        picks.append(int(rng.choice(cand)))
    for i in picks:
        w = ws[i]
        gr = po.Grid(w.n, w.L)
        p = po.Params(dt=0.05, Q=w.Q, q_over_m=w.q_over_m)
        xo, vo, ho = po.run(w.x, w.v, gr, p, 4)
        assert _pos_err(xs[i], xo, w) <= 1e-4, i
        assert np.max(np.abs(vs[i] - vo)) <= 1e-4 * np.max(np.abs(vo)), i
        assert hist[-1][i]["Wx"] == pytest.approx(ho[-1]["Wx"], rel=1e-4)
        assert hist[-1][i]["Q"] == pytest.approx(ho[-1]["Q"], rel=1e-6)
