"""Stray-triggered re-binning of pic_step (needs a GPU).

With params.stray_rebin > 0 the device decides before every step whether to
re-bin, from the number of particles the last push left outside their tile's
guard.  Binning only reorders the store, and the fixed-point deposit sums
integers, so the trajectory in load order is bit-for-bit the same whatever
the re-binning schedule; it must also follow the FP64 oracle (Section 3.1
cycle, Section 3.2 scheme) within the one-step tolerances.
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
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()

FIXED = capi.PIC_OPT_FIXED_DEPOSIT


def _fast_landau():
    # ~1.5 cells per step: the 4^3 tiles with one guard layer lose particles
    # within a step or two of each re-binning
    w = pi.landau(n=16, ppc=8, seed=41)
    w.v *= 3.0
    return w


def _run(w, steps, **kw):
    sim = Simulation.from_workload(w, tile=4, guard=1, options=FIXED, **kw)
    sim.step(steps)
    x, v = sim.particles()
    stats = sim.rebin_stats()
    sim.deposit()
    rho, _ = sim.field()
    sim.close()
    return x, v, rho, stats


def test_strays_trigger_rebinning_and_the_run_matches_the_oracle():
    w = _fast_landau()
    steps = 8
    x, v, rho, (rebins, _) = _run(w, steps, sort_period=-1, stray_rebin=1e-12)
    # the load's binning plus at least one stray-triggered re-binning, and not
    # a re-binning before the first push (no strays yet)
    assert 2 <= rebins <= steps
    xo, vo, _ = po.run(w.x, w.v, po.Grid(w.n, w.L),
                       po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q), steps)
    L = np.asarray(w.L)
    d = x - xo
    d -= L * np.round(d / L)
    assert np.max(np.abs(d) / (L / np.asarray(w.n))) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
    g = po.Grid(w.n, w.L)
    rho_o = po.deposit(po.wrap(xo + 0.5 * w.dt * vo, g), g, w.Q / w.n_particles)
    assert np.max(np.abs(rho - rho_o)) <= 1e-4 * np.max(np.abs(rho_o))


def test_rebinning_schedule_does_not_change_the_trajectory():
    """Adaptive, every-step and never re-binning give bit-identical states."""
    w = _fast_landau()
    xa, va, ra, (na, _) = _run(w, 6, sort_period=-1, stray_rebin=1e-12)
    xp, vp, rp, (np_, _) = _run(w, 6, sort_period=1)
    xn, vn, rn, (nn, sn) = _run(w, 6, sort_period=-1)
    assert nn == 1 and sn > 0          # only the load's binning; strays pile up
    assert np_ == 6                    # load + before each step but the first
    assert 1 < na < 6
    for a, b in ((xa, xp), (va, vp), (ra, rp), (xa, xn), (va, vn), (ra, rn)):
        assert np.array_equal(a, b)


def test_no_strays_no_rebinning():
    """Slow particles never leave their guard: the gate stays shut."""
    w = pi.landau(n=16, ppc=8, seed=42)
    w.v *= 0.01
    _, _, _, (rebins, strays) = _run(w, 5, sort_period=-1, stray_rebin=1e-12)
    assert rebins == 1 and strays == 0


def test_threshold_and_period_combine():
    """A high threshold leaves only the period: before steps 3 and 5 of 6,
    as the host-side period schedules it."""
    w = _fast_landau()
    _, _, _, (rebins, _) = _run(w, 6, sort_period=2, stray_rebin=0.99)
    _, _, _, (host, _) = _run(w, 6, sort_period=2)
    assert rebins == host == 1 + 2


def test_stray_rebinning_inside_a_cuda_graph_equals_eager_steps():
    """The decision is taken on the device, so a captured graph re-bins
    exactly as the eager calls do."""
    w = _fast_landau()
    xe, ve, _, (ne, _) = _run(w, 6, sort_period=-1, stray_rebin=1e-12)
    sim = Simulation.from_workload(w, tile=4, guard=1, options=FIXED, sort_period=-1,
                                   stray_rebin=1e-12)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    capi.pic_set_stream(sim.handle, s.cuda_stream)
    with torch.cuda.stream(s):
        sim.step(2)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sim.step(2)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    capi.pic_set_stream(sim.handle, torch.cuda.current_stream().cuda_stream)
    x, v = sim.particles()
    n, _ = sim.rebin_stats()
    sim.close()
    assert np.array_equal(x, xe) and np.array_equal(v, ve)
    assert n == ne
