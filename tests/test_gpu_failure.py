"""Failure detection without a GPU fault (needs a GPU).

The staged kernels wait for their bulk copies on mbarriers with a bounded
wait.  pic_selftest_timeout runs one such wait with nothing to wait for: it
must give up within its limit, raise PIC_FLAG_TIMEOUT, report
PIC_ERR_TIMEOUT, and leave the context usable.  Nothing here faults, traps or
hangs the GPU: the wait is bounded in time and no copy is in flight.
"""
import time

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


def test_a_bounded_wait_that_runs_out_is_reported_and_the_context_survives():
    w = pi.landau(n=16, ppc=8, seed=51)
    sim = Simulation.from_workload(w, diag_every=1)
    t0 = time.perf_counter()
    rc = capi.pic_selftest_timeout(sim.handle)
    secs = time.perf_counter() - t0
    assert rc == capi.PIC_ERR_TIMEOUT
    assert secs < 30.0
    assert sim.flags() & capi.PIC_FLAG_TIMEOUT
    sim.step(1)
    with pytest.raises(capi.PicError) as e:
        sim.diagnostics()
    assert e.value.code == capi.PIC_ERR_TIMEOUT
    # cleared, the same context runs on and matches the oracle
    assert sim.flags(clear=True) & capi.PIC_FLAG_TIMEOUT
    assert sim.flags() == 0
    sim.step(2)
    x, v = sim.particles()
    hist = sim.diagnostics()
    sim.close()
    assert len(hist) == 3
    xo, vo, _ = po.run(w.x, w.v, po.Grid(w.n, w.L), po.Params(dt=w.dt, Q=w.Q), 3)
    L = np.asarray(w.L)
    d = x - xo
    d -= L * np.round(d / L)
    assert np.max(np.abs(d) / (L / np.asarray(w.n))) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
