"""The fused push reads E along three paths that must give the same bits
(needs a GPU).

`k_push_deposit` gathers E (Section 3.1 step 3) from a shared-memory copy of
its tile's box when that copy fits three blocks per SM, with the box extent
compiled in for 8^3 tiles with two guard layers; particles outside the box,
and every particle when the copy does not fit, read the x-paired grid. All
paths read the same E values and interpolate them in the same order, and the
fixed-point deposit sums integers, so a run gives bit-identical particles and
charge density whichever path each particle takes. Without re-binning after
the load, particles drift out of their tiles' boxes, so the grid path runs
beside the shared one within a launch.
"""
import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2205_11052_gb300 import capi  # noqa: E402
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()

# (tile, guard): the staged box with the compiled-in extent (13 slots per
# axis), a staged box of another shape (13 x 13 x 11 slots), and a box too
# large to stage for three blocks per SM (15^3 slots: E from the grid)
PATHS = {
    "staged_constant_box": ((8, 8, 8), 2),
    "staged_runtime_box": ((8, 8, 6), 2),
    "grid_only": ((8, 8, 8), 3),
}


def _run(w, tile, guard, steps=6):
    sim = Simulation.from_workload(w, tile=tile, guard=guard, sort_period=-1,
                                   options=capi.PIC_OPT_FIXED_DEPOSIT)
    sim.step(steps)
    x, v = sim.particles()
    rho, _ = sim.field()
    _, strays = sim.rebin_stats()
    flags = sim.flags()
    sim.close()
    return x, v, rho, strays, flags


def test_staged_and_grid_gathers_give_the_same_bits():
    # dt = 0.3 moves a thermal particle about 0.8 cells per step on this grid
    w = pi.landau(n=32, ppc=8, alpha=0.2, seed=21, dt=0.3)
    runs = {name: _run(w, *cfg) for name, cfg in PATHS.items()}
    ref = runs["staged_constant_box"]
    assert ref[4] == 0
    # particles left their boxes, so both gather paths and the stray deposit ran
    assert ref[3] > w.n_particles // 100
    for name, got in runs.items():
        assert got[4] == 0, name
        for a, b, what in zip(ref[:3], got[:3], ("x", "v", "rho")):
            assert np.array_equal(a, b), f"{name}: {what} differs"
