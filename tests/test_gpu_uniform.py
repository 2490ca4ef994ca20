"""The uniform plasma test (Section 4.4) on the GPU against the oracle: random
displacements in [-h, h) from the shared SplitMix64 stream replace the gather
and push; deposit, solve and diagnostics as usual (needs a GPU)."""
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

MOVE = capi.PIC_OPT_UNIFORM_MOVE
SEED = 0x5EED


def _oracle(w, n_steps):
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    x, v, hist = w.x, w.v, []
    for n in range(n_steps):
        x, v, d = po.step_uniform(x, v, g, p, n, SEED, with_diag=True)
        hist.append(d)
    return x, v, hist


def _pos_err(x, xo, w):
    L = np.asarray(w.L)
    d = x - xo
    d -= L * np.round(d / L)
    return np.max(np.abs(d) / (L / np.asarray(w.n)))


@pytest.mark.parametrize("options", [MOVE, MOVE | capi.PIC_OPT_FIXED_DEPOSIT], ids=["fp32", "fixed"])
@pytest.mark.parametrize("split", [False, True], ids=["step", "split-calls"])
def test_uniform_move_matches_oracle(options, split):
    w = pi.uniform_plasma(n=(12, 10, 8), ppc=6, L=(3.0, 2.5, 2.0), seed=21)
    n_steps = 6
    sim = Simulation.from_workload(w, options=options, seed=SEED, diag_every=1, sort_period=2)
    if split:
        for _ in range(n_steps):
            sim.sort()
            sim.deposit()
            sim.field_solve()
            sim.gather_push()
    else:
        sim.step(n_steps)
    x, v = sim.particles()
    xo, vo, ho = _oracle(w, n_steps)
    assert _pos_err(x, xo, w) <= 1e-5
    assert np.max(np.abs(v - vo)) <= 1e-6 * np.max(np.abs(vo))
    if not split:
        hist = sim.diagnostics()
        assert len(hist) == n_steps
        for d, do in zip(hist, ho):
            for key in ("Wx", "Wy", "Wz"):
                assert d[key] == pytest.approx(do[key], rel=1e-4)
            assert d["Q"] == pytest.approx(do["Q"], rel=1e-6)
    assert sim.flags() == 0
    sim.close()


def test_uniform_move_is_rejected_where_it_has_no_meaning():
    w = pi.uniform_plasma(n=8, ppc=2, seed=22)
    sim = Simulation.from_workload(w, options=MOVE, seed=SEED)
    with pytest.raises(capi.PicError) as e:
        sim.adjoint_forward(3)
    assert e.value.code == capi.PIC_ERR_ARG
    sim.close()
