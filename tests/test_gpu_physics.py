"""Physics of the CUDA path at the benchmark scales (GPU).

* Same input as the oracle: weak Landau damping on a 32^3 grid with 64
  particles per cell (2,097,152 particles), 200 steps, against the stored FP64
  oracle history (tests/golden, written by make_physics_goldens.py): the
  (1,0,0) mode of E_x and W_x at every step.
* Landau damping at 128^3 x 64 per cell (134,217,728 particles, Section 4.1:
  alpha = 0.05, k = 0.5, L = 4 pi, dt = 0.05), 200 steps: the fitted rate
  against the same fit of the oracle's noise-free 1D lattice at the same
  alpha (2%), and against the linear root 1.41566 - 0.15336i.  The oracle's
  lattice itself, fitted on t in (2, 10), decays about 3% faster than the
  linear root (finite amplitude and the damped transients in the window), so
  the linear root is held to 5% and the frequency to 1%.
* Bump-on-tail growth (Section 4.2 family; velocity mixture
  0.9 N(0,1) + 0.1 N(4, 0.3^2), L = 20 pi) seeded at k = 0.3 (mode 3) with
  alpha = 1e-3 on starts that are quiet along the wave vector.  On the quiet
  1D lattice of the stored oracle history (64 cells, the 64^3 grid's
  resolution) the GPU's fastest root matches the oracle's (1%) and the
  two-Maxwellian root 0.92925 + 0.21093i (2%).  At 64^3 x 16 per cell
  (4,194,304 particles) the transverse positions and velocities are random
  draws whose field noise scatters the resonant beam particles; that slows
  the growth by a few percent, so the linear root is held to 5% there.  The
  benchmark's own bump-on-tail input (alpha = 0.05 at k = 0.1) saturates the
  beam mode at once, so there only its two Langmuir roots (1.08464 and
  -0.98988) are checked.
* Two-stream instability (Section 4.2, Eq. twostream_f: beams at -pi/2 and
  +pi/2, spread 0.1, k = 0.5), seeded with alpha = 1e-3: on the quiet 1D
  lattice of the stored oracle history the GPU's growth rate matches the
  oracle's (1%) and the kinetic root 0.31824i (2%).  (In 3D the cold beams
  are also unstable at oblique wave vectors, which random transverse
  positions seed; those modes outgrow k = 0.5 and drive it nonlinearly, so
  the rate is checked on the lattice.)
* Strong Landau damping (alpha = 0.5, Section 5.3) on 16^3 x 16 per cell,
  200 steps: the W_x history against the stored oracle history (the same
  input), to 1e-4 of its peak.
"""
import json
import math
import os

import numpy as np
import pytest

import bench
import pic_inputs as pi
from tests import dispersion
from tests.fits import damped_cosine, fastest_root, pencil

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BOT_SPECIES = ((0.9, 0.0, 1.0), (0.1, 4.0, 0.3))


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    return np.array(g["t_field"]), np.array([complex(*m) for m in g["mode"]]), g


def _run(w, n_steps):
    sim = Simulation.from_workload(w, diag_every=1, diag_capacity=n_steps + 8, **bench.LAUNCH)
    sim.step(n_steps)
    hist = sim.diagnostics(n_steps + 8)
    flags = sim.flags()
    sim.close()
    assert flags == 0
    t = np.array([d["t_field"] for d in hist])
    c = np.array([d["mode"] for d in hist])
    return t, c, hist


def test_landau_history_matches_oracle_at_32_cubed():
    to, co, g = _golden("landau_32x32x32_ppc64_history.json")
    w = pi.landau(n=32, ppc=64, seed=1001)
    t, c, hist = _run(w, 200)
    assert np.array_equal(t, to)
    scale = np.max(np.abs(co))
    err = np.max(np.abs(c - co)) / scale
    print(f"32^3 mode history: max deviation {err:.2e} of the peak")
    assert err <= 1e-4
    Wx = np.array([d["Wx"] for d in hist])
    Wxo = np.array(g["Wx"])
    assert np.max(np.abs(Wx - Wxo)) <= 1e-4 * np.max(Wxo)
    root = dispersion.root(0.5, 1.4 - 0.15j)
    gg, wg = damped_cosine(t, c, 2.0, 10.0, root)
    go, wo = damped_cosine(to, co, 2.0, 10.0, root)
    assert gg == pytest.approx(go, rel=0.02)
    assert wg == pytest.approx(wo, rel=0.01)


def test_landau_damping_rate_at_128_cubed():
    tl, cl, _ = _golden("landau_lattice_1d_history.json")
    w = pi.by_name("landau_128")
    Q = w.Q
    t, c, hist = _run(w, 200)
    del w
    root = dispersion.root(0.5, 1.4 - 0.15j)
    gamma, omega = damped_cosine(t, c, 2.0, 10.0, root)
    g_lat, w_lat = damped_cosine(tl, cl, 2.0, 10.0, root)
    print(f"landau 128^3: gamma {gamma:.5f} (oracle lattice {g_lat:.5f}, linear {root.imag:.5f}), "
          f"omega {omega:.5f} (linear {root.real:.5f})")
    assert gamma == pytest.approx(g_lat, rel=0.02)
    assert gamma == pytest.approx(root.imag, rel=0.05)
    assert omega == pytest.approx(root.real, rel=0.01)
    # the deposit conserves charge exactly
    assert all(abs(d["Q"] - Q) <= 1e-6 * abs(Q) for d in hist)


def test_bump_on_tail_growth_rate_matches_oracle_on_a_quiet_lattice():
    to, co, _ = _golden("bump_on_tail_quiet_1d_history.json")
    # the input of the stored history (make_physics_goldens.bump_on_tail_quiet_1d)
    w = pi.bump_on_tail_quiet(n=(64, 1, 1), L=20.0 * math.pi, axis=0, m=3, alpha=1e-3,
                              ms=256, mv=512)
    t, c, _ = _run(w, 400)
    assert np.array_equal(t, to)
    root = dispersion.root(0.3, 0.93 + 0.21j, species=BOT_SPECIES)
    gamma, omega = fastest_root(t, c, 5.0, 20.0)
    g_o, w_o = fastest_root(to, co, 5.0, 20.0)
    print(f"bump-on-tail lattice, k = 0.3: gamma {gamma:.5f} (oracle {g_o:.5f}, linear "
          f"{root.imag:.5f}), omega {omega:.5f} (oracle {w_o:.5f})")
    assert gamma == pytest.approx(g_o, rel=0.01)
    assert omega == pytest.approx(w_o, rel=0.005)
    assert gamma == pytest.approx(root.imag, rel=0.02)


def test_bump_on_tail_growth_rate_at_64_cubed():
    w = pi.bump_on_tail_quiet(n=64, L=20.0 * math.pi, axis=2, m=3, alpha=1e-3, ms=4096, mv=1024)
    assert w.n_particles == 64 ** 3 * 16
    t, c, _ = _run(w, 400)
    root = dispersion.root(0.3, 0.93 + 0.21j, species=BOT_SPECIES)
    gamma, omega = fastest_root(t, c, 5.0, 20.0)
    print(f"bump-on-tail 64^3, k = 0.3: gamma {gamma:.5f} (linear {root.imag:.5f}), "
          f"omega {omega:.5f} (linear {root.real:.5f})")
    assert gamma == pytest.approx(root.imag, rel=0.05)
    assert omega == pytest.approx(root.real, rel=0.01)


def test_bump_on_tail_langmuir_roots_at_64_cubed():
    w = pi.by_name("bump_on_tail_64")
    t, c, _ = _run(w, 400)
    sel = (t >= 0.5) & (t <= 20.0)
    s, a = pencil(c[sel], t[1] - t[0], M=3)
    top = np.argsort(-np.abs(a))[:2]
    found = sorted(abs(s[i].imag) for i in top)
    fast = dispersion.root(0.1, 1.0 + 0.0j, species=BOT_SPECIES)
    slow = dispersion.root(0.1, -1.0 + 0.0j, species=BOT_SPECIES)
    want = sorted([abs(fast.real), abs(slow.real)])
    print(f"bump-on-tail 64^3, k = 0.1: Langmuir roots {found} (linear {want})")
    assert found[0] == pytest.approx(want[0], rel=0.005)
    assert found[1] == pytest.approx(want[1], rel=0.005)
    assert all(abs(s[i].real) < 0.01 for i in top)


TSI_SPECIES = ((0.5, -0.5 * math.pi, 0.1), (0.5, 0.5 * math.pi, 0.1))


def _two_stream(n, ms, mv):
    return pi.bump_on_tail_quiet(n=n, L=4.0 * math.pi, axis=0, m=1, alpha=1e-3, ms=ms, mv=mv,
                                 eps=0.5, v_beam=0.5 * math.pi, sigma_beam=0.1, sigma_bulk=0.1,
                                 u_bulk=-0.5 * math.pi)


def test_two_stream_growth_rate_matches_oracle_on_a_quiet_lattice():
    to, co, _ = _golden("two_stream_quiet_1d_history.json")
    # the input of the stored history (make_physics_goldens.two_stream_quiet_1d)
    w = _two_stream((32, 1, 1), 64, 512)
    t, c, _ = _run(w, 400)
    assert np.array_equal(t, to)
    root = dispersion.root(0.5, 0.3j, species=TSI_SPECIES)
    gamma, omega = fastest_root(t, c, 4.0, 18.0)
    g_o, _ = fastest_root(to, co, 4.0, 18.0)
    print(f"two-stream lattice: gamma {gamma:.5f} (oracle {g_o:.5f}, kinetic {root.imag:.5f})")
    assert gamma == pytest.approx(g_o, rel=0.01)
    assert gamma == pytest.approx(root.imag, rel=0.02)
    assert omega < 0.01


def test_strong_landau_history_matches_oracle():
    to, _, g = _golden("strong_landau_16_history.json")
    w = pi.landau(n=16, ppc=16, alpha=0.5, seed=1007)
    t, _, hist = _run(w, 200)
    assert np.array_equal(t, to)
    Wx = np.array([d["Wx"] for d in hist])
    Wxo = np.array(g["Wx"])
    err = np.max(np.abs(Wx - Wxo)) / np.max(Wxo)
    print(f"strong Landau 16^3: W_x history deviation {err:.2e} of the peak")
    assert err <= 1e-4
