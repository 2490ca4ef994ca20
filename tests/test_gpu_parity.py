"""CUDA path vs the FP64 oracle on identical seeded inputs (needs a GPU).

Tolerances (FP32 particle store, FP32 tile accumulation, FP32 cuFFT):
  rho, E        max |gpu - oracle| <= 1e-5 max |oracle|
  one step      |dx| <= 1e-5 h per axis, |dv| <= 1e-5 max |v|
  diagnostics   W_d, K to 1e-5 relative per step, Q to 1e-6, P absolute
                against m_p N_p v_th.
Several results are correct up to summation order (FP32 atomics), so no
comparison below is bit-exact except the integer work (sort permutation,
counts), which is checked exactly.
"""
import math

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

TOL = 1e-5


def _grid(w):
    return po.Grid(w.n, w.L)


def _params(w):
    return po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q, B=w.B, wz2=w.wz2)


def _pos_err_in_cells(x, xo, w):
    L = np.asarray(w.L)
    d = x - xo
    d -= L * np.round(d / L)
    return np.max(np.abs(d) / (L / np.asarray(w.n)))


def _ragged():
    w = pi.uniform_plasma(n=(12, 10, 6), ppc=1, L=(3.0, 2.0, 1.5), seed=77)
    # 1001 particles: ragged against every block and vector width
    w.x = w.x[:1001].copy()
    w.v = w.v[:1001].copy()
    w.Q = -4.5
    # exact boundary positions: 0, nextafter(L, 0), exactly on nodes
    L = np.asarray(w.L)
    h = L / np.asarray(w.n)
    w.x[0] = 0.0
    w.x[1] = np.nextafter(L, 0.0)
    w.x[2] = 0.5 * h
    w.x[3] = L - 0.5 * h
    w.v[:4] = 0.0
    return w


def _penning_small():
    return pi.penning(n=32, n_particles=200_000, L=20.0, sigma=(1.0, 1.0, 2.0), seed=5,
                      Q=-1562.5, wz2=1.0)


WORKLOADS = {
    "landau16": lambda: pi.landau(n=16, ppc=8, seed=1000),
    "penning32": _penning_small,
    "ragged": _ragged,
    "bot16": lambda: pi.bump_on_tail(n=16, ppc=4, seed=9),
}


@pytest.fixture(params=sorted(WORKLOADS))
def workload(request):
    return WORKLOADS[request.param]()


# --------------------------------------------------------------------- load

def test_load_and_readback_roundtrip(workload):
    w = workload
    sim = Simulation.from_workload(w)
    x, v = sim.particles()
    assert _pos_err_in_cells(x, w.x, w) < 1e-6
    assert np.max(np.abs(v - w.v)) <= 1e-6 * max(1.0, np.max(np.abs(w.v)))
    assert np.all((x >= 0) & (x < np.asarray(w.L)))
    assert sim.flags() == 0
    sim.close()


# ------------------------------------------------------------------- deposit

def _oracle_half_step_positions(w):
    return po.wrap(w.x + 0.5 * w.dt * w.v, _grid(w))


@pytest.mark.parametrize("options", [0, 1], ids=["fp32", "fixed"])
def test_deposit_matches_oracle(workload, options):
    w = workload
    sim = Simulation.from_workload(w, options=options)
    sim.deposit()
    rho, _ = sim.field()
    qp = w.Q / w.n_particles
    rho_o = po.deposit(_oracle_half_step_positions(w), _grid(w), qp)
    err = np.max(np.abs(rho - rho_o))
    assert err <= TOL * np.max(np.abs(rho_o)), err / np.max(np.abs(rho_o))
    # total charge: h^3 sum rho = Q_e
    g = _grid(w)
    assert abs(float(np.sum(rho.astype(np.float64))) * g.cell_volume - w.Q) <= 1e-5 * abs(w.Q)
    sim.close()


@pytest.mark.parametrize("options", [0, 1], ids=["fp32", "fixed"])
@pytest.mark.parametrize("tile,guard,chunk", [((4, 4, 4), 1, 64), ((8, 8, 8), 2, 4095),
                                              ((16, 8, 4), 3, 1000), ((5, 3, 7), 1, 33)])
def test_deposit_is_independent_of_tiling(tile, guard, chunk, options):
    w = pi.landau(n=(20, 12, 14), ppc=6, seed=3, alpha=0.3)
    sim = Simulation.from_workload(w, tile=tile, guard=guard, chunk=chunk, options=options)
    sim.deposit()
    rho, _ = sim.field()
    rho_o = po.deposit(_oracle_half_step_positions(w), _grid(w), w.Q / w.n_particles)
    assert np.max(np.abs(rho - rho_o)) <= TOL * np.max(np.abs(rho_o))
    sim.close()


@pytest.mark.parametrize("n,tile,ppc", [((32, 32, 32), (2, 2, 2), 4),     # 4096 tiles: 1 coarse pass
                                         ((64, 64, 32), (2, 2, 2), 2),     # 16384 tiles: 2 passes
                                         ((36, 20, 28), (3, 2, 2), 3),     # 1680 tiles, ragged keys
                                         ((32, 32, 32), (2, 2, 2), 0.1)])  # sparse: slices overflow
def test_first_binning_of_arbitrary_order_with_many_tiles(n, tile, ppc):
    """The load's coarse pre-passes (tile key >> shift) and the full-key pass
    bin particles given in random order: readback, deposit and one step agree
    with the oracle."""
    n_cells = int(np.prod(n))
    w = pi.landau(n=n, ppc=max(1, int(ppc)), seed=31, alpha=0.2)
    if ppc < 1:
        keep = int(ppc * n_cells)
        w.x = w.x[:keep].copy()
        w.v = w.v[:keep].copy()
    rng = np.random.default_rng(5)
    order = rng.permutation(w.x.shape[0])
    w.x = w.x[order].copy()
    w.v = w.v[order].copy()
    sim = Simulation.from_workload(w, tile=tile, options=1)
    x, v = sim.particles()
    assert _pos_err_in_cells(x, w.x, w) < 1e-6
    assert np.max(np.abs(v - w.v)) <= 1e-6 * max(1.0, np.max(np.abs(w.v)))
    sim.deposit()
    rho, _ = sim.field()
    rho_o = po.deposit(_oracle_half_step_positions(w), _grid(w), w.Q / w.n_particles)
    assert np.max(np.abs(rho - rho_o)) <= TOL * np.max(np.abs(rho_o))
    sim.step(1)
    x1, v1 = sim.particles()
    xo, vo = po.step(w.x, w.v, _grid(w), _params(w))
    assert _pos_err_in_cells(x1, xo, w) <= 1e-5
    assert np.max(np.abs(v1 - vo)) <= 1e-5 * np.max(np.abs(vo))
    assert sim.flags() == 0
    sim.close()


@pytest.mark.parametrize("options", [0, 1], ids=["fp32", "fixed"])
def test_deposit_of_strays_after_many_steps_without_rebinning(options):
    """Particles far outside their tile since the last sort still deposit exactly."""
    w = pi.landau(n=16, ppc=8, seed=4)
    w.v *= 6.0              # ~3 cells per step
    sim = Simulation.from_workload(w, sort_period=-1, guard=1, options=options)
    xo, vo = w.x.copy(), w.v.copy()
    g, p = _grid(w), _params(w)
    for _ in range(5):
        sim.step(1)
        xo, vo = po.step(xo, vo, g, p)
    sim.deposit()
    rho, _ = sim.field()
    rho_o = po.deposit(po.wrap(xo + 0.5 * w.dt * vo, g), g, w.Q / w.n_particles)
    assert np.max(np.abs(rho - rho_o)) <= 1e-4 * np.max(np.abs(rho_o))
    sim.close()


def test_fixed_point_deposit_is_deterministic_and_conserves_charge():
    """Integer tile sums do not depend on the order of the atomics: two
    deposits of the same particles (re-binned in between, which changes the
    order within tiles) give bit-identical rho."""
    w = _penning_small()
    sim = Simulation.from_workload(w, options=capi.PIC_OPT_FIXED_DEPOSIT)
    sim.deposit()
    rho1, _ = sim.field()
    sim.sort()
    sim.deposit()
    rho2, _ = sim.field()
    assert np.array_equal(rho1, rho2)
    g = _grid(w)
    assert abs(float(np.sum(rho1.astype(np.float64))) * g.cell_volume - w.Q) <= 1e-6 * abs(w.Q)
    sim.close()


# --------------------------------------------------------------- field solve

@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, -2, 1), (3, 1, -2)])
def test_field_solve_single_mode_closed_form(m):
    n, L = (16, 20, 12), (2.0, 3.0, 5.0)
    sim = Simulation(n=n, L=L, n_particles=1, dt=0.1)
    h = np.asarray(L) / np.asarray(n)
    k = np.array([2 * math.pi * m[d] / L[d] for d in range(3)])
    zz, yy, xx = np.meshgrid(*[(np.arange(n[d]) + 0.5) * h[d] for d in (2, 1, 0)], indexing="ij")
    ph = k[0] * xx + k[1] * yy + k[2] * zz
    sim.set_rho(np.cos(ph))
    sim.field_solve()
    _, E = sim.field()
    k2 = float(k @ k)
    for d in range(3):
        exact = k[d] * np.sin(ph) / k2
        assert np.max(np.abs(E[d] - exact)) <= 2e-6 * max(1.0, np.max(np.abs(k)) / k2)
    sim.close()


def test_field_solve_matches_oracle(workload):
    w = workload
    sim = Simulation.from_workload(w)
    sim.deposit()
    sim.field_solve()
    _, E = sim.field()
    g = _grid(w)
    rho_o = po.deposit(_oracle_half_step_positions(w), g, w.Q / w.n_particles)
    E_o = po.solve_field(rho_o, g)
    err = np.max(np.abs(E - E_o))
    assert err <= TOL * np.max(np.abs(E_o)), err / np.max(np.abs(E_o))
    sim.close()


# --------------------------------------------------------------- full steps

def test_one_step_matches_oracle(workload):
    w = workload
    sim = Simulation.from_workload(w)
    sim.step(1)
    x, v = sim.particles()
    xo, vo = po.step(w.x, w.v, _grid(w), _params(w))
    assert _pos_err_in_cells(x, xo, w) <= TOL
    assert np.max(np.abs(v - vo)) <= TOL * np.max(np.abs(vo))
    assert sim.counts() == (w.n_particles, 1)
    sim.close()


def test_separate_calls_equal_one_step():
    w = pi.landau(n=16, ppc=8, seed=11)
    sim = Simulation.from_workload(w)
    sim.deposit()
    sim.field_solve()
    sim.gather_push()
    x, v = sim.particles()
    xo, vo = po.step(w.x, w.v, _grid(w), _params(w))
    assert _pos_err_in_cells(x, xo, w) <= TOL
    assert np.max(np.abs(v - vo)) <= TOL * np.max(np.abs(vo))
    sim.close()


def test_step_after_split_calls_redeposits_the_stale_density():
    """pic_gather_push leaves rho stale; the next pic_step deposits first."""
    w = pi.landau(n=16, ppc=8, seed=12)
    sim = Simulation.from_workload(w)
    sim.deposit()
    sim.field_solve()
    sim.gather_push()
    sim.step(2)
    x, v = sim.particles()
    xo, vo, _ = po.run(w.x, w.v, _grid(w), _params(w), 3)
    assert _pos_err_in_cells(x, xo, w) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
    sim.close()


@pytest.mark.parametrize("sort_period,options", [(1, 0), (3, 0), (-1, 0), (2, 1), (4, 1)])
def test_twenty_steps_and_diagnostics_match_oracle(sort_period, options):
    """Landau damping, 16^3 grid, 8 particles per cell, dt = 0.05, 20 steps."""
    w = pi.landau(n=16, ppc=8, seed=1000, n_steps=20)
    sim = Simulation.from_workload(w, diag_every=1, sort_period=sort_period, options=options)
    sim.step(w.n_steps)
    x, v = sim.particles()
    hist = sim.diagnostics()
    xo, vo, ho = po.run(w.x, w.v, _grid(w), _params(w), w.n_steps, mode=w.mode,
                        mode_comp=w.mode_comp)
    assert _pos_err_in_cells(x, xo, w) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
    assert len(hist) == len(ho) == w.n_steps
    mp = w.Q / w.n_particles / w.q_over_m
    for a, b in zip(hist, ho):
        assert a["step"] == b["step"]
        assert a["t_field"] == pytest.approx(b["t_field"], rel=1e-15)
        for key in ("Wx", "Wy", "Wz", "K"):
            assert a[key] == pytest.approx(b[key], rel=1e-4), key
        assert a["Q"] == pytest.approx(b["Q"], rel=1e-6)
        for key in ("Px", "Py", "Pz"):
            assert abs(a[key] - b[key]) <= 1e-6 * abs(mp) * w.n_particles
        assert abs(a["mode"] - b["mode"]) <= 1e-4 * abs(b["mode"]) + 1e-7
    sim.close()


@pytest.mark.parametrize("options", [0, 1], ids=["fp32", "fixed"])
def test_penning_boris_steps_match_oracle(options):
    w = _penning_small()
    sim = Simulation.from_workload(w, options=options)
    sim.step(5)
    x, v = sim.particles()
    xo, vo, _ = po.run(w.x, w.v, _grid(w), _params(w), 5)
    assert _pos_err_in_cells(x, xo, w) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
    sim.close()


@pytest.mark.parametrize("B", [(0.0, 0.0, 0.0), (0.0, 0.0, 2.0)])
def test_quadrupole_across_the_periodic_seam(B):
    """Particles everywhere in the box, including the half cells next to the
    seam where the quadrupole field jumps by wz2 L: the push must take the
    position in [0, L) (the oracle's) and not the stencil base's image."""
    w = pi.bump_on_tail(n=8, ppc=4, seed=5, alpha=0.2, k=0.5)
    w.dt, w.wz2, w.B = 0.1, 0.3, B
    h = np.asarray(w.L) / np.asarray(w.n)
    w.x[:8] = 0.25 * h           # inside [0, h/2) on every axis
    w.v[:8] = 0.0
    sim = Simulation.from_workload(w)
    sim.step(5)
    x, v = sim.particles()
    xo, vo, _ = po.run(w.x, w.v, _grid(w), _params(w), 5)
    assert _pos_err_in_cells(x, xo, w) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
    sim.close()


def test_lone_penning_particle_follows_the_oracle_orbit():
    w = pi.single_particle(x0=(10.7, 9.6, 11.1), v0=(0.3, -0.2, 0.1), n=(16, 16, 16),
                           L=(20.0, 20.0, 20.0), Q=0.0, dt=0.005, n_steps=400)
    sim = Simulation.from_workload(w)
    sim.step(w.n_steps)
    x, v = sim.particles()
    xo, vo, _ = po.run(w.x, w.v, _grid(w), _params(w), w.n_steps)
    assert np.max(np.abs(x - xo)) < 1e-4
    assert np.max(np.abs(v - vo)) < 1e-4
    sim.close()


# --------------------------------------------------------------- edge cases

def test_zero_particles():
    sim = Simulation(n=(8, 8, 8), L=(1.0, 1.0, 1.0), n_particles=0, dt=0.1, diag_every=1)
    sim.load(np.zeros((0, 3)), np.zeros((0, 3)))
    sim.step(2)
    rho, E = sim.field()
    assert np.all(rho == 0) and np.all(E == 0)
    hist = sim.diagnostics()
    assert len(hist) == 2 and hist[-1]["Q"] == 0.0 and hist[-1]["K"] == 0.0
    x, v = sim.particles()
    assert x.shape == (0, 3)
    sim.close()


def test_lone_particle_feels_no_self_force():
    w = pi.single_particle(x0=(0.37, 0.81, 0.52), v0=(0.0, 0.0, 0.0), n=(8, 6, 10),
                           L=(1.0, 1.2, 0.9), Q=-1.0, dt=0.1, Bz=0.0, wz2=0.0)
    sim = Simulation.from_workload(w)
    sim.step(3)
    _, E = sim.field()
    x, v = sim.particles()
    assert np.max(np.abs(v)) <= 1e-5 * np.max(np.abs(E)) * 0.3
    sim.close()


def test_reduced_axes_one_dimensional_grid():
    """An (Nx, 1, 1) grid runs the 1D problem (quiet Landau lattice)."""
    w = pi.landau_lattice_1d(nx=32, mx=32, mv=256, n_steps=40)
    sim = Simulation.from_workload(w, diag_every=1)
    sim.step(w.n_steps)
    hist = sim.diagnostics()
    _, _, ho = po.run(w.x, w.v, _grid(w), _params(w), w.n_steps)
    for a, b in zip(hist, ho):
        # the field decays: compare against its initial scale
        assert abs(a["mode"] - b["mode"]) <= 1e-4 * abs(ho[0]["mode"])
        assert abs(a["Wx"] - b["Wx"]) <= 1e-4 * ho[0]["Wx"]
    sim.close()


def test_capacity_and_flag_errors():
    sim = Simulation(n=(8, 8, 8), L=(1.0, 1.0, 1.0), n_particles=10, dt=0.1)
    with pytest.raises(capi.PicError) as e:
        sim.load(np.zeros((11, 3)), np.zeros((11, 3)))
    assert e.value.code == capi.PIC_ERR_CAPACITY
    x = np.full((10, 3), 0.5)
    x[3, 1] = np.nan
    sim.load(x, np.zeros((10, 3)))
    assert sim.flags() & capi.PIC_FLAG_NONFINITE
    with pytest.raises(capi.PicError) as e:
        sim.diagnostics()
    assert e.value.code == capi.PIC_ERR_DEVICE_FLAG
    sim.flags(clear=True)
    assert sim.flags() == 0
    sim.close()


def test_device_sources_and_destinations():
    w = pi.landau(n=16, ppc=2, seed=21)
    xd = torch.from_numpy(w.x).cuda()
    vd = torch.from_numpy(w.v).cuda()
    sim = Simulation(n=w.n, L=w.L, n_particles=w.n_particles, dt=w.dt, Q=w.Q)
    sim.load(xd, vd)
    sim.step(2)
    x, v = sim.particles(device=True)
    xh, vh = sim.particles()
    assert np.array_equal(x.cpu().numpy(), xh)
    assert np.array_equal(v.cpu().numpy(), vh)
    sim.close()


def test_cuda_graph_replay_matches_oracle():
    """pic_step enqueues only capturable work: replaying a captured 2-step
    graph three times equals six steps."""
    w = pi.landau(n=16, ppc=8, seed=31)
    sim = Simulation.from_workload(w, sort_period=1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    capi.pic_set_stream(sim.handle, s.cuda_stream)
    with torch.cuda.stream(s):
        sim.step(1)                 # warm up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sim.step(2)
    for _ in range(3):
        g.replay()               # on the current stream
    torch.cuda.synchronize()
    capi.pic_set_stream(sim.handle, torch.cuda.current_stream().cuda_stream)
    x, v = sim.particles()
    xo, vo, _ = po.run(w.x, w.v, _grid(w), _params(w), 7)
    assert _pos_err_in_cells(x, xo, w) <= 1e-4
    assert np.max(np.abs(v - vo)) <= 1e-4 * np.max(np.abs(vo))
    sim.close()


def test_load_and_readback_through_page_locked_host_buffers():
    """Page-locked host arrays are read and written in place by the load and
    unload kernels; the result equals the staged path for pageable arrays."""
    w = pi.landau(n=(12, 10, 6), ppc=5, seed=31, alpha=0.2)
    xs = torch.from_numpy(w.x).pin_memory()
    vs = torch.from_numpy(w.v).pin_memory()
    fixed = capi.PIC_OPT_FIXED_DEPOSIT     # deterministic deposit: equal bits expected
    a = Simulation.from_workload(w, options=fixed)
    b = Simulation(n=w.n, L=w.L, n_particles=w.n_particles, dt=w.dt, q_over_m=w.q_over_m, Q=w.Q,
                   options=fixed)
    capi.pic_load_particles(b.handle, xs.data_ptr(), vs.data_ptr(), w.n_particles, False)
    b.n_particles = w.n_particles
    a.step(3)
    b.step(3)
    xa, va = a.particles()
    xo = torch.empty((w.n_particles, 3), dtype=torch.float64).pin_memory()
    vo = torch.empty((w.n_particles, 3), dtype=torch.float64).pin_memory()
    capi.pic_get_particles(b.handle, xo.data_ptr(), vo.data_ptr(), False)
    assert np.array_equal(xa, xo.numpy()) and np.array_equal(va, vo.numpy())
    a.close()
    b.close()


def test_large_page_locked_load_bins_ranges_while_loading():
    """Above 2^22 particles a page-locked load is split into ranges, each
    binned on a side stream while the next one is read; the run equals the
    staged path for pageable arrays bit for bit (fixed-point deposit)."""
    w = pi.landau(n=(64, 64, 32), ppc=33, seed=41, alpha=0.2)
    extra = 777                                    # a ragged last range
    rng = np.random.default_rng(8)
    order = rng.permutation(w.x.shape[0])[: (1 << 22) + extra]
    w.x = w.x[order].copy()
    w.v = w.v[order].copy()
    xs = torch.from_numpy(w.x).pin_memory()
    vs = torch.from_numpy(w.v).pin_memory()
    fixed = capi.PIC_OPT_FIXED_DEPOSIT
    a = Simulation.from_workload(w, tile=(4, 4, 4), options=fixed)
    b = Simulation(n=w.n, L=w.L, n_particles=w.n_particles, dt=w.dt, q_over_m=w.q_over_m, Q=w.Q,
                   tile=(4, 4, 4), options=fixed)
    capi.pic_load_particles(b.handle, xs.data_ptr(), vs.data_ptr(), w.n_particles, False)
    b.n_particles = w.n_particles
    assert b.flags() == 0
    xb, vb = b.particles()
    assert _pos_err_in_cells(xb, w.x, w) < 1e-6
    assert np.max(np.abs(vb - w.v)) <= 1e-6 * max(1.0, np.max(np.abs(w.v)))
    a.step(2)
    b.step(2)
    xa, va = a.particles()
    xb, vb = b.particles()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    ra, _ = a.field()
    rb, _ = b.field()
    assert np.array_equal(ra, rb)
    a.close()
    b.close()
