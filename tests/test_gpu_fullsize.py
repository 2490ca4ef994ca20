"""Parity at the full benchmark sizes, in the benchmark's launch configuration.

One step of the 128^3 x 64-per-cell Landau workload (134,217,728 particles)
and of the 256^3 Penning bunch (1.3e8 particles): rho and E are compared
against the oracle on every node, the pushed particles on a random sample of
1,000,000 (the oracle evaluates its gather and push particle by particle, so a
sample is exact for those particles).  The oracle's deposit is summed over
particle chunks (it is linear in the particle set).

The fused gather + push + deposit kernel that pic_step runs is checked the
same way on the third step of each workload (after two steps, so its work
items span particles that have drifted since their re-binning): the density
it deposits against the oracle's deposit of the positions it wrote, on every
node, and the pushed particles of a sample against the oracle's step from the
state before it.
"""
import numpy as np
import pytest

import pic_inputs as pi
from oracle import pic_oracle as po

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

import bench  # noqa: E402  (launch configuration of the benchmark)
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()


# the benchmark's launch settings for each workload
LAUNCHES = {"landau_128": dict(bench.LAUNCH),
            "penning_256": dict(bench.LAUNCH, sort_period=2, guard=3)}


def _oracle_rho(xh, grid, qp, chunk=1 << 22):
    rho = np.zeros(grid.shape)
    for s in range(0, xh.shape[0], chunk):
        rho += po.deposit(xh[s:s + chunk], grid, qp)
    return rho


@pytest.mark.parametrize("name", ["landau_128", "penning_256"])
def test_full_size_one_step_on_every_node_and_a_particle_sample(name):
    w = pi.by_name(name)
    sim = Simulation.from_workload(w, **bench.LAUNCH)
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q, B=w.B, wz2=w.wz2)
    qp = w.Q / w.n_particles
    xh = po.wrap(w.x + 0.5 * w.dt * w.v, g)

    sim.deposit()
    rho, _ = sim.field()
    rho_o = _oracle_rho(xh, g, qp)
    assert np.max(np.abs(rho - rho_o)) <= 1e-5 * np.max(np.abs(rho_o))

    sim.field_solve()
    _, E = sim.field()
    E_o = po.solve_field(rho_o, g)
    assert np.max(np.abs(E - E_o)) <= 1e-5 * np.max(np.abs(E_o))

    sim.gather_push()
    x1, v1 = sim.particles()
    idx = np.random.default_rng(0).choice(w.n_particles, 1_000_000, replace=False)
    e = po.gather(xh[idx], E_o, g)
    if p.wz2:
        e = e + po.external_field(xh[idx], g, p.wz2)
    v1_o = po.boris_kick(w.v[idx], e, p.q_over_m, p.B, p.dt)
    x1_o = po.wrap(xh[idx] + 0.5 * p.dt * v1_o, g)
    L = np.asarray(w.L)
    d = x1[idx] - x1_o
    d -= L * np.round(d / L)
    assert np.max(np.abs(d) / (L / np.asarray(w.n))) <= 1e-5
    assert np.max(np.abs(v1[idx] - v1_o)) <= 1e-5 * np.max(np.abs(v1_o))
    assert sim.flags() == 0
    sim.close()


@pytest.mark.parametrize("name", ["landau_128", "penning_256"])
def test_full_size_fused_step_on_every_node_and_a_particle_sample(name):
    w = pi.by_name(name)
    sim = Simulation.from_workload(w, **LAUNCHES[name])
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q, B=w.B, wz2=w.wz2)
    qp = w.Q / w.n_particles
    del w
    sim.step(2)
    x2, v2 = sim.particles()
    sim.step(1)                        # (re-bin if due,) solve, fused gather + push + deposit
    x3, v3 = sim.particles()
    rho3, _ = sim.field()              # what the fused kernel deposited
    assert sim.flags() == 0
    sim.close()

    rho_o = _oracle_rho(po.wrap(x3 + 0.5 * p.dt * v3, g), g, qp)
    assert np.max(np.abs(rho3 - rho_o)) <= 1e-5 * np.max(np.abs(rho_o))
    del rho_o

    xh2 = po.wrap(x2 + 0.5 * p.dt * v2, g)
    E2_o = po.solve_field(_oracle_rho(xh2, g, qp), g)
    idx = np.random.default_rng(1).choice(x2.shape[0], 1_000_000, replace=False)
    e = po.gather(xh2[idx], E2_o, g)
    if p.wz2:
        e = e + po.external_field(xh2[idx], g, p.wz2)
    v3_o = po.boris_kick(v2[idx], e, p.q_over_m, p.B, p.dt)
    x3_o = po.wrap(xh2[idx] + 0.5 * p.dt * v3_o, g)
    L = np.asarray(g.L)
    d = x3[idx] - x3_o
    d -= L * np.round(d / L)
    assert np.max(np.abs(d) / (L / np.asarray(g.n))) <= 1e-5
    assert np.max(np.abs(v3[idx] - v3_o)) <= 1e-5 * np.max(np.abs(v3_o))
