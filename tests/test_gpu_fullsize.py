"""Parity at the full benchmark sizes, in the benchmark's launch configuration.

One step of the 128^3 x 64-per-cell Landau workload (134,217,728 particles)
and of the 256^3 Penning bunch (1.3e8 particles): rho and E are compared
against the oracle on every node, the pushed particles on a random sample of
1,000,000 (the oracle evaluates its gather and push particle by particle, so a
sample is exact for those particles).  The oracle's deposit is summed over
particle chunks (it is linear in the particle set).
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
