"""One step of the paper's strong-scaling case A on one GPU (needs a GPU).

Case A of Table strong_scaling_setup: weak Landau damping on a 512^3 grid
with 8 particles per cell (1,073,741,824 particles), dt = 0.5 h (Section
5.1).  The oracle cannot deposit a billion particles in a test's time, so
each stage is checked where the oracle's work stays small:

  rho   on the 32^3 corner block of nodes, against the oracle's deposit of
        every particle whose CIC stencil reaches that block;
  E     on every node, against the oracle's field solve of the GPU's rho
        (checked above where it can be);
  push  on 1,000,000 sampled particles, against the oracle's gather of that
        field, Boris kick and drift, particle by particle.
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

import bench  # noqa: E402  (launch configuration of the benchmark)
from paper_2205_11052_gb300 import capi  # noqa: E402
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()

N = 512
BLOCK = 32


def test_case_a_one_step_on_a_node_block_every_node_of_E_and_a_particle_sample():
    L = 4.0 * math.pi
    dt = 0.5 * L / N
    w = pi.landau(n=N, ppc=8, seed=1007, dt=dt)
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q)
    qp = w.Q / w.n_particles
    sim = Simulation.from_workload(w, **bench.LAUNCH)
    sim.deposit()
    ng = N ** 3
    rho_d = torch.empty(ng, dtype=torch.float32, device="cuda")
    capi.pic_get_field(sim.handle, rho_d.data_ptr(), 0, True)
    sim.field_solve()
    E4_d = torch.empty(ng * 4, dtype=torch.float32, device="cuda")
    capi.pic_get_field(sim.handle, 0, E4_d.data_ptr(), True)
    sim.gather_push()
    x1_d, v1_d = sim.particles(device=True)
    assert sim.flags() == 0
    sim.close()
    idx = np.sort(np.random.default_rng(3).choice(w.n_particles, 1_000_000, replace=False))
    it = torch.from_numpy(idx).cuda()
    x1 = x1_d[it].cpu().numpy()
    v1 = v1_d[it].cpu().numpy()
    del x1_d, v1_d
    rho = rho_d.cpu().numpy().reshape(g.shape)
    E = E4_d.view(N, N, N, 4)[..., :3].permute(3, 0, 1, 2).contiguous().cpu().numpy()
    del rho_d, E4_d
    torch.cuda.empty_cache()

    # rho on the corner block: particles whose stencil base is N-1 or 0..BLOCK-1 per axis
    h = L / N
    sel = []
    for s in range(0, w.n_particles, 1 << 25):
        xh = po.wrap(w.x[s:s + (1 << 25)] + 0.5 * dt * w.v[s:s + (1 << 25)], g)
        base = np.floor(xh / h - 0.5).astype(np.int64) % N
        near = np.all((base < BLOCK) | (base == N - 1), axis=1)
        sel.append(xh[near])
    xs = np.concatenate(sel)
    rho_o = po.deposit(xs, g, qp)[:BLOCK, :BLOCK, :BLOCK]
    assert xs.shape[0] > 8 * BLOCK ** 3 // 2
    assert np.max(np.abs(rho[:BLOCK, :BLOCK, :BLOCK] - rho_o)) <= 1e-5 * np.max(np.abs(rho_o))

    # E on every node from the GPU's rho
    E_o = po.solve_field(rho.astype(np.float64), g)
    assert np.max(np.abs(E - E_o)) <= 1e-5 * np.max(np.abs(E_o))

    # the push of the sample
    xh = po.wrap(w.x[idx] + 0.5 * dt * w.v[idx], g)
    e = po.gather(xh, E_o, g)
    v1_o = po.boris_kick(w.v[idx], e, p.q_over_m, p.B, p.dt)
    x1_o = po.wrap(xh + 0.5 * dt * v1_o, g)
    d = x1 - x1_o
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) / h <= 1e-5
    assert np.max(np.abs(v1 - v1_o)) <= 1e-5 * np.max(np.abs(v1_o))
