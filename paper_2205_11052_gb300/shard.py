"""Particle-sharded runs over several GPUs of one node.

The paper distributes both particles and field over MPI ranks (Section 2,
Section 5: particle exchange, halo exchange, a distributed FFT).  The
particle kernels of this library shard more simply: every rank (one GPU)
holds a contiguous share of the particles and a full copy of the grid.  Per
step each rank deposits its own particles, one sum all-reduce of rho makes
every copy the total density, every rank solves the field on its copy
(redundantly: the solve is a few percent of a step), and gather and push stay
local.  No particle ever moves between ranks.

The exchange is written against four callables (deposit, solve, push and the
all-reduce), so the same driver runs the CUDA library on GPUs with NCCL, and
the test suite checks its logic on CPU ranks over gloo.
"""
from __future__ import annotations

from . import capi


def shard_range(n_total: int, world: int, rank: int):
    """[start, stop) of this rank's particles: contiguous, sizes differing by
    at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(n_total), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_charge(total_charge: float, n_total: int, start: int, stop: int) -> float:
    """Charge carried by a shard: every particle keeps q_p = Q_e / N of the
    whole run (Section 3.2 normalisation), so a shard of n particles carries
    Q_e n / N."""
    return float(total_charge) * (stop - start) / float(n_total)


class ShardedStep:
    """One step of the sharded cycle: deposit -> all-reduce(rho) -> solve ->
    gather + push, plus a re-binning every `sort_period` steps."""

    def __init__(self, deposit, allreduce_rho, solve, push, sort=None, sort_period=0):
        self.deposit = deposit
        self.allreduce_rho = allreduce_rho
        self.solve = solve
        self.push = push
        self.sort = sort
        self.sort_period = int(sort_period)
        self.steps = 0

    def step(self, n: int = 1):
        for _ in range(int(n)):
            if self.sort is not None and self.sort_period > 0 and self.steps > 0 and \
                    self.steps % self.sort_period == 0:
                self.sort()
            self.deposit()
            self.allreduce_rho()
            self.solve()
            self.push()
            self.steps += 1


def sharded_simulation(w, rank: int, world: int, dist=None, sort_period: int = 4, **kw):
    """A Simulation holding this rank's share of workload `w` and the
    ShardedStep that advances it with the ranks' densities summed each step
    (`dist` = torch.distributed with an initialised process group, or None
    for a single rank).  Returns (sim, stepper, (start, stop))."""
    import torch

    from .sim import Simulation

    start, stop = shard_range(w.n_particles, world, rank)
    sim = Simulation(n=w.n, L=w.L, n_particles=stop - start, dt=w.dt, q_over_m=w.q_over_m,
                     Q=shard_charge(w.Q, w.n_particles, start, stop), B=w.B, wz2=w.wz2,
                     mode=w.mode, mode_comp=w.mode_comp, sort_period=-1, **kw)
    sim.load(w.x[start:stop], w.v[start:stop])
    ng = sim.n[0] * sim.n[1] * sim.n[2]
    rho = torch.empty(ng, dtype=torch.float32, device=sim.device)

    def allreduce_rho():
        if dist is None or world == 1:
            return
        # the library and the collective share the stream, so the copy, the
        # sum and the copy back are ordered with the deposit and the solve
        capi.pic_get_field(sim.handle, rho.data_ptr(), 0, True)
        with torch.cuda.stream(sim.stream):
            dist.all_reduce(rho)
        capi.pic_set_rho(sim.handle, rho.data_ptr(), True)

    stepper = ShardedStep(sim.deposit, allreduce_rho, sim.field_solve, sim.gather_push,
                          sort=sim.sort, sort_period=sort_period)
    return sim, stepper, (start, stop)
