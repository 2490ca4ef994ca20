"""The multi-rank paths on CPU: world_size 2 over gloo.

bench.py --gpus N runs N independent replicas (the step needs no exchange
between ranks); its only collective is the max of the ranks' times, and the
job's throughput is all ranks' particle-steps over that max.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_throughput(1000, world, 4, slowest * 1e-3)
    out[rank] = (slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 15.0
    assert value == pytest.approx(1000 * 2 * 4 / 0.015)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10, 1, 2, 0.5) == 40.0


# ---------------------------------------------------------------- particle sharding
#
# The sharded cycle of paper_2205_11052_gb300.shard (each rank deposits its
# own particles onto a full grid, one sum all-reduce of rho, redundant solve,
# local gather + push) driven on two gloo ranks with the FP64 oracle's
# functions as the per-rank compute: the summed density of the two halves is
# the oracle's density of the whole set, and three sharded steps reproduce
# the unsharded run particle for particle.

def _shard_worker(rank, world, port, out):
    import numpy as np

    import pic_inputs as pi
    from oracle import pic_oracle as po
    from paper_2205_11052_gb300.shard import ShardedStep, shard_charge, shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = pi.landau(n=8, ppc=4, seed=21, alpha=0.3)     # 2048 particles
    g = po.Grid(w.n, w.L)
    s0, s1 = shard_range(w.n_particles, world, rank)
    q_p = shard_charge(w.Q, w.n_particles, s0, s1) / (s1 - s0)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    st = {"x": w.x[s0:s1].copy(), "v": w.v[s0:s1].copy()}

    def deposit():
        st["xh"] = po.wrap(st["x"] + 0.5 * p.dt * st["v"], g)
        st["rho"] = torch.from_numpy(po.deposit(st["xh"], g, q_p))

    def allreduce_rho():
        st["rho_local"] = st["rho"].clone()
        dist.all_reduce(st["rho"])

    def solve():
        st["E"] = po.solve_field(st["rho"].numpy(), g)

    def push():
        e = po.gather(st["xh"], st["E"], g)
        st["v"] = po.boris_kick(st["v"], e, p.q_over_m, p.B, p.dt)
        st["x"] = po.wrap(st["xh"] + 0.5 * p.dt * st["v"], g)

    stepper = ShardedStep(deposit, allreduce_rho, solve, push)
    stepper.step(1)
    first_rho = st["rho"].numpy().copy()
    stepper.step(2)
    out[rank] = (s0, s1, first_rho, st["x"], st["v"])
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_cycle_on_two_gloo_ranks_equals_the_whole_run():
    import numpy as np

    import pic_inputs as pi
    from oracle import pic_oracle as po

    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    w = pi.landau(n=8, ppc=4, seed=21, alpha=0.3)
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    rho_whole = po.deposit(po.wrap(w.x + 0.5 * p.dt * w.v, g), g, w.Q / w.n_particles)
    scale = np.max(np.abs(rho_whole))
    for r in range(world):
        assert np.max(np.abs(res[r][2] - rho_whole)) <= 1e-13 * scale
    x3, v3, _ = po.run(w.x, w.v, g, p, 3)
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == w.n_particles
    for r in range(world):
        s0, s1, _, x, v = res[r]
        d = x - x3[s0:s1]
        d -= np.asarray(w.L) * np.round(d / np.asarray(w.L))
        assert np.max(np.abs(d)) < 1e-11 and np.max(np.abs(v - v3[s0:s1])) < 1e-11


def test_shard_ranges_cover_the_particles_and_keep_the_particle_charge():
    from paper_2205_11052_gb300.shard import shard_charge, shard_range

    for n, world in ((10, 3), (7, 8), (1 << 20, 8), (0, 2)):
        spans = [shard_range(n, world, r) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        sizes = [b - a for a, b in spans]
        assert max(sizes) - min(sizes) <= 1
        if n:
            assert sum(shard_charge(-3.0, n, a, b) for a, b in spans) == pytest.approx(-3.0)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
