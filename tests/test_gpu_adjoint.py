"""GPU adjoint vs the FP64 oracle: J, dJ/dx0, dJ/dv0, dJ/dalpha (needs a GPU).

Tolerances: the GPU runs FP32 particles and grids, so gradients are compared
at 1e-4 of their largest component against the oracle's discrete adjoint and
against central differences of the oracle's objective (the accuracy the GPU
gradient is held to); J itself to 1e-5.
"""
import numpy as np
import pytest

import pic_inputs as pi
from oracle import pic_oracle as po

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2205_11052_gb300 import capi  # noqa: E402
from paper_2205_11052_gb300.autograd import final_field_energy  # noqa: E402
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()

FIXED = capi.PIC_OPT_FIXED_DEPOSIT


def _small(alpha=0.2, seed=5):
    w = pi.bump_on_tail(n=8, ppc=4, seed=seed, alpha=alpha, k=0.5)   # L = 4 pi, 2048 particles
    w.dt = 0.1
    return w


def _oracle(w, n_steps, weights, wz2=0.0, B=(0.0, 0.0, 0.0)):
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m, wz2=wz2, B=B)
    return po.run_with_gradient(w.x, w.v, g, p, n_steps, weights)


@pytest.mark.parametrize("options", [0, FIXED], ids=["fp32", "fixed"])
@pytest.mark.parametrize("wz2,weights,B", [(0.0, (0.0, 0.0, 1.0), (0.0, 0.0, 0.0)),
                                           (0.3, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0)),
                                           (0.3, (1.0, 1.0, 1.0), (0.0, 0.0, 5.0)),
                                           (0.0, (0.0, 1.0, 1.0), (1.0, -2.0, 3.0))],
                         ids=["plain", "quadrupole", "penning", "oblique-B"])
def test_gradient_matches_oracle_adjoint(options, wz2, weights, B):
    w = _small()
    n_steps = 6
    sim = Simulation.from_workload(w, wz2=wz2, B=B, options=options)
    J = sim.adjoint_forward(n_steps, weights, checkpoint_every=4)
    gx, gv = sim.adjoint_backward()
    Jo, gxo, gvo = _oracle(w, n_steps, weights, wz2, B)
    assert J == pytest.approx(Jo, rel=1e-5)
    assert np.max(np.abs(gx - gxo)) <= 1e-4 * np.max(np.abs(gxo))
    assert np.max(np.abs(gv - gvo)) <= 1e-4 * np.max(np.abs(gvo))
    # the call left the loaded state in place
    x, v = sim.particles()
    L = np.asarray(w.L)
    d = x - w.x
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) < 1e-5 and np.max(np.abs(v - w.v)) < 1e-6
    assert sim.counts()[1] == 0
    sim.close()


def test_gradient_matches_central_differences_of_the_oracle():
    w = _small()
    n_steps, weights = 6, (0.0, 0.0, 1.0)
    sim = Simulation.from_workload(w, options=FIXED)
    sim.adjoint_forward(n_steps, weights, checkpoint_every=2)
    gx, gv = sim.adjoint_backward()
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q)
    rng = np.random.default_rng(3)
    dX, dV = rng.standard_normal(w.x.shape), rng.standard_normal(w.v.shape)
    eps = 1e-5
    Jp = po.run_with_gradient(w.x + eps * dX, w.v + eps * dV, g, p, n_steps, weights)[0]
    Jm = po.run_with_gradient(w.x - eps * dX, w.v - eps * dV, g, p, n_steps, weights)[0]
    fd = (Jp - Jm) / (2 * eps)
    ad = float(np.sum(gx * dX) + np.sum(gv * dV))
    assert abs(ad - fd) <= 1e-4 * abs(fd)
    sim.close()


def test_amplitude_gradient_against_oracle_differences():
    """dJ/dalpha = <dJ/dx0, dx0/dalpha> (FP64 dot on the GPU) vs the central
    difference of the oracle's J over re-sampled particles (fixed uniforms)."""
    alpha, k, eps = 0.2, 0.5, 1e-6
    w = _small(alpha)
    n_steps, weights = 6, (0.0, 0.0, 1.0)
    sim = Simulation.from_workload(w, options=FIXED)
    sim.adjoint_forward(n_steps, weights, checkpoint_every=3)
    gx, _ = sim.adjoint_backward(device=True)
    dxa = np.zeros_like(w.x)
    dxa[:, 2] = po.cosine_sample_dalpha(w.x[:, 2], alpha, k)
    ad = sim.dot(gx, torch.from_numpy(dxa).cuda())
    wp, wm = _small(alpha + eps), _small(alpha - eps)
    fd = (_oracle(wp, n_steps, weights)[0] - _oracle(wm, n_steps, weights)[0]) / (2 * eps)
    assert ad == pytest.approx(fd, rel=1e-4)
    sim.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    """With the deterministic deposit the forward pass (and so J) is the same
    bits for every checkpoint interval; the gradients agree to FP32 rounding
    (the adjoint's own field deposit sums in FP32 in arbitrary order)."""
    w = pi.bump_on_tail(n=16, ppc=4, seed=8, alpha=0.1, k=0.25)
    out = []
    for K in (1, 3, 16):
        sim = Simulation.from_workload(w, options=FIXED)
        J = sim.adjoint_forward(16, (0.0, 0.0, 1.0), checkpoint_every=K)
        gx, gv = sim.adjoint_backward()
        out.append((J, gx, gv))
        sim.close()
    for J, gx, gv in out[1:]:
        assert J == out[0][0]
        assert np.max(np.abs(gx - out[0][1])) <= 1e-5 * np.max(np.abs(out[0][1]))
        assert np.max(np.abs(gv - out[0][2])) <= 1e-5 * np.max(np.abs(out[0][2]))


def test_longer_run_against_oracle_adjoint():
    """40 steps of a 16^3 bump-on-tail (16,384 particles), 5 segments."""
    w = pi.bump_on_tail(n=16, ppc=4, seed=8, alpha=0.1, k=0.25)
    n_steps, weights = 40, (0.0, 0.0, 1.0)
    sim = Simulation.from_workload(w, options=FIXED)
    J = sim.adjoint_forward(n_steps, weights, checkpoint_every=8)
    gx, gv = sim.adjoint_backward()
    Jo, gxo, gvo = _oracle(w, n_steps, weights)
    assert J == pytest.approx(Jo, rel=1e-4)
    assert np.max(np.abs(gx - gxo)) <= 1e-3 * np.max(np.abs(gxo))
    assert np.max(np.abs(gv - gvo)) <= 1e-3 * np.max(np.abs(gvo))
    sim.close()


def test_autograd_function_returns_the_library_gradients():
    w = _small()
    sim = Simulation.from_workload(w, options=FIXED)
    x0 = torch.from_numpy(w.x).cuda().requires_grad_(True)
    v0 = torch.from_numpy(w.v).cuda().requires_grad_(True)
    J = final_field_energy(x0, v0, sim, 6, (0.0, 0.0, 1.0), 2)
    (2.0 * J).backward()
    Jo, gxo, gvo = _oracle(w, 6, (0.0, 0.0, 1.0))
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-5)
    assert np.max(np.abs(x0.grad.cpu().numpy() - 2 * gxo)) <= 2e-4 * np.max(np.abs(gxo))
    assert np.max(np.abs(v0.grad.cpu().numpy() - 2 * gvo)) <= 2e-4 * np.max(np.abs(gvo))
    sim.close()


def test_penning_gradient_against_central_differences_of_the_oracle():
    """A Penning-trap bunch (B_z = 5, quadrupole with axial frequency 1) on a
    16^3 grid: <dJ/d(x0, v0), delta> against the central difference of the
    oracle's J, through 10 Boris steps."""
    w = pi.penning(n=16, n_particles=4096, L=20.0, seed=9)
    n_steps, weights = 10, (1.0, 1.0, 1.0)
    sim = Simulation.from_workload(w, options=FIXED)
    sim.adjoint_forward(n_steps, weights, checkpoint_every=4)
    gx, gv = sim.adjoint_backward()
    sim.close()
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m, B=w.B, wz2=w.wz2)
    rng = np.random.default_rng(4)
    dX, dV = rng.standard_normal(w.x.shape), rng.standard_normal(w.v.shape)
    eps = 1e-5
    Jp = po.run_with_gradient(w.x + eps * dX, w.v + eps * dV, g, p, n_steps, weights)[0]
    Jm = po.run_with_gradient(w.x - eps * dX, w.v - eps * dV, g, p, n_steps, weights)[0]
    fd = (Jp - Jm) / (2 * eps)
    ad = float(np.sum(gx * dX) + np.sum(gv * dV))
    assert ad == pytest.approx(fd, rel=1e-4)


def test_adjoint_rejects_small_buffers_and_missing_forward():
    w = _small()
    sim = Simulation.from_workload(w)
    buf = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.PicError) as e:
        capi.pic_adjoint_forward(sim.handle, 4, 2, (1.0, 1.0, 1.0), buf.data_ptr(), 1024)
    assert e.value.code == capi.PIC_ERR_CAPACITY
    with pytest.raises(capi.PicError) as e:
        sim.adjoint_backward()
    assert e.value.code == capi.PIC_ERR_STATE
    sim.close()


def test_directional_derivative_with_the_benchmark_settings():
    """The bump-on-tail velocity mixture and seed wave (k = 0.1, alpha = 0.05)
    on a 16^3 grid with 16 particles per cell (65,536 particles), 40 steps,
    the benchmark's launch settings (re-binning every 4 steps, fixed-point
    deposit), checkpoints every 20 steps: <dJ/d(x0, v0), delta> against the
    central difference of the oracle's J along delta."""
    import bench

    w = pi.bump_on_tail(n=16, ppc=16, seed=11)
    n_steps, weights = 40, (0.0, 0.0, 1.0)
    sim = Simulation.from_workload(w, **bench.LAUNCH)
    J = sim.adjoint_forward(n_steps, weights, checkpoint_every=20)
    gx, gv = sim.adjoint_backward()
    sim.close()
    rng = np.random.default_rng(5)
    dX, dV = rng.standard_normal(w.x.shape), rng.standard_normal(w.v.shape)
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q)
    eps = 1e-6
    Jp = po.run_with_gradient(w.x + eps * dX, w.v + eps * dV, g, p, n_steps, weights)[0]
    Jm = po.run_with_gradient(w.x - eps * dX, w.v - eps * dV, g, p, n_steps, weights)[0]
    fd = (Jp - Jm) / (2 * eps)
    ad = float(np.sum(gx * dX) + np.sum(gv * dV))
    J0 = po.run_with_gradient(w.x, w.v, g, p, n_steps, weights)[0]
    assert J == pytest.approx(J0, rel=1e-4)
    assert ad == pytest.approx(fd, rel=1e-3)


PARAMS = capi.PIC_OPT_ADJOINT_PARAMS


@pytest.mark.parametrize("wz2,B", [(0.3, (0.0, 0.0, 5.0)), (0.0, (1.0, -2.0, 3.0)),
                                   (0.3, (0.0, 0.0, 0.0))],
                         ids=["penning", "oblique-B", "quadrupole-B0"])
@pytest.mark.parametrize("every", [4, 5], ids=["checkpoints", "kept"])
def test_parameter_gradient_matches_oracle(wz2, B, every):
    """dJ/dB_ext and dJ/d(wz2) against the oracle's reverse sweep, with
    recomputed segments and with the trajectory kept; the state gradients are
    unchanged by the option."""
    w = _small()
    n_steps, weights = 6, (1.0, 1.0, 1.0)
    sim = Simulation.from_workload(w, wz2=wz2, B=B, options=FIXED | PARAMS)
    sim.adjoint_forward(n_steps, weights, checkpoint_every=every)
    gx, gv = sim.adjoint_backward()
    gp = np.asarray(sim.adjoint_param_gradient())
    sim.close()
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m, wz2=wz2, B=B)
    _, gxo, gvo, gBo, gwo = po.run_with_gradient(w.x, w.v, g, p, n_steps, weights,
                                                 param_grad=True)
    assert np.max(np.abs(gx - gxo)) <= 1e-4 * np.max(np.abs(gxo))
    assert np.max(np.abs(gv - gvo)) <= 1e-4 * np.max(np.abs(gvo))
    ref = np.append(gBo, gwo)
    assert np.max(np.abs(gp - ref)) <= 1e-4 * np.max(np.abs(ref)), (gp, ref)


def test_penning_parameter_gradient_against_central_differences_of_the_oracle():
    """A Penning bunch through 10 Boris steps: dJ/dB_z and dJ/d(wz2) from the
    GPU against central differences of the oracle's J in B_z and wz2."""
    w = pi.penning(n=16, n_particles=4096, L=20.0, seed=9)
    n_steps, weights = 10, (1.0, 1.0, 1.0)
    sim = Simulation.from_workload(w, options=FIXED | PARAMS)
    sim.adjoint_forward(n_steps, weights, checkpoint_every=4)
    sim.adjoint_backward()
    gp = sim.adjoint_param_gradient()
    sim.close()
    g = po.Grid(w.n, w.L)
    eps = 1e-5

    def J(B, wz2):
        p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m, B=B, wz2=wz2)
        return po.run_with_gradient(w.x, w.v, g, p, n_steps, weights)[0]

    Bz = w.B[2]
    fd_b = (J((w.B[0], w.B[1], Bz + eps), w.wz2) - J((w.B[0], w.B[1], Bz - eps), w.wz2)) / (2 * eps)
    fd_w = (J(w.B, w.wz2 + eps) - J(w.B, w.wz2 - eps)) / (2 * eps)
    assert gp[2] == pytest.approx(fd_b, rel=1e-3)
    assert gp[3] == pytest.approx(fd_w, rel=1e-3)


def test_parameter_gradient_needs_the_option_and_a_backward_pass():
    w = _small()
    sim = Simulation.from_workload(w, wz2=0.3, options=FIXED)
    sim.adjoint_forward(3, (1.0, 1.0, 1.0))
    sim.adjoint_backward()
    with pytest.raises(capi.PicError):
        sim.adjoint_param_gradient()
    sim.close()
    sim = Simulation.from_workload(w, wz2=0.3, options=FIXED | PARAMS)
    with pytest.raises(capi.PicError):
        sim.adjoint_param_gradient()
    sim.adjoint_forward(3, (1.0, 1.0, 1.0))
    with pytest.raises(capi.PicError):
        sim.adjoint_param_gradient()
    sim.adjoint_backward()
    assert np.all(np.isfinite(sim.adjoint_param_gradient()))
    sim.close()


def test_two_hundred_steps_at_the_benchmark_settings_against_stored_oracle_gradients():
    """The bump-on-tail adjoint workload's settings (velocity mixture,
    1 + 0.05 cos(k z), dt = 0.05, 200 steps, W_z of the last field) on a
    16^3 x 16 grid with the 64^3 workload's cell size, run as benchmarked:
    checkpoints every 20 steps, re-binning every 4, fixed-point deposit.
    Compared with the FP64 oracle's values stored by
    tests/golden/make_adjoint_goldens.py: J; dJ/dalpha against the oracle's
    central difference over re-sampled inputs (the gradient accuracy
    target, 1e-4); dJ/dx0 and dJ/dv0 of 512 particles against the oracle's
    discrete adjoint.  Over 200 steps of an unstable plasma the FP32 and
    FP64 trajectories separate, so the per-particle comparison is held to
    the looser bound the arithmetic supports (see the design notes)."""
    import json
    import os

    import bench

    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "bump_on_tail_16_adjoint_200.json")))
    s = gold["setup"]
    w = pi.bump_on_tail(n=s["n"], ppc=s["ppc"], seed=s["seed"], alpha=s["alpha"], k=s["k"])
    assert w.n_particles == s["n_particles"] and w.dt == s["dt"]
    sim = Simulation.from_workload(w, **bench.LAUNCH)
    J = sim.adjoint_forward(s["n_steps"], tuple(s["weights"]), checkpoint_every=20)
    gx, gv = sim.adjoint_backward(device=True)
    dxa = torch.zeros_like(gx)
    dxa[:, 2] = torch.from_numpy(pi.sample_cosine_density_dalpha(
        w.x[:, 2], s["alpha"], s["k"])).to(gx.device)
    dJ_da = sim.dot(gx, dxa)
    gx, gv = gx.cpu().numpy(), gv.cpu().numpy()
    sim.close()
    assert J == pytest.approx(gold["J"], rel=1e-5)
    assert dJ_da == pytest.approx(gold["dJ_dalpha_central_difference"], rel=1e-4)
    assert dJ_da == pytest.approx(gold["dJ_dalpha_adjoint"], rel=1e-4)
    idx = np.asarray(gold["sample"])
    ex = np.max(np.abs(gx[idx] - np.asarray(gold["gx"]))) / gold["max_abs_gx"]
    ev = np.max(np.abs(gv[idx] - np.asarray(gold["gv"]))) / gold["max_abs_gv"]
    print(f"200-step adjoint: J rel {abs(J / gold['J'] - 1):.2e}, dJ/dalpha rel "
          f"{abs(dJ_da / gold['dJ_dalpha_central_difference'] - 1):.2e}, "
          f"dJ/dx0 {ex:.2e}, dJ/dv0 {ev:.2e} of their maxima")
    # observed on a GB300: J 9e-7, dJ/dalpha 7e-6, dJ/dx0 5e-4 and dJ/dv0 5e-4
    # of their maxima; the per-particle gradients carry the FP32/FP64
    # separation of 200 unstable steps
    assert ex <= 2e-3 and ev <= 2e-3
