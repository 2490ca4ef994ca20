"""Pins of the FP64 oracle against what the scheme and the physics fix.

None of these compares the oracle with itself: each checks a closed form,
an invariant, a brute-force evaluation or textbook plasma theory, chosen so
that a dropped term, a wrong sign or index or a transposed axis fails.
"""
import math

import numpy as np
import pytest

import pic_inputs as pi
from oracle import pic_oracle as po
from tests import dispersion

RNG = np.random.default_rng(12345)

# a deliberately non-cubic grid so transposed axes show up
GRID = po.Grid(n=(6, 5, 8), L=(2.0, 3.1, 2.6))


def _random_positions(grid, n, rng):
    return rng.random((n, 3)) * np.asarray(grid.L)


# ---------------------------------------------------------------- deposit

def test_deposit_conserves_charge():
    """CIC weights sum to one, so h^3 sum_g rho_g = sum_p q_p (Section 3.2)."""
    x = _random_positions(GRID, 5000, RNG)
    q = -0.37
    rho = po.deposit(x, GRID, q)
    total = rho.sum() * GRID.cell_volume
    assert abs(total - q * x.shape[0]) <= 1e-13 * abs(q * x.shape[0])


def test_deposit_matches_bruteforce_tent_functions():
    """Floor-based stencil == node-by-node minimum-image tent functions."""
    for grid in (po.Grid((4, 3, 5), (1.0, 1.5, 2.0)), po.Grid((2, 6, 3), (3.0, 1.0, 0.7))):
        x = _random_positions(grid, 40, RNG)
        # include boundary cases: exactly 0, just below L, exactly on a node
        x[0] = 0.0
        x[1] = np.nextafter(np.asarray(grid.L), 0.0)
        x[2] = 0.5 * grid.h
        a = po.deposit(x, grid, 1.3)
        b = po.deposit_bruteforce(x, grid, 1.3)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_particle_on_node_deposits_to_that_node_only():
    grid = GRID
    h = grid.h
    g = (3, 2, 5)
    x = np.array([[(g[0] + 0.5) * h[0], (g[1] + 0.5) * h[1], (g[2] + 0.5) * h[2]]])
    rho = po.deposit(x, grid, 2.0)
    expect = np.zeros(grid.shape)
    expect[g[2], g[1], g[0]] = 2.0 / grid.cell_volume
    assert np.max(np.abs(rho - expect)) <= 1e-12 * expect.max()


def test_particle_midway_splits_evenly_across_the_periodic_seam():
    """x = 0 lies halfway between node N-1 (at L - h/2) and node 0 (at h/2)."""
    grid = po.Grid((4, 4, 4), (1.0, 1.0, 1.0))
    x = np.array([[0.0, 0.125, 0.125]])   # y, z on nodes 0
    rho = po.deposit(x, grid, 1.0) * grid.cell_volume
    assert rho[0, 0, 0] == pytest.approx(0.5, abs=1e-15)
    assert rho[0, 0, 3] == pytest.approx(0.5, abs=1e-15)
    assert rho.sum() == pytest.approx(1.0, abs=1e-15)


# ---------------------------------------------------------------- field solve

@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, -2, 1), (2, 1, -3)])
def test_single_mode_poisson_closed_form(m):
    """rho = cos(k.x) -> phi = cos(k.x)/|k|^2 -> E = k sin(k.x)/|k|^2 (Eq. potential)."""
    grid = po.Grid((8, 10, 12), (2.0, 3.0, 5.0))
    h = grid.h
    k = np.array([2 * math.pi * m[d] / grid.L[d] for d in range(3)])
    zz, yy, xx = np.meshgrid(*[(np.arange(grid.n[d]) + 0.5) * h[d] for d in (2, 1, 0)], indexing="ij")
    phase = k[0] * xx + k[1] * yy + k[2] * zz
    rho = np.cos(phase)
    E, phi = po.solve_field(rho, grid, return_potential=True)
    k2 = float(np.dot(k, k))
    for d in range(3):
        assert np.max(np.abs(E[d] - k[d] * np.sin(phase) / k2)) < 1e-12
    assert np.max(np.abs(phi - np.cos(phase) / k2)) < 1e-12


def test_uniform_background_only_removes_the_mean():
    grid = GRID
    rho = RNG.standard_normal(grid.shape)
    E1 = po.solve_field(rho, grid)
    E2 = po.solve_field(rho + 7.5, grid)
    assert np.max(np.abs(E1 - E2)) < 1e-12


def test_nyquist_gradient_is_zeroed():
    """A pure Nyquist density along x gives E_x = 0 (no derivative at k = pi/h)."""
    grid = po.Grid((8, 4, 4), (1.0, 1.0, 1.0))
    rho = np.zeros(grid.shape)
    rho[:, :, :] = (-1.0) ** np.arange(8)[None, None, :]
    E = po.solve_field(rho, grid)
    assert np.max(np.abs(E)) < 1e-13


# ------------------------------------------------- deposit / gather pairing

def test_zero_self_force():
    """A lone particle feels no force from its own field: the spectral
    gradient with zeroed Nyquist modes is an antisymmetric circulant and the
    gather uses the deposit's weights."""
    grid = GRID
    for _ in range(20):
        x = _random_positions(grid, 1, RNG)
        rho = po.deposit(x, grid, 1.0)
        E = po.solve_field(rho, grid)
        f = po.gather(x, E, grid)
        scale = np.max(np.abs(E))
        assert np.max(np.abs(f)) <= 1e-13 * scale


def test_momentum_conservation_of_self_forces():
    """sum_p q_p E(x_p) = h^3 sum_g rho_g E_g = 0 for any particle set."""
    grid = GRID
    x = _random_positions(grid, 3000, RNG)
    q = -0.2
    rho = po.deposit(x, grid, q)
    E = po.solve_field(rho, grid)
    F = q * po.gather(x, E, grid).sum(axis=0)
    scale = abs(q) * x.shape[0] * np.max(np.abs(E))
    assert np.max(np.abs(F)) <= 1e-13 * scale


def test_gather_is_transpose_of_deposit():
    """<G(x) E, w> = h^3 <E, D_w(x)> with the same CIC weights."""
    grid = GRID
    x = _random_positions(grid, 400, RNG)
    E = RNG.standard_normal((3,) + grid.shape)
    w = RNG.standard_normal((400, 3))
    lhs = float(np.sum(po.gather(x, E, grid) * w))
    rhs = sum(grid.cell_volume * float(np.sum(E[d] * po.deposit(x, grid, w[:, d]))) for d in range(3))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_mode_coefficient_of_a_cosine():
    grid = po.Grid((16, 8, 8), (4.0, 1.0, 1.0))
    xx = (np.arange(16) + 0.5) * grid.h[0]
    f = np.broadcast_to(0.3 * np.cos(2 * math.pi * xx / 4.0)[None, None, :], grid.shape)
    c = po.mode_coefficient(np.array(f), (1, 0, 0))
    assert abs(c) == pytest.approx(0.15, rel=1e-12)


# ---------------------------------------------------------------- push

def test_boris_pure_magnetic_rotation_angle():
    """With E = 0 the Boris rotation angle per step is 2 arctan(w_c dt / 2)."""
    B = (0.0, 0.0, 5.0)
    dt = 0.05       # w_c dt = |q/m| B dt = 0.25
    v = np.array([[1.0, 0.0, 0.3]])
    v1 = po.boris_kick(v, np.zeros((1, 3)), -1.0, B, dt)
    ang = math.atan2(v1[0, 1], v1[0, 0])
    assert abs(ang) == pytest.approx(2 * math.atan(0.125), abs=1e-14)
    assert abs(2 * math.atan(0.125) - 0.24870999) < 1e-8
    # q/m = -1, B along +z: electrons gyrate counter-clockwise seen from +z
    assert ang > 0
    assert np.linalg.norm(v1) == pytest.approx(np.linalg.norm(v), rel=1e-15)
    assert v1[0, 2] == v[0, 2]


def test_boris_without_b_is_a_plain_kick():
    e = RNG.standard_normal((5, 3))
    v = RNG.standard_normal((5, 3))
    v1 = po.boris_kick(v, e, -1.0, (0.0, 0.0, 0.0), 0.05)
    assert np.max(np.abs(v1 - (v - 0.05 * e))) < 1e-15


def test_free_streaming_step_and_wrap():
    grid = po.Grid((8, 8, 8), (1.0, 2.0, 3.0))
    x = np.array([[0.99, 1.0, 0.01]])
    v = np.array([[1.0, -0.5, -1.0]])
    p = po.Params(dt=0.05, Q=0.0)
    x1, v1 = po.step(x, v, grid, p)
    expect = np.mod(x + 0.05 * v, np.asarray(grid.L))
    assert np.max(np.abs(x1 - expect)) < 1e-15
    assert np.all(v1 == v)


def _trap_map(dt, wz2, Bz=5.0):
    """The 6x6 linear one-step map of a lone particle about the trap centre."""
    grid = po.Grid((8, 8, 8), (20.0, 20.0, 20.0))
    p = po.Params(dt=dt, Q=0.0, B=(0.0, 0.0, Bz), wz2=wz2)
    c = np.full(3, 10.0)
    M = np.empty((6, 6))
    eps = 1e-2
    for col in range(6):
        s = np.zeros(6)
        s[col] = eps
        x1, v1 = po.step((c + s[:3])[None], s[3:][None], grid, p)
        M[:, col] = np.concatenate([x1[0] - c, v1[0]]) / eps
    return M


@pytest.mark.parametrize("wz2", [1.0, 1.5])
def test_penning_single_particle_frequencies(wz2):
    """Cyclotron, magnetron (E x B) and axial frequencies of the ideal trap:
    w+- = (wc +- sqrt(wc^2 - 2 wz^2)) / 2, wz = sqrt(wz2) (Section 4.3)."""
    wc = 5.0
    dt = 0.005
    lam = np.linalg.eigvals(_trap_map(dt, wz2))
    freqs = sorted(set(np.round(np.abs(np.angle(lam)) / dt, 9)))
    wp = 0.5 * (wc + math.sqrt(wc * wc - 2 * wz2))
    wm = 0.5 * (wc - math.sqrt(wc * wc - 2 * wz2))
    expect = sorted([wm, math.sqrt(wz2), wp])
    assert len(freqs) == 3
    for f, e in zip(freqs, expect):
        assert f == pytest.approx(e, rel=1e-3)
    if wz2 == 1.0:
        assert wp == pytest.approx(4.89792, abs=1e-5)
        assert wm == pytest.approx(0.10208, abs=1e-5)
    # the map is symplectic-like: every eigenvalue on the unit circle
    assert np.max(np.abs(np.abs(lam) - 1.0)) < 1e-12


# ---------------------------------------------------------------- physics

def test_dispersion_root_for_landau_k_half():
    w = dispersion.root(0.5, 1.4 - 0.15j)
    assert w.real == pytest.approx(1.41566, abs=2e-5)
    assert w.imag == pytest.approx(-0.15336, abs=2e-5)


@pytest.mark.slow
def test_landau_damping_rate_and_frequency():
    """Weak Landau damping, k = 0.5 (Section 4.1, Eq. landau_f): the x mode
    of E_x oscillates at Re(w) and decays at Im(w) of the kinetic dispersion
    relation.  Quiet 1D lattice start (32 cells, 128 x 1024 particles) at
    alpha = 0.01, small enough that the linear rate holds; the least damped
    root is separated from the ballistic transient and the heavier roots by
    a six-exponential matrix pencil on t in [4, 14].  The grid's CIC
    smoothing alone moves the root by 0.7% at this resolution."""
    from tests.fits import pencil

    w = pi.landau_lattice_1d(nx=32, mx=128, mv=1024, alpha=0.01, n_steps=300)
    grid = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    _, _, hist = po.run(w.x, w.v, grid, p, w.n_steps)
    t = np.array([d["t_field"] for d in hist])
    c = np.array([d["mode"] for d in hist])
    root = dispersion.root(0.5, 1.4 - 0.15j)
    sel = (t >= 4.0) & (t <= 14.0)
    s, a = pencil(c[sel], t[1] - t[0], 6)
    near = [i for i in range(len(s)) if abs(abs(s[i].imag) - root.real) < 0.1]
    i = max(near, key=lambda j: abs(a[j]))
    assert s[i].real == pytest.approx(root.imag, rel=0.02)
    assert abs(s[i].imag) == pytest.approx(root.real, rel=0.005)
    # charge is exact and the lattice start has zero net momentum
    assert hist[-1]["Q"] == pytest.approx(w.Q, rel=1e-13)
    assert abs(hist[-1]["Px"]) < 1e-9 * abs(w.Q)


def test_bump_on_tail_growth_rate_on_a_quiet_lattice():
    """Bump-on-tail (Section 4.2 family): electrons 0.9 N(0,1) + 0.1 N(4, 0.3^2),
    seeded at k = 0.3 with alpha = 1e-3 on a quiet 1D lattice (32 cells,
    64 x 512 particles).  The most strongly growing root fitted on t in
    [5, 20] matches the two-Maxwellian dispersion root 0.92925 + 0.21093i."""
    from tests.fits import fastest_root

    w = pi.bump_on_tail_quiet(n=(32, 1, 1), L=2.0 * math.pi / 0.3, axis=0, m=1, alpha=1e-3,
                              ms=64, mv=512)
    grid = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    _, _, hist = po.run(w.x, w.v, grid, p, 400)
    t = np.array([d["t_field"] for d in hist])
    c = np.array([d["mode"] for d in hist])
    gamma, omega = fastest_root(t, c, 5.0, 20.0)
    root = dispersion.root(0.3, 0.93 + 0.21j, species=((0.9, 0.0, 1.0), (0.1, 4.0, 0.3)))
    assert gamma == pytest.approx(root.imag, rel=0.02)
    assert omega == pytest.approx(root.real, rel=0.005)


def test_two_stream_growth_rate_on_a_quiet_lattice():
    """Symmetric two-stream instability (Section 4.2, Eq. twostream_f: beams at
    v = -pi/2 and +pi/2 with spread 0.1, k = 0.5), seeded with alpha = 1e-3
    on a quiet 1D lattice (32 cells, 64 x 512 particles).  The fastest root
    fitted on t in [4, 18] is purely growing at the kinetic root 0.31824i."""
    from tests.fits import fastest_root

    w = pi.bump_on_tail_quiet(n=(32, 1, 1), L=4.0 * math.pi, axis=0, m=1, alpha=1e-3, ms=64,
                              mv=512, eps=0.5, v_beam=0.5 * math.pi, sigma_beam=0.1,
                              sigma_bulk=0.1, u_bulk=-0.5 * math.pi)
    grid = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    _, _, hist = po.run(w.x, w.v, grid, p, 400)
    t = np.array([d["t_field"] for d in hist])
    c = np.array([d["mode"] for d in hist])
    gamma, omega = fastest_root(t, c, 4.0, 18.0)
    root = dispersion.root(0.5, 0.3j, species=((0.5, -0.5 * math.pi, 0.1),
                                              (0.5, 0.5 * math.pi, 0.1)))
    assert abs(root.real) < 1e-9
    assert gamma == pytest.approx(root.imag, rel=0.02)
    assert omega < 0.01


def test_splitmix64_matches_its_published_outputs():
    """The first outputs of SplitMix64 from seeds 0 and 1234567 as published
    with the generator's reference implementation."""
    c = np.array([1, 2, 3], dtype=np.uint64)
    assert [int(r) for r in po.splitmix64(0, c)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                    0x06C45D188009454F]
    assert [int(r) for r in po.splitmix64(1234567, c[:2])] == [6457827717110365317,
                                                              3203168211198807973]


def test_uniform_displacements_are_uniform_and_keep_velocities():
    """Section 4.4: displacements fill [-1, 1) cells uniformly (mean 0,
    variance 1/3), differ by step, particle and axis, and the step leaves
    the velocities alone."""
    d = po.uniform_displacement(5, np.arange(200_000), seed=7)
    assert d.min() >= -1.0 and d.max() < 1.0
    assert abs(d.mean()) < 3e-3 and abs(d.var() - 1.0 / 3.0) < 3e-3
    assert not np.array_equal(d, po.uniform_displacement(6, np.arange(200_000), seed=7))
    assert abs(np.corrcoef(d[:, 0], d[:, 1])[0, 1]) < 1e-2
    w = pi.uniform_plasma(n=8, ppc=4, seed=3)
    g = po.Grid(w.n, w.L)
    x1, v1 = po.step_uniform(w.x, w.v, g, po.Params(dt=0.05, Q=w.Q), 0, seed=7)
    assert np.array_equal(v1, w.v)
    dx = x1 - w.x
    dx -= np.asarray(w.L) * np.round(dx / np.asarray(w.L))
    assert np.all(np.abs(dx) <= np.asarray(g.h) + 1e-12)


def test_diagnostics_field_energy_of_a_known_field():
    grid = po.Grid((8, 8, 8), (2.0, 2.0, 2.0))
    E = np.zeros((3,) + grid.shape)
    E[1] = 3.0
    d = po.diagnostics(np.ones(grid.shape), E, None, grid, po.Params(dt=0.1, Q=-8.0), 0)
    assert d["Wy"] == pytest.approx(9.0 * 8.0, rel=1e-14)
    assert d["Wx"] == 0.0 and d["Wz"] == 0.0
    assert d["Q"] == pytest.approx(8.0, rel=1e-14)


def test_diagnostics_momentum_and_kinetic_energy_of_two_particles():
    """Two electrons of a species with Q_e = -3 and q/m = -2 (Section 3.2:
    q_p = -1.5, m_p = q_p / (q/m) = 0.75) moving at (1, 2, 3) and (-3, 0, 1):
    the total momentum is (-1.5, 1.5, 3) and the kinetic energy 9, worked
    out by hand."""
    grid = po.Grid((4, 4, 4), (2.0, 2.0, 2.0))
    v = np.array([[1.0, 2.0, 3.0], [-3.0, 0.0, 1.0]])
    E = np.zeros((3,) + grid.shape)
    d = po.diagnostics(np.zeros(grid.shape), E, v, grid, po.Params(dt=0.1, Q=-3.0, q_over_m=-2.0), 2)
    assert (d["Px"], d["Py"], d["Pz"]) == pytest.approx((-1.5, 1.5, 3.0), rel=1e-15)
    assert d["K"] == pytest.approx(9.0, rel=1e-15)


def _work_and_impulse_residuals(n_steps=6):
    """Run a strongly driven Penning-like bunch (self field, quadrupole and
    B) and return the largest residuals of the work-energy theorem
    K_{n+1} - K_n = sum_p q_p e_p . (x_{n+1} - x_n) and of the Lorentz
    impulse P_{n+1} - P_n = sum_p q_p (dt e_p + (x_{n+1} - x_n) x B),
    relative to |K| and |P| scales.  Both hold exactly for the synchronised
    Boris step: the rotation does no work and v_{n+1} - v_n solves
    v1 = v0 + dt (q/m) [e + (v0 + v1)/2 x B] (Eq. momentum_eqn), while the
    drift-kick-drift positions move by dt (v_n + v_{n+1}) / 2.  The field e_p
    is the gathered self field plus the quadrupole at the half-step
    position; displacements come from the positions alone (minimum image)."""
    w = pi.landau(n=8, ppc=4, seed=11, alpha=0.4)
    grid = po.Grid(w.n, w.L)
    B = np.array([0.3, -0.2, 2.0])
    p = po.Params(dt=0.1, Q=w.Q, q_over_m=-1.7, B=tuple(B), wz2=0.8)
    L = np.asarray(w.L)
    N = w.x.shape[0]
    qp = p.Q / N
    x, v = w.x.copy(), w.v.copy()
    prev = None
    res_k = res_p = 0.0
    for _ in range(n_steps):
        xh = po.wrap(x + 0.5 * p.dt * v, grid)
        e = po.gather(xh, po.solve_field(po.deposit(xh, grid, qp), grid), grid)
        e = e + po.external_field(xh, grid, p.wz2)
        x1, v1, d = po.step(x, v, grid, p, with_diag=True)
        dx = x1 - x
        dx -= L * np.round(dx / L)
        if prev is not None:
            work = qp * float(np.sum(e * dx))
            impulse = qp * (p.dt * e.sum(axis=0) + np.cross(dx, B).sum(axis=0))
            dK = d["K"] - prev["K"]
            dP = np.array([d["Px"] - prev["Px"], d["Py"] - prev["Py"], d["Pz"] - prev["Pz"]])
            res_k = max(res_k, abs(dK - work) / abs(work))
            res_p = max(res_p, float(np.max(np.abs(dP - impulse))) / float(np.max(np.abs(impulse))))
        prev = d
        x, v = x1, v1
    return res_k, res_p


def test_kinetic_energy_and_momentum_follow_work_and_impulse():
    """K and P of the diagnostics change by exactly the work and the impulse
    of the fields on the particles (see _work_and_impulse_residuals): this
    fixes the 1/2 of K, m_p = q_p / (q/m) with its sign and the sums over
    particles independently of how the diagnostics are written."""
    res_k, res_p = _work_and_impulse_residuals()
    assert res_k < 1e-9
    assert res_p < 1e-9


@pytest.mark.parametrize("mistake", ["K without 1/2", "m_p with the wrong sign", "P without m_p"])
def test_work_and_impulse_pins_catch_planted_mistakes(monkeypatch, mistake):
    """The pin above fails for each plausible slip in the oracle's K and P."""
    good = po.diagnostics

    def planted(rho, E, v_new, grid, params, n_particles, mode=(1, 0, 0), mode_comp=0):
        d = good(rho, E, v_new, grid, params, n_particles, mode, mode_comp)
        mp = params.Q / n_particles / params.q_over_m
        if mistake == "K without 1/2":
            d["K"] *= 2.0
        elif mistake == "m_p with the wrong sign":
            d["K"], d["Px"], d["Py"], d["Pz"] = -d["K"], -d["Px"], -d["Py"], -d["Pz"]
        else:
            d["Px"], d["Py"], d["Pz"] = d["Px"] / mp, d["Py"] / mp, d["Pz"] / mp
        return d

    monkeypatch.setattr(po, "diagnostics", planted)
    res_k, res_p = _work_and_impulse_residuals(n_steps=3)
    assert max(res_k, res_p) > 0.5


def test_momentum_is_conserved_by_the_self_field():
    """With B = E_ext = 0 only the self field acts, whose forces sum to zero
    (CIC deposit and gather are transposes, the spectral gradient is odd), so
    P stays at its nonzero initial value to rounding over 20 steps."""
    w = pi.landau(n=8, ppc=8, seed=21, alpha=0.3)
    grid = po.Grid(w.n, w.L)
    p = po.Params(dt=0.1, Q=w.Q)
    v0 = w.v + np.array([0.3, -0.2, 0.1])
    mp = (w.Q / w.x.shape[0]) / p.q_over_m
    P0 = mp * v0.sum(axis=0)
    _, _, hist = po.run(w.x, v0, grid, p, 20)
    scale = abs(mp) * float(np.sum(np.abs(v0)))
    for d in hist:
        P = np.array([d["Px"], d["Py"], d["Pz"]])
        assert np.max(np.abs(P - P0)) < 1e-12 * scale
    assert np.max(np.abs(P0)) > 1e-3 * scale


@pytest.mark.parametrize("Bz", [0.0, 5.0])
def test_time_reversibility_with_self_field(Bz):
    """The drift-kick-drift step with the field taken at x_{n+1/2} is exactly
    time-reversible: stepping (x_n, -v_n) under -B retraces the orbit.  An
    evaluation of the self or external field at x_n instead breaks this."""
    w = pi.landau(n=8, ppc=4, seed=7, alpha=0.3)
    grid = po.Grid(w.n, w.L)
    fwd = po.Params(dt=0.1, Q=w.Q, B=(0.0, 0.0, Bz), wz2=0.2)
    bwd = po.Params(dt=0.1, Q=w.Q, B=(0.0, 0.0, -Bz), wz2=0.2)
    x, v = w.x.copy(), w.v.copy()
    for _ in range(5):
        x, v = po.step(x, v, grid, fwd)
    v = -v
    for _ in range(5):
        x, v = po.step(x, v, grid, bwd)
    dx = x - w.x
    dx -= np.asarray(grid.L) * np.round(dx / np.asarray(grid.L))
    assert np.max(np.abs(dx)) < 1e-10
    assert np.max(np.abs(-v - w.v)) < 1e-10


# ---------------------------------------------------------------- adjoint

def test_field_solve_transpose_identity():
    """<S rho, lamE> = <rho, S^T lamE> for the spectral field operator."""
    grid = GRID
    rho = RNG.standard_normal(grid.shape)
    lamE = RNG.standard_normal((3,) + grid.shape)
    lhs = float(np.sum(po.solve_field(rho, grid) * lamE))
    rhs = float(np.sum(rho * po.solve_field_transpose(lamE, grid)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_cic_weight_gradients_are_derivatives_of_the_weights():
    grid = GRID
    x = _random_positions(grid, 50, RNG)
    nodes, w, dw = po.cic_weight_gradients(x, grid)
    eps = 1e-7 * float(np.min(grid.h))
    for j in range(3):
        e = np.zeros(3)
        e[j] = eps
        n_p, w_p = po.cic_stencil(x + e, grid)
        n_m, w_m = po.cic_stencil(x - e, grid)
        same = np.all(n_p == nodes, axis=1) & np.all(n_m == nodes, axis=1)
        fd = (w_p - w_m) / (2 * eps)
        assert np.max(np.abs(fd[same] - dw[same, :, j])) < 1e-6 / float(np.min(grid.h))


@pytest.mark.parametrize("wz2,weights,B", [(0.0, (0.0, 0.0, 1.0), (0.0, 0.0, 0.0)),
                                           (0.3, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0)),
                                           (0.3, (1.0, 1.0, 1.0), (0.0, 0.0, 5.0)),
                                           (0.0, (0.0, 1.0, 1.0), (1.0, -2.0, 3.0))])
def test_adjoint_matches_central_differences(wz2, weights, B):
    """Directional derivative of J along a random (dx0, dv0) equals the
    adjoint's inner product (J = final weighted field energy, 6 steps), with
    and without the Boris rotation (R^T in the reverse step)."""
    w = pi.bump_on_tail(n=8, ppc=4, seed=5, alpha=0.2, k=0.5)
    grid = po.Grid(w.n, w.L)
    p = po.Params(dt=0.1, Q=w.Q, wz2=wz2, B=B)
    J, dx, dv = po.run_with_gradient(w.x, w.v, grid, p, 6, weights)
    rng = np.random.default_rng(1)
    dX = rng.standard_normal(w.x.shape)
    dV = rng.standard_normal(w.v.shape)
    eps = 1e-5
    Jp = po.run_with_gradient(w.x + eps * dX, w.v + eps * dV, grid, p, 6, weights)[0]
    Jm = po.run_with_gradient(w.x - eps * dX, w.v - eps * dV, grid, p, 6, weights)[0]
    fd = (Jp - Jm) / (2 * eps)
    ad = float(np.sum(dx * dX) + np.sum(dv * dV))
    assert abs(fd - ad) <= 1e-6 * abs(ad)


def test_boris_rotation_matrix_is_the_kick_without_field():
    """R from the unit-vector kicks is orthogonal, rotates about B by
    2 arctan(|q/m| |B| dt / 2), and reproduces boris_kick for any (v, e)."""
    p = po.Params(dt=0.05, Q=-1.0, B=(0.0, 0.0, 5.0))
    R = po.boris_rotation(p)
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
    ang = math.atan2(R[1, 0], R[0, 0])
    assert abs(abs(ang) - 2.0 * math.atan(0.5 * 5.0 * 0.05)) < 1e-14
    rng = np.random.default_rng(2)
    v, e = rng.standard_normal(3), rng.standard_normal(3)
    h = 0.5 * p.dt * p.q_over_m
    kick = po.boris_kick(v, e, p.q_over_m, p.B, p.dt)
    assert np.allclose(kick, R @ v + h * (R @ e + e), atol=1e-14)


def test_gradient_with_respect_to_the_perturbation_amplitude():
    """dJ/dalpha through the inverse-transform sample x0(u; alpha) (fixed u)
    equals the central difference of J over regenerated particles."""
    alpha, k = 0.2, 0.5
    grid_args = dict(n=8, ppc=4, seed=5, k=k)
    w = pi.bump_on_tail(alpha=alpha, **grid_args)
    grid = po.Grid(w.n, w.L)
    p = po.Params(dt=0.1, Q=w.Q)
    wts = (0.0, 0.0, 1.0)
    J, dx, _ = po.run_with_gradient(w.x, w.v, grid, p, 6, wts)
    dadz = po.cosine_sample_dalpha(w.x[:, 2], alpha, k)
    ad = float(np.sum(dx[:, 2] * dadz))
    eps = 1e-6
    wp = pi.bump_on_tail(alpha=alpha + eps, **grid_args)
    wm = pi.bump_on_tail(alpha=alpha - eps, **grid_args)
    assert np.array_equal(wp.v, w.v) and np.array_equal(wp.x[:, :2], w.x[:, :2])
    fd = (po.run_with_gradient(wp.x, wp.v, grid, p, 6, wts)[0]
          - po.run_with_gradient(wm.x, wm.v, grid, p, 6, wts)[0]) / (2 * eps)
    assert abs(fd - ad) <= 1e-5 * abs(ad)


@pytest.mark.parametrize("wz2,B", [(0.3, (0.0, 0.0, 5.0)), (0.0, (1.0, -2.0, 3.0)),
                                   (0.3, (0.0, 0.0, 0.0))])
def test_parameter_gradients_match_central_differences(wz2, B):
    """dJ/dB_k and dJ/d(wz2) from the reverse sweep equal central differences
    of J over the field parameters (the particles' initial state fixed),
    including the sensitivity to a magnetic field at B = 0."""
    w = pi.bump_on_tail(n=8, ppc=4, seed=5, alpha=0.2, k=0.5)
    grid = po.Grid(w.n, w.L)
    wts = (1.0, 1.0, 1.0)
    p = po.Params(dt=0.1, Q=w.Q, wz2=wz2, B=B)
    J, _, _, gB, gw = po.run_with_gradient(w.x, w.v, grid, p, 6, wts, param_grad=True)
    eps = 1e-5
    for k in range(3):
        Bp = list(B)
        Bm = list(B)
        Bp[k] += eps
        Bm[k] -= eps
        Jp = po.run_with_gradient(w.x, w.v, grid, po.Params(dt=0.1, Q=w.Q, wz2=wz2, B=tuple(Bp)), 6, wts)[0]
        Jm = po.run_with_gradient(w.x, w.v, grid, po.Params(dt=0.1, Q=w.Q, wz2=wz2, B=tuple(Bm)), 6, wts)[0]
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - gB[k]) <= 1e-6 * max(abs(fd), 1e-3 * J), (k, fd, gB[k])
    Jp = po.run_with_gradient(w.x, w.v, grid, po.Params(dt=0.1, Q=w.Q, wz2=wz2 + eps, B=B), 6, wts)[0]
    Jm = po.run_with_gradient(w.x, w.v, grid, po.Params(dt=0.1, Q=w.Q, wz2=wz2 - eps, B=B), 6, wts)[0]
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - gw) <= 1e-6 * max(abs(fd), 1e-3 * J), (fd, gw)


def test_boris_rotation_derivative_matches_central_differences():
    """boris_rotation_dt against central differences of the rotation in t."""
    rng = np.random.default_rng(4)
    vm = rng.standard_normal((5, 3))
    t = np.array([0.3, -0.2, 0.5])
    d = po.boris_rotation_dt(vm, t)

    def f(tt):
        s = 2.0 * tt / (1.0 + float(np.dot(tt, tt)))
        return vm + np.cross(vm + np.cross(vm, tt), s)

    eps = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        fd = (f(t + e) - f(t - e)) / (2 * eps)
        assert np.max(np.abs(fd - d[:, k, :])) < 1e-8
