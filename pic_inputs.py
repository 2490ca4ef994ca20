"""Seeded synthetic workloads for the electrostatic PIC step (inputs only).

This module draws initial particle phase space for the mini-apps of the paper
(Section 4: Landau damping, bump-on-tail / two-stream, Penning trap, uniform
plasma) and returns plain FP64 arrays.  It holds none of the PIC method's
arithmetic (no deposit, field solve, gather or push): both the CUDA path and
the FP64 oracle consume what it returns, so parity measures only the method.

Sampling follows Section 3.2: separable densities are drawn by inverse
transform sampling (Newton iteration on the CDF), Maxwellians by normal
draws.  Every draw comes from ``numpy.random.Generator(PCG64(seed))`` so runs
are deterministic (the paper's device RNG is only statistically
reproducible; here the seed fixes every value).  An optional "quiet start"
replaces the pseudo-random uniforms with a randomly shifted Halton sequence,
which lowers sampling noise for the damping-rate checks on small problems.

Positions are returned as an (N, 3) array in [0, L_d), velocities as (N, 3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "landau",
    "bump_on_tail",
    "two_stream",
    "penning",
    "uniform_plasma",
    "single_particle",
    "halton",
    "by_name",
]


@dataclasses.dataclass
class Workload:
    """One initial condition plus the physical parameters it is run with."""

    name: str
    n: tuple            # grid nodes (Nx, Ny, Nz)
    L: tuple            # box lengths (Lx, Ly, Lz); periodic box [0, L)^3
    x: np.ndarray       # (N, 3) float64 positions
    v: np.ndarray       # (N, 3) float64 velocities
    q_over_m: float     # -1 for electrons in normalised units (Section 3.2)
    Q: float            # total electron charge Q_e
    dt: float
    B: tuple = (0.0, 0.0, 0.0)   # uniform external magnetic field
    wz2: float = 0.0             # quadrupole strength (axial frequency squared)
    n_steps: int = 20
    mode: tuple = (1, 0, 0)      # Fourier mode tracked by the diagnostics
    mode_comp: int = 0           # field component of that mode (0=x, 1=y, 2=z)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_particles(self) -> int:
        return int(self.x.shape[0])


# --------------------------------------------------------------------------
# uniform sources
# --------------------------------------------------------------------------

def _vdc(idx: np.ndarray, base: int) -> np.ndarray:
    """Radical inverse of integers ``idx`` in ``base`` (van der Corput)."""
    out = np.zeros(idx.shape, dtype=np.float64)
    f = 1.0 / base
    i = idx.astype(np.int64).copy()
    scale = f
    while np.any(i > 0):
        out += (i % base) * scale
        i //= base
        scale *= f
    return out


_PRIMES = (2, 3, 5, 7, 11, 13, 17, 19)


def halton(n: int, dim: int, rng: np.random.Generator, start: int = 1) -> np.ndarray:
    """(n, dim) Halton points with a random Cranley-Patterson shift per axis."""
    idx = np.arange(start, start + n, dtype=np.int64)
    shift = rng.random(dim)
    cols = [np.mod(_vdc(idx, _PRIMES[d]) + shift[d], 1.0) for d in range(dim)]
    return np.stack(cols, axis=1)


def _normals_from_uniform(u: np.ndarray) -> np.ndarray:
    from scipy.special import ndtri

    # keep strictly inside (0, 1) so the inverse CDF stays finite
    eps = 1e-12
    return ndtri(np.clip(u, eps, 1.0 - eps))


# --------------------------------------------------------------------------
# inverse transform sampling of 1 + alpha cos(k x) on [0, L)
# --------------------------------------------------------------------------

def sample_cosine_density(u: np.ndarray, L: float, alpha: float, k: float,
                          iters: int = 4) -> np.ndarray:
    """Invert F(x) = (x + (alpha/k) sin(k x)) / L = u by Newton iteration.

    Valid when k L is a multiple of 2 pi (the perturbation integrates to zero)
    and |alpha| < 1 (F strictly increasing).  The start x0 = uL - (alpha/k)
    sin(k uL) is exact to first order in alpha, so a few quadratically
    converging steps reach rounding level; more are taken if the residual says
    so.  The map u -> x is smooth in alpha.
    """
    target = u * L
    x = target - (alpha / k) * np.sin(k * target)
    for it in range(64):
        g = x + (alpha / k) * np.sin(k * x) - target
        dg = 1.0 + alpha * np.cos(k * x)
        x -= g / dg
        np.clip(x, 0.0, L, out=x)
        if it + 1 >= iters and np.max(np.abs(g), initial=0.0) < 1e-13 * L:
            break
    x = np.where(x >= L, 0.0, x)
    return x


def sample_cosine_density_dalpha(x: np.ndarray, alpha: float, k: float) -> np.ndarray:
    """Derivative in alpha of the sample sample_cosine_density(u, L, alpha, k)
    at fixed u, expressed through the sample x itself: differentiating
    x + (alpha/k) sin(k x) = u L gives dx/dalpha = -(sin(k x)/k) / (1 + alpha cos(k x)).
    The Jacobian of this input generator, for gradients of a run with respect
    to the perturbation amplitude."""
    return -(np.sin(k * x) / k) / (1.0 + alpha * np.cos(k * x))


def _chunked(N: int, seed: int, chunk: int, fill, workers=None):
    """Run fill(rng, start, stop) over [0, N) in chunks, each with its own
    stream spawned from ``seed`` (deterministic for any worker count)."""
    import concurrent.futures as cf
    import os

    starts = list(range(0, N, chunk))
    seqs = np.random.SeedSequence(seed).spawn(max(1, len(starts)))
    jobs = [(np.random.Generator(np.random.PCG64(seqs[i])), s, min(N, s + chunk))
            for i, s in enumerate(starts)]
    nw = workers or min(len(jobs), os.cpu_count() or 1, 32)
    if nw <= 1 or len(jobs) <= 1:
        for j in jobs:
            fill(*j)
        return
    with cf.ThreadPoolExecutor(max_workers=nw) as ex:
        list(ex.map(lambda j: fill(*j), jobs))


def _wrap(x: np.ndarray, L) -> np.ndarray:
    L = np.asarray(L, dtype=np.float64)
    y = np.mod(x, L)
    return np.where(y >= L, 0.0, y)


# --------------------------------------------------------------------------
# mini-apps
# --------------------------------------------------------------------------

def landau(n=16, ppc=8, alpha=0.05, k=0.5, seed=1000, dt=0.05, n_steps=20,
           form="product", quiet=False, chunk=1 << 20) -> Workload:
    """Landau damping initial condition (Section 4.1, Eq. landau_f).

    ``form="product"`` draws the paper's density
    (1 + a cos kx)(1 + a cos ky)(1 + a cos kz) per axis by inverse transform;
    ``form="literal"`` draws 1 + a cos kx cos ky cos kz by rejection.
    Velocities are Maxwellian with unit thermal speed.  Q_e = -L^3.
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(int(a) for a in n)
    L = 2.0 * math.pi / k
    Ls = (L, L, L)
    N = int(nn[0] * nn[1] * nn[2] * ppc)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((N, 3), dtype=np.float64)
    v = np.empty((N, 3), dtype=np.float64)
    if form == "product":
        if quiet:
            shift = rng.random(6)
            for s in range(0, N, chunk):
                e = min(N, s + chunk)
                idx = np.arange(s + 1, e + 1, dtype=np.int64)
                u = np.stack([np.mod(_vdc(idx, _PRIMES[d]) + shift[d], 1.0)
                              for d in range(6)], axis=1)
                for d in range(3):
                    x[s:e, d] = sample_cosine_density(u[:, d], L, alpha, k)
                v[s:e] = _normals_from_uniform(u[:, 3:6])
        else:
            def fill(g, s, e):
                u = g.random((e - s, 3))
                for d in range(3):
                    x[s:e, d] = sample_cosine_density(u[:, d], L, alpha, k)
                v[s:e] = g.standard_normal((e - s, 3))

            _chunked(N, seed, chunk, fill)
    elif form == "literal":
        filled = 0
        while filled < N:
            m = int((N - filled) * 1.2) + 64
            cand = rng.random((m, 3)) * L
            acc = rng.random(m) * (1.0 + abs(alpha))
            dens = 1.0 + alpha * np.cos(k * cand[:, 0]) * np.cos(k * cand[:, 1]) * np.cos(k * cand[:, 2])
            keep = cand[acc < dens]
            take = min(N - filled, keep.shape[0])
            x[filled:filled + take] = keep[:take]
            filled += take
        v[:] = rng.standard_normal((N, 3))
    else:
        raise ValueError(f"unknown density form {form!r}")
    x = _wrap(x, Ls)
    return Workload(name=f"landau_{nn[0]}x{nn[1]}x{nn[2]}_ppc{ppc}", n=nn, L=Ls, x=x, v=v,
                    q_over_m=-1.0, Q=-(L ** 3), dt=dt, n_steps=n_steps, mode=(1, 0, 0),
                    mode_comp=0, meta=dict(alpha=alpha, k=k, form=form, seed=seed,
                                           ppc=ppc, quiet=quiet))


def bump_on_tail(n=64, ppc=16, alpha=0.05, k=0.1, seed=1003, dt=0.05, n_steps=200,
                 eps=0.1, v_beam=4.0, sigma_beam=0.3, sigma_bulk=1.0, chunk=1 << 20) -> Workload:
    """Bump-on-tail initial condition on [0, 2 pi / k)^3.

    Density 1 + alpha cos(k z) (Eq. twostream_f's spatial factor) drawn by
    inverse transform in z, uniform in x and y.  v_x, v_y ~ N(0, sigma_bulk^2);
    v_z from the mixture (1 - eps) N(0, sigma_bulk^2) + eps N(v_beam, sigma_beam^2).
    The default parameters are the bump-on-tail adjoint workload (64^3 grid,
    16 particles per cell, k = 0.1, alpha = 0.05, eps = 0.1, beam 4 +- 0.3).
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(int(a) for a in n)
    L = 2.0 * math.pi / k
    Ls = (L, L, L)
    N = int(nn[0] * nn[1] * nn[2] * ppc)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((N, 3), dtype=np.float64)
    v = np.empty((N, 3), dtype=np.float64)
    def fill(r, s, e):
        m = e - s
        u = r.random((m, 3))
        x[s:e, 0] = u[:, 0] * L
        x[s:e, 1] = u[:, 1] * L
        x[s:e, 2] = sample_cosine_density(u[:, 2], L, alpha, k)
        g = r.standard_normal((m, 3))
        beam = r.random(m) < eps
        v[s:e, 0] = sigma_bulk * g[:, 0]
        v[s:e, 1] = sigma_bulk * g[:, 1]
        v[s:e, 2] = np.where(beam, v_beam + sigma_beam * g[:, 2], sigma_bulk * g[:, 2])

    _chunked(N, seed, chunk, fill)
    x = _wrap(x, Ls)
    return Workload(name=f"bump_on_tail_{nn[0]}x{nn[1]}x{nn[2]}_ppc{ppc}", n=nn, L=Ls, x=x, v=v,
                    q_over_m=-1.0, Q=-(L ** 3), dt=dt, n_steps=n_steps, mode=(0, 0, 1),
                    mode_comp=2, meta=dict(alpha=alpha, k=k, eps=eps, v_beam=v_beam,
                                           sigma_beam=sigma_beam, seed=seed, ppc=ppc))


def two_stream(n=32, ppc=8, alpha=0.01, k=0.5, seed=1005, dt=0.05, n_steps=200,
               eps=0.5, sigma=0.1, vb1=-math.pi / 2, vb2=math.pi / 2, chunk=1 << 20) -> Workload:
    """Two-stream / bump-on-tail family with equal thermal spread (Eq. twostream_f).

    The paper's two-stream case is eps = 0.5, sigma = 0.1, k = 0.5,
    alpha = 0.01, beams at v_z = -pi/2 and +pi/2; its bump-on-tail case is
    eps = 0.1, sigma = 1/sqrt(2), k = 0.21, alpha = 0.01, beams at 0 and 4.
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(int(a) for a in n)
    L = 2.0 * math.pi / k
    Ls = (L, L, L)
    N = int(nn[0] * nn[1] * nn[2] * ppc)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((N, 3), dtype=np.float64)
    v = np.empty((N, 3), dtype=np.float64)
    def fill(r, s, e):
        m = e - s
        u = r.random((m, 3))
        x[s:e, 0] = u[:, 0] * L
        x[s:e, 1] = u[:, 1] * L
        x[s:e, 2] = sample_cosine_density(u[:, 2], L, alpha, k)
        g = r.standard_normal((m, 3))
        second = r.random(m) < eps
        v[s:e] = sigma * g
        v[s:e, 2] += np.where(second, vb2, vb1)

    _chunked(N, seed, chunk, fill)
    x = _wrap(x, Ls)
    return Workload(name=f"two_stream_{nn[0]}x{nn[1]}x{nn[2]}_ppc{ppc}", n=nn, L=Ls, x=x, v=v,
                    q_over_m=-1.0, Q=-(L ** 3), dt=dt, n_steps=n_steps, mode=(0, 0, 1),
                    mode_comp=2, meta=dict(alpha=alpha, k=k, eps=eps, sigma=sigma, seed=seed))


def penning(n=256, n_particles=130_000_000, L=20.0, sigma=(1.0, 1.0, 2.0), Bz=5.0,
            wz2=1.0, Q=-1562.5, seed=1002, dt=0.05, n_steps=100, chunk=1 << 20) -> Workload:
    """Penning trap bunch (Section 4.3): Gaussian in all phase-space variables.

    Positions ~ N(L/2, sigma_d^2) per axis (wrapped into the periodic box),
    velocities ~ N(0, 1).  B = (0, 0, Bz); the quadrupole external field has
    axial frequency sqrt(wz2).  The paper's own setting is sigma =
    (0.15, 0.05, 0.2) L with wz2 = 30 / L = 1.5; the large-bunch workload uses
    sigma = (1, 1, 2) and wz2 = 1.
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(int(a) for a in n)
    Ls = (L, L, L)
    N = int(n_particles)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((N, 3), dtype=np.float64)
    v = np.empty((N, 3), dtype=np.float64)
    sig = np.asarray(sigma, dtype=np.float64)
    def fill(r, s, e):
        m = e - s
        x[s:e] = 0.5 * L + sig * r.standard_normal((m, 3))
        v[s:e] = r.standard_normal((m, 3))

    _chunked(N, seed, chunk, fill)
    x = _wrap(x, Ls)
    return Workload(name=f"penning_{nn[0]}x{nn[1]}x{nn[2]}_np{N}", n=nn, L=Ls, x=x, v=v,
                    q_over_m=-1.0, Q=float(Q), dt=dt, B=(0.0, 0.0, float(Bz)), wz2=float(wz2),
                    n_steps=n_steps, mode=(0, 0, 1), mode_comp=2,
                    meta=dict(sigma=tuple(sig), seed=seed))


def uniform_plasma(n=32, ppc=8, L=None, seed=1004, dt=0.05, n_steps=20, chunk=1 << 20) -> Workload:
    """Uniform positions and unit Maxwellian velocities (Section 4.4's layout)."""
    nn = (n, n, n) if np.isscalar(n) else tuple(int(a) for a in n)
    if L is None:
        L = 4.0 * math.pi
    Ls = (L, L, L) if np.isscalar(L) else tuple(float(a) for a in L)
    N = int(nn[0] * nn[1] * nn[2] * ppc)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((N, 3), dtype=np.float64)
    v = np.empty((N, 3), dtype=np.float64)
    Lv = np.asarray(Ls)
    def fill(r, s, e):
        x[s:e] = r.random((e - s, 3)) * Lv
        v[s:e] = r.standard_normal((e - s, 3))

    _chunked(N, seed, chunk, fill)
    x = _wrap(x, Ls)
    return Workload(name=f"uniform_{nn[0]}x{nn[1]}x{nn[2]}_ppc{ppc}", n=nn, L=Ls, x=x, v=v,
                    q_over_m=-1.0, Q=-float(np.prod(Lv)), dt=dt, n_steps=n_steps,
                    meta=dict(seed=seed, ppc=ppc))


def single_particle(x0, v0, n=(16, 16, 16), L=(20.0, 20.0, 20.0), Q=0.0, dt=0.005,
                    Bz=5.0, wz2=1.0, n_steps=1000) -> Workload:
    """One particle in the trap fields (no self-field when Q = 0)."""
    x = np.asarray(x0, dtype=np.float64).reshape(1, 3)
    v = np.asarray(v0, dtype=np.float64).reshape(1, 3)
    return Workload(name="single_particle", n=tuple(n), L=tuple(L), x=x.copy(), v=v.copy(),
                    q_over_m=-1.0, Q=float(Q), dt=dt, B=(0.0, 0.0, Bz), wz2=wz2,
                    n_steps=n_steps)


def by_name(name: str, **kw) -> Workload:
    """Named workloads used by the tests and the benchmark.

    landau_16        16^3 grid, 8 per cell (32,768 particles), L = 4 pi, 20 steps
    landau_128       128^3 grid, 64 per cell (134,217,728 particles), 200 steps
    penning_256      256^3 grid on [0, 20)^3, 1.3e8 particles, Bz = 5, wz = 1
    bump_on_tail_64  64^3 grid on [0, 20 pi)^3, 16 per cell (4,194,304 particles)
    """
    table = {
        "landau_16": lambda: landau(n=16, ppc=8, seed=1000, n_steps=20),
        "landau_128": lambda: landau(n=128, ppc=64, seed=1001, n_steps=200),
        "penning_256": lambda: penning(seed=1002),
        "bump_on_tail_64": lambda: bump_on_tail(seed=1003),
    }
    if name not in table:
        raise KeyError(name)
    w = table[name]()
    for key, val in kw.items():
        setattr(w, key, val)
    return w


def landau_lattice_1d(nx=32, mx=256, mv=128, alpha=0.05, k=0.5, dt=0.05, n_steps=300,
                      vmax=6.0) -> Workload:
    """Quiet 1D-1V Landau start on an (nx, 1, 1) grid: a phase-space lattice.

    x takes mx stratified inverse-transform samples of 1 + alpha cos(k x);
    v_x takes mv stratified samples of N(0, 1) (truncated at +-vmax); every
    (x, v_x) pair is present once, so the sampling noise of the k mode is
    absent and the recurrence time 2 pi / (k dv) lies far beyond the run.
    With one node along y and z the 3D scheme reduces exactly to 1D.
    """
    from scipy.special import ndtr, ndtri

    L = 2.0 * math.pi / k
    ux = (np.arange(mx, dtype=np.float64) + 0.5) / mx
    xs = sample_cosine_density(ux, L, alpha, k)
    c = ndtr(vmax)
    uv = (1.0 - c) + (2.0 * c - 1.0) * (np.arange(mv, dtype=np.float64) + 0.5) / mv
    vs = ndtri(uv)
    X, V = np.meshgrid(xs, vs, indexing="ij")
    N = mx * mv
    x = np.zeros((N, 3), dtype=np.float64)
    v = np.zeros((N, 3), dtype=np.float64)
    x[:, 0] = X.ravel()
    x[:, 1] = 0.5 * L
    x[:, 2] = 0.5 * L
    v[:, 0] = V.ravel()
    Ls = (L, L, L)
    return Workload(name=f"landau_lattice_{nx}x1x1", n=(nx, 1, 1), L=Ls, x=_wrap(x, Ls), v=v,
                    q_over_m=-1.0, Q=-(L ** 3), dt=dt, n_steps=n_steps, mode=(1, 0, 0),
                    mode_comp=0, meta=dict(alpha=alpha, k=k, mx=mx, mv=mv))


def _mixture_quantiles(u: np.ndarray, eps: float, v_beam: float, sigma_beam: float,
                       sigma_bulk: float, u_bulk: float = 0.0) -> np.ndarray:
    """Inverse CDF of (1 - eps) N(u_bulk, sigma_bulk^2) + eps N(v_beam, sigma_beam^2) at u,
    by bisection (monotone CDF; 80 halvings reach double precision)."""
    from scipy.special import ndtr

    lo = np.full(u.shape, min(u_bulk - 12.0 * sigma_bulk, v_beam - 12.0 * sigma_beam))
    hi = np.full(u.shape, max(u_bulk + 12.0 * sigma_bulk, v_beam + 12.0 * sigma_beam))
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        F = (1.0 - eps) * ndtr((mid - u_bulk) / sigma_bulk) + eps * ndtr((mid - v_beam) / sigma_beam)
        below = F < u
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def bump_on_tail_quiet(n=(64, 64, 64), L=20.0 * math.pi, axis=2, m=3, alpha=1e-3, ms=4096,
                       mv=1024, eps=0.1, v_beam=4.0, sigma_beam=0.3, sigma_bulk=1.0, seed=1006,
                       dt=0.05, n_steps=300, u_bulk=0.0) -> Workload:
    """Bump-on-tail start that is quiet along one axis, for growth-rate checks.

    Along `axis`: ms stratified inverse-transform samples of the density
    1 + alpha cos(k s), k = 2 pi m / L, paired with every one of mv stratified
    samples of the velocity mixture (1 - eps) N(u_bulk, sigma_bulk^2) +
    eps N(v_beam, sigma_beam^2): ms * mv particles (u_bulk = -v_beam, eps = 1/2
    and equal spreads give the symmetric two-stream case).  The Fourier modes
    (0, 0, j) (for axis 2) of the charge then carry no sampling noise, so the
    seeded mode m grows from its seed alone.  The transverse positions are
    uniform and the transverse velocities N(0, sigma_bulk^2), both seeded
    random draws (on a grid with one node across, their values do not enter).
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(int(a) for a in n)
    Ls = (L, L, L)
    k = 2.0 * math.pi * m / L
    us = (np.arange(ms, dtype=np.float64) + 0.5) / ms
    s = sample_cosine_density(us, L, alpha, k)
    uv = (np.arange(mv, dtype=np.float64) + 0.5) / mv
    vs = _mixture_quantiles(uv, eps, v_beam, sigma_beam, sigma_bulk, u_bulk)
    S, V = np.meshgrid(s, vs, indexing="ij")
    N = ms * mv
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.random((N, 3)) * L
    v = sigma_bulk * rng.standard_normal((N, 3))
    x[:, axis] = S.ravel()
    v[:, axis] = V.ravel()
    mode = [0, 0, 0]
    mode[axis] = m
    return Workload(name=f"bump_on_tail_quiet_{nn[0]}x{nn[1]}x{nn[2]}_m{m}", n=nn, L=Ls,
                    x=_wrap(x, Ls), v=v, q_over_m=-1.0, Q=-(L ** 3), dt=dt, n_steps=n_steps,
                    mode=tuple(mode), mode_comp=axis,
                    meta=dict(alpha=alpha, k=k, m=m, eps=eps, v_beam=v_beam, u_bulk=u_bulk,
                              sigma_beam=sigma_beam, ms=ms, mv=mv, seed=seed))
