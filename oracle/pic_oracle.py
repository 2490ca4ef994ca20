"""FP64 CPU oracle for the electrostatic PIC step -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module.  The product path (the CUDA library and its Python
binding) never calls it and shares no code with it.

It restates, in plain numpy FP64, the scheme of Section 3 of the paper
(arXiv 2205.11052) as this project reads it:

  * Section 3.1, steps 1-4 (Eq. Vlasov, Eq. potential, Eq. momentum_eqn):
    scatter -> Poisson solve -> gather -> push, electrons in a uniform
    neutralising ion background (the k = 0 mode of the charge is dropped).
  * Section 3.2: normalised units (q/m = -1, eps0 = 1); a cell-centred grid
    with constant spacing h_d = L_d / N_d per axis, nodes at (g + 1/2) h;
    cloud-in-cell (CIC) shape for scatter and gather; periodic in x, y, z;
    FFT spectral solve; the synchronised Boris integrator giving x and v at
    integer steps.

Readings where the paper is silent (each is listed in the design notes):
  * CIC base index i = floor(x/h - 1/2) mod N, fraction f = x/h - 1/2 - i.
    A particle on a node puts all its weight on that node.
  * The deposit produces the charge density rho_g = sum_p q_p W / h^3.
  * Poisson: -Lap(phi) = rho with the continuous symbol |k|^2,
    k_d = 2 pi m_d / L_d, m_d in FFT order [-N/2, N/2).  E = -grad(phi) taken
    spectrally, E^_d = -i k_d rho^ / |k|^2, with the k = 0 mode and each
    axis' Nyquist component of k_d set to zero (so E is real and the
    real-space kernel is antisymmetric).
  * Time stepping: drift-kick-drift.  x_h = x_n + dt/2 v_n; the kick is the
    Boris rotation with E evaluated at x_h (self field plus the external
    quadrupole); x_{n+1} = x_h + dt/2 v_{n+1}.  Field diagnostics therefore
    refer to t_{n+1/2}.
  * External quadrupole E_ext = wz2 * (-(x-cx)/2, -(y-cy)/2, (z-cz)), the
    paper's Penning field written with its axial frequency squared wz2
    (Section 4.3 has wz2 = 30/L).
  * Uniform particle charge q_p = Q / N_p and mass m_p = q_p / (q/m).

Every function below cites the passage it follows.  Nothing here is blocked,
fused or reordered beyond what those passages state.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Grid",
    "Params",
    "cic_stencil",
    "deposit",
    "deposit_bruteforce",
    "solve_field",
    "gather",
    "external_field",
    "boris_kick",
    "wrap",
    "step",
    "run",
    "diagnostics",
    "mode_coefficient",
]


@dataclasses.dataclass(frozen=True)
class Grid:
    """Periodic cell-centred grid on [0, L)^3 (Section 3.2)."""

    n: tuple   # (Nx, Ny, Nz)
    L: tuple   # (Lx, Ly, Lz)

    @property
    def h(self) -> np.ndarray:
        return np.asarray(self.L, dtype=np.float64) / np.asarray(self.n, dtype=np.float64)

    @property
    def cell_volume(self) -> float:
        h = self.h
        return float(h[0] * h[1] * h[2])

    @property
    def shape(self) -> tuple:
        """numpy shape of a field array: (Nz, Ny, Nx), x fastest."""
        return (self.n[2], self.n[1], self.n[0])

    @property
    def n_nodes(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])


@dataclasses.dataclass(frozen=True)
class Params:
    """Physical parameters of one run (Section 3.1 and Section 4)."""

    dt: float
    q_over_m: float = -1.0             # Section 3.2 normalisation
    Q: float = -1.0                    # total electron charge Q_e
    B: tuple = (0.0, 0.0, 0.0)         # uniform external magnetic field
    wz2: float = 0.0                   # quadrupole strength (axial frequency squared)


def wrap(x: np.ndarray, grid: Grid) -> np.ndarray:
    """Periodic boundary condition in all directions (Section 3.2)."""
    L = np.asarray(grid.L, dtype=np.float64)
    y = np.mod(x, L)
    return np.where(y >= L, y - L, y)


# ---------------------------------------------------------------------------
# scatter (Section 3.1 step 1; Section 3.2: cell-centred grid, CIC shape)
# ---------------------------------------------------------------------------

def cic_stencil(x: np.ndarray, grid: Grid):
    """CIC stencil of each particle on the cell-centred grid.

    Returns (nodes, weights): nodes is (N, 8) int64 linear node indices
    g = i + Nx (j + Ny k), weights is (N, 8) float64, both ordered by the
    corner bits (a, b, c) = (bit0, bit1, bit2) of the corner number.
    """
    h = grid.h
    n = np.asarray(grid.n, dtype=np.int64)
    s = x / h - 0.5                      # node g sits at (g + 1/2) h
    base = np.floor(s)
    f = s - base
    base = base.astype(np.int64) % n
    nodes = np.empty((x.shape[0], 8), dtype=np.int64)
    weights = np.empty((x.shape[0], 8), dtype=np.float64)
    for corner in range(8):
        a, b, c = corner & 1, (corner >> 1) & 1, (corner >> 2) & 1
        ix = (base[:, 0] + a) % n[0]
        iy = (base[:, 1] + b) % n[1]
        iz = (base[:, 2] + c) % n[2]
        wx = f[:, 0] if a else 1.0 - f[:, 0]
        wy = f[:, 1] if b else 1.0 - f[:, 1]
        wz = f[:, 2] if c else 1.0 - f[:, 2]
        nodes[:, corner] = ix + n[0] * (iy + n[1] * iz)
        weights[:, corner] = wx * wy * wz
    return nodes, weights


def deposit(x: np.ndarray, grid: Grid, q) -> np.ndarray:
    """Electron charge density rho_g = sum_p q_p W(x_g - x_p) / h^3.

    Section 3.1 step 1 ("scatter") with the CIC shape of Section 3.2.
    ``q`` is a scalar particle charge or an (N,) array of per-particle
    weights (the latter is the transpose of ``gather``).  Returns an array of
    shape (Nz, Ny, Nx).
    """
    nodes, w = cic_stencil(x, grid)
    qq = np.broadcast_to(np.asarray(q, dtype=np.float64), (x.shape[0],))
    rho = np.bincount(nodes.ravel(), weights=(w * qq[:, None]).ravel(),
                      minlength=grid.n_nodes)
    return (rho / grid.cell_volume).reshape(grid.shape)


def deposit_bruteforce(x: np.ndarray, grid: Grid, q: float) -> np.ndarray:
    """Independent CIC deposit for tiny cases: node-by-node tent functions.

    rho_g = sum_p q Prod_d max(0, 1 - |minimage(x_g,d - x_p,d)| / h_d) / h^3,
    evaluated with explicit loops over every particle and every node (no
    base-index arithmetic), so it shares no step with ``deposit``.
    """
    h = grid.h
    L = np.asarray(grid.L, dtype=np.float64)
    nx, ny, nz = grid.n
    rho = np.zeros(grid.shape, dtype=np.float64)
    for p in range(x.shape[0]):
        for kz in range(nz):
            for jy in range(ny):
                for ix in range(nx):
                    node = np.array([(ix + 0.5) * h[0], (jy + 0.5) * h[1], (kz + 0.5) * h[2]])
                    d = node - x[p]
                    d = d - L * np.round(d / L)
                    w = np.prod(np.maximum(0.0, 1.0 - np.abs(d) / h))
                    rho[kz, jy, ix] += q * w
    return rho / grid.cell_volume


# ---------------------------------------------------------------------------
# field solve (Section 3.1 step 2; Eq. potential; Section 3.2: FFT solver)
# ---------------------------------------------------------------------------

def _wavenumbers(grid: Grid):
    """Per-axis integer mode numbers in FFT order and the k vectors."""
    ks, kgrad = [], []
    for d in range(3):
        N = grid.n[d]
        m = np.fft.fftfreq(N, d=1.0 / N)        # 0, 1, ..., -N/2, ..., -1 (integers)
        k = 2.0 * math.pi * m / grid.L[d]
        kg = k.copy()
        if N % 2 == 0:
            kg[m == -(N // 2)] = 0.0             # Nyquist: no derivative
        ks.append(k)
        kgrad.append(kg)
    return ks, kgrad


def solve_field(rho: np.ndarray, grid: Grid, return_potential: bool = False):
    """E = -grad(phi) with -Lap(phi) = rho - rho_i (Eq. potential, eps0 = 1).

    The uniform ion background rho_i only cancels the k = 0 mode, which is set
    to zero.  Spectral: E^_d = -i k_d rho^ / |k|^2.  Returns E with shape
    (3, Nz, Ny, Nx) (components x, y, z).
    """
    rho_hat = np.fft.fftn(rho)                   # axes (z, y, x)
    ks, kgrad = _wavenumbers(grid)
    KZ, KY, KX = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
    GZ, GY, GX = np.meshgrid(kgrad[2], kgrad[1], kgrad[0], indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    phi_hat = rho_hat / k2
    phi_hat[0, 0, 0] = 0.0
    E = np.empty((3,) + grid.shape, dtype=np.float64)
    for d, G in enumerate((GX, GY, GZ)):
        E[d] = np.fft.ifftn(-1j * G * phi_hat).real
    if return_potential:
        return E, np.fft.ifftn(phi_hat).real
    return E


def mode_coefficient(field: np.ndarray, m: tuple) -> complex:
    """Fourier coefficient (1/N_g) sum_g F_g exp(-2 pi i m.g/N) of one mode."""
    F = np.fft.fftn(field) / field.size
    nz, ny, nx = field.shape
    return complex(F[m[2] % nz, m[1] % ny, m[0] % nx])


# ---------------------------------------------------------------------------
# gather and push (Section 3.1 steps 3-4, Eq. momentum_eqn; Section 3.2)
# ---------------------------------------------------------------------------

def gather(x: np.ndarray, E: np.ndarray, grid: Grid) -> np.ndarray:
    """Interpolate grid E to the particles with the scatter's CIC weights."""
    nodes, w = cic_stencil(x, grid)
    out = np.empty((x.shape[0], 3), dtype=np.float64)
    for d in range(3):
        Ed = E[d].ravel()
        out[:, d] = np.sum(w * Ed[nodes], axis=1)
    return out


def external_field(x: np.ndarray, grid: Grid, wz2: float) -> np.ndarray:
    """Quadrupole trap field of Section 4.3, centred in the box."""
    c = 0.5 * np.asarray(grid.L, dtype=np.float64)
    d = x - c
    return wz2 * np.stack([-0.5 * d[:, 0], -0.5 * d[:, 1], d[:, 2]], axis=1)


def boris_kick(v: np.ndarray, e: np.ndarray, q_over_m: float, B, dt: float) -> np.ndarray:
    """One velocity update of Eq. momentum_eqn over dt by the Boris rotation.

    Solves v1 = v0 + dt (q/m) [e + (v0 + v1)/2 x B] exactly: half electric
    kick, rotation about B by angle 2 arctan(|q/m| |B| dt / 2), half kick.
    """
    B = np.asarray(B, dtype=np.float64)
    vm = v + 0.5 * dt * q_over_m * e
    t = 0.5 * dt * q_over_m * B
    s = 2.0 * t / (1.0 + float(np.dot(t, t)))
    vprime = vm + np.cross(vm, t)
    vp = vm + np.cross(vprime, s)
    return vp + 0.5 * dt * q_over_m * e


# ---------------------------------------------------------------------------
# one synchronised step and the diagnostics
# ---------------------------------------------------------------------------

def diagnostics(rho: np.ndarray, E: np.ndarray, v_new: np.ndarray, grid: Grid,
                params: Params, n_particles: int, mode=(1, 0, 0), mode_comp=0) -> dict:
    """Field energies int E_d^2 dV (Figs. Landau_damping_rate, TSI_BTI),
    total charge, momentum and kinetic energy of the electrons."""
    dV = grid.cell_volume
    qp = params.Q / n_particles if n_particles else 0.0
    mp = qp / params.q_over_m
    out = {
        "Wx": dV * float(np.sum(E[0] ** 2)),
        "Wy": dV * float(np.sum(E[1] ** 2)),
        "Wz": dV * float(np.sum(E[2] ** 2)),
        "Q": dV * float(np.sum(rho)),
        "mode": mode_coefficient(E[mode_comp], mode),
    }
    if v_new is not None and n_particles:
        P = mp * np.sum(v_new, axis=0)
        out.update(Px=float(P[0]), Py=float(P[1]), Pz=float(P[2]),
                   K=0.5 * mp * float(np.sum(v_new * v_new)))
    return out


def step(x: np.ndarray, v: np.ndarray, grid: Grid, params: Params, with_diag=False,
         mode=(1, 0, 0), mode_comp=0):
    """Advance synchronised (x_n, v_n) to (x_{n+1}, v_{n+1}).

    Drift-kick-drift reading of the synchronised Boris scheme (Section 3.2):
    1. x_h = x_n + dt/2 v_n, periodic wrap
    2. scatter: rho = deposit(x_h)                  (Section 3.1 step 1)
    3. solve: E = -grad phi, -Lap phi = rho - rho_i  (step 2)
    4. gather: e = G(x_h) E + E_ext(x_h)             (step 3)
    5. Boris kick v_n -> v_{n+1} with e and B_ext      (step 4)
    6. x_{n+1} = x_h + dt/2 v_{n+1}, periodic wrap
    """
    N = x.shape[0]
    dt = params.dt
    qp = params.Q / N if N else 0.0
    xh = wrap(x + 0.5 * dt * v, grid)
    rho = deposit(xh, grid, qp)
    E = solve_field(rho, grid)
    e = gather(xh, E, grid)
    if params.wz2 != 0.0:
        e = e + external_field(xh, grid, params.wz2)
    v1 = boris_kick(v, e, params.q_over_m, params.B, dt)
    x1 = wrap(xh + 0.5 * dt * v1, grid)
    if with_diag:
        return x1, v1, diagnostics(rho, E, v1, grid, params, N, mode, mode_comp)
    return x1, v1


def run(x: np.ndarray, v: np.ndarray, grid: Grid, params: Params, n_steps: int,
        mode=(1, 0, 0), mode_comp=0, diag_every: int = 1):
    """n_steps synchronised steps; returns (x, v, list of per-step diagnostics)."""
    hist = []
    for n in range(n_steps):
        want = diag_every > 0 and (n % diag_every == diag_every - 1 or diag_every == 1)
        if want:
            x, v, d = step(x, v, grid, params, True, mode, mode_comp)
            d["step"] = n
            d["t_field"] = (n + 0.5) * params.dt
            d["t"] = (n + 1) * params.dt
            hist.append(d)
        else:
            x, v = step(x, v, grid, params)
    return x, v, hist


# ---------------------------------------------------------------------------
# discrete adjoint (not in the paper: gradient of the final field energy)
#
# The step above, written on the half-step positions y_n = x_{n+1/2}:
#     e_n     = G(y_n) S D(y_n) + E_ext(y_n)
#     v_{n+1} = v_n + c e_n,            c = dt q/m      (B = 0)
#     y_{n+1} = y_n + dt v_{n+1}
# with y_0 = x_0 + dt/2 v_0.  The objective is the weighted field energy of
# the field the last of n_steps steps uses,
#     J = sum_d w_d h^3 sum_g E_d,g^2,   E = S D(y_{n_steps - 1}).
# Its reverse sweep, step by step, is the plain chain rule of these lines:
#     lv_tot = lv' + dt ly'
#     le     = c lv_tot                          (adjoint of e)
#     ly     = ly' + (dG/dy . E)^T le            (weight gradients, E fixed)
#              + Ext^T le                        (linear quadrupole)
#              + (dD/dy)^T S^T G^T le            (through the self field)
#     lv     = lv_tot
# with S^T = -S for the spectral gradient (purely imaginary, odd symbol).
# ---------------------------------------------------------------------------

def cic_weight_gradients(x: np.ndarray, grid: Grid):
    """(nodes, weights, dweights): dweights[:, corner, j] = dW/dx_j."""
    h = grid.h
    n = np.asarray(grid.n, dtype=np.int64)
    s = x / h - 0.5
    base = np.floor(s)
    f = s - base
    base = base.astype(np.int64) % n
    N = x.shape[0]
    nodes = np.empty((N, 8), dtype=np.int64)
    w = np.empty((N, 8), dtype=np.float64)
    dw = np.empty((N, 8, 3), dtype=np.float64)
    for corner in range(8):
        bits = (corner & 1, (corner >> 1) & 1, (corner >> 2) & 1)
        fac = []
        dfac = []
        for d in range(3):
            if bits[d]:
                fac.append(f[:, d])
                dfac.append(np.full(N, 1.0 / h[d]))
            else:
                fac.append(1.0 - f[:, d])
                dfac.append(np.full(N, -1.0 / h[d]))
        ix = (base[:, 0] + bits[0]) % n[0]
        iy = (base[:, 1] + bits[1]) % n[1]
        iz = (base[:, 2] + bits[2]) % n[2]
        nodes[:, corner] = ix + n[0] * (iy + n[1] * iz)
        w[:, corner] = fac[0] * fac[1] * fac[2]
        dw[:, corner, 0] = dfac[0] * fac[1] * fac[2]
        dw[:, corner, 1] = fac[0] * dfac[1] * fac[2]
        dw[:, corner, 2] = fac[0] * fac[1] * dfac[2]
    return nodes, w, dw


def solve_field_transpose(lamE: np.ndarray, grid: Grid) -> np.ndarray:
    """S^T applied to a field adjoint (3, Nz, Ny, Nx) -> rho adjoint.

    S_d has the symbol -i k_d / |k|^2 (k = 0 and the Nyquist gradient zeroed);
    as a real operator its transpose has the conjugate symbol +i k_d / |k|^2.
    """
    ks, kgrad = _wavenumbers(grid)
    KZ, KY, KX = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
    GZ, GY, GX = np.meshgrid(kgrad[2], kgrad[1], kgrad[0], indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    acc = np.zeros(grid.shape, dtype=np.complex128)
    for d, G in enumerate((GX, GY, GZ)):
        acc += 1j * G / k2 * np.fft.fftn(lamE[d])
    acc[0, 0, 0] = 0.0
    return np.fft.ifftn(acc).real


def field_energy(y: np.ndarray, grid: Grid, params: Params, weights=(1.0, 1.0, 1.0)) -> float:
    """J = sum_d w_d h^3 sum_g E_d^2 with E = S D(y)."""
    qp = params.Q / y.shape[0]
    E = solve_field(deposit(y, grid, qp), grid)
    return float(sum(weights[d] * grid.cell_volume * np.sum(E[d] ** 2) for d in range(3)))


def field_energy_gradient(y: np.ndarray, grid: Grid, params: Params, weights=(1.0, 1.0, 1.0)):
    """dJ/dy for J = field_energy(y): (dD/dy)^T S^T (2 h^3 w E)."""
    N = y.shape[0]
    qp = params.Q / N
    E = solve_field(deposit(y, grid, qp), grid)
    lamE = np.stack([2.0 * weights[d] * grid.cell_volume * E[d] for d in range(3)])
    lamrho = solve_field_transpose(lamE, grid)
    nodes, _, dw = cic_weight_gradients(y, grid)
    lr = lamrho.ravel()[nodes]                      # (N, 8)
    return (qp / grid.cell_volume) * np.einsum("pc,pcj->pj", lr, dw)


# ---------------------------------------------------------------------------
# uniform plasma test (Section 4.4)
# ---------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(seed: int, c: np.ndarray) -> np.ndarray:
    """The c-th outputs (c >= 1, uint64 array) of the SplitMix64 generator
    seeded with `seed` (Steele, Lea and Flood, 2014): state seed + c * golden
    gamma, then the two xor-shift-multiply rounds and a final xor-shift."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + np.asarray(c, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_displacement(n: int, pid: np.ndarray, seed: int) -> np.ndarray:
    """(N, 3) displacements in cell units, uniform in [-1, 1): axis d of particle
    pid in step n uses output c = ((n 2^32) + pid) 4 + d + 1, u = its top 24
    bits times 2^-24, displacement 2u - 1."""
    pid = np.asarray(pid, dtype=np.uint64)
    base = (np.uint64(n) << np.uint64(32)) + pid
    out = np.empty((pid.shape[0], 3), dtype=np.float64)
    for d in range(3):
        c = base * np.uint64(4) + np.uint64(d + 1)
        u = (splitmix64(seed, c) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
        out[:, d] = 2.0 * u - 1.0
    return out


def step_uniform(x: np.ndarray, v: np.ndarray, grid: Grid, params: Params, n: int, seed: int,
                 pid=None, with_diag=False, mode=(1, 0, 0), mode_comp=0):
    """One step of the uniform plasma test: the scatter and field solve of the
    drift-kick-drift cycle (at x_h = x_n + dt/2 v_n), then every particle
    moves by a uniform random displacement in [-h, h) per axis instead of the
    gather and push; velocities unchanged."""
    N = x.shape[0]
    qp = params.Q / N if N else 0.0
    xh = wrap(x + 0.5 * params.dt * v, grid)
    rho = deposit(xh, grid, qp)
    E = solve_field(rho, grid)
    if pid is None:
        pid = np.arange(N)
    x1 = wrap(x + uniform_displacement(n, pid, seed) * np.asarray(grid.h), grid)
    if with_diag:
        return x1, v, diagnostics(rho, E, v, grid, params, N, mode, mode_comp)
    return x1, v


def boris_rotation(params: Params) -> np.ndarray:
    """The rotation R of the Boris kick: boris_kick(v, e) = R v + (dt q/m / 2)(R + I) e.
    Its columns are the kicks of the unit vectors with e = 0."""
    return np.stack([boris_kick(np.eye(3)[j], np.zeros(3), params.q_over_m, params.B, params.dt)
                     for j in range(3)], axis=1)


def adjoint_step(y: np.ndarray, lam_y: np.ndarray, lam_v: np.ndarray, grid: Grid,
                 params: Params):
    """Pull (lam_y, lam_v) of (y_{n+1}, v_{n+1}) back to (y_n, v_n).

    The step is v' = R v + h (R + I) e(y), y' = y + dt v' (h = dt q/m / 2,
    R the Boris rotation, the identity without B), so with
    lv_tot = lam_v + dt lam_y: lam_v(n) = R^T lv_tot and the field sees
    le = h (R^T + I) lv_tot (= 2 h lv_tot without B)."""
    N = y.shape[0]
    qp = params.Q / N if N else 0.0
    c = params.dt * params.q_over_m
    E = solve_field(deposit(y, grid, qp), grid)
    lv_tot = lam_v + params.dt * lam_y
    if any(b != 0.0 for b in params.B):
        R = boris_rotation(params)
        le = 0.5 * c * (lv_tot @ R + lv_tot)        # rows: (R^T lv)^T = lv^T R
        lv_out = lv_tot @ R
    else:
        le = c * lv_tot
        lv_out = lv_tot
    nodes, w, dw = cic_weight_gradients(y, grid)
    # (dG/dy . E)^T le : sum_corner dW/dy_j (le . E_corner)
    Eg = np.stack([E[d].ravel()[nodes] for d in range(3)], axis=-1)     # (N, 8, 3)
    s = np.einsum("pcd,pd->pc", Eg, le)
    ly = lam_y + np.einsum("pc,pcj->pj", s, dw)
    if params.wz2 != 0.0:
        ly = ly + params.wz2 * le * np.array([-0.5, -0.5, 1.0])
    # through the self field: G^T le -> S^T -> (dD/dy)^T
    lamE = np.stack([deposit(y, grid, le[:, d]) * grid.cell_volume for d in range(3)])
    lamrho = solve_field_transpose(lamE, grid)
    lr = lamrho.ravel()[nodes]
    ly = ly + (qp / grid.cell_volume) * np.einsum("pc,pcj->pj", lr, dw)
    return ly, lv_out


def boris_rotation_dt(vm: np.ndarray, t: np.ndarray) -> np.ndarray:
    """d/dt_k of the Boris rotation f(t) = vm + (vm + vm x t) x s(t),
    s = 2t / (1 + |t|^2), for each row vm: (N, 3 (k), 3).

    d(vm x t)/dt_k = vm x e_k and ds/dt_k = (2 / (1 + |t|^2)) (e_k - t_k s)."""
    D = 1.0 + float(np.dot(t, t))
    s = 2.0 * t / D
    w = vm + np.cross(vm, t)
    out = np.empty((vm.shape[0], 3, 3), dtype=np.float64)
    for k in range(3):
        ek = np.zeros(3)
        ek[k] = 1.0
        ds = (2.0 / D) * (ek - t[k] * s)
        out[:, k, :] = np.cross(np.cross(vm, ek), s) + np.cross(w, ds)
    return out


def param_gradient_terms(y: np.ndarray, v: np.ndarray, e: np.ndarray, lam_y: np.ndarray,
                         lam_v: np.ndarray, grid: Grid, params: Params):
    """Contribution of one step to dJ/dB_ext (3) and dJ/d(wz2).

    The step is v' = R(B) vm + h e, vm = v + h e, h = dt q/m / 2,
    t = h B, e = G(y) E + wz2 Q(y) with Q(y) = (-(y-c)_x/2, -(y-c)_y/2, (y-c)_z)
    (Section 4.3), and y' = y + dt v'.  With lv_tot = lam_v + dt lam_y (the
    adjoint of v'), dJ/dB_k gets sum_p lv_tot . h df/dt_k(vm) and dJ/dwz2 gets
    sum_p lv_tot . dv'/dwz2 = sum_p le . Q(y), le = h (R^T + I) lv_tot."""
    h = 0.5 * params.dt * params.q_over_m
    t = h * np.asarray(params.B, dtype=np.float64)
    lv_tot = lam_v + params.dt * lam_y
    vm = v + h * e
    dB = h * np.einsum("pj,pkj->k", lv_tot, boris_rotation_dt(vm, t))
    R = boris_rotation(params)
    le = h * (lv_tot @ R + lv_tot)
    c = 0.5 * np.asarray(grid.L, dtype=np.float64)
    d = y - c
    Q = np.stack([-0.5 * d[:, 0], -0.5 * d[:, 1], d[:, 2]], axis=1)
    dwz2 = float(np.sum(le * Q))
    return dB, dwz2


def run_with_gradient(x0: np.ndarray, v0: np.ndarray, grid: Grid, params: Params,
                      n_steps: int, weights=(1.0, 1.0, 1.0), param_grad: bool = False):
    """J of the field used by the last of n_steps steps, and dJ/dx0, dJ/dv0
    (with param_grad, also dJ/dB_ext (3) and dJ/d(wz2)).

    Forward: y_0 = x_0 + dt/2 v_0, then n_steps - 1 updates of (y, v); the
    objective is the field energy at y_{n_steps-1}.  The forward states are
    kept (the oracle stores them all; it has no checkpointing)."""
    dt = params.dt
    N = x0.shape[0]
    qp = params.Q / N
    ys = [wrap(x0 + 0.5 * dt * v0, grid)]
    vs, es = [], []
    v = v0.copy()
    for _ in range(n_steps - 1):
        y = ys[-1]
        E = solve_field(deposit(y, grid, qp), grid)
        e = gather(y, E, grid)
        if params.wz2 != 0.0:
            e = e + external_field(y, grid, params.wz2)
        vs.append(v)
        es.append(e)
        v = boris_kick(v, e, params.q_over_m, params.B, dt)
        ys.append(wrap(y + dt * v, grid))
    J = field_energy(ys[-1], grid, params, weights)
    ly = field_energy_gradient(ys[-1], grid, params, weights)
    lv = np.zeros_like(ly)
    gB = np.zeros(3)
    gw = 0.0
    for n in range(n_steps - 2, -1, -1):
        if param_grad:
            dB, dw = param_gradient_terms(ys[n], vs[n], es[n], ly, lv, grid, params)
            gB += dB
            gw += dw
        ly, lv = adjoint_step(ys[n], ly, lv, grid, params)
    dx0 = ly
    dv0 = lv + 0.5 * dt * ly
    if param_grad:
        return J, dx0, dv0, gB, gw
    return J, dx0, dv0


def cosine_sample_dalpha(x: np.ndarray, alpha: float, k: float) -> np.ndarray:
    """d x / d alpha of the inverse-transform sample x(u; alpha) of
    1 + alpha cos(k x): from x + (alpha/k) sin(k x) = u L at fixed u."""
    return -(np.sin(k * x) / k) / (1.0 + alpha * np.cos(k * x))
