"""Convenience wrapper around the C ABI: torch supplies device memory and the
stream, the CUDA library does all the work.

    sim = Simulation(n=(16, 16, 16), L=(4*pi,)*3, n_particles=N, dt=0.05, Q=-L**3)
    sim.load(x, v)          # (N, 3) float64 host or CUDA arrays
    sim.step(20)
    hist = sim.diagnostics()
    x, v = sim.particles()
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi


def _i3(v):
    v = tuple(int(a) for a in (v if np.ndim(v) else (v, v, v)))
    return (C.c_int32 * 3)(*v)


def _d3(v):
    v = tuple(float(a) for a in (v if np.ndim(v) else (v, v, v)))
    return (C.c_double * 3)(*v)


def make_structs(n, L, n_particles, dt, q_over_m=-1.0, Q=-1.0, B=(0.0, 0.0, 0.0), wz2=0.0,
                 tile=(0, 0, 0), guard=0, sort_period=0, diag_every=0, diag_capacity=0,
                 mode=(1, 0, 0), mode_comp=0, block=0, chunk=0, options=0, seed=0,
                 stray_rebin=0.0):
    grid = capi.pic_grid_t(_i3(n), _d3(L))
    species = capi.pic_species_t(float(q_over_m), float(Q), int(n_particles))
    params = capi.pic_params_t(float(dt), _d3(B), float(wz2), _i3(tile), int(guard),
                               int(sort_period), int(diag_every), int(diag_capacity),
                               _i3(mode), int(mode_comp), int(block), int(chunk), int(options),
                               int(seed), float(stray_rebin))
    return grid, species, params


class Simulation:
    """One PIC run bound to a torch-allocated device arena and CUDA stream."""

    def __init__(self, n, L, n_particles, dt, q_over_m=-1.0, Q=-1.0, B=(0.0, 0.0, 0.0),
                 wz2=0.0, tile=(0, 0, 0), guard=0, sort_period=0, diag_every=0,
                 diag_capacity=0, mode=(1, 0, 0), mode_comp=0, block=0, chunk=0, options=0,
                 seed=0, stray_rebin=0.0, device=None, stream=None):
        import torch

        self.n = tuple(int(a) for a in (n if np.ndim(n) else (n, n, n)))
        self.L = tuple(float(a) for a in (L if np.ndim(L) else (L, L, L)))
        self.capacity = int(n_particles)
        self.dt = float(dt)
        grid, species, params = make_structs(self.n, self.L, n_particles, dt, q_over_m, Q, B, wz2,
                                             tile, guard, sort_period, diag_every, diag_capacity,
                                             mode, mode_comp, block, chunk, options, seed,
                                             stray_rebin)
        self.handle = capi.pic_create(grid, species, params)
        self._closed = False
        self.sizes = capi.pic_buffer_sizes(self.handle)
        self.device = torch.device(device) if device is not None else torch.device("cuda",
                                                                                   torch.cuda.current_device())
        self.arena = torch.empty(int(self.sizes.workspace_bytes), dtype=torch.uint8,
                                 device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        capi.pic_bind_workspace(self.handle, self.arena.data_ptr(), int(self.sizes.workspace_bytes),
                                self.stream.cuda_stream)
        self.n_particles = 0

    @classmethod
    def from_workload(cls, w, **kw):
        """Build from a ``pic_inputs.Workload``-like object and load its particles."""
        args = dict(n=w.n, L=w.L, n_particles=w.n_particles, dt=w.dt, q_over_m=w.q_over_m,
                    Q=w.Q, B=w.B, wz2=w.wz2, mode=w.mode, mode_comp=w.mode_comp)
        args.update(kw)
        sim = cls(**args)
        sim.load(w.x, w.v)
        return sim

    # ------------------------------------------------------------------ I/O
    def load(self, x, v):
        import torch

        if isinstance(x, torch.Tensor):
            assert x.dtype == torch.float64 and v.dtype == torch.float64
            x = x.contiguous()
            v = v.contiguous()
            n = int(x.shape[0])
            capi.pic_load_particles(self.handle, x.data_ptr(), v.data_ptr(), n, x.is_cuda)
            self._keep = (x, v)      # device sources are read asynchronously
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            v = np.ascontiguousarray(v, dtype=np.float64)
            n = int(x.shape[0])
            capi.pic_load_particles(self.handle, x.ctypes.data, v.ctypes.data, n, False)
        self.n_particles = n

    def particles(self, device: bool = False):
        """Synchronised (x_n, v_n) in load order as (N, 3) float64 arrays."""
        import torch

        N = self.n_particles
        if device:
            x = torch.empty((N, 3), dtype=torch.float64, device=self.device)
            v = torch.empty((N, 3), dtype=torch.float64, device=self.device)
            capi.pic_get_particles(self.handle, x.data_ptr(), v.data_ptr(), True)
            return x, v
        x = np.empty((N, 3), dtype=np.float64)
        v = np.empty((N, 3), dtype=np.float64)
        capi.pic_get_particles(self.handle, x.ctypes.data, v.ctypes.data, False)
        return x, v

    def field(self):
        """(rho, E): rho as (Nz, Ny, Nx) float32, E as (3, Nz, Ny, Nx) float32."""
        nx, ny, nz = self.n
        rho = np.empty((nz, ny, nx), dtype=np.float32)
        E4 = np.empty((nz, ny, nx, 4), dtype=np.float32)
        capi.pic_get_field(self.handle, rho.ctypes.data, E4.ctypes.data, False)
        return rho, np.ascontiguousarray(np.moveaxis(E4[..., :3], -1, 0))

    def set_rho(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float32)
        assert rho.size == self.n[0] * self.n[1] * self.n[2]
        capi.pic_set_rho(self.handle, rho.ctypes.data, False)

    # ------------------------------------------------------------------ cycle
    def sort(self):
        capi.pic_sort(self.handle)

    def deposit(self):
        capi.pic_deposit(self.handle)

    def field_solve(self):
        capi.pic_field_solve(self.handle)

    def gather_push(self):
        capi.pic_gather_push(self.handle)

    def step(self, n: int = 1):
        capi.pic_step(self.handle, int(n))

    def counts(self):
        return capi.pic_get_counts(self.handle)

    def rebin_stats(self):
        """(re-binnings since the load, strays since the last re-binning decision)."""
        return capi.pic_rebin_stats(self.handle)

    def diagnostics(self, max_records: int = 1 << 16):
        recs = capi.pic_diagnostics(self.handle, max_records)
        out = []
        for r in recs:
            out.append(dict(step=r.step, t_field=r.t_field, Wx=r.Wx, Wy=r.Wy, Wz=r.Wz, Q=r.Q,
                            mode=complex(r.mode_re, r.mode_im), t=r.t, Px=r.Px, Py=r.Py,
                            Pz=r.Pz, K=r.K))
        return out

    # ------------------------------------------------------------------ adjoint
    def adjoint_forward(self, n_steps: int, weights=(1.0, 1.0, 1.0), checkpoint_every: int = 20):
        """J = sum_d w_d h^3 sum_g E_d^2 of the field of the last of n_steps steps
        from the loaded state; keeps checkpoints for adjoint_backward."""
        import torch

        nbytes = capi.pic_adjoint_buffer_bytes(self.handle, int(n_steps), int(checkpoint_every))
        if getattr(self, "_adj_buf", None) is None or self._adj_buf.numel() < nbytes:
            self._adj_buf = None
            self._adj_buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return capi.pic_adjoint_forward(self.handle, int(n_steps), int(checkpoint_every),
                                        weights, self._adj_buf.data_ptr(), int(self._adj_buf.numel()))

    def adjoint_backward(self, scale: float = 1.0, device: bool = False):
        """(scale dJ/dx0, scale dJ/dv0) as (N, 3) float64 arrays in load order."""
        import torch

        N = self.n_particles
        if device:
            gx = torch.empty((N, 3), dtype=torch.float64, device=self.device)
            gv = torch.empty((N, 3), dtype=torch.float64, device=self.device)
            capi.pic_adjoint_backward(self.handle, float(scale), gx.data_ptr(), gv.data_ptr(), True)
            return gx, gv
        gx = np.empty((N, 3), dtype=np.float64)
        gv = np.empty((N, 3), dtype=np.float64)
        capi.pic_adjoint_backward(self.handle, float(scale), gx.ctypes.data, gv.ctypes.data, False)
        return gx, gv

    def adjoint_param_gradient(self):
        """(dJ/dB_x, dJ/dB_y, dJ/dB_z, dJ/d(wz2)) of the last adjoint_backward
        (the run must be created with options including PIC_OPT_ADJOINT_PARAMS)."""
        return capi.pic_adjoint_param_gradient(self.handle)

    def dot(self, a, b) -> float:
        """FP64 sum of a * b over two CUDA float64 tensors of equal size."""
        a = a.contiguous()
        b = b.contiguous()
        assert a.numel() == b.numel() and a.is_cuda and b.is_cuda
        return capi.pic_dot_f64(self.handle, a.data_ptr(), b.data_ptr(), a.numel())

    def flags(self, clear: bool = False) -> int:
        return capi.pic_device_flags(self.handle, clear)

    def close(self):
        if not self._closed:
            try:
                self.stream.synchronize()
            except Exception:
                pass
            capi.pic_destroy(self.handle)
            self._closed = True

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
