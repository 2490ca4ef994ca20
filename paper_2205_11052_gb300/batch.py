"""Batched ensembles: many independent PIC runs advanced by one set of launches.

    ens = Ensemble([(n, L, x, v, Q), ...], dt=0.05, diag_every=1)
    ens.step(100)
    hist = ens.diagnostics()      # hist[record][instance] -> dict
    xs, vs = ens.particles()      # lists per instance

torch supplies the arena and the stream; every phase runs in the CUDA
library (pic_batch_* in include/pic.h).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .sim import _d3, _i3, make_structs


class Ensemble:
    def __init__(self, members, dt, q_over_m=-1.0, B=(0.0, 0.0, 0.0), wz2=0.0, tile=(0, 0, 0),
                 guard=0, sort_period=0, diag_every=0, diag_capacity=0, mode=(1, 0, 0),
                 mode_comp=0, chunk=0, options=0, block=0, device=None, stream=None):
        """members: sequence of (n, L, x, v, Q) with x, v (N_i, 3) float64 arrays."""
        import torch

        self.members = list(members)
        insts = []
        for n, L, x, v, Q in self.members:
            insts.append(capi.pic_instance_t(_i3(n), _d3(L), int(np.asarray(x).shape[0]), float(Q)))
        self.counts = [int(np.asarray(m[2]).shape[0]) for m in self.members]
        _, _, params = make_structs((2, 1, 1), (1.0, 1.0, 1.0), 0, dt, q_over_m, 0.0, B, wz2, tile,
                                    guard, sort_period, diag_every, diag_capacity, mode, mode_comp,
                                    block, chunk, options)
        self.handle = capi.pic_batch_create(insts, q_over_m, params)
        self._closed = False
        self.sizes = capi.pic_batch_buffer_sizes(self.handle)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.arena = torch.empty(int(self.sizes.workspace_bytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        capi.pic_batch_bind_workspace(self.handle, self.arena.data_ptr(),
                                      int(self.sizes.workspace_bytes), self.stream.cuda_stream)
        x = np.ascontiguousarray(np.concatenate([np.asarray(m[2]) for m in self.members]), np.float64)
        v = np.ascontiguousarray(np.concatenate([np.asarray(m[3]) for m in self.members]), np.float64)
        capi.pic_batch_load_particles(self.handle, x.ctypes.data, v.ctypes.data, False)

    @property
    def n_inst(self):
        return len(self.members)

    def step(self, n: int = 1):
        capi.pic_batch_step(self.handle, int(n))

    def capture(self, n: int = 1):
        """Capture n steps into a CUDA graph (one launch of the whole ensemble
        for all n steps); each ``replay()`` of the returned graph advances every
        instance by n steps.  The ensemble moves to a private stream and takes
        one eager step first, so that the captured launches find their state
        initialised."""
        import torch

        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        self.set_stream(s)
        with torch.cuda.stream(s):
            self.step(1)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.step(n)
        return g

    def set_stream(self, stream):
        self.stream = stream
        capi.pic_batch_set_stream(self.handle, stream.cuda_stream)

    def diagnostics(self, max_records: int = 4096):
        recs = capi.pic_batch_diagnostics(self.handle, max_records, self.n_inst)
        return [[dict(step=r.step, t_field=r.t_field, Wx=r.Wx, Wy=r.Wy, Wz=r.Wz, Q=r.Q,
                      mode=complex(r.mode_re, r.mode_im), t=r.t, Px=r.Px, Py=r.Py, Pz=r.Pz,
                      K=r.K) for r in row] for row in recs]

    def particles(self):
        N = sum(self.counts)
        x = np.empty((N, 3), dtype=np.float64)
        v = np.empty((N, 3), dtype=np.float64)
        capi.pic_batch_get_particles(self.handle, x.ctypes.data, v.ctypes.data, False)
        offs = np.cumsum([0] + self.counts)
        return ([x[offs[i]:offs[i + 1]] for i in range(self.n_inst)],
                [v[offs[i]:offs[i + 1]] for i in range(self.n_inst)])

    def close(self):
        if not self._closed:
            try:
                self.stream.synchronize()
            except Exception:
                pass
            capi.pic_batch_destroy(self.handle)
            self._closed = True

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
