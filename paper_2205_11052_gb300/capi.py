"""ctypes binding of the C ABI in ``include/pic.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
computation of its own: all device work runs in the CUDA library.  Loading
fails loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

PIC_OK = 0
PIC_ERR_ARG = -1
PIC_ERR_CAPACITY = -2
PIC_ERR_CUDA = -3
PIC_ERR_CUFFT = -4
PIC_ERR_DEVICE_FLAG = -5
PIC_ERR_TIMEOUT = -6
PIC_ERR_STATE = -7

PIC_FLAG_NONFINITE = 1
PIC_FLAG_BAD_CELL = 2
PIC_FLAG_TIMEOUT = 4

ERROR_NAMES = {
    PIC_ERR_ARG: "PIC_ERR_ARG",
    PIC_ERR_CAPACITY: "PIC_ERR_CAPACITY",
    PIC_ERR_CUDA: "PIC_ERR_CUDA",
    PIC_ERR_CUFFT: "PIC_ERR_CUFFT",
    PIC_ERR_DEVICE_FLAG: "PIC_ERR_DEVICE_FLAG",
    PIC_ERR_TIMEOUT: "PIC_ERR_TIMEOUT",
    PIC_ERR_STATE: "PIC_ERR_STATE",
}


class pic_grid_t(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("L", C.c_double * 3)]


class pic_species_t(C.Structure):
    _fields_ = [("q_over_m", C.c_double), ("total_charge", C.c_double),
                ("n_particles", C.c_int64)]


class pic_params_t(C.Structure):
    _fields_ = [("dt", C.c_double), ("B_ext", C.c_double * 3), ("wz2", C.c_double),
                ("tile", C.c_int32 * 3), ("guard", C.c_int32), ("sort_period", C.c_int32),
                ("diag_every", C.c_int32), ("diag_capacity", C.c_int32),
                ("mode", C.c_int32 * 3), ("mode_comp", C.c_int32), ("block", C.c_int32),
                ("chunk", C.c_int32), ("options", C.c_int32), ("seed", C.c_uint64),
                ("stray_rebin", C.c_double)]


PIC_OPT_FIXED_DEPOSIT = 1
PIC_OPT_UNIFORM_MOVE = 2
PIC_OPT_ADJOINT_PARAMS = 4


class pic_bufsizes_t(C.Structure):
    _fields_ = [("workspace_bytes", C.c_size_t), ("workspace_align", C.c_size_t),
                ("particle_capacity", C.c_int64), ("grid_nodes", C.c_int64),
                ("staging_particles", C.c_int64)]


class pic_diag_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("t_field", C.c_double), ("Wx", C.c_double),
                ("Wy", C.c_double), ("Wz", C.c_double), ("Q", C.c_double),
                ("mode_re", C.c_double), ("mode_im", C.c_double), ("t", C.c_double),
                ("Px", C.c_double), ("Py", C.c_double), ("Pz", C.c_double), ("K", C.c_double)]


class pic_instance_t(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("L", C.c_double * 3), ("n_particles", C.c_int64),
                ("total_charge", C.c_double)]


pic_handle_t = C.c_void_p
pic_batch_t = C.c_void_p

# name -> (restype, argtypes)
_SIGNATURES = {
    "pic_create": (C.c_int, [C.POINTER(pic_grid_t), C.POINTER(pic_species_t),
                             C.POINTER(pic_params_t), C.POINTER(pic_handle_t)]),
    "pic_buffer_sizes": (C.c_int, [pic_handle_t, C.POINTER(pic_bufsizes_t)]),
    "pic_bind_workspace": (C.c_int, [pic_handle_t, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pic_set_stream": (C.c_int, [pic_handle_t, C.c_void_p]),
    "pic_destroy": (None, [pic_handle_t]),
    "pic_last_error": (C.c_char_p, []),
    "pic_load_particles": (C.c_int, [pic_handle_t, C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "pic_get_particles": (C.c_int, [pic_handle_t, C.c_void_p, C.c_void_p, C.c_int]),
    "pic_get_field": (C.c_int, [pic_handle_t, C.c_void_p, C.c_void_p, C.c_int]),
    "pic_set_rho": (C.c_int, [pic_handle_t, C.c_void_p, C.c_int]),
    "pic_get_counts": (C.c_int, [pic_handle_t, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pic_rebin_stats": (C.c_int, [pic_handle_t, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pic_selftest_timeout": (C.c_int, [pic_handle_t]),
    "pic_sort": (C.c_int, [pic_handle_t]),
    "pic_deposit": (C.c_int, [pic_handle_t]),
    "pic_field_solve": (C.c_int, [pic_handle_t]),
    "pic_gather_push": (C.c_int, [pic_handle_t]),
    "pic_step": (C.c_int, [pic_handle_t, C.c_int]),
    "pic_diagnostics": (C.c_int, [pic_handle_t, C.POINTER(pic_diag_t), C.c_int,
                                  C.POINTER(C.c_int)]),
    "pic_device_flags": (C.c_int, [pic_handle_t, C.POINTER(C.c_int32), C.c_int]),
    "pic_field_energy_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                           C.c_void_p, C.c_void_p]),
    "pic_adjoint_buffer_bytes": (C.c_int, [pic_handle_t, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "pic_adjoint_forward": (C.c_int, [pic_handle_t, C.c_int, C.c_int, C.POINTER(C.c_double),
                                      C.c_void_p, C.c_size_t, C.POINTER(C.c_double)]),
    "pic_adjoint_backward": (C.c_int, [pic_handle_t, C.c_double, C.c_void_p, C.c_void_p, C.c_int]),
    "pic_adjoint_param_gradient": (C.c_int, [pic_handle_t, C.POINTER(C.c_double)]),
    "pic_dot_f64": (C.c_int, [pic_handle_t, C.c_void_p, C.c_void_p, C.c_int64,
                              C.POINTER(C.c_double)]),
    "pic_batch_create": (C.c_int, [C.POINTER(pic_instance_t), C.c_int, C.c_double,
                                   C.POINTER(pic_params_t), C.POINTER(pic_batch_t)]),
    "pic_batch_buffer_sizes": (C.c_int, [pic_batch_t, C.POINTER(pic_bufsizes_t)]),
    "pic_batch_bind_workspace": (C.c_int, [pic_batch_t, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pic_batch_set_stream": (C.c_int, [pic_batch_t, C.c_void_p]),
    "pic_batch_destroy": (None, [pic_batch_t]),
    "pic_batch_load_particles": (C.c_int, [pic_batch_t, C.c_void_p, C.c_void_p, C.c_int]),
    "pic_batch_step": (C.c_int, [pic_batch_t, C.c_int]),
    "pic_batch_diagnostics": (C.c_int, [pic_batch_t, C.POINTER(pic_diag_t), C.c_int,
                                        C.POINTER(C.c_int)]),
    "pic_batch_get_particles": (C.c_int, [pic_batch_t, C.c_void_p, C.c_void_p, C.c_int]),
    "pic_enable_timers": (C.c_int, [pic_handle_t, C.c_int]),
    "pic_read_timers": (C.c_int, [pic_handle_t, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
}

PHASES = ("sort", "deposit", "solve", "push", "diag")

_lib = None


class PicError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        self.code = code
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {message}")


def library_path() -> str:
    return _build.LIB_PATH


def load_library(path: str | None = None):
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(
            f"CUDA library {p} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` "
            "(there is no CPU fallback)")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGNATURES)


def check(code: int, where: str) -> int:
    if code != PIC_OK:
        msg = load_library().pic_last_error()
        raise PicError(code, where, msg.decode() if msg else "")
    return code


def _call(name, *args):
    return getattr(load_library(), name)(*args)


# Thin wrappers with the C names ------------------------------------------------

def pic_create(grid: pic_grid_t, species: pic_species_t, params: pic_params_t) -> pic_handle_t:
    h = pic_handle_t()
    check(_call("pic_create", C.byref(grid), C.byref(species), C.byref(params), C.byref(h)),
          "pic_create")
    return h


def pic_buffer_sizes(h) -> pic_bufsizes_t:
    out = pic_bufsizes_t()
    check(_call("pic_buffer_sizes", h, C.byref(out)), "pic_buffer_sizes")
    return out


def pic_bind_workspace(h, dev_ptr: int, nbytes: int, stream: int) -> None:
    check(_call("pic_bind_workspace", h, C.c_void_p(dev_ptr), C.c_size_t(nbytes),
                C.c_void_p(stream)), "pic_bind_workspace")


def pic_set_stream(h, stream: int) -> None:
    check(_call("pic_set_stream", h, C.c_void_p(stream)), "pic_set_stream")


def pic_destroy(h) -> None:
    _call("pic_destroy", h)


def pic_last_error() -> str:
    m = _call("pic_last_error")
    return m.decode() if m else ""


def pic_load_particles(h, x_ptr: int, v_ptr: int, n: int, src_is_device: bool) -> None:
    check(_call("pic_load_particles", h, C.c_void_p(x_ptr), C.c_void_p(v_ptr), C.c_int64(n),
                C.c_int(1 if src_is_device else 0)), "pic_load_particles")


def pic_get_particles(h, x_ptr: int, v_ptr: int, dst_is_device: bool) -> None:
    check(_call("pic_get_particles", h, C.c_void_p(x_ptr), C.c_void_p(v_ptr),
                C.c_int(1 if dst_is_device else 0)), "pic_get_particles")


def pic_get_field(h, rho_ptr: int | None, E_ptr: int | None, dst_is_device: bool) -> None:
    check(_call("pic_get_field", h, C.c_void_p(rho_ptr or 0), C.c_void_p(E_ptr or 0),
                C.c_int(1 if dst_is_device else 0)), "pic_get_field")


def pic_set_rho(h, rho_ptr: int, src_is_device: bool) -> None:
    check(_call("pic_set_rho", h, C.c_void_p(rho_ptr), C.c_int(1 if src_is_device else 0)),
          "pic_set_rho")


def pic_get_counts(h):
    n, s = C.c_int64(), C.c_int64()
    check(_call("pic_get_counts", h, C.byref(n), C.byref(s)), "pic_get_counts")
    return n.value, s.value


def pic_selftest_timeout(h) -> int:
    """Status of one bounded device wait that is left to run out (PIC_ERR_TIMEOUT expected)."""
    return int(_call("pic_selftest_timeout", h))


def pic_rebin_stats(h):
    """(re-binnings since the load, strays since the last re-binning decision)."""
    r, s = C.c_int64(), C.c_int64()
    check(_call("pic_rebin_stats", h, C.byref(r), C.byref(s)), "pic_rebin_stats")
    return int(r.value), int(s.value)


def pic_sort(h) -> None:
    check(_call("pic_sort", h), "pic_sort")


def pic_deposit(h) -> None:
    check(_call("pic_deposit", h), "pic_deposit")


def pic_field_solve(h) -> None:
    check(_call("pic_field_solve", h), "pic_field_solve")


def pic_gather_push(h) -> None:
    check(_call("pic_gather_push", h), "pic_gather_push")


def pic_step(h, n: int) -> None:
    check(_call("pic_step", h, C.c_int(n)), "pic_step")


def pic_diagnostics(h, max_records: int):
    buf = (pic_diag_t * max(1, max_records))()
    n = C.c_int()
    code = _call("pic_diagnostics", h, buf, C.c_int(max_records), C.byref(n))
    recs = [buf[i] for i in range(n.value)]
    check(code, "pic_diagnostics")
    return recs


def pic_device_flags(h, clear: bool = False) -> int:
    f = C.c_int32()
    check(_call("pic_device_flags", h, C.byref(f), C.c_int(1 if clear else 0)), "pic_device_flags")
    return f.value


def pic_enable_timers(h, enable: bool = True) -> None:
    check(_call("pic_enable_timers", h, C.c_int(1 if enable else 0)), "pic_enable_timers")


def pic_read_timers(h):
    """{phase: (ms, calls)} plus the library's kernel-launch count."""
    ms = (C.c_double * len(PHASES))()
    calls = (C.c_int64 * len(PHASES))()
    launches = C.c_int64()
    check(_call("pic_read_timers", h, ms, calls, C.byref(launches)), "pic_read_timers")
    return {p: (ms[i], calls[i]) for i, p in enumerate(PHASES)}, launches.value


PIC_NOALLOC_MAX_NODES = 134217728


def pic_field_energy_noalloc(rho_ptr: int, E_ptr: int, n_nodes: int, cell_volume: float,
                             out_ptr: int, stream: int) -> None:
    """(Wx, Wy, Wz, Q) into 4 device doubles at out_ptr; allocates nothing."""
    check(_call("pic_field_energy_noalloc", C.c_void_p(rho_ptr), C.c_void_p(E_ptr),
                C.c_int64(n_nodes), C.c_double(cell_volume), C.c_void_p(out_ptr),
                C.c_void_p(stream)), "pic_field_energy_noalloc")


def pic_adjoint_buffer_bytes(h, n_steps: int, checkpoint_every: int) -> int:
    out = C.c_size_t()
    check(_call("pic_adjoint_buffer_bytes", h, C.c_int(n_steps), C.c_int(checkpoint_every),
                C.byref(out)), "pic_adjoint_buffer_bytes")
    return out.value


def pic_adjoint_forward(h, n_steps: int, checkpoint_every: int, weights, buf_ptr: int,
                        nbytes: int) -> float:
    w = (C.c_double * 3)(*[float(a) for a in weights])
    J = C.c_double()
    check(_call("pic_adjoint_forward", h, C.c_int(n_steps), C.c_int(checkpoint_every), w,
                C.c_void_p(buf_ptr), C.c_size_t(nbytes), C.byref(J)), "pic_adjoint_forward")
    return J.value


def pic_adjoint_backward(h, scale: float, gx_ptr: int, gv_ptr: int, dst_is_device: bool) -> None:
    check(_call("pic_adjoint_backward", h, C.c_double(scale), C.c_void_p(gx_ptr),
                C.c_void_p(gv_ptr), C.c_int(1 if dst_is_device else 0)), "pic_adjoint_backward")


def pic_adjoint_param_gradient(h):
    """(dJ/dB_x, dJ/dB_y, dJ/dB_z, dJ/d(wz2)) of the last backward pass."""
    out = (C.c_double * 4)()
    check(_call("pic_adjoint_param_gradient", h, out), "pic_adjoint_param_gradient")
    return tuple(out)


def pic_dot_f64(h, a_ptr: int, b_ptr: int, n: int) -> float:
    out = C.c_double()
    check(_call("pic_dot_f64", h, C.c_void_p(a_ptr), C.c_void_p(b_ptr), C.c_int64(n),
                C.byref(out)), "pic_dot_f64")
    return out.value


def pic_batch_create(instances, q_over_m: float, params: pic_params_t):
    arr = (pic_instance_t * len(instances))(*instances)
    b = pic_batch_t()
    check(_call("pic_batch_create", arr, C.c_int(len(instances)), C.c_double(q_over_m),
                C.byref(params), C.byref(b)), "pic_batch_create")
    return b


def pic_batch_buffer_sizes(b) -> pic_bufsizes_t:
    out = pic_bufsizes_t()
    check(_call("pic_batch_buffer_sizes", b, C.byref(out)), "pic_batch_buffer_sizes")
    return out


def pic_batch_bind_workspace(b, dev_ptr: int, nbytes: int, stream: int) -> None:
    check(_call("pic_batch_bind_workspace", b, C.c_void_p(dev_ptr), C.c_size_t(nbytes),
                C.c_void_p(stream)), "pic_batch_bind_workspace")


def pic_batch_set_stream(b, stream: int) -> None:
    check(_call("pic_batch_set_stream", b, C.c_void_p(stream)), "pic_batch_set_stream")


def pic_batch_destroy(b) -> None:
    _call("pic_batch_destroy", b)


def pic_batch_load_particles(b, x_ptr: int, v_ptr: int, src_is_device: bool) -> None:
    check(_call("pic_batch_load_particles", b, C.c_void_p(x_ptr), C.c_void_p(v_ptr),
                C.c_int(1 if src_is_device else 0)), "pic_batch_load_particles")


def pic_batch_step(b, n: int) -> None:
    check(_call("pic_batch_step", b, C.c_int(n)), "pic_batch_step")


def pic_batch_diagnostics(b, max_records: int, n_inst: int):
    buf = (pic_diag_t * max(1, max_records * n_inst))()
    n = C.c_int()
    code = _call("pic_batch_diagnostics", b, buf, C.c_int(max_records), C.byref(n))
    recs = [[buf[r * n_inst + i] for i in range(n_inst)] for r in range(n.value)]
    check(code, "pic_batch_diagnostics")
    return recs


def pic_batch_get_particles(b, x_ptr: int, v_ptr: int, dst_is_device: bool) -> None:
    check(_call("pic_batch_get_particles", b, C.c_void_p(x_ptr), C.c_void_p(v_ptr),
                C.c_int(1 if dst_is_device else 0)), "pic_batch_get_particles")
