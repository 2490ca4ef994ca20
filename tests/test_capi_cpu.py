"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function declared in include/pic.h, and validates configurations."""
import ctypes as C
import os
import re

import pytest

from paper_2205_11052_gb300 import build, capi
from paper_2205_11052_gb300.sim import make_structs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load_library()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(pic_\w+)\s*\(", src, re.M))
    return names


def test_every_declared_function_is_exported(lib):
    declared = _declared()
    assert "pic_step" in declared and "pic_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
    # and the binding knows each of them under the same name
    assert declared == set(capi.exported_symbols())


def _create(**kw):
    args = dict(n=(16, 16, 16), L=(1.0, 1.0, 1.0), n_particles=1000, dt=0.1)
    args.update(kw)
    return capi.pic_create(*make_structs(**args))


def test_create_and_sizes_without_gpu(lib):
    h = _create()
    s = capi.pic_buffer_sizes(h)
    assert s.workspace_bytes > 16 ** 3 * (4 + 16) + 2 * 1000 * 32
    assert s.workspace_align == 256
    assert s.grid_nodes == 16 ** 3
    assert s.particle_capacity == 1000
    capi.pic_destroy(h)


@pytest.mark.parametrize("kw", [
    dict(n=(0, 4, 4)), dict(n=(1, 4, 4)), dict(n=(4, 2000, 4)), dict(L=(1.0, -1.0, 1.0)),
    dict(L=(1.0, float("nan"), 1.0)), dict(dt=0.0), dict(dt=float("inf")),
    dict(n_particles=-1), dict(n_particles=2 ** 31), dict(q_over_m=0.0),
    dict(mode=(9, 0, 0)), dict(mode_comp=3), dict(block=48), dict(block=512),
    dict(chunk=8), dict(chunk=4096), dict(guard=-1), dict(B=(0.0, float("nan"), 0.0)),
    dict(options=8), dict(stray_rebin=-1e-3), dict(stray_rebin=float("nan")),
])
def test_create_rejects_bad_configs(lib, kw):
    with pytest.raises(capi.PicError) as e:
        _create(**kw)
    assert e.value.code == capi.PIC_ERR_ARG
    assert capi.pic_last_error()


def test_calls_before_binding_are_state_errors(lib):
    h = _create()
    with pytest.raises(capi.PicError) as e:
        capi.pic_step(h, 1)
    assert e.value.code == capi.PIC_ERR_STATE
    with pytest.raises(capi.PicError) as e:
        capi.pic_deposit(h)
    assert e.value.code == capi.PIC_ERR_STATE
    with pytest.raises(capi.PicError) as e:
        capi.pic_rebin_stats(h)
    assert e.value.code == capi.PIC_ERR_STATE
    assert capi.pic_selftest_timeout(h) == capi.PIC_ERR_STATE
    capi.pic_destroy(h)


def test_small_arena_is_a_capacity_error_before_any_device_work(lib):
    h = _create()
    s = capi.pic_buffer_sizes(h)
    rc = lib.pic_bind_workspace(h, C.c_void_p(256), C.c_size_t(s.workspace_bytes - 1), None)
    assert rc == capi.PIC_ERR_CAPACITY
    rc = lib.pic_bind_workspace(h, C.c_void_p(100), C.c_size_t(s.workspace_bytes), None)
    assert rc == capi.PIC_ERR_ARG
    capi.pic_destroy(h)


def test_library_missing_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        # a fresh loader pointed at a path that does not exist
        capi._lib_saved = capi._lib
        try:
            capi._lib = None
            capi.load_library(str(tmp_path / "nope.so"))
        finally:
            capi._lib = capi._lib_saved


def test_batch_create_validates_and_sizes_without_gpu(lib):
    from paper_2205_11052_gb300.sim import _d3, _i3

    _, _, params = make_structs((2, 1, 1), (1.0, 1.0, 1.0), 0, 0.1)
    good = [capi.pic_instance_t(_i3((16, 16, 16)), _d3((1.0, 1.0, 1.0)), 100, -1.0),
            capi.pic_instance_t(_i3((24, 8, 12)), _d3((2.0, 1.0, 1.5)), 50, -2.0)]
    b = capi.pic_batch_create(good, -1.0, params)
    s = capi.pic_batch_buffer_sizes(b)
    assert s.grid_nodes == 16 ** 3 + 24 * 8 * 12
    assert s.particle_capacity == 150
    capi.pic_batch_destroy(b)
    bad = [capi.pic_instance_t(_i3((16, 0, 16)), _d3((1.0, 1.0, 1.0)), 100, -1.0)]
    with pytest.raises(capi.PicError) as e:
        capi.pic_batch_create(bad, -1.0, params)
    assert e.value.code == capi.PIC_ERR_ARG
    with pytest.raises(capi.PicError):
        capi.pic_batch_create(good, 0.0, params)


def test_adjoint_buffer_with_parameter_gradients_without_gpu(lib):
    """PIC_OPT_ADJOINT_PARAMS adds each stored step's velocities (3 arrays per
    step of the reversed segment) and the per-block partials of the parameter
    sums (10 doubles for each of the 152 * 3 * 2 reverse-push blocks, plus 10)."""
    def align(b):
        return (b + 255) // 256 * 256

    n_p, n_steps, K = 1000, 30, 8
    a = _create(n_particles=n_p)
    b = _create(n_particles=n_p, options=capi.PIC_OPT_ADJOINT_PARAMS)
    sa = capi.pic_adjoint_buffer_bytes(a, n_steps, K)
    sb = capi.pic_adjoint_buffer_bytes(b, n_steps, K)
    assert sb - sa == K * 3 * align(4 * n_p) + align(8 * 10 * (152 * 3 * 2 + 1))
    with pytest.raises(capi.PicError) as e:
        capi.pic_adjoint_param_gradient(b)
    assert e.value.code == capi.PIC_ERR_STATE
    capi.pic_destroy(a)
    capi.pic_destroy(b)
