"""GPU test of pic_field_energy_noalloc, the reduction that allocates nothing.

It serves callers that may not allocate device memory while running (a host
application that owns a fixed memory budget, or a time-critical loop where
cudaMalloc is forbidden): its scratch lives in a static device array of the
library.  Here it is called twice in a row through the C ABI on the density
and field of a loaded state, and each result must match the FP64 field
energies and charge that pic_step's own diagnostics report for that field.  The larger grid
goes first so that partials left in the shared scratch by the first call
would corrupt the second if a call read any slot it did not write.
"""
import gc

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2205_11052_gb300 import capi  # noqa: E402
from paper_2205_11052_gb300.build import build  # noqa: E402
from paper_2205_11052_gb300.sim import Simulation  # noqa: E402

build()

REL = 1e-12   # both sides are FP64 sums of the same FP32 grid data


def _one_call(w):
    """Deposit and solve the loaded state, reduce that field with the
    allocation-free entry point, then take one pic_step: its diagnostic record
    of step 0 is computed from the same rho and E."""
    sim = Simulation.from_workload(w, diag_every=1)
    sim.deposit()
    sim.field_solve()
    nx, ny, nz = w.n
    ng = nx * ny * nz
    rho = torch.empty(ng, dtype=torch.float32, device="cuda")
    E = torch.empty(4 * ng, dtype=torch.float32, device="cuda")
    capi.pic_get_field(sim.handle, rho.data_ptr(), E.data_ptr(), True)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    dV = float(np.prod(np.asarray(w.L) / np.asarray(w.n)))
    capi.pic_field_energy_noalloc(rho.data_ptr(), E.data_ptr(), ng, dV, out.data_ptr(),
                                  sim.stream.cuda_stream)
    sim.stream.synchronize()
    got = out.cpu().numpy()
    sim.step(1)
    rec = sim.diagnostics()[-1]
    assert rec["step"] == 0
    sim.close()
    return got, np.array([rec["Wx"], rec["Wy"], rec["Wz"], rec["Q"]])


def test_noalloc_reduction_matches_step_diagnostics_on_two_calls():
    big = pi.landau(n=(64, 48, 40), ppc=2, seed=12, alpha=0.3)     # 30 blocks of partials
    small = pi.landau(n=(16, 16, 16), ppc=8, seed=13, alpha=0.3)   # 1 block
    for w in (big, small):
        got, want = _one_call(w)
        assert np.all(np.isfinite(got))
        for g, e in zip(got, want):
            assert g == pytest.approx(e, rel=REL)


def test_noalloc_calls_leave_device_memory_untouched():
    """After a first call on the device (its one-time set-up), further calls
    change neither the device's free memory nor torch's allocations, and
    repeat the first result bit for bit."""
    w = pi.landau(n=(32, 32, 24), ppc=2, seed=14, alpha=0.2)
    sim = Simulation.from_workload(w)
    sim.deposit()
    sim.field_solve()
    ng = int(np.prod(w.n))
    rho = torch.empty(ng, dtype=torch.float32, device="cuda")
    E = torch.empty(4 * ng, dtype=torch.float32, device="cuda")
    capi.pic_get_field(sim.handle, rho.data_ptr(), E.data_ptr(), True)
    outs = [torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(3)]
    dV = float(np.prod(np.asarray(w.L) / np.asarray(w.n)))
    st = sim.stream.cuda_stream
    capi.pic_field_energy_noalloc(rho.data_ptr(), E.data_ptr(), ng, dV, outs[0].data_ptr(), st)
    torch.cuda.synchronize()
    gc.collect()        # objects of earlier tests must not free memory inside the window
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for o in outs[1:]:
        capi.pic_field_energy_noalloc(rho.data_ptr(), E.data_ptr(), ng, dV, o.data_ptr(), st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() <= torch_bytes0
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    sim.close()


def test_noalloc_rejects_oversized_and_bad_arguments():
    capi.load_library()
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.PicError) as e:
        capi.pic_field_energy_noalloc(x.data_ptr(), x.data_ptr(), capi.PIC_NOALLOC_MAX_NODES + 1,
                                      1.0, out.data_ptr(), 0)
    assert e.value.code == capi.PIC_ERR_CAPACITY
    with pytest.raises(capi.PicError) as e:
        capi.pic_field_energy_noalloc(x.data_ptr(), x.data_ptr(), 0, 1.0, out.data_ptr(), 0)
    assert e.value.code == capi.PIC_ERR_ARG
