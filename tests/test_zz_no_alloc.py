"""Allocation-free diagnostics (lbm_diag_noalloc), called through the C ABI.

Some callers may not allocate device memory while they run: a program whose
device memory is all handed out by its own pool allocator, or a tight
time-stepping loop where cudaMalloc/cudaFree would synchronise the device.
For them the library offers one entry point that works on the caller's own
population array with a fixed scratch array compiled into the library.

This test checks that it reports the same mass, momentum, per-slice liquid
area and per-slice maximum density as the context-based lbm_diag, on two
calls in a row (host outputs, then device outputs), for FP64 and FP32
population arrays and for the FP16 / BF16 deviation formats (read from the
context's own stored copy, with a reference density and scale other than 1);
and that a state with a non-positive density is reported as LBM_ENONFINITE
with the outputs still written.  The file is named so that pytest collects
it last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import inputs, lbm  # noqa: E402

RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


def _close(a, b, scale):
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= 1e-12 * scale


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_noalloc_diagnostics_match_lbm_diag_on_two_calls(storage):
    nx, ny, nz = 48, 40, 72
    code = lbm.STORAGE[storage]
    tdtype = torch.float64 if storage == "f64" else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    with lbm.Lattice(nx, ny, nz, storage=storage) as L:
        L.init_ligament(10.0, 0.05, RL, RV)
        f64 = torch.empty((19, nz, ny, nx), dtype=torch.float64, device="cuda")
        for call in range(2):
            L.step(25)
            ref = L.diag(RL, RV)
            L.get_populations(f64)  # the caller's own copy of the state
            f = f64.to(tdtype)      # exact for FP32: the values came from FP32
            on_device = call  # first call: host outputs; second: device outputs
            if on_device:
                mass_t = torch.zeros(1, dtype=torch.float64, device="cuda")
                mom_t = torch.zeros(3, dtype=torch.float64, device="cuda")
                area_t = torch.zeros(nz, dtype=torch.float64, device="cuda")
                mx_t = torch.zeros(nz, dtype=torch.float64, device="cuda")
                st = lbm.lbm_diag_noalloc(f.data_ptr(), code, nx, ny, nz, 1.0, 1.0, RL, RV,
                                          mass_t.data_ptr(), mom_t.data_ptr(), area_t.data_ptr(),
                                          mx_t.data_ptr(), 1, stream)
                mass, mom = float(mass_t.item()), mom_t.cpu().numpy()
                area, mx = area_t.cpu().numpy(), mx_t.cpu().numpy()
            else:
                m = ctypes.c_double()
                mo = (ctypes.c_double * 3)()
                area, mx = np.empty(nz), np.empty(nz)
                st = lbm.lbm_diag_noalloc(f.data_ptr(), code, nx, ny, nz, 1.0, 1.0, RL, RV,
                                          ctypes.addressof(m), ctypes.addressof(mo), area.ctypes.data,
                                          mx.ctypes.data, 0, stream)
                mass, mom = m.value, np.array(mo[:])
            assert st == lbm.LBM_OK, call
            assert _close(mass, ref["mass"], ref["mass"]), call
            assert _close(mom, ref["mom"], ref["mass"]), call
            assert _close(area, ref["area_z"], nx * ny), call
            assert _close(mx, ref["maxrho_z"], 1.0), call


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_noalloc_diagnostics_of_16_bit_deviation_storage(storage):
    """The caller passes the context's stored 16-bit copy as it is, with the
    rho_ref and dev_scale that encoded it; two calls in a row."""
    nx, ny, nz = 40, 36, 50
    rho_ref, scale = 0.8, 2.0
    stream = torch.cuda.current_stream().cuda_stream
    with lbm.Lattice(nx, ny, nz, storage=storage, rho_ref=rho_ref, dev_scale=scale) as L:
        L.init_ligament(8.0, 0.05, RL, RV)
        for call in range(2):
            L.step(15 + call)
            ref = L.diag(RL, RV)
            f = L.stored_populations()
            m = ctypes.c_double()
            mo = (ctypes.c_double * 3)()
            area, mx = np.empty(nz), np.empty(nz)
            st = lbm.lbm_diag_noalloc(f.data_ptr(), lbm.STORAGE[storage], nx, ny, nz, rho_ref, scale, RL, RV,
                                      ctypes.addressof(m), ctypes.addressof(mo), area.ctypes.data,
                                      mx.ctypes.data, 0, stream)
            assert st == lbm.LBM_OK, call
            assert _close(m.value, ref["mass"], ref["mass"]), call
            assert _close(np.array(mo[:]), ref["mom"], ref["mass"]), call
            assert _close(area, ref["area_z"], nx * ny), call
            assert _close(mx, ref["maxrho_z"], 1.0), call


def test_noalloc_diagnostics_flag_a_non_positive_density():
    nx, ny, nz = 32, 32, 24
    stream = torch.cuda.current_stream().cuda_stream
    with lbm.Lattice(nx, ny, nz, storage="f32") as L:
        L.init_ligament(6.0, 0.05, RL, RV)
        f = torch.empty((19, nz, ny, nx), dtype=torch.float64, device="cuda")
        L.get_populations(f)
    f32 = f.to(torch.float32)
    f32[:, 5, 7, 9] = -0.01  # rho = -0.19 in one cell
    m = ctypes.c_double()
    mo = (ctypes.c_double * 3)()
    area, mx = np.full(nz, -1.0), np.full(nz, -1.0)
    st = lbm.lbm_diag_noalloc(f32.data_ptr(), lbm.STORAGE["f32"], nx, ny, nz, 1.0, 1.0, RL, RV,
                              ctypes.addressof(m), ctypes.addressof(mo), area.ctypes.data, mx.ctypes.data, 0,
                              stream)
    assert st == lbm.LBM_ENONFINITE
    want = float(f32.double().sum())
    assert abs(m.value - want) <= 1e-6 * abs(want)  # float sums over runs of 8 cells
    assert (area >= 0).all() and (mx > 0).all()
