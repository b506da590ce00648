"""pfl_phi_moments_static: the phase-field reduction for callers that may not
allocate device memory (an application whose GPU memory all belongs to its own
pool, a plugin handed fixed buffers, a loop that cannot afford an allocation's
synchronisation).  It must give the same sums as pfl_diag, which reduces the
same field with workspace scratch, on consecutive calls that share the static
scratch array.  Collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2206_11637_gb300 import _lib as L
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _entry():
    from paper_2206_11637_gb300 import build
    build.build_library()
    lib = L.load()
    fn = lib.pfl_phi_moments_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p]
    return lib, fn


def _static_sums(fn, phi_dev, p, fp64, stream=None):
    out = np.full(8, np.nan)
    nf = ctypes.c_longlong(-1)
    stream = (torch.cuda.current_stream() if stream is None else stream).cuda_stream
    st = fn(ctypes.c_void_p(phi_dev.data_ptr()), 1 if fp64 else 0, p.nx, p.ny, p.nz,
            out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nf), ctypes.c_void_p(stream))
    return st, out, nf.value


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_scratch_reduction_matches_pfl_diag(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib, fn = _entry()
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, u0, p0 = W.rising_bubble(24, 40, 20, D=10.0, xi=4.0, M=0.05)
    s = Simulation(p, phi0, u0, p0, precision=precision)
    fp64 = precision == "fp64"
    for call, steps in enumerate((30, 17)):   # two calls in a row, on changing fields
        s.step(steps)
        ref, nf_ref = s.diag()
        phi_dev = torch.empty(p.cells, dtype=torch.float64, device="cuda")
        s.fields(out={"phi": phi_dev})
        if not fp64:
            phi_dev = phi_dev.to(torch.float32)   # exact: the FP32 path keeps phi in FP32
        st, out, nf = _static_sums(fn, phi_dev, p, fp64)
        assert st == L.PFL_OK, lib.pfl_last_error()
        assert nf == nf_ref == 0
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-9), (call, out, ref)


def test_static_scratch_rejects_oversized_lattice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib, fn = _entry()
    phi = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = np.zeros(8)
    st = fn(ctypes.c_void_p(phi.data_ptr()), 1, 2048, 2048, 1024, out.ctypes.data_as(ctypes.c_void_p), None, None)
    assert st == L.PFL_ERR_ARG
    assert "at most" in lib.pfl_last_error().decode()


def test_static_scratch_keeps_current_device_and_runs_on_a_second_stream():
    """The call leaves the caller's current device as it was, and a call on a
    second stream, ordered after the first by synchronisation, gives the same
    sums as pfl_diag."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib, fn = _entry()
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, u0, p0 = W.rising_bubble(24, 40, 20, D=10.0, xi=4.0, M=0.05)
    s = Simulation(p, phi0, u0, p0, precision="fp64")
    s.step(11)
    ref, _ = s.diag()
    phi_dev = torch.empty(p.cells, dtype=torch.float64, device="cuda")
    s.fields(out={"phi": phi_dev})
    before = torch.cuda.current_device()
    st, out, nf = _static_sums(fn, phi_dev, p, True)
    assert st == L.PFL_OK, lib.pfl_last_error()
    assert torch.cuda.current_device() == before
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    st, out2, nf2 = _static_sums(fn, phi_dev, p, True, stream=side)
    assert st == L.PFL_OK, lib.pfl_last_error()
    assert torch.cuda.current_device() == before
    assert np.allclose(out2, ref, rtol=1e-12, atol=1e-9)
    assert np.array_equal(out, out2)


def test_static_scratch_on_a_device_that_is_not_current():
    """phi held by another GPU: the sums come from that GPU's scratch and the
    caller's current device stays current."""
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    lib, fn = _entry()
    p, phi0, _, _ = W.static_drop(20, 6.0)
    torch.cuda.set_device(0)
    phi_other = torch.from_numpy(phi0.reshape(-1).copy()).to("cuda:1")
    with torch.cuda.device(1):
        other_stream = torch.cuda.current_stream()
    st, out, nf = _static_sums(fn, phi_other, p, True, stream=other_stream)
    assert st == L.PFL_OK, lib.pfl_last_error()
    assert torch.cuda.current_device() == 0
    assert abs(out[0] - phi0.sum()) <= 1e-9 * phi0.sum()
