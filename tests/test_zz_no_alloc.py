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


def _static_sums(fn, phi_dev, p, fp64):
    out = np.full(8, np.nan)
    nf = ctypes.c_longlong(-1)
    stream = torch.cuda.current_stream().cuda_stream
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
