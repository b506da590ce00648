"""Failure detection through the C-ABI: a non-finite value planted from the
host.

The paper reports runs of its PFLBM that went unstable (sections "Rising
bubble" and "Taylor bubble": small mobilities, coarse bubbles).  The library
detects such a run without faulting the GPU: pfl_diag counts the cells whose
phi is NaN or Inf and returns PFL_ERR_UNSTABLE.  The failure is made on the
host -- a NaN written into one population through pfl_set_populations -- and
nothing here traps or waits on the device.  The context stays usable: later
steps run, spread the NaN to the neighbours, and the count grows.
"""
import numpy as np
import pytest

from paper_2206_11637_gb300 import _lib as L
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_planted_nan_is_counted_and_reported(precision):
    from paper_2206_11637_gb300.pflbm import Simulation
    p = W.Params(16, 12, 10, (0,) * 6, 1.0, 1e-3, 1 / 60, 1 / 60, 1e-4, 0.02, 4.0)
    phi0 = np.ones(p.shape)
    s = Simulation(p, phi0, precision=precision)
    s.step(2)
    _, nf = s.diag(check=False)
    assert nf == 0 and s.lib.pfl_diag(s.ctx, None, None) == L.PFL_OK

    h, g = s.populations()
    h[3, 4, 5, 6] = np.nan               # one population of cell (x 6, y 5, z 4)
    s.set_populations(h, g)
    _, nf = s.diag(check=False)
    assert nf == 1
    assert s.lib.pfl_diag(s.ctx, None, None) == L.PFL_ERR_UNSTABLE
    assert "non-finite" in s.lib.pfl_last_error().decode()

    s.step(3)                            # the context still steps; the NaN spreads
    _, nf3 = s.diag(check=False)
    assert nf3 > 1
    assert s.lib.pfl_diag(s.ctx, None, None) == L.PFL_ERR_UNSTABLE
    s.close()
