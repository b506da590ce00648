"""The library's calls leave the caller's current device as they found it.

A context (or a batch) lives on the device that holds its workspace.  Each
call of the C-ABI makes that device current while it runs and gives the
caller's current device back before it returns, so the caller's own CUDA work
keeps going to the device it chose.  With two devices, a context on the
device that is not current gives the same states as one on the current device.
"""
import numpy as np
import pytest

from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


def _bubble():
    return W.rising_bubble(24, 40, 20, D=10.0, xi=4.0, M=0.05)


def _exercise(s, expect):
    """Every kind of single-lattice call, checking the current device after each."""
    s.step(8)
    assert torch.cuda.current_device() == expect
    s.fields()
    assert torch.cuda.current_device() == expect
    s.diag()
    s.max_speed()
    s.interface_height(3, 3)
    assert torch.cuda.current_device() == expect
    state = s.save()
    s.step(3)
    s.load(state)
    s.populations()
    assert torch.cuda.current_device() == expect
    s.set_graph_steps(4)
    s.step(9)
    assert torch.cuda.current_device() == expect


def test_calls_keep_the_current_device():
    from paper_2206_11637_gb300.pflbm import Simulation
    from paper_2206_11637_gb300.batch import Batch
    before = torch.cuda.current_device()
    p, phi0, u0, p0 = _bubble()
    s = Simulation(p, phi0, u0, p0, precision="fp32")
    assert torch.cuda.current_device() == before
    _exercise(s, before)
    s.close()
    assert torch.cuda.current_device() == before
    b = Batch(W.batched_sweep(4, small=True), precision="fp32", tune=False)
    b.step(5)
    b.diag(check=False)
    b.fields(1)
    b.close()
    assert torch.cuda.current_device() == before


def test_context_on_a_device_that_is_not_current():
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    from paper_2206_11637_gb300.pflbm import Simulation
    torch.cuda.set_device(0)
    p, phi0, u0, p0 = _bubble()
    other = Simulation(p, phi0, u0, p0, precision="fp64", device="cuda:1")
    assert torch.cuda.current_device() == 0
    _exercise(other, 0)
    here = Simulation(p, phi0, u0, p0, precision="fp64", device="cuda:0")
    _exercise(here, 0)
    a, b = other.fields(), here.fields()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    other.close()
    here.close()
    assert torch.cuda.current_device() == 0
