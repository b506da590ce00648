"""Parity at the full workload sizes, in the launch configuration the
benchmark times: one GPU step from a GPU state compared with one oracle step
from the same state (the oracle cannot follow millions of cells for many
steps), plus properties that hold at any size (finite fields, conserved mass).
"""
import numpy as np
import pytest

import oracle
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


def rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("fp16s", 2e-3)])
def test_capillary_wave_200x400_one_step(precision, tol):
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, _, _ = W.capillary_wave(200)        # 200 x 400 x 1, walls in y
    s = Simulation(p, phi0, precision=precision)
    s.step(101)                                  # odd count: state left by an even step
    h, g = s.populations()
    o = oracle.from_params(p, phi0)
    o.set_populations(h, g)
    s.step(1)
    o.step(1, 0)
    phi, _, pr, u = s.fields()
    ophi, _, opr, ou = o.fields()
    assert rel(phi, ophi) < tol
    assert rel(u, ou) < tol * 50


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_rising_bubble_full_size_properties(precision):
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, _, _ = W.rising_bubble()            # 128 x 384 x 128, walls everywhere
    s = Simulation(p, phi0, precision=precision)
    m0 = s.mass()
    s.step(200)
    out, nf = s.diag()
    assert nf == 0
    tol = 1e-5 if precision == "fp32" else 2e-3
    assert abs(out[0] - m0) / m0 < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("fp16s", 2e-3)])
def test_rising_bubble_128x384x128_one_step(precision, tol):
    """The full 6.29 M-cell bubble (walls everywhere, gravity, hydrostatic
    start): one GPU step against one oracle step from the same populations."""
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, u0, p0 = W.rising_bubble()
    s = Simulation(p, phi0, u0, p0, precision=precision)
    s.step(11)
    h, g = s.populations()
    o = oracle.from_params(p, phi0, u0, p0)
    o.set_populations(h, g)
    del h, g
    s.step(1)
    o.step(1, 0)
    phi, _, _, u = s.fields()
    ophi, _, _, ou = o.fields()
    assert np.all(np.isfinite(phi))
    assert rel(phi, ophi) < tol
    assert rel(u, ou) < tol * 50


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_drop_impact_512x384x512_properties(precision):
    """The 100.7 M-cell vertical impact (the benchmark's largest lattice), in
    the launch configuration it is timed in: 40 steps stay finite and
    conserve phi (34 GB of FP32 state on the device)."""
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, u0, p0 = W.drop_impact()
    s = Simulation(p, phi0, u0, p0, precision=precision)
    m0 = s.mass()
    s.step(40)
    out, nf = s.diag()
    assert nf == 0
    tol = 1e-5 if precision == "fp32" else 2e-3
    assert abs(out[0] - m0) / m0 < tol
    del s
    torch.cuda.empty_cache()
