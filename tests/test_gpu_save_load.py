"""Saved states (pfl_save / pfl_load): a run saved at step t and resumed in a
second context reaches bitwise the state the first run reaches, in every
precision (FP16S keeps its rounding seeds: the step count is part of the
state), on both engines, with solid cells, and through host and device
buffers.  Mismatched lattices, short buffers and foreign bytes are refused.
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


def sim(p, phi0, u0=None, p0=None, precision="fp64"):
    from paper_2206_11637_gb300.pflbm import Simulation
    return Simulation(p, phi0, u0, p0, precision=precision)


def state(s):
    h, g = s.populations()
    return [h, g] + list(s.fields())


def bubble():
    return W.rising_bubble(20, 36, 20, D=10.0, xi=4.0, M=0.05)


def drop_on_block():
    p = W.Params(24, 24, 16, (0, 0, 1, 1, 0, 0), 1.0, 0.01, 0.02, 0.05, 2e-4, 0.03, 4.0, (0.0, -2e-6, 0.0))
    x, y, z = W.coords(p)
    p.solid = ((np.abs(x - 11.5) < 5) & (y < 6) & (np.abs(z - 7.5) < 4)).astype(np.uint8)
    phi0 = W.sphere(p, (11.5, 14.0, 7.5), 5.0, heavy_inside=True)
    return p, phi0, None, None


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("engine", [0, 1])
def test_resume_is_bitwise(precision, engine):
    p, phi0, u0, p0 = bubble()
    p.engine = engine
    a = sim(p, phi0, u0, p0, precision)
    a.step(37)                  # odd: the in-place engine's swapped layout
    saved = a.save()
    a.step(45)
    ref = state(a)
    b = sim(p, np.full(p.shape, 0.5), None, None, precision)
    b.step(3)                   # another state and step count, overwritten by the load
    b.load(saved)
    assert b.time == 37
    b.step(45)
    for x, y in zip(state(b), ref):
        assert np.array_equal(x, y)


def test_resume_with_solids_through_a_device_buffer():
    p, phi0, u0, p0 = drop_on_block()
    a = sim(p, phi0, u0, p0, "fp16s")
    a.step(40)
    buf = torch.empty(int(a.lib.pfl_state_bytes(a.ctx)), dtype=torch.uint8, device="cuda")
    a.save(buf)
    a.step(40)
    ref = state(a)
    b = sim(p, np.full(p.shape, 0.5), None, None, "fp16s")   # same solid cells, another state
    b.load(buf)
    b.step(40)
    for x, y in zip(state(b), ref):
        assert np.array_equal(x, y)


def test_load_refusals():
    from paper_2206_11637_gb300 import _lib as L
    p, phi0, u0, p0 = bubble()
    a = sim(p, phi0, u0, p0, "fp32")
    a.step(4)
    saved = a.save()
    s = a.lib
    # short buffer on save and on load
    small = np.zeros(100, np.uint8)
    assert s.pfl_save(a.ctx, small.ctypes.data, small.nbytes) == L.PFL_ERR_ARG
    assert s.pfl_load(a.ctx, saved.ctypes.data, saved.nbytes - 1) == L.PFL_ERR_ARG
    # not a state
    junk = np.zeros(saved.nbytes, np.uint8)
    assert s.pfl_load(a.ctx, junk.ctypes.data, junk.nbytes) == L.PFL_ERR_ARG
    # another precision, another lattice
    b = sim(p, phi0, u0, p0, "fp16s")
    assert s.pfl_load(b.ctx, saved.ctypes.data, saved.nbytes) == L.PFL_ERR_ARG
    q, phi1, _, _ = W.rising_bubble(20, 36, 22, D=10.0, xi=4.0, M=0.05)
    c = sim(q, phi1, None, None, "fp32")
    assert s.pfl_load(c.ctx, saved.ctypes.data, saved.nbytes) == L.PFL_ERR_ARG
    # a state with solid cells into a context without them
    pd, phid, _, _ = drop_on_block()
    d = sim(pd, phid, None, None, "fp32")
    sd = d.save()
    pd.solid = None
    e = sim(pd, phid, None, None, "fp32")
    assert s.pfl_load(e.ctx, sd.ctypes.data, sd.nbytes) == L.PFL_ERR_STATE
    # the refused loads left the contexts usable
    a.step(2)
    assert a.time == 6
