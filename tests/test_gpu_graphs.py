"""Graph-replayed steps (pfl_step advances whole runs of graph_k fused steps by
replaying a CUDA graph) against steps launched one by one: bitwise equal
states in every precision, including the FP16 stochastic rounding, whose
seeds the replayed launches read from the device step count.  Step counts
that are not multiples of graph_k, several graph states (a replay started at
an odd step) and the argument checks."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("case", ["wave", "bubble", "wave_d2q9"])
def test_graph_replay_equals_single_launches(precision, case):
    build = {"wave": lambda: W.capillary_wave(40, ny=48, a0=1.5, xi=5.0, sigma=1e-4, nu=0.01),
             "bubble": lambda: W.rising_bubble(20, 36, 20, D=10.0, xi=4.0, M=0.05),
             "wave_d2q9": lambda: W.capillary_wave(40, ny=48, a0=1.5, xi=5.0, sigma=1e-4, nu=0.01)}[case]
    out = []
    for k in (0, 8):
        p, phi0, u0, p0 = build()
        if case == "wave_d2q9":
            p.h_lattice = 9
        s = sim(p, phi0, u0, p0, precision)
        s.set_graph_steps(k)
        s.step(3)        # graphs start at an odd step: the other (ab, cur) state
        s.step(21)       # two replays and five single launches
        s.fields()       # a read between runs
        s.step(16)
        out.append(state(s))
        assert s.time == 40
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_graph_steps_argument_checks():
    from paper_2206_11637_gb300 import _lib as L
    p, phi0, u0, p0 = W.static_drop(16, 5.0)
    s = sim(p, phi0, u0, p0, "fp32")
    for bad in (-2, 3, 4098):
        assert s.lib.pfl_set_graph_steps(s.ctx, bad) == L.PFL_ERR_ARG
    s.set_graph_steps(2)
    s.step(5)
    s.set_graph_steps(0)
    s.step(5)
    assert s.time == 10


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_interface_height_matches_the_fields(precision):
    """pfl_interface_height equals the host's first-crossing interpolation on
    the same phi, in every column tried; a column without a crossing is NaN."""
    import analytic as A
    p, phi0, u0, p0 = W.capillary_wave(48, ny=40, a0=2.0, xi=4.0, sigma=1e-3, nu=0.01)
    s = sim(p, phi0, u0, p0, precision)
    s.step(50)
    phi = s.phi()
    for x in (0, 7, 47):
        want = A.interface_height(phi[0, :, x])
        assert s.interface_height(x, 0) == want
    q, _, _, _ = W.static_drop(16, 5.0)
    d = sim(q, np.ones(q.shape), None, None, precision)
    assert np.isnan(d.interface_height(3, 3))
    from paper_2206_11637_gb300 import _lib as L
    y = np.zeros(1)
    assert d.lib.pfl_interface_height(d.ctx, 16, 0, y.ctypes.data) == L.PFL_ERR_ARG
