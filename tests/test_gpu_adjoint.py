"""Discrete adjoint of the stream-collide step against central finite
differences of the forward GPU path (FP64), against the exact derivative of
the CPU oracle (forward-mode dual numbers), and FP32 against FP64.

J is a linear functional of phi at chosen steps (bubble rise velocity, wave
mode amplitude); the gradient is taken with respect to M, xi and sigma.  The
bar is 1e-3 relative error per component against central differences with a
relative step of 1e-4 (truncation error of order 1e-8).
"""
import copy

import numpy as np
import pytest

from paper_2206_11637_gb300 import objectives as O
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PARAMS = ("mobility", "xi", "sigma")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


def forward_J(p, phi0, u0, p0, n, obs, precision="fp64"):
    from paper_2206_11637_gb300.pflbm import Simulation
    s = Simulation(p, phi0, u0, p0, precision=precision)
    J = 0.0
    for step, w in sorted(obs, key=lambda t: t[0]):
        s.step(step - s.time)
        J += float(np.dot(w, s.phi().reshape(-1)))
    return J


def fd_grad(p, phi0, u0, p0, n, obs, rel=1e-4):
    g = []
    for name in PARAMS:
        v = getattr(p, name)
        d = rel * v
        pp, pm = copy.copy(p), copy.copy(p)
        setattr(pp, name, v + d)
        setattr(pm, name, v - d)
        g.append((forward_J(pp, phi0, u0, p0, n, obs) - forward_J(pm, phi0, u0, p0, n, obs)) / (2 * d))
    return np.array(g)


def adjoint(p, phi0, u0, p0, n, obs, precision="fp64"):
    from paper_2206_11637_gb300.pflbm import Simulation
    s = Simulation(p, phi0, u0, p0, precision=precision)
    J, g = s.adjoint(n, obs)
    return J, g, s


def bubble_case():
    p, phi0, u0, p0 = W.rising_bubble(20, 36, 20, D=10.0, xi=4.0, M=0.05)
    n = 50                      # K = 8: seven checkpoints, the last segment partial
    return p, phi0, u0, p0, n, O.rise_velocity_weights(p, phi0, 20, n)


def wave_case():
    p, phi0, u0, p0 = W.capillary_wave(32, ny=32, a0=1.0, xi=4.0, M=0.02, sigma=1e-3, nu=0.02)
    n = 64
    return p, phi0, u0, p0, n, [(n, O.wave_mode_weights(p, 32.0)), (n // 2, 0.5 * O.wave_mode_weights(p, 32.0))]


@pytest.mark.parametrize("case", [bubble_case, wave_case])
def test_adjoint_matches_finite_differences(case):
    p, phi0, u0, p0, n, obs = case()
    J, g, s = adjoint(p, phi0, u0, p0, n, obs)
    assert s.time == n
    Jf = forward_J(p, phi0, u0, p0, n, obs)
    assert abs(J - Jf) <= 1e-12 * max(1.0, abs(Jf))
    gfd = fd_grad(p, phi0, u0, p0, n, obs)
    assert np.all(np.abs(gfd) > 0)
    rel = np.abs(g - gfd) / np.abs(gfd)
    assert np.all(rel < 1e-3), (g, gfd, rel)


@pytest.mark.parametrize("case", [bubble_case, wave_case])
def test_adjoint_matches_oracle_tangent(case):
    """Against the exact derivative of the FP64 CPU oracle (forward-mode
    dual numbers through the same update): both are exact up to rounding, so
    the bar is 1e-6 relative, a thousand times tighter than the finite
    differences above."""
    import oracle
    p, phi0, u0, p0, n, obs = case()
    J, g, _ = adjoint(p, phi0, u0, p0, n, obs)
    for k, name in enumerate(PARAMS):
        Jo, dJo = oracle.tangent(p, phi0, u0, p0, n, obs, name)
        assert abs(J - Jo) <= 1e-10 * max(1e-12, abs(Jo)), (J, Jo)
        assert abs(g[k] - dJo) <= 1e-6 * abs(dJo), (name, g[k], dJo)


def test_adjoint_same_on_both_engines():
    """The in-place engine's reverse sweep replays through the live arrays and
    copies each state; the fused engine's steps from slot to slot."""
    import dataclasses
    p, phi0, u0, p0, n, obs = bubble_case()
    J0, g0, s0 = adjoint(p, phi0, u0, p0, n, obs)
    J1, g1, s1 = adjoint(dataclasses.replace(p, engine=1), phi0, u0, p0, n, obs)
    assert abs(J0 - J1) <= 1e-13 * abs(J0)
    assert np.all(np.abs(g0 - g1) <= 1e-12 * np.abs(g0)), (g0, g1)
    assert np.array_equal(s0.phi(), s1.phi())


def test_adjoint_leaves_forward_state():
    p, phi0, u0, p0, n, obs = bubble_case()
    _, _, s = adjoint(p, phi0, u0, p0, n, obs)
    from paper_2206_11637_gb300.pflbm import Simulation
    r = Simulation(p, phi0, u0, p0, precision="fp64")
    r.step(n)
    assert np.abs(s.phi() - r.phi()).max() < 1e-13
    h1, g1 = s.populations()
    h2, g2 = r.populations()
    assert np.abs(h1 - h2).max() < 1e-13 and np.abs(g1 - g2).max() < 1e-13
    s.step(3)                        # the context steps on from where the forward run ended
    r.step(3)
    assert np.abs(s.phi() - r.phi()).max() < 1e-13


def test_fp32_adjoint_close_to_fp64():
    p, phi0, u0, p0, n, obs = wave_case()
    _, g64, _ = adjoint(p, phi0, u0, p0, n, obs, "fp64")
    _, g32, _ = adjoint(p, phi0, u0, p0, n, obs, "fp32")
    assert np.all(np.abs(g32 - g64) / np.abs(g64) < 1e-2), (g32, g64)


def test_full_size_bubble_adjoint_matches_finite_differences():
    """The 128x384x128 FP32 bubble (6.29 M cells, walls, gravity, hydrostatic
    start) over 2000 steps, J the mean rise velocity over the last 500, sqrt(n)
    checkpoints: the adjoint gradient against central differences of forward
    FP32 runs with a relative step of 1e-2 (FP32 rounding makes smaller steps
    noisy).  Measured on a GB300: within 1.1e-3 per component.  (At 4000 steps
    J is no longer smooth in the parameters -- FP64 central differences in
    sigma do not converge as the step shrinks -- and the exact derivative the
    adjoint returns is far from any finite difference.)"""
    p, phi0, u0, p0 = W.rising_bubble()
    n = 2000
    obs = O.rise_velocity_weights(p, phi0, n - n // 4, n)
    J, g, s = adjoint(p, phi0, u0, p0, n, obs, "fp32")
    del s
    torch.cuda.empty_cache()
    fd = []
    for name in PARAMS:
        v = getattr(p, name)
        pp, pm = copy.copy(p), copy.copy(p)
        setattr(pp, name, v * 1.01)
        setattr(pm, name, v * 0.99)
        fd.append((forward_J(pp, phi0, u0, p0, n, obs, "fp32") - forward_J(pm, phi0, u0, p0, n, obs, "fp32"))
                  / (0.02 * v))
        torch.cuda.empty_cache()
    fd = np.array(fd)
    assert np.all(np.abs(g - fd) <= 1e-2 * np.abs(fd)), (g, fd)


def test_adjoint_rejects_fp16s_and_bad_observations():
    from paper_2206_11637_gb300.pflbm import Simulation
    from paper_2206_11637_gb300 import _lib as L
    p, phi0, u0, p0, n, obs = wave_case()
    s = Simulation(p, phi0, u0, p0, precision="fp16s")
    with pytest.raises(L.PFLError) as e:
        s.adjoint(n, obs)
    assert e.value.status == L.PFL_ERR_STATE
    s = Simulation(p, phi0, u0, p0, precision="fp64")
    with pytest.raises(L.PFLError) as e:
        s.adjoint(n, [(n + 1, obs[0][1])])
    assert e.value.status == L.PFL_ERR_ARG


def test_autograd_function():
    from paper_2206_11637_gb300.autograd import RolloutSetup, rollout
    p, phi0, u0, p0, n, obs = wave_case()
    setup = RolloutSetup(p, phi0, n, obs, u0, p0, precision="fp64")
    M = torch.tensor(p.mobility, dtype=torch.float64, requires_grad=True)
    xi = torch.tensor(p.xi, dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(p.sigma, dtype=torch.float64, requires_grad=True)
    J = rollout(M, xi, sg, setup)
    (3.0 * J).backward()
    _, g, _ = adjoint(p, phi0, u0, p0, n, obs)
    assert abs(J.item() - forward_J(p, phi0, u0, p0, n, obs)) < 1e-12
    got = np.array([M.grad.item(), xi.grad.item(), sg.grad.item()])
    assert np.allclose(got, 3.0 * g, rtol=1e-12, atol=0)


def wave_frequency_case():
    """Capillary wave L x L (depth L / 2, the paper's set-up), sigma 1e-3,
    nu 0.002, rho ratio 1000, xi 4, M 0.02: the interface height of column
    x = 0 every 40 steps from a quarter period to 1.5 periods; J = the
    fitted angular frequency."""
    import analytic as A
    L = 32
    p, phi0, u0, p0 = W.capillary_wave(L, ny=L, a0=1.0, xi=4.0, M=0.02, sigma=1e-3, nu=0.002)
    k = 2 * np.pi / L
    w0 = A.capillary_omega0(p.sigma, k, p.rho_h, p.rho_l)
    T = 2 * np.pi / w0
    steps = list(range(int(T / 4) // 40 * 40, int(1.5 * T), 40))
    return p, phi0, u0, p0, steps, w0


def frequency_forward(p, phi0, u0, p0, steps, w0, precision="fp64"):
    from paper_2206_11637_gb300.pflbm import Simulation
    obj = O.WaveFrequency(steps, w0)
    s = Simulation(p, phi0, u0, p0, precision=precision)
    for t in steps:
        s.step(t - s.time)
        obj.record(t, s.phi())
    return obj


def test_wave_frequency_gradient():
    """Gradient of the capillary-wave frequency with respect to (M, xi,
    sigma), the wave objective the adjoint is built for: seed fields from a
    forward pass (the fit's implicit derivative times the derivative of the
    interpolated interface height), one adjoint of those seeds.  Checked
    against central differences of the whole pipeline (forward run, height,
    fit) at 1e-3, against the oracle's exact derivative of the same seeded
    functional at 1e-6, and d omega / d sigma against the dispersion relation
    omega^2 proportional to sigma (within 10 %)."""
    import oracle
    p, phi0, u0, p0, steps, w0 = wave_frequency_case()
    obj = frequency_forward(p, phi0, u0, p0, steps, w0)
    omega = obj.value()
    assert abs(omega / w0 - 1) < 0.15
    seeds = obj.seeds(p.shape)
    n = steps[-1]
    _, g, _ = adjoint(p, phi0, u0, p0, n, seeds)
    fd = []
    for name in PARAMS:
        v = getattr(p, name)
        d = 1e-4 * v
        pp, pm = copy.copy(p), copy.copy(p)
        setattr(pp, name, v + d)
        setattr(pm, name, v - d)
        fd.append((frequency_forward(pp, phi0, u0, p0, steps, w0).value()
                   - frequency_forward(pm, phi0, u0, p0, steps, w0).value()) / (2 * d))
    fd = np.array(fd)
    assert np.all(np.abs(g - fd) <= 1e-3 * np.abs(fd)), (g, fd)
    for k, name in enumerate(PARAMS):
        _, dJo = oracle.tangent(p, phi0, u0, p0, n, seeds, name)
        assert abs(g[k] - dJo) <= 1e-6 * abs(dJo), (name, g[k], dJo)
    assert abs(g[2] / (omega / (2 * p.sigma)) - 1) < 0.10, (g[2], omega / (2 * p.sigma))


def test_objective_rollout_autograd():
    from paper_2206_11637_gb300.autograd import RolloutSetup, objective_rollout
    p, phi0, u0, p0, steps, w0 = wave_frequency_case()
    setup = RolloutSetup(p, phi0, steps[-1], None, u0, p0, precision="fp64")
    M = torch.tensor(p.mobility, dtype=torch.float64, requires_grad=True)
    xi = torch.tensor(p.xi, dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(p.sigma, dtype=torch.float64, requires_grad=True)
    J = objective_rollout(M, xi, sg, setup, O.WaveFrequency(steps, w0))
    J.backward()
    obj = frequency_forward(p, phi0, u0, p0, steps, w0)
    assert abs(J.item() - obj.value()) <= 1e-12 * obj.value()
    _, g, _ = adjoint(p, phi0, u0, p0, steps[-1], obj.seeds(p.shape))
    got = np.array([M.grad.item(), xi.grad.item(), sg.grad.item()])
    assert np.allclose(got, g, rtol=1e-12, atol=0)
