"""The oracle's exact parameter derivatives (forward-mode, dual numbers)
against central finite differences of the oracle's own FP64 forward run.

The same templated arithmetic runs once in doubles (the oracle) and once in
dual numbers (value, derivative with respect to M, xi or sigma).  Central
differences with a relative step of 1e-4 carry a truncation error of order
1e-8 relative, so 1e-5 catches any wrong derivative rule (a product, quotient
or square root differentiated wrongly, a parameter whose seed is lost) while
leaving room for the truncation.  These derivatives are the CPU reference of
the GPU adjoint (tests/test_gpu_adjoint.py).
"""
import copy

import numpy as np
import pytest

import oracle
from paper_2206_11637_gb300 import objectives as O
from paper_2206_11637_gb300 import workloads as W


def J_forward(p, phi0, u0, p0, obs):
    o = oracle.from_params(p, phi0, u0, p0)
    J = 0.0
    for t, w in sorted(obs, key=lambda x: x[0]):
        o.step(t - o.time)
        J += float(np.dot(w, o.fields()[0].reshape(-1)))
    return J


def bubble():
    # walls on every face, gravity, hydrostatic start: every force term active
    p, phi0, u0, p0 = W.rising_bubble(10, 16, 10, D=6.0, xi=3.0, M=0.05)
    n = 30
    return p, phi0, u0, p0, n, O.rise_velocity_weights(p, phi0, 10, n)


def wave():
    # periodic x, walls in y, observations at two steps
    p, phi0, u0, p0 = W.capillary_wave(16, ny=16, a0=1.0, xi=3.0, M=0.03, sigma=1e-3, nu=0.05)
    n = 24
    w = O.wave_mode_weights(p, 16.0)
    return p, phi0, u0, p0, n, [(n, w), (n // 2, 0.5 * w)]


@pytest.mark.parametrize("qh", [15, 27, 9])
@pytest.mark.parametrize("case", [bubble, wave])
@pytest.mark.parametrize("param", ["mobility", "xi", "sigma"])
def test_tangent_matches_central_differences(case, param, qh):
    if qh == 9 and case is bubble:
        pytest.skip("D2Q9 is the 2-D lattice; the bubble is 3-D")
    p, phi0, u0, p0, n, obs = case()
    p.h_lattice = qh
    J, dJ = oracle.tangent(p, phi0, u0, p0, n, obs, param)
    assert abs(J - J_forward(p, phi0, u0, p0, obs)) <= 1e-12 * max(1.0, abs(J))
    v = getattr(p, param)
    d = 1e-4 * v
    pp, pm = copy.copy(p), copy.copy(p)
    setattr(pp, param, v + d)
    setattr(pm, param, v - d)
    fd = (J_forward(pp, phi0, u0, p0, obs) - J_forward(pm, phi0, u0, p0, obs)) / (2 * d)
    assert fd != 0.0
    assert abs(dJ - fd) <= 1e-5 * abs(fd), (dJ, fd)


def test_tangent_of_an_unobserved_start_is_zero():
    # J = W . phi(0) does not depend on the parameters
    p, phi0, u0, p0, n, obs = bubble()
    for param in ("mobility", "xi", "sigma"):
        _, dJ = oracle.tangent(p, phi0, u0, p0, n, [(0, obs[0][1])], param)
        assert dJ == 0.0


def random_tiny(qh):
    """A 5 x 6 x 4 lattice (5 x 6 in 2-D) with walls in y, gravity and uniform
    random phi, u and p*: every cell is an interface cell with steep
    gradients, so every branch of the update carries derivative."""
    rng = np.random.Generator(np.random.PCG64(4242))
    nz = 1 if qh == 9 else 4
    p = W.Params(5, 6, nz, (0, 0, 1, 1, 0, 0), 1.0, 0.1, 0.05, 0.1, 1e-3, 0.05, 3.0, (0.0, -1e-5, 0.0),
                 h_lattice=qh)
    phi0 = rng.uniform(0.05, 0.95, p.shape)
    u0 = rng.uniform(-1e-3, 1e-3, (3,) + p.shape)
    if nz == 1:
        u0[2] = 0.0
    p0 = rng.uniform(-1e-3, 1e-3, p.shape)
    n = 12
    return p, phi0, u0, p0, n, [(n, rng.standard_normal(p.cells)), (5, rng.standard_normal(p.cells))]


@pytest.mark.parametrize("qh", [15, 27, 9])
@pytest.mark.parametrize("param", ["mobility", "xi", "sigma"])
def test_tangent_on_random_fields(param, qh):
    """Against central differences at relative steps 1e-3 and 1e-4: the
    difference is within 1e-6 at 1e-4 (measured <= 4e-8), and where the
    truncation error dominates at 1e-3 it falls by the factor 100 of a
    second-order difference."""
    p, phi0, u0, p0, n, obs = random_tiny(qh)
    J, dJ = oracle.tangent(p, phi0, u0, p0, n, obs, param)
    assert abs(J - J_forward(p, phi0, u0, p0, obs)) <= 1e-12 * max(1.0, abs(J))
    v = getattr(p, param)
    err = []
    for rel in (1e-3, 1e-4):
        pp, pm = copy.copy(p), copy.copy(p)
        setattr(pp, param, v * (1 + rel))
        setattr(pm, param, v * (1 - rel))
        fd = (J_forward(pp, phi0, u0, p0, obs) - J_forward(pm, phi0, u0, p0, obs)) / (2 * rel * v)
        err.append(abs(dJ - fd) / abs(fd))
    assert err[1] <= 1e-6, err
    if err[0] > 1e-7:                 # truncation-dominated at the larger step
        assert 50 < err[0] / err[1] < 200, err
