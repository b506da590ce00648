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
