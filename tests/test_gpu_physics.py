"""Physics checks of the GPU path against what the paper fixes.

- Laplace: static 3D drop, p_in - p_out = 2 sigma / R.  The FP64 jump falls
  short of 2 sigma / R by a deficit that does not depend on R and shrinks as
  (1 / xi)^2 -- the second-order error of the stencil across a diffuse
  interface resolved by xi cells -- so the test checks the second-order decay
  between xi = 4 and xi = 8 and a deficit below 1.5 % at xi = 8 (R = 26); FP32
  and shifted-FP16 storage within 1 % of the FP64 jump at xi = 5, R = 16.
- Capillary wave (200 x 400 x 1, sigma 1e-4, nu 0.01, xi 5, M 0.02): the
  oscillation frequency from zero crossings of the interface height at x = 0
  (section "Capillary wave"), FP32 and FP16S within 1 % of FP64; FP64 against
  Prosperetti's model.
- Gravity wave (section "Gravity wave": L x L x 1, Re 10, omega_H 1.99, rho
  ratio 1000, xi 5, M 0.02, hydrostatic start): the fitted angular frequency
  approaches omega0 = sqrt(g k tanh(k d)) from below as L grows (0.96 at L 50,
  0.98 at L 100) and is within 3 % at L 100; FP32 and FP16S within 1 % of
  FP64; the fitted amplitude decay stays below Lamb's 2 nu k^2 (the paper
  finds the PFLBM underestimates this damping).
- Convergence at the paper's wave parameters (L x L, Re 10, omega_H 1.99,
  xi 5, M 0.02): the period error against Prosperetti shrinks as L grows.
"""
import math

import numpy as np
import pytest

import analytic as A
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


def radius_from_volume(V, xi):
    """R of a tanh-profile sphere holding V: V = 4 pi (R^3 / 3 + R pi^2 xi^2 / 48)."""
    R = (3 * V / (4 * math.pi)) ** (1 / 3)
    for _ in range(50):
        f = R ** 3 / 3 + R * math.pi ** 2 * xi ** 2 / 48 - V / (4 * math.pi)
        R -= f / (R * R + math.pi ** 2 * xi ** 2 / 48)
    return R


def laplace_jump(precision, n=64, R=16.0, steps=3000, xi=5.0):
    p, phi0, _, _ = W.static_drop(n, R, xi=xi, nu=1.0 / 6.0)
    s = sim(p, phi0, precision=precision)
    s.step(steps)
    phi, _, pr, _ = s.fields()
    c = n // 2
    p_in = pr[c - 2:c + 2, c - 2:c + 2, c - 2:c + 2].mean()
    p_out = pr[0:3, 0:3, 0:3].mean()
    return p_in - p_out, radius_from_volume(phi.sum(), p.xi), p


def test_radius_from_volume_inverts_the_profile():
    for R in (10.0, 16.0, 24.0):
        p, phi0, _, _ = W.static_drop(int(4 * R), R)
        assert abs(radius_from_volume(phi0.sum(), p.xi) / R - 1) < 2e-3


def test_laplace_3d_drop_converges_in_xi():
    # steps scale with xi^2: the interface relaxes diffusively over xi
    dp4, R4, p4 = laplace_jump("fp64", n=64, R=16.0, steps=3840, xi=4.0)
    dp8, R8, p8 = laplace_jump("fp64", n=104, R=26.0, steps=15360, xi=8.0)
    d4 = 1 - dp4 / (2 * p4.sigma / R4)
    d8 = 1 - dp8 / (2 * p8.sigma / R8)
    assert 0 < d8 < 0.015, (d4, d8)
    assert 2.5 < d4 / d8 < 8.0, (d4, d8)    # second order: 4


def test_laplace_3d_drop_by_precision():
    dp64, R64, p = laplace_jump("fp64")
    assert abs(dp64 / (2 * p.sigma / R64) - 1) < 0.04, (dp64, R64)
    for prec in ("fp32", "fp16s"):
        dp, _, _ = laplace_jump(prec)
        assert abs(dp / dp64 - 1) < 0.01, (prec, dp, dp64)


def crossings(ts, a):
    return np.array([ts[i] + a[i] / (a[i] - a[i + 1]) * (ts[i + 1] - ts[i])
                     for i in range(len(a) - 1) if (a[i] > 0) != (a[i + 1] > 0)])


def wave_history(p, phi0, precision, t_end, nsamp=160):
    s = sim(p, phi0, precision=precision)
    dt = max(1, int(t_end / nsamp))
    ts, amp = [], []
    depth = (p.ny - 1) / 2.0
    while s.time <= t_end:
        ts.append(s.time)
        amp.append(A.interface_height(s.phi()[0, :, 0]) - depth)
        s.step(dt)
    return np.array(ts, float), np.array(amp)


def fitted_period(ts, amp, T):
    """Period of a0 exp(-g t) cos(w t + phase) + offset fitted after t = T / 10."""
    from scipy.optimize import curve_fit
    f = lambda t, a, g, w, ph, c: a * np.exp(-g * t) * np.cos(w * t + ph) + c
    m = ts > 0.1 * T
    popt, _ = curve_fit(f, ts[m], amp[m], p0=[amp[0], 1e-6, 2 * math.pi / T, 0.0, 0.0], maxfev=20000)
    return 2 * math.pi / popt[2]


def test_capillary_wave_frequency_by_precision():
    p, phi0, _, _ = W.capillary_wave(200)            # 200 x 400 x 1
    k = 2 * math.pi / 200
    T = 2 * math.pi / A.capillary_omega0(p.sigma, k, p.rho_h, p.rho_l)
    periods = {}
    for prec in ("fp64", "fp32", "fp16s"):
        ts, amp = wave_history(p, phi0, prec, 2.2 * T)
        periods[prec] = fitted_period(ts, amp, T)
    for prec in ("fp32", "fp16s"):
        assert abs(periods[prec] / periods["fp64"] - 1) < 0.01, periods
    # FP64 against the model: the diffuse interface lengthens the period (see the convergence test)
    assert 1.0 < periods["fp64"] / T < 1.2, (periods, T)


def paper_wave(L):
    nu = (1.0 / 1.99 - 0.5) / 3.0
    a0 = 0.01 * L
    w0 = 10.0 * nu / (a0 * L)                        # Re = a0 w0 L / nu = 10
    k = 2 * math.pi / L
    sigma = w0 ** 2 * (1.0 + 1e-3) / k ** 3
    p, phi0, _, _ = W.capillary_wave(L, ny=L, a0=a0, xi=5.0, M=0.02, sigma=sigma, nu=nu)
    return p, phi0, w0, k, nu, a0


def test_capillary_wave_converges_with_resolution():
    errs = []
    for L in (50, 100):
        p, phi0, w0, k, nu, a0 = paper_wave(L)
        T = 2 * math.pi / w0
        ts, amp = wave_history(p, phi0, "fp64", 1.3 * T, nsamp=130)
        an = A.prosperetti(ts, k, nu, p.rho_h, p.rho_l, p.sigma, a0)
        c_sim, c_an = crossings(ts, amp), crossings(ts, an)
        assert len(c_sim) >= 2 and len(c_an) >= 2
        errs.append(abs((c_sim[1] - c_sim[0]) / (c_an[1] - c_an[0]) - 1))
    assert errs[1] < errs[0], errs
    assert errs[1] < 0.05, errs


def damped_fit(ts, amp, T, w0, g0):
    """(omega, decay rate) of a0 exp(-g t) cos(w t + phase) + offset fitted after t = T / 10."""
    from scipy.optimize import curve_fit
    f = lambda t, a, g, w, ph, c: a * np.exp(-g * t) * np.cos(w * t + ph) + c
    m = ts > 0.1 * T
    popt, _ = curve_fit(f, ts[m], amp[m], p0=[amp[0], g0, w0, 0.0, 0.0], maxfev=20000)
    return popt[2], popt[1]


def gravity_wave_fit(L, precision, periods=2.2, nsamp=180):
    p, phi0, u0, p0 = W.gravity_wave(L)
    k, d = 2 * math.pi / L, 0.5 * L
    w0 = A.gravity_omega0(abs(p.gravity[1]), k, d)
    g0 = A.gravity_damping(p.nu_h, k)
    T = 2 * math.pi / w0
    s = sim(p, phi0, u0, p0, precision=precision)
    dt = max(1, int(periods * T / nsamp))
    ts, amp = [], []
    while s.time <= periods * T:
        ts.append(s.time)
        amp.append(A.interface_height(s.phi()[0, :, 0]) - (L - 1) / 2.0)
        s.step(dt)
    w, g = damped_fit(np.array(ts, float), np.array(amp), T, w0, g0)
    return w / w0, g / g0


def test_gravity_wave_dispersion():
    w50, _ = gravity_wave_fit(50, "fp64")
    w100, g100 = gravity_wave_fit(100, "fp64")
    assert abs(w100 - 1) < 0.03, (w50, w100)
    assert abs(w100 - 1) < abs(w50 - 1), (w50, w100)
    assert 0.5 < g100 < 1.0, g100
    for prec in ("fp32", "fp16s"):
        w, _ = gravity_wave_fit(100, prec)
        assert abs(w / w100 - 1) < 0.01, (prec, w, w100)
