"""Closed-form solutions the paper uses to validate the PFLBM (test helpers).

prosperetti  -- small-amplitude viscous capillary wave, section "Capillary
                wave", analytical model (Prosperetti 1981): amplitude a(t) from
                the four roots of the quartic and complementary error functions.
gravity_omega0, gravity_damping -- standing gravity wave, section "Gravity
                wave": omega0^2 = g k tanh(k d), decay a0 exp(-2 nu k^2 t).
poiseuille   -- body-force driven channel with halfway walls.
two_layer_poiseuille -- two immiscible layers with different density and
                dynamic viscosity; continuity of velocity and shear stress.
"""
import numpy as np
from scipy.special import erfc, wofz


def capillary_omega0(sigma, k, rho_h, rho_l):
    return np.sqrt(sigma * k ** 3 / (rho_h + rho_l))


def gravity_omega0(g, k, d):
    """Linear standing gravity wave over depth d (section "Gravity wave")."""
    return np.sqrt(g * k * np.tanh(k * d))


def gravity_damping(nu, k):
    """Viscous amplitude decay rate of a gravity wave, a0 exp(-2 nu k^2 t)."""
    return 2.0 * nu * k * k


def prosperetti(t, k, nu, rho_h, rho_l, sigma, a0):
    t = np.asarray(t, dtype=np.float64)
    w02 = sigma * k ** 3 / (rho_h + rho_l)
    beta = rho_l * rho_h / (rho_l + rho_h) ** 2
    nk2 = nu * k * k
    coeffs = [1.0, -4.0 * beta * np.sqrt(nk2), 2.0 * (1.0 - 6.0 * beta) * nk2,
              4.0 * (1.0 - 3.0 * beta) * nk2 ** 1.5, (1.0 - 4.0 * beta) * nk2 ** 2 + w02]
    z = np.roots(coeffs).astype(np.complex128)
    first = 4.0 * (1.0 - 4.0 * beta) * nk2 ** 2 / (8.0 * (1.0 - 4.0 * beta) * nk2 ** 2 + w02) * a0 * erfc(np.sqrt(nk2 * t))
    total = np.zeros_like(t, dtype=np.complex128)
    st = np.sqrt(t)
    for i in range(4):
        Zi = np.prod([z[j] - z[i] for j in range(4) if j != i])
        # exp(z^2 t) erfc(z sqrt t) = w(i z sqrt t)  (Faddeeva function)
        total += z[i] / Zi * (w02 * a0 / (z[i] ** 2 - nk2)) * np.exp(-nk2 * t) * wofz(1j * z[i] * st)
    return first + total.real


def poiseuille(y, H, g, nu):
    """u(y) for cells y = 0..H-1 between halfway walls at -1/2 and H - 1/2."""
    yy = np.asarray(y, dtype=np.float64) + 0.5
    return g / (2.0 * nu) * yy * (H - yy)


def two_layer_poiseuille(y, H, h1, g, rho1, mu1, rho2, mu2):
    """Layer 1 (rho1, mu1) occupies 0 < s < h1, layer 2 above, walls at s = 0, H.

    s = y + 1/2.  mu_k u'' = -rho_k g; u(0) = u(H) = 0; u and mu u' continuous.
    """
    s = np.asarray(y, dtype=np.float64) + 0.5
    # u1 = -rho1 g s^2 / (2 mu1) + A1 s ; u2 = -rho2 g (s - H)^2 / (2 mu2) + A2 (s - H)
    # continuity at s = h1 of u and mu u' -> 2x2 system in A1, A2
    d = h1 - H
    a11, a12 = h1, -d
    b1 = rho1 * g * h1 ** 2 / (2 * mu1) - rho2 * g * d ** 2 / (2 * mu2)
    a21, a22 = mu1, -mu2
    b2 = rho1 * g * h1 - rho2 * g * d
    det = a11 * a22 - a12 * a21
    A1 = (b1 * a22 - a12 * b2) / det
    A2 = (a11 * b2 - a21 * b1) / det
    u1 = -rho1 * g * s ** 2 / (2 * mu1) + A1 * s
    u2 = -rho2 * g * (s - H) ** 2 / (2 * mu2) + A2 * (s - H)
    return np.where(s < h1, u1, u2)


def interface_height(phi_column):
    """First phi = 0.5 crossing along y, going up from the heavy side (linear)."""
    c = np.asarray(phi_column)
    for j in range(len(c) - 1):
        if c[j] >= 0.5 > c[j + 1]:
            return j + (c[j] - 0.5) / (c[j] - c[j + 1])
    return np.nan
