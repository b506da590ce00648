"""Linear objectives J = sum_x W(x) phi(x, t) for the adjoint (weight fields).

Bubble rise velocity: the centroid of the light phase, y_c = sum (1 - phi) y /
sum (1 - phi).  The denominator V = sum (1 - phi) is conserved by the
conservative Allen-Cahn model, so y_c = (sum y - sum phi y) / V is linear in
phi, and the mean rise velocity between steps t_a < t_b is
  (y_c(t_b) - y_c(t_a)) / (t_b - t_a) = sum W_b phi(t_b) + sum W_a phi(t_a) + const,
  W_b = -y / (V (t_b - t_a)),  W_a = +y / (V (t_b - t_a)).

Wave mode amplitude: for a heavy layer below an interface y = d + a(x, t),
sum_y phi(x, y) = d + a(x) + const per column, so
  A(t) = (2 / nx) sum_x cos(k x) sum_y phi(x, y, t)
is the amplitude of the cos(k x) mode of the interface height.
"""
import numpy as np


def rise_velocity_weights(p, phi0, t_a, t_b):
    """[(t_a, W_a), (t_b, W_b)] for the mean rise velocity along +y."""
    z, y, x = np.meshgrid(np.arange(p.nz, dtype=np.float64), np.arange(p.ny, dtype=np.float64),
                          np.arange(p.nx, dtype=np.float64), indexing="ij")
    V = float(np.sum(1.0 - phi0))
    w = y.reshape(-1) / (V * (t_b - t_a))
    return [(t_a, w.copy()), (t_b, -w)]


def rise_velocity_constant(p, phi0, t_a, t_b):
    """The phi-independent part of the rise velocity (zero: sum y cancels)."""
    return 0.0


def wave_mode_weights(p, wavelength):
    """W(x, y, z) = (2 / nx) cos(2 pi x / wavelength) / nz."""
    z, y, x = np.meshgrid(np.arange(p.nz, dtype=np.float64), np.arange(p.ny, dtype=np.float64),
                          np.arange(p.nx, dtype=np.float64), indexing="ij")
    return (2.0 / p.nx * np.cos(2.0 * np.pi * x / wavelength) / p.nz).reshape(-1)
