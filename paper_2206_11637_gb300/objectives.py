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


# ---------------------------------------------------------------------------
# Capillary-wave frequency: a nonlinear objective through seed fields.
#
# The adjoint differentiates J = sum_o sum_x W_o(x) phi(x, t_o) for fixed weight
# fields.  A nonlinear J(phi(t_1), ..., phi(t_K)) is differentiated by taking
# the weights W_o = dJ / dphi(t_o), evaluated on a forward pass: the gradient
# of that linear functional at the forward solution is dJ / dtheta (chain
# rule).  The wave's angular frequency is such a J:
#   interface height  zeta_k = j + (phi_j - 1/2) / (phi_j - phi_{j+1}) of the
#                     column (x, z) at step t_k, j the first cell from the
#                     heavy side with phi_j >= 1/2 > phi_{j+1} (the amplitude
#                     the paper reads at phi = 1/2 at x = 0);
#   fit               zeta(t) ~ A exp(-gamma t) cos(omega t + psi) + c by least
#                     squares over the observations;
#   J = omega         with d omega / d zeta_k from the implicit function
#                     theorem at the optimum theta* of F = 1/2 sum r_k^2,
#                     r_k = f(t_k; theta) - zeta_k:  d theta / d zeta_k =
#                     H^-1 J_k, H = sum_k (J_k J_k^T + r_k d2f_k) the full
#                     Hessian of F and J_k = df(t_k) / dtheta.

def interface_crossing(col):
    """(j, zeta, dzeta/dphi_j, dzeta/dphi_{j+1}) of the first phi = 1/2
    crossing of a column going up from the heavy side."""
    col = np.asarray(col, dtype=np.float64)
    for j in range(len(col) - 1):
        if col[j] >= 0.5 > col[j + 1]:
            d = col[j] - col[j + 1]
            return j, j + (col[j] - 0.5) / d, (0.5 - col[j + 1]) / (d * d), (col[j] - 0.5) / (d * d)
    raise ValueError("the column has no phi = 1/2 crossing")


def _damped_cosine(t, th):
    A, g, w, ps, c = th
    E = np.exp(-g * t)
    C, S = np.cos(w * t + ps), np.sin(w * t + ps)
    f = A * E * C + c
    # first derivatives in the order (A, gamma, omega, psi, c)
    J = np.stack([E * C, -t * A * E * C, -t * A * E * S, -A * E * S, np.ones_like(t)], axis=1)
    # second derivatives, (K, 5, 5)
    H = np.zeros((len(t), 5, 5))
    H[:, 0, 1] = H[:, 1, 0] = -t * E * C
    H[:, 0, 2] = H[:, 2, 0] = -t * E * S
    H[:, 0, 3] = H[:, 3, 0] = -E * S
    H[:, 1, 1] = t * t * A * E * C
    H[:, 1, 2] = H[:, 2, 1] = t * t * A * E * S
    H[:, 1, 3] = H[:, 3, 1] = t * A * E * S
    H[:, 2, 2] = -t * t * A * E * C
    H[:, 2, 3] = H[:, 3, 2] = -t * A * E * C
    H[:, 3, 3] = -A * E * C
    return f, J, H


def fit_damped_cosine(t, zeta, omega_guess):
    """Least-squares theta = (A, gamma, omega, psi, c) of the damped cosine
    through (t, zeta), by Gauss-Newton from a guess built on omega_guess;
    returns (theta, d omega / d zeta) with the latter from the full Hessian."""
    t = np.asarray(t, dtype=np.float64)
    zeta = np.asarray(zeta, dtype=np.float64)
    c0 = float(np.mean(zeta))
    # linear least squares for the amplitude and phase at the guessed frequency
    B = np.stack([np.cos(omega_guess * t), -np.sin(omega_guess * t), np.ones_like(t)], axis=1)
    a, b, c0 = np.linalg.lstsq(B, zeta, rcond=None)[0]
    th = np.array([np.hypot(a, b), 0.0, omega_guess, np.arctan2(b, a), c0])
    for _ in range(200):
        f, J, _ = _damped_cosine(t, th)
        r = f - zeta
        step = np.linalg.lstsq(J, -r, rcond=None)[0]
        th = th + step
        if np.all(np.abs(step) <= 1e-15 * np.maximum(np.abs(th), 1e-300) + 1e-300):
            break
    f, J, Hf = _damped_cosine(t, th)
    r = f - zeta
    H = J.T @ J + np.einsum("k,kij->ij", r, Hf)
    dth = np.linalg.solve(H, J.T)          # (5, K): d theta / d zeta_k
    return th, dth[2]


class WaveFrequency:
    """J = omega of the damped cosine fitted to the interface height of the
    column (x, z) at the observation steps.  Use: record(step, phi) for every
    observation step of a forward run, then value() and seeds(shape)."""

    def __init__(self, steps, omega_guess, x=0, z=0):
        self.steps = [int(s) for s in steps]
        self.omega_guess = float(omega_guess)
        self.x, self.z = int(x), int(z)
        self.cross = {}

    def record(self, step, phi):
        """phi: (nz, ny, nx) field at `step`."""
        self.cross[int(step)] = interface_crossing(np.asarray(phi)[self.z, :, self.x])

    def _fit(self):
        t = np.array(self.steps, dtype=np.float64)
        zeta = np.array([self.cross[s][1] for s in self.steps])
        return fit_damped_cosine(t, zeta, self.omega_guess)

    def value(self):
        return float(self._fit()[0][2])

    def seeds(self, shape):
        """[(step, W)] with W = d omega / d phi(step) (two cells per step)."""
        nz, ny, nx = shape
        _, dw = self._fit()
        out = []
        for k, s in enumerate(self.steps):
            j, _, dj, dj1 = self.cross[s]
            W = np.zeros(shape)
            W[self.z, j, self.x] = dw[k] * dj
            W[self.z, j + 1, self.x] = dw[k] * dj1
            out.append((s, W.reshape(-1)))
        return out
