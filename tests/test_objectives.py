"""Host side of the nonlinear adjoint objective (no GPU): the interface
crossing of a column and its derivative, the damped-cosine fit and the
implicit-function derivative of its frequency, against central differences."""
import numpy as np

from paper_2206_11637_gb300 import objectives as O


def test_interface_crossing_and_its_derivative():
    col = np.array([1.0, 0.99, 0.8, 0.3, 0.05, 0.0])
    j, z, dj, dj1 = O.interface_crossing(col)
    assert j == 2 and abs(z - (2 + 0.3 / 0.5)) < 1e-15
    for idx, d in ((j, dj), (j + 1, dj1)):
        e = 1e-7
        cp, cm = col.copy(), col.copy()
        cp[idx] += e
        cm[idx] -= e
        fd = (O.interface_crossing(cp)[1] - O.interface_crossing(cm)[1]) / (2 * e)
        assert abs(fd - d) < 1e-7 * abs(d)


def test_fit_recovers_a_damped_cosine_exactly():
    t = np.arange(0.0, 4000.0, 50.0)
    th0 = np.array([0.8, 1.5e-4, 2.2e-3, -0.7, 15.5])
    z, _, _ = O._damped_cosine(t, th0)
    th, _ = O.fit_damped_cosine(t, z, 2.0e-3)
    assert np.allclose(th, th0, rtol=1e-9, atol=1e-12)


def test_frequency_derivative_matches_central_differences():
    t = np.arange(0.0, 3000.0, 40.0)
    th0 = np.array([1.0, 2e-4, 2.7e-3, 0.3, 15.5])
    z, _, _ = O._damped_cosine(t, th0)
    z = z + 0.01 * np.random.default_rng(1).standard_normal(len(t))   # residuals: the Hessian term matters
    _, dw = O.fit_damped_cosine(t, z, 2.5e-3)
    for k in (0, 3, 20, 50, len(t) - 1):
        e = 1e-6
        zp, zm = z.copy(), z.copy()
        zp[k] += e
        zm[k] -= e
        fd = (O.fit_damped_cosine(t, zp, 2.5e-3)[0][2] - O.fit_damped_cosine(t, zm, 2.5e-3)[0][2]) / (2 * e)
        assert abs(fd - dw[k]) <= 1e-6 * np.abs(dw).max()


def test_wave_frequency_seeds_are_two_cells_per_step():
    nz, ny, nx = 1, 16, 8
    steps = list(range(0, 2000, 50))
    obj = O.WaveFrequency(steps, 3e-3)
    yy = np.arange(ny, dtype=np.float64)
    for s in steps:
        zeta = 7.5 + 0.8 * np.exp(-1e-4 * s) * np.cos(3e-3 * s)
        phi = np.broadcast_to((0.5 - 0.5 * np.tanh((yy - zeta) / 2.0))[None, :, None], (nz, ny, nx)).copy()
        obj.record(s, phi)
    assert abs(obj.value() - 3e-3) < 1e-4
    seeds = obj.seeds((nz, ny, nx))
    assert [s for s, _ in seeds] == steps
    for _, W in seeds:
        assert np.count_nonzero(W) <= 2 and W.shape == (nz * ny * nx,)
