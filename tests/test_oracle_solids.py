"""Solid cells in the oracle (voxelised walls: links into a solid cell bounce
back half-way, stencil reads of a solid neighbour return the reading cell's
phi, solid cells are not updated).

- A channel whose walls are rows of solid cells in a periodic box equals the
  channel between no-slip faces exactly (single phase: the same links bounce).
- Hagen-Poiseuille flow in a tube voxelised on the lattice: the flow rate and
  the centre-line speed within the staircase error of the voxel tube (its
  cross-section is 3.45 % larger than the circle at D = 8 and 16).
- A two-phase drop falling onto a solid block conserves phi to 1e-12 and
  leaves the solid cells' populations zero.
"""
import math

import numpy as np

import oracle
from paper_2206_11637_gb300 import workloads as W


def test_solid_rows_equal_no_slip_faces():
    H, g, nu = 16, 1e-6, 1 / 8
    p, phi0, _, _ = W.poiseuille(H, nx=4, g=g, nu=nu)
    a = oracle.from_params(p, phi0)
    a.step(2000, 0)
    q = W.Params(4, H + 2, 1, (0,) * 6, 1.0, 1e-3, nu, nu, 1e-4, 0.02, 5.0, (g, 0.0, 0.0))
    mask = np.zeros(q.shape, np.uint8)
    mask[:, 0, :] = mask[:, -1, :] = 1
    q.solid = mask
    b = oracle.from_params(q, np.ones(q.shape))
    b.step(2000, 0)
    ua, ub = a.fields()[3], b.fields()[3]
    assert np.array_equal(ub[:, :, 1:-1, :], ua)
    assert np.all(ub[:, :, 0, :] == 0) and np.all(ub[:, :, -1, :] == 0)


def test_hagen_poiseuille_in_a_voxel_tube():
    for D in (8, 16):
        p, phi0, _, _ = W.hagen_poiseuille(D)
        o = oracle.from_params(p, phi0)
        o.step(int(9 * D * D / p.nu_h), 0)
        u = o.fields()[3][1]
        fluid = p.solid == 0
        Q = u[fluid].sum() / p.ny
        Qa = math.pi * p.gravity[1] * (D / 2) ** 4 / (8 * p.nu_h)
        ua = p.gravity[1] * (D / 2) ** 2 / (4 * p.nu_h)
        assert abs(Q / Qa - 1) < 0.06, (D, Q / Qa)
        assert abs(u.max() / ua - 1) < 0.03, (D, u.max() / ua)
        assert np.all(u[~fluid] == 0)


def drop_on_block():
    p = W.Params(32, 32, 24, (0, 0, 1, 1, 0, 0), 1.0, 0.01, 0.02, 0.05, 2e-4, 0.03, 4.0, (0.0, -2e-6, 0.0))
    x, y, z = W.coords(p)
    p.solid = ((np.abs(x - 15.5) < 6) & (y < 8) & (np.abs(z - 11.5) < 5)).astype(np.uint8)
    phi0 = W.sphere(p, (15.5, 18.0, 11.5), 6.0, heavy_inside=True)
    u0 = np.zeros((3,) + p.shape)
    u0[1] = -0.01 * phi0
    return p, phi0, u0, None


def test_drop_on_a_solid_block_conserves_phi():
    p, phi0, u0, _ = drop_on_block()
    o = oracle.from_params(p, phi0, u0)
    m0 = o.fields()[0].sum()
    o.step(300, 0)
    phi = o.fields()[0]
    assert abs(phi.sum() - m0) / m0 < 1e-12
    h, g = o.populations()
    solid = p.solid != 0
    assert np.all(h[:, solid] == 0) and np.all(g[:, solid] == 0)
    assert np.all(phi[solid] == 0)


def test_taylor_bubble_setup():
    """The Taylor bubble's tube is closed (every cell on the x and z faces is
    solid), the gas cylinder has the stated volume, and the hydrostatic start
    puts zero pressure at the bubble's top."""
    D = 32
    p, phi0, _, p0 = W.taylor_bubble(D)
    s = p.solid.astype(bool)
    assert p.shape == (D + 2, 10 * D, D + 2)
    assert s[0].all() and s[-1].all() and s[:, :, 0].all() and s[:, :, -1].all()
    gas = (1.0 - phi0)[~s].sum()
    vol = math.pi * (0.375 * D) ** 2 * 3 * D
    assert abs(gas / vol - 1) < 0.03, gas / vol
    rho = p.rho_l + phi0 * (p.rho_h - p.rho_l)
    pres = p0 * rho / 3.0
    g = abs(p.gravity[1])
    c = (D + 1) // 2
    col = pres[c, :, c]              # the tube's axis, through the gas
    assert abs(col[4 * D]) < 2 * g and abs(col[4 * D - 1]) < 2 * g
    # liquid above the bubble: p = -rho_h g (y - y_top)
    y = np.arange(5 * D, 6 * D)
    assert np.allclose(col[y], -g * (y - (4 * D - 0.5)), rtol=0, atol=2 * g)
