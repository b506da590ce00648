"""Solid cells (pfl_set_solid) on the GPU against the oracle, and the Taylor
bubble (section "Taylor bubble") against the paper.

- FP64 within 1e-10 of the oracle on fluid cells: a drop falling onto a solid
  block, a small Taylor bubble in a voxel tube, and a 2-D channel (D2Q9) past
  a solid post; FP32 within 1e-5 and shifted FP16 within 1e-3 on phi.
- A channel walled by solid rows equals the channel between no-slip faces
  bitwise on the GPU as well (single phase).
- pfl_set_solid refuses a context created without solids, a call after the
  first step, and the adjoint refuses a solid lattice.
- Taylor bubble, D = 64, FP32: the Reynolds number from the bubble's rise
  between t* = 10 and 15 (t* = t sqrt(g / D), as in the paper), against the
  paper's PFLBM 26.83 (experiment 27) within 5 %.
"""
import math

import numpy as np
import pytest

import golden
import oracle
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = 0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


def sim(p, phi0, u0=None, p0=None, precision="fp64"):
    from paper_2206_11637_gb300.pflbm import Simulation
    return Simulation(p, phi0, u0, p0, precision=precision)


def rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def drop_on_block():
    p = W.Params(32, 32, 24, (0, 0, 1, 1, 0, 0), 1.0, 0.01, 0.02, 0.05, 2e-4, 0.03, 4.0, (0.0, -2e-6, 0.0))
    x, y, z = W.coords(p)
    p.solid = ((np.abs(x - 15.5) < 6) & (y < 8) & (np.abs(z - 11.5) < 5)).astype(np.uint8)
    phi0 = W.sphere(p, (15.5, 18.0, 11.5), 6.0, heavy_inside=True)
    u0 = np.zeros((3,) + p.shape)
    u0[1] = -0.01 * phi0
    return p, phi0, u0, None


def small_taylor():
    # the paper's fluids are unstable in a D = 16 tube (as it reports for
    # small D); a milder pair (density and viscosity ratio 100, Bo = 20,
    # Mo = 1) keeps the same geometry
    return W.taylor_bubble(16, Bo=20.0, Mo=1.0, rho_ratio=100.0, mu_ratio=100.0)


def channel_post_2d():
    p = W.Params(64, 34, 1, (0,) * 6, 1.0, 0.01, 0.05, 0.05, 2e-4, 0.03, 4.0, (1e-6, 0.0, 0.0), h_lattice=9)
    x, y, z = W.coords(p)
    p.solid = ((y < 1) | (y > 32) | ((x - 20.0) ** 2 + (y - 16.5) ** 2 < 16)).astype(np.uint8)
    phi0 = W.cylinder_z(p, (44.0, 16.5), 7.0, heavy_inside=True)
    return p, phi0, None, None


# the small Taylor bubble amplifies rounding about tenfold per 30 steps (the
# oracle against itself with phi0 perturbed by 1e-16 shows the same): 150 steps
CASES = {"drop_on_block": (drop_on_block, 300), "small_taylor": (small_taylor, 150),
         "channel_post_d2q9": (channel_post_2d, 400)}


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_parity_with_solids(name):
    build, steps = CASES[name]
    p, phi0, u0, p0 = build()
    s = sim(p, phi0, u0, p0, "fp64")
    o = oracle.from_params(p, phi0, u0, p0)
    s.step(steps)
    o.step(steps, THREADS)
    fluid = p.solid == 0
    for a, b in zip(s.fields(), o.fields()):
        a, b = np.asarray(a), np.asarray(b)
        if a.ndim == 4:
            a, b = a[:, fluid], b[:, fluid]
        else:
            assert np.all(a[~fluid] == 0) and np.all(b[~fluid] == 0)
            a, b = a[fluid], b[fluid]
        assert rel(a, b) <= 1e-10


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16s", 1e-3)])
def test_reduced_precision_with_solids(precision, tol):
    p, phi0, u0, p0 = drop_on_block()
    s = sim(p, phi0, u0, p0, precision)
    o = oracle.from_params(p, phi0, u0, p0)
    s.step(300)
    o.step(300, THREADS)
    fluid = p.solid == 0
    assert rel(s.fields()[0][fluid], o.fields()[0][fluid]) <= tol


def test_solid_rows_equal_no_slip_faces_gpu():
    H, g, nu = 16, 1e-6, 1 / 8
    p, phi0, _, _ = W.poiseuille(H, nx=4, g=g, nu=nu)
    a = sim(p, phi0)
    a.step(500)
    q = W.Params(4, H + 2, 1, (0,) * 6, 1.0, 1e-3, nu, nu, 1e-4, 0.02, 5.0, (g, 0.0, 0.0))
    mask = np.zeros(q.shape, np.uint8)
    mask[:, 0, :] = mask[:, -1, :] = 1
    q.solid = mask
    b = sim(q, np.ones(q.shape))
    b.step(500)
    assert np.array_equal(b.fields()[3][:, :, 1:-1, :], a.fields()[3])


def test_solid_calls_refused():
    from paper_2206_11637_gb300 import _lib as L
    from paper_2206_11637_gb300 import objectives as O
    p, phi0, u0, p0 = drop_on_block()
    mask = p.solid
    p.solid = None
    s = sim(p, phi0, u0, p0)
    m = np.ascontiguousarray(mask.reshape(-1), dtype=np.uint8)
    assert s.lib.pfl_set_solid(s.ctx, m.ctypes.data) == L.PFL_ERR_STATE       # created without solids
    p.solid = mask
    s = sim(p, phi0, u0, p0)
    s.step(1)
    assert s.lib.pfl_set_solid(s.ctx, m.ctypes.data) == L.PFL_ERR_STATE       # after the first step
    with pytest.raises(L.PFLError):
        s.adjoint(4, [(4, np.ones(p.cells) / p.cells)])


def test_taylor_bubble_reynolds_number():
    """Paper's fluids and D = 64 with xi = 3.5: its xi = 3 blows up within the
    first time unit in this model (oracle and GPU alike), 3.5 is the nearest
    stable width.  The centroid rises steadily from t* = 6 on."""
    D = 64
    p, phi0, u0, p0 = W.taylor_bubble(D, xi=3.5)
    s = sim(p, phi0, u0, p0, "fp32")
    t_unit = 1.0 / math.sqrt(abs(p.gravity[1]) / D)
    ys = []
    for ts in (10.0, 15.0):
        s.step(int(round(ts * t_unit)) - s.time)
        ys.append(W.gas_centroid_y(s.phi(), p.solid))
    _, nf = s.diag(check=False)
    assert nf == 0
    U = (ys[1] - ys[0]) / (5.0 * t_unit)
    Re = U * D / p.nu_h
    paper, _ = golden.taylor_bubble_re()
    assert abs(Re / paper[D] - 1) < 0.05, Re
