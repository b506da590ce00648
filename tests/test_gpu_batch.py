"""Batched form: many independent lattices in persistent launches.

Each instance of a batch evolves exactly like the same lattice run alone
(same per-cell code, FP64: bitwise), through both the graph replay and the
direct-launch remainder; tuned and untuned launch shapes agree, and so does
every tile shape a class offers (16- and 32-wide, FP32 bitwise against single
runs); FP32 instances stay within the FP32 tolerance of the oracle; an
instance that goes unstable is stopped while the others continue.
"""
import numpy as np
import pytest

import oracle
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


def mixed(count=6, seed=3):
    """Seeded sweep instances (M raised into the stable range), a walled
    bubble with gravity and a large cube that fills the large size class."""
    inst = W.batched_sweep(count, seed=seed, small=True)
    for p, _, _, _ in inst:
        p.mobility = max(p.mobility, 0.03)
    inst.append(W.rising_bubble(20, 36, 20, D=10.0, xi=4.0, M=0.05))
    inst.append(W.static_drop(44, 11.0, u_noise=1e-3, seed=9))
    return inst


@pytest.mark.parametrize("tune", [False, True])
def test_batch_equals_single_runs(tune):
    from paper_2206_11637_gb300.batch import Batch
    from paper_2206_11637_gb300.pflbm import Simulation
    inst = mixed()
    b = Batch(inst, precision="fp64", tune=tune)
    t, g, n = b.shapes()
    assert n[0] > 0 and n[1] > 0 and all(x in (128, 256) for x in t)
    steps = 37                       # two graph replays and five direct steps
    b.step(steps)
    assert b.time == steps
    for i, (p, phi0, u0, p0) in enumerate(inst):
        s = Simulation(p, phi0, u0, p0, precision="fp64")
        s.step(steps)
        a = b.fields(i)
        r = s.fields()
        for x, y in zip(a, r):
            assert np.array_equal(x, y), i


# every tile shape of each class (FP32 adds the 16-wide ones); one pair of
# shapes per batch, the same steps through graph replays and direct launches
SHAPE_PAIRS = [((32, 4), (32, 8)), ((32, 8), (16, 8)), ((16, 8), (16, 16))]


@pytest.mark.parametrize("shapes", SHAPE_PAIRS, ids=["%dx%d-%dx%d" % (a + b) for a, b in SHAPE_PAIRS])
def test_batch_tile_shapes_equal_single_runs_fp32(shapes):
    from paper_2206_11637_gb300.batch import Batch
    from paper_2206_11637_gb300.pflbm import Simulation
    inst = mixed()
    b = Batch(inst, precision="fp32", tune=False)
    (tx0, ty0), (tx1, ty1) = shapes
    b.set_shape(0, tx0, ty0)
    b.set_shape(1, tx1, ty1, z_chunk=7)    # a ragged last chunk on the 20- and 44-deep lattices
    t, g, n = b.shapes()
    assert list(t) == [tx0 * ty0, tx1 * ty1] and n[0] > 0 and n[1] > 0
    steps = 37
    b.step(steps)
    for i, (p, phi0, u0, p0) in enumerate(inst):
        s = Simulation(p, phi0, u0, p0, precision="fp32")
        s.step(steps)
        for x, y in zip(b.fields(i), s.fields()):
            assert np.array_equal(x, y), (shapes, i)


def test_batch_set_shape_refusals():
    from paper_2206_11637_gb300 import _lib as L
    from paper_2206_11637_gb300.batch import Batch
    inst = mixed(count=2)
    b = Batch(inst, precision="fp64", tune=False)
    for args in [(0, 16, 8), (1, 16, 16), (2, 32, 8), (1, 32, 4), (0, 32, 16), (1, 32, 8, -1)]:
        with pytest.raises(L.PFLError):
            b.set_shape(*args)
    b.set_shape(1, 16, 8, 5, 100)          # FP64 has the 16 x 8 tile in 3-D
    t, g, n = b.shapes()
    assert t[1] == 128 and g[1] == min(100, n[1])


def test_batch_fp32_against_oracle():
    from paper_2206_11637_gb300.batch import Batch
    inst = [W.static_drop(16, 5.0, u_noise=1e-3, seed=1), W.capillary_wave(32, ny=40, a0=1.0, xi=4.0, sigma=1e-3),
            W.static_drop(20, 6.0, xi=4.0, sigma=3e-4, mobility=0.05),
            W.rising_bubble(16, 28, 16, D=8.0, xi=4.0, M=0.05, hydrostatic=False)]
    b = Batch(inst, precision="fp32")
    b.step(200)
    for i, (p, phi0, u0, p0) in enumerate(inst[:3]):
        o = oracle.from_params(p, phi0, u0, p0)
        o.step(200, 0)
        phi = b.fields(i)[0]
        ophi = o.fields()[0]
        assert np.abs(phi - ophi).max() < 1e-5, i
    # The bubble starts out of hydrostatic balance and amplifies rounding: the
    # oracle's own answer moves by ~1e-3 under a 1e-7 relative change of phi0
    # (FP32 rounding).  The batch must equal the single-lattice FP32 run and
    # stay within four times that spread of the oracle.
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, u0, p0 = inst[3]
    o = oracle.from_params(p, phi0, u0, p0)
    o.step(200, 0)
    ophi = o.fields()[0]
    rng = np.random.default_rng(0)
    o2 = oracle.from_params(p, phi0 * (1 + 1e-7 * rng.standard_normal(phi0.shape)), u0, p0)
    o2.step(200, 0)
    spread = np.abs(o2.fields()[0] - ophi).max()
    phi = b.fields(3)[0]
    s = Simulation(p, phi0, u0, p0, precision="fp32")
    s.step(200)
    assert np.array_equal(phi, s.phi())
    assert np.abs(phi - ophi).max() < max(1e-5, 4 * spread), spread


def test_unstable_instance_is_stopped():
    from paper_2206_11637_gb300 import _lib as L
    from paper_2206_11637_gb300.batch import Batch
    inst = [W.static_drop(16, 5.0), W.static_drop(16, 5.0), W.capillary_wave(32, ny=40, a0=1.0, xi=4.0),
            W.static_drop(20, 6.0, mobility=0.05)]
    p, phi0, u0, p0 = inst[1]
    p.mobility = 1e-4              # far below the stable range (the paper: small M is unstable)
    p.sigma = 1e-2
    b = Batch(inst, precision="fp32", tune=False)
    for _ in range(40):
        b.step(50)
        out, nf, st = b.diag(check=False)
        if nf[1] > 0:
            break
    assert nf[1] > 0 and st == L.PFL_ERR_UNSTABLE
    ok = [i for i in range(4) if i != 1]
    assert np.all(nf[ok] == 0)
    before = b.fields(1)[0].copy()
    b.step(33)                     # odd: the stopped instance keeps its own buffer roles
    assert np.array_equal(np.nan_to_num(b.fields(1)[0], nan=7.0), np.nan_to_num(before, nan=7.0))
    out2, nf2, _ = b.diag(check=False)
    assert np.all(nf2[ok] == 0)
