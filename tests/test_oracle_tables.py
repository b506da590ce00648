"""Pins of the oracle's lattice tables and moment machinery (no GPU).

Checks against what the mathematics fixes: weights sum to one, odd moments
vanish, the second moment is c_s^2 I and the fourth is isotropic (the
properties the equilibria rely on, section "The lattice Boltzmann method");
the moment matrices are invertible and weighted-orthogonal; and the MRT
collision with all rates equal reduces to BGK (Eq. BGK is the special case of
Eq. mrt with a single rate).
"""
import itertools

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("q", [15, 27])
def test_lattice_isotropy(q):
    t = oracle.tables(q)
    c, w = t["c"].astype(float), t["w"]
    assert c.shape == (q, 3) and len({tuple(r) for r in t["c"]}) == q
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, CS2 * np.eye(3), atol=1e-15)
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(third, 0.0, atol=1e-16)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(fourth, iso, atol=1e-15)
    for i in range(q):
        assert np.array_equal(t["c"][t["opp"][i]], -t["c"][i])


def test_canonical_order():
    """Velocity order of the C interface: cz, cy, cx over -1, 0, 1 (cx fastest)."""
    t27 = oracle.tables(27)
    expect = [(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)]
    assert [tuple(r) for r in t27["c"]] == expect
    t15 = oracle.tables(15)
    expect15 = [v for v in expect if sum(a * a for a in v) != 2]
    assert [tuple(r) for r in t15["c"]] == expect15
    assert list(t15["opp"]) == [14 - i for i in range(15)]
    assert list(t27["opp"]) == [26 - i for i in range(27)]


@pytest.mark.parametrize("q", [15, 27])
def test_moment_matrices(q):
    t = oracle.tables(q)
    M, Minv, w, c, deg = t["M"], t["Minv"], t["w"], t["c"].astype(float), t["degree"]
    assert np.abs(M @ Minv - np.eye(q)).max() < 1e-13
    assert np.abs(Minv @ M - np.eye(q)).max() < 1e-13
    G = M @ np.diag(w) @ M.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-14 and np.all(np.diag(G) > 0)
    # grading: each moment row is orthogonal (weighted) to every monomial of lower degree
    for k in range(q):
        for a, b, cc in itertools.product(range(3), repeat=3):
            if a + b + cc < deg[k]:
                mono = c[:, 0] ** a * c[:, 1] ** b * c[:, 2] ** cc
                assert abs(np.sum(w * M[k] * mono)) < 1e-13
    # degrees 0..2 span exactly {1, c, cc}: counts 1, 3, 6
    assert [int(np.sum(deg == d)) for d in range(3)] == [1, 3, 6]


@pytest.mark.parametrize("q", [15, 27, 9])
def test_mrt_equal_rates_is_bgk(q):
    rng = np.random.Generator(np.random.PCG64(7))
    f, feq, src = rng.random(q), rng.random(q), rng.standard_normal(q) * 1e-3
    om = 1.37
    out = oracle.mrt_collide(q, f, feq, src, np.full(q, om))
    bgk = f - om * (f - feq) + (1 - om / 2) * src
    assert np.abs(out - bgk).max() < 1e-13


@pytest.mark.parametrize("q", [15, 27, 9])
def test_collision_conserves_zeroth_moment(q):
    t = oracle.tables(q)
    rng = np.random.Generator(np.random.PCG64(11))
    f = rng.random(q)
    feq = rng.random(q)
    feq *= f.sum() / feq.sum()
    src = t["w"] * (t["c"] @ rng.standard_normal(3))       # first-order source only
    rates = np.where(t["degree"] == 0, 0.0, np.where(t["degree"] == 2, 1.6, 1.0))
    out = oracle.mrt_collide(q, f, feq, src, rates)
    assert abs(out.sum() - f.sum()) < 1e-14
    # degree >= 3 moments relax at rate 1 to the equilibrium's, degree 2 at 1.6
    M = t["M"]
    m, meq, mo = M @ f, M @ feq, M @ out
    hi = t["degree"] >= 3
    assert np.abs(mo[hi] - meq[hi]).max() < 1e-13
    two = t["degree"] == 2
    assert np.abs(mo[two] - (m[two] - 1.6 * (m[two] - meq[two]))).max() < 1e-13


def test_d2q9_lattice():
    """D2Q9, the 2-D lattice of both sets: the cz = 0 slice of D3Q27 in the
    canonical order, weights 4/9, 1/9, 1/36, isotropic to 4th order in the
    plane, and a weighted-orthogonal moment basis graded 1, 2, 3 over degrees
    0, 1, 2."""
    t = oracle.tables(9)
    c, w = t["c"].astype(float), t["w"]
    expect = [(cx, cy, 0) for cy in (-1, 0, 1) for cx in (-1, 0, 1)]
    assert [tuple(r) for r in t["c"]] == expect
    assert list(t["opp"]) == [8 - i for i in range(9)]
    assert np.allclose(w, [1 / 36, 1 / 9, 1 / 36, 1 / 9, 4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36], atol=1e-16)
    c2 = c[:, :2]
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c2, c2), CS2 * np.eye(2), atol=1e-15)
    d = np.eye(2)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c2, c2, c2, c2), iso, atol=1e-15)
    M, Minv, deg = t["M"], t["Minv"], t["degree"]
    assert np.abs(M @ Minv - np.eye(9)).max() < 1e-13
    G = M @ np.diag(w) @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-14
    assert [int(np.sum(deg == k)) for k in range(5)] == [1, 2, 3, 2, 1]


@pytest.mark.parametrize("q", [27, 9])
def test_stencil_weights_factor_per_axis(q):
    """The weights of the phi stencil (D3Q27 in 3-D, D2Q9 in 2-D) are products
    of one 1-D weight per axis, w1(0) = 2/3 and w1(+-1) = 1/6: the property the
    adjoint's transposed stencil uses to sum plane by plane."""
    t = oracle.tables(q)
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    dims = 3 if q == 27 else 2
    for ci, wi in zip(t["c"], t["w"]):
        assert abs(wi - np.prod([w1[int(ci[a])] for a in range(dims)])) < 1e-16
