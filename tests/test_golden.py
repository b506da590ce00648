"""The paper's printed values under tests/golden/ parse into the shapes the
GPU tests use, agree with the measurement schedule of the impact module, and
carry the signs and trends the paper's captions state (cavity depths below
the initial surface, crowns opening with time)."""
import golden
from paper_2206_11637_gb300 import impact as I


def test_taylor_bubble_table():
    re, exp = golden.taylor_bubble_re()
    assert set(re) == {64, 128}
    assert exp == 27.0
    for v in re.values():
        assert abs(v / exp - 1) < 0.01      # the paper's PFLBM agrees with the experiment within 1 %


def test_drop_tables():
    for case in ("vertical", "oblique"):
        times, tab = golden.drop_table(case)
        assert tuple(times) == I.TIMES[case]
        for D in (20, 40, 80):
            h, d = tab[("h_ca", D)], tab[("d_cr", D)]
            assert len(h) == len(d) == len(times)
            assert all(v < 0 for v in h)
            assert all(b > a for a, b in zip(d, d[1:]))
