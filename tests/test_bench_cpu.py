"""Host-side logic of bench.py (no GPU): the Wilson interval behind the FER statistics and the
frame ranges of the statistics pass."""
import math

import pytest

import bench


def test_wilson_interval_known_values():
    """Wilson score interval p' +- h / (1 + z^2/n), p' = (p + z^2/2n) / (1 + z^2/n): checked against
    values worked out from that formula by hand and against its limiting properties."""
    z = 1.959963984540054
    # k = 0: lower bound 0, upper bound z^2 / (n + z^2)
    lo, hi = bench.wilson_ci(0, 100)
    assert lo == pytest.approx(0.0, abs=1e-15) and hi == pytest.approx(z * z / (100 + z * z), rel=1e-12)
    # k = n: the mirror image
    lo, hi = bench.wilson_ci(100, 100)
    assert hi == pytest.approx(1.0, abs=1e-15) and lo == pytest.approx(100 / (100 + z * z), rel=1e-12)
    # symmetric around 1/2 for k = n/2
    lo, hi = bench.wilson_ci(50, 100)
    assert lo + hi == pytest.approx(1.0, abs=1e-12)
    assert hi - lo == pytest.approx(2 * z * math.sqrt(0.25 / 100 + z * z / 40000) / (1 + z * z / 100), rel=1e-12)
    # a small proportion at the sizes of the FER statistics: contains p, and the normal
    # approximation's half-width is close for many errors
    lo, hi = bench.wilson_ci(597, 10 ** 6)
    assert lo < 597e-6 < hi
    assert (hi - lo) / 2 == pytest.approx(z * math.sqrt(597e-6 * (1 - 597e-6) / 1e6), rel=0.01)
    assert bench.wilson_ci(0, 0) == [0.0, 1.0]


def test_statistics_ranges_are_distinct():
    """Range r of rank q covers frames STATS_FRAME0 + (r world + q) B ... : no two (rank, range)
    pairs overlap, and none meets the timed batch's frames (below 2^32)."""
    B, world, ranges = 100_000, 4, 10
    spans = sorted((bench.STATS_FRAME0 + (r * world + q) * B, B) for r in range(ranges) for q in range(world))
    for (a, n), (b, _) in zip(spans, spans[1:]):
        assert a + n <= b
    assert spans[0][0] >= 1 << 32
    assert bench.STATS_SEED != bench.SEED


def test_oracle_one_core_leg_restores_threads():
    """The one-thread oracle timing reports one core and leaves the oracle's thread count as it
    found it (the all-cores leg and the reference arm run after it)."""
    oracle = pytest.importorskip("oracle")
    before = oracle.num_threads()
    r = bench.oracle_one_core(2.5, bench.SEED + 98, min_seconds=0.0)
    assert r["cores"] == 1 and r["frames"] == 64 and r["value"] > 0
    assert oracle.num_threads() == before
