"""Host logic of the design search on CPU: the spline coordinates and the
search box of the choice of nested populations."""
import numpy as np

import workloads
from paper_2005_10494_gb300.search import r_search_box


def _per_r(best):
    pairs = workloads.paper_r_pairs()
    assert len(pairs) == 171
    return [(a, b, 1.0 - (a - best[0]) ** 2 - (b - best[1]) ** 2) for a, b in pairs]


def test_box_is_inside_the_data_and_around_the_best_pair():
    per_r = _per_r((0.45, 0.15))
    pts, vals, lo, hi = r_search_box(per_r)
    assert pts.shape == (171, 2) and vals.shape == (171,)
    np.testing.assert_allclose(pts[:, 1], [b / a for a, b, _ in per_r])
    ib = int(np.argmax(vals))
    assert np.all(lo <= pts[ib]) and np.all(pts[ib] <= hi)
    assert np.all(lo >= pts.min(0)) and np.all(hi <= pts.max(0))
    assert hi[0] - lo[0] <= 4 * 0.05 + 1e-12


def test_box_keeps_r3_above_the_smallest_evaluated_r3():
    # best pair at the smallest r3: the rectangle in (r2, r3/r2) would reach
    # r3 = lo_r2 * min(r3/r2) < 0.05 without the bound
    for best in ((0.35, 0.05), (0.3, 0.05), (0.9, 0.05), (0.1, 0.05)):
        pts, vals, lo, hi = r_search_box(_per_r(best))
        assert lo[0] * lo[1] >= 0.05 - 1e-12, (best, lo)
        assert lo[1] <= hi[1]
        # every corner of the box keeps 1 > r2 > r3 > 0
        for r2 in (lo[0], hi[0]):
            for v in (lo[1], hi[1]):
                assert 1.0 > r2 > r2 * v > 0.0


def test_box_with_one_r2_value_uses_the_default_step():
    per_r = [(0.5, b, 1.0 - (b - 0.2) ** 2) for b in (0.05, 0.1, 0.2, 0.3, 0.4)]
    pts, vals, lo, hi = r_search_box(per_r)
    assert lo[0] == hi[0] == 0.5                      # the data span one r2
    assert lo[1] <= 0.2 / 0.5 <= hi[1]
    assert lo[0] * lo[1] >= 0.05 - 1e-12
