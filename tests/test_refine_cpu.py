"""Host logic of the positivity refinement (Section 3.2): the windows."""
import numpy as np


def test_windows_follow_the_paper():
    # +-25% around non-negative pixels; [0, |s| + 15%] for negative ones
    from paper_1101_5803_gb300.refine import windows
    lo, hi = windows([2.0, 0.0, -1.0, 4.0, -0.2])
    np.testing.assert_allclose(lo, [1.5, 0.0, 0.0, 3.0, 0.0])
    np.testing.assert_allclose(hi, [2.5, 0.0, 1.15, 5.0, 0.23])
    assert np.all(lo >= 0) and np.all(hi >= lo)
