"""KGC selection rules (Algorithm 2 and the appendix aggregation rules) on hand-checked cases."""
import numpy as np

from paper_2408_06197_b300 import kgc


def test_permutation_mask_worked_example():
    # Section "Masked-based Encrypted Sorting": 5 clients, keep clients 1, 3, 5 (1-based)
    P = kgc.permutation_mask(5, [0, 2, 4])
    e = np.eye(5, dtype=np.int64)
    assert np.array_equal(P, np.stack([e[0], e[2], e[4], np.zeros(5, np.int64), np.zeros(5, np.int64)]))
    assert kgc.mask_weights(5, [0, 2, 4], average=False).tolist() == [1, 0, 1, 0, 1]
    assert np.allclose(kgc.mask_weights(5, [0, 2, 4], average=True), [1 / 3, 0, 1 / 3, 0, 1 / 3])


def test_krum_scores_hand_computed():
    pts = np.array([0.0, 1.0, 2.0, 10.0])
    d = (pts[:, None] - pts[None, :]) ** 2
    # n=4, f=1: n-f-2 = 1 nearest neighbour
    assert kgc.krum_scores(d, 1).tolist() == [1.0, 1.0, 1.0, 64.0]
    assert kgc.krum_select(d, 1, 1) == [0]          # tie -> lower index
    assert kgc.krum_select(d, 1, 3) == [0, 1, 2]
    # f=0: 2 nearest
    assert kgc.krum_scores(d, 0).tolist() == [5.0, 2.0, 5.0, 145.0]
    assert kgc.krum_select(d, 0, 2) == [1, 0]


def test_median_select():
    pts = np.array([0.0, 1.0, 5.0, 6.0, 20.0])
    d = np.abs(pts[:, None] - pts[None, :])
    sums = d.sum(axis=1)
    assert kgc.median_select(d) == int(np.argsort(sums, kind="stable")[2])
