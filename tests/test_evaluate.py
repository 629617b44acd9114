"""Host-side geometry scores of evaluate.py (Chamfer distance and F-score of
Sec. 4.1) against closed forms on synthetic point sets (CPU only)."""
import numpy as np
import pytest

pytest.importorskip("scipy")
torch = pytest.importorskip("torch")

from paper_2412_03451_gb300 import evaluate as E


def _grid(n=40, spacing=0.01):
    u, v = np.meshgrid(np.arange(n) * spacing, np.arange(n) * spacing)
    return np.stack([u.ravel(), v.ravel(), np.zeros(u.size)], 1)


def test_identical_sets_score_zero_and_one():
    P = _grid()
    s = E.chamfer_fscore(P, P.copy())
    assert s["chamfer_m"] == 0.0 and s["accuracy_m"] == 0.0 and s["fscore"] == 1.0


@pytest.mark.parametrize("d,f", [(0.03, 1.0), (0.07, 0.0)])
def test_offset_plane_closed_form(d, f):
    # a plane of points moved by d along its normal: every nearest neighbour is exactly d away
    P = _grid()
    Q = P + np.array([0.0, 0.0, d])
    s = E.chamfer_fscore(Q, P, thresh=0.05)
    assert s["accuracy_m"] == pytest.approx(d, abs=1e-5)
    assert s["completeness_m"] == pytest.approx(d, abs=1e-5)
    assert s["chamfer_m"] == pytest.approx(d, abs=1e-5)
    assert s["fscore"] == f


def test_partial_coverage_splits_precision_and_recall():
    # prediction covers half of the ground truth exactly: precision 1, recall 1/2 (far half),
    # F = 2 * 1 * 0.5 / 1.5
    gt = _grid(40)
    pred = gt[gt[:, 0] < 0.195]
    far = gt[:, 0] > 0.195 + 0.05
    s = E.chamfer_fscore(pred, gt, thresh=0.05)
    recall = 1.0 - far.mean()
    assert s["accuracy_m"] == 0.0
    assert s["fscore"] == pytest.approx(2 * recall / (1 + recall), abs=1e-4)


def test_empty_prediction():
    s = E.chamfer_fscore(np.zeros((0, 3)), _grid(5))
    assert s["fscore"] == 0.0 and s["chamfer_m"] is None
