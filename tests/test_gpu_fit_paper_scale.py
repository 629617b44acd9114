"""The paper-scale single-scene configuration end to end on the GPU: the synthetic
8x10x3 m room, 3,000 planes from the random surface start, 2,000 optimisation
iterations of 8 of its 64 views at 640x480, every step replayed from its camera
batch's CUDA graph with lambda, the filter margin and Adam's bias corrections
read from the device schedule (Eq. 10).  The fit must finish without a tile-list
overflow and bring the mean depth error over all 64 views below 2 cm."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_thousand_graph_replayed_iterations_reach_two_centimetres():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import bench
    wl = bench.Workload(0, (8, 8), "cuda:0")
    err0 = bench.depth_error_all_views(wl)
    out = bench.run_fit(wl, 2000)
    assert out["iterations"] == 2000 and wl.fit.ite == 2000
    assert out["depth_err_m_after"] < 0.02, out
    assert err0 > 0.1, err0          # the start is far from the ground truth
    assert out["ms_per_step"] > 0.0
