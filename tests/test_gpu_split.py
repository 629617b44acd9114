"""Plane splitting on the GPU (ps_radii_grad_accum, ps_split_planes) against the
FP64 oracle: decisions, ranks, scene layout and moments exactly, geometry to
FP32 rounding."""
import numpy as np
import pytest

from oracle import split_oracle as SO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _case(seed, sizes):
    rng = np.random.default_rng(seed)
    P = int(sum(sizes))
    c = rng.normal(size=(P, 3)).astype(np.float32)
    q = rng.normal(size=(P, 4)).astype(np.float32)
    r = rng.uniform(0.05, 1.0, size=(P, 4)).astype(np.float32)
    # per-axis sums spread around the threshold 0.2 x n_iter (n_iter = 10)
    acc = rng.uniform(0.0, 4.0, size=(P, 2))
    # keep every decision clear of FP32 rounding: sums away from the threshold (2.0)
    # and the two axes apart
    acc[np.abs(acc - 2.0) < 1e-3] += 0.01
    close = np.abs(acc[:, 0] - acc[:, 1]) < 1e-3
    acc[close, 0] += 0.01
    acc = acc.astype(np.float32)
    if P > 3:
        q[3] = 0.0                      # degenerate rotation: never split
        acc[3] = 10.0
    ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    return c, q, r, acc, ptr


def _run(torch, c, q, r, acc, ptr, n_iter, tau, capacity=None):
    from paper_2412_03451_gb300 import binding as B
    P = len(c)
    dev = "cuda"
    flat = torch.from_numpy(np.concatenate([c.ravel(), q.ravel(), r.ravel()])).to(dev)
    m = torch.arange(11 * P, dtype=torch.float32, device=dev) + 1
    v = -m
    cap = 2 * P if capacity is None else capacity
    out = torch.full((11 * max(cap, 1),), np.nan, device=dev)
    mo = torch.full_like(out, np.nan)
    vo = torch.full_like(out, np.nan)
    ptr_d = torch.from_numpy(ptr).to(dev)
    ptr_o = torch.full_like(ptr_d, -1)
    rank = torch.full((P + 1,), -1, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    acc_d = torch.from_numpy(acc).to(dev)
    B.ps_split_planes(flat, m, v, ptr_d, acc_d, n_iter, tau, out, mo, vo, ptr_o, cap, rank, cnt)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), mo.cpu().numpy(), vo.cpu().numpy(), ptr_o.cpu().numpy(),
            rank.cpu().numpy(), int(cnt.item()), m.cpu().numpy())


@pytest.mark.parametrize("sizes", [[37], [5, 0, 1200, 3], [1, 1], [3000]])
def test_split_matches_oracle(torch, sizes):
    c, q, r, acc, ptr = _case(len(sizes) * 7 + sizes[0], sizes)
    n_iter, tau = 10, 0.2
    out, mo, vo, ptr_o, rank, cnt, m = _run(torch, c, q, r, acc, ptr, n_iter, tau)
    ref = SO.split_planes(c, q, r, ptr, acc.astype(np.float64), n_iter, tau, m=m, v=-m)
    assert cnt == ref["count"]
    assert np.array_equal(rank, ref["split_rank"])
    assert np.array_equal(ptr_o, ref["plane_ptr"])
    Pn = cnt
    got_c = out[:3 * Pn].reshape(Pn, 3)
    got_q = out[3 * Pn:7 * Pn].reshape(Pn, 4)
    got_r = out[7 * Pn:11 * Pn].reshape(Pn, 4)
    assert np.allclose(got_c, ref["center"], rtol=1e-5, atol=2e-6)
    assert np.array_equal(got_q, ref["quat"].astype(np.float32))
    assert np.allclose(got_r, ref["radii"], rtol=1e-6, atol=1e-7)
    assert np.array_equal(mo[:11 * Pn], ref["m"].astype(np.float32))
    assert np.array_equal(vo[:11 * Pn], ref["v"].astype(np.float32))


def test_capacity_too_small_writes_only_the_count(torch):
    c, q, r, acc, ptr = _case(11, [50])
    acc[:] = 9.0
    out, mo, vo, ptr_o, rank, cnt, _ = _run(torch, c, q, r, acc, ptr, 10, 0.2, capacity=60)
    ref = SO.split_planes(c, q, r, ptr, acc, 10, 0.2)
    assert cnt == ref["count"] > 60
    assert np.array_equal(rank, ref["split_rank"])
    assert np.all(np.isnan(out)) and np.all(ptr_o == -1)


def test_accumulation_matches_oracle(torch):
    from paper_2412_03451_gb300 import binding as B
    rng = np.random.default_rng(4)
    P = 1001
    g = rng.normal(size=(P, 4)).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, size=P).astype(np.float32)
    acc = torch.zeros((P, 2), device="cuda")
    gd = torch.from_numpy(g).cuda()
    B.ps_radii_grad_accum(gd, acc, scale=0.25)
    B.ps_radii_grad_accum(gd, acc, plane_scale=torch.from_numpy(scale).cuda())
    torch.cuda.synchronize()
    ref = SO.radii_grad_accum(SO.radii_grad_accum(np.zeros((P, 2)), g, 0.25), g, scale)
    assert np.allclose(acc.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)


def _partition(g):
    out = {}
    for i, x in enumerate(g):
        out.setdefault(int(x), []).append(i)
    return sorted(tuple(v) for k, v in out.items() if k >= 0)


@pytest.mark.parametrize("max_offset", [0.001, 0.1])
def test_merge_matches_oracle_on_room_rectangles(torch, max_offset):
    from paper_2412_03451_gb300 import binding as B
    from paper_2412_03451_gb300 import scenes as S
    room = S.large_room(1000, n_rect=2000, n_views=4)
    gt = room.gt
    P = gt.K
    q = gt.quat.copy()
    q[5] = 0.0                                  # degenerate: no group
    flat = torch.from_numpy(np.concatenate([gt.center.ravel(), q.ravel(), gt.radii.ravel()])).cuda()
    c0 = np.asarray(room.size, np.float64) / 2
    g = torch.full((P,), -7, dtype=torch.int32, device="cuda")
    reps = torch.full((P,), -7, dtype=torch.int32, device="cuda")
    ng = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ps_merge_planes(flat, P, c0, 25.0, max_offset, g, reps, ng)
    torch.cuda.synchronize()
    g_ref, reps_ref = SO.merge_planes(gt.center, q, gt.radii, c0, 25.0, max_offset)
    n = int(ng.item())
    assert n == len(reps_ref)
    gg = g.cpu().numpy()
    assert gg[5] == -1 and g_ref[5] == -1
    assert _partition(gg) == _partition(g_ref)
    # the rooms' faces lie on a few dozen planes: most rectangles merge
    assert n < 0.1 * P
