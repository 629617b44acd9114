"""The allocation-free backward (ps_splat_bwd_noalloc) against ps_splat_bwd.

Some callers of this library cannot allocate device memory -- an engine whose
device memory belongs to a fixed arena, a real-time loop that must not enter
the CUDA allocator, a plug-in host without a device allocator -- so they cannot
pass the scratch buffer that ps_splat_bwd needs.  ps_splat_bwd_noalloc keeps
that scratch in an array compiled into the library.  This test calls it
through the C ABI twice in a row (the second call must not see the first
call's leftovers) and checks both results against ps_splat_bwd with a
caller-provided buffer, within the tolerance the other gradient comparisons
use for float-atomic ordering.  It also checks that a frame too large for the
static array is refused.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_backward_matches_workspace_backward():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2412_03451_gb300 import binding as B
    from paper_2412_03451_gb300 import scenes as S
    from paper_2412_03451_gb300 import splat as SP

    lib = B.load()
    fn = lib.ps_splat_bwd_noalloc
    P, LL = ctypes.c_void_p, ctypes.c_longlong
    fn.argtypes = [P, P, P, P, P, P, P, LL, P, P, P, P, P, P, P]
    fn.restype = ctypes.c_int

    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 1)
    cams = room.cams
    V, H, W = cams.V, cams.H, cams.W
    r = SP.Renderer([H] * V, [W] * V, [0] * V, [0, init.K])
    r.set_cameras(cams.w2c, cams.intr)
    flat = SP.planes_to_flat(init.center, init.quat, init.radii, "cuda")
    lam = 20.0
    r.ensure_capacity(flat, lam)
    r.forward(flat, lam)
    gtD, gtN, _ = O.raycast(room.gt.center, room.gt.quat, room.gt.radii, cams.w2c, cams.intr, H, W)
    r.loss(torch.from_numpy(gtD.astype(np.float32).reshape(-1)).cuda(),
           torch.from_numpy(gtN.astype(np.float32).reshape(-1, 3)).cuda())

    ref = torch.zeros_like(flat)
    r.backward(flat, ref)               # existing entry point, caller-provided scratch
    torch.cuda.synchronize()
    ref = ref.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(ref) > 0

    pl = r.planes_struct(flat)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    K = init.K
    for call in range(2):
        g = torch.zeros_like(flat)
        gc, gq, gr = SP.flat_views(g, K)
        code = fn(ctypes.byref(pl), ctypes.byref(r.frame), ctypes.byref(r.settings),
                  r.rec.data_ptr(), r.tile_key.data_ptr(), r.tile_ptr.data_ptr(), r.tile_ent.data_ptr(),
                  r.capacity, r.dLdD.data_ptr(), r.dLdN.data_ptr(), gc.data_ptr(), gq.data_ptr(),
                  gr.data_ptr(), r.status.data_ptr(), stream)
        assert code == B.PS_OK, B.ps_status_string(code)
        torch.cuda.synchronize()
        got = g.cpu().numpy().astype(np.float64)
        for a, b in ((0, 3 * K), (3 * K, 7 * K), (7 * K, 11 * K)):
            assert np.linalg.norm(got[a:b] - ref[a:b]) <= 1e-5 * np.linalg.norm(ref[a:b]) + 1e-6, call
    assert int(r.status.item()) == 0

    # a frame with more records than the static array holds is refused before any launch
    big = B.PsFrame()
    big.n_views, big.n_records, big.n_tiles, big.max_K = 1, 65537, 1, 65537
    big.n_pixels, big.views = 1, r.frame.views
    code = fn(ctypes.byref(pl), ctypes.byref(big), ctypes.byref(r.settings), r.rec.data_ptr(),
              r.tile_key.data_ptr(), r.tile_ptr.data_ptr(), r.tile_ent.data_ptr(), r.capacity,
              r.dLdD.data_ptr(), r.dLdN.data_ptr(), gc.data_ptr(), gq.data_ptr(), gr.data_ptr(),
              r.status.data_ptr(), stream)
    assert code == B.PS_ERR_ARG
