"""PlaneSplatFunction: the torch.autograd.Function around the C ABI.

Its forward is projection, binning and the forward splat (Sec. 3.2, Eq. 4-13);
its backward is the hand-written adjoint kernel ps_splat_bwd.  Checked on the
64-plane room through torch.autograd.grad of a scalar of (D, N):

  * against the oracle's analytic FP64 adjoint, per plane and group,
    ||g - g*|| <= 1e-3 ||g*|| + 1e-6 max ||g*|| (upstream weights zeroed where
    FP32 rounding could flip a branch, the filter, the order or the range);
  * against FP64 central differences of the oracle's render for the planes with
    the largest gradients (upstream weights zeroed wherever such a flip lies
    within the difference step);
  * when the renderer renders something else (other planes, other cameras)
    between the forward and .backward(), the gradient is unchanged.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_03451_gb300 import scenes as S

from gpu_cases import Z_NEAR32, f32, grad_errors, oracle_render, record

pytestmark = pytest.mark.gpu

LAM = 20.0


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 1)
    cams = room.cams
    o = oracle_render(init, cams, LAM)
    rng = np.random.default_rng(21)
    wD = rng.normal(size=o["depth"].shape)
    wN = rng.normal(size=o["normal"].shape)
    ill = (o["ill"] & 12) != 0
    wD[ill] = 0.0
    wN[ill] = 0.0
    return room, init, cams, wD.astype(np.float32), wN.astype(np.float32)


def _renderer(cams, K):
    from paper_2412_03451_gb300 import splat as SP
    V = cams.V
    r = SP.Renderer([cams.H] * V, [cams.W] * V, [0] * V, [0, K])
    r.set_cameras(cams.w2c, cams.intr)
    return r


def _grad(r, init, wD, wN, interfere=None):
    import torch
    from paper_2412_03451_gb300 import splat as SP
    flat = SP.planes_to_flat(init.center, init.quat, init.radii, "cuda").requires_grad_(True)
    D, N = SP.PlaneSplatFunction.apply(flat, r, LAM)
    if interfere is not None:
        interfere(r, flat.detach())
    s = (D * torch.from_numpy(wD.reshape(-1)).cuda()).sum() + \
        (N * torch.from_numpy(wN.reshape(-1, 3)).cuda()).sum()
    (g,) = torch.autograd.grad(s, flat)
    torch.cuda.synchronize()
    return D.detach().cpu().numpy(), g.cpu().numpy().astype(np.float64)


def _split(g, K):
    return g[:3 * K].reshape(K, 3), g[3 * K:7 * K].reshape(K, 4), g[7 * K:].reshape(K, 4)


def test_autograd_gradient_matches_oracle_adjoint(setup):
    room, init, cams, wD, wN = setup
    r = _renderer(cams, init.K)
    D, g = _grad(r, init, wD, wN)
    oc, oq, orr = O.backward(init.center, init.quat, init.radii, cams.w2c, cams.intr, cams.H,
                             cams.W, f32(LAM), wD, wN, z_near=Z_NEAR32)
    res = {k: grad_errors(a, b) for k, a, b in zip(("center", "quat", "radii"), _split(g, init.K),
                                                   (oc, oq, orr))}
    record("autograd_vs_oracle", **{k: list(v) for k, v in res.items()})
    for k, (nbad, worst) in res.items():
        assert nbad == 0, (k, nbad, worst)


def test_autograd_gradient_matches_central_differences(setup):
    room, init, cams, _, _ = setup
    H, W, K = cams.H, cams.W, init.K
    lam32 = f32(LAM)
    h = 1e-6
    # upstream weights zeroed wherever a branch, the filter, the order or the range could
    # flip within the step (the oracle's flags at eta = 1e-4, no smooth criterion)
    ob = O.render(init.center, init.quat, init.radii, cams.w2c, cams.intr, H, W, lam32,
                  z_near=Z_NEAR32, eta=1e-4, tol_d=np.inf, tol_n=np.inf)
    rng = np.random.default_rng(22)
    wD = rng.normal(size=ob["depth"].shape)
    wN = rng.normal(size=ob["normal"].shape)
    bad = ob["ill"] != 0
    wD[bad] = 0.0
    wN[bad] = 0.0
    wD, wN = wD.astype(np.float32), wN.astype(np.float32)
    r = _renderer(cams, K)
    _, g = _grad(r, init, wD, wN)
    gc, gq, gr = _split(g, K)
    gpu = np.concatenate([gc, gq, gr], 1)
    pick = np.argsort(-np.linalg.norm(gpu, axis=1))[:8]

    def J(c, q, rr):
        o = O.render(c, q, rr, cams.w2c, cams.intr, H, W, lam32, z_near=Z_NEAR32)
        return float(np.sum(wD * o["depth"]) + np.sum(wN * o["normal"]))

    base = [init.center.astype(np.float64), init.quat.astype(np.float64),
            init.radii.astype(np.float64)]
    fd = np.zeros((len(pick), 11))
    for n, k in enumerate(pick):
        col = 0
        for grp in range(3):
            for e in range(base[grp].shape[1]):
                plus = [b.copy() for b in base]
                minus = [b.copy() for b in base]
                plus[grp][k, e] += h
                minus[grp][k, e] -= h
                fd[n, col] = (J(*plus) - J(*minus)) / (2 * h)
                col += 1
    err = np.linalg.norm(gpu[pick] - fd, axis=1)
    bound = 1e-3 * np.linalg.norm(fd, axis=1) + 1e-6 * np.linalg.norm(fd, axis=1).max()
    record("autograd_vs_fd", worst=float((err / bound).max()))
    assert (err <= bound).all(), np.sort(err / bound)[-4:]


def test_autograd_backward_survives_a_render_in_between(setup):
    room, init, cams, wD, wN = setup
    r = _renderer(cams, init.K)
    D0, g0 = _grad(r, init, wD, wN)

    def interfere(rr, flat):
        # other planes at another lambda, then other cameras: both overwrite the
        # renderer's records, tile lists and view descriptors before .backward()
        moved = flat.clone()
        moved[: 3 * init.K] += 0.05
        rr.forward(moved, 100.0)
        rr.set_cameras(cams.w2c[::-1].copy(), cams.intr[::-1].copy())
        rr.forward(flat, 7.0)

    D1, g1 = _grad(r, init, wD, wN, interfere=interfere)
    assert np.array_equal(D0, D1)
    # the same lists: only the order of float atomics differs
    for a, b in zip(_split(g1, init.K), _split(g0, init.K)):
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-7
