"""The C ABI library builds, loads and exports every entry point that
include/ps.h declares; host-side planning and argument checks work without a
GPU (no compute calls are made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2412_03451_gb300 import _build, binding
    _build.build()
    return binding.load()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ps_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_path(lib):
    names = declared_functions()
    for fn in ("ps_project_cull", "ps_bin_tiles", "ps_splat_fwd", "ps_splat_bwd", "ps_loss",
               "ps_adam_step"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_exports_match_header(lib):
    from paper_2412_03451_gb300 import binding
    assert set(binding.EXPORTS) <= declared_functions()
    assert binding.ps_version() >= 1


def test_struct_sizes_match_header(lib):
    from paper_2412_03451_gb300 import binding as B
    assert ctypes.sizeof(B.PsView) == 128
    assert ctypes.sizeof(B.PsSettings) == 64
    assert ctypes.sizeof(B.PsStepState) == 24
    assert ctypes.sizeof(B.PsFrame) == 32


def test_plan_views_host_only(lib):
    from paper_2412_03451_gb300 import binding as B
    H, W = [96, 48, 480], [128, 64, 640]
    w2c = np.tile(np.eye(3, 4, dtype=np.float32), (3, 1, 1))
    intr = np.tile(np.array([100, 100, 64, 48], np.float32), (3, 1))
    views, frame = B.ps_plan_views(H, W, [0, 1, 1], [0, 10, 25], w2c, intr, 16, 16)
    assert frame.n_views == 3 and frame.max_K == 15
    assert frame.n_records == 10 + 15 + 15
    assert frame.n_tiles == 6 * 8 + 3 * 4 + 30 * 40
    assert frame.n_pixels == 96 * 128 + 48 * 64 + 480 * 640
    assert [v.tile_off for v in views] == [0, 48, 60]
    assert [v.rec_off for v in views] == [0, 10, 25]
    assert [v.plane_off for v in views] == [0, 10, 10]
    assert [v.pix_off for v in views] == [0, 96 * 128, 96 * 128 + 48 * 64]


def test_plan_views_rejects_bad_input(lib):
    from paper_2412_03451_gb300 import binding as B
    w2c = np.tile(np.eye(3, 4, dtype=np.float32), (2, 1, 1))
    intr = np.tile(np.array([100, 100, 64, 48], np.float32), (2, 1))
    with pytest.raises(B.PsError):
        B.ps_plan_views([96, 96], [128, 128], [1, 0], [0, 5, 9], w2c, intr, 16, 16)   # unsorted scenes
    with pytest.raises(B.PsError):
        B.ps_plan_views([96, 0], [128, 128], [0, 0], [0, 5], w2c, intr, 16, 16)       # empty image
    with pytest.raises(B.PsError):
        B.ps_plan_views([96, 96], [128, 128], [0, 0], [0, 5], w2c, intr, 0, 16)       # bad tile


def test_null_arguments_rejected_before_launch(lib):
    from paper_2412_03451_gb300 import binding as B
    s = B.make_settings(20.0, B.filter_margin(20.0))
    assert lib.ps_project_cull(None, None, ctypes.byref(s), None, None, None, None, None) == B.PS_ERR_ARG
    assert lib.ps_splat_fwd(None, ctypes.byref(s), None, None, None, None, 0, None, None, None,
                            None, 0, None, None) == B.PS_ERR_ARG
    assert lib.ps_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, 0.0,
                            None) == B.PS_ERR_ARG
    assert lib.ps_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 0, 0.0,
                            None) == B.PS_ERR_ARG
    # the state form: no schedule, a negative clamp start, null parameter arrays
    state = ctypes.create_string_buffer(64)
    assert lib.ps_adam_step_state(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, None, 0.0, 0,
                                  None) == B.PS_ERR_ARG
    assert lib.ps_adam_step_state(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, state, 0.0, -1,
                                  None) == B.PS_ERR_ARG
    assert lib.ps_adam_step_state(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, state, 0.0, 0,
                                  None) == B.PS_ERR_ARG
    assert B.ps_status_string(B.PS_ERR_CAPACITY) == "tile-list capacity exceeded"


def test_settings_validation(lib):
    from paper_2412_03451_gb300 import binding as B
    views, frame = B.ps_plan_views([96], [128], [0], [0, 4], np.eye(3, 4, dtype=np.float32)[None],
                                   np.array([[100, 100, 64, 48]], np.float32), 16, 16)
    frame.views = 256          # a non-null placeholder: every call below fails its checks first
    dummy = ctypes.c_void_p(256)
    for bad in (dict(M=0), dict(M=65), dict(tile_w=12, tile_h=12), dict(lam=0.0)):
        kw = dict(lam=20.0, delta=0.1, M=30, tile_w=16, tile_h=16)
        kw.update(bad)
        s = B.make_settings(kw.pop("lam"), kw.pop("delta"), **kw)
        code = lib.ps_splat_fwd(ctypes.byref(frame), ctypes.byref(s), dummy, dummy, dummy, dummy,
                                1, dummy, dummy, None, dummy, 256, None, None)
        assert code == B.PS_ERR_ARG, bad


def test_plane_set_operations_reject_bad_arguments(lib):
    # host-side checks of the splitting and merging entry points: nothing is launched
    from paper_2412_03451_gb300 import binding as B
    d = ctypes.c_void_p(256)
    split = lib.ps_split_planes
    # no scenes, negative planes, zero iterations, negative threshold, capacity below P
    assert split(d, None, None, 0, d, 4, d, 10, 0.2, d, None, None, d, 8, d, d, None) == B.PS_ERR_ARG
    assert split(d, None, None, 1, d, -1, d, 10, 0.2, d, None, None, d, 8, d, d, None) == B.PS_ERR_ARG
    assert split(d, None, None, 1, d, 4, d, 0, 0.2, d, None, None, d, 8, d, d, None) == B.PS_ERR_ARG
    assert split(d, None, None, 1, d, 4, d, 10, -1.0, d, None, None, d, 8, d, d, None) == B.PS_ERR_ARG
    assert split(d, None, None, 1, d, 4, d, 10, 0.2, d, None, None, d, 3, d, d, None) == B.PS_ERR_ARG
    assert split(d, None, None, 1, None, 4, d, 10, 0.2, d, None, None, d, 8, d, d, None) == B.PS_ERR_ARG
    centre = (ctypes.c_float * 3)(0, 0, 0)
    merge = lib.ps_merge_planes
    assert merge(d, 8193, centre, 25.0, 0.001, d, d, d, None) == B.PS_ERR_ARG      # above 8,192
    assert merge(d, 4, centre, 95.0, 0.001, d, d, d, None) == B.PS_ERR_ARG        # angle > 90
    assert merge(d, 4, centre, 25.0, -1.0, d, d, d, None) == B.PS_ERR_ARG         # negative offset
    assert merge(d, 4, None, 25.0, 0.001, d, d, d, None) == B.PS_ERR_ARG
    assert lib.ps_radii_grad_accum(None, None, 1.0, 4, None, None) == B.PS_ERR_ARG


def test_wait_selftest_rejects_bad_arguments(lib):
    # a status word is required and the poll count is bounded (1 .. 2^24): nothing is launched
    from paper_2412_03451_gb300 import binding as B
    d = ctypes.c_void_p(256)
    assert lib.ps_wait_selftest(None, 1000, None) == B.PS_ERR_ARG
    assert lib.ps_wait_selftest(d, 0, None) == B.PS_ERR_ARG
    assert lib.ps_wait_selftest(d, (1 << 24) + 1, None) == B.PS_ERR_ARG


def test_gaussian_flag_checks(lib):
    from paper_2412_03451_gb300 import binding as B
    views, frame = B.ps_plan_views([96], [128], [0], [0, 4], np.eye(3, 4, dtype=np.float32)[None],
                                   np.array([[100, 100, 64, 48]], np.float32), 16, 16)
    frame.views = 256
    dummy = ctypes.c_void_p(256)
    for flags, delta in ((B.PS_GAUSSIAN | B.PS_HARD, B.gauss_extent()), (B.PS_GAUSSIAN, 0.0)):
        s = B.make_settings(20.0, delta, flags=flags)
        code = lib.ps_splat_fwd(ctypes.byref(frame), ctypes.byref(s), dummy, dummy, dummy, dummy,
                                1, dummy, dummy, None, dummy, 256, None, None)
        assert code == B.PS_ERR_ARG, flags


def test_schedule_functions_host_only(lib):
    # Eq. 10 and the filter margin of Eq. 7-8 / Sec. 3.2, computed by the library on the host,
    # against the oracle's independent definitions and closed forms
    import math
    from oracle import oracle as O
    from paper_2412_03451_gb300 import binding as B
    for ite in (0, 1, 999, 1000, 2000, 5703, 5704, 10000):
        assert B.lambda_schedule(ite) == O.lambda_schedule(ite)
    assert B.lambda_schedule(0) == pytest.approx(20.0 / math.e, rel=1e-15)
    assert B.lambda_schedule(1000) == pytest.approx(20.0, rel=1e-15)
    assert B.lambda_schedule(10 ** 6) == 300.0
    for lam in (7.36, 20.0, 300.0):
        d = B.filter_margin(lam)
        assert d == pytest.approx(O.filter_margin(lam), rel=1e-15)
        # 2 sigmoid(-5 lam delta) = w_min
        assert 2.0 / (1.0 + math.exp(5.0 * lam * d)) == pytest.approx(1e-4, rel=1e-12)
    assert math.isnan(B.filter_margin(0.0)) and math.isnan(B.filter_margin(1.0, 1.5))
    k = B.gauss_extent()
    assert math.exp(-0.5 * k * k) == pytest.approx(1e-4, rel=1e-12)
    raw = B.step_schedule(5, first=998, lam_offset=2)
    st = (B.PsStepState * 5).from_buffer_copy(raw)
    for i, e in enumerate(st):
        ite = 998 + i
        assert e.step == ite + 1
        assert e.lambda_ == np.float32(O.lambda_schedule(ite + 2))
        assert e.delta == pytest.approx(O.filter_margin(float(np.float32(O.lambda_schedule(ite + 2)))),
                                        rel=1e-15)
        assert e.bc1 == np.float32(1.0 - np.float64(np.float32(0.9)) ** (ite + 1))
        assert e.bc2 == np.float32(1.0 - np.float64(np.float32(0.999)) ** (ite + 1))
    # argument checks happen on the host
    arr = (B.PsStepState * 1)()
    assert lib.ps_step_schedule(-1, 1, 0, 0.9, 0.999, 1e-4, arr) == B.PS_ERR_ARG
    assert lib.ps_step_schedule(0, 1, 0, 1.0, 0.999, 1e-4, arr) == B.PS_ERR_ARG
    assert lib.ps_step_schedule(0, 1, 0, 0.9, 0.999, 0.0, arr) == B.PS_ERR_ARG
    assert lib.ps_step_schedule(0, 1, 0, 0.9, 0.999, 1e-4, None) == B.PS_ERR_ARG
    assert lib.ps_step_schedule(0, 0, 0, 0.9, 0.999, 1e-4, None) == B.PS_OK
