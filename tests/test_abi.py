"""The C ABI without a GPU: libsff.so builds for sm_103a, loads, exports
every function include/sff.h declares, and rejects invalid arguments on the
host before anything reaches CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sff.h")


@pytest.fixture(scope="module")
def sff():
    import paper_1710_10096_gb300 as sff
    sff.build()
    return sff


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sff_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("sff_features", "sff_match_views", "sff_match_quad", "sff_consistency_filter", "sff_emit_seeds"):
        assert n in names


def test_every_declared_symbol_is_exported(sff):
    L = ctypes.CDLL(sff.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_default_params_are_the_papers(sff):
    p = sff.default_params()
    # Sec. 5: k = 3 subscales (+ full resolution), 12 iterations, tau_c = 1, s_c = 150
    assert (p.num_scales, p.iterations, p.tau_c, p.region_min) == (4, 12, 1, 150)
    assert (p.tau_r, p.quant_shift, p.knn_temporal, p.knn_epipolar) == (1, 4, 4, 2)


def test_sizes(sff):
    p = sff.default_params()
    assert sff.pyramid_bytes(1242, 375, p) == 4 * 1242 * 375 * 52
    assert sff.pyramid_bytes(7, 100, p) == 0  # below the minimum size
    assert sff.pyramid_bytes(16385, 100, p) == 0
    ws = sff.workspace_bytes(1242, 375, p)
    assert ws >= 3 * 1242 * 375 * 4 and ws % 256 == 0
    bad = sff.default_params(num_scales=5)
    assert sff.workspace_bytes(64, 64, bad) == 0


def test_status_strings(sff):
    L = sff.lib()
    assert L.sff_status_string(0) == b"ok"
    assert L.sff_status_string(-1) == b"invalid argument"
    assert L.sff_status_string(-3) == b"workspace too small"


def test_argument_errors_without_gpu(sff):
    L = sff.lib()
    p = sff.default_params()
    P = ctypes.byref(p)
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: every call below fails validation first
    null = ctypes.c_void_p(0)
    ws = sff.workspace_bytes(64, 48, p)
    # null pointers
    assert L.sff_features(null, 64, 48, 192, P, fake, fake, ws, null) == -1
    # bad sizes / pitch / params
    assert L.sff_features(fake, 7, 48, 192, P, fake, fake, ws, null) == -1
    assert L.sff_features(fake, 64, 48, 100, P, fake, fake, ws, null) == -1
    bad = sff.default_params(knn_temporal=9)
    assert L.sff_features(fake, 64, 48, 192, ctypes.byref(bad), fake, fake, ws, null) == -1
    # misaligned pyramid
    assert L.sff_features(fake, 64, 48, 192, P, ctypes.c_void_p(0x10008), fake, ws, null) == -1
    # workspace too small
    assert L.sff_features(fake, 64, 48, 192, P, fake, fake, 16, null) == -3
    assert L.sff_match_views(fake, fake, fake, fake, 64, 48, 2, 1, P, fake, fake, fake, ws, null) == -1
    assert L.sff_match_views(fake, fake, fake, fake, 64, 48, 0, 1, P, fake, fake, fake, 0, null) == -3
    assert L.sff_match_quad(fake, fake, fake, null, 64, 48, 1, P, fake, fake, fake, fake, fake, ws, null) == -1
    assert L.sff_match_quad(fake, fake, fake, fake, 64, 48, 1, P, fake, fake, fake, fake, fake, 0, null) == -3
    assert L.sff_consistency_filter(fake, fake, fake, null, 64, 48, P, fake, fake, fake, ws, null) == -1
    assert L.sff_emit_seeds(fake, fake, fake, fake, 64, 48, fake, -1, fake, fake, ws, null) == -1
    assert L.sff_emit_seeds(fake, fake, fake, fake, 64, 48, fake, 10, fake, fake, 0, null) == -3


def test_product_path_has_no_oracle_dependency():
    # the package and its CUDA sources never reference the oracle
    pkg = os.path.join(ROOT, "paper_1710_10096_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("oracle-", ""), os.path.join(dirpath, f)


def test_tuning_space(sff):
    assert sff.default_tuning().as_tuple() in sff.TUNING_SPACE
    for cand in sff.TUNING_SPACE:
        assert sff.make_tuning(*cand).as_tuple() == cand
    with pytest.raises(sff.SffError):
        sff.make_tuning(3, 32, 8)


def test_extension_rows_without_gpu(sff):
    # defaults, workspace sizes and argument checks of the paper-order,
    # disparity-fill, interpolation and SIFT-cost entry points: all on the
    # host, before anything reaches CUDA
    L = sff.lib()
    p = sff.default_params()
    P = ctypes.byref(p)
    fake = ctypes.c_void_p(0x10000)
    null = ctypes.c_void_p(0)
    ws = sff.workspace_bytes(64, 48, p)
    # paper order
    assert L.sff_match_views_sequential(fake, fake, fake, fake, 64, 48, 2, 1, P, fake, fake, fake, ws, null) == -1
    assert L.sff_match_views_sequential(fake, fake, fake, fake, 64, 48, 0, 1, P, fake, fake, fake, 0, null) == -3
    # disparity fill: defaults (Hirschmueller-style penalties), parameter limits
    sp = sff.default_sgm_params()
    assert (sp.max_disp, sp.p1, sp.p2) == (128, 10, 120)
    assert sff.sgm_workspace_bytes(64, 48, sp) >= 64 * 48 * (2 * 8 + 9 * 128)
    for bad in (dict(max_disp=96), dict(max_disp=512), dict(p1=-1), dict(p1=30, p2=20), dict(p2=194)):
        assert sff.sgm_workspace_bytes(64, 48, sff.default_sgm_params(**bad)) == 0
    SP = ctypes.byref(sp)
    sws = sff.sgm_workspace_bytes(64, 48, sp)
    assert L.sff_sgm(null, fake, 192, 64, 48, SP, fake, fake, sws, null) == -1
    assert L.sff_sgm(fake, fake, 100, 64, 48, SP, fake, fake, sws, null) == -1      # pitch < 3 W
    assert L.sff_sgm(fake, fake, 192, 64, 48, SP, ctypes.c_void_p(0x10001), fake, sws, null) == -1  # odd disp
    assert L.sff_sgm(fake, fake, 192, 64, 48, SP, fake, fake, 16, null) == -3
    assert L.sff_emit_seeds_geo(fake, fake, fake, fake, null, 64, 48, P, fake, 10, fake, fake, ws, null) == -1
    assert L.sff_emit_seeds_geo(fake, fake, fake, fake, fake, 64, 48, P, fake, 10, fake, fake, 0, null) == -3
    # interpolation: defaults of Sec. 5 and the principal point at the centre
    ip = sff.default_interp_params(101, 40, 700.0, 0.5)
    assert (ip.k_geo, ip.k_motion, ip.alpha, ip.dist_unit) == (160, 80, 2.2, 20.0)
    assert (ip.cx, ip.cy, ip.focal, ip.baseline) == (50.0, 19.5, 700.0, 0.5)
    IP = ctypes.byref(ip)
    with pytest.raises(sff.SffError):
        sff.default_interp_params(64, 48, 0.0, 0.5)
    iws = sff.interp_workspace_bytes(64, 48, 400)
    assert iws > 0 and sff.interp_workspace_bytes(7, 48, 400) == 0 and sff.interp_workspace_bytes(64, 48, -1) == 0
    assert L.sff_interpolate(null, fake, 400, 64, 48, IP, fake, fake, iws, null) == -1
    assert L.sff_interpolate(fake, fake, 400, 64, 48, IP, ctypes.c_void_p(0x10004), fake, iws, null) == -1  # field
    assert L.sff_interpolate(fake, fake, 400, 64, 48, IP, fake, fake, 16, null) == -3
    for bad in (dict(k_geo=0), dict(k_motion=1025), dict(alpha=-1.0), dict(dist_unit=0.0)):
        b = sff.default_interp_params(64, 48, 700.0, 0.5, **bad)
        assert L.sff_interpolate(fake, fake, 400, 64, 48, ctypes.byref(b), fake, fake, iws, null) == -1
    # SIFT-PCA cost
    assert sff.sift_workspace_bytes(64, 48) > 64 * 48 * 4 * 128 and sff.sift_workspace_bytes(64, 7) == 0
    four = (ctypes.c_void_p * 4)(fake, fake, fake, fake)
    some_null = (ctypes.c_void_p * 4)(fake, null, fake, fake)
    fws = sff.sift_workspace_bytes(64, 48)
    assert L.sff_sift_features(four, 192, 64, 48, P, some_null, fake, fws, null) == -1
    assert L.sff_sift_features(four, 192, 64, 48, P, four, fake, 16, null) == -3
    assert L.sff_match_views_sift(fake, fake, fake, fake, fake, fake, fake, ctypes.c_void_p(0x10004), 64, 48, 0, 1, P,
                                  fake, fake, fake, ws, null) == -1  # phi not 16-byte aligned
    assert L.sff_match_views_sift(fake, fake, fake, fake, fake, fake, fake, fake, 64, 48, 0, 1, P, fake, fake, fake,
                                  0, null) == -3


def test_batch_arguments_without_gpu(sff):
    # sff_run_batch checks every quad before its first launch; each call
    # below carries at least one invalid field, so none reaches CUDA
    L = sff.lib()
    p = sff.default_params()
    P = ctypes.byref(p)
    null = ctypes.c_void_p(0)
    w, h = 64, 48
    qws = sff.quad_workspace_bytes(w, h, p)
    assert qws > 0

    def quad(**over):
        q = sff.QuadDesc()
        for k in range(4):
            q.rgb[k] = 0x10000
            q.pyramid[k] = 0x20000
        q.pitch_bytes, q.width, q.height, q.seed = 3 * w, w, h, 1
        q.fwd, q.fwd_cost, q.inv, q.inv_cost = 0x30000, 0x40000, 0x50000, 0x60000
        q.keep, q.cerr, q.seeds, q.capacity, q.count = 0x70000, 0x80000, 0x90000, 400, 0xa0000
        q.workspace, q.workspace_bytes = 0xb0000, qws
        for k, v in over.items():
            setattr(q, k, v)
        return q

    def run(quads, params=P):
        arr = (sff.QuadDesc * max(1, len(quads)))(*quads)
        return L.sff_run_batch(arr, len(quads), params, None, null)

    bad_quads = [dict(width=7), dict(pitch_bytes=3 * w - 1), dict(workspace=0), dict(capacity=-1), dict(fwd=0),
                 dict(count=0), dict(seeds=0), dict(fwd=0x30004), dict(fwd_cost=0x40002), dict(workspace=0xb0010)]
    for over in bad_quads:
        assert run([quad(**over)]) == -1, over
    assert run([quad(workspace_bytes=qws - 1)]) == -3
    # a bad quad after a good one is still caught before any launch
    assert run([quad(), quad(keep=0)]) == -1
    assert run([quad(), quad(workspace_bytes=16)]) == -3
    # the batch itself
    assert L.sff_run_batch(None, 1, P, None, null) == -1
    assert run([]) == -1
    assert run([quad(width=7)] * (sff.MAX_BATCH + 1)) == -1
    bad = sff.default_params(num_scales=9)
    assert run([quad(width=7)], ctypes.byref(bad)) == -1
