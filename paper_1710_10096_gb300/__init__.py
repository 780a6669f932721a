"""SceneFlowFields sparse four-view matching stage on GB300 (sm_103a).

Python binding of libsff.so (C ABI in include/sff.h).  This module only
marshals arguments: every step of the stage -- features, initialisation,
propagation, random search, consistency/region filter, seeds -- runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if libsff.so is missing or cannot be loaded, every call
raises.

Paper: Schuster et al., "SceneFlowFields: Dense Interpolation of Sparse Scene
Flow Correspondences", WACV 2018, Sec. 3.1-3.2.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Params", "Tuning", "SffError", "default_params", "default_tuning", "make_tuning", "pyramid_bytes",
           "workspace_bytes", "quad_workspace_bytes", "features", "match_views", "match_quad", "match_quad_tuned",
           "consistency_filter", "emit_seeds", "run_batch", "QuadBuffers", "BatchMatcher", "QuadMatcher",
           "sift_workspace_bytes", "sift_features", "match_views_sift",
           "SgmParams", "default_sgm_params", "sgm_workspace_bytes", "sgm", "emit_seeds_geo",
           "InterpParams", "default_interp_params", "interp_workspace_bytes", "interpolate", "interp_status",
           "SEED_DTYPE", "lib", "build"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsff.so")
EMPTY_COST = 2147483647
FEATURE_BYTES = 48
WHOLE_RECORD_STRIDE = 2  # scales with a coarser grid keep whole records (see split_pyramid)
_lib = None


class SffError(RuntimeError):
    """A library call failed; `status` holds its SFF_ERR_* code (None for
    checks of the binding itself)."""

    def __init__(self, msg: str, status: int = None):
        super().__init__(msg)
        self.status = status


# status codes of include/sff.h
OK, ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT, ERR_CAPACITY = 0, -1, -2, -3, -4, -5


class Params(ctypes.Structure):
    """sff_params of include/sff.h."""
    _fields_ = [("num_scales", ctypes.c_int32), ("iterations", ctypes.c_int32), ("tau_c", ctypes.c_int32),
                ("region_min", ctypes.c_int32), ("tau_r", ctypes.c_int32), ("quant_shift", ctypes.c_int32),
                ("knn_temporal", ctypes.c_int32), ("knn_epipolar", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    """sff_tuning of include/sff.h: work distribution, never changes results."""
    _fields_ = [("lanes_per_pixel", ctypes.c_int32), ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("min_ctas", ctypes.c_int32), ("coarse", (ctypes.c_int32 * 5) * 3),
                ("group_mb", ctypes.c_int32), ("pair_fields", ctypes.c_int32), ("alternate_order", ctypes.c_int32),
                ("features_form", ctypes.c_int32), ("pdl", ctypes.c_int32), ("fuse", ctypes.c_int32),
                ("tma", ctypes.c_int32), ("overlap", ctypes.c_int32)]

    def as_tuple(self):
        """(lanes, tile_x, tile_y) of scale 0 (the throughput-form space)."""
        return (self.lanes_per_pixel, self.tile_x, self.tile_y)

    def scale_variants(self):
        """[(lanes, slots, tile_x, tile_y, min_ctas)] of scales 0..3; all zero = derived."""
        return [(self.lanes_per_pixel, self.slots, self.tile_x, self.tile_y, self.min_ctas)] + \
            [tuple(self.coarse[k][j] for j in range(5)) for k in range(3)]


TILES = ((64, 16), (32, 16), (64, 8), (32, 8), (16, 8), (8, 8))
TUNING_SPACE = [(l, tx, ty) for l in (1, 2, 4) for (tx, ty) in TILES]


def _lat_fits(group: int, tx: int, ty: int) -> bool:
    # one group of lanes per colour-0 slot of the (tx + 1) x (ty + 1) region
    return (group * ((tx + 2) // 2) * (ty + 1) + 31) // 32 * 32 <= 1024


# Every variant (lanes, slots, tile_x, tile_y, min_ctas) of the iteration
# kernel: the throughput form (slots 0), its one-lane tiles also with a
# register budget for min_ctas resident CTAs per SM, and the latency form
# (slots 1 or 4) on every tile whose region fits one cell per lane group in
# 1024 threads.
VARIANT_SPACE = [(l, 0, tx, ty, 0) for l in (1, 2, 4) for (tx, ty) in TILES] + \
    [(1, 0, 64, 16, 2), (1, 0, 32, 16, 3), (1, 0, 32, 16, 4), (1, 0, 32, 8, 6), (1, 0, 32, 8, 7), (1, 0, 32, 8, 8),
     (1, 0, 16, 8, 12)] + \
    [(l, c, tx, ty, 0) for (l, c) in ((1, 1), (2, 1), (4, 1), (1, 4), (2, 4), (4, 4)) for (tx, ty) in TILES
     if _lat_fits(l * c, tx, ty)]

# Scale-0 variants that also exist with TMA-staged reference records
# (sff_tuning.tma).
TMA_SPACE = [(1, 0, 32, 16, 0), (1, 0, 32, 16, 3), (1, 0, 32, 8, 0), (1, 0, 32, 8, 7)]

# Variants that also exist in the fused form (all iterations of a coarse
# scale in one cooperative launch: sff_tuning.fuse).
FUSED_SPACE = [(1, 0, 32, 16, 0), (1, 0, 32, 16, 4), (1, 0, 32, 8, 0), (1, 0, 32, 8, 7), (2, 0, 32, 8, 0),
               (1, 1, 32, 16, 0), (1, 1, 32, 8, 0), (1, 1, 16, 8, 0), (1, 1, 8, 8, 0), (2, 1, 32, 8, 0),
               (2, 1, 16, 8, 0), (2, 1, 8, 8, 0), (1, 4, 16, 8, 0), (1, 4, 8, 8, 0), (2, 4, 8, 8, 0)]


class QuadDesc(ctypes.Structure):
    """sff_quad of include/sff.h."""
    _fields_ = [("rgb", ctypes.c_void_p * 4), ("pitch_bytes", ctypes.c_int32), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("seed", ctypes.c_uint64), ("pyramid", ctypes.c_void_p * 4),
                ("fwd", ctypes.c_void_p), ("fwd_cost", ctypes.c_void_p), ("inv", ctypes.c_void_p),
                ("inv_cost", ctypes.c_void_p), ("keep", ctypes.c_void_p), ("cerr", ctypes.c_void_p),
                ("seeds", ctypes.c_void_p), ("capacity", ctypes.c_int32), ("count", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


MAX_BATCH = 32


class InterpParams(ctypes.Structure):
    """sff_interp_params: neighbourhood sizes, weight kernel and camera (Sec. 3.2)."""
    _fields_ = [("k_geo", ctypes.c_int32), ("k_motion", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("dist_unit", ctypes.c_double), ("focal", ctypes.c_double), ("baseline", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


class SgmParams(ctypes.Structure):
    """sff_sgm_params: disparity range and penalties of the disparity fill."""
    _fields_ = [("max_disp", ctypes.c_int32), ("p1", ctypes.c_int32), ("p2", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    """sff_kernel_time of include/sff.h."""
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int32), ("units", ctypes.c_int32),
                ("total_ms", ctypes.c_double)]


def profile_enable(on: bool = True) -> None:
    """Bracket every library kernel launch with CUDA events (sff_profile_enable)."""
    _check(lib().sff_profile_enable(1 if on else 0), "sff_profile_enable")


def profile_collect(with_units: bool = False) -> dict:
    """{kernel name: (launches, total ms)} of the launches recorded since
    enabling; with_units: (launches, total ms, work units), the units being
    iterations for the iteration kernel (a fused scale is one launch of all
    its iterations) and launches for the others."""
    cap = 64
    buf = (KernelTime * cap)()
    n = ctypes.c_int32(0)
    _check(lib().sff_profile_collect(buf, cap, ctypes.byref(n)), "sff_profile_collect")
    if with_units:
        return {buf[k].name.decode(): (buf[k].launches, buf[k].total_ms, buf[k].units)
                for k in range(min(n.value, cap))}
    return {buf[k].name.decode(): (buf[k].launches, buf[k].total_ms) for k in range(min(n.value, cap))}


# sff_seed of include/sff.h
SEED_DTYPE = np.dtype([("x", "<i2"), ("y", "<i2"), ("u", "<i2"), ("v", "<i2"), ("d0", "<i2"), ("d1", "<i2"),
                       ("cost", "<i4"), ("cerr", "u1"), ("kind", "u1"), ("pad", "u1", (2,))])
assert SEED_DTYPE.itemsize == 20


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """Loads libsff.so; raises SffError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SffError(f"{LIB_PATH} is missing: build it with paper_1710_10096_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        PP = ctypes.POINTER(Params)
        L.sff_default_params.argtypes = [PP]
        L.sff_default_params.restype = i32
        L.sff_pyramid_bytes.argtypes = [i32, i32, PP]
        L.sff_pyramid_bytes.restype = sz
        L.sff_workspace_bytes.argtypes = [i32, i32, PP]
        L.sff_workspace_bytes.restype = sz
        L.sff_features.argtypes = [P, i32, i32, i32, PP, P, P, sz, P]
        L.sff_features.restype = i32
        L.sff_features_tc.argtypes = [P, i32, i32, i32, PP, P, P, sz, P]
        L.sff_features_tc.restype = i32
        L.sff_features_pairs.argtypes = [P, i32, i32, i32, PP, P, P, sz, P]
        L.sff_features_pairs.restype = i32
        L.sff_match_views.argtypes = [P, P, P, P, i32, i32, i32, ctypes.c_uint64, PP, P, P, P, sz, P]
        L.sff_match_views.restype = i32
        L.sff_match_views_sequential.argtypes = [P, P, P, P, i32, i32, i32, ctypes.c_uint64, PP, P, P, P, sz, P]
        L.sff_match_views_sequential.restype = i32
        L.sff_match_quad.argtypes = [P, P, P, P, i32, i32, ctypes.c_uint64, PP, P, P, P, P, P, sz, P]
        L.sff_match_quad.restype = i32
        L.sff_match_quad_tuned.argtypes = [P, P, P, P, i32, i32, ctypes.c_uint64, PP, ctypes.POINTER(Tuning), P, P, P,
                                           P, P, sz, P]
        L.sff_match_quad_tuned.restype = i32
        L.sff_default_tuning.argtypes = [ctypes.POINTER(Tuning)]
        L.sff_default_tuning.restype = i32
        L.sff_tuning_supported.argtypes = [ctypes.POINTER(Tuning)]
        L.sff_tuning_supported.restype = i32
        L.sff_quad_workspace_bytes.argtypes = [i32, i32, PP]
        L.sff_quad_workspace_bytes.restype = sz
        L.sff_run_batch.argtypes = [ctypes.POINTER(QuadDesc), i32, PP, ctypes.POINTER(Tuning), P]
        L.sff_run_batch.restype = i32
        L.sff_consistency_filter.argtypes = [P, P, P, P, i32, i32, PP, P, P, P, sz, P]
        L.sff_consistency_filter.restype = i32
        L.sff_emit_seeds.argtypes = [P, P, P, P, i32, i32, P, i32, P, P, sz, P]
        L.sff_emit_seeds.restype = i32
        L.sff_emit_seeds_noalloc.argtypes = [P, P, P, P, i32, i32, P, i32, P, P]
        L.sff_emit_seeds_noalloc.restype = i32
        L.sff_sift_workspace_bytes.argtypes = [i32, i32]
        L.sff_sift_workspace_bytes.restype = sz
        L.sff_sift_features.argtypes = [ctypes.POINTER(P), i32, i32, i32, PP, ctypes.POINTER(P), P, sz, P]
        L.sff_sift_features.restype = i32
        L.sff_match_views_sift.argtypes = [P, P, P, P, P, P, P, P, i32, i32, i32, ctypes.c_uint64, PP, P, P, P, sz, P]
        L.sff_match_views_sift.restype = i32
        SP = ctypes.POINTER(SgmParams)
        L.sff_default_sgm_params.argtypes = [SP]
        L.sff_default_sgm_params.restype = i32
        L.sff_sgm_workspace_bytes.argtypes = [i32, i32, SP]
        L.sff_sgm_workspace_bytes.restype = sz
        L.sff_sgm.argtypes = [P, P, i32, i32, i32, SP, P, P, sz, P]
        L.sff_sgm.restype = i32
        L.sff_emit_seeds_geo.argtypes = [P, P, P, P, P, i32, i32, PP, P, i32, P, P, sz, P]
        L.sff_emit_seeds_geo.restype = i32
        IP = ctypes.POINTER(InterpParams)
        L.sff_default_interp_params.argtypes = [i32, i32, ctypes.c_double, ctypes.c_double, IP]
        L.sff_default_interp_params.restype = i32
        L.sff_interp_workspace_bytes.argtypes = [i32, i32, i32]
        L.sff_interp_workspace_bytes.restype = sz
        L.sff_interpolate.argtypes = [P, P, i32, i32, i32, IP, P, P, sz, P]
        L.sff_interpolate.restype = i32
        L.sff_interp_status.argtypes = [P, i32, i32, i32, ctypes.POINTER(ctypes.c_uint32)]
        L.sff_interp_status.restype = i32
        L.sff_profile_enable.argtypes = [i32]
        L.sff_profile_enable.restype = i32
        L.sff_profile_collect.argtypes = [ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
        L.sff_profile_collect.restype = i32
        L.sff_device_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint32), i32]
        L.sff_device_timeouts.restype = i32
        L.sff_device_drain_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
        L.sff_device_drain_timeouts.restype = i32
        L.sff_device_status.argtypes = [ctypes.c_void_p, i32]
        L.sff_device_status.restype = i32
        L.sff_debug_knn_withhold.argtypes = [i32, i32]
        L.sff_debug_knn_withhold.restype = i32
        L.sff_debug_barrier_withhold.argtypes = [i32, i32]
        L.sff_debug_barrier_withhold.restype = i32
        L.sff_int_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        L.sff_int_peak.restype = i32
        L.sff_status_string.argtypes = [i32]
        L.sff_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise SffError(f"{what}: {lib().sff_status_string(status).decode()} ({status})", status)


def default_params(**overrides) -> Params:
    p = Params()
    _check(lib().sff_default_params(ctypes.byref(p)), "sff_default_params")
    for k, v in overrides.items():
        setattr(p, k, int(v))
    return p


def pyramid_bytes(width: int, height: int, params: Params = None) -> int:
    params = params or default_params()
    return lib().sff_pyramid_bytes(width, height, ctypes.byref(params))


def workspace_bytes(width: int, height: int, params: Params = None) -> int:
    params = params or default_params()
    return lib().sff_workspace_bytes(width, height, ctypes.byref(params))


def _ptr(t) -> int:
    return t.data_ptr()


def _stream(stream) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def _buf(t, nbytes: int, what: str):
    """A buffer the library writes or reads densely: a contiguous CUDA tensor
    of at least `nbytes` bytes.  The C ABI sees only its pointer, so the size
    is checked here."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    if _nbytes(t) < nbytes:
        raise ValueError(f"{what}: {_nbytes(t)} bytes, at least {nbytes} needed")
    return t.data_ptr()


def _image(t, what: str, shape=None) -> int:
    """An H x W x 3 uint8 CUDA image whose rows may be padded (pixels packed);
    returns its row pitch in bytes."""
    if not getattr(t, "is_cuda", False) or t.dim() != 3 or t.shape[2] != 3 or t.element_size() != 1:
        raise ValueError(f"{what}: expected a CUDA uint8 [H, W, 3] tensor")
    if t.stride(2) != 1 or t.stride(1) != 3 or t.stride(0) < 3 * t.shape[1]:
        raise ValueError(f"{what}: pixels must be packed, rows at a pitch of at least 3 W bytes")
    if shape is not None and tuple(t.shape[:2]) != tuple(shape):
        raise ValueError(f"{what}: shape {tuple(t.shape[:2])}, expected {tuple(shape)}")
    return t.stride(0)


def _pyramids(pyrs, width: int, height: int, params: Params, what: str):
    pb = pyramid_bytes(width, height, params)
    if pb == 0:
        raise SffError(f"{what}: invalid size {width}x{height} or parameters")
    return [_buf(t, pb, f"{what} pyramid") for t in pyrs]


def features(rgb, pyramid, workspace, params: Params = None, stream=None, tensor: bool = False,
             form: int = None) -> None:
    """sff_features on a [H, W, 3] uint8 CUDA tensor (rows may be padded), in
    the transform form `form` (0: sff_features, separable; 1: sff_features_tc;
    2: sff_features_pairs; all give the same pyramid); tensor=True is form 1."""
    params = params or default_params()
    if form is None:
        form = 1 if tensor else 0
    name = {0: "sff_features", 1: "sff_features_tc", 2: "sff_features_pairs"}[int(form)]
    pitch = _image(rgb, name + " rgb")
    h, w = rgb.shape[0], rgb.shape[1]
    (pp,) = _pyramids([pyramid], w, h, params, name)
    _check(getattr(lib(), name)(_ptr(rgb), w, h, pitch, ctypes.byref(params), pp, _buf(workspace, 0, "workspace"),
                                _nbytes(workspace), _stream(stream)), name)


def match_views(pyr_ref, pyr_temporal, pyr_stereo, pyr_cross, width: int, height: int, mirror: int, seed: int,
                field, cost, workspace, params: Params = None, stream=None) -> None:
    """sff_match_views; field [H, W, 4] int16 and cost [H, W] int32 CUDA tensors."""
    params = params or default_params()
    pr = _pyramids([pyr_ref, pyr_temporal, pyr_stereo, pyr_cross], width, height, params, "sff_match_views")
    _check(lib().sff_match_views(*pr, width, height, int(mirror), int(seed) & (2 ** 64 - 1), ctypes.byref(params),
                                 _buf(field, 8 * width * height, "field"), _buf(cost, 4 * width * height, "cost"),
                                 _buf(workspace, 0, "workspace"), _nbytes(workspace), _stream(stream)),
           "sff_match_views")


def match_views_sequential(pyr_ref, pyr_temporal, pyr_stereo, pyr_cross, width: int, height: int, mirror: int,
                           seed: int, field, cost, workspace, params: Params = None, stream=None) -> None:
    """sff_match_views_sequential: the paper's in-place raster sweeps instead of
    checkerboard half-steps (slow; reproduces the sequential scan exactly)."""
    params = params or default_params()
    pr = _pyramids([pyr_ref, pyr_temporal, pyr_stereo, pyr_cross], width, height, params,
                   "sff_match_views_sequential")
    _check(lib().sff_match_views_sequential(*pr, width, height, int(mirror), int(seed) & (2 ** 64 - 1),
                                            ctypes.byref(params), _buf(field, 8 * width * height, "field"),
                                            _buf(cost, 4 * width * height, "cost"), _buf(workspace, 0, "workspace"),
                                            _nbytes(workspace), _stream(stream)),
           "sff_match_views_sequential")


def match_quad(pyr_l0, pyr_r0, pyr_l1, pyr_r1, width: int, height: int, seed: int, fwd, fwd_cost, inv, inv_cost,
               workspace, params: Params = None, stream=None) -> None:
    """sff_match_quad: forward field of L0 and inverse field of R1 in shared launches."""
    params = params or default_params()
    n = width * height
    pr = _pyramids([pyr_l0, pyr_r0, pyr_l1, pyr_r1], width, height, params, "sff_match_quad")
    _check(lib().sff_match_quad(*pr, width, height, int(seed) & (2 ** 64 - 1), ctypes.byref(params),
                                _buf(fwd, 8 * n, "fwd"), _buf(fwd_cost, 4 * n, "fwd_cost"), _buf(inv, 8 * n, "inv"),
                                _buf(inv_cost, 4 * n, "inv_cost"), _buf(workspace, 0, "workspace"),
                                _nbytes(workspace), _stream(stream)),
           "sff_match_quad")


def default_tuning() -> Tuning:
    t = Tuning()
    _check(lib().sff_default_tuning(ctypes.byref(t)), "sff_default_tuning")
    return t


def make_tuning(lanes: int, tile_x: int, tile_y: int, slots: int = 0, coarse=None, group_mb: int = 0,
                pair_fields: int = 0, min_ctas: int = 0, alternate_order: int = 0, features_form: int = 0,
                pdl: int = 0, fuse: int = 0, tma: int = 0, overlap: int = 1) -> Tuning:
    """sff_tuning: scale 0 (lanes, slots, tile, min_ctas); coarse = [(lanes, slots, tile_x,
    tile_y[, min_ctas])] for scales 1.. (None or all-zero entries: derived from the grid
    size); group_mb: the batch's scale-0 sweep schedule (0: all quads in every launch);
    pair_fields: a quad's two fields alternate tile by tile in each launch; alternate_order,
    pdl, fuse: per-scale bits of the launch schedule; tma: scale-0 reference records staged by
    tensor copies; overlap: the finer scales' features on a second stream while the coarse
    scales match (see sff_tuning)."""
    t = Tuning(lanes, tile_x, tile_y, slots, min_ctas)
    t.group_mb = int(group_mb)
    t.pair_fields = int(pair_fields)
    t.alternate_order = int(alternate_order)
    t.features_form = int(features_form)
    t.pdl = int(pdl)
    t.fuse = int(fuse)
    t.tma = int(tma)
    t.overlap = int(overlap)
    for k, v in enumerate(coarse or []):
        v = tuple(v) + (0,) * (5 - len(v))
        for j in range(5):
            t.coarse[k][j] = int(v[j])
    if not lib().sff_tuning_supported(ctypes.byref(t)):
        raise SffError(f"unsupported tuning {(lanes, tile_x, tile_y, slots, coarse)}")
    return t


def match_quad_tuned(pyr_l0, pyr_r0, pyr_l1, pyr_r1, width: int, height: int, seed: int, tuning: Tuning, fwd,
                     fwd_cost, inv, inv_cost, workspace, params: Params = None, stream=None) -> None:
    """sff_match_quad_tuned: match_quad with an explicit work distribution."""
    params = params or default_params()
    n = width * height
    pr = _pyramids([pyr_l0, pyr_r0, pyr_l1, pyr_r1], width, height, params, "sff_match_quad_tuned")
    _check(lib().sff_match_quad_tuned(*pr, width, height, int(seed) & (2 ** 64 - 1), ctypes.byref(params),
                                      ctypes.byref(tuning), _buf(fwd, 8 * n, "fwd"), _buf(fwd_cost, 4 * n, "fwd_cost"),
                                      _buf(inv, 8 * n, "inv"), _buf(inv_cost, 4 * n, "inv_cost"),
                                      _buf(workspace, 0, "workspace"), _nbytes(workspace), _stream(stream)),
           "sff_match_quad_tuned")


def split_pyramid(pyr, width: int, height: int, params: Params = None):
    """(features [S, H, W, 48] int8, norms [S, H, W] int32) of a pyramid buffer.
    Scales with grid stride 2^s < WHOLE_RECORD_STRIDE hold their 48-byte
    records as three planes of 16-byte chunks ([chunk][y][x]), coarser scales
    as whole records ([y][x][48]); the features are returned as records (a copy)."""
    import torch
    params = params or default_params()
    S, np_ = params.num_scales, width * height
    blocks = pyr[:S * np_ * FEATURE_BYTES].view(torch.int8).view(S, np_ * FEATURE_BYTES)
    scales = []
    for s in range(S):
        if (1 << s) < WHOLE_RECORD_STRIDE:
            scales.append(blocks[s].view(3, height, width, FEATURE_BYTES // 3).permute(1, 2, 0, 3)
                          .reshape(height, width, FEATURE_BYTES))
        else:
            scales.append(blocks[s].view(height, width, FEATURE_BYTES))
    feat = torch.stack(scales)
    norm = pyr[S * np_ * FEATURE_BYTES:S * np_ * (FEATURE_BYTES + 4)].view(torch.int32).view(S, height, width)
    return feat, norm


def consistency_filter(fwd, fwd_cost, inv, inv_cost, keep, cerr, workspace, params: Params = None,
                       stream=None) -> None:
    """fwd, inv: CUDA int16 [H, W, 4]; costs: int32 [H, W]; keep, cerr: uint8 [H, W], overwritten."""
    params = params or default_params()
    h, w = fwd.shape[0], fwd.shape[1]
    n = w * h
    _check(lib().sff_consistency_filter(_buf(fwd, 8 * n, "fwd"), _buf(fwd_cost, 4 * n, "fwd_cost"),
                                        _buf(inv, 8 * n, "inv"), _buf(inv_cost, 4 * n, "inv_cost"), w, h,
                                        ctypes.byref(params), _buf(keep, n, "keep"), _buf(cerr, n, "cerr"),
                                        _buf(workspace, 0, "workspace"), _nbytes(workspace), _stream(stream)),
           "sff_consistency_filter")


def emit_seeds(fwd, fwd_cost, keep, cerr, seeds, capacity: int, count, workspace, stream=None) -> None:
    """seeds: CUDA uint8 tensor of >= 20 * capacity bytes; count: CUDA int32 tensor [1]."""
    h, w = fwd.shape[0], fwd.shape[1]
    n = w * h
    _check(lib().sff_emit_seeds(_buf(fwd, 8 * n, "fwd"), _buf(fwd_cost, 4 * n, "fwd_cost"), _buf(keep, n, "keep"),
                                _buf(cerr, n, "cerr"), w, h, _buf(seeds, 20 * capacity, "seeds"), capacity,
                                _buf(count, 4, "count"), _buf(workspace, 0, "workspace"), _nbytes(workspace),
                                _stream(stream)), "sff_emit_seeds")


def sift_workspace_bytes(width: int, height: int) -> int:
    return lib().sff_sift_workspace_bytes(width, height)


def sift_features(images, phis, workspace, params: Params = None, stream=None) -> None:
    """images: 4 CUDA uint8 [H, W, 3] with one row pitch; phis: 4 CUDA float32
    [S, H, W, 4], overwritten with phi of Eq. 1's SIFT-PCA features."""
    params = params or default_params()
    if len(images) != 4 or len(phis) != 4:
        raise ValueError("sff_sift_features: four images and four phi buffers")
    h, w = images[0].shape[0], images[0].shape[1]
    pitch = _image(images[0], "sff_sift_features image")
    if any(_image(im, "sff_sift_features image", (h, w)) != pitch for im in images):
        raise ValueError("sff_sift_features: the four images must share one row pitch")
    ip = (ctypes.c_void_p * 4)(*[_ptr(im) for im in images])
    pp = (ctypes.c_void_p * 4)(*[_buf(p, 16 * params.num_scales * w * h, "phi") for p in phis])
    _check(lib().sff_sift_features(ip, pitch, w, h, ctypes.byref(params), pp, _buf(workspace, 0, "workspace"),
                                   _nbytes(workspace), _stream(stream)), "sff_sift_features")


def match_views_sift(pyr_ref, pyr_temporal, pyr_stereo, pyr_cross, phi_ref, phi_temporal, phi_stereo, phi_cross,
                     width: int, height: int, mirror: int, seed: int, field, cost, workspace,
                     params: Params = None, stream=None) -> None:
    """One field with the cost of Eq. 1 on SIFT-PCA features; cost holds float bit patterns."""
    params = params or default_params()
    pr = _pyramids([pyr_ref, pyr_temporal, pyr_stereo, pyr_cross], width, height, params, "sff_match_views_sift")
    ph = [_buf(p, 16 * params.num_scales * width * height, "phi") for p in (phi_ref, phi_temporal, phi_stereo,
                                                                          phi_cross)]
    _check(lib().sff_match_views_sift(*pr, *ph, width, height, int(mirror), int(seed) & (2 ** 64 - 1),
                                      ctypes.byref(params), _buf(field, 8 * width * height, "field"),
                                      _buf(cost, 4 * width * height, "cost"), _buf(workspace, 0, "workspace"),
                                      _nbytes(workspace), _stream(stream)),
           "sff_match_views_sift")


def default_sgm_params(**overrides) -> SgmParams:
    p = SgmParams()
    _check(lib().sff_default_sgm_params(ctypes.byref(p)), "sff_default_sgm_params")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def sgm_workspace_bytes(width: int, height: int, params: SgmParams = None) -> int:
    return lib().sff_sgm_workspace_bytes(width, height, ctypes.byref(params or default_sgm_params()))


def sgm(left, right, disp, workspace, params: SgmParams = None, stream=None) -> None:
    """left, right: CUDA uint8 [H, W, 3] (L0, R0, same row pitch); disp: CUDA int16 [H, W]."""
    h, w = left.shape[0], left.shape[1]
    pitch = _image(left, "sff_sgm left")
    if _image(right, "sff_sgm right", (h, w)) != pitch:
        raise ValueError("sff_sgm: left and right must share one row pitch")
    _check(lib().sff_sgm(_ptr(left), _ptr(right), pitch, w, h, ctypes.byref(params or default_sgm_params()),
                         _buf(disp, 2 * w * h, "disp"), _buf(workspace, 0, "workspace"), _nbytes(workspace),
                         _stream(stream)), "sff_sgm")


def emit_seeds_geo(fwd, fwd_cost, keep, cerr, sgm_disp, seeds, capacity: int, count, workspace,
                   params: Params = None, stream=None) -> None:
    """As emit_seeds, with disparity-only seeds (kind 1) where d0 agrees with sgm_disp."""
    h, w = fwd.shape[0], fwd.shape[1]
    n = w * h
    _check(lib().sff_emit_seeds_geo(_buf(fwd, 8 * n, "fwd"), _buf(fwd_cost, 4 * n, "fwd_cost"), _buf(keep, n, "keep"),
                                    _buf(cerr, n, "cerr"), _buf(sgm_disp, 2 * n, "sgm_disp"), w, h,
                                    ctypes.byref(params or default_params()), _buf(seeds, 20 * capacity, "seeds"),
                                    capacity, _buf(count, 4, "count"), _buf(workspace, 0, "workspace"),
                                    _nbytes(workspace), _stream(stream)), "sff_emit_seeds_geo")


def default_interp_params(width: int, height: int, focal: float, baseline: float, **overrides) -> InterpParams:
    p = InterpParams()
    _check(lib().sff_default_interp_params(width, height, float(focal), float(baseline), ctypes.byref(p)),
           "sff_default_interp_params")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def interp_workspace_bytes(width: int, height: int, capacity: int) -> int:
    return lib().sff_interp_workspace_bytes(width, height, capacity)


def interpolate(seeds, count, capacity: int, width: int, height: int, params: InterpParams, field, workspace,
                stream=None) -> None:
    """seeds: CUDA tensor of >= 20 * capacity bytes; count: CUDA int32 [1];
    field: CUDA float32 [H][W][4] (u, v, d0, d1), overwritten."""
    _check(lib().sff_interpolate(_buf(seeds, 20 * capacity, "seeds"), _buf(count, 4, "count"), capacity, width,
                                 height, ctypes.byref(params), _buf(field, 16 * width * height, "field"),
                                 _buf(workspace, 0, "workspace"), _nbytes(workspace), _stream(stream)),
           "sff_interpolate")


def interp_status(workspace, width: int, height: int, capacity: int) -> int:
    """Error bits the last interpolate on `workspace` set (0: none)."""
    v = ctypes.c_uint32(0)
    _check(lib().sff_interp_status(_ptr(workspace), width, height, capacity, ctypes.byref(v)), "sff_interp_status")
    return v.value


def device_timeouts(reset: bool = False) -> int:
    """Device-side bounded waits that gave up (0 in any valid run)."""
    v = ctypes.c_uint32(0)
    _check(lib().sff_device_timeouts(ctypes.byref(v), 1 if reset else 0), "sff_device_timeouts")
    return v.value


def device_drain_timeouts() -> int:
    """Of the waits that gave up, the drains of work already issued (0 unless
    the hardware did not finish issued copies or MMAs within ten wait limits)."""
    v = ctypes.c_uint32(0)
    _check(lib().sff_device_drain_timeouts(ctypes.byref(v)), "sff_device_drain_timeouts")
    return v.value


def device_status(stream=None, reset: bool = False) -> int:
    """sff_device_status: waits for `stream`, returns OK, ERR_TIMEOUT (a
    bounded device wait gave up: results invalid), ERR_CAPACITY (a seed
    buffer was too small) or ERR_CUDA."""
    return int(lib().sff_device_status(_stream(stream), 1 if reset else 0))


def check_device_status(stream=None, what: str = "device status") -> None:
    """Raises SffError (with .status) unless device_status(stream, reset=True) is OK."""
    _check(device_status(stream, reset=True), what)


def int_peak(kind: str = "dp4a", stream=None) -> float:
    """Measured integer throughput (ops/s) of the current device: "dp4a" or "imad"."""
    v = ctypes.c_double(0.0)
    _check(lib().sff_int_peak({"dp4a": 0, "imad": 1}[kind], ctypes.byref(v), _stream(stream)), "sff_int_peak")
    return v.value


def debug_knn_withhold(step: int, wait_limit_us: int = 0) -> None:
    """sff_debug_knn_withhold: failure injection for tests (step -1: off)."""
    _check(lib().sff_debug_knn_withhold(int(step), int(wait_limit_us)), "sff_debug_knn_withhold")


def debug_barrier_withhold(barrier: int, wait_limit_us: int = 0) -> None:
    """sff_debug_barrier_withhold: failure injection for tests (barrier -1: off)."""
    _check(lib().sff_debug_barrier_withhold(int(barrier), int(wait_limit_us)), "sff_debug_barrier_withhold")


def seed_capacity(width: int, height: int) -> int:
    return ((width + 2) // 3) * ((height + 2) // 3)


def seeds_to_numpy(seeds_bytes: np.ndarray, count: int) -> np.ndarray:
    return np.frombuffer(np.ascontiguousarray(seeds_bytes).tobytes(), SEED_DTYPE)[:count].copy()


def quad_workspace_bytes(width: int, height: int, params: Params = None) -> int:
    params = params or default_params()
    return lib().sff_quad_workspace_bytes(width, height, ctypes.byref(params))


class QuadBuffers:
    """Device buffers of one W x H quad: input images, pyramids, fields,
    filter masks, seeds and scratch."""

    def __init__(self, width: int, height: int, params: Params, device, per_call_workspaces: int = 0):
        import torch
        self.width, self.height = int(width), int(height)
        w, h = self.width, self.height
        pb = pyramid_bytes(w, h, params)
        qb = quad_workspace_bytes(w, h, params)
        if pb == 0 or qb == 0:
            raise SffError(f"invalid size {w}x{h} or parameters")
        u8 = dict(dtype=torch.uint8, device=device)
        self.dev_in = torch.empty((4, h, w, 3), **u8)  # L0, R0, L1, R1
        self.pyr = [torch.empty(pb, **u8) for _ in range(4)]
        self.workspace = torch.empty(qb, **u8)
        self.fwd = torch.empty((h, w, 4), dtype=torch.int16, device=device)
        self.inv = torch.empty((h, w, 4), dtype=torch.int16, device=device)
        self.fwd_cost = torch.empty((h, w), dtype=torch.int32, device=device)
        self.inv_cost = torch.empty((h, w), dtype=torch.int32, device=device)
        self.keep = torch.empty((h, w), **u8)
        self.cerr = torch.empty((h, w), **u8)
        self.capacity = seed_capacity(w, h)
        self.seeds = torch.empty(20 * self.capacity, **u8)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)

    def desc(self, images, seed: int) -> QuadDesc:
        imgs = list(images) if images is not None else list(self.dev_in.unbind(0))
        pitch = imgs[0].stride(0)
        for im in imgs:
            if _image(im, "quad image", (self.height, self.width)) != pitch:
                raise ValueError("quad images: the four images must share one row pitch")
        d = QuadDesc()
        for k in range(4):
            d.rgb[k] = imgs[k].data_ptr()
            d.pyramid[k] = self.pyr[k].data_ptr()
        d.pitch_bytes, d.width, d.height, d.seed = pitch, self.width, self.height, int(seed) & (2 ** 64 - 1)
        d.fwd, d.fwd_cost = self.fwd.data_ptr(), self.fwd_cost.data_ptr()
        d.inv, d.inv_cost = self.inv.data_ptr(), self.inv_cost.data_ptr()
        d.keep, d.cerr = self.keep.data_ptr(), self.cerr.data_ptr()
        d.seeds, d.capacity, d.count = self.seeds.data_ptr(), self.capacity, self.count.data_ptr()
        d.workspace, d.workspace_bytes = self.workspace.data_ptr(), _nbytes(self.workspace)
        return d

    def seeds_numpy(self) -> np.ndarray:
        n = int(self.count.item())
        return seeds_to_numpy(self.seeds.cpu().numpy(), min(n, self.capacity))


def run_batch(descs, params: Params = None, tuning: Tuning = None, stream=None) -> None:
    """sff_run_batch on a list of QuadDesc (at most MAX_BATCH)."""
    params = params or default_params()
    arr = (QuadDesc * len(descs))(*descs)
    _check(lib().sff_run_batch(arr, len(descs), ctypes.byref(params), ctypes.byref(tuning) if tuning else None,
                               _stream(stream)), "sff_run_batch")


class BatchMatcher:
    """Buffers for a fixed list of quad sizes; run() matches all of them in
    shared launches (sff_run_batch), capture() records that into a CUDA graph.

    streams > 1 splits the quads into that many groups (quad k in group
    k % streams, so every group holds a mix of the sizes) and runs one
    sff_run_batch per group, each on its own stream forked from the caller's
    and joined back: the latency-bound phases of one group (the coarse scales,
    the K-NN) then run beside the throughput-bound ones of another.  Every
    quad's outputs are the same whatever the grouping."""

    def __init__(self, sizes, params: Params = None, device="cuda", tuning: Tuning = None, streams: int = 1):
        import torch
        if not 1 <= len(sizes) <= MAX_BATCH:
            raise SffError(f"a batch holds 1..{MAX_BATCH} quads")
        self.params = params or default_params()
        self.tuning = tuning or default_tuning()
        self.device = torch.device(device)
        self.quads = [QuadBuffers(w, h, self.params, self.device) for (w, h) in sizes]
        self.streams = streams
        self._group_streams = []

    @property
    def streams(self) -> int:
        return self._streams

    @streams.setter
    def streams(self, n: int) -> None:
        if not 1 <= int(n) <= len(self.quads):
            raise SffError(f"streams must be 1..{len(self.quads)}")
        self._streams = int(n)

    def load(self, k: int, L0, R0, L1, R1) -> None:
        """Copy host (or device) images of quad k into its device input buffer."""
        import torch
        for j, im in enumerate((L0, R0, L1, R1)):
            self.quads[k].dev_in[j].copy_(torch.as_tensor(np.ascontiguousarray(im)) if isinstance(im, np.ndarray) else im,
                                          non_blocking=True)

    def run(self, seeds, stream=None) -> None:
        descs = [q.desc(None, sd) for q, sd in zip(self.quads, seeds)]
        if self._streams == 1:
            run_batch(descs, self.params, self.tuning, stream)
            return
        import torch
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        while len(self._group_streams) < self._streams:
            self._group_streams.append(torch.cuda.Stream(device=self.device))
        groups = self._group_streams[:self._streams]
        for gs in groups:
            gs.wait_stream(main)
        for g, gs in enumerate(groups):
            run_batch(descs[g::self._streams], self.params, self.tuning, gs)
        for gs in groups:
            main.wait_stream(gs)

    def capture(self, seeds):
        """A CUDA graph replaying run(seeds) on the current input buffers."""
        import torch
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.run(seeds, s)  # warm-up outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(seeds, torch.cuda.current_stream(self.device))
        return g


class QuadMatcher:
    """One W x H quad.  run() works on CUDA images already on the device;
    run_host() takes host arrays, copies them in, runs the stage and copies
    the seeds back.

    mode "batch" runs the whole stage with sff_run_batch (one quad); mode
    "calls" runs the four calls sff_features x4, sff_match_quad,
    sff_consistency_filter and sff_emit_seeds.  Both give identical results.
    """

    def __init__(self, width: int, height: int, params: Params = None, device="cuda", tuning: Tuning = None,
                 mode: str = "batch"):
        import torch
        self.params = params or default_params()
        self.tuning = tuning or default_tuning()
        self.device = torch.device(device)
        self.mode = mode
        self.buf = QuadBuffers(width, height, self.params, self.device)
        b = self.buf
        self.width, self.height = b.width, b.height
        self.pyr, self.fwd, self.inv, self.fwd_cost, self.inv_cost = b.pyr, b.fwd, b.inv, b.fwd_cost, b.inv_cost
        self.keep, self.cerr, self.seeds, self.count, self.capacity = b.keep, b.cerr, b.seeds, b.count, b.capacity
        self.workspace = b.workspace
        self._host_in = None

    def run(self, L0, R0, L1, R1, seed: int, stream=None):
        """All four calls on device images; returns (seeds bytes tensor, count tensor)."""
        p = self.params
        if self.mode == "batch":
            run_batch([self.buf.desc((L0, R0, L1, R1), seed)], p, self.tuning, stream)
            return self.seeds, self.count
        ws = workspace_bytes(self.width, self.height, p)
        w = self.workspace[:ws]
        for img, pyr in zip((L0, R0, L1, R1), self.pyr):
            features(img, pyr, w, p, stream, form=self.tuning.features_form)
        pL0, pR0, pL1, pR1 = self.pyr
        match_quad_tuned(pL0, pR0, pL1, pR1, self.width, self.height, seed, self.tuning, self.fwd, self.fwd_cost,
                         self.inv, self.inv_cost, w, p, stream)
        consistency_filter(self.fwd, self.fwd_cost, self.inv, self.inv_cost, self.keep, self.cerr, w, p, stream)
        emit_seeds(self.fwd, self.fwd_cost, self.keep, self.cerr, self.seeds, self.capacity, self.count, w, stream)
        return self.seeds, self.count

    def run_host(self, L0, R0, L1, R1, seed: int, stream=None) -> np.ndarray:
        """Host images in, host seeds out (pinned staging, copies on `stream`)."""
        import torch
        h, w = self.height, self.width
        if self._host_in is None:
            self._host_in = torch.empty((4, h, w, 3), dtype=torch.uint8).pin_memory()
            self._host_seeds = torch.empty(20 * self.capacity, dtype=torch.uint8).pin_memory()
            self._host_count = torch.empty(1, dtype=torch.int32).pin_memory()
        for k, img in enumerate((L0, R0, L1, R1)):
            self._host_in[k].copy_(torch.as_tensor(np.ascontiguousarray(img)))
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.stream(s):
            self.buf.dev_in.copy_(self._host_in, non_blocking=True)
            self.run(*self.buf.dev_in.unbind(0), seed=seed, stream=s)
            self._host_count.copy_(self.count, non_blocking=True)
            self._host_seeds.copy_(self.seeds, non_blocking=True)
        s.synchronize()
        n = int(self._host_count.item())
        return seeds_to_numpy(self._host_seeds[:20 * min(n, self.capacity)].numpy(), n)

    @property
    def dev_in(self):
        return self.buf.dev_in

    @property
    def h2d_bytes(self) -> int:
        return 4 * self.height * self.width * 3

    @property
    def d2h_bytes(self) -> int:
        return 4 + 20 * self.capacity
