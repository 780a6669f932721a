"""CPU oracle of the sparse four-view matching stage -- TEST INFRASTRUCTURE.

``sff_oracle.c`` states, in plain C loops, what the CUDA path must compute
(SceneFlowFields Sec. 3.1-3.2).  Only tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  It shares no code with the CUDA path.

This module compiles the C file with gcc (``build()``) and marshals numpy
arrays to it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sff_oracle.c")
_SRC_INTERP = os.path.join(_HERE, "sff_interp_oracle.c")
_SRC_SGM = os.path.join(_HERE, "sff_sgm_oracle.c")
_SRC_SIFT = os.path.join(_HERE, "sff_sift_oracle.c")
SOURCES = (_SRC, _SRC_INTERP, _SRC_SGM, _SRC_SIFT)
# SFF_ORACLE_LIB names a library built elsewhere by compile_library() (the
# planted-mistake tests load a deliberately broken copy this way)
_PREBUILT = os.environ.get("SFF_ORACLE_LIB")
_LIB = _PREBUILT or os.path.join(_HERE, "liboracle.so")
_lib = None

NF = 48
EMPTY = np.iinfo(np.int32).max
# order_mode bits: readings switched back towards the paper's own procedure
SEQUENTIAL_SCAN, KDTREE_INIT, SEQUENTIAL_RNG = 1, 2, 4


class Params(ctypes.Structure):
    """Method parameters (Sec. 5 values plus the stated readings)."""
    _fields_ = [("num_scales", ctypes.c_int32), ("iterations", ctypes.c_int32), ("tau_c", ctypes.c_int32),
                ("region_min", ctypes.c_int32), ("tau_r", ctypes.c_int32), ("quant_shift", ctypes.c_int32),
                ("knn_temporal", ctypes.c_int32), ("knn_epipolar", ctypes.c_int32), ("order_mode", ctypes.c_int32)]


def default_params(**over) -> Params:
    p = dict(num_scales=4, iterations=12, tau_c=1, region_min=150, tau_r=1, quant_shift=4,
             knn_temporal=4, knn_epipolar=2, order_mode=0)
    p.update(over)
    return Params(**p)


SEED_DTYPE = np.dtype([("x", "<i2"), ("y", "<i2"), ("u", "<i2"), ("v", "<i2"), ("d0", "<i2"), ("d1", "<i2"),
                       ("cost", "<i4"), ("cerr", "u1"), ("kind", "u1"), ("pad", "u1", (2,))])
assert SEED_DTYPE.itemsize == 20


def compile_library(sources, out: str) -> str:
    """gcc (OpenMP) of the given C files into the shared library `out`."""
    tmp = out + f".tmp{os.getpid()}"
    # no contracted multiply-adds: the float and double sums follow their
    # written order, as the CUDA path's do; explicit fma() calls stay (only
    # where a reading names them), correctly rounded
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-ffp-contract=off", *sources,
                           "-lm", "-o", tmp])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, OpenMP)."""
    if _PREBUILT:
        return _LIB
    newest = max(os.path.getmtime(p) for p in (*SOURCES, __file__))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        compile_library(SOURCES, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32 = ctypes.c_int32
        L.sffo_features.argtypes = [P, i32, i32, ctypes.POINTER(Params), P, P]
        L.sffo_smooth.argtypes = [P, i32, i32, i32, P]
        L.sffo_match_views.argtypes = [P, P, P, P, i32, i32, i32, ctypes.c_uint64, ctypes.POINTER(Params), P, P]
        L.sffo_consistency_check.argtypes = [P, P, P, P, i32, i32, ctypes.POINTER(Params), P, P]
        L.sffo_region_filter.argtypes = [P, P, i32, i32, ctypes.POINTER(Params), P]
        L.sffo_consistency_filter.argtypes = [P, P, P, P, i32, i32, ctypes.POINTER(Params), P, P]
        L.sffo_emit_seeds.argtypes = [P, P, P, P, i32, i32, P, i32]
        L.sffo_emit_seeds.restype = i32
        L.sffo_philox4x32_10.argtypes = [P, P, P]
        L.sffo_rs_offset.argtypes = [ctypes.c_uint32, i32]
        L.sffo_rs_offset.restype = i32
        L.sffo_wht8x8.argtypes = [P, P]
        L.sffo_walsh_matrix.argtypes = [P]
        L.sffo_coef_order.argtypes = [P, P]
        L.sffo_cost.argtypes = [P, P, P, P, i32, i32, i32, i32, i32, P]
        L.sffo_cost.restype = i32
        L.sffi_seed_models.argtypes = [P, i32, ctypes.POINTER(InterpParams), P, P, P]
        L.sffi_seed_models_of.argtypes = [P, i32, ctypes.POINTER(InterpParams), P, i32, P, P, P]
        L.sffi_interpolate_pixels.argtypes = [P, i32, ctypes.POINTER(InterpParams), P, P, P, P, i32, P, P]
        L.sffi_nearest.argtypes = [P, i32, i32, i32, i32, i32, P, P, P]
        L.sffi_set_threads.argtypes = [i32]
        L.sffs_set_threads.argtypes = [i32]
        L.sfft_set_threads.argtypes = [i32]
        L.sfft_orientation_bin.argtypes = [i32, i32]
        L.sfft_orientation_bin.restype = i32
        L.sfft_descriptors.argtypes = [P, i32, i32, i32, P]
        L.sfft_pca.argtypes = [P, ctypes.c_int64, P, P]
        L.sfft_project.argtypes = [P, ctypes.c_int64, P, P, P]
        L.sfft_phi.argtypes = [P, i32, i32, i32, P, P, P]
        L.sfft_cost.argtypes = [P, P, P, P, i32, i32, i32, i32, i32, i32, P]
        L.sfft_cost.restype = ctypes.c_float
        L.sffo_match_views_sift.argtypes = [P, P, P, P, P, P, P, P, i32, i32, i32, ctypes.c_uint64,
                                            ctypes.POINTER(Params), P, P]
        L.sffs_grey.argtypes = [P, i32, i32, i32, P]
        L.sffs_census.argtypes = [P, i32, i32, P]
        L.sffs_cost_volume.argtypes = [P, P, i32, i32, i32, P]
        L.sffs_path.argtypes = [P, i32, i32, i32, i32, i32, i32, i32, P]
        L.sffs_sgm_from_cost.argtypes = [P, i32, i32, i32, i32, i32, P]
        L.sffs_sgm.argtypes = [P, P, i32, i32, i32, ctypes.POINTER(SgmParams), P]
        L.sffs_emit_seeds_geo.argtypes = [P, P, P, P, P, i32, i32, i32, P, i32]
        L.sffs_emit_seeds_geo.restype = i32
        L.sffo_set_threads.argtypes = [i32]
        L.sffo_get_threads.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    lib().sffo_set_threads(int(n))
    lib().sffi_set_threads(int(n))
    lib().sffs_set_threads(int(n))
    lib().sfft_set_threads(int(n))


def get_threads() -> int:
    return lib().sffo_get_threads()


def smooth(img: np.ndarray, s: int) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    h, w, _ = img.shape
    out = np.empty_like(img)
    lib().sffo_smooth(_p(img), w, h, s, _p(out))
    return out


def features(img: np.ndarray, params: Params = None):
    """Features of one RGB uint8 image: (feat [S,H,W,48] int8, norm [S,H,W] int32)."""
    params = params or default_params()
    img = np.ascontiguousarray(img, np.uint8)
    h, w, _ = img.shape
    S = params.num_scales
    feat = np.empty((S, h, w, NF), np.int8)
    norm = np.empty((S, h, w), np.int32)
    lib().sffo_features(_p(img), w, h, ctypes.byref(params), _p(feat), _p(norm))
    return feat, norm


def match_views(f_ref, f_tmp, f_ste, f_crs, mirror: int, seed: int, params: Params = None):
    params = params or default_params()
    S, h, w, _ = f_ref.shape
    field = np.empty((h, w, 4), np.int16)
    cost = np.empty((h, w), np.int32)
    lib().sffo_match_views(_p(f_ref), _p(f_tmp), _p(f_ste), _p(f_crs), w, h, int(mirror), int(seed) & (2**64 - 1),
                           ctypes.byref(params), _p(field), _p(cost))
    return field, cost


def consistency_check(fwd, fwd_cost, inv, inv_cost, params: Params = None):
    params = params or default_params()
    h, w, _ = fwd.shape
    keep = np.empty((h, w), np.uint8)
    cerr = np.empty((h, w), np.uint8)
    lib().sffo_consistency_check(_p(fwd), _p(fwd_cost), _p(inv), _p(inv_cost), w, h, ctypes.byref(params),
                                 _p(keep), _p(cerr))
    return keep, cerr


def region_filter(fwd, fwd_cost, keep, params: Params = None):
    params = params or default_params()
    h, w, _ = fwd.shape
    keep = np.ascontiguousarray(keep, np.uint8).copy()
    lib().sffo_region_filter(_p(fwd), _p(fwd_cost), w, h, ctypes.byref(params), _p(keep))
    return keep


def consistency_filter(fwd, fwd_cost, inv, inv_cost, params: Params = None):
    params = params or default_params()
    h, w, _ = fwd.shape
    keep = np.empty((h, w), np.uint8)
    cerr = np.empty((h, w), np.uint8)
    lib().sffo_consistency_filter(_p(fwd), _p(fwd_cost), _p(inv), _p(inv_cost), w, h, ctypes.byref(params),
                                  _p(keep), _p(cerr))
    return keep, cerr


def emit_seeds(fwd, fwd_cost, keep, cerr):
    h, w, _ = fwd.shape
    cap = ((w + 2) // 3) * ((h + 2) // 3)
    out = np.zeros(cap, SEED_DTYPE)
    n = lib().sffo_emit_seeds(_p(fwd), _p(fwd_cost), _p(keep), _p(cerr), w, h, _p(out), cap)
    return out[:n]


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.empty(4, np.uint32)
    lib().sffo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def rs_offset(r: int, n: int) -> int:
    return lib().sffo_rs_offset(ctypes.c_uint32(r), n)


def wht8x8(patch) -> np.ndarray:
    p = np.ascontiguousarray(patch, np.int32).reshape(8, 8)
    out = np.empty((8, 8), np.int32)
    lib().sffo_wht8x8(_p(p), _p(out))
    return out


def walsh_matrix() -> np.ndarray:
    out = np.empty((8, 8), np.int32)
    lib().sffo_walsh_matrix(_p(out))
    return out


def coef_order():
    ky = np.empty(16, np.int32)
    kx = np.empty(16, np.int32)
    lib().sffo_coef_order(_p(ky), _p(kx))
    return ky, kx


def cost(f_ref, f_tmp, f_ste, f_crs, mirror, px, py, u):
    """Cost of vector u at pixel (px, py); features of ONE scale, [H,W,48]."""
    h, w, _ = f_ref.shape
    uu = np.ascontiguousarray(u, np.int16)
    return lib().sffo_cost(_p(f_ref), _p(f_tmp), _p(f_ste), _p(f_crs), w, h, int(mirror), px, py, _p(uu))


def run_quad(L0, R0, L1, R1, seed: int, params: Params = None):
    """The whole stage on one quad: features, forward and inverse fields,
    consistency + region filter, seeds.  Returns a dict of numpy arrays."""
    params = params or default_params()
    fL0, nL0 = features(L0, params)
    fR0, nR0 = features(R0, params)
    fL1, nL1 = features(L1, params)
    fR1, nR1 = features(R1, params)
    fwd, fwd_cost = match_views(fL0, fL1, fR0, fR1, 0, seed, params)
    inv, inv_cost = match_views(fR1, fR0, fL1, fL0, 1, seed, params)
    keep, cerr = consistency_filter(fwd, fwd_cost, inv, inv_cost, params)
    seeds = emit_seeds(fwd, fwd_cost, keep, cerr)
    return dict(feat=(fL0, fR0, fL1, fR1), norm=(nL0, nR0, nL1, nR1), fwd=fwd, fwd_cost=fwd_cost, inv=inv,
                inv_cost=inv_cost, keep=keep, cerr=cerr, seeds=seeds)


# ---------------------------------------------------------------------------
# Dense interpolation of the seeds (Sec. 3.2), sff_interp_oracle.c


class InterpParams(ctypes.Structure):
    """Neighbourhood sizes and kernel of Sec. 5 (160 / 80 seeds, alpha = 2.2),
    the distance unit of the Euclidean reading, and the pinhole camera."""
    _fields_ = [("k_geo", ctypes.c_int32), ("k_motion", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("dist_unit", ctypes.c_double), ("focal", ctypes.c_double), ("baseline", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


def interp_params(width: int, height: int, focal: float, baseline: float, **over) -> InterpParams:
    p = dict(k_geo=160, k_motion=80, alpha=2.2, dist_unit=20.0, focal=float(focal), baseline=float(baseline),
             cx=(width - 1) / 2.0, cy=(height - 1) / 2.0)
    p.update(over)
    return InterpParams(**p)


def seed_models(seeds, params: InterpParams, which=None):
    """(plane [n, 3], affine [n, 15] = [A | t] rows then the centre, motion
    neighbour count [n]) of every seed, or only of the seeds listed in
    `which` (the other rows stay zero)."""
    seeds = np.ascontiguousarray(seeds, SEED_DTYPE)
    n = len(seeds)
    plane = np.zeros((max(n, 1), 3), np.float64)
    affine = np.zeros((max(n, 1), 15), np.float64)
    motion = np.zeros(max(n, 1), np.int32)
    if which is None:
        lib().sffi_seed_models(_p(seeds) if n else None, n, ctypes.byref(params), _p(plane), _p(affine), _p(motion))
    else:
        which = np.ascontiguousarray(np.unique(np.asarray(which, np.int64)), np.int32)
        assert n == 0 or (which.min(initial=0) >= 0 and which.max(initial=0) < n)
        if len(which):
            lib().sffi_seed_models_of(_p(seeds), n, ctypes.byref(params), _p(which), len(which), _p(plane),
                                      _p(affine), _p(motion))
    return plane[:n], affine[:n], motion[:n]


def closest_seeds(seeds, pixels):
    """Closest seed [m] of the listed pixels [m, 2] (x, y), ties to the lower index."""
    seeds = np.ascontiguousarray(seeds, SEED_DTYPE)
    pixels = np.asarray(pixels, np.int64).reshape(-1, 2)
    return np.array([nearest_seeds(seeds, int(x), int(y), 1)[0][0] for x, y in pixels], np.int32)


def interpolate_pixels(seeds, params: InterpParams, pixels, models=None):
    """Interpolated (u, v, d0, d1) float32 [m, 4] and closest seed [m] at the
    listed pixels [m, 2] (x, y)."""
    seeds = np.ascontiguousarray(seeds, SEED_DTYPE)
    plane, affine, motion = models if models is not None else seed_models(seeds, params)
    pixels = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
    m = len(pixels)
    out = np.zeros((max(m, 1), 4), np.float32)
    closest = np.zeros(max(m, 1), np.int32)
    plane = np.ascontiguousarray(plane, np.float64)
    affine = np.ascontiguousarray(affine, np.float64)
    motion = np.ascontiguousarray(motion, np.int32)
    lib().sffi_interpolate_pixels(_p(seeds) if len(seeds) else None, len(seeds), ctypes.byref(params),
                                  _p(plane) if len(seeds) else None, _p(affine) if len(seeds) else None,
                                  _p(motion) if len(seeds) else None, _p(pixels), m, _p(out), _p(closest))
    return out[:m], closest[:m]


def interpolate(seeds, width: int, height: int, params: InterpParams):
    """Dense interpolated field float32 [H, W, 4] (u, v, d0, d1)."""
    ys, xs = np.mgrid[0:height, 0:width]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    out, _ = interpolate_pixels(seeds, params, pix)
    return out.reshape(height, width, 4)


def nearest_seeds(seeds, x: int, y: int, k: int, motion_only: bool = False):
    """Indices and squared distances of the k nearest seeds to (x, y)."""
    seeds = np.ascontiguousarray(seeds, SEED_DTYPE)
    idx = np.zeros(max(k, 1), np.int32)
    d2 = np.zeros(max(k, 1), np.int64)
    cnt = ctypes.c_int32(0)
    lib().sffi_nearest(_p(seeds), len(seeds), x, y, k, int(motion_only), _p(idx), _p(d2), ctypes.byref(cnt))
    return idx[:cnt.value], d2[:cnt.value]


# ---------------------------------------------------------------------------
# Disparity fill by semi-global matching (Sec. 3.1, last paragraph),
# sff_sgm_oracle.c


class SgmParams(ctypes.Structure):
    """Disparity range D and the SGM penalties P1, P2."""
    _fields_ = [("max_disp", ctypes.c_int32), ("p1", ctypes.c_int32), ("p2", ctypes.c_int32)]


def sgm_params(**over) -> SgmParams:
    p = dict(max_disp=128, p1=10, p2=120)
    p.update(over)
    return SgmParams(**p)


def grey(rgb):
    rgb = np.ascontiguousarray(rgb, np.uint8)
    h, w, _ = rgb.shape
    out = np.empty((h, w), np.uint8)
    lib().sffs_grey(_p(rgb), 3 * w, w, h, _p(out))
    return out


def census(grey_img):
    g = np.ascontiguousarray(grey_img, np.uint8)
    h, w = g.shape
    out = np.empty((h, w), np.uint64)
    lib().sffs_census(_p(g), w, h, _p(out))
    return out


def cost_volume(cl, cr, max_disp: int):
    cl = np.ascontiguousarray(cl, np.uint64)
    cr = np.ascontiguousarray(cr, np.uint64)
    h, w = cl.shape
    out = np.empty((h, w, max_disp), np.uint8)
    lib().sffs_cost_volume(_p(cl), _p(cr), w, h, max_disp, _p(out))
    return out


def path_costs(C, p1: int, p2: int, rx: int, ry: int):
    """L_r [H, W, D] uint16 of direction (rx, ry) over the cost volume C [H, W, D] uint8."""
    C = np.ascontiguousarray(C, np.uint8)
    h, w, d = C.shape
    out = np.empty((h, w, d), np.uint16)
    lib().sffs_path(_p(C), w, h, d, p1, p2, rx, ry, _p(out))
    return out


def sgm_from_cost(C, p1: int, p2: int):
    C = np.ascontiguousarray(C, np.uint8)
    h, w, d = C.shape
    out = np.empty((h, w), np.int16)
    lib().sffs_sgm_from_cost(_p(C), w, h, d, p1, p2, _p(out))
    return out


def sgm(left, right, params: SgmParams = None):
    """SGM disparity map int16 [H, W] of L0 (left) against R0 (right)."""
    params = params or sgm_params()
    left = np.ascontiguousarray(left, np.uint8)
    right = np.ascontiguousarray(right, np.uint8)
    h, w, _ = left.shape
    out = np.empty((h, w), np.int16)
    lib().sffs_sgm(_p(left), _p(right), 3 * w, w, h, ctypes.byref(params), _p(out))
    return out


def emit_seeds_geo(fwd, fwd_cost, keep, cerr, sgm_disp, tau_c: int = 1):
    """Seeds with the disparity fill: the jointly consistent seed of a 3x3
    block, else its best disparity-only pixel (kind 1)."""
    h, w, _ = fwd.shape
    cap = ((w + 2) // 3) * ((h + 2) // 3)
    out = np.zeros(cap, SEED_DTYPE)
    f = np.ascontiguousarray(fwd, np.int16)
    c = np.ascontiguousarray(fwd_cost, np.int32)
    k = np.ascontiguousarray(keep, np.uint8)
    e = np.ascontiguousarray(cerr, np.uint8)
    g = np.ascontiguousarray(sgm_disp, np.int16)
    n = lib().sffs_emit_seeds_geo(_p(f), _p(c), _p(k), _p(e), _p(g), w, h, tau_c, _p(out), cap)
    return out[:min(n, cap)]


# ---------------------------------------------------------------------------
# The paper's own matching cost (Eq. 1 with SIFT-PCA features),
# sff_sift_oracle.c


def orientation_bin(dx: int, dy: int) -> int:
    return lib().sfft_orientation_bin(int(dx), int(dy))


def sift_descriptors(rgb_s, s: int):
    """Descriptors uint8 [H, W, 128] of a scale-s smoothed image."""
    rgb_s = np.ascontiguousarray(rgb_s, np.uint8)
    h, w, _ = rgb_s.shape
    out = np.empty((h, w, 128), np.uint8)
    lib().sfft_descriptors(_p(rgb_s), w, h, s, _p(out))
    return out


def sift_pca(desc):
    d = np.ascontiguousarray(desc, np.uint8).reshape(-1, 128)
    mean = np.empty(128, np.float64)
    axes = np.empty((3, 128), np.float64)
    lib().sfft_pca(_p(d), len(d), _p(mean), _p(axes))
    return mean, axes


def sift_project(desc, mean, axes):
    d = np.ascontiguousarray(desc, np.uint8)
    flat = d.reshape(-1, 128)
    out = np.empty((len(flat), 4), np.float32)
    mean = np.ascontiguousarray(mean, np.float64)
    axes = np.ascontiguousarray(axes, np.float64)
    lib().sfft_project(_p(flat), len(flat), _p(mean), _p(axes), _p(out))
    return out.reshape(d.shape[:-1] + (4,))


def sift_phi(images, num_scales: int = 4):
    """phi float32 [4][S, H, W, 4] of the four images (L0, R0, L1, R1 or any
    order), with the principal axes (mean [128], axes [3, 128])."""
    imgs = [np.ascontiguousarray(im, np.uint8) for im in images]
    h, w, _ = imgs[0].shape
    phis = [np.empty((num_scales, h, w, 4), np.float32) for _ in range(4)]
    ip = (ctypes.c_void_p * 4)(*[im.ctypes.data for im in imgs])
    pp = (ctypes.c_void_p * 4)(*[ph.ctypes.data for ph in phis])
    mean = np.empty(128, np.float64)
    axes = np.empty((3, 128), np.float64)
    lib().sfft_phi(ip, w, h, num_scales, pp, _p(mean), _p(axes))
    return phis, mean, axes


def sift_cost(phi_ref, phi_tmp, phi_ste, phi_crs, n: int, mirror: int, px: int, py: int, u):
    """The float cost of vector u at (px, py); phi_* [H, W, 4] of one scale."""
    h, w, _ = phi_ref.shape
    a = [np.ascontiguousarray(x, np.float32) for x in (phi_ref, phi_tmp, phi_ste, phi_crs)]
    uu = np.ascontiguousarray(u, np.int16)
    return lib().sfft_cost(_p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), w, h, n, -1 if mirror else 1, px, py, _p(uu))


def match_views_sift(f_ref, f_tmp, f_ste, f_crs, phi_ref, phi_tmp, phi_ste, phi_crs, w: int, h: int, mirror: int,
                     seed: int, params: Params = None):
    """One field with the SIFT-PCA cost; costs as int32 bit patterns of the floats."""
    params = params or default_params()
    field = np.empty((h, w, 4), np.int16)
    cost = np.empty((h, w), np.int32)
    f = [np.ascontiguousarray(x, np.int8) for x in (f_ref, f_tmp, f_ste, f_crs)]
    ph = [np.ascontiguousarray(x, np.float32) for x in (phi_ref, phi_tmp, phi_ste, phi_crs)]
    lib().sffo_match_views_sift(*[_p(x) for x in f], *[_p(x) for x in ph], w, h, int(mirror),
                                int(seed) & (2 ** 64 - 1), ctypes.byref(params), _p(field), _p(cost))
    return field, cost
