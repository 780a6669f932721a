"""Seeded synthetic stereo quads for the four-view matching stage.

This module is the one piece of code shared by the CUDA path's tests and
benchmarks and by the CPU oracle's: it draws the inputs.  It contains no part
of the matching method (no features, no costs, no propagation) -- only a small
ray caster over textured planes and boxes, with camera and object motion, that
produces the four RGB uint8 images of a rectified stereo quad

    L0 = I_l^0,  R0 = I_r^0,  L1 = I_l^1,  R1 = I_r^1          (Sec. 3)

and the ground truth scene flow u = (u, v, d0, d1) of every L0 pixel together
with an occlusion mask.  The scene families follow the shapes of the paper's
evaluation data (KITTI driving scenes, Sec. 5, Tab. 1-2; MPI Sintel movie
scenes, Tab. 3), which are not available here:

* ``planes``  -- a few textured planes, static camera, two rigid movers.
* ``driving`` -- ground plane, boxes and planes, forward ego-motion with yaw,
                 three independent rigid movers.
* ``movie``   -- surfaces deformed by a Gaussian-RBF displacement field plus
                 two rigid movers, large motion, sensor noise, per-view gain.
* ``shift``   -- a textured image shifted by constant integer offsets: the
                 ground truth is exact and identical at every pixel.

Everything is float64 numpy driven by ``numpy.random.default_rng(seed)``, so a
given (family, size, seed) gives the same quad on every run of one machine.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["Quad", "make_quad", "make_shift_quad", "CONFIG_SIZES", "ground_truth", "scene_ranges", "SEED_RECORD",
           "sparse_seeds"]

# (family, width, height) of the named workloads.
CONFIG_SIZES = {
    "planes_256x80": ("planes", 256, 80),
    "driving_1242x375": ("driving", 1242, 375),
    "movie_1024x436": ("movie", 1024, 436),
    "planes_640x192": ("planes", 640, 192),
    "planes_512x160": ("planes", 512, 160),
}


@dataclasses.dataclass
class Quad:
    L0: np.ndarray  # [H, W, 3] uint8, left image at t0 (reference)
    R0: np.ndarray  # right image at t0
    L1: np.ndarray  # left image at t1
    R1: np.ndarray  # right image at t1
    gt: np.ndarray  # [H, W, 4] float64 ground truth (u, v, d0, d1) per L0 pixel
    occluded: np.ndarray  # [H, W] bool: not visible in all four views
    focal: float
    baseline: float
    out_of_frame: np.ndarray = None  # [H, W] bool: of those, leaving the frame of a view

    def ranges(self) -> dict:
        """Measured ranges of the scene (scene_ranges)."""
        return scene_ranges(self.gt, self.occluded, self.out_of_frame)

    @property
    def width(self) -> int:
        return self.L0.shape[1]

    @property
    def height(self) -> int:
        return self.L0.shape[0]

    def images(self):
        return self.L0, self.R0, self.L1, self.R1


# ----------------------------------------------------------------------------
# geometry helpers


def _rot(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * k + (1 - np.cos(angle)) * (k @ k)


@dataclasses.dataclass
class _Surface:
    c: np.ndarray  # centre at t0 (world)
    a1: np.ndarray  # in-plane unit axis 1 at t0
    a2: np.ndarray  # in-plane unit axis 2 at t0
    e1: float  # half extent along a1
    e2: float  # half extent along a2
    R: np.ndarray  # rigid rotation t0 -> t1 about c
    t: np.ndarray  # rigid translation t0 -> t1
    lattice: list  # per channel, per octave: (cell, grid array)
    tint: np.ndarray  # 3 channel tints
    deform: object = None  # callable (s, t) -> (ds, dt) at t1, or None

    def pose(self, time: int):
        if time == 0:
            return self.c, self.a1, self.a2
        return self.c + self.t, self.R @ self.a1, self.R @ self.a2


def _make_texture(rng, e1, e2, cell, octaves=3, margin=0.25):
    """Value-noise lattices (one per channel and octave) covering the surface."""
    lat = []
    for _ch in range(3):
        per = []
        for o in range(octaves):
            h = cell * (2.0 ** o)
            n1 = int(np.ceil(2 * e1 * (1 + margin) / h)) + 3
            n2 = int(np.ceil(2 * e2 * (1 + margin) / h)) + 3
            per.append((h, rng.random((n1, n2))))
        lat.append(per)
    return lat


def _noise(lattice_ch, s, t, e1, e2, margin=0.25):
    val = np.zeros_like(s)
    wsum = 0.0
    for o, (h, g) in enumerate(lattice_ch):
        fs = (s + e1 * (1 + margin)) / h
        ft = (t + e2 * (1 + margin)) / h
        i0 = np.clip(np.floor(fs).astype(np.int64), 0, g.shape[0] - 2)
        j0 = np.clip(np.floor(ft).astype(np.int64), 0, g.shape[1] - 2)
        a = np.clip(fs - i0, 0.0, 1.0)
        b = np.clip(ft - j0, 0.0, 1.0)
        a = a * a * (3 - 2 * a)
        b = b * b * (3 - 2 * b)
        v = (g[i0, j0] * (1 - a) * (1 - b) + g[i0 + 1, j0] * a * (1 - b)
             + g[i0, j0 + 1] * (1 - a) * b + g[i0 + 1, j0 + 1] * a * b)
        w = 0.5 ** o
        val += w * v
        wsum += w
    return val / wsum


@dataclasses.dataclass
class _Camera:
    C: np.ndarray  # centre of the left camera (world)
    R: np.ndarray  # camera -> world rotation of the left camera
    f: float
    cx: float
    cy: float
    B: float

    def centre(self, right: bool):
        return self.C + (self.R @ np.array([self.B, 0.0, 0.0]) if right else 0.0)

    def project(self, X: np.ndarray, right: bool):
        """X [..., 3] world -> (x, y, Z) in the chosen camera."""
        Xc = (X - self.C) @ self.R  # world -> left camera coordinates
        if right:
            Xc = Xc - np.array([self.B, 0.0, 0.0])
        Z = Xc[..., 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            x = self.f * Xc[..., 0] / Z + self.cx
            y = self.f * Xc[..., 1] / Z + self.cy
        return x, y, Z


def _surface_bbox(S: _Surface, cam: _Camera, right: bool, time: int, pad: float):
    """Screen-space bounding box of a surface, or None when it may cross the camera plane."""
    c, a1, a2 = S.pose(time)
    g = 1.3 if S.deform is not None else 1.0
    corners = np.array([c + g * (i * S.e1 * a1 + j * S.e2 * a2) for i in (-1, 1) for j in (-1, 1)])
    x, y, Z = cam.project(corners, right)
    if np.any(Z <= 1e-3):
        return None
    return x.min() - pad, x.max() + pad, y.min() - pad, y.max() + pad


def _raycast(surfs, cam: _Camera, right: bool, time: int, xs, ys):
    """Nearest surface hit for rays through image positions (xs, ys).

    Returns (surface id or -1, depth Z in the camera, intrinsic s, intrinsic t).
    The depth equals the ray parameter because the camera-frame direction has
    unit z component.
    """
    xs = np.asarray(xs, np.float64)
    ys = np.asarray(ys, np.float64)
    dxc = (xs - cam.cx) / cam.f
    dyc = (ys - cam.cy) / cam.f
    R = cam.R
    dw = [R[i, 0] * dxc + R[i, 1] * dyc + R[i, 2] for i in range(3)]
    o = cam.centre(right)
    best = np.full(xs.shape, np.inf)
    sid = np.full(xs.shape, -1, np.int64)
    bs = np.zeros(xs.shape)
    bt = np.zeros(xs.shape)
    for j, S in enumerate(surfs):
        bb = _surface_bbox(S, cam, right, time, pad=2.0)
        if bb is None:
            idx = np.nonzero(np.ones(xs.shape, bool).ravel())[0]
        else:
            m = (xs >= bb[0]) & (xs <= bb[1]) & (ys >= bb[2]) & (ys <= bb[3])
            idx = np.nonzero(m.ravel())[0]
        if idx.size == 0:
            continue
        c, a1, a2 = S.pose(time)
        n = np.cross(a1, a2)
        d0, d1, d2 = (dw[0].ravel()[idx], dw[1].ravel()[idx], dw[2].ravel()[idx])
        den = d0 * n[0] + d1 * n[1] + d2 * n[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = ((c - o) @ n) / den
        with np.errstate(invalid="ignore", over="ignore"):
            r0 = o[0] - c[0] + lam * d0
            r1 = o[1] - c[1] + lam * d1
            r2 = o[2] - c[2] + lam * d2
            s = r0 * a1[0] + r1 * a1[1] + r2 * a1[2]
            t = r0 * a2[0] + r1 * a2[1] + r2 * a2[2]
        if S.deform is not None and time == 1:
            # intrinsic coordinates: invert p = q + D(q) by fixed-point iteration
            qs, qt = s.copy(), t.copy()
            for _ in range(6):
                ds, dt = S.deform(qs, qt)
                qs, qt = s - ds, t - dt
            s, t = qs, qt
        flat_best = best.ravel()
        ok = (lam > 1e-6) & (np.abs(s) <= S.e1) & (np.abs(t) <= S.e2) & (lam < flat_best[idx])
        sel = idx[ok]
        best.ravel()[sel] = lam[ok]
        sid.ravel()[sel] = j
        bs.ravel()[sel] = s[ok]
        bt.ravel()[sel] = t[ok]
    return sid, best, bs, bt


def _world_point(S: _Surface, time: int, s, t):
    c, a1, a2 = S.pose(time)
    if S.deform is not None and time == 1:
        ds, dt = S.deform(s, t)
        s, t = s + ds, t + dt
    return c + s[..., None] * a1 + t[..., None] * a2


def _shade(surfs, sid, s, t):
    out = np.zeros(sid.shape + (3,))
    for j, S in enumerate(surfs):
        m = sid == j
        if not m.any():
            continue
        for ch in range(3):
            nz = _noise(S.lattice[ch], s[m], t[m], S.e1, S.e2)
            out[..., ch][m] = S.tint[ch] * (0.25 + 0.75 * nz)
    return out


def _render(surfs, cam, right, time, W, H, ss=2):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    acc = np.zeros((H, W, 3))
    offs = [(-0.25, -0.25), (0.25, -0.25), (-0.25, 0.25), (0.25, 0.25)] if ss == 2 else [(0.0, 0.0)]
    for ox, oy in offs:
        sid, _, s, t = _raycast(surfs, cam, right, time, xs + ox, ys + oy)
        acc += _shade(surfs, sid, s, t)
    return acc / len(offs)


def _ground_truth(surfs, cam0: _Camera, cam1: _Camera, W, H):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    sid, Z0, s, t = _raycast(surfs, cam0, False, 0, xs, ys)
    X0 = np.zeros((H, W, 3))
    X1 = np.zeros((H, W, 3))
    for j, S in enumerate(surfs):
        m = sid == j
        X0[m] = _world_point(S, 0, s[m], t[m])
        X1[m] = _world_point(S, 1, s[m], t[m])
    x1, y1, Z1 = cam1.project(X1, False)
    f, B = cam0.f, cam0.B
    gt = np.stack([x1 - xs, y1 - ys, f * B / Z0, f * B / Z1], -1)
    # visibility of the same surface point in R0, L1 and R1
    vis = sid >= 0
    oof = np.zeros((H, W), bool)
    for cam, right, time, X in ((cam0, True, 0, X0), (cam1, False, 1, X1), (cam1, True, 1, X1)):
        px, py, Zp = cam.project(X, right)
        inside = (px >= -0.5) & (px <= W - 0.5) & (py >= -0.5) & (py <= H - 0.5) & (Zp > 0)
        sid2, Z2, _, _ = _raycast(surfs, cam, right, time, np.where(inside, px, 0.0), np.where(inside, py, 0.0))
        same = (sid2 == sid) & (np.abs(Z2 - Zp) <= 0.01 * np.abs(Zp) + 1e-3)
        vis &= inside & same
        oof |= (sid >= 0) & ~inside
    return gt, ~vis, oof


def scene_ranges(gt: np.ndarray, occluded: np.ndarray, out_of_frame: np.ndarray = None) -> dict:
    """Ranges of a scene's ground truth over its visible pixels: disparity d0,
    flow u and v, the fraction of pixels hidden by another surface in some
    view while inside every frame ("occluded"), and of pixels leaving a
    view's frame ("out_of_frame")."""
    vis = ~occluded
    r = {"d0_px": [round(float(gt[..., 2][vis].min()), 1), round(float(gt[..., 2][vis].max()), 1)],
         "u_px": [round(float(gt[..., 0][vis].min()), 1), round(float(gt[..., 0][vis].max()), 1)],
         "v_px": [round(float(gt[..., 1][vis].min()), 1), round(float(gt[..., 1][vis].max()), 1)]}
    if out_of_frame is not None:
        r["occluded"] = round(float((occluded & ~out_of_frame).mean()), 4)
        r["out_of_frame"] = round(float(out_of_frame.mean()), 4)
    else:
        r["not_visible"] = round(float(occluded.mean()), 4)
    return r


def _finish(img, rng, noise_sigma=0.0, gain=1.0):
    img = img * gain
    if noise_sigma > 0:
        img = img + rng.normal(0.0, noise_sigma, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def _rand_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _box_faces(centre, size, yaw):
    """Three visible-ish faces of an axis-aligned box (front, left, right) as planes."""
    R = _rot(np.array([0.0, 1.0, 0.0]), yaw)
    w, h, d = size
    faces = []
    # front face (normal -z), side faces (normal +-x), top face (normal -y)
    faces.append((centre + R @ np.array([0, 0, -d / 2]), R @ np.array([1.0, 0, 0]), R @ np.array([0, 1.0, 0]), w / 2, h / 2))
    faces.append((centre + R @ np.array([-w / 2, 0, 0]), R @ np.array([0, 0, 1.0]), R @ np.array([0, 1.0, 0]), d / 2, h / 2))
    faces.append((centre + R @ np.array([w / 2, 0, 0]), R @ np.array([0, 0, 1.0]), R @ np.array([0, 1.0, 0]), d / 2, h / 2))
    faces.append((centre + R @ np.array([0, -h / 2, 0]), R @ np.array([1.0, 0, 0]), R @ np.array([0, 0, 1.0]), w / 2, d / 2))
    return faces


def _surface(rng, c, a1, a2, e1, e2, depth, f, R=None, t=None, deform=None, px_per_cell=3.0):
    cell = max(depth / f * px_per_cell, 1e-3)
    return _Surface(c=np.asarray(c, float), a1=np.asarray(a1, float), a2=np.asarray(a2, float), e1=e1, e2=e2,
                    R=np.eye(3) if R is None else R, t=np.zeros(3) if t is None else np.asarray(t, float),
                    lattice=_make_texture(rng, e1, e2, cell), tint=90.0 + 165.0 * rng.random(3),
                    deform=deform)


# ----------------------------------------------------------------------------
# scene families


def _scene_planes(rng, W, H):
    f = 200.0 * W / 256.0
    B = 0.54
    surfs = []
    # back wall far enough that it fills the view
    zb = 25.0 + 10 * rng.random()
    half_w = zb * (W / 2 + 40) / f
    half_h = zb * (H / 2 + 40) / f
    surfs.append(_surface(rng, [0, 0, zb], [1, 0, 0], [0, 1, 0], half_w, half_h, zb, f))
    movers = {1, 2}
    for k in range(5):
        # the two movers near the camera, so that their 0.2-0.3 m translation
        # gives flows up to ~16 px
        z = 3.8 + 1.7 * rng.random() if k in movers else 3.6 + 14.0 * rng.random()
        x = (rng.random() - 0.5) * z * W / f * 0.8
        y = (rng.random() - 0.5) * z * H / f * 0.6
        n = np.array([rng.normal() * 0.3, rng.normal() * 0.2, -1.0])
        n /= np.linalg.norm(n)
        a1 = np.cross([0, 1.0, 0], n)
        a1 /= np.linalg.norm(a1)
        a2 = np.cross(n, a1)
        e1 = z * W / f * (0.08 + 0.12 * rng.random())
        e2 = z * H / f * (0.12 + 0.2 * rng.random())
        R = None
        t = None
        if k in movers:
            R = _rot(_rand_unit(rng), np.deg2rad(2.0) * rng.random())
            ang = 2 * np.pi * rng.random()
            t = np.array([np.cos(ang), 0.5 * np.sin(ang), 0.3 * rng.normal()])
            t *= (0.2 + 0.1 * rng.random()) / np.linalg.norm(t)
        surfs.append(_surface(rng, [x, y, z], a1, a2, e1, e2, z, f, R, t))
    cam0 = _Camera(C=np.zeros(3), R=np.eye(3), f=f, cx=(W - 1) / 2, cy=(H - 1) / 2, B=B)
    # small ego-motion so that static surfaces also move in the image
    cam1 = _Camera(C=np.array([0.08 * rng.normal(), 0.03 * rng.normal(), 0.2 * rng.random()]), R=np.eye(3),
                   f=f, cx=cam0.cx, cy=cam0.cy, B=B)
    return surfs, cam0, cam1, dict(noise=0.0, gain=(1.0, 1.0, 1.0, 1.0))


def _scene_driving(rng, W, H):
    f = 721.0 * W / 1242.0
    B = 0.54
    surfs = []
    # ground plane y = +1.65 (y points down), extending far ahead
    surfs.append(_surface(rng, [0, 1.65, 60.0], [1, 0, 0], [0, 0, 1], 60.0, 58.0, 15.0, f, px_per_cell=6.0))
    # far back wall ("sky" / distant buildings): disparities below 1 px
    zb = 450.0
    surfs.append(_surface(rng, [0, -10.0, zb], [1, 0, 0], [0, 1, 0], zb * (W / 2 + 200) / f, zb * (H / 2 + 60) / f, zb, f))
    # side walls (building facades)
    for side in (-1, 1):
        x = side * (7.0 + 3.0 * rng.random())
        surfs.append(_surface(rng, [x, -2.0, 55.0], [0, 0, 1], [0, 1, 0], 50.0, 3.7, 20.0, f))
    # a car parked on the left 3.04-3.08 m ahead: disparities up to 128 px,
    # and flows near -150 px under the forward ego-motion where its face
    # stays inside all four frames
    zc = 3.04 + 0.04 * rng.random()
    car = np.array([1.7, 1.4, 3.8])
    for (c, a1, a2, e1, e2) in _box_faces(np.array([-(1.45 + 0.25 * rng.random()), 1.65 - 0.7, zc + car[2] / 2]),
                                          car, 0.0):
        surfs.append(_surface(rng, c, a1, a2, e1, e2, zc, f))
    # static boxes: with the ground, the back wall, the two facades, the car
    # and the three movers, 20 planes / boxes
    n_obj = 0
    while n_obj < 12:
        z = 4.5 + 20.0 * rng.random()
        x = (rng.random() - 0.5) * 12.0
        if n_obj < 3:  # posts and signs: thin and tall
            size = np.array([0.3 + 0.4 * rng.random(), 2.5 + 2.0 * rng.random(), 0.3 + 0.4 * rng.random()])
        else:
            size = np.array([0.6 + 2.0 * rng.random(), 0.8 + 2.0 * rng.random(), 0.6 + 3.0 * rng.random()])
        y = 1.65 - size[1] / 2
        if z - size[2] / 2 < 4.0:
            continue
        for (c, a1, a2, e1, e2) in _box_faces(np.array([x, y, z]), size, rng.normal() * 0.3):
            surfs.append(_surface(rng, c, a1, a2, e1, e2, z, f))
        n_obj += 1
    # three independently moving boxes
    for _ in range(3):
        z = 7.0 + 20.0 * rng.random()
        x = (rng.random() - 0.5) * 10.0
        size = np.array([1.6, 1.4, 3.5])
        R = _rot(np.array([0, 1.0, 0]), np.deg2rad(4.0) * (rng.random() - 0.5))
        t = np.array([(rng.random() - 0.5) * 1.0, 0.0, 0.5 + 1.5 * rng.random()])
        for (c, a1, a2, e1, e2) in _box_faces(np.array([x, 1.65 - 0.7, z]), size, rng.normal() * 0.2):
            S = _surface(rng, c, a1, a2, e1, e2, z, f)
            # rotation about the box centre: express as rotation about face centre + translation
            box_c = np.array([x, 1.65 - 0.7, z])
            S.R = R
            S.t = (R @ (c - box_c) + box_c + t) - c
            surfs.append(S)
    cam0 = _Camera(C=np.zeros(3), R=np.eye(3), f=f, cx=(W - 1) / 2, cy=(H - 1) / 2, B=B)
    yaw = np.deg2rad(1.0) * (1 if rng.random() < 0.5 else -1)
    R1 = _rot(np.array([0, 1.0, 0]), yaw)
    cam1 = _Camera(C=np.array([0.0, 0.0, 1.0]), R=R1, f=f, cx=cam0.cx, cy=cam0.cy, B=B)
    return surfs, cam0, cam1, dict(noise=0.0, gain=(1.0, 1.0, 1.0, 1.0))


def _rbf_field(rng, centres=16, amp=0.6, sigma=1.5):
    cs = rng.normal(size=(centres, 2)) * 2.0
    ws = rng.normal(size=(centres, 2)) * amp

    def deform(s, t):
        ds = np.zeros_like(s)
        dt = np.zeros_like(t)
        for (c0, c1), (w0, w1) in zip(cs, ws):
            g = np.exp(-((s - c0) ** 2 + (t - c1) ** 2) / (2 * sigma * sigma))
            ds += w0 * g
            dt += w1 * g
        return ds, dt

    return deform


def _scene_movie(rng, W, H):
    f = 500.0 * W / 1024.0
    B = 0.2
    surfs = []
    zb = 30.0
    surfs.append(_surface(rng, [0, 0, zb], [1, 0, 0], [0, 1, 0], zb * (W / 2 + 260) / f, zb * (H / 2 + 260) / f, zb, f))
    for k in range(11):
        z = 2.0 + 14.0 * rng.random()
        x = (rng.random() - 0.5) * z * W / f * 0.9
        y = (rng.random() - 0.5) * z * H / f * 0.7
        n = np.array([rng.normal() * 0.4, rng.normal() * 0.3, -1.0])
        n /= np.linalg.norm(n)
        a1 = np.cross([0, 1.0, 0], n)
        a1 /= np.linalg.norm(a1)
        a2 = np.cross(n, a1)
        e1 = z * W / f * (0.06 + 0.12 * rng.random())
        e2 = z * H / f * (0.1 + 0.2 * rng.random())
        R = _rot(_rand_unit(rng), np.deg2rad(3.0) * rng.random())
        t = _rand_unit(rng) * 0.25 * rng.random()
        surfs.append(_surface(rng, [x, y, z], a1, a2, e1, e2, z, f, R, t,
                              deform=_rbf_field(rng, amp=0.04 * z, sigma=0.5 * max(e1, e2))))
    # two fast rigid movers (105-155 px sideways before the camera's own motion)
    for _ in range(2):
        z = 3.0 + 4.0 * rng.random()
        x = (rng.random() - 0.5) * z * W / f * 0.5
        y = (rng.random() - 0.5) * z * H / f * 0.4
        e1 = z * W / f * 0.08
        e2 = z * H / f * 0.12
        R = _rot(_rand_unit(rng), np.deg2rad(5.0) * rng.random())
        lateral = (0.42 + 0.2 * rng.random()) * (1 if rng.random() < 0.5 else -1)
        t = np.array([lateral, (rng.random() - 0.5) * 0.8, -0.2 * rng.random()]) * z / f * 250
        surfs.append(_surface(rng, [x, y, z], [1, 0, 0], [0, 1, 0], e1, e2, z, f, R, t))
    cam0 = _Camera(C=np.zeros(3), R=np.eye(3), f=f, cx=(W - 1) / 2, cy=(H - 1) / 2, B=B)
    cam1 = _Camera(C=np.array([0.15, 0.0, 0.3]), R=_rot(np.array([0, 1.0, 0]), np.deg2rad(1.5)), f=f,
                   cx=cam0.cx, cy=cam0.cy, B=B)
    gains = tuple(0.9 + 0.2 * rng.random() for _ in range(4))
    return surfs, cam0, cam1, dict(noise=2.0, gain=gains)


_FAMILIES = {"planes": _scene_planes, "driving": _scene_driving, "movie": _scene_movie}


def make_quad(family: str, width: int, height: int, seed: int, supersample: int = 2,
              with_gt: bool = True) -> Quad:
    """Render one rectified stereo quad of the given scene family and size."""
    rng = np.random.default_rng(seed)
    surfs, cam0, cam1, extra = _FAMILIES[family](rng, width, height)
    imgs = []
    for k, (cam, right, time) in enumerate(((cam0, False, 0), (cam0, True, 0), (cam1, False, 1), (cam1, True, 1))):
        img = _render(surfs, cam, right, time, width, height, ss=supersample)
        imgs.append(_finish(img, rng, extra["noise"], extra["gain"][k]))
    L0, R0, L1, R1 = imgs
    if with_gt:
        gt, occ, oof = _ground_truth(surfs, cam0, cam1, width, height)
    else:
        gt, occ, oof = np.zeros((height, width, 4)), np.zeros((height, width), bool), None
    return Quad(L0, R0, L1, R1, gt, occ, cam0.f, cam0.B, oof)


def ground_truth(family: str, width: int, height: int, seed: int):
    """(gt [H, W, 4], occluded [H, W], focal, baseline) of the scene that
    make_quad(family, width, height, seed) renders, without rendering it."""
    rng = np.random.default_rng(seed)
    surfs, cam0, cam1, _ = _FAMILIES[family](rng, width, height)
    gt, occ, _ = _ground_truth(surfs, cam0, cam1, width, height)
    return gt, occ, cam0.f, cam0.B


# 20-byte seed record of the sparse matches (x, y, u, v, d0, d1, cost, cerr)
SEED_RECORD = np.dtype([("x", "<i2"), ("y", "<i2"), ("u", "<i2"), ("v", "<i2"), ("d0", "<i2"), ("d1", "<i2"),
                        ("cost", "<i4"), ("cerr", "u1"), ("kind", "u1"), ("pad", "u1", (2,))])


def sparse_seeds(gt: np.ndarray, occluded: np.ndarray, seed: int, keep: float = 0.6, noise: float = 0.0,
                 outliers: float = 0.0, block: int = 3) -> np.ndarray:
    """Synthetic sparse matches with the structure of the matching stage's
    output: at most one pixel per non-overlapping block x block cell
    (anchored at (0, 0)), in cell raster order.  Each cell draws a pixel
    uniformly inside it; a visible pixel is kept with probability `keep` and
    carries its ground-truth vector plus Gaussian noise of `noise` px, a
    fraction `outliers` of them a uniform random vector instead, rounded to
    integers with disparities >= 0.  cost and cerr are random."""
    rng = np.random.default_rng(seed)
    H, W = occluded.shape
    gbw, gbh = -(-W // block), -(-H // block)
    by, bx = np.mgrid[0:gbh, 0:gbw]
    x = np.minimum(W - 1, bx * block + rng.integers(0, block, bx.shape))
    y = np.minimum(H - 1, by * block + rng.integers(0, block, by.shape))
    take = (rng.random(bx.shape) < keep) & ~occluded[y, x]
    x, y = x[take], y[take]
    vec = gt[y, x] + noise * rng.standard_normal((len(x), 4))
    bad = rng.random(len(x)) < outliers
    span = np.array([W / 4, H / 8, W / 8, W / 8])
    vec[bad] = rng.uniform(-1, 1, (int(bad.sum()), 4)) * span
    vec = np.rint(vec)
    vec[:, 2:] = np.clip(np.abs(vec[:, 2:]), 0, 32767)
    vec = np.clip(vec, -32768, 32767)
    out = np.zeros(len(x), SEED_RECORD)
    out["x"], out["y"] = x, y
    out["u"], out["v"], out["d0"], out["d1"] = vec[:, 0], vec[:, 1], vec[:, 2], vec[:, 3]
    out["cost"] = rng.integers(0, 1 << 20, len(x))
    out["cerr"] = rng.integers(0, 4, len(x))
    return out


def make_named(name: str, seed: int, **kw) -> Quad:
    family, w, h = CONFIG_SIZES[name]
    return make_quad(family, w, h, seed, **kw)


def random_images(width: int, height: int, seed: int, n: int = 4):
    """Independent uniform-noise RGB images (no scene structure)."""
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 256, (height, width, 3), dtype=np.uint8) for _ in range(n)]


def make_shift_quad(width: int, height: int, seed: int, u: int, v: int, d0: int, d1: int,
                    cell: float = 3.0) -> Quad:
    """Quad whose views are integer shifts of one value-noise texture.

    L0(x, y) = T(x, y); R0(x, y) = T(x + d0, y); L1(x, y) = T(x - u, y - v);
    R1(x, y) = T(x - u + d1, y - v), so every L0 pixel has the exact scene
    flow (u, v, d0, d1).  Pixels whose correspondences leave an image are
    flagged occluded.
    """
    rng = np.random.default_rng(seed)
    m = 2 * (abs(u) + abs(v) + abs(d0) + abs(d1)) + 8
    Wt, Ht = width + 2 * m, height + 2 * m
    ys, xs = np.mgrid[0:Ht, 0:Wt].astype(np.float64)
    lat = _make_texture(rng, Wt / 2, Ht / 2, cell)
    tex = np.stack([_noise(lat[c], xs - Wt / 2, ys - Ht / 2, Wt / 2, Ht / 2) for c in range(3)], -1)
    tex = np.clip(np.rint(255 * (0.1 + 0.9 * tex)), 0, 255).astype(np.uint8)

    def crop(ox, oy):
        return np.ascontiguousarray(tex[m + oy:m + oy + height, m + ox:m + ox + width])

    L0 = crop(0, 0)
    R0 = crop(d0, 0)
    L1 = crop(-u, -v)
    R1 = crop(-u + d1, -v)
    gt = np.broadcast_to(np.array([u, v, d0, d1], float), (height, width, 4)).copy()
    ys, xs = np.mgrid[0:height, 0:width]
    occ = ~((xs - d0 >= 0) & (xs + u < width) & (xs + u >= 0) & (ys + v >= 0) & (ys + v < height)
            & (xs + u - d1 >= 0) & (xs + u - d1 < width))
    return Quad(L0, R0, L1, R1, gt, occ, 1.0, 1.0)
