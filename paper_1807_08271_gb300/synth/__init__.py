"""Seeded synthetic RGB-D inputs shaped like Kinect-class sequences.

This module produces INPUTS only: intensity images in [0, 1] and inverse-depth
maps (1/m, hole = 0) rendered by a CPU ray caster (``raycast.c``) from scenes of
textured boxes, plus ground-truth poses.  It contains none of the alignment or
fusion arithmetic, so both the CUDA path and the FP64 oracle can consume it.

Workload recipes (the paper evaluates on TUM RGB-D Kinect sequences, 640x480 at
30 Hz; these seeded renders stand in for them):

* ``make_pair``      one frame pair: 6 random textured planes/boxes 0.5-5 m in
                     front of the camera, relative pose with a rotation angle
                     ~U(0, 2 deg) about a uniform axis and a translation
                     ~U(0, 3 cm) in a uniform direction.
* ``make_room`` + ``make_trajectory`` + ``render_sequence``
                     a procedural room of textured boxes and a smooth (C2 cubic
                     B-spline) trajectory limited to 0.5 m/s and 30 deg/s.

Noise model (applied by ``apply_noise``): depth noise sigma_z = 1.5e-3 z^2,
intensity noise sigma = 2/255, 10 % i.i.d. missing depth, and depth outside
[0.5, 5] m marked as a hole (W = 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raycast.c")
_LIB_PATH = os.path.join(_HERE, "_raycast.so")
_lock = threading.Lock()
_lib = None

BOX_STRIDE = 20


def build_raycaster(force: bool = False) -> str:
    """Compile the ray caster into an in-tree shared object (gcc)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build_raycaster()
            lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            lib.rgbid_synth_raycast.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp,
                                                ctypes.c_int, fp, dp, dp, dp]
            lib.rgbid_synth_raycast.restype = None
            _lib = lib
    return _lib


# ----------------------------------------------------------------------------- textures

def perlin_tile(rng: np.random.Generator, size: int = 512, periods=(4, 8, 16, 32, 64, 128),
                persistence: float = 0.6) -> np.ndarray:
    """Periodic fractal 2D gradient (Perlin) noise tile, rescaled to [0, 1]."""
    acc = np.zeros((size, size), dtype=np.float64)
    amp = 1.0
    coords = np.arange(size, dtype=np.float64)
    for n in periods:
        ang = rng.uniform(0.0, 2.0 * np.pi, size=(n, n))
        gx, gy = np.cos(ang), np.sin(ang)
        X = coords * (n / size)
        i0 = np.floor(X).astype(np.int64)
        f = X - i0
        i1 = (i0 + 1) % n
        fade = f * f * f * (f * (f * 6.0 - 15.0) + 10.0)
        fy_, fx_ = np.meshgrid(f, f, indexing="ij")
        uy, ux = np.meshgrid(fade, fade, indexing="ij")
        iy0, ix0 = np.meshgrid(i0, i0, indexing="ij")
        iy1, ix1 = np.meshgrid(i1, i1, indexing="ij")

        def corner(iy, ix, dy, dx):
            return gx[iy, ix] * dx + gy[iy, ix] * dy

        n00 = corner(iy0, ix0, fy_, fx_)
        n10 = corner(iy0, ix1, fy_, fx_ - 1.0)
        n01 = corner(iy1, ix0, fy_ - 1.0, fx_)
        n11 = corner(iy1, ix1, fy_ - 1.0, fx_ - 1.0)
        top = n00 + (n10 - n00) * ux
        bot = n01 + (n11 - n01) * ux
        acc += amp * (top + (bot - top) * uy)
        amp *= persistence
    lo, hi = np.percentile(acc, 0.5), np.percentile(acc, 99.5)
    return np.clip((acc - lo) / (hi - lo), 0.0, 1.0).astype(np.float32)


# ----------------------------------------------------------------------------- geometry helpers

def rotation_about(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix about a unit axis (used only to place objects and cameras)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    x, y, z = a
    c, s = np.cos(angle), np.sin(angle)
    C = 1.0 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def random_relative_pose(rng: np.random.Generator, max_angle_deg: float, max_trans: float) -> np.ndarray:
    """4x4 pose: rotation angle ~U(0, max) about a uniform axis; translation ~U(0, max) m."""
    T = np.eye(4)
    T[:3, :3] = rotation_about(random_unit(rng), np.deg2rad(rng.uniform(0.0, max_angle_deg)))
    T[:3, 3] = random_unit(rng) * rng.uniform(0.0, max_trans)
    return T


class Scene:
    """A list of oriented textured boxes plus their texture tiles."""

    def __init__(self, textures: np.ndarray):
        self.textures = np.ascontiguousarray(textures, dtype=np.float32)
        self.boxes: list[np.ndarray] = []
        self.light = np.array([0.3, -0.8, -0.5]) / np.linalg.norm([0.3, -0.8, -0.5])

    def add_box(self, center, R, half, tex_id, texel=0.005, inside=False, rng=None):
        b = np.zeros(BOX_STRIDE)
        b[0:3] = center
        b[3:12] = np.asarray(R, dtype=np.float64).reshape(9)
        b[12:15] = half
        b[15] = 1.0 if inside else 0.0
        b[16] = tex_id
        b[17] = texel
        if rng is not None:
            b[18:20] = rng.uniform(0, 4096, size=2)
        self.boxes.append(b)

    def render(self, K, width: int, height: int, T_wc: np.ndarray):
        """Noise-free render: (intensity, depth z) as float64 arrays; z = 0 where no hit."""
        lib = _load()
        boxes = np.ascontiguousarray(np.stack(self.boxes), dtype=np.float64)
        Kd = np.ascontiguousarray(np.asarray(K, dtype=np.float64))
        Tw = np.ascontiguousarray(np.asarray(T_wc, dtype=np.float64))
        light = np.ascontiguousarray(self.light, dtype=np.float64)
        z = np.zeros((height, width), dtype=np.float64)
        inten = np.zeros((height, width), dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.rgbid_synth_raycast(width, height, Kd.ctypes.data_as(dp), Tw.ctypes.data_as(dp),
                                len(self.boxes), boxes.ctypes.data_as(dp), self.textures.shape[1],
                                self.textures.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                light.ctypes.data_as(dp), z.ctypes.data_as(dp), inten.ctypes.data_as(dp))
        return inten, z


def apply_noise(inten, z, rng, sigma_z_coef=1.5e-3, sigma_i=2.0 / 255.0, hole_frac=0.10,
                z_min=0.5, z_max=5.0, noise=True):
    """Sensor model -> (I float32 in [0,1], W float32 inverse depth, 0 = hole)."""
    hit = z > 0
    if noise:
        zn = z + rng.standard_normal(z.shape) * sigma_z_coef * z * z
        In = inten + rng.standard_normal(z.shape) * sigma_i
        drop = rng.random(z.shape) < hole_frac
    else:
        zn, In, drop = z, inten, np.zeros(z.shape, dtype=bool)
    valid = hit & (zn >= z_min) & (zn <= z_max) & ~drop
    W = np.zeros(z.shape, dtype=np.float64)
    W[valid] = 1.0 / zn[valid]
    return np.clip(In, 0.0, 1.0).astype(np.float32), W.astype(np.float32)


# ----------------------------------------------------------------------------- scenes

def make_object_scene(rng: np.random.Generator, K, width: int, n_objects: int = 6,
                      n_textures: int = 6, tex_size: int = 512) -> Scene:
    """Random planes/boxes 0.5-5 m in front of a camera at the origin (looking +z)."""
    tex = np.stack([perlin_tile(rng, tex_size) for _ in range(n_textures)])
    sc = Scene(tex)
    fx, cx = K[0], K[2]
    half_fov = (width * 0.5) / fx
    # a large tilted backdrop plane fills the view behind the objects
    zb = rng.uniform(3.5, 4.6)
    Rb = rotation_about([1, 0, 0], np.deg2rad(rng.uniform(-25, 25))) @ \
        rotation_about([0, 1, 0], np.deg2rad(rng.uniform(-25, 25)))
    sc.add_box([0.0, 0.0, zb], Rb, [4.0, 4.0, 0.002], int(rng.integers(n_textures)), rng=rng)
    for _ in range(n_objects - 1):
        z = rng.uniform(0.8, 3.0)
        x = z * half_fov * rng.uniform(-0.8, 0.8)
        y = z * half_fov * 0.75 * rng.uniform(-0.8, 0.8)
        if rng.random() < 0.4:
            half = [rng.uniform(0.25, 0.7), rng.uniform(0.25, 0.7), 0.002]   # a plane
        else:
            half = list(rng.uniform(0.1, 0.45, size=3))                        # a box
        sc.add_box([x, y, z], random_rotation(rng), half, int(rng.integers(n_textures)), rng=rng)
    return sc


def make_room(rng: np.random.Generator, n_boxes: int = 20, n_textures: int = 10,
              tex_size: int = 512) -> Scene:
    """Procedural room (6 x 3 x 6 m, y pointing down) with textured boxes."""
    tex = np.stack([perlin_tile(rng, tex_size) for _ in range(n_textures)])
    sc = Scene(tex)
    sc.add_box([0.0, 0.0, 0.0], np.eye(3), [3.0, 1.5, 3.0], int(rng.integers(n_textures)),
               texel=0.006, inside=True, rng=rng)
    placed = 0
    while placed < n_boxes:
        x, z = rng.uniform(-2.7, 2.7, size=2)
        if max(abs(x), abs(z)) < 1.5:          # keep the camera's region free
            continue
        half = rng.uniform(0.15, 0.55, size=3)
        on_floor = rng.random() < 0.6
        y = 1.5 - half[1] if on_floor else rng.uniform(-1.2, 1.0)
        R = rotation_about([0, 1, 0], rng.uniform(0, 2 * np.pi))
        if not on_floor:
            R = R @ random_rotation(rng)
        sc.add_box([x, y, z], R, half, int(rng.integers(n_textures)), rng=rng)
        placed += 1
    return sc


def _bspline(ctrl: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Uniform cubic B-spline (C2) through control rows, evaluated at tau in [0, n-3)."""
    i = np.clip(np.floor(tau).astype(np.int64), 0, len(ctrl) - 4)
    s = (tau - i)[:, None]
    b0 = (1 - s) ** 3 / 6.0
    b1 = (3 * s ** 3 - 6 * s ** 2 + 4) / 6.0
    b2 = (-3 * s ** 3 + 3 * s ** 2 + 3 * s + 1) / 6.0
    b3 = s ** 3 / 6.0
    return b0 * ctrl[i] + b1 * ctrl[i + 1] + b2 * ctrl[i + 2] + b3 * ctrl[i + 3]


def _ypr(yaw, pitch, roll):
    return rotation_about([0, 1, 0], yaw) @ rotation_about([1, 0, 0], pitch) @ rotation_about([0, 0, 1], roll)


def _rot_angle(R):
    c = np.clip((np.trace(R) - 1.0) * 0.5, -1.0, 1.0)
    return float(np.arccos(c))


def make_trajectory(rng: np.random.Generator, n_frames: int = 300, fps: float = 30.0,
                    v_max: float = 0.5, w_max_deg: float = 30.0, yaw_step_deg: float = 70.0) -> np.ndarray:
    """Smooth random camera-to-world poses [n, 4, 4] inside the room's free region.

    Control poses once per second (yaw random walk of +-yaw_step_deg, pitch
    +-10 deg, roll +-5 deg) are joined by a cubic B-spline; the excursion about
    the mean is then scaled down until speed <= v_max and angular rate <= w_max.
    """
    n_ctrl = int(np.ceil(n_frames / fps)) + 4
    pos = np.column_stack([rng.uniform(-0.9, 0.9, n_ctrl), rng.uniform(-0.3, 0.3, n_ctrl),
                           rng.uniform(-0.9, 0.9, n_ctrl)])
    yaw = np.cumsum(rng.uniform(-np.deg2rad(yaw_step_deg), np.deg2rad(yaw_step_deg), n_ctrl))
    ang = np.column_stack([yaw, rng.uniform(-np.deg2rad(10), np.deg2rad(10), n_ctrl),
                           rng.uniform(-np.deg2rad(5), np.deg2rad(5), n_ctrl)])
    tau = np.arange(n_frames) / fps
    P = _bspline(pos, tau)
    A = _bspline(ang, tau)
    for _ in range(30):
        Rs = [_ypr(*a) for a in A]
        v = np.linalg.norm(np.diff(P, axis=0), axis=1).max() * fps
        w = max(_rot_angle(Rs[k].T @ Rs[k + 1]) for k in range(n_frames - 1)) * fps
        sp = min(1.0, 0.98 * v_max / max(v, 1e-12))
        sa = min(1.0, 0.98 * np.deg2rad(w_max_deg) / max(w, 1e-12))
        if sp >= 1.0 and sa >= 1.0:
            break
        P = P.mean(0) + sp * (P - P.mean(0))
        A = A.mean(0) + sa * (A - A.mean(0))
    T = np.tile(np.eye(4), (n_frames, 1, 1))
    for k in range(n_frames):
        T[k, :3, :3] = _ypr(*A[k])
        T[k, :3, 3] = P[k]
    return T


# ----------------------------------------------------------------------------- workloads

def pinhole(width: int, height: int, f0: float = 525.0, w0: int = 640):
    """Kinect-class intrinsics scaled to a resolution: f = 525 W/640, c = (W-1)/2."""
    f = f0 * width / w0
    return (f, f, (width - 1) / 2.0, (height - 1) / 2.0)


def make_pair(seed: int, width: int = 160, height: int = 120, K=None, noise: bool = True,
              max_angle_deg: float = 2.0, max_trans: float = 0.03, n_objects: int = 6):
    """One synthetic frame pair A (reference, at the origin) and B at pose T_gt = A_T_B.

    Returns a dict with float32 planes I_A, W_A, I_B, W_B, the intrinsics K
    (fx, fy, cx, cy) and the 4x4 ground truth T_gt (X_A = R X_B + t)."""
    if K is None:
        K = pinhole(width, height)
    rng = np.random.default_rng(seed)
    scene = make_object_scene(rng, K, width, n_objects=n_objects)
    T_gt = random_relative_pose(rng, max_angle_deg, max_trans)
    iA, zA = scene.render(K, width, height, np.eye(4))
    iB, zB = scene.render(K, width, height, T_gt)
    I_A, W_A = apply_noise(iA, zA, rng, noise=noise)
    I_B, W_B = apply_noise(iB, zB, rng, noise=noise)
    return dict(I_A=I_A, W_A=W_A, I_B=I_B, W_B=W_B, K=tuple(float(k) for k in K), T_gt=T_gt,
                seed=seed, width=width, height=height)


def render_sequence(seed: int = 0, n_frames: int = 300, width: int = 640, height: int = 480,
                    noise: bool = True, yaw_step_deg: float = 70.0):
    """The 30 Hz room sequence: dict with I [n,h,w], W [n,h,w] (float32), K, T_wc [n,4,4]."""
    rng = np.random.default_rng(seed)
    scene = make_room(rng)
    T = make_trajectory(rng, n_frames, yaw_step_deg=yaw_step_deg)
    K = pinhole(width, height)
    I = np.zeros((n_frames, height, width), dtype=np.float32)
    W = np.zeros((n_frames, height, width), dtype=np.float32)
    for k in range(n_frames):
        ik, zk = scene.render(K, width, height, T[k])
        I[k], W[k] = apply_noise(ik, zk, rng, noise=noise)
    return dict(I=I, W=W, K=tuple(float(k) for k in K), T_wc=T, seed=seed, width=width, height=height)


BATCH_SIZES = ((320, 240), (640, 480), (960, 720), (1280, 960))


def batch_levels(width: int) -> int:
    """Pyramid levels of a batch pair: halve down to an 80-pixel-wide coarsest level."""
    return 1 + int(np.floor(np.log2(width / 80.0)))


def batch_iters(levels: int) -> list:
    """Gauss-Newton iterations per level, finest first: 10 at the coarsest, 5 elsewhere."""
    return [5] * (levels - 1) + [10]


def make_batch(seed: int = 0, n: int = 64, sizes=BATCH_SIZES, max_angle_deg: float = 10.0, max_trans: float = 0.2,
               init_angle_deg: float = 2.0, init_trans: float = 0.03, noise: bool = True):
    """Loop-closure-verification-like batch: n independent pairs, an equal share at
    each resolution of ``sizes`` (shuffled), ground truth A_T_B with angle
    ~U(0, max_angle_deg) and translation ~U(0, max_trans) m, and an initial guess
    T_init = T_gt dT with dT ~ U(0, init_angle_deg) / U(0, init_trans) (the
    perturbed seed pose a RANSAC stage would hand to the dense check).
    Returns a list of make_pair dicts with T_init, levels and iters added."""
    rng = np.random.default_rng(seed)
    res = [sizes[i % len(sizes)] for i in range(n)]
    order = rng.permutation(n)
    res = [res[i] for i in order]
    out = []
    for (w, h) in res:
        pair_seed = int(rng.integers(0, 2**31 - 1))
        p = make_pair(pair_seed, w, h, noise=noise, max_angle_deg=max_angle_deg, max_trans=max_trans)
        dT = random_relative_pose(rng, init_angle_deg, init_trans)
        p["T_init"] = p["T_gt"] @ dT
        L = batch_levels(w)
        p["levels"] = L
        p["iters"] = batch_iters(L)
        out.append(p)
    return out
