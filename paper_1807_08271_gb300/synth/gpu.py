"""GPU rendering of large sets of synthetic frame pairs (training inputs).

Same scene family and sensor model as ``make_pair`` (random textured planes
and boxes 0.8-3 m in front of a tilted backdrop 3.5-4.6 m away; depth noise
sigma_z = 1.5e-3 z^2, intensity noise 2/255, 10 % missing depth, depth outside
[0.5, 5] m dropped), drawn with vectorised numpy from one seed, rendered by
``raycast_gpu.cu`` in single precision and noised with a seeded torch
generator on the device.  Textures come from a shared bank of Perlin tiles.
It produces INPUTS only and holds none of the alignment arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

from . import BOX_STRIDE, perlin_tile, pinhole

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raycast_gpu.cu")
_LIB_PATH = os.path.join(_HERE, "_raycast_gpu.so")
_lock = threading.Lock()
_lib = None
N_BOX = 6
LIGHT = np.array([0.3, -0.8, -0.5]) / np.linalg.norm([0.3, -0.8, -0.5])


def build_gpu_raycaster(force: bool = False) -> str:
    """Compile raycast_gpu.cu for sm_103a into an in-tree shared object (nvcc)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC", "-shared",
                    _SRC, "-o", _LIB_PATH + ".tmp"], check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_gpu_raycaster())
            vp = ctypes.c_void_p
            lib.synth_render_gpu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                             vp, vp, vp, ctypes.c_int, vp, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_float), vp, vp, vp]
            lib.synth_render_gpu.restype = ctypes.c_int
            _lib = lib
    return _lib


class TextureBank:
    """n Perlin tiles (tex_size^2 each) on the device."""

    def __init__(self, seed: int, n: int = 48, tex_size: int = 512, device="cuda"):
        import torch
        rng = np.random.default_rng(seed)
        tiles = np.stack([perlin_tile(rng, tex_size) for _ in range(n)]).astype(np.float32)
        self.n, self.size = n, tex_size
        self.tex = torch.from_numpy(tiles).to(device)


def _rot_x(a):
    c, s = np.cos(a), np.sin(a)
    R = np.zeros(a.shape + (3, 3))
    R[..., 0, 0] = 1
    R[..., 1, 1], R[..., 1, 2], R[..., 2, 1], R[..., 2, 2] = c, -s, s, c
    return R


def _rot_y(a):
    c, s = np.cos(a), np.sin(a)
    R = np.zeros(a.shape + (3, 3))
    R[..., 1, 1] = 1
    R[..., 0, 0], R[..., 0, 2], R[..., 2, 0], R[..., 2, 2] = c, s, -s, c
    return R


def _axis_angle(axis, ang):
    """Rotations about unit axes [..., 3] by angles [...] (Rodrigues)."""
    K = np.zeros(axis.shape[:-1] + (3, 3))
    x, y, z = axis[..., 0], axis[..., 1], axis[..., 2]
    K[..., 0, 1], K[..., 0, 2], K[..., 1, 0] = -z, y, z
    K[..., 1, 2], K[..., 2, 0], K[..., 2, 1] = -x, -y, x
    s, c = np.sin(ang)[..., None, None], np.cos(ang)[..., None, None]
    return np.eye(3) + s * K + (1 - c) * (K @ K)


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _random_rotations(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                     2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                     2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], axis=1).reshape(n, 3, 3)


def object_scenes(rng, n: int, K, width: int, n_tex: int) -> np.ndarray:
    """[n, N_BOX, BOX_STRIDE] float32: a backdrop plane and five planes/boxes per scene."""
    fx = K[0]
    half_fov = (width * 0.5) / fx
    S = np.zeros((n, N_BOX, BOX_STRIDE))
    zb = rng.uniform(3.5, 4.6, n)
    Rb = _rot_x(np.deg2rad(rng.uniform(-25, 25, n))) @ _rot_y(np.deg2rad(rng.uniform(-25, 25, n)))
    S[:, 0, 2] = zb
    S[:, 0, 3:12] = Rb.reshape(n, 9)
    S[:, 0, 12:15] = [4.0, 4.0, 0.002]
    S[:, 0, 16] = rng.integers(0, n_tex, n)
    S[:, 0, 17] = 0.005
    S[:, 0, 18:20] = rng.uniform(0, 4096, (n, 2))
    for k in range(1, N_BOX):
        z = rng.uniform(0.8, 3.0, n)
        S[:, k, 0] = z * half_fov * rng.uniform(-0.8, 0.8, n)
        S[:, k, 1] = z * half_fov * 0.75 * rng.uniform(-0.8, 0.8, n)
        S[:, k, 2] = z
        plane = rng.random(n) < 0.4
        half = rng.uniform(0.1, 0.45, (n, 3))
        half[plane, 0] = rng.uniform(0.25, 0.7, plane.sum())
        half[plane, 1] = rng.uniform(0.25, 0.7, plane.sum())
        half[plane, 2] = 0.002
        S[:, k, 3:12] = _random_rotations(rng, n).reshape(n, 9)
        S[:, k, 12:15] = half
        S[:, k, 16] = rng.integers(0, n_tex, n)
        S[:, k, 17] = 0.005
        S[:, k, 18:20] = rng.uniform(0, 4096, (n, 2))
    return S.astype(np.float32)


def relative_poses(rng, n: int, max_angle_deg: float, max_trans: float) -> np.ndarray:
    """[n, 4, 4]: rotation angle ~U(0, max) about a uniform axis, translation ~U(0, max) m."""
    T = np.tile(np.eye(4), (n, 1, 1))
    T[:, :3, :3] = _axis_angle(_unit(rng, n), np.deg2rad(rng.uniform(0, max_angle_deg, n)))
    T[:, :3, 3] = _unit(rng, n) * rng.uniform(0, max_trans, n)[:, None]
    return T


def render_pairs(bank: TextureBank, scenes, T_gt, width: int, height: int, K, stream=None):
    """Noise-free renders of A (at the origin) and B (at T_gt) for every scene:
    (depth [n, 2, h, w], intensity [n, 2, h, w]) float32 device tensors."""
    import torch
    dev = bank.tex.device
    n = scenes.shape[0]
    T = np.zeros((n, 2, 4, 4), dtype=np.float32)
    T[:, 0] = np.eye(4)
    T[:, 1] = T_gt
    Td = torch.from_numpy(T.reshape(2 * n, 16)).to(dev)
    scene_of = torch.arange(n, dtype=torch.int32, device=dev).repeat_interleave(2)
    boxes = torch.from_numpy(np.ascontiguousarray(scenes)).to(dev)
    depth = torch.empty((n, 2, height, width), dtype=torch.float32, device=dev)
    inten = torch.empty_like(depth)
    Kf = (ctypes.c_float * 4)(*[float(k) for k in K])
    light = (ctypes.c_float * 3)(*[float(v) for v in LIGHT])
    s = torch.cuda.current_stream(dev) if stream is None else stream
    code = _load().synth_render_gpu(2 * n, width, height, Kf, Td.data_ptr(), scene_of.data_ptr(), boxes.data_ptr(),
                                    N_BOX, bank.tex.data_ptr(), bank.size, light, depth.data_ptr(),
                                    inten.data_ptr(), s.cuda_stream)
    if code != 0:
        raise RuntimeError(f"synth_render_gpu failed ({code})")
    return depth, inten


def noise_gpu(depth, inten, gen, sigma_z_coef=1.5e-3, sigma_i=2.0 / 255.0, hole_frac=0.10, z_min=0.5, z_max=5.0):
    """The sensor model of ``apply_noise`` on device tensors -> (I, W) float32."""
    import torch
    hit = depth > 0
    zn = depth + torch.randn(depth.shape, generator=gen, device=depth.device) * sigma_z_coef * depth * depth
    In = inten + torch.randn(depth.shape, generator=gen, device=depth.device) * sigma_i
    drop = torch.rand(depth.shape, generator=gen, device=depth.device) < hole_frac
    valid = hit & (zn >= z_min) & (zn <= z_max) & ~drop
    W = torch.where(valid, 1.0 / torch.where(valid, zn, torch.ones_like(zn)), torch.zeros_like(zn))
    return In.clamp(0.0, 1.0), W


def make_pairs_gpu(seed: int, n: int, bank: TextureBank, width: int = 640, height: int = 480,
                   max_angle_deg: float = 10.0, max_trans: float = 0.15):
    """n noisy pairs: dict with I, W [n, 2, h, w] (index 0 = A, 1 = B) device
    tensors, the intrinsics K and the ground truth T_gt [n, 4, 4] (A_T_B, numpy)."""
    import torch
    rng = np.random.default_rng(seed)
    K = pinhole(width, height)
    scenes = object_scenes(rng, n, K, width, bank.n)
    T_gt = relative_poses(rng, n, max_angle_deg, max_trans)
    depth, inten = render_pairs(bank, scenes, T_gt, width, height, K)
    gen = torch.Generator(device=bank.tex.device)
    gen.manual_seed(int(rng.integers(0, 2**62)))
    I, W = noise_gpu(depth, inten, gen)
    return dict(I=I, W=W, K=tuple(float(k) for k in K), T_gt=T_gt)
