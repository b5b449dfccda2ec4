"""Thin Python binding of ``librgbid`` (the C ABI declared in ``include/rgbid.h``).

Argument marshalling only: every step of the alignment and fusion runs in the
library's CUDA kernels.  PyTorch supplies device memory (tensors whose
``data_ptr()`` is passed through) and streams (``torch.cuda.Stream``); the
functions below carry the same names as the C entry points.  There is no CPU
fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_size_t, c_uint8, c_void_p

import numpy as np

from . import build as _build

MAX_LEVELS = 6
MAX_SAMPLES = 19200
PLANES_F32 = 0
PLANES_BF16_F16 = 1

OK = 0
ERR_INVALID_ARG = 1
ERR_CUDA = 2
ERR_WORKSPACE = 3
ERR_DEGENERATE = 4
ERR_TIMEOUT = 5
ERR_UNSUPPORTED = 6
WARP_PER_LEVEL = 0
WARP_FULL_RESOLUTION = 1


class Intrinsics(Structure):
    _fields_ = [("fx", c_double), ("fy", c_double), ("cx", c_double), ("cy", c_double)]


class Level(Structure):
    _fields_ = [("width", c_int), ("height", c_int), ("pitch", c_int), ("pad_", c_int),
                ("K", Intrinsics), ("IW", c_void_p)]


class Pyramid(Structure):
    _fields_ = [("levels", c_int), ("precision", c_int), ("lv", Level * MAX_LEVELS)]


KERNEL_SWEEP = 0
KERNEL_ROBUST = 1
KERNEL_BATCH = 2
KERNEL_LEVEL = 3
KERNEL_SPLIT = 4


class Timing(Structure):
    _fields_ = [("ev_start", POINTER(c_void_p)), ("ev_end", POINTER(c_void_p)), ("capacity", c_int),
                ("kernel", c_int), ("count", c_int), ("pad_", c_int), ("units", ctypes.c_longlong)]


class AlignParams(Structure):
    _fields_ = [("levels", c_int), ("iters", c_int * MAX_LEVELS), ("scale_iters", c_int),
                ("bisect_steps", c_int), ("sample_cap", c_int), ("estimate_nu", c_int),
                ("min_valid", c_int), ("warp_mode", c_int), ("nu0", c_double), ("nu_lo", c_double),
                ("nu_hi", c_double), ("timing", POINTER(Timing)), ("level_iters", c_void_p),
                ("no_level_kernel", c_int), ("pad2_", c_int)]


class AlignResult(Structure):
    _fields_ = [("T", c_double * 16), ("H", c_double * 36), ("g", c_double * 6), ("mu", c_double * 2),
                ("sigma", c_double * 2), ("nu", c_double * 2), ("cost", c_double), ("n_valid", c_int * 2),
                ("iters_done", c_int), ("iters_skipped", c_int), ("status", c_int), ("pad_", c_int)]


RESULT_BYTES = ctypes.sizeof(AlignResult)


class BatchItem(Structure):
    _fields_ = [("ref", Pyramid), ("cur", Pyramid), ("T_init", c_double * 16), ("levels", c_int),
                ("iters", c_int * MAX_LEVELS), ("pad_", c_int), ("result", c_void_p)]


class Bilateral(Structure):
    _fields_ = [("radius", c_int), ("pad_", c_int), ("sigma_s", c_double), ("sigma_r_I", c_double),
                ("sigma_r_W", c_double)]


class BatchConfig(Structure):
    _fields_ = [("cluster", c_int), ("rows_per_warp", c_int), ("n_clusters", c_int), ("pad_", c_int)]

    def as_tuple(self):
        return (self.cluster, self.rows_per_warp, self.n_clusters)

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/rgbid.h
SIGNATURES = [
    ("rgbid_status_string", c_char_p, [c_int]),
    ("rgbid_default_params", None, [POINTER(AlignParams)]),
    ("rgbid_pyramid_bytes", c_size_t, [c_int, c_int, c_int, c_int]),
    ("rgbid_build_pyramid", c_int, [c_void_p, c_void_p, c_int, c_int, c_int, Intrinsics, c_int, c_int,
                                    c_void_p, c_size_t, POINTER(Pyramid), c_void_p]),
    ("rgbid_align_workspace_bytes", c_size_t, [POINTER(Pyramid), POINTER(AlignParams)]),
    ("rgbid_align_launches", c_int, [POINTER(Pyramid), POINTER(AlignParams)]),
    ("rgbid_align", c_int, [POINTER(Pyramid), POINTER(Pyramid), c_void_p, c_int, POINTER(AlignParams),
                            c_void_p, c_size_t, c_void_p, c_void_p]),
    ("rgbid_align_noalloc", c_int, [POINTER(Pyramid), POINTER(Pyramid), c_void_p, c_int, POINTER(AlignParams),
                                    c_void_p, c_void_p]),
    ("rgbid_eval_step", c_int, [POINTER(Pyramid), POINTER(Pyramid), c_int, POINTER(c_double), c_void_p,
                                POINTER(AlignParams), c_void_p, c_size_t, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p]),
    ("rgbid_fuse_keyframe", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_int,
                                    c_int, Intrinsics, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    ("rgbid_init_keyframe", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_int,
                                    c_int, c_void_p]),
    ("rgbid_default_bilateral", None, [POINTER(Bilateral)]),
    ("rgbid_covariance_workspace_bytes", c_size_t, [POINTER(Pyramid)]),
    ("rgbid_covariance", c_int, [POINTER(Pyramid), POINTER(Pyramid), c_void_p, c_int, POINTER(AlignParams),
                                 POINTER(Bilateral), c_void_p, c_size_t, c_void_p, c_void_p, c_void_p]),
    ("rgbid_fuse_or_switch_keyframe", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int,
                                              c_int, c_int, Intrinsics, c_void_p, c_void_p, c_int, c_void_p,
                                              c_void_p]),
    ("rgbid_covisibility", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_int, c_int, Intrinsics,
                                   c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("rgbid_keyframe_decide", c_int, [c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
    ("rgbid_predict_pose", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rgbid_compose_pose", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("rgbid_align_batched_workspace_bytes", c_size_t, []),
    ("rgbid_batch_check_item", c_int, [POINTER(BatchItem), c_int]),
    ("rgbid_batch_resident_clusters", c_int, [c_int, POINTER(BatchConfig), POINTER(c_int)]),
    ("rgbid_align_batched", c_int, [c_void_p, c_int, c_int, POINTER(AlignParams), POINTER(BatchConfig),
                                    c_void_p, c_size_t, c_void_p]),
    ("rgbid_batch_autotune", c_int, [c_void_p, c_int, c_int, POINTER(AlignParams), c_void_p, c_size_t, c_int,
                                     POINTER(BatchConfig), POINTER(ctypes.c_float), c_void_p]),
    ("rgbid_probe_wait_timeout", c_int, [ctypes.c_longlong, c_void_p, c_void_p]),
    ("rgbid_probe_mailbox_timeout", c_int, [ctypes.c_longlong, c_void_p, c_size_t, c_void_p, c_void_p]),
    ("rgbid_nu_constant_series", c_int, [c_double, c_double, POINTER(ctypes.c_float), c_int]),
    ("rgbid_net_param_count", c_size_t, []),
    ("rgbid_net_param_offset", c_size_t, [c_int, c_int]),
    ("rgbid_net_workspace_bytes", c_size_t, [c_int]),
    ("rgbid_net_wait_timeouts", ctypes.c_uint, []),
    ("rgbid_debug_bounds_violations", c_int, [POINTER(ctypes.c_ulonglong)]),
    ("rgbid_debug_phase_stamps", c_int, [POINTER(ctypes.c_longlong), c_int]),
    ("rgbid_net_init", c_int, [c_void_p, ctypes.c_ulonglong, c_void_p]),
    ("rgbid_net_inputs", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    ("rgbid_net_forward", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("rgbid_net_backward", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("rgbid_net_loss", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("rgbid_net_adam", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, c_void_p]),
    ("rgbid_net_plan", c_int, [c_void_p, c_int, POINTER(ctypes.c_float), c_int, c_void_p, c_void_p, c_void_p,
                               c_void_p]),
]


class RgbidError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {status_name(code)} ({code})")
        self.code = code


def lib():
    """Load (building first if needed) the in-tree librgbid.so, or with the environment
    variable RGBID_LIBRARY=checked the bounds-checked test build librgbid_checked.so
    (RGBID_LIBRARY=phases: the phase-stamped diagnostic build librgbid_phases.so)."""
    global _lib
    with _lock:
        if _lib is None:
            variant = os.environ.get("RGBID_LIBRARY")
            path = _build.build(checked=variant == "checked", phases=variant == "phases")
            L = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_name(code: int) -> str:
    names = {0: "RGBID_OK", 1: "RGBID_ERR_INVALID_ARG", 2: "RGBID_ERR_CUDA", 3: "RGBID_ERR_WORKSPACE",
             4: "RGBID_ERR_DEGENERATE", 5: "RGBID_ERR_TIMEOUT", 6: "RGBID_ERR_UNSUPPORTED"}
    return names.get(code, "RGBID_UNKNOWN_STATUS")


def _check(fn: str, code: int):
    if code != OK:
        raise RgbidError(fn, code)


def _stream_ptr(stream) -> c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


def _ptr(t) -> c_void_p:
    return c_void_p(0 if t is None else t.data_ptr())


# ----------------------------------------------------------------------------- entry points
def rgbid_status_string(code: int) -> str:
    return lib().rgbid_status_string(code).decode()


def rgbid_default_params(levels: int | None = None, iters=None) -> AlignParams:
    p = AlignParams()
    lib().rgbid_default_params(ctypes.byref(p))
    if levels is not None:
        p.levels = levels
    if iters is not None:
        for i in range(MAX_LEVELS):
            p.iters[i] = int(iters[i]) if i < len(iters) else 0
    return p


def rgbid_pyramid_bytes(width: int, height: int, levels: int, precision: int = PLANES_F32) -> int:
    return int(lib().rgbid_pyramid_bytes(width, height, levels, precision))


def rgbid_build_pyramid(I0, W0, K0, levels: int, precision: int, storage, stream=None) -> Pyramid:
    """Build a pyramid from float32 CUDA tensors I0, W0 [h, w] into ``storage`` (uint8 CUDA tensor)."""
    h, w = I0.shape[-2], I0.shape[-1]
    pitch0 = I0.stride(-2)
    assert W0.stride(-2) == pitch0 and I0.stride(-1) == 1 and W0.stride(-1) == 1
    out = Pyramid()
    K = Intrinsics(*[float(k) for k in K0])
    code = lib().rgbid_build_pyramid(_ptr(I0), _ptr(W0), pitch0, w, h, K, levels, precision, _ptr(storage),
                                     storage.numel() * storage.element_size(), ctypes.byref(out),
                                     _stream_ptr(stream))
    _check("rgbid_build_pyramid", code)
    return out


def rgbid_align_workspace_bytes(ref: Pyramid, params: AlignParams) -> int:
    return int(lib().rgbid_align_workspace_bytes(ctypes.byref(ref), ctypes.byref(params)))


def rgbid_align_launches(ref: Pyramid, params: AlignParams) -> int:
    """Kernel launches one rgbid_align call enqueues with these arguments (-1: invalid)."""
    return int(lib().rgbid_align_launches(ctypes.byref(ref), ctypes.byref(params)))


def rgbid_align(ref: Pyramid, cur: Pyramid, T_init, params: AlignParams, workspace, result, stream=None):
    """Enqueue an alignment.  ``T_init``: None (identity), a host array of 16
    doubles, or a CUDA float64 tensor of 16 elements (read on the device)."""
    if T_init is None:
        tp, on_dev = c_void_p(0), 0
    elif hasattr(T_init, "is_cuda") and T_init.is_cuda:
        tp, on_dev = _ptr(T_init), 1
    else:
        arr = np.ascontiguousarray(np.asarray(T_init, dtype=np.float64).reshape(16))
        tp, on_dev = c_void_p(arr.ctypes.data), 0
    code = lib().rgbid_align(ctypes.byref(ref), ctypes.byref(cur), tp, on_dev, ctypes.byref(params),
                             _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(result),
                             _stream_ptr(stream))
    _check("rgbid_align", code)


def rgbid_align_noalloc(ref: Pyramid, cur: Pyramid, T_init, params: AlignParams, result, stream=None):
    """rgbid_align with the library's fixed internal scratch (no workspace argument)."""
    if T_init is None:
        tp, on_dev = c_void_p(0), 0
    elif hasattr(T_init, "is_cuda") and T_init.is_cuda:
        tp, on_dev = _ptr(T_init), 1
    else:
        arr = np.ascontiguousarray(np.asarray(T_init, dtype=np.float64).reshape(16))
        tp, on_dev = c_void_p(arr.ctypes.data), 0
    code = lib().rgbid_align_noalloc(ctypes.byref(ref), ctypes.byref(cur), tp, on_dev, ctypes.byref(params),
                                     _ptr(result), _stream_ptr(stream))
    _check("rgbid_align_noalloc", code)


def rgbid_eval_step(ref: Pyramid, cur: Pyramid, level: int, T, robust, params: AlignParams, workspace,
                    r_I=None, r_W=None, mask_I=None, mask_W=None, result=None, stream=None):
    Ta = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    if robust is not None:
        ra = np.ascontiguousarray(np.asarray(robust, dtype=np.float64).reshape(6))
        rp = c_void_p(ra.ctypes.data)
    else:
        rp = c_void_p(0)
    code = lib().rgbid_eval_step(ctypes.byref(ref), ctypes.byref(cur), level,
                                 Ta.ctypes.data_as(POINTER(c_double)), rp, ctypes.byref(params), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), _ptr(r_I), _ptr(r_W),
                                 _ptr(mask_I), _ptr(mask_W), _ptr(result), _stream_ptr(stream))
    _check("rgbid_eval_step", code)


def rgbid_fuse_keyframe(I_kf, W_kf, C_kf, I_k, W_k, K, T_kf_k, sigma_W, fuse_intensity: bool = True, stream=None):
    """Fuse frame k into the keyframe in place.  ``T_kf_k``/``sigma_W`` are either
    host values (16-array, float) or CUDA float64 tensors (read on the device)."""
    h, w = W_kf.shape[-2], W_kf.shape[-1]
    on_dev = hasattr(T_kf_k, "is_cuda") and T_kf_k.is_cuda
    keep = []
    if on_dev:
        tp, sp = _ptr(T_kf_k), _ptr(sigma_W)
    else:
        Ta = np.ascontiguousarray(np.asarray(T_kf_k, dtype=np.float64).reshape(16))
        sa = np.array([float(sigma_W)], dtype=np.float64)
        keep += [Ta, sa]
        tp, sp = c_void_p(Ta.ctypes.data), c_void_p(sa.ctypes.data)
    Ki = Intrinsics(*[float(k) for k in K])
    code = lib().rgbid_fuse_keyframe(_ptr(I_kf), _ptr(W_kf), _ptr(C_kf), W_kf.stride(-2), _ptr(I_k), _ptr(W_k),
                                     W_k.stride(-2), w, h, Ki, tp, sp, 1 if on_dev else 0,
                                     1 if fuse_intensity else 0, _stream_ptr(stream))
    _check("rgbid_fuse_keyframe", code)


def rgbid_default_bilateral(**overrides) -> Bilateral:
    f = Bilateral()
    lib().rgbid_default_bilateral(ctypes.byref(f))
    for k, v in overrides.items():
        setattr(f, k, v)
    return f


def new_covariance_workspace(ref: Pyramid, device="cuda"):
    import torch
    n = lib().rgbid_covariance_workspace_bytes(ctypes.byref(ref))
    return torch.zeros(max(int(n), 256), dtype=torch.uint8, device=device)


def rgbid_covariance(ref: Pyramid, cur: Pyramid, T, params: AlignParams, filt: Bilateral, workspace, d_result,
                     d_sigma, stream=None):
    """The covariance iteration at pose ``T`` (host 4x4 or a CUDA float64 tensor of 16):
    ``d_result`` (result tensor) receives H_filt and the iteration's statistics,
    ``d_sigma`` (CUDA float64 tensor of 36) receives H_filt^-1."""
    keep = []
    if hasattr(T, "is_cuda") and T.is_cuda:
        tp, on_dev = _ptr(T), 1
    else:
        Ta = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
        keep.append(Ta)
        tp, on_dev = c_void_p(Ta.ctypes.data), 0
    code = lib().rgbid_covariance(ctypes.byref(ref), ctypes.byref(cur), tp, on_dev, ctypes.byref(params),
                                  ctypes.byref(filt), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                  _ptr(d_result), _ptr(d_sigma), _stream_ptr(stream))
    _check("rgbid_covariance", code)


def _pose_sigma_args(T, sigma_W, keep):
    """(pose pointer, sigma pointer, on_device) for host values or CUDA float64 tensors."""
    on_dev = hasattr(T, "is_cuda") and T.is_cuda
    if on_dev:
        return _ptr(T), _ptr(sigma_W), 1
    Ta = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    sa = np.array([float(sigma_W)], dtype=np.float64)
    keep += [Ta, sa]
    return c_void_p(Ta.ctypes.data), c_void_p(sa.ctypes.data), 0


def rgbid_fuse_or_switch_keyframe(I_kf, W_kf, C_kf, I_k, W_k, K, T_kf_k, sigma_W, d_switch,
                                  fuse_intensity: bool = True, stream=None):
    """Fuse frame k into the keyframe, or (device int ``d_switch`` set) make it the
    keyframe.  ``T_kf_k`` and ``sigma_W`` are CUDA float64 tensors."""
    h, w = W_kf.shape[-2], W_kf.shape[-1]
    code = lib().rgbid_fuse_or_switch_keyframe(_ptr(I_kf), _ptr(W_kf), _ptr(C_kf), W_kf.stride(-2), _ptr(I_k),
                                               _ptr(W_k), W_k.stride(-2), w, h, Intrinsics(*[float(k) for k in K]),
                                               _ptr(T_kf_k), _ptr(sigma_W), 1 if fuse_intensity else 0,
                                               _ptr(d_switch), _stream_ptr(stream))
    _check("rgbid_fuse_or_switch_keyframe", code)


def rgbid_covisibility(I_A, W_A, I_B, W_B, K, T_AB, sigma_W, d_counts, d_ratio=None, stream=None):
    """Dense covisibility counts (device uint32[4]: S_V(A->B), S_H(A), S_V(B->A), S_H(B))
    and optionally the ratio (device float32[1]).  ``T_AB``/``sigma_W`` are host
    values or CUDA float64 tensors."""
    h, w = W_A.shape[-2], W_A.shape[-1]
    keep = []
    tp, sp, on_dev = _pose_sigma_args(T_AB, sigma_W, keep)
    code = lib().rgbid_covisibility(_ptr(I_A), _ptr(W_A), W_A.stride(-2), _ptr(I_B), _ptr(W_B), W_B.stride(-2), w, h,
                                    Intrinsics(*[float(k) for k in K]), tp, sp, on_dev, _ptr(d_counts),
                                    _ptr(d_ratio) if d_ratio is not None else None, _stream_ptr(stream))
    _check("rgbid_covisibility", code)


def rgbid_keyframe_decide(d_counts, threshold: float, T_k, T1, T2, d_switch, d_ratio=None, stream=None):
    code = lib().rgbid_keyframe_decide(_ptr(d_counts), float(threshold), _ptr(T_k), _ptr(T1), _ptr(T2),
                                       _ptr(d_switch), _ptr(d_ratio) if d_ratio is not None else None,
                                       _stream_ptr(stream))
    _check("rgbid_keyframe_decide", code)


def rgbid_init_keyframe(I_kf, W_kf, C_kf, I_k, W_k, stream=None):
    h, w = W_kf.shape[-2], W_kf.shape[-1]
    code = lib().rgbid_init_keyframe(_ptr(I_kf), _ptr(W_kf), _ptr(C_kf), W_kf.stride(-2), _ptr(I_k), _ptr(W_k),
                                     W_k.stride(-2), w, h, _stream_ptr(stream))
    _check("rgbid_init_keyframe", code)


def rgbid_predict_pose(T_km1, T_km2, T_out, stream=None):
    _check("rgbid_predict_pose", lib().rgbid_predict_pose(_ptr(T_km1), _ptr(T_km2), _ptr(T_out), _stream_ptr(stream)))


def rgbid_compose_pose(A, invert_A: bool, B, T_out, stream=None):
    _check("rgbid_compose_pose", lib().rgbid_compose_pose(_ptr(A), 1 if invert_A else 0, _ptr(B), _ptr(T_out),
                                                          _stream_ptr(stream)))


def rgbid_align_batched_workspace_bytes() -> int:
    return int(lib().rgbid_align_batched_workspace_bytes())


def rgbid_batch_check_item(item: BatchItem, precision: int) -> int:
    """Host-side check of one item descriptor; returns the status code (no raise)."""
    return int(lib().rgbid_batch_check_item(ctypes.byref(item), precision))


def rgbid_batch_resident_clusters(precision: int, cfg: BatchConfig | None = None) -> int:
    n = c_int(0)
    code = lib().rgbid_batch_resident_clusters(precision, ctypes.byref(cfg) if cfg is not None else None,
                                               ctypes.byref(n))
    _check("rgbid_batch_resident_clusters", code)
    return n.value


def rgbid_align_batched(d_items, n_items: int, precision: int, params: AlignParams, cfg: BatchConfig | None,
                        workspace, stream=None):
    """Enqueue the persistent batched alignment.  ``d_items``: CUDA uint8 tensor
    holding ``n_items`` BatchItem descriptors; ``workspace``: zeroed CUDA uint8
    tensor of rgbid_align_batched_workspace_bytes()."""
    code = lib().rgbid_align_batched(_ptr(d_items), n_items, precision, ctypes.byref(params),
                                     ctypes.byref(cfg) if cfg is not None else None, _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), _stream_ptr(stream))
    _check("rgbid_align_batched", code)


def rgbid_batch_autotune(d_items, n_items: int, precision: int, params: AlignParams, workspace, reps: int = 3,
                         stream=None):
    """Time every launch shape on this batch; returns (best BatchConfig, its median ms)."""
    best = BatchConfig()
    ms = ctypes.c_float(0.0)
    code = lib().rgbid_batch_autotune(_ptr(d_items), n_items, precision, ctypes.byref(params), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), reps, ctypes.byref(best),
                                      ctypes.byref(ms), _stream_ptr(stream))
    _check("rgbid_batch_autotune", code)
    return best, float(ms.value)


def rgbid_nu_constant_series(nu_lo: float = 2.0, nu_hi: float = 10.0, n: int = 22):
    """Host-computed Chebyshev coefficients of the nu equation's constant part (see rgbid.h)."""
    out = (ctypes.c_float * n)()
    k = lib().rgbid_nu_constant_series(nu_lo, nu_hi, out, n)
    if k < 0:
        _check("rgbid_nu_constant_series", -k)
    return list(out)[:k]


def rgbid_probe_wait_timeout(budget_cycles: int, d_timeouts, stream=None):
    """One cluster-reduction round with the partials withheld: every wait runs out (see rgbid.h)."""
    _check("rgbid_probe_wait_timeout", lib().rgbid_probe_wait_timeout(budget_cycles, _ptr(d_timeouts),
                                                                      _stream_ptr(stream)))


def rgbid_probe_mailbox_timeout(budget_cycles: int, d_scratch, d_out, stream=None):
    """The split level kernel's mailbox wait on a counter nothing advances (see rgbid.h):
    d_out (4 device ints) gets the timeouts, both waits' verdicts and the error flag."""
    _check("rgbid_probe_mailbox_timeout",
           lib().rgbid_probe_mailbox_timeout(budget_cycles, _ptr(d_scratch), d_scratch.numel() * d_scratch.element_size(),
                                             _ptr(d_out), _stream_ptr(stream)))


NET_IN_H, NET_IN_W, NET_IN_C, NET_OUT, NET_LAYERS = 60, 80, 4, 7, 6
NET_TWIST_SCALE = 0.1


def rgbid_net_param_count() -> int:
    return int(lib().rgbid_net_param_count())


def rgbid_net_param_offset(layer: int, what: int) -> int:
    return int(lib().rgbid_net_param_offset(layer, what))


def rgbid_net_workspace_bytes(batch: int) -> int:
    return int(lib().rgbid_net_workspace_bytes(batch))


def rgbid_debug_bounds_violations() -> int | None:
    """Out-of-plane gather indices counted since the library was loaded (the
    bounds-checked build); None for the product library, which does not check."""
    n = ctypes.c_ulonglong(0)
    rc = lib().rgbid_debug_bounds_violations(ctypes.byref(n))
    if rc == ERR_UNSUPPORTED:
        return None
    _check("rgbid_debug_bounds_violations", rc)
    return int(n.value)


def rgbid_debug_phase_stamps():
    """The split kernel's phase stamps of the phase-stamped build as a [levels, 16, 16]
    int64 array (ns), or None for a build without them."""
    n = MAX_LEVELS * 16 * 16
    buf = (ctypes.c_longlong * n)()
    rc = lib().rgbid_debug_phase_stamps(buf, n)
    if rc == ERR_UNSUPPORTED:
        return None
    _check("rgbid_debug_phase_stamps", rc)
    return np.array(buf, dtype=np.int64).reshape(MAX_LEVELS, 16, 16)


def rgbid_net_wait_timeouts() -> int:
    """Tensor-core waits of the network's GEMMs that ran out on the current device (0 when healthy)."""
    return int(lib().rgbid_net_wait_timeouts())


def rgbid_net_init(params, seed: int, stream=None):
    _check("rgbid_net_init", lib().rgbid_net_init(_ptr(params), seed, _stream_ptr(stream)))


def rgbid_net_inputs(d_items, n: int, precision: int, x, stream=None):
    _check("rgbid_net_inputs", lib().rgbid_net_inputs(_ptr(d_items), n, precision, _ptr(x), _stream_ptr(stream)))


def rgbid_net_forward(params, x, batch: int, y, workspace, stream=None):
    _check("rgbid_net_forward", lib().rgbid_net_forward(_ptr(params), _ptr(x), batch, _ptr(y), _ptr(workspace),
                                                        workspace.numel() * workspace.element_size(),
                                                        _stream_ptr(stream)))


def rgbid_net_backward(params, x, batch: int, dy, grad, workspace, stream=None):
    _check("rgbid_net_backward", lib().rgbid_net_backward(_ptr(params), _ptr(x), batch, _ptr(dy), _ptr(grad),
                                                          _ptr(workspace),
                                                          workspace.numel() * workspace.element_size(),
                                                          _stream_ptr(stream)))


def rgbid_net_loss(y, target, batch: int, dy, loss, stream=None):
    _check("rgbid_net_loss", lib().rgbid_net_loss(_ptr(y), _ptr(target), batch, _ptr(dy), _ptr(loss),
                                                  _stream_ptr(stream)))


def rgbid_net_adam(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                   eps: float = 1e-8, stream=None):
    _check("rgbid_net_adam", lib().rgbid_net_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1,
                                                  beta2, eps, _stream_ptr(stream)))


def rgbid_net_plan(y, n: int, max_log_var, d_in, d_out, skipped=None, stream=None):
    """``max_log_var``: thresholds of tiers 1.. (tier k skips k coarse levels)."""
    thr = (ctypes.c_float * max(1, len(max_log_var)))(*[float(t) for t in max_log_var])
    _check("rgbid_net_plan", lib().rgbid_net_plan(_ptr(y), n, thr, len(max_log_var), _ptr(d_in), _ptr(d_out),
                                                  _ptr(skipped), _stream_ptr(stream)))


# ----------------------------------------------------------------------------- conveniences
def parse_result(buf) -> dict:
    """Decode an rgbid_align_result held in a (device or host) uint8 tensor."""
    raw = bytes(buf.detach().cpu().numpy().tobytes()[:RESULT_BYTES])
    r = AlignResult.from_buffer_copy(raw)
    return dict(T=np.array(r.T).reshape(4, 4), H=np.array(r.H).reshape(6, 6), g=np.array(r.g),
                mu=list(r.mu), sigma=list(r.sigma), nu=list(r.nu), cost=r.cost, n_valid=list(r.n_valid),
                iters_done=r.iters_done, iters_skipped=r.iters_skipped, status=r.status)


def result_tensor(n: int = 1, device="cuda"):
    import torch
    return torch.zeros((n, RESULT_BYTES), dtype=torch.uint8, device=device)


class DevicePyramid:
    """A pyramid plus the device storage that backs it."""

    def __init__(self, width: int, height: int, levels: int, precision: int = PLANES_F32, device="cuda"):
        import torch
        self.width, self.height, self.levels, self.precision = width, height, levels, precision
        nbytes = rgbid_pyramid_bytes(width, height, levels, precision)
        if nbytes == 0:
            raise ValueError("invalid pyramid shape")
        self.storage = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.desc = None

    def build(self, I0, W0, K0, stream=None) -> "DevicePyramid":
        self.desc = rgbid_build_pyramid(I0, W0, K0, self.levels, self.precision, self.storage, stream)
        return self

    def level_planes(self, l: int):
        """(I, W) float32 host arrays of level l (for tests and inspection)."""
        import torch
        L = self.desc.lv[l]
        off = L.IW - self.storage.data_ptr()
        bpp = 8 if self.precision == PLANES_F32 else 4
        raw = self.storage[off:off + L.pitch * L.height * bpp].cpu().numpy()
        if self.precision == PLANES_F32:
            a = raw.view(np.float32).reshape(L.height, L.pitch, 2)[:, :L.width]
            return a[..., 0].copy(), a[..., 1].copy()
        u = raw.view(np.uint16).reshape(L.height, L.pitch, 2)[:, :L.width]
        I = (u[..., 0].astype(np.uint32) << 16).view(np.float32)
        W = u[..., 1].copy().view(np.float16).astype(np.float32)
        return I.copy(), W


class KernelTimer:
    """Caller-owned CUDA events that rgbid_align records around one kernel's launches."""

    def __init__(self, kernel: int, capacity: int):
        import torch
        self.events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(capacity)]
        for a, b in self.events:          # torch creates the CUDA event on first record
            a.record()
            b.record()
        torch.cuda.synchronize()
        assert all(a.cuda_event and b.cuda_event for a, b in self.events)
        self._starts = (c_void_p * capacity)(*[e[0].cuda_event for e in self.events])
        self._ends = (c_void_p * capacity)(*[e[1].cuda_event for e in self.events])
        self.t = Timing(ctypes.cast(self._starts, POINTER(c_void_p)), ctypes.cast(self._ends, POINTER(c_void_p)),
                        capacity, kernel, 0, 0, 0)

    def attach(self, params: AlignParams):
        params.timing = ctypes.pointer(self.t)

    def reset(self):
        self.t.count = 0
        self.t.units = 0

    def total_ms(self) -> float:
        """Sum of the recorded launch durations (call after synchronising)."""
        return float(sum(s.elapsed_time(e) for s, e in self.events[:self.t.count]))


def new_workspace(ref: Pyramid, params: AlignParams, device="cuda"):
    import torch
    return torch.empty(rgbid_align_workspace_bytes(ref, params), dtype=torch.uint8, device=device)
