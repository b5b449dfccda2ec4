"""Frame-to-keyframe tracking front-end over the C ABI ("Camera tracking" and
"Keyframe fusion" of the paper's RGB-ID SLAM system).

Per frame k, entirely enqueued on one CUDA stream (no host round trip):
  1. build the frame's pyramid;
  2. initial guess by the constant-velocity model
     kf_T_k(0) = kf_T_{k-1} (kf_T_{k-2})^-1 kf_T_{k-1};
  3. align the frame to the keyframe (coarse-to-fine IRLS);
  4. either fuse the frame into the keyframe with the estimated pose and the
     final sigma_W of the alignment, or, every ``kf_every`` frames, make the
     frame the new keyframe (after its own alignment, without fusing it into
     the outgoing one) and re-express the motion model's poses in it;
  5. rebuild the keyframe's pyramid.
Each frame's result (pose relative to its keyframe, robust parameters, ...) is
copied to a device array so that the host reads them once at the end.
"""
from __future__ import annotations

import numpy as np

from . import rgbid as R


class Tracker:
    def __init__(self, width: int, height: int, K, levels: int = 4, iters=(5, 5, 5, 10), kf_every: int = 20,
                 precision: int = R.PLANES_F32, fuse_intensity: bool = True, max_frames: int = 4096,
                 device="cuda"):
        import torch
        self.torch = torch
        self.w, self.h, self.K = width, height, tuple(float(k) for k in K)
        self.kf_every = kf_every
        self.fuse_intensity = fuse_intensity
        self.device = device
        self.params = R.rgbid_default_params(levels=levels, iters=iters)
        self.cur = R.DevicePyramid(width, height, levels, precision, device)
        self.kfp = R.DevicePyramid(width, height, levels, precision, device)
        f32 = dict(dtype=torch.float32, device=device)
        self.I_kf = torch.zeros((height, width), **f32)
        self.W_kf = torch.zeros((height, width), **f32)
        self.C_kf = torch.zeros((height, width), **f32)
        self.res = R.result_tensor(1, device)
        self.results = torch.zeros((max_frames, R.RESULT_BYTES), dtype=torch.uint8, device=device)
        f64 = dict(dtype=torch.float64, device=device)
        eye = torch.eye(4, **f64).reshape(16)
        self.T1 = eye.clone()      # kf_T_{k-1}
        self.T2 = eye.clone()      # kf_T_{k-2}
        self.Tinit = eye.clone()
        self.Tnew = eye.clone()
        self.ws = None
        self.k = 0
        self.is_kf = np.zeros(max_frames, dtype=bool)

    def _T_view(self):
        return self.res[0, 0:128].view(self.torch.float64)

    def _sigmaW_view(self):
        off = 8 * (16 + 36 + 6 + 2 + 1)
        return self.res[0, off:off + 8].view(self.torch.float64)

    def step(self, I, W, stream=None):
        """Process one frame (float32 CUDA tensors [h, w])."""
        torch = self.torch
        k = self.k
        if k == 0:
            R.rgbid_init_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, stream)
            self.kfp.build(self.I_kf, self.W_kf, self.K, stream)
            if self.ws is None:
                self.ws = R.new_workspace(self.kfp.desc, self.params, self.device)
            self.T1.copy_(torch.eye(4, dtype=torch.float64, device=self.device).reshape(16))
            self.T2.copy_(self.T1)
            self.is_kf[0] = True
            self.k = 1
            return
        self.cur.build(I, W, self.K, stream)
        R.rgbid_predict_pose(self.T1, self.T2, self.Tinit, stream)
        R.rgbid_align(self.kfp.desc, self.cur.desc, self.Tinit, self.params, self.ws, self.res, stream)
        self.results[k].copy_(self.res[0])
        if k % self.kf_every == 0:
            # new keyframe = this frame; poses of frames k-1 and k re-expressed in it
            R.rgbid_compose_pose(self._T_view(), True, self.T1, self.Tnew, stream)   # k_T_{k-1}
            self.T2.copy_(self.Tnew)
            self.T1.copy_(torch.eye(4, dtype=torch.float64, device=self.device).reshape(16))
            R.rgbid_init_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, stream)
            self.is_kf[k] = True
        else:
            R.rgbid_fuse_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, self.K, self._T_view(),
                                  self._sigmaW_view(), self.fuse_intensity, stream)
            self.T2.copy_(self.T1)
            self.T1.copy_(self._T_view())
        self.kfp.build(self.I_kf, self.W_kf, self.K, stream)
        self.k = k + 1

    def trajectory(self):
        """World-from-camera poses of the processed frames (frame 0 = identity), on the host."""
        n = self.k
        T_world = [np.eye(4)]
        T_wkf = np.eye(4)
        for k in range(1, n):
            r = R.parse_result(self.results[k])
            Tk = T_wkf @ r["T"]
            T_world.append(Tk)
            if self.is_kf[k]:
                T_wkf = Tk
        return np.stack(T_world)

    def frame_results(self):
        return [R.parse_result(self.results[k]) for k in range(1, self.k)]
