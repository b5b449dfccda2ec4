"""Frame-to-keyframe tracking front-end over the C ABI ("Camera tracking" and
"Keyframe fusion" of the paper's RGB-ID SLAM system).

Per frame k, entirely enqueued on one CUDA stream (no host round trip):
  1. build the frame's pyramid;
  2. initial guess by the constant-velocity model
     kf_T_k(0) = kf_T_{k-1} (kf_T_{k-2})^-1 kf_T_{k-1};
  3. align the frame to the keyframe (coarse-to-fine IRLS);
  4. either fuse the frame into the keyframe with the estimated pose and the
     final sigma_W of the alignment, or make the frame the new keyframe (after
     its own alignment, without fusing it into the outgoing one) and
     re-express the motion model's poses in it: every ``kf_every`` frames, or,
     with ``kf_covisibility``, when the dense covisibility ratio of the aligned
     frame with the keyframe falls below that threshold (0.7 in the paper),
     decided on the device;
  5. rebuild the keyframe's pyramid.
Each frame's result (pose relative to its keyframe, robust parameters, ...) is
copied to a device array so that the host reads them once at the end.

With ``graphs=True`` (the default) steps 1-5 of a frame are one CUDA graph
replay: each frame kind (fusing, keyframe-switching) and staging slot has a
graph, captured after the first eager frame of its kind, which reads the frame
from that slot's fixed staging pair; per frame the host then copies the frame
into staging (or finds it there), replays the graph and copies the frame's
result into the result array, instead of enqueueing some fifty launches.  Two
slots let a caller upload frame k+1 (``staging(slot)``) while frame k runs.  The per-launch timing hook of the
alignment (``params.timing``) needs the eager path, which step() takes while
it is attached.  With ``level_kernel=False`` every level of the alignment runs by
the per-iteration kernels (the library's default runs a level whose systematic
sample is every pixel in one persistent cluster launch).
"""
from __future__ import annotations

import numpy as np

from . import rgbid as R


class Tracker:
    def __init__(self, width: int, height: int, K, levels: int = 4, iters=(5, 5, 5, 10), kf_every: int = 20,
                 precision: int = R.PLANES_F32, fuse_intensity: bool = True, max_frames: int = 4096,
                 device="cuda", graphs: bool = True, kf_covisibility: float | None = None,
                 level_kernel: bool = True):
        import torch
        self.torch = torch
        self.w, self.h, self.K = width, height, tuple(float(k) for k in K)
        self.kf_every = kf_every
        self.kf_covisibility = kf_covisibility
        self.fuse_intensity = fuse_intensity
        self.device = device
        self.params = R.rgbid_default_params(levels=levels, iters=iters)
        self.params.no_level_kernel = 0 if level_kernel else 1
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
        self.eye16 = eye.clone()
        self.ws = None
        self.k = 0
        self.is_kf = np.zeros(max_frames, dtype=bool)
        if kf_covisibility is not None:
            # device-side decision: counts, flag and ratio of the current frame, and per-frame copies
            self.counts = torch.zeros(4, dtype=torch.int32, device=device)
            self.d_switch = torch.zeros(1, dtype=torch.int32, device=device)
            self.d_ratio = torch.zeros(1, dtype=torch.float32, device=device)
            self.kf_flags = torch.zeros(max_frames, dtype=torch.int32, device=device)
            self.ratios = torch.zeros(max_frames, dtype=torch.float32, device=device)
        self.graphs = graphs
        self._graph = {}          # (frame kind (True: keyframe switch), staging slot) -> CUDA graph of steps 1-5
        # two staging pairs for the graphs (slot 0 also takes frames passed from elsewhere)
        self._stage = [(torch.zeros((height, width), **f32), torch.zeros((height, width), **f32))
                       for _ in range(2)] if graphs else []
        self.I_in, self.W_in = self._stage[0] if graphs else (None, None)

    def _T_view(self):
        return self.res[0, 0:128].view(self.torch.float64)

    def _sigmaW_view(self):
        off = 8 * (16 + 36 + 6 + 2 + 1)
        return self.res[0, off:off + 8].view(self.torch.float64)

    def align_launches(self) -> int:
        """Kernel launches of one frame's alignment (initialisation to closing launch);
        available once the first frame has been stepped."""
        return R.rgbid_align_launches(self.kfp.desc, self.params)

    def staging(self, slot: int):
        """The (I, W) staging pair of ``slot`` (0 or 1): a frame copied there may be
        passed to step() as is, and is read by the graph without another copy.
        Staging exists only with ``graphs=True``."""
        if not self.graphs:
            raise ValueError("staging slots exist only for a tracker built with graphs=True")
        if slot not in (0, 1):
            raise ValueError(f"staging slot must be 0 or 1, got {slot}")
        return self._stage[slot]

    def step(self, I, W, stream=None):
        """Process one frame (float32 CUDA tensors [h, w]) on ``stream`` (a
        torch.cuda.Stream; None: the current stream)."""
        torch = self.torch
        k = self.k
        if k == 0:
            R.rgbid_init_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, stream)
            self.kfp.build(self.I_kf, self.W_kf, self.K, stream)
            if self.ws is None:
                self.ws = R.new_workspace(self.kfp.desc, self.params, self.device)
            self.T1.copy_(self.eye16)
            self.T2.copy_(self.T1)
            self.is_kf[0] = True
            self.k = 1
            return
        # with the covisibility policy every frame has the same kind: the device decides
        kf = self.kf_covisibility is None and k % self.kf_every == 0
        s = stream if stream is not None else torch.cuda.current_stream()
        slot = 1 if self.graphs and I is self._stage[1][0] and W is self._stage[1][1] else 0
        with torch.cuda.stream(s):
            eager = not self.graphs or bool(self.params.timing)   # a NULL timing pointer is falsy
            g = None if eager else self._graph.get((kf, slot))
            if g is not None:
                SI, SW = self._stage[slot]
                if I is not SI:             # a caller may fill the staging pair itself
                    SI.copy_(I, non_blocking=True)
                if W is not SW:
                    SW.copy_(W, non_blocking=True)
                g.replay()
            else:
                self._frame(I, W, kf, s)
            self.results[k].copy_(self.res[0], non_blocking=True)
            if self.kf_covisibility is not None:
                self.kf_flags[k:k + 1].copy_(self.d_switch, non_blocking=True)
                self.ratios[k:k + 1].copy_(self.d_ratio, non_blocking=True)
        if self.graphs and not self.params.timing and (kf, slot) not in self._graph:
            self._capture(kf, slot)
        self.is_kf[k] = kf
        self.k = k + 1

    def _frame(self, I, W, kf: bool, stream):
        """Steps 1-5 for frame data I, W; touches no host state, so it can be captured."""
        self.cur.build(I, W, self.K, stream)
        R.rgbid_predict_pose(self.T1, self.T2, self.Tinit, stream)
        R.rgbid_align(self.kfp.desc, self.cur.desc, self.Tinit, self.params, self.ws, self.res, stream)
        if self.kf_covisibility is not None:
            # covisibility of the aligned frame with the keyframe, the decision, and fusion or switch
            R.rgbid_covisibility(self.I_kf, self.W_kf, I, W, self.K, self._T_view(), self._sigmaW_view(),
                                 self.counts, None, stream)
            R.rgbid_keyframe_decide(self.counts, self.kf_covisibility, self._T_view(), self.T1, self.T2,
                                    self.d_switch, self.d_ratio, stream)
            R.rgbid_fuse_or_switch_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, self.K, self._T_view(),
                                            self._sigmaW_view(), self.d_switch, self.fuse_intensity, stream)
        elif kf:
            # new keyframe = this frame; poses of frames k-1 and k re-expressed in it
            R.rgbid_compose_pose(self._T_view(), True, self.T1, self.Tnew, stream)   # k_T_{k-1}
            self.T2.copy_(self.Tnew)
            self.T1.copy_(self.eye16)
            R.rgbid_init_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, stream)
        else:
            R.rgbid_fuse_keyframe(self.I_kf, self.W_kf, self.C_kf, I, W, self.K, self._T_view(),
                                  self._sigmaW_view(), self.fuse_intensity, stream)
            self.T2.copy_(self.T1)
            self.T1.copy_(self._T_view())
        self.kfp.build(self.I_kf, self.W_kf, self.K, stream)

    def _capture(self, kf: bool, slot: int):
        """Capture steps 1-5 of a frame of this kind, reading staging pair ``slot`` (nothing runs)."""
        torch = self.torch
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        SI, SW = self._stage[slot]
        with torch.cuda.graph(g):
            self._frame(SI, SW, kf, torch.cuda.current_stream())
        self._graph[(kf, slot)] = g

    def save_state(self, path: str):
        """Write what the next frame depends on to an .npz file: the frame count, the
        keyframe planes, the motion model's poses and the per-frame results so far.
        A tracker built with the same arguments continues after ``load_state`` with
        the bits an uninterrupted run would give."""
        torch = self.torch
        torch.cuda.synchronize(self.device)
        arrays = dict(k=np.array(self.k), I_kf=self.I_kf.cpu().numpy(), W_kf=self.W_kf.cpu().numpy(),
                      C_kf=self.C_kf.cpu().numpy(), T1=self.T1.cpu().numpy(), T2=self.T2.cpu().numpy(),
                      is_kf=self.is_kf[:self.k].copy(), results=self.results[:self.k].cpu().numpy())
        if self.kf_covisibility is not None:
            arrays.update(kf_flags=self.kf_flags[:self.k].cpu().numpy(), ratios=self.ratios[:self.k].cpu().numpy())
        np.savez(path, **arrays)

    def load_state(self, path: str, stream=None):
        """Restore a state written by ``save_state`` and rebuild the keyframe pyramid."""
        torch = self.torch
        d = np.load(path)
        k = int(d["k"])
        if k > self.results.shape[0] or d["I_kf"].shape != tuple(self.I_kf.shape):
            raise ValueError("saved state does not fit this tracker")
        if ("kf_flags" in d) != (self.kf_covisibility is not None):
            raise ValueError("saved state and tracker differ in the keyframe policy")
        for name in ("I_kf", "W_kf", "C_kf", "T1", "T2"):
            getattr(self, name).copy_(torch.from_numpy(d[name]))
        self.results[:k].copy_(torch.from_numpy(d["results"]))
        if self.kf_covisibility is not None:
            self.kf_flags[:k].copy_(torch.from_numpy(d["kf_flags"]))
            self.ratios[:k].copy_(torch.from_numpy(d["ratios"]))
        self.is_kf[:] = False
        self.is_kf[:k] = d["is_kf"]
        if k > 0:
            self.kfp.build(self.I_kf, self.W_kf, self.K, stream)
            if self.ws is None:
                self.ws = R.new_workspace(self.kfp.desc, self.params, self.device)
        self.k = k

    def keyframe_flags(self) -> np.ndarray:
        """Per processed frame: True where the frame became the keyframe (frame 0 included)."""
        flags = self.is_kf[:self.k].copy()
        if self.kf_covisibility is not None:
            flags[1:] = self.kf_flags[1:self.k].cpu().numpy() != 0
        return flags

    def covisibility_ratios(self) -> np.ndarray:
        """Per processed frame k >= 1: its covisibility ratio with the keyframe it was aligned to."""
        return self.ratios[1:self.k].cpu().numpy().astype(np.float64)

    def trajectory(self):
        """World-from-camera poses of the processed frames (frame 0 = identity), on the host."""
        n = self.k
        is_kf = self.keyframe_flags()
        T_world = [np.eye(4)]
        T_wkf = np.eye(4)
        for k in range(1, n):
            r = R.parse_result(self.results[k])
            Tk = T_wkf @ r["T"]
            T_world.append(Tk)
            if is_kf[k]:
                T_wkf = Tk
        return np.stack(T_world)

    def frame_results(self):
        return [R.parse_result(self.results[k]) for k in range(1, self.k)]
