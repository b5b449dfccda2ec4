"""The learned initialiser: network state on the device, training steps, and the
confidence-gated plan that starts batched alignments from the network's pose.

Argument marshalling over the ``rgbid_net_*`` entry points of ``librgbid``:
every pass of the network (forward, backward, loss, Adam, input packing, plan)
runs in the library's kernels.  The network is described in ``include/rgbid.h``.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import rgbid as R

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "init_net.npz")


def so3_log_np(R) -> np.ndarray:
    """Rotation vector of a rotation matrix (label conversion on the host)."""
    R = np.asarray(R, dtype=np.float64)
    c = np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)
    th = float(np.arccos(c))
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    if th < 1e-6:
        return 0.5 * v
    if np.pi - th < 1e-4:
        # near pi: axis from the diagonal of (R + I) / 2
        B = (R + np.eye(3)) / 2.0
        k = int(np.argmax(np.diag(B)))
        a = B[:, k] / np.sqrt(B[k, k])
        return th * a / np.linalg.norm(a)
    return th / (2.0 * np.sin(th)) * v


def twist_of_pose(T) -> np.ndarray:
    """(t, w) of the decoupled pose T = [exp([w]x), t; 0, 1] (the network's target)."""
    T = np.asarray(T, dtype=np.float64)
    return np.concatenate([T[:3, 3], so3_log_np(T[:3, :3])])


class InitNet:
    """Parameters (float32 master copy), Adam moments and a workspace for
    batches of up to ``max_batch`` inputs."""

    def __init__(self, max_batch: int = 256, seed: int = 0, device="cuda"):
        import torch
        self.device = torch.device(device)
        P = R.rgbid_net_param_count()
        self.params = torch.empty(P, dtype=torch.float32, device=self.device)
        R.rgbid_net_init(self.params, seed)
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.max_batch = max_batch
        self.ws = torch.empty(R.rgbid_net_workspace_bytes(max_batch), dtype=torch.uint8, device=self.device)
        self.y = torch.zeros((max_batch, R.NET_OUT), dtype=torch.float32, device=self.device)
        self.dy = torch.zeros_like(self.y)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0
        self.meta = {}

    def forward(self, x, n: int):
        """y [n, 7] (a view of the net's output buffer) for inputs x [n, 60, 80, 4] bf16."""
        assert 1 <= n <= self.max_batch and x.is_contiguous()
        R.rgbid_net_forward(self.params, x, n, self.y, self.ws)
        return self.y[:n]

    def train_step(self, x, target, n: int, lr: float):
        """Forward, loss, backward and one Adam step; returns the loss (device tensor)."""
        self.forward(x, n)
        R.rgbid_net_loss(self.y, target, n, self.dy, self.loss)
        R.rgbid_net_backward(self.params, x, n, self.dy, self.grad, self.ws)
        self.step += 1
        R.rgbid_net_adam(self.params, self.grad, self.m, self.v, self.step, lr)
        return self.loss

    def save(self, path: str, **meta):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        self.meta.update(meta)
        np.savez_compressed(path, params=self.params.cpu().numpy(), meta=json.dumps(self.meta))

    @classmethod
    def load(cls, path: str = WEIGHTS, max_batch: int = 256, device="cuda") -> "InitNet":
        import torch
        d = np.load(path)
        net = cls(max_batch=max_batch, device=device)
        p = torch.from_numpy(d["params"].astype(np.float32))
        if p.numel() != net.params.numel():
            raise ValueError("weights do not match the network's parameter layout")
        net.params.copy_(p)
        net.meta = json.loads(str(d["meta"]))
        return net


class LearnedPlanner:
    """For a batch of n items: network inputs from each pair's 80x60 pyramid
    level, the forward pass, and the plan kernel that copies the pristine items
    and, for an item whose predicted log-variance is below ``thresholds[k - 1]``
    (largest such k), starts it from the proposal with its k coarsest levels
    skipped; other items run the plain alignment."""

    def __init__(self, net: InitNet, n: int, precision: int, thresholds):
        import torch
        assert n <= net.max_batch, "planner batch larger than the network's workspace"
        self.net, self.n, self.precision = net, n, precision
        self.thresholds = [float(t) for t in thresholds]
        self.x = torch.zeros((max(1, n), R.NET_IN_H, R.NET_IN_W, R.NET_IN_C), dtype=torch.bfloat16,
                             device=net.device)
        self.skipped = torch.zeros(max(1, n), dtype=torch.int32, device=net.device)

    def plan(self, d_src, d_dst, stream=None):
        R.rgbid_net_inputs(d_src, self.n, self.precision, self.x, stream)
        R.rgbid_net_forward(self.net.params, self.x, self.n, self.net.y, self.net.ws, stream)
        R.rgbid_net_plan(self.net.y, self.n, self.thresholds, d_src, d_dst, self.skipped, stream)


class LearnedAligner:
    """Frame pairs one at a time (the per-pair alignment) with the learned start:
    the network's inputs are packed from the pair's 80x60 levels, the forward
    pass and the plan run on the device, and rgbid_align reads the planned start
    pose and per-level iteration counts from device memory, so nothing waits for
    the host.  ``levels``/``iters`` give the plain schedule (the fallback).

    The pairs' descriptors live in a device table uploaded once by
    ``set_pairs`` (a copy from pageable memory would stall the stream if it
    were made per alignment); ``align(slot, ...)`` copies the pair's item into a
    fixed device slot and, with ``graphs=True`` (the default), replays one CUDA
    graph of the network's launches (input packing, the forward GEMMs and their
    split-K reductions, the plan) on it: a dozen small launches whose enqueue
    would otherwise cost more than their work."""

    def __init__(self, net: InitNet, thresholds, precision: int = R.PLANES_F32, levels: int = 4,
                 iters=(5, 5, 5, 10), params: R.AlignParams | None = None, graphs: bool = True):
        import torch
        self.net, self.precision = net, precision
        self.thresholds = [float(t) for t in thresholds]
        self.levels, self.iters = levels, list(iters)
        self.params = params if params is not None else R.rgbid_default_params(levels=levels, iters=iters)
        dev = net.device
        self.x = torch.zeros((1, R.NET_IN_H, R.NET_IN_W, R.NET_IN_C), dtype=torch.bfloat16, device=dev)
        self.skipped = torch.zeros(1, dtype=torch.int32, device=dev)
        self.d_src = None
        self.n = 0
        self.graphs = graphs
        self._graph = None
        import ctypes
        size = ctypes.sizeof(R.BatchItem)
        # the current pair's item (input of the network and of the plan) and its plan
        self.d_one = torch.zeros(size, dtype=torch.uint8, device=dev)
        self.d_plan = torch.zeros(size, dtype=torch.uint8, device=dev)

    def set_pairs(self, pairs):
        """pairs: list of (ref, cur) pyramid descriptors; uploads their items."""
        import ctypes
        import torch
        n = len(pairs)
        table = (R.BatchItem * max(1, n))()
        for i, (ref, cur) in enumerate(pairs):
            it = table[i]
            it.ref, it.cur = ref, cur
            for k in (0, 5, 10, 15):
                it.T_init[k] = 1.0
            it.levels = self.levels
            for l in range(R.MAX_LEVELS):
                it.iters[l] = self.iters[l] if l < len(self.iters) else 0
        raw = np.frombuffer(bytes(table), dtype=np.uint8)[: n * ctypes.sizeof(R.BatchItem)].copy()
        self.d_src = torch.from_numpy(raw).to(self.net.device)
        self.pairs = list(pairs)
        self.n = n

    def _plan(self, stream=None):
        """The network on the item in d_one and the plan into d_plan (no host state)."""
        R.rgbid_net_inputs(self.d_one, 1, self.precision, self.x, stream)
        R.rgbid_net_forward(self.net.params, self.x, 1, self.net.y, self.net.ws, stream)
        R.rgbid_net_plan(self.net.y, 1, self.thresholds, self.d_one, self.d_plan, self.skipped, stream)

    def align(self, slot: int, workspace, result, stream=None):
        """Enqueue the learned-start alignment of pair ``slot`` into ``result``."""
        import ctypes
        import torch
        assert 0 <= slot < self.n
        size = ctypes.sizeof(R.BatchItem)
        s = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            self.d_one.copy_(self.d_src[slot * size:(slot + 1) * size], non_blocking=True)
            if self.graphs:
                if self._graph is None:
                    torch.cuda.synchronize()
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g):
                        self._plan()
                    self._graph = g
                self._graph.replay()
            else:
                self._plan(s)
        self.params.level_iters = self.d_plan.data_ptr() + R.BatchItem.iters.offset
        ref, cur = self.pairs[slot]
        R.rgbid_align(ref, cur, _DevicePtr(self.d_plan.data_ptr() + R.BatchItem.T_init.offset), self.params,
                      workspace, result, stream)


class _DevicePtr:
    """A raw device address that rgbid.rgbid_align accepts as an on-device T_init."""
    is_cuda = True

    def __init__(self, ptr: int):
        self._p = ptr

    def data_ptr(self) -> int:
        return self._p


def main(argv=None):
    """Time training steps (random inputs) and batch-1 inference of the network
    (a command-line check of the network kernels)."""
    import argparse

    import torch
    ap = argparse.ArgumentParser(prog="python -m paper_1807_08271_gb300.learned")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--steps", type=int, default=20)
    a = ap.parse_args(argv)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    net = InitNet(max_batch=a.batch, seed=1)
    x = (torch.randn(a.batch, R.NET_IN_H, R.NET_IN_W, R.NET_IN_C, device="cuda", generator=gen) * 0.5)
    x = x.to(torch.bfloat16).contiguous()
    t = torch.randn(a.batch, 6, device="cuda", generator=gen)
    for _ in range(5):
        net.train_step(x, t, a.batch, 1e-3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        net.train_step(x, t, a.batch, 1e-3)
    e1.record()
    torch.cuda.synchronize()
    print(f"training step (batch {a.batch}): {e0.elapsed_time(e1) / a.steps:.3f} ms, loss {float(net.loss):.4f}")
    x1 = x[:1].contiguous()
    for _ in range(5):
        net.forward(x1, 1)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        net.forward(x1, 1)
    e1.record()
    torch.cuda.synchronize()
    print(f"forward (batch 1): {e0.elapsed_time(e1) / a.steps:.3f} ms")


if __name__ == "__main__":
    main()
