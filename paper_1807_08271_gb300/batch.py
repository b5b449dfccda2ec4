"""Batched alignment executor over ``rgbid_align_batched``.

Holds what one persistent launch needs: the device table of item descriptors
(largest pairs first, so the device queue hands out the longest alignments
before the short ones), the per-item result records, the queue workspace, the
launch shape chosen by the library's autotuner (cached per resolution mix of
the batch), and an optional CUDA graph of the launch.  All alignment work runs
in the library's kernel; this class only arranges arguments.
"""
from __future__ import annotations

import ctypes
import json
import os
from collections import Counter

import numpy as np

from . import rgbid as R


def resolution_key(items, precision: int) -> str:
    """Order-free signature of a batch: the multiset of (width, height, levels,
    iterations) of its pairs plus the plane precision."""
    c = Counter((it["ref"].lv[0].width, it["ref"].lv[0].height, it["levels"], tuple(it["iters"])) for it in items)
    parts = [f"{w}x{h}:L{L}:{'-'.join(map(str, its))}*{n}" for (w, h, L, its), n in sorted(c.items())]
    return f"p{precision}|" + ",".join(parts)


class BatchAligner:
    """Many frame/keyframe alignments in one launch.

    ``items``: list of dicts with ``ref``/``cur`` (rgbid.Pyramid descriptors of
    device pyramids), ``T_init`` (4x4, or None for the identity), ``levels`` and
    ``iters`` (per level, finest first).  Results come back in the given order.
    """

    def __init__(self, items, precision: int = R.PLANES_F32, params: R.AlignParams | None = None,
                 device="cuda", tune_cache: str | None = None, planner_factory=None):
        import torch
        self.precision = precision
        self.params = params if params is not None else R.rgbid_default_params()
        self.items = list(items)
        self.n = len(self.items)
        self.results = R.result_tensor(self.n, device=device)
        self.workspace = torch.zeros(R.rgbid_align_batched_workspace_bytes(), dtype=torch.uint8, device=device)
        self.tune_cache_path = tune_cache
        self._cache = self._load_cache()
        self.config: R.BatchConfig | None = None
        self.graph = None
        # largest first: level-0 pixels times finest-level iterations approximates the work
        order = sorted(range(self.n), key=lambda i: -self._cost(self.items[i]))
        table = (R.BatchItem * max(1, self.n))()
        base = self.results.data_ptr()
        for slot, i in enumerate(order):
            it = self.items[i]
            d = table[slot]
            d.ref = it["ref"]
            d.cur = it["cur"]
            T = np.eye(4) if it.get("T_init") is None else np.asarray(it["T_init"], dtype=np.float64)
            for k, v in enumerate(T.reshape(16)):
                d.T_init[k] = float(v)
            d.levels = int(it["levels"])
            its = list(it["iters"])
            for l in range(R.MAX_LEVELS):
                d.iters[l] = int(its[l]) if l < len(its) else 0
            d.result = base + i * R.RESULT_BYTES
            code = R.rgbid_batch_check_item(d, precision)
            if code != R.OK:
                raise R.RgbidError(f"rgbid_batch_check_item(item {i})", code)
        self.order = order
        raw = np.frombuffer(bytes(table), dtype=np.uint8)[: self.n * ctypes.sizeof(R.BatchItem)]
        self.d_items = torch.from_numpy(raw.copy()).to(device)
        self.key = resolution_key(self.items, precision)
        # with a learned planner the pristine table stays in d_src and every run
        # writes the planned items (start pose, skipped levels) into d_items
        self.planner = planner_factory(self.n, precision) if planner_factory is not None else None
        self.d_src = self.d_items.clone() if self.planner is not None else None
        if self.planner is not None:
            self.key += "|learned"

    @staticmethod
    def _cost(it) -> float:
        L0 = it["ref"].lv[0]
        return float(L0.width * L0.height) * (1.0 + float(sum(it["iters"])))

    # ------------------------------------------------------------------ shape tuning
    def _load_cache(self) -> dict:
        if self.tune_cache_path and os.path.exists(self.tune_cache_path):
            with open(self.tune_cache_path) as f:
                return json.load(f)
        return {}

    def _store_cache(self):
        if self.tune_cache_path:
            tmp = self.tune_cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self._cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.tune_cache_path)

    def tune(self, reps: int = 3, force: bool = False, stream=None) -> R.BatchConfig:
        """Pick the launch shape: the cached one for this resolution mix, else run
        the library's autotuner on this batch and cache its answer."""
        if self.planner is not None:
            self.planner.plan(self.d_src, self.d_items, stream)    # tune on the planned work
        hit = self._cache.get(self.key)
        if hit is not None and not force:
            self.config = R.BatchConfig(hit["cluster"], hit["rows_per_warp"], hit["n_clusters"], 0)
            return self.config
        cfg, ms = R.rgbid_batch_autotune(self.d_items, self.n, self.precision, self.params, self.workspace, reps,
                                         stream)
        self._cache[self.key] = dict(cluster=cfg.cluster, rows_per_warp=cfg.rows_per_warp,
                                     n_clusters=cfg.n_clusters, ms=ms)
        self._store_cache()
        self.config = cfg
        return cfg

    # ------------------------------------------------------------------ execution
    def run(self, stream=None):
        """Enqueue the batch: one kernel launch (plus, with a learned planner, the
        network's input packing, forward pass and plan before it)."""
        if self.planner is not None:
            self.planner.plan(self.d_src, self.d_items, stream)
        R.rgbid_align_batched(self.d_items, self.n, self.precision, self.params, self.config, self.workspace,
                              stream)

    def capture(self):
        """Capture the launch in a CUDA graph (after the shape is fixed) for replay()."""
        import torch
        R.rgbid_batch_resident_clusters(self.precision, self.config)   # set-up happens outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def result(self, i: int) -> dict:
        return R.parse_result(self.results[i])

    def all_results(self) -> list[dict]:
        host = self.results.cpu()
        return [R.parse_result(host[i]) for i in range(self.n)]


def main(argv=None):
    """Align a seeded batch of same-size synthetic pairs with a given launch shape
    and print the per-launch time (a command-line check of the batched kernel)."""
    import argparse

    import torch

    from . import synth
    ap = argparse.ArgumentParser(prog="python -m paper_1807_08271_gb300.batch")
    ap.add_argument("--size", default="1280x960", help="pair resolution WxH")
    ap.add_argument("--pairs", type=int, default=16)
    ap.add_argument("--cluster", type=int, default=8)
    ap.add_argument("--rows", type=int, default=1)
    ap.add_argument("--runs", type=int, default=3)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--precision", choices=["f32", "bf16"], default="f32")
    a = ap.parse_args(argv)
    w, h = (int(v) for v in a.size.split("x"))
    prec = R.PLANES_BF16_F16 if a.precision == "bf16" else R.PLANES_F32
    pairs = synth.make_batch(seed=a.seed, n=a.pairs, sizes=((w, h),))
    keep, items = [], []
    for p in pairs:
        PA = R.DevicePyramid(w, h, p["levels"], prec).build(torch.from_numpy(p["I_A"]).cuda(),
                                                            torch.from_numpy(p["W_A"]).cuda(), p["K"])
        PB = R.DevicePyramid(w, h, p["levels"], prec).build(torch.from_numpy(p["I_B"]).cuda(),
                                                            torch.from_numpy(p["W_B"]).cuda(), p["K"])
        keep += [PA, PB]
        items.append(dict(ref=PA.desc, cur=PB.desc, T_init=p["T_init"], levels=p["levels"], iters=p["iters"]))
    B = BatchAligner(items, precision=prec)
    B.config = R.BatchConfig(a.cluster, a.rows, 0, 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(a.runs):
        e0.record()
        B.run()
        e1.record()
        torch.cuda.synchronize()
        print(f"run {k}: {e0.elapsed_time(e1):.3f} ms")
    res = B.all_results()
    print("status", sorted(set(r["status"] for r in res)), "iterations", res[0]["iters_done"])


if __name__ == "__main__":
    main()
