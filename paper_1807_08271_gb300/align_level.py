"""Align one pyramid level of the 640x480 sequence's first frame pair on its own.

``python -m paper_1807_08271_gb300.align_level --level 3 --iters 10 --reps 5`` builds
both frames' 4-level pyramids, makes a one-level pyramid of level ``--level`` and runs
``rgbid_align`` on it ``--reps`` times: one launch of the kernel that level gets in the
sequence (80x60: the level kernel), between the initialisation and the closing launch.
A way to time or profile one level's kernel in isolation.  160x120 and larger levels
run in the split kernel (a cooperative launch), which ncu does not profile.
"""
from __future__ import annotations

import argparse


def main(argv=None):
    import torch

    from . import rgbid as R
    from . import synth

    ap = argparse.ArgumentParser(prog="python -m paper_1807_08271_gb300.align_level")
    ap.add_argument("--level", type=int, default=3, help="pyramid level of the 640x480 frames (0 = finest)")
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args(argv)
    if not 0 <= a.level < 4:
        ap.error("--level must be 0..3")
    seq = synth.render_sequence(0, n_frames=2)
    full = [R.DevicePyramid(640, 480, 4).build(torch.from_numpy(seq["I"][k]).cuda(),
                                               torch.from_numpy(seq["W"][k]).cuda(), seq["K"]) for k in (0, 1)]
    one = []
    for p in full:
        d = R.Pyramid()
        d.levels = 1
        d.precision = p.desc.precision
        d.lv[0] = p.desc.lv[a.level]
        one.append(d)
    params = R.rgbid_default_params(levels=1, iters=[a.iters])
    ws = R.new_workspace(one[0], params)
    res = R.result_tensor()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        R.rgbid_align(one[0], one[1], None, params, ws, res)
    e1.record()
    torch.cuda.synchronize()
    g = R.parse_result(res)
    L = one[0].lv[0]
    print(f"level {a.level} ({L.width}x{L.height}), {a.iters} iterations, {R.rgbid_align_launches(one[0], params)} "
          f"launches: {e0.elapsed_time(e1) / a.reps:.3f} ms per alignment, status {g['status']}, "
          f"iterations {g['iters_done']}")
    return 0 if g["status"] == R.OK else 1


if __name__ == "__main__":
    raise SystemExit(main())
