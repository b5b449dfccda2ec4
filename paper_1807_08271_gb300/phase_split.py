"""Phase table of the split kernel on a 640x480 pair of the sequence's camera.

``RGBID_LIBRARY=phases python -m paper_1807_08271_gb300.phase_split`` loads the
phase-stamped build (librgbid_phases.so, -DRGBID_PHASE_STAMPS), aligns one synthetic
640x480 pair 30 times with the sequence's schedule and prints, per split-kernel level,
the median time of each phase of iterations 1-4 from the stamps that thread 0 of the
cluster's CTA 0 and of the first helper CTA write (rgbid_debug_phase_stamps).  Where ncu
does not profile the split kernel's cooperative launch, this is its phase evidence.
"""
from __future__ import annotations

import os

import numpy as np

CLUSTER = ["wait for the helpers' partials", "sum the partials, solve, update", "publish the pose",
           "sample residuals", "counts round", "10 fixed-point rounds", "nu sums, gathered to CTA 0",
           "bisection, publish the parameters"]
HELPER = [("sees the pose after its publication", 9, 3), ("pixel pass", 10, 9),
          ("sees the parameters after their publication", 11, 8), ("accumulate and post", 12, 11)]


def main(argv=None):
    import argparse

    import torch

    from . import rgbid as R
    from . import synth

    ap = argparse.ArgumentParser(prog="RGBID_LIBRARY=phases python -m paper_1807_08271_gb300.phase_split")
    ap.add_argument("--reps", type=int, default=30)
    a = ap.parse_args(argv)
    if os.environ.get("RGBID_LIBRARY") != "phases":
        ap.error("run with RGBID_LIBRARY=phases (the phase-stamped build)")
    pair = synth.make_pair(4, 640, 480, K=(525.0, 525.0, 319.5, 239.5), max_angle_deg=2.0, max_trans=0.03)
    P = [R.DevicePyramid(640, 480, 4).build(torch.from_numpy(pair[i]).cuda(), torch.from_numpy(pair[w]).cuda(),
                                            pair["K"]) for i, w in (("I_A", "W_A"), ("I_B", "W_B"))]
    params = R.rgbid_default_params(levels=4, iters=[5, 5, 5, 10])
    ws = R.new_workspace(P[0].desc, params)
    res = R.result_tensor()
    print(f"launches per alignment: {R.rgbid_align_launches(P[0].desc, params)}")
    runs = []
    for rep in range(a.reps):
        R.rgbid_align(P[0].desc, P[1].desc, None, params, ws, res)
        st = R.rgbid_debug_phase_stamps()
        if st is None:
            raise SystemExit("the loaded library has no phase stamps")
        if rep >= min(5, a.reps - 1):
            runs.append(st.astype(np.float64))
    A = np.stack(runs)   # [runs, level, iteration, phase]
    for level, name in ((2, "160x120"), (1, "320x240"), (0, "640x480")):
        L = A[:, level]
        if not np.any(L[:, 1:5, 0]):
            continue
        print(f"level {level} ({name}), us, iterations 1-4 (median over {A.shape[0]} alignments)")
        for k, nm in enumerate(CLUSTER):
            d = [np.median(L[:, it, k + 1] - L[:, it, k]) / 1e3 for it in range(1, 5)]
            print(f"  {nm:44s} " + " ".join(f"{x:6.2f}" for x in d))
        d = [np.median(L[:, it + 1, 0] - L[:, it, 0]) / 1e3 for it in range(1, 4)]
        print(f"  {'iteration':44s} " + " ".join(f"{x:6.2f}" for x in d))
        for nm, k1, k0 in HELPER:
            d = [np.median(L[:, it, k1] - L[:, it, k0]) / 1e3 for it in range(1, 5)]
            print(f"  helper {nm:37s} " + " ".join(f"{x:6.2f}" for x in d))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
