"""Write tests/golden/seq640_oracle.json: the FP64 oracle's tracking of the seeded
300-frame 640x480 room sequence (seed 0; 4 levels, [5, 5, 5, 10] iterations
finest first, keyframe switch every 20 frames, every other frame fused), once
on the float32 planes and once on the reduced-precision pyramids (bfloat16
intensity, binary16 inverse depth).  Per frame it stores the alignment's pose
kf_T_k, the world pose, status, iteration count and final robust parameters;
for the final keyframe it stores I, W and C on a 16-pixel grid (offset 3) and
the plane sums over the pixels fused at least once.  Calls only oracle/ and the
seeded input generator; the two plane sets run in two spawned processes.

With --covisibility THR it writes tests/golden/seq640_covis_oracle.json
instead: the first --frames frames of the same sequence on the float32 planes,
tracked with the keyframe switched whenever the covisibility ratio of the
aligned frame with its keyframe falls below THR, with each frame's ratio and
switch decision.

    python tests/golden/make_seq_oracle_poses.py [--frames N] [--covisibility THR]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

GRID = (slice(3, None, 16), slice(3, None, 16))
SEQ_FRAMES = 300


def _track(args):
    import oracle as O
    from paper_1807_08271_gb300 import synth
    reduced, n, covis = args
    # the benchmark's 300-frame sequence (its trajectory depends on its length), first n frames tracked
    seq = synth.render_sequence(0, n_frames=SEQ_FRAMES)
    o = O.track_sequence(seq["I"], seq["W"], seq["K"], levels=4, iters=(5, 5, 5, 10),
                         kf_every=None if covis is not None else 20, reduced=reduced, kf_covisibility=covis,
                         n_frames=n)
    frames = []
    for k, r in enumerate(o["results"], start=1):
        frames.append({"k": k, "T": r["T"].reshape(-1).tolist(), "T_world": o["T_world"][k].reshape(-1).tolist(),
                       "status": int(r["status"]), "iters_done": int(r["iters_done"]),
                       "n_valid": [int(v) for v in r["n_valid"]],
                       "sigma": [float(s) for s in r["robust"]["sigma"]],
                       "nu": [float(v) for v in r["robust"]["nu"]]})
        if covis is not None:
            frames[-1]["covisibility"] = float(o["covisibility"][k - 1])
            frames[-1]["switch"] = bool(o["covisibility"][k - 1] < covis)
    I, W, C = o["keyframe"]
    fused = C > 1
    kf = {"grid": "rows 3::16, columns 3::16", "I": I[GRID].tolist(), "W": W[GRID].tolist(), "C": C[GRID].tolist(),
          "n_fused": int(fused.sum()), "sum_W_fused": float(W[fused].sum()), "sum_I_fused": float(I[fused].sum()),
          "sum_C_fused": float(C[fused].sum())}
    return reduced, {"frames": frames, "keyframe": kf}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--covisibility", type=float, default=None)
    a = ap.parse_args()
    if a.covisibility is not None:
        _, res = _track((False, a.frames, a.covisibility))
        out = {"config": f"640x480 room sequence, seed 0, first {a.frames} of its 300 frames, 4 levels, iterations [5, 5, 5, 10] "
                         f"finest first, keyframe switch when the covisibility ratio falls below {a.covisibility}, "
                         "FP64 oracle (oracle.track_sequence)", "threshold": a.covisibility, "fp32_planes": res}
        with open(os.path.join(HERE, "seq640_covis_oracle.json"), "w") as f:
            json.dump(out, f)
        return
    with mp.get_context("spawn").Pool(2) as pool:
        res = dict(pool.map(_track, [(False, a.frames, None), (True, a.frames, None)]))
    out = {"config": f"640x480 room sequence, seed 0, {a.frames} frames, 4 levels, iterations [5, 5, 5, 10] finest "
                     "first, keyframe every 20 frames, FP64 oracle (oracle.track_sequence)",
           "fp32_planes": res[False], "reduced_planes": res[True]}
    with open(os.path.join(HERE, "seq640_oracle.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
