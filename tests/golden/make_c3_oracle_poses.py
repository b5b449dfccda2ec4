"""Write tests/golden/c3_oracle_poses.json: the FP64 oracle's alignment of every
pair of the 64-pair loop-closure batch (seed 0: 16 pairs each at 320x240,
640x480, 960x720 and 1280x960, shuffled; relative poses up to 10 deg / 20 cm;
started from the ground truth perturbed by up to 2 deg / 3 cm; levels
1 + floor(log2(W/80)), 10 iterations at the coarsest level and 5 elsewhere).
Calls only oracle/ and the seeded input generator.  The pairs are aligned in
worker processes (spawned, one pair per task); every pair's arithmetic is the
single-threaded oracle's, so the result does not depend on the worker count.

    python tests/golden/make_c3_oracle_poses.py [--workers N] [--reduced]

With --reduced the pyramids are those of the reduced-precision form (bfloat16
intensity, binary16 inverse depth) and the output is c3_oracle_poses_reduced.json.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402


def _align(args):
    import oracle as O
    i, p, reduced = args
    build = O.build_pyramid_reduced if reduced else O.build_pyramid
    A = build(p["I_A"], p["W_A"], p["K"], p["levels"])
    B = build(p["I_B"], p["W_B"], p["K"], p["levels"])
    o = O.align(A, B, p["T_init"], O.AlignParams(levels=p["levels"], iters=tuple(p["iters"])))
    return i, {"width": p["width"], "height": p["height"], "levels": p["levels"], "iters": list(p["iters"]),
               "T": o["T"].reshape(-1).tolist(), "T_gt": p["T_gt"].reshape(-1).tolist(),
               "T_init": np.asarray(p["T_init"]).reshape(-1).tolist(), "status": int(o["status"]),
               "iters_done": int(o["iters_done"]), "n_valid": [int(v) for v in o["n_valid"]],
               "sigma": [float(s) for s in o["robust"]["sigma"]], "nu": [float(v) for v in o["robust"]["nu"]]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--reduced", action="store_true")
    a = ap.parse_args()
    from paper_1807_08271_gb300 import synth
    pairs = synth.make_batch(seed=0, n=64)
    # largest first, so the long alignments do not end up last
    order = sorted(range(len(pairs)), key=lambda i: -pairs[i]["width"])
    tasks = [(i, pairs[i], a.reduced) for i in order]
    out = {"config": "64-pair loop-closure batch, seed 0 (synth.make_batch); FP64 oracle per pair from T_init"
                     + ("; reduced-precision pyramids (bfloat16 I, binary16 W)" if a.reduced else ""),
           "pairs": {}}
    with mp.get_context("spawn").Pool(a.workers) as pool:
        for i, rec in pool.imap_unordered(_align, tasks):
            out["pairs"][str(i)] = rec
            print(i, rec["width"], flush=True)
    out["pairs"] = {k: out["pairs"][k] for k in sorted(out["pairs"], key=int)}
    name = "c3_oracle_poses_reduced.json" if a.reduced else "c3_oracle_poses.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
