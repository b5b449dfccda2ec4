"""Write tests/golden/c0_oracle_poses.json: the FP64 oracle's alignment of the
160x120 pair of every seed 0..99 (3 levels, [5, 5, 10] iterations finest first,
identity start), with the ground truth.  Calls only oracle/ and the seeded input
generator.

    python tests/golden/make_c0_oracle_poses.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1807_08271_gb300 import synth  # noqa: E402


def main():
    out = {"config": "160x120 pairs, seeds 0..99, 3 levels, iterations [5, 5, 10] finest first, identity start",
           "seeds": {}}
    for seed in range(100):
        p = synth.make_pair(seed)
        A = O.build_pyramid(p["I_A"], p["W_A"], p["K"], 3)
        B = O.build_pyramid(p["I_B"], p["W_B"], p["K"], 3)
        o = O.align(A, B, None, O.AlignParams())
        out["seeds"][str(seed)] = {"T": o["T"].reshape(-1).tolist(), "T_gt": p["T_gt"].reshape(-1).tolist(),
                                   "status": int(o["status"]), "iters_done": int(o["iters_done"]),
                                   "n_valid": [int(v) for v in o["n_valid"]]}
        print(seed, flush=True)
    with open(os.path.join(HERE, "c0_oracle_poses.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
