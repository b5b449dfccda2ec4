"""FP64 CPU oracle for the RGBiD-SLAM dense alignment and keyframe fusion.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link anything under ``oracle/``: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA path; the only shared module is the seeded input generator, which holds
none of the method's arithmetic.

Every function restates the paper's definition in plain numpy float64, one
formula per step, with no blocking, fusion or reordering.  See
``rgbid_oracle`` for the per-function citations (paper section and equation
labels) and the readings taken where the paper is silent or garbled.
"""
from .rgbid_oracle import *  # noqa: F401,F403
from . import cnn_oracle  # noqa: F401  (the learned initialiser's network)
