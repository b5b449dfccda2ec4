"""Pins of the oracle's treatment of non-finite input (reading R19: a pixel
whose I or W is not a finite number carries no measurement).

Checked against hand arithmetic on a 2x2 block, invariants that hold for any
input, and the locality of the bilinear taps in fusion, so that a non-finite
value leaking into a mean, a validity test or a fusion update fails a test."""
import numpy as np

import oracle as O
from paper_1807_08271_gb300 import synth


def test_pyramid_block_with_nonfinite_children_by_hand():
    I = np.full((4, 4), 0.5)
    W = np.full((4, 4), 0.4)
    # the top-left 2x2 block: (0,0) valid, (0,1) NaN intensity, (1,0) +inf depth, (1,1) valid
    I[0, 0], I[0, 1], I[1, 0], I[1, 1] = 0.2, np.nan, 0.6, 0.4
    W[0, 0], W[0, 1], W[1, 0], W[1, 1] = 0.5, 0.8, np.inf, 0.25
    pyr = O.build_pyramid(I, W, (4.0, 4.0, 1.5, 1.5), 2)
    L0, L1 = pyr
    assert L0.I[0, 1] == 0.0 and L0.W[0, 1] == 0.0          # NaN intensity: a hole with I = 0
    assert L0.I[1, 0] == 0.6 and L0.W[1, 0] == 0.0          # +inf depth: a hole, I kept
    assert L1.I[0, 0] == ((0.2 + 0.0) + (0.6 + 0.4)) / 4     # 0.3, in the (a+b)+(c+d) order of R1
    assert L1.W[0, 0] == (0.5 + 0.25) / 2                    # mean of the two measurements
    assert L1.I[0, 1] == 0.5 and L1.W[0, 1] == 0.4           # untouched blocks


def test_pyramid_of_any_input_is_finite_and_holes_are_the_nonfinite_pixels():
    rng = np.random.default_rng(5)
    h, w = 48, 64
    I = rng.random((h, w))
    W = rng.uniform(0.2, 2.0, (h, w))
    bad = rng.random((h, w))
    I[bad < 0.03] = np.nan
    I[(bad >= 0.03) & (bad < 0.05)] = np.inf
    I[(bad >= 0.05) & (bad < 0.06)] = -np.inf
    W[(bad >= 0.06) & (bad < 0.09)] = np.nan
    W[(bad >= 0.09) & (bad < 0.11)] = np.inf
    W[(bad >= 0.11) & (bad < 0.12)] = -np.inf
    pyr = O.build_pyramid(I, W, synth.pinhole(w, h), 3)
    for L in pyr:
        assert np.all(np.isfinite(L.I)) and np.all(np.isfinite(L.W)) and np.all(L.W >= 0)
    assert np.array_equal(pyr[0].W > 0, bad >= 0.12)
    # the reduced-precision form rounds the same finite levels
    for L in O.build_pyramid_reduced(I, W, synth.pinhole(w, h), 3):
        assert np.all(np.isfinite(L.I)) and np.all(np.isfinite(L.W))


def test_alignment_with_nonfinite_pixels_stays_on_ground_truth():
    p = synth.make_pair(0)
    rng = np.random.default_rng(9)
    IB, WB = p["I_B"].astype(np.float64), p["W_B"].astype(np.float64)
    IA, WA = p["I_A"].astype(np.float64), p["W_A"].astype(np.float64)
    for img, val in ((IB, np.nan), (WB, np.inf), (IB, -np.inf), (WA, np.nan), (IA, np.inf)):
        m = rng.random(img.shape) < 0.01
        img[m] = val
    A = O.build_pyramid(IA, WA, p["K"], 3)
    B = O.build_pyramid(IB, WB, p["K"], 3)
    r = O.align(A, B, None, O.AlignParams())
    assert r["status"] == O.OK and np.all(np.isfinite(r["T"])) and np.all(np.isfinite(r["H"]))
    E = O.se3_inv(p["T_gt"]) @ r["T"]
    assert np.linalg.norm(O.so3_log(E[:3, :3])) < 2e-3 and np.linalg.norm(E[:3, 3]) < 2e-3


def test_fusion_never_reads_a_nonfinite_tap():
    p = synth.make_pair(3, noise=True)
    I, W = p["I_A"].astype(np.float64), p["W_A"].astype(np.float64)
    C = np.ones_like(W)
    clean = O.fuse(I, W, C, I, W, p["K"], np.eye(4), 1e-3)
    rng = np.random.default_rng(2)
    S = rng.random(W.shape) < 0.02
    Ik, Wk = I.copy(), W.copy()
    half = rng.random(W.shape) < 0.5
    Ik[S & half] = np.nan
    Wk[S & ~half] = np.inf
    I2, W2, C2, gate = O.fuse(I, W, C, Ik, Wk, p["K"], np.eye(4), 1e-3)
    assert np.all(np.isfinite(I2)) and np.all(np.isfinite(W2)) and np.all(np.isfinite(C2))
    # at the identity every keyframe pixel's 2x2 tap block contains the pixel itself
    assert not gate[S].any()
    assert np.array_equal(W2[S], W[S]) and np.array_equal(I2[S], I[S]) and np.array_equal(C2[S], C[S])
    # pixels whose 3x3 neighbourhood avoids S fuse exactly as with the clean frame
    near = np.zeros_like(S)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            near |= np.roll(np.roll(S, dy, axis=0), dx, axis=1)
    far = ~near
    far[0, :] = far[-1, :] = far[:, 0] = far[:, -1] = False
    assert gate[far].sum() > 0.5 * far.sum()
    for got, want in zip((I2, W2, C2, gate), clean):
        assert np.array_equal(got[far], want[far])


def test_fusion_skips_nonfinite_keyframe_pixels():
    p = synth.make_pair(3, noise=True)
    I, W = p["I_A"].astype(np.float64), p["W_A"].astype(np.float64)
    C = np.ones_like(W)
    Wkf, Ikf = W.copy(), I.copy()
    Wkf[10:14, 20:30] = np.inf
    Ikf[30:32, 40:50] = np.nan
    I2, W2, C2, gate = O.fuse(Ikf, Wkf, C, I, W, p["K"], np.eye(4), 1e-3)
    assert not gate[10:14, 20:30].any() and not gate[30:32, 40:50].any()
    assert np.all(np.isinf(W2[10:14, 20:30])) and np.all(np.isnan(I2[30:32, 40:50]))   # left as given
    assert np.array_equal(C2[10:14, 20:30], C[10:14, 20:30])
    other = np.ones_like(gate)
    other[10:14, 20:30] = other[30:32, 40:50] = False
    assert np.all(np.isfinite(W2[other])) and np.all(np.isfinite(I2[other])) and gate.sum() > 0.5 * (W > 0).sum()
