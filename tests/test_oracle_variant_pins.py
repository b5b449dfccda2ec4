"""Pins of the oracle's paper variants around the alignment path:

* the bilateral filter and the covariance iteration ("Dense motion estimation",
  the paragraph after the update rule: Sigma = H_filt^-1 from one more,
  non-updating iteration with {I_A, W_A} bilateral-filtered before their
  gradients are taken; reading R20);
* the dense covisibility ratio ("Dense frame covisibility ratio": S_H, S_V, the
  3 sigma_W visibility test, the minimum over both directions; reading R21);
* the literal warp-then-downsample mode ("Iterative optimisation": the warped
  images downsampled to the current level; reading R22).

Each is checked against closed forms, library routines (scipy's correlation),
independent per-pixel loops, or special cases that reduce to the plain method.
"""
import numpy as np
import pytest
import scipy.ndimage

import oracle as O
from paper_1807_08271_gb300 import synth

ROB = dict(mu=[0.004, -0.0015], sigma=[0.045, 0.012], nu=[3.5, 7.25])


# ----------------------------------------------------------------------------- bilateral filter
def _bilateral_loop(I, W, F):
    h, w = I.shape
    r = F.radius
    I_f = np.zeros((h, w)); W_f = np.zeros((h, w))
    for y in range(h):
        for x in range(w):
            nI = dI = nW = dW = 0.0
            for yy in range(max(0, y - r), min(h, y + r + 1)):
                for xx in range(max(0, x - r), min(w, x + r + 1)):
                    d2 = (yy - y) ** 2 + (xx - x) ** 2
                    gs = np.exp(-d2 / (2 * F.sigma_s ** 2))
                    k = gs * np.exp(-(I[y, x] - I[yy, xx]) ** 2 / (2 * F.sigma_r_I ** 2))
                    nI += k * I[yy, xx]; dI += k
                    if W[yy, xx] > 0:
                        k = gs * np.exp(-(W[y, x] - W[yy, xx]) ** 2 / (2 * F.sigma_r_W ** 2))
                        nW += k * W[yy, xx]; dW += k
            I_f[y, x] = nI / dI
            W_f[y, x] = nW / dW if W[y, x] > 0 else 0.0
    return I_f, W_f


def test_bilateral_filter_against_a_per_pixel_loop():
    rng = np.random.default_rng(60)
    h, w = 11, 14
    I = rng.random((h, w))
    W = rng.uniform(0.2, 0.6, (h, w))
    W[rng.random((h, w)) < 0.2] = 0.0
    F = O.BilateralParams(radius=2, sigma_s=1.3, sigma_r_I=0.2, sigma_r_W=0.05)
    I_f, W_f = O.bilateral_filter(I, W, F)
    I_l, W_l = _bilateral_loop(I, W, F)
    assert np.allclose(I_f, I_l, rtol=1e-13, atol=1e-15) and np.allclose(W_f, W_l, rtol=1e-13, atol=1e-15)
    assert np.array_equal(W_f > 0, W > 0)                     # holes stay holes, no hole is filled


def test_bilateral_filter_without_range_term_is_a_normalised_gaussian_blur():
    rng = np.random.default_rng(61)
    I = rng.random((30, 40))
    F = O.BilateralParams(radius=3, sigma_s=1.7, sigma_r_I=1e9, sigma_r_W=1e9)
    I_f, W_f = O.bilateral_filter(I, np.ones_like(I), F)
    d = np.arange(-3, 4)
    k = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * 1.7 ** 2))
    expect = (scipy.ndimage.correlate(I, k, mode="constant", cval=0.0)
              / scipy.ndimage.correlate(np.ones_like(I), k, mode="constant", cval=0.0))
    assert np.allclose(I_f, expect, rtol=1e-13)
    assert np.allclose(W_f, 1.0, rtol=1e-15)


def test_bilateral_filter_special_cases():
    rng = np.random.default_rng(62)
    I = rng.random((9, 12))
    W = rng.uniform(0.3, 0.5, (9, 12))
    I0, W0 = O.bilateral_filter(I, W, O.BilateralParams(radius=0))
    assert np.array_equal(I0, I) and np.array_equal(W0, W)
    c = np.full((9, 12), 0.37)
    Ic, Wc = O.bilateral_filter(c, c, O.BilateralParams())
    assert np.allclose(Ic, 0.37, rtol=1e-15) and np.allclose(Wc, 0.37, rtol=1e-15)
    # a step far above the range sigma is preserved on both sides
    step = np.where(np.arange(12)[None, :] < 6, 0.2, 0.8) * np.ones((9, 1))
    Is, _ = O.bilateral_filter(step, np.ones_like(step), O.BilateralParams(sigma_r_I=0.02))
    assert np.allclose(Is, step, atol=1e-12)


# ----------------------------------------------------------------------------- covariance
def _pair(seed=5, w=160, h=120, levels=3, noise=True):
    p = synth.make_pair(seed, w, h, noise=noise)
    return p, O.build_pyramid(p["I_A"], p["W_A"], p["K"], levels), O.build_pyramid(p["I_B"], p["W_B"], p["K"], levels)


def test_covariance_without_filtering_is_the_inverse_of_the_final_step_hessian():
    p, A, B = _pair()
    r = O.align(A, B, None, O.AlignParams())
    c = O.covariance(A, B, r["T"], O.AlignParams(), O.BilateralParams(radius=0))
    st = O.eval_step(A, B, 0, r["T"], None, O.AlignParams())
    assert c["ok"] and np.array_equal(c["H"], st["H"])
    assert np.allclose(c["Sigma"] @ c["H"], np.eye(6), atol=1e-9)
    assert np.allclose(c["Sigma"], c["Sigma"].T, rtol=1e-10, atol=0)
    np.linalg.cholesky(c["Sigma"])


def test_covariance_filters_only_the_gradients():
    """Residuals, masks and robust parameters of the extra iteration are those of
    the unfiltered evaluation at the same pose; the Hessian is the one assembled
    with the gradients of the per-pixel-loop filtered planes."""
    p, A, B = _pair(seed=6, w=80, h=60, levels=2)
    r = O.align(A, B, None, O.AlignParams(levels=2, iters=(5, 10)))
    F = O.BilateralParams()
    c = O.covariance(A, B, r["T"], O.AlignParams(levels=2, iters=(5, 10)), F)
    st = O.eval_step(A, B, 0, r["T"], None, O.AlignParams(levels=2, iters=(5, 10)))
    s = c["step"]
    for key in ("r_I", "r_W", "mask_I", "mask_W"):
        assert np.array_equal(s[key], st[key]), key
    assert s["robust"] == st["robust"]
    I_l, W_l = _bilateral_loop(A[0].I, A[0].W, F)
    manual = O.eval_step(A, B, 0, r["T"], s["robust"], O.AlignParams(levels=2, iters=(5, 10)), grad_planes=(I_l, W_l))
    scale = np.sqrt(np.outer(np.diag(c["H"]), np.diag(c["H"])))
    assert np.all(np.abs(manual["H"] - c["H"]) <= 1e-10 * scale)
    # smoothing the noisy gradients lowers the information: the covariance grows
    assert np.trace(c["H"]) < np.trace(st["H"])
    assert np.linalg.det(c["Sigma"]) > np.linalg.det(np.linalg.inv(st["H"]))


def test_covariance_of_a_featureless_reference_is_degenerate():
    p, A, B = _pair(seed=7, w=80, h=60, levels=1)
    Z = [O.Level(l.I, np.zeros_like(l.W), l.K) for l in A]
    c = O.covariance(Z, B, np.eye(4), O.AlignParams(levels=1, iters=(1,)))
    assert not c["ok"] and not c["Sigma"].any()


# ----------------------------------------------------------------------------- covisibility
def _plane(h=60, w=80, W0=0.5):
    K = (65.625, 65.625, 39.5, 29.5)
    rng = np.random.default_rng(63)
    return K, rng.random((h, w)), np.full((h, w), W0)


def test_covisibility_of_a_frontal_plane_shifted_by_a_fraction_of_pixels():
    """A frontal plane seen after a sideways move by (3.3, -2.6) pixels: every
    pixel shifts by that amount, so the visible pixels are those whose nearest
    pixel after the shift is in the image, (w - 3)(h - 3) in each direction."""
    h, w = 60, 80
    K, I, W = _plane(h, w)
    T = np.eye(4)
    T[0, 3] = -3.3 / (K[0] * 0.5)
    T[1, 3] = 2.6 / (K[1] * 0.5)
    c = O.covisibility_ratio(I, W, I, W, K, T, 1e-3)
    expect = (w - 3) * (h - 3) / (w * h)
    assert c["counts"][0] == ((w - 3) * (h - 3), w * h) and c["counts"][1] == ((w - 3) * (h - 3), w * h)
    assert c["vr"] == c["vr_AB"] == c["vr_BA"] == expect


def test_covisibility_occlusion_and_holes_brute_force():
    """Random inverse depth with holes and an occluding patch in B: S_V and S_H
    counted pixel by pixel, and the ratio is the minimum over both directions."""
    rng = np.random.default_rng(64)
    h, w = 24, 32
    K = (26.0, 26.0, 15.5, 11.5)
    IA, IB = rng.random((h, w)), rng.random((h, w))
    WA = 0.5 + 0.02 * rng.random((h, w))
    WA[rng.random((h, w)) < 0.1] = 0
    WB = 0.5 + 0.02 * rng.random((h, w))
    WB[rng.random((h, w)) < 0.1] = 0
    WB[5:12, 8:20] = 0.9                                   # an occluder in B only
    T = O.se3_exp([0.03, -0.02, 0.01, 0.01, -0.015, 0.02])
    sigma_W = 0.01
    c = O.covisibility_ratio(IA, WA, IB, WB, K, T, sigma_W)

    def count(Wa, Wb, Tab):
        R, t = Tab[:3, :3], Tab[:3, 3]
        vis = valid = 0
        for y in range(h):
            for x in range(w):
                if not Wa[y, x] > 0:
                    continue
                valid += 1
                XA = np.array([(x - K[2]) / K[0], (y - K[3]) / K[1], 1.0]) / Wa[y, x]
                XB = R.T @ (XA - t)
                if not XB[2] > 0:
                    continue
                ub, vb = K[0] * XB[0] / XB[2] + K[2], K[1] * XB[1] / XB[2] + K[3]
                xn, yn = int(np.floor(ub + 0.5)), int(np.floor(vb + 0.5))      # nearest pixel
                if not (0 <= xn <= w - 1 and 0 <= yn <= h - 1):
                    continue
                if Wb[yn, xn] > 0 and abs(Wb[yn, xn] - 1.0 / XB[2]) < 3 * sigma_W:
                    vis += 1
        return vis, valid

    ab = count(WA, WB, T)
    ba = count(WB, WA, O.se3_inv(T))
    assert c["counts"] == (ab, ba)
    assert c["vr"] == min(ab[0] / ab[1], ba[0] / ba[1])
    assert c["vr_AB"] != c["vr_BA"]
    assert 0.3 < c["vr"] < 0.95


def test_covisibility_of_identical_frames_is_one():
    """Identical frames (with holes), T = I: every valid pixel maps onto itself."""
    p = synth.make_pair(10, 160, 120)
    c = O.covisibility_ratio(p["I_A"], p["W_A"], p["I_A"], p["W_A"], p["K"], np.eye(4), 1e-3)
    assert c["vr"] == 1.0 and c["counts"][0][1] == int((p["W_A"] > 0).sum())
    # the ratio of a frame pair is below one and falls as the motion grows
    T = p["T_gt"]
    c1 = O.covisibility_ratio(p["I_A"], p["W_A"], p["I_B"], p["W_B"], p["K"], T, 1.5e-3)
    big = O.se3_exp([0.1, 0.0, 0.0, 0.0, 0.05, 0.0]) @ T
    c2 = O.covisibility_ratio(p["I_A"], p["W_A"], p["I_B"], p["W_B"], p["K"], big, 1.5e-3)
    assert 0.5 < c1["vr"] < 1.0 and c2["vr"] < c1["vr"]


def test_tracking_switches_keyframe_on_covisibility():
    """With the covisibility policy a keyframe is replaced exactly on the frames
    whose ratio to it falls below the threshold, and every other frame is fused."""
    seq = synth.render_sequence(seed=0, n_frames=24, width=160, height=120)
    out = O.track_sequence(seq["I"], seq["W"], seq["K"], levels=2, iters=(3, 4), kf_every=None,
                           kf_covisibility=0.75)
    vr = np.array(out["covisibility"])
    assert len(vr) == 23 and (vr > 0).all() and (vr <= 1).all()
    switched = vr < 0.75
    assert 1 <= switched.sum() <= 8
    # the ratio right after a switch is measured against the new keyframe: it
    # recovers above the threshold
    after = np.argwhere(switched).ravel() + 1
    assert all(vr[i] > vr[i - 1] for i in after if i < len(vr))


# ----------------------------------------------------------------------------- warp at full resolution
def test_full_resolution_warp_is_the_plain_warp_at_level_zero():
    p, A, B = _pair(seed=8)
    T = p["T_gt"]
    a = O.eval_step(A, B, 0, T, ROB, O.AlignParams())
    b = O.eval_step(A, B, 0, T, ROB, O.AlignParams(warp_mode="full"))
    for key in ("r_I", "r_W", "mask_I", "mask_W", "H", "g"):
        assert np.array_equal(a[key], b[key]), key


def _brute_full(pA, pB, level, T):
    """Warped maps at level 0 pixel by pixel, reduced to `level` by nested loops."""
    A0, B0 = pA[0], pB[0]
    h, w = A0.I.shape
    K = A0.K
    R, t = T[:3, :3], T[:3, 3]
    Is, Ws = np.zeros((h, w)), np.zeros((h, w))
    vI, vW = np.zeros((h, w), bool), np.zeros((h, w), bool)
    for y in range(h):
        for x in range(w):
            if not A0.W[y, x] > 0:
                continue
            XA = np.array([(x - K[2]) / K[0], (y - K[3]) / K[1], 1.0]) / A0.W[y, x]
            XB = R.T @ (XA - t)
            if not XB[2] > 0:
                continue
            ub, vb = K[0] * XB[0] / XB[2] + K[2], K[1] * XB[1] / XB[2] + K[3]
            x0, y0 = int(np.floor(ub)), int(np.floor(vb))
            if not (0 <= x0 <= w - 2 and 0 <= y0 <= h - 2):
                continue
            ax, ay = ub - x0, vb - y0
            bil = lambda M: ((1 - ay) * ((1 - ax) * M[y0, x0] + ax * M[y0, x0 + 1])
                             + ay * ((1 - ax) * M[y0 + 1, x0] + ax * M[y0 + 1, x0 + 1]))
            Is[y, x], vI[y, x] = bil(B0.I), True
            taps = [B0.W[y0, x0], B0.W[y0, x0 + 1], B0.W[y0 + 1, x0], B0.W[y0 + 1, x0 + 1]]
            if min(taps) > 0:
                zt = (R @ (np.array([(ub - K[2]) / K[0], (vb - K[3]) / K[1], 1.0]) / bil(B0.W)) + t)[2]
                if zt > 0:
                    Ws[y, x], vW[y, x] = 1.0 / zt, True
    for _ in range(level):
        h, w = h // 2, w // 2
        nI, nW = np.zeros((h, w)), np.zeros((h, w))
        nvI, nvW = np.zeros((h, w), bool), np.zeros((h, w), bool)
        for y in range(h):
            for x in range(w):
                for (src, val, dst, dval) in ((Is, vI, nI, nvI), (Ws, vW, nW, nvW)):
                    kids = [(src[2 * y + a, 2 * x + b], val[2 * y + a, 2 * x + b]) for a in (0, 1) for b in (0, 1)]
                    good = [k for k, ok in kids if ok]
                    if good:
                        dst[y, x] = sum(good) / len(good)
                        dval[y, x] = True
        Is, Ws, vI, vW = nI, nW, nvI, nvW
    return Is, vI, Ws, vW


@pytest.mark.parametrize("level", [1, 2])
def test_full_resolution_warp_against_per_pixel_loops(level):
    rng = np.random.default_rng(70 + level)
    h, w = 24, 32
    K = (26.0, 26.0, 15.5, 11.5)
    IA, IB = rng.random((h, w)), rng.random((h, w))
    WA, WB = rng.uniform(0.3, 0.6, (h, w)), rng.uniform(0.3, 0.6, (h, w))
    WA[rng.random((h, w)) < 0.15] = 0
    WB[rng.random((h, w)) < 0.15] = 0
    pA = O.build_pyramid(IA, WA, K, level + 1)
    pB = O.build_pyramid(IB, WB, K, level + 1)
    T = O.se3_exp([0.05, -0.03, 0.02, 0.02, -0.03, 0.01])
    st = O.eval_step(pA, pB, level, T, ROB, O.AlignParams(levels=level + 1, warp_mode="full"))
    Is, vI, Ws, vW = _brute_full(pA, pB, level, T)
    A = pA[level]
    hh, ww = A.I.shape
    for y in range(hh):
        for x in range(ww):
            interior = 1 <= x <= ww - 2 and 1 <= y <= hh - 2
            mI = bool(A.W[y, x] > 0 and interior and vI[y, x])
            nb = interior and min(A.W[y, x - 1], A.W[y, x + 1], A.W[y - 1, x], A.W[y + 1, x]) > 0
            mW = bool(mI and vW[y, x] and nb)
            assert st["mask_I"][y, x] == mI and st["mask_W"][y, x] == mW, (y, x)
            if mI:
                assert abs(st["r_I"][y, x] - (Is[y, x] - A.I[y, x])) < 1e-13
            if mW:
                assert abs(st["r_W"][y, x] - (Ws[y, x] - A.W[y, x])) < 1e-13
    assert st["mask_I"].sum() > 0.2 * hh * ww and st["mask_W"].sum() > 0


def test_full_resolution_warp_recovers_the_pose_of_noise_free_renders():
    p, A, B = _pair(seed=9, noise=False)
    r = O.align(A, B, None, O.AlignParams(warp_mode="full"))
    E = O.se3_inv(p["T_gt"]) @ r["T"]
    assert r["status"] == O.OK
    assert np.linalg.norm(O.so3_log(E[:3, :3])) < 5e-4 and np.linalg.norm(E[:3, 3]) < 5e-4
