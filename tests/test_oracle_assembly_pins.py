"""Pins of the oracle's weighting, normal-equation assembly, robust-parameter
selection and tracking bookkeeping against things other than the oracle.

* the IRLS weights against the score of scipy's Student-t density
  ("Error distribution and robust optimisation", eqs. Student_pdf and
  minimisationIRLS: w(r) = -(d/dr log p(r)) / (r - mu));
* H, g and the cost against an independent per-pixel loop that rebuilds every
  term from the paper's formulas with explicit 3x3 / 3x6 matrices
  ("Dense motion estimation": eqs. res_int, res_depth, DeltaX, the normal
  weight lambda_n, minimisationIRLS);
* g against the central finite difference of the weighted cost
  E(xi) = 1/2 sum w r(exp(xi)^-1 T)^2 with the weights held fixed, H against
  the same sum assembled from finite-difference Jacobians, and the step
  H xi = -g against a decrease of E ("Iterative optimisation");
* nu_I <- max(nu_I, nu_W) and the masked systematic sample on hand-built
  residual sets;
* the tracking front-end's keyframe switch, constant-velocity guess and pose
  composition against the same quantities recomposed from world poses
  ("Camera tracking", "Keyframe fusion").
"""
import numpy as np
import pytest
import scipy.stats

import oracle as O
from paper_1807_08271_gb300 import synth

# distinct parameters per channel, so that a swapped channel index shows
ROB = dict(mu=[0.004, -0.0015], sigma=[0.045, 0.012], nu=[3.5, 7.25])


def _pair(seed=2, w=160, h=120, levels=1, noise=True):
    p = synth.make_pair(seed, w, h, noise=noise)
    A = O.build_pyramid(p["I_A"], p["W_A"], p["K"], levels)
    B = O.build_pyramid(p["I_B"], p["W_B"], p["K"], levels)
    return p, A, B


def _off_pose(p, seed=0):
    """Ground truth perturbed by a small motion, so residuals are non-zero and
    warped points fall between pixel nodes."""
    rng = np.random.default_rng(100 + seed)
    return O.se3_exp(np.concatenate([rng.uniform(-4e-3, 4e-3, 3), rng.uniform(-3e-3, 3e-3, 3)])) @ p["T_gt"]


# ----------------------------------------------------------------------------- weights
def test_weights_are_the_student_t_score_over_the_residual():
    """w_I = -(d/dr log f_St(r | mu_I, sigma_I, nu_I)) / (r - mu_I) and
    w_W / lambda_n the same with the W channel's parameters, the derivative taken
    numerically from scipy's log-density."""
    p, A, B = _pair()
    st = O.eval_step(A, B, 0, _off_pose(p), ROB)
    for c, (r, w, m) in enumerate(((st["r_I"], st["w_I"], st["mask_I"]),
                                   (st["r_W"], st["w_W"], st["mask_W"]))):
        mu, sig, nu = ROB["mu"][c], ROB["sigma"][c], ROB["nu"][c]
        rr = r[m]
        d = rr - mu
        keep = np.abs(d) > 1e-3 * sig            # the quotient is ill-conditioned at r = mu
        rr, d = rr[keep], d[keep]
        hstep = 1e-6 * sig
        lp = lambda x: scipy.stats.t.logpdf(x, nu, loc=mu, scale=sig)
        score = (lp(rr + hstep) - lp(rr - hstep)) / (2 * hstep)
        expect = -score / d
        got = w[m][keep]
        if c == 1:
            got = got / st["lam"][m][keep]
        assert rr.size > 5000
        assert np.allclose(got, expect, rtol=1e-6), c
    # outside the masks nothing is weighted
    assert not st["w_I"][~st["mask_I"]].any() and not st["w_W"][~st["mask_W"]].any()


def test_a_channel_without_scale_gets_no_weight():
    p, A, B = _pair()
    rob = dict(mu=[0.0, 0.0], sigma=[0.05, 0.0], nu=[5.0, 5.0])
    st = O.eval_step(A, B, 0, _off_pose(p), rob)
    assert st["w_I"][st["mask_I"]].min() > 0
    assert not st["w_W"].any()


# ----------------------------------------------------------------------------- normal equations
def _brute_force_terms(IA, WA, IB, WB, K, T, rob):
    """Every pixel's residuals, Jacobians, normal weight and IRLS weights from the
    paper's formulas with explicit matrices, summed into H, g and the cost."""
    h, w = IA.shape
    fx, fy, cx, cy = K
    Km = np.array([[fx, 0.0, cx], [0.0, fy, cy], [0.0, 0.0, 1.0]])
    Ki = np.linalg.inv(Km)
    R, t = T[:3, :3], T[:3, 3]
    ez = np.array([0.0, 0.0, 1.0])
    H = np.zeros((6, 6)); g = np.zeros(6); cost = 0.0
    n = [0, 0]

    def skew(x):
        return np.array([[0.0, -x[2], x[1]], [x[2], 0.0, -x[0]], [-x[1], x[0], 0.0]])

    def student_w(r, c):
        # -(d/dr log f_St) / (r - mu) of f_St ~ (1 + ((r - mu)/sigma)^2 / nu)^(-(nu + 1)/2)
        mu, sig, nu = rob["mu"][c], rob["sigma"][c], rob["nu"][c]
        return (nu + 1.0) / (nu * sig * sig + (r - mu) ** 2)

    for y in range(1, h - 1):
        for x in range(1, w - 1):
            if not WA[y, x] > 0:
                continue
            p = np.array([x, y, 1.0])
            XA = (Ki @ p) / WA[y, x]
            XB = R.T @ (XA - t)
            if not XB[2] > 0:
                continue
            pb = Km @ (XB / XB[2])
            x0, y0 = int(np.floor(pb[0])), int(np.floor(pb[1]))
            if not (0 <= x0 <= w - 2 and 0 <= y0 <= h - 2):
                continue
            ax, ay = pb[0] - x0, pb[1] - y0

            def bil(M):
                return ((1 - ay) * ((1 - ax) * M[y0, x0] + ax * M[y0, x0 + 1])
                        + ay * ((1 - ax) * M[y0 + 1, x0] + ax * M[y0 + 1, x0 + 1]))

            Mx = np.hstack([np.eye(3), -skew(XA)])                 # [I | -[X_A]x]
            KP = Km - np.outer(p, ez)                               # K - p e_z^T
            dI = np.array([(IA[y, x + 1] - IA[y, x - 1]) / 2, (IA[y + 1, x] - IA[y - 1, x]) / 2, 0.0])
            rI = bil(IB) - IA[y, x]
            JI = (WA[y, x] * (dI @ KP)) @ Mx
            wI = student_w(rI, 0)
            H += wI * np.outer(JI, JI); g += wI * JI * rI; cost += wI * rI * rI
            n[0] += 1
            taps = [WB[y0, x0], WB[y0, x0 + 1], WB[y0 + 1, x0], WB[y0 + 1, x0 + 1]]
            nb = [WA[y, x - 1], WA[y, x + 1], WA[y - 1, x], WA[y + 1, x]]
            if min(taps) > 0 and min(nb) > 0:
                zt = (R @ ((Ki @ pb) / bil(WB)) + t)[2]
                if zt > 0:
                    Wg = 1.0 / zt
                    rW = Wg - WA[y, x]
                    dW = np.array([(WA[y, x + 1] - WA[y, x - 1]) / 2, (WA[y + 1, x] - WA[y - 1, x]) / 2, 0.0])
                    JW = (WA[y, x] * (dW @ KP + Wg * ez)) @ Mx
                    nu_ = dW @ KP / WA[y, x] + ez                  # surface normal (unnormalised)
                    ray = Ki @ p
                    lam = (nu_ / np.linalg.norm(nu_)) @ ray / np.linalg.norm(ray)
                    wW = lam * student_w(rW, 1)
                    H += wW * np.outer(JW, JW); g += wW * JW * rW; cost += wW * rW * rW
                    n[1] += 1
    return H, g, cost, n


@pytest.mark.parametrize("hw", [(6, 8), (12, 16), (30, 40)])
def test_normal_equations_against_an_independent_per_pixel_loop(hw):
    h, w = hw
    rng = np.random.default_rng(40 + h)
    K = (w * 0.8, w * 0.8, (w - 1) / 2, (h - 1) / 2)
    IA, IB = rng.random((h, w)), rng.random((h, w))
    WA, WB = rng.uniform(0.3, 0.6, (h, w)), rng.uniform(0.3, 0.6, (h, w))
    WA[rng.random((h, w)) < 0.15] = 0
    WB[rng.random((h, w)) < 0.15] = 0
    T = O.se3_exp([0.05, -0.03, 0.02, 0.02, -0.03, 0.01])
    st = O.eval_step([O.Level(IA, WA, K)], [O.Level(IB, WB, K)], 0, T, ROB)
    H, g, cost, n = _brute_force_terms(IA, WA, IB, WB, K, T, ROB)
    assert n[0] > 0 and n[1] > 0 and st["n_valid"] == n
    scale = np.sqrt(np.outer(np.diag(H), np.diag(H)))
    assert np.abs(st["H"] - H).max() <= 1e-12 * scale.max()
    assert np.allclose(st["H"], H, rtol=1e-11, atol=1e-13 * scale.max())
    assert np.allclose(st["g"], g, rtol=1e-11, atol=1e-13 * np.abs(g).max())
    assert abs(st["cost"] - cost) <= 1e-12 * cost


def _smooth_offset_pair(h=120, w=160):
    """A smooth textured slanted plane without holes (A), and B = A with every
    intensity raised by 0.05: at T = I the intensity residual is 0.05 everywhere
    and the inverse-depth residual 0, and the Jacobians of A's central
    differences are those of B's bilinear surface at the pixel nodes (reading R3)."""
    K = (131.25, 131.25, 79.5, 59.5)
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    q = np.stack([(u - K[2]) / K[0], (v - K[3]) / K[1], np.ones((h, w))], -1)
    WA = (q @ np.array([0.25, -0.15, 1.0])) / 2.5
    IA = 0.5 + 0.2 * np.sin(0.31 * u + 0.1) * np.cos(0.23 * v) + 0.1 * np.sin(0.013 * u * v)
    return [O.Level(IA, WA, K)], [O.Level(IA + 0.05, WA.copy(), K)]


def _frozen_cost(A, B, T, wI, wW, mI):
    """E = 1/2 sum w r^2 with the weights of the evaluation point; the
    inverse-depth residuals vanish at that point, so pixels whose W mask changes
    with the pose change E by O(h^2) only."""
    st = O.eval_step(A, B, 0, T, ROB)
    assert np.array_equal(st["mask_I"], mI)
    return 0.5 * (np.sum(wI * st["r_I"] ** 2) + np.sum(wW * st["r_W"] ** 2)), st


def test_g_is_the_gradient_of_the_weighted_cost_with_weights_held():
    """g_k = dE/dxi_k at xi = 0 for E(xi) = 1/2 sum w r(exp(xi)^-1 T)^2 with the
    weights of the evaluation point held fixed: central differences."""
    A, B = _smooth_offset_pair()
    T = np.eye(4)
    st = O.eval_step(A, B, 0, T, ROB)
    assert np.allclose(st["r_I"][st["mask_I"]], 0.05, atol=1e-13) and np.abs(st["r_W"]).max() < 1e-13
    args = (st["w_I"], st["w_W"], st["mask_I"])
    h = 1e-9
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6); e[k] = h
        Ep, _ = _frozen_cost(A, B, O.se3_inv(O.se3_exp(e)) @ T, *args)
        Em, _ = _frozen_cost(A, B, O.se3_inv(O.se3_exp(-e)) @ T, *args)
        fd[k] = (Ep - Em) / (2 * h)
    scale = np.sqrt(np.diag(st["H"]) * st["cost"])       # |g_k| <= sqrt(H_kk cost)
    assert np.abs(st["g"]).min() > 5e-4 * scale.max()      # a gradient worth checking
    assert np.all(np.abs(fd - st["g"]) <= 1e-7 * scale), (fd, st["g"])


def test_h_is_the_weighted_sum_of_finite_difference_jacobian_products():
    """H = sum w J J^T with J the central finite difference of the residuals
    (both channels), on the pair where those Jacobians are exact."""
    A, B = _smooth_offset_pair()
    T = np.eye(4)
    st = O.eval_step(A, B, 0, T, ROB)
    h = 1e-7
    JI = np.zeros(st["r_I"].shape + (6,))
    JW = np.zeros_like(JI)
    keepW = st["mask_W"].copy()
    for k in range(6):
        e = np.zeros(6); e[k] = h
        sp = O.eval_step(A, B, 0, O.se3_inv(O.se3_exp(e)) @ T, ROB)
        sm = O.eval_step(A, B, 0, O.se3_inv(O.se3_exp(-e)) @ T, ROB)
        assert np.array_equal(sp["mask_I"], st["mask_I"]) and np.array_equal(sm["mask_I"], st["mask_I"])
        keepW &= sp["mask_W"] & sm["mask_W"]
        JI[..., k] = (sp["r_I"] - sm["r_I"]) / (2 * h)
        JW[..., k] = (sp["r_W"] - sm["r_W"]) / (2 * h)
    # the W mask of the slanted plane without holes only loses border pixels
    assert keepW.sum() == st["mask_W"].sum()
    Hfd = np.einsum("hw,hwi,hwj->ij", st["w_I"], JI, JI) + np.einsum("hw,hwi,hwj->ij", st["w_W"], JW, JW)
    scale = np.sqrt(np.outer(np.diag(st["H"]), np.diag(st["H"])))
    assert np.all(np.abs(Hfd - st["H"]) <= 1e-5 * scale), np.abs(Hfd - st["H"]) / scale
    # both channels carry weight in H
    HW = np.einsum("hw,hwi,hwj->ij", st["w_W"], JW, JW)
    assert np.trace(HW) > 1e-3 * np.trace(st["H"])


def test_the_step_solving_h_xi_equals_minus_g_lowers_the_weighted_cost():
    p, A, B = _pair(seed=4)
    T = _off_pose(p, 2)
    st = O.eval_step(A, B, 0, T, ROB)
    xi = np.linalg.solve(st["H"], -st["g"])
    E0 = 0.5 * (np.sum(st["w_I"] * st["r_I"] ** 2) + np.sum(st["w_W"] * st["r_W"] ** 2))
    E = lambda x: (lambda s: 0.5 * (np.sum(st["w_I"] * np.where(s["mask_I"] & st["mask_I"], s["r_I"], 0) ** 2)
                                    + np.sum(st["w_W"] * np.where(s["mask_W"] & st["mask_W"], s["r_W"], 0) ** 2)))(
        O.eval_step(A, B, 0, O.se3_inv(O.se3_exp(x)) @ T, ROB))
    assert E(xi) < 0.9 * E0
    assert E(-xi) > E0                                    # the opposite direction climbs
    T_new, xi2, ok = O.solve_update(st["H"], st["g"], T, 10 ** 6, 60)
    assert ok and np.allclose(xi2, xi, rtol=1e-12)
    assert np.allclose(T_new, O.se3_inv(O.se3_exp(xi)) @ T, atol=1e-15)


# ----------------------------------------------------------------------------- robust parameters
def test_nu_of_the_intensity_channel_is_raised_to_the_inverse_depth_channel():
    """nu_I <- max(nu_I, nu_W): heavy-tailed intensity residuals (nu_I near 3) with
    Gaussian inverse-depth residuals (nu_W at the upper bound 10) give nu_I = 10;
    the opposite case keeps nu_I; a channel without residuals leaves the other."""
    rng = np.random.default_rng(50)
    heavy = scipy.stats.t.rvs(3, scale=0.03, size=19000, random_state=51)
    gauss = rng.normal(0.0, 0.002, 17000)
    P = O.AlignParams()
    nu_heavy = O.estimate_nu(heavy, *O.location_scale(heavy))
    assert 2.4 < nu_heavy < 3.8
    out = O.robust_params(heavy, gauss, P)
    assert out["nu"] == [10.0, 10.0] and out["ok"] == [True, True]
    out = O.robust_params(gauss, heavy, P)
    assert out["nu"][0] == 10.0 and out["nu"][1] == nu_heavy
    out = O.robust_params(heavy, np.zeros(0), P)
    assert out["nu"] == [nu_heavy, P.nu0] and out["ok"] == [True, False]
    assert out["n"] == [19000, 0]
    # without nu estimation both stay at nu0
    out = O.robust_params(heavy, gauss, O.AlignParams(estimate_nu=False))
    assert out["nu"] == [P.nu0, P.nu0]


def test_robust_parameters_come_from_the_masked_systematic_sample():
    """A 200x150 level has stride 2: the estimated (mu, sigma, nu) per channel are
    those of the residuals at u = 0, v = 0 (mod 2) that pass that channel's mask,
    collected here pixel by pixel."""
    p = synth.make_pair(6, 200, 150)
    A = O.build_pyramid(p["I_A"], p["W_A"], p["K"], 1)
    B = O.build_pyramid(p["I_B"], p["W_B"], p["K"], 1)
    T = _off_pose(p, 3)
    st = O.eval_step(A, B, 0, T, None)
    s = O.sample_stride(200, 150)
    assert s == 2
    picked = [[], []]
    for y in range(0, 150, s):
        for x in range(0, 200, s):
            if st["mask_I"][y, x]:
                picked[0].append(st["r_I"][y, x])
            if st["mask_W"][y, x]:
                picked[1].append(st["r_W"][y, x])
    assert len(picked[1]) < len(picked[0]) <= 100 * 75
    assert st["robust"]["n"] == [len(picked[0]), len(picked[1])]
    P = O.AlignParams()
    for c in range(2):
        mu, sig = O.location_scale(np.array(picked[c]), P.nu0, P.scale_iters)
        assert st["robust"]["mu"][c] == mu and st["robust"]["sigma"][c] == sig
    # every mask-passing pixel off the sample grid is left out: using them all changes the scale
    allI = st["r_I"][st["mask_I"]]
    assert O.location_scale(allI)[1] != st["robust"]["sigma"][0]


# ----------------------------------------------------------------------------- tracking front-end
def test_track_sequence_bookkeeping_against_world_poses(monkeypatch):
    """Keyframe switch every 3 frames on a short sequence.  Recomposed from the
    world poses the tracker reports: every guess is the projected constant-velocity
    prediction T_wkf^-1 W_{k-1} W_{k-2}^-1 W_{k-1} in the current keyframe, every
    world pose is the keyframe's world pose times the alignment, frames 3j replace
    the keyframe without being fused, the others are fused with the final sigma_W
    of their own alignment, and the last keyframe is the last switch frame fused
    with the frames after it."""
    seq = synth.render_sequence(seed=3, n_frames=8, width=160, height=120)
    K = seq["K"]
    calls = []
    fuses = []
    real_align, real_fuse = O.align, O.fuse

    def spy_align(A, B, T_init=None, P=None):
        r = real_align(A, B, T_init, P)
        calls.append(dict(T_init=np.array(T_init), T=r["T"].copy(), sigma_W=r["robust"]["sigma"][1]))
        return r

    def spy_fuse(I_kf, W_kf, C_kf, I_k, W_k, K_, T, sigma_W, fuse_intensity=True):
        fuses.append(dict(T=np.array(T), sigma_W=sigma_W, I_k=np.array(I_k)))
        return real_fuse(I_kf, W_kf, C_kf, I_k, W_k, K_, T, sigma_W, fuse_intensity)

    monkeypatch.setattr(O.rgbid_oracle, "align", spy_align)
    monkeypatch.setattr(O.rgbid_oracle, "fuse", spy_fuse)
    out = O.rgbid_oracle.track_sequence(seq["I"], seq["W"], K, levels=2, iters=(3, 4), kf_every=3)
    Wd = out["T_world"]
    assert len(calls) == 7 and Wd.shape == (8, 4, 4) and np.array_equal(Wd[0], np.eye(4))
    kf_of = lambda k: 3 * ((k - 1) // 3)                      # the keyframe frame k is aligned to
    for k in range(1, 8):
        c = calls[k - 1]
        T_wkf = Wd[kf_of(k)]
        # the reported world pose composes the keyframe's with the alignment
        assert np.allclose(Wd[k], T_wkf @ c["T"], atol=1e-14)
        if k == 1:
            expect = np.eye(4)
        else:
            Wm1 = Wd[k - 1]
            Wm2 = Wd[k - 2] if k - 2 >= 0 else np.eye(4)
            expect = O.se3_project(O.se3_inv(T_wkf) @ Wm1 @ O.se3_inv(Wm2) @ Wm1)
        assert np.allclose(c["T_init"], expect, atol=1e-11), k
    # fused frames: all but the switch frames, each with its own final sigma_W and pose
    fused = [k for k in range(1, 8) if k % 3 != 0]
    assert len(fuses) == len(fused)
    for f, k in zip(fuses, fused):
        assert np.array_equal(f["I_k"], seq["I"][k].astype(np.float64))
        assert f["sigma_W"] == calls[k - 1]["sigma_W"] and np.array_equal(f["T"], calls[k - 1]["T"])
    # the last keyframe: frame 6 fused with frame 7
    I6, W6 = O.measurement_planes(seq["I"][6], seq["W"][6])
    Ie, We, Ce, _ = real_fuse(I6, W6, np.ones_like(W6), seq["I"][7], seq["W"][7], K, calls[6]["T"],
                              calls[6]["sigma_W"])
    I_kf, W_kf, C_kf = out["keyframe"]
    assert np.array_equal(I_kf, Ie) and np.array_equal(W_kf, We) and np.array_equal(C_kf, Ce)
    # and the tracking stays on the rendered trajectory
    Tw = [O.se3_inv(seq["T_wc"][0]) @ seq["T_wc"][k] for k in range(8)]
    for k in range(8):
        E = O.se3_inv(Tw[k]) @ Wd[k]
        assert np.linalg.norm(O.so3_log(E[:3, :3])) < 5e-3 and np.linalg.norm(E[:3, 3]) < 5e-3
