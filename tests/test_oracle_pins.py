"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, an invariant, a library
routine that implements the same mathematics independently (scipy's matrix
exponential, Student-t density, MLE fit, root finder), or brute force on tiny
inputs, chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
import scipy.stats

import oracle as O
from paper_1807_08271_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Lie groups
def _thetas():
    rng = np.random.default_rng(1)
    out = [np.zeros(3), np.array([1e-9, -2e-9, 3e-10]), np.array([0.0, 0.0, 3.0])]
    for mag in (1e-6, 1e-3, 0.1, 1.0, 2.5, 3.1):
        out.append(synth.random_unit(rng) * mag)
    return out


@pytest.mark.parametrize("theta", _thetas())
def test_so3_exp_is_rotation_and_matches_expm(theta):
    R = O.so3_exp(theta)
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1.0) < 1e-14
    # textbook matrix exponential of [theta]x (scipy's Pade implementation)
    assert np.allclose(R, scipy.linalg.expm(O.hat(theta)), atol=1e-14)


@pytest.mark.parametrize("theta", [t for t in _thetas() if np.linalg.norm(t) < 3.05])
def test_so3_log_inverts_exp(theta):
    assert np.allclose(O.so3_log(O.so3_exp(theta)), theta, atol=1e-12)


def test_se3_exp_is_decoupled():
    xi = np.array([0.3, -0.2, 0.1, 0.4, -0.5, 0.2])
    T = O.se3_exp(xi)
    assert np.array_equal(T[:3, 3], xi[:3])            # translation is not coupled to rotation
    assert np.allclose(T[:3, :3], scipy.linalg.expm(O.hat(xi[3:])), atol=1e-14)
    assert np.allclose(O.se3_log(T), xi, atol=1e-13)
    assert np.allclose(O.se3_inv(T) @ T, np.eye(4), atol=1e-14)


# ----------------------------------------------------------------------------- pyramid & intrinsics
def test_level_intrinsics_chain_matches_paper_cameras():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    K640 = g["intrinsics_640"]["value"]
    K160 = g["intrinsics_160"]["value"]
    assert O.level_intrinsics(K640, 2) == tuple(K160)
    assert O.level_intrinsics(K640, 1) == (262.5, 262.5, 159.5, 119.5)


def test_downsample_brute_force_with_holes_and_odd_sizes():
    rng = np.random.default_rng(3)
    for h, w in [(6, 8), (7, 9), (12, 16), (5, 5)]:
        I = rng.random((h, w))
        W = rng.random((h, w)) + 0.2
        W[rng.random((h, w)) < 0.3] = 0.0
        I1, W1 = O.downsample(I, W)
        assert I1.shape == (h // 2, w // 2)
        for y in range(h // 2):
            for x in range(w // 2):
                kids_i = [I[2 * y, 2 * x], I[2 * y, 2 * x + 1], I[2 * y + 1, 2 * x], I[2 * y + 1, 2 * x + 1]]
                kids_w = [W[2 * y, 2 * x], W[2 * y, 2 * x + 1], W[2 * y + 1, 2 * x], W[2 * y + 1, 2 * x + 1]]
                assert abs(I1[y, x] - sum(kids_i) / 4) < 1e-15
                good = [k for k in kids_w if k > 0]
                expect = sum(good) / len(good) if good else 0.0
                assert abs(W1[y, x] - expect) < 1e-15


def test_pyramid_of_affine_plane_equals_direct_projection_at_each_level():
    """A plane has inverse depth affine in pixel coordinates; with intensity affine
    in level-0 pixels the 2x2 box mean equals the value at the child-block
    centre.  Both must equal the direct formula evaluated through K_l: this pins
    the box mean and the principal-point update together."""
    K0 = (525.0, 525.0, 319.5, 239.5)
    n, d = np.array([0.2, -0.3, 1.0]), 2.5            # plane n.X = d
    h, w = 480, 640
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)

    def plane_maps(K, uu, vv):
        fx, fy, cx, cy = K
        qx, qy = (uu - cx) / fx, (vv - cy) / fy
        Wp = (n[0] * qx + n[1] * qy + n[2]) / d
        # intensity defined on the ray direction, affine in level-0 pixels
        u0 = K0[0] * qx + K0[2]
        v0 = K0[1] * qy + K0[3]
        return 0.3 + 1e-3 * u0 - 4e-4 * v0, Wp

    I0, W0 = plane_maps(K0, u, v)
    pyr = O.build_pyramid(I0, W0, K0, 4)
    for l in range(1, 4):
        Kl = O.level_intrinsics(K0, l)
        hl, wl = pyr[l].W.shape
        vl, ul = np.mgrid[0:hl, 0:wl].astype(np.float64)
        Ie, We = plane_maps(Kl, ul, vl)
        assert np.max(np.abs(pyr[l].W - We)) < 1e-13
        assert np.max(np.abs(pyr[l].I - Ie)) < 1e-13


def test_gradients_exact_on_quadratics_and_border_rules():
    h, w = 9, 11
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    I = 0.1 + 0.02 * u - 0.03 * v + 1e-3 * u * u + 2e-3 * u * v - 5e-4 * v * v
    W = 0.5 + 0.01 * u + 0.02 * v + 3e-4 * u * u
    W[4, 6] = 0.0                                         # a hole
    gIx, gIy, gWx, gWy, interior, gWv = O.gradients(I, W)
    dIdu = 0.02 + 2e-3 * u + 2e-3 * v
    dIdv = -0.03 + 2e-3 * u - 1e-3 * v
    assert np.allclose(gIx[interior], dIdu[interior], atol=1e-14)
    assert np.allclose(gIy[interior], dIdv[interior], atol=1e-14)
    assert not interior[0].any() and not interior[-1].any() and not interior[:, 0].any() and not interior[:, -1].any()
    # the four 4-neighbours of the hole lose their W gradient; the hole's own gradient
    # is valid since its neighbours are valid (mask_W also needs W_A > 0 there)
    for (y, x) in [(4, 5), (4, 7), (3, 6), (5, 6)]:
        assert not gWv[y, x]
    assert gWv[4, 6] and gWv[2, 2]


def test_bilinear_reproduces_bilinear_functions_and_bounds():
    h, w = 7, 9
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    f = 0.3 + 0.1 * u - 0.2 * v + 0.05 * u * v
    rng = np.random.default_rng(4)
    x = rng.uniform(-1.5, w + 0.5, 500)
    y = rng.uniform(-1.5, h + 0.5, 500)
    val, valid, _ = O.bilinear(f, x, y)
    inside = (x >= 0) & (np.floor(x) + 1 <= w - 1) & (y >= 0) & (np.floor(y) + 1 <= h - 1)
    assert np.array_equal(valid, inside)
    exact = 0.3 + 0.1 * x - 0.2 * y + 0.05 * x * y
    assert np.allclose(val[valid], exact[valid], atol=1e-14)
    # the last column/row itself is not bilinear-valid (needs x0 + 1 <= w - 1)
    _, vv, _ = O.bilinear(f, np.array([w - 1.0, w - 1.5]), np.array([1.0, 1.0]))
    assert list(vv) == [False, True]


# ----------------------------------------------------------------------------- residuals & Jacobians
def _pair_levels(seed=0, noise=False, w=160, h=120, levels=3):
    p = synth.make_pair(seed, w, h, noise=noise)
    A = O.build_pyramid(p["I_A"], p["W_A"], p["K"], levels)
    B = O.build_pyramid(p["I_B"], p["W_B"], p["K"], levels)
    return p, A, B


FIXED = dict(mu=[0.0, 0.0], sigma=[0.05, 0.01], nu=[5.0, 5.0])


def test_zero_residual_and_gradient_at_identity_on_identical_frames():
    p, A, _ = _pair_levels(1)
    st = O.eval_step(A, A, 0, np.eye(4), FIXED)
    assert np.max(np.abs(st["r_I"])) <= 1e-12
    assert np.max(np.abs(st["r_W"])) <= 1e-12
    assert np.max(np.abs(st["g"])) <= 1e-9 * np.sqrt(np.max(np.diag(st["H"])))
    np.linalg.cholesky(st["H"])                            # H is SPD
    W = A[0].W
    _, _, _, _, interior, _ = O.gradients(A[0].I, W)
    assert np.array_equal(st["mask_I"], (W > 0) & interior & np.pad(np.ones((119, 159), bool), ((0, 1), (0, 1))))


def test_true_pose_transfers_plane_inverse_depth_exactly():
    """Noise-free render of a single plane: at the ground-truth pose the warped
    inverse depth of B equals W_A (inverse depth is affine on a plane, so the
    bilinear transfer is exact up to float32 storage)."""
    rng = np.random.default_rng(11)
    K = synth.pinhole(160, 120)
    sc = synth.Scene(np.stack([synth.perlin_tile(rng, 128)]))
    Rb = synth.rotation_about([1, 0.3, 0], np.deg2rad(20))
    sc.add_box([0.1, -0.05, 2.2], Rb, [5.0, 5.0, 0.001], 0)
    T = O.se3_exp([0.02, -0.01, 0.015, 0.01, -0.02, 0.015])
    iA, zA = sc.render(K, 160, 120, np.eye(4))
    iB, zB = sc.render(K, 160, 120, T)
    IA, WA = synth.apply_noise(iA, zA, rng, noise=False)
    IB, WB = synth.apply_noise(iB, zB, rng, noise=False)
    A = O.build_pyramid(IA, WA, K, 1)
    B = O.build_pyramid(IB, WB, K, 1)
    st = O.eval_step(A, B, 0, T, FIXED)
    m = st["mask_W"]
    assert m.sum() > 10000
    rel = np.abs(st["r_W"][m]) / A[0].W[m]
    assert rel.max() < 5e-6                                # float32 storage of W
    # a wrong pose does not transfer exactly
    st2 = O.eval_step(A, B, 0, O.se3_exp([0.0, 0, 0.01, 0, 0, 0]) @ T, FIXED)
    m2 = st2["mask_W"]
    assert (np.abs(st2["r_W"][m2]) / A[0].W[m2]).min() > 100 * rel.max()


@pytest.mark.parametrize("level", [0, 1])
def test_jacobian_matches_central_differences_at_identity(level):
    """J of eqs. res_int / res_depth equals the central finite difference of the
    nonlinear residual under T(xi) = exp(xi)^-1 at xi = 0 (identical frames)."""
    p, A, _ = _pair_levels(2, noise=False)
    st = O.eval_step(A, A, level, np.eye(4), FIXED)
    h = 1e-6
    ok = st["mask_I"] & st["mask_W"]
    for k in range(6):
        e = np.zeros(6); e[k] = h
        sp = O.eval_step(A, A, level, O.se3_inv(O.se3_exp(e)), FIXED)
        sm = O.eval_step(A, A, level, O.se3_inv(O.se3_exp(-e)), FIXED)
        both = ok & sp["mask_I"] & sm["mask_I"] & sp["mask_W"] & sm["mask_W"]
        fdI = (sp["r_I"] - sm["r_I"]) / (2 * h)
        fdW = (sp["r_W"] - sm["r_W"]) / (2 * h)
        JI, JW = st["J_I"][..., k], st["J_W"][..., k]
        sI = np.abs(JI[both]).max()
        sW = np.abs(JW[both]).max()
        assert np.abs(fdI[both] - JI[both]).max() < 2e-4 * sI, k
        assert np.abs(fdW[both] - JW[both]).max() < 2e-4 * sW, k


def test_normal_weight_is_cosine_between_plane_normal_and_ray():
    K = (131.25, 131.25, 79.5, 59.5)
    h, w = 120, 160
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    n, d = np.array([0.35, -0.2, 1.0]), 2.0
    q = np.stack([(u - K[2]) / K[0], (v - K[3]) / K[1], np.ones((h, w))], -1)
    W = (q @ n) / d
    I = 0.5 + 0.001 * u
    A = [O.Level(I, W, K)]
    st = O.eval_step(A, A, 0, np.eye(4), FIXED)
    cosang = (q @ n) / (np.linalg.norm(q, axis=-1) * np.linalg.norm(n))
    m = st["mask_W"]
    assert m.sum() > 15000
    assert np.allclose(st["lam"][m], cosang[m], atol=1e-12)
    # frontal plane: lambda is the cosine of the ray angle
    A2 = [O.Level(I, np.full((h, w), 0.5), K)]
    st2 = O.eval_step(A2, A2, 0, np.eye(4), FIXED)
    assert np.allclose(st2["lam"][st2["mask_W"]], (1 / np.linalg.norm(q, axis=-1))[st2["mask_W"]], atol=1e-14)


def test_brute_force_tiny_images_against_per_pixel_loops():
    """8x6 and 16x12 images: every pixel's masks and residuals recomputed by an
    independent per-pixel loop."""
    rng = np.random.default_rng(5)
    for (h, w) in [(6, 8), (12, 16)]:
        K = (w * 0.8, w * 0.8, (w - 1) / 2, (h - 1) / 2)
        IA, IB = rng.random((h, w)), rng.random((h, w))
        WA, WB = rng.uniform(0.3, 0.6, (h, w)), rng.uniform(0.3, 0.6, (h, w))
        WA[rng.random((h, w)) < 0.15] = 0
        WB[rng.random((h, w)) < 0.15] = 0
        T = O.se3_exp([0.05, -0.03, 0.02, 0.02, -0.03, 0.01])
        st = O.eval_step([O.Level(IA, WA, K)], [O.Level(IB, WB, K)], 0, T, FIXED)
        R, t = T[:3, :3], T[:3, 3]
        for y in range(h):
            for x in range(w):
                mI = mW = False
                rI = rW = 0.0
                if WA[y, x] > 0 and 1 <= x <= w - 2 and 1 <= y <= h - 2:
                    XA = np.array([(x - K[2]) / K[0], (y - K[3]) / K[1], 1.0]) / WA[y, x]
                    XB = R.T @ (XA - t)
                    if XB[2] > 0:
                        ub = K[0] * XB[0] / XB[2] + K[2]
                        vb = K[1] * XB[1] / XB[2] + K[3]
                        x0, y0 = int(np.floor(ub)), int(np.floor(vb))
                        if 0 <= x0 <= w - 2 and 0 <= y0 <= h - 2:
                            ax, ay = ub - x0, vb - y0
                            bil = lambda M: ((1 - ay) * ((1 - ax) * M[y0, x0] + ax * M[y0, x0 + 1])
                                             + ay * ((1 - ax) * M[y0 + 1, x0] + ax * M[y0 + 1, x0 + 1]))
                            mI, rI = True, bil(IB) - IA[y, x]
                            taps = [WB[y0, x0], WB[y0, x0 + 1], WB[y0 + 1, x0], WB[y0 + 1, x0 + 1]]
                            nb = [WA[y, x - 1], WA[y, x + 1], WA[y - 1, x], WA[y + 1, x]]
                            if min(taps) > 0 and min(nb) > 0:
                                wb = bil(WB)
                                Xp = np.array([(ub - K[2]) / K[0], (vb - K[3]) / K[1], 1.0]) / wb
                                zt = (R @ Xp + t)[2]
                                if zt > 0:
                                    mW, rW = True, 1.0 / zt - WA[y, x]
                assert st["mask_I"][y, x] == mI and st["mask_W"][y, x] == mW, (y, x)
                assert abs(st["r_I"][y, x] - rI) < 1e-13 and abs(st["r_W"][y, x] - rW) < 1e-13


# ----------------------------------------------------------------------------- robust statistics
def test_location_scale_gaussian_limit_is_mean_and_population_std():
    r = np.random.default_rng(6).normal(0.3, 0.7, 5000)
    mu, sigma = O.location_scale(r, nu=1e15, iters=3)
    assert abs(mu - np.mean(r)) < 1e-12 and abs(sigma - np.std(r)) < 1e-12


def test_location_scale_fixed_point_matches_student_t_mle():
    r = scipy.stats.t.rvs(4, loc=0.02, scale=0.05, size=19200, random_state=7)
    mu, sigma = O.location_scale(r, nu=5.0, iters=400)
    x = (r - mu) / sigma
    w = (5.0 + 1) / (5.0 + x * x)
    assert abs(np.sum(w * (r - mu))) < 1e-10 * np.sum(np.abs(r))
    assert abs(np.sum(1 - w * x * x)) < 1e-8 * r.size
    _, loc, scale = scipy.stats.t.fit(r, f0=5.0, loc=0.0, scale=0.05)
    # scipy's optimiser stops near the optimum; the fixed point is at least as likely
    assert abs(mu - loc) < 1e-5 and abs(sigma - scale) / scale < 2e-4
    ll = lambda m, s: np.sum(scipy.stats.t.logpdf(r, 5.0, loc=m, scale=s))
    assert ll(mu, sigma) >= ll(loc, scale) - 1e-9


def test_nu_equation_is_twice_the_likelihood_derivative():
    r = scipy.stats.t.rvs(3, loc=0.0, scale=0.1, size=4000, random_state=8)
    mu, sigma = 0.01, 0.09
    x = (r - mu) / sigma
    for nu in (2.0, 3.7, 6.0, 10.0):
        eps = 1e-5
        ll = lambda n: np.sum(scipy.stats.t.logpdf(r, n, loc=mu, scale=sigma))
        fd = (ll(nu + eps) - ll(nu - eps)) / (2 * eps)
        assert abs(O.nu_equation(nu, x) - 2 * fd) < 1e-5 * r.size


def test_nu_bisection_agrees_with_brent_root_of_the_likelihood():
    r = scipy.stats.t.rvs(4, loc=0.0, scale=0.05, size=19200, random_state=9)
    mu, sigma = O.location_scale(r, 5.0, 10)
    nu = O.estimate_nu(r, mu, sigma)
    x = (r - mu) / sigma
    dll = lambda n: np.sum(scipy.stats.t.logpdf(r, n + 1e-6, loc=mu, scale=sigma)
                           - scipy.stats.t.logpdf(r, n - 1e-6, loc=mu, scale=sigma))
    root = scipy.optimize.brentq(dll, 2.0, 10.0, xtol=1e-10)
    assert abs(nu - root) < 2e-5
    assert 3.4 < nu < 4.8                                  # recovers the generating nu


def test_nu_clamps_to_bounds():
    g = np.random.default_rng(10).normal(0, 1, 19200)
    mu, sigma = O.location_scale(g, 5.0, 10)
    # Gaussian residuals (with the scale fitted at nu = 5): the likelihood in nu is
    # still rising or flat at the top of the interval
    assert O.estimate_nu(g, mu, sigma) >= 9.5
    c = scipy.stats.cauchy.rvs(size=19200, random_state=10)
    mu, sigma = O.location_scale(c, 5.0, 10)
    assert O.estimate_nu(c, mu, sigma) == 2.0             # Cauchy: heavier than nu = 2


def test_sample_stride_is_smallest_integer_under_cap():
    expect = {(640, 480): 4, (320, 240): 2, (160, 120): 1, (80, 60): 1,
              (960, 720): 6, (1280, 960): 8, (480, 360): 3}
    for (w, h), s in expect.items():
        assert O.sample_stride(w, h) == s
        got = O.sample_stride(w, h)
        assert int(np.ceil(w / got)) * int(np.ceil(h / got)) <= 19200
        if got > 1:
            assert int(np.ceil(w / (got - 1))) * int(np.ceil(h / (got - 1))) > 19200


def test_paper_constants_are_the_oracle_defaults():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    P = O.AlignParams()
    assert P.nu0 == g["nu_default"]["value"]
    assert [P.nu_lo, P.nu_hi] == g["nu_interval"]["value"]
    assert P.sample_cap == g["sample_cap"]["value"]


# ----------------------------------------------------------------------------- end to end
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pose_recovery_noise_free(seed):
    p, A, B = _pair_levels(seed, noise=False)
    r = O.align(A, B, None, O.AlignParams())
    E = O.se3_inv(p["T_gt"]) @ r["T"]
    assert np.linalg.norm(O.so3_log(E[:3, :3])) < 5e-4
    assert np.linalg.norm(E[:3, 3]) < 5e-4
    assert r["status"] == O.OK


@pytest.mark.parametrize("seed", [4, 5])
def test_pose_recovery_noisy(seed):
    p, A, B = _pair_levels(seed, noise=True)
    r = O.align(A, B, None, O.AlignParams())
    E = O.se3_inv(p["T_gt"]) @ r["T"]
    # a few times the noise-propagated standard deviation from H^-1
    cov = np.linalg.inv(r["H"])
    assert np.linalg.norm(O.so3_log(E[:3, :3])) < max(2e-3, 6 * np.sqrt(np.trace(cov[3:, 3:])))
    assert np.linalg.norm(E[:3, 3]) < max(2e-3, 6 * np.sqrt(np.trace(cov[:3, :3])))


def test_identical_frames_stay_at_identity_and_all_holes_are_degenerate():
    p, A, _ = _pair_levels(0)
    r = O.align(A, A, None, O.AlignParams())
    assert np.array_equal(r["T"], np.eye(4))               # sigma = 0 -> no weight -> no step
    assert r["status"] == O.DEGENERATE
    # a reference frame without any inverse depth gives no residual at all
    Z = [O.Level(l.I, np.zeros_like(l.W), l.K) for l in A]
    r2 = O.align(Z, A, O.se3_exp([0.01, 0, 0, 0, 0, 0]), O.AlignParams())
    assert np.array_equal(r2["T"], O.se3_exp([0.01, 0, 0, 0, 0, 0]))
    assert r2["status"] == O.DEGENERATE and r2["n_valid"] == [0, 0]


# ----------------------------------------------------------------------------- fusion
def test_fusion_identity_identical_frame():
    p = synth.make_pair(3, noise=True)
    I, W = p["I_A"].astype(np.float64), p["W_A"].astype(np.float64)
    C = np.ones_like(W)
    I2, W2, C2, gate = O.fuse(I, W, C, I, W, p["K"], np.eye(4), 1e-3)
    assert gate.sum() > 0.6 * (W > 0).sum()
    assert np.allclose(W2, W, atol=1e-14, rtol=1e-14) and np.allclose(I2, I, atol=1e-14)
    assert np.array_equal(C2[gate], np.full(gate.sum(), 2.0))   # C_k = 1 exactly
    assert np.array_equal(C2[~gate], C[~gate])


def test_fusion_frontal_plane_moved_along_axis_closed_form():
    K = (131.25, 131.25, 79.5, 59.5)
    h, w = 120, 160
    z1, dz = 2.0, 0.1
    W_kf = np.full((h, w), 1 / z1)
    W_k = np.full((h, w), 1 / (z1 - dz))                      # camera moved dz forward
    T = np.eye(4); T[2, 3] = dz                                # kf_T_k
    I = np.full((h, w), 0.4)
    I2, W2, C2, gate = O.fuse(I, W_kf, np.ones((h, w)), I, W_k, K, T, 1e-3)
    assert gate[5:-5, 5:-5].all()
    assert np.allclose(W2[gate], 1 / z1, rtol=1e-14)
    assert np.allclose(C2[gate], 1 + (z1 / (z1 - dz)) ** 4, rtol=1e-12)


def test_fusion_weight_is_inverse_square_of_transfer_derivative():
    p = synth.make_pair(4, noise=False)
    K = p["K"]
    T = p["T_gt"]
    I_kf, W_kf = p["I_A"].astype(np.float64), p["W_A"].astype(np.float64)
    I_k, W_k = p["I_B"].astype(np.float64), p["W_B"].astype(np.float64)
    _, _, Ck, gate = O.fuse(I_kf, W_kf, np.zeros_like(W_kf), I_k, W_k, K, T, 10.0)
    A = O.Level(I_kf, W_kf, K)
    eps = 1e-6
    wp_p = O.inverse_geometric_warp(A, O.Level(I_k, W_k * (1 + eps), K), T)
    wp_m = O.inverse_geometric_warp(A, O.Level(I_k, W_k * (1 - eps), K), T)
    wp0 = O.inverse_geometric_warp(A, O.Level(I_k, W_k, K), T)
    Wp0 = np.where(gate, wp0["W_Bp"], 1.0)
    d = (wp_p["W_Bw"] - wp_m["W_Bw"]) / (2 * eps * Wp0)
    assert gate.sum() > 5000
    assert np.allclose(Ck[gate], 1 / d[gate] ** 2, rtol=1e-6)


def test_fusion_of_equal_weight_frames_is_the_arithmetic_mean():
    rng = np.random.default_rng(12)
    h, w = 30, 40
    K = (32.8, 32.8, 19.5, 14.5)
    W0 = rng.uniform(0.4, 0.6, (h, w))
    I0 = rng.random((h, w))
    I, W, C = I0.copy(), W0.copy(), np.ones((h, w))
    Ws, Is = [W0], [I0]
    every = np.ones((h, w), bool)
    for k in range(5):
        Wk = W0 + rng.uniform(-1e-3, 1e-3, (h, w))
        Ik = rng.random((h, w))
        I, W, C, gate = O.fuse(I, W, C, Ik, Wk, K, np.eye(4), 1.0)
        every &= gate
        Ws.append(Wk); Is.append(Ik)
    # at T = I the warp lands on pixel nodes; nodes whose computed coordinate
    # rounds just below an integer on the first row/column fail the bounds test
    assert every.sum() > 0.9 * (h - 1) * (w - 1)
    assert np.allclose(W[every], np.mean(np.stack(Ws), 0)[every], rtol=1e-12)
    assert np.allclose(I[every], np.mean(np.stack(Is), 0)[every], rtol=1e-12)
    assert np.array_equal(C[every], np.full(every.sum(), 6.0))


def test_so3_projection_is_nearest_rotation():
    rng = np.random.default_rng(21)
    R0 = synth.random_rotation(rng)
    assert np.allclose(O.so3_project(R0), R0, atol=1e-14)          # rotations are fixed points
    E = 1e-4 * rng.normal(size=(3, 3))
    P = O.so3_project(R0 + E)
    assert np.allclose(P.T @ P, np.eye(3), atol=1e-14) and abs(np.linalg.det(P) - 1) < 1e-14
    # nearest in Frobenius norm: no random rotation near R0 is closer
    for _ in range(50):
        Q = R0 @ O.so3_exp(1e-4 * rng.normal(size=3))
        assert np.linalg.norm(R0 + E - P) <= np.linalg.norm(R0 + E - Q) + 1e-15


def test_constant_velocity_drift_is_removed_by_projection():
    """Without re-projection the rotation drift of T1 T2^-1 T1 grows ~2.4x per frame."""
    T2 = np.eye(4)
    T1 = O.se3_exp([0.01, 0, 0, 0, 0.01, 0])
    T1[:3, :3] *= 1 + 1e-12                                         # rounding-sized drift
    free, proj = (T1.copy(), T2.copy()), (T1.copy(), T2.copy())
    for _ in range(30):
        a, b = free
        free = (a @ O.se3_inv(b) @ a, a)
        a, b = proj
        proj = (O.se3_project(a @ O.se3_inv(b) @ a), a)
    orth = lambda T: np.abs(T[:3, :3].T @ T[:3, :3] - np.eye(3)).max()
    assert orth(free[0]) > 1e-3
    assert orth(proj[0]) < 1e-14


def test_reduced_precision_rounding_matches_torch_conversions():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    x = np.concatenate([rng.random(4000), rng.uniform(0.1, 3.0, 4000), [0.0, 1.0, 0.5, 2.0 ** -10]]).astype(np.float32)
    # exact ties of the bfloat16 grid round to even
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], dtype=np.float32)
    x = np.concatenate([x, ties])
    ref_bf = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x), ref_bf)
    assert list(O.round_bf16(ties)) == [1.0, 1.0 + 4 * 2.0 ** -8]
    ref_h = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(O.round_f16(x), ref_h)


def test_reduced_pyramid_rounds_every_level_of_the_fp64_pyramid():
    p = synth.make_pair(1)
    full = O.build_pyramid(p["I_A"], p["W_A"], p["K"], 3)
    red = O.build_pyramid_reduced(p["I_A"], p["W_A"], p["K"], 3)
    for a, b in zip(full, red):
        assert np.array_equal(b.I, O.round_bf16(a.I)) and np.array_equal(b.W, O.round_f16(a.W))
        assert np.array_equal(b.W > 0, a.W > 0)
        assert np.max(np.abs(b.I - a.I)) <= 2.0 ** -9 and np.max(np.abs(b.W - a.W) / np.where(a.W > 0, a.W, 1)) <= 2.0 ** -11
