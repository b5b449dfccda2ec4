"""Plain FP64 oracle of RGBiD-SLAM's data-parallel hot path (arXiv 1807.08271).

TEST INFRASTRUCTURE ONLY (see the package header): the product never imports it.

Notation follows the paper.  A is the reference frame (the keyframe), B the
current frame; ``T = A_T_B`` maps B's coordinates into A's (X_A = R X_B + t).
Pixels are ``p = (u, v, 1)`` with u the column and v the row index;
``K = (fx, fy, cx, cy)``; an inverse-depth hole is ``W = 0``.  All arithmetic is
float64; the float32 input planes are widened exactly.

Citations name the paper's section and equation label:
  * "Preliminaries"   - SO(3)/SE(3) exp and log, the decoupled SE(3) maps.
  * "Warping functions" - eq. 3d_registration and the inverse geometric warping.
  * "Dense motion estimation" - eqs. intCons, depthCons, DeltaX, res_int,
    res_depth, minimisationIRLS, the normal weight lambda_n, the update rule;
    "Error distribution and robust optimisation" - eqs. Student_pdf,
    logLikelihood_St, the location/scale equations, robustnessValue, the
    N = 19200 systematic sample; "Dense frame covisibility ratio" - the 3 sigma_W
    visibility test.
  * "Keyframe fusion" (section "RGB-ID SLAM system") - the weighted mean and the
    weight C_k from propagating inverse-depth variance through eq. 3d_registration.

Readings taken where the paper is silent, ambiguous or garbled (R1..R17):
  R1  pyramid: 2x2 box mean of I; W = mean of the valid (> 0) children, 0 if
      none; summation order (a+b)+(c+d); odd sizes drop the last row/column;
      K_{l+1}: f/2 and c <- (c + 0.5)/2 - 0.5.
  R2  B is warped directly at each pyramid level with K_l.
  R3  gradients are central differences in level pixels; border pixels have
      none; grad W needs all four neighbours > 0.
  R4  software bilinear: x0 = floor(x), valid iff 0 <= x0 and x0 + 1 <= w - 1
      (same for y).
  R5  mask_I = W_A > 0, interior, Z_B > 0, bilinear-valid;
      mask_W = mask_I, all four W_B taps > 0, grad W_A valid, transferred Z > 0.
  R6  sample stride s = smallest integer with ceil(w/s) ceil(h/s) <= 19200;
      samples at u = 0 mod s and v = 0 mod s that pass the channel's mask.
  R7  W_B^gamma(p) = 1 / e_z^T (R K^-1 p_B / W_B(p_B) + t).
  R8  lambda_n uses the ray K^-1 p for p and n = n_u / |n_u|.
  R9  (mu, sigma) at nu = 5: mu0 = 0, sigma0 = sqrt(mean r^2), 10 fixed
      iterations of the linear system with lagged weights (mu first, then
      sigma^2 = (1/n) sum w (r - mu_new)^2); sigma < 1e-12 -> channel weight 0.
  R10 nu by bisection on eq. robustnessValue over [2, 10] with mu, sigma fixed:
      f(10) >= 0 -> 10, f(2) <= 0 -> 2, else 20 halvings and the midpoint.
      nu_I <- max(nu_I, nu_W) when both channels are valid.
  R11 Rodrigues with (1 - cos|theta|)/|theta|^2 (the printed 1/|theta| is a
      typo); Taylor terms below |theta| = 1e-8.
  R12 iterations per level are given coarsest-last in ``iters`` (index = level,
      0 = finest); levels are visited coarse to fine.
  R13 fusion weight C_k = (dW*/dW_B)^-2 at W_B(p_B); intensity is averaged
      with the same weights behind the same gate.
  R14 sigma_W of the fusion gate is passed in (the frame's final alignment).
  R16 an iteration is skipped (no update, status DEGENERATE) when the valid
      residual count is below ``min_valid`` or H is not positive definite.
  R18 the constant-velocity guess T1 T2^-1 T1 is projected onto SE(3) (nearest
      rotation); otherwise rounding drift of the rotation block compounds by
      ~2.4x per frame and tracking is lost after a few dozen frames.
  R19 a pixel whose I or W is not a finite number carries no measurement (the
      paper's sensor gives finite intensities and marks missing depth only):
      it enters the pyramid and the keyframe as a hole, W = 0, with I = 0
      where I is not finite; in fusion such a keyframe pixel or frame-k tap is
      not a measurement.
  R20 covariance: the extra iteration runs at the finest level at the final
      pose, estimates (mu, sigma, nu) on the systematic sample like any
      iteration, and takes the bilateral-filtered planes only where the paper
      names them, in the gradients of {I_A, W_A} (the Jacobians and lambda_n);
      the warp, residuals, masks and W_A itself stay unfiltered.  The bilateral
      filter (parameters unstated: radius, sigma_s and the range sigmas are
      configuration) weighs the (2r+1)^2 window inside the image by
      exp(-d^2 / 2 sigma_s^2) exp(-(f(p) - f(q))^2 / 2 sigma_r^2); W only over
      valid (> 0) neighbours, holes stay holes.
  R21 covisibility: S_V counts a valid pixel of A whose transfer lies in front
      of B and whose nearest pixel of B, floor(p_B + 1/2), lies in the image,
      holds a valid W_B and passes |W_B - w_B| < 3 sigma_W with w_B = 1 / Z_B
      (the ratio only counts, so no interpolation of W_B is needed; with four
      valid taps required, 10 % scattered holes alone would cut every ratio to
      about 0.65); sigma_W is the frame's final one (as R14).  The tracker
      switches keyframe, optionally, when min(vr_AB, vr_BA) between the
      keyframe and the aligned frame falls below the threshold (0.7 in the
      paper); the switch frame is handled as in R15.
  R22 warp-then-downsample mode: B is warped at level 0 with K_0; the warped
      maps I_B*, W_B* (valid where mask_I's, resp. mask_W's warp conditions
      hold at level 0) are reduced to level l by R1's rule applied to both,
      each with its own validity (mean of the valid children, valid when one
      is); level l's masks are A's conditions there plus that validity.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import digamma

# ----------------------------------------------------------------------------- status codes
OK = 0
DEGENERATE = 4


# ----------------------------------------------------------------------------- Lie groups
def hat(w) -> np.ndarray:
    """Skew-symmetric matrix [w]x ("Preliminaries")."""
    w = np.asarray(w, dtype=np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def vee(S) -> np.ndarray:
    return np.array([S[2, 1], S[0, 2], S[1, 0]], dtype=np.float64)


def so3_exp(theta) -> np.ndarray:
    """exp([theta]x) by Rodrigues' formula ("Preliminaries"), reading R11."""
    theta = np.asarray(theta, dtype=np.float64)
    th = float(np.linalg.norm(theta))
    S = hat(theta)
    if th < 1e-8:
        return np.eye(3) + S + 0.5 * (S @ S)
    return np.eye(3) + (np.sin(th) / th) * S + ((1.0 - np.cos(th)) / (th * th)) * (S @ S)


def so3_log(R) -> np.ndarray:
    """log(R): |theta| = arccos((tr R - 1)/2), [theta]x = |theta| (R - R^T)/(2 sin|theta|)."""
    R = np.asarray(R, dtype=np.float64)
    c = np.clip((np.trace(R) - 1.0) * 0.5, -1.0, 1.0)
    th = float(np.arccos(c))
    if th < 1e-8:
        return vee(0.5 * (R - R.T))
    return vee(th * (R - R.T) / (2.0 * np.sin(th)))


def se3_exp(xi) -> np.ndarray:
    """Decoupled SE(3) exponential ("Preliminaries"): [exp([theta]x), v; 0, 1] with xi = (v, theta)."""
    xi = np.asarray(xi, dtype=np.float64)
    T = np.eye(4)
    T[:3, :3] = so3_exp(xi[3:6])
    T[:3, 3] = xi[0:3]
    return T


def se3_log(T) -> np.ndarray:
    """Decoupled SE(3) logarithm: (t, log R)."""
    T = np.asarray(T, dtype=np.float64)
    return np.concatenate([T[:3, 3], so3_log(T[:3, :3])])


def so3_project(R) -> np.ndarray:
    """Nearest rotation matrix (polar factor U V^T of the SVD), reading R18: the
    constant-velocity composition is re-projected onto SO(3) because rounding
    drift in the rotation block grows ~2.4x per frame through T1 T2^-1 T1."""
    U, _, Vt = np.linalg.svd(np.asarray(R, dtype=np.float64))
    P = U @ Vt
    if np.linalg.det(P) < 0:
        U[:, -1] = -U[:, -1]
        P = U @ Vt
    return P


def se3_project(T) -> np.ndarray:
    T = np.asarray(T, dtype=np.float64).copy()
    T[:3, :3] = so3_project(T[:3, :3])
    T[3] = (0.0, 0.0, 0.0, 1.0)
    return T


def se3_inv(T) -> np.ndarray:
    T = np.asarray(T, dtype=np.float64)
    Ti = np.eye(4)
    Ti[:3, :3] = T[:3, :3].T
    Ti[:3, 3] = -T[:3, :3].T @ T[:3, 3]
    return Ti


# ----------------------------------------------------------------------------- pyramid
@dataclass
class Level:
    I: np.ndarray   # float64 [h, w]
    W: np.ndarray   # float64 [h, w], 0 = hole
    K: tuple        # (fx, fy, cx, cy) at this level


def measurement_planes(I, W):
    """Level-0 planes with every non-finite pixel made a hole (reading R19):
    W = 0 where I or W is not finite, I = 0 where I is not finite; every other
    pixel unchanged."""
    I = np.asarray(I, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    fin_I = np.isfinite(I)
    return np.where(fin_I, I, 0.0), np.where(fin_I & np.isfinite(W), W, 0.0)


def downsample(I, W):
    """One pyramid step ("Iterative optimisation": downsample {I_A, W_A}), reading R1."""
    I = np.asarray(I, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    h2, w2 = I.shape[0] // 2, I.shape[1] // 2
    ia, ib = I[0:2 * h2:2, 0:2 * w2:2], I[0:2 * h2:2, 1:2 * w2:2]
    ic, id_ = I[1:2 * h2:2, 0:2 * w2:2], I[1:2 * h2:2, 1:2 * w2:2]
    I1 = ((ia + ib) + (ic + id_)) / 4.0
    kids = [W[0:2 * h2:2, 0:2 * w2:2], W[0:2 * h2:2, 1:2 * w2:2],
            W[1:2 * h2:2, 0:2 * w2:2], W[1:2 * h2:2, 1:2 * w2:2]]
    valid = [k > 0 for k in kids]
    z = [np.where(v, k, 0.0) for k, v in zip(kids, valid)]
    n = valid[0].astype(np.float64) + valid[1] + valid[2] + valid[3]
    s = (z[0] + z[1]) + (z[2] + z[3])
    W1 = np.where(n > 0, s / np.where(n > 0, n, 1.0), 0.0)
    return I1, W1


def level_intrinsics(K0, level: int) -> tuple:
    """K at a pyramid level (reading R1): f halves; c <- (c + 0.5)/2 - 0.5 per step."""
    fx, fy, cx, cy = (float(k) for k in K0)
    for _ in range(level):
        fx, fy = fx / 2.0, fy / 2.0
        cx, cy = (cx + 0.5) / 2.0 - 0.5, (cy + 0.5) / 2.0 - 0.5
    return (fx, fy, cx, cy)


def build_pyramid(I0, W0, K0, levels: int) -> list:
    """Image pyramid {I, W} per level, finest first (level 0: reading R19)."""
    I, W = measurement_planes(I0, W0)
    pyr = [Level(I, W, tuple(float(k) for k in K0))]
    for l in range(1, levels):
        I, W = downsample(I, W)
        pyr.append(Level(I, W, level_intrinsics(K0, l)))
    return pyr


def round_bf16(x) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even), via float32, as float64.

    Storage of the reduced-precision form: each level's intensity is held as
    bfloat16."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = r.astype(np.uint32).view(np.float32)
    out = np.where(np.isnan(f), f, out)
    return out.astype(np.float64)


def round_f16(x) -> np.ndarray:
    """Round to IEEE binary16 (round to nearest even), via float32, as float64 (the
    reduced-precision form's inverse-depth storage)."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def build_pyramid_reduced(I0, W0, K0, levels: int) -> list:
    """Pyramid of the reduced-precision form: every level computed from level 0
    as in ``build_pyramid``, then I rounded to bfloat16 and W to binary16."""
    return [Level(round_bf16(l.I), round_f16(l.W), l.K) for l in build_pyramid(I0, W0, K0, levels)]


def gradients(I, W):
    """Central-difference gradients of I and W (reading R3).

    Returns gIx, gIy, gWx, gWy (0 where undefined), ``interior`` (not on the
    border) and ``gW_valid`` (interior and all four W neighbours > 0)."""
    h, w = I.shape
    gIx = np.zeros((h, w)); gIy = np.zeros((h, w))
    gWx = np.zeros((h, w)); gWy = np.zeros((h, w))
    gIx[:, 1:-1] = (I[:, 2:] - I[:, :-2]) / 2.0
    gIy[1:-1, :] = (I[2:, :] - I[:-2, :]) / 2.0
    gWx[:, 1:-1] = (W[:, 2:] - W[:, :-2]) / 2.0
    gWy[1:-1, :] = (W[2:, :] - W[:-2, :]) / 2.0
    interior = np.zeros((h, w), dtype=bool)
    interior[1:-1, 1:-1] = True
    Wv = W > 0
    nb = np.zeros((h, w), dtype=bool)
    nb[1:-1, 1:-1] = Wv[1:-1, 2:] & Wv[1:-1, :-2] & Wv[2:, 1:-1] & Wv[:-2, 1:-1]
    return gIx, gIy, gWx, gWy, interior, interior & nb


def bilinear(img, x, y):
    """Bilinear interpolation at (x, y) (reading R4).

    Returns (value, valid, taps) where taps = (v00, v10, v01, v11) are the four
    neighbours (x0,y0), (x0+1,y0), (x0,y0+1), (x0+1,y0+1)."""
    h, w = img.shape
    x0 = np.floor(x)
    y0 = np.floor(y)
    valid = (x0 >= 0) & (x0 + 1 <= w - 1) & (y0 >= 0) & (y0 + 1 <= h - 1)
    xi = np.where(valid, x0, 0).astype(np.int64)
    yi = np.where(valid, y0, 0).astype(np.int64)
    ax = np.where(valid, x - x0, 0.0)
    ay = np.where(valid, y - y0, 0.0)
    v00 = img[yi, xi]; v10 = img[yi, xi + 1]
    v01 = img[yi + 1, xi]; v11 = img[yi + 1, xi + 1]
    val = (1 - ay) * ((1 - ax) * v00 + ax * v10) + ay * ((1 - ax) * v01 + ax * v11)
    return np.where(valid, val, 0.0), valid, (v00, v10, v01, v11)


# ----------------------------------------------------------------------------- warping
def inverse_geometric_warp(A: Level, B: Level, T):
    """Inverse geometric warping of B towards A ("Warping functions", eq. 3d_registration
    and the two relations of the inverse geometric warping; readings R4, R5, R7).

    For each pixel p of A: X_A = K^-1 p / W_A(p), X_B = R^T (X_A - t), p_B = pi(X_B);
    I_B*(p) = I_B(p_B) and W_B*(p) = B's inverse depth at p_B transferred into A."""
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    fx, fy, cx, cy = A.K
    h, w = A.W.shape
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    q = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones((h, w))], axis=-1)   # K^-1 p
    WA = A.W
    validA = WA > 0
    X_A = q / np.where(validA, WA, 1.0)[..., None]
    X_B = (X_A - t) @ R                      # rows of R^T (X_A - t)
    Z_B = X_B[..., 2]
    front = Z_B > 0
    Zs = np.where(front, Z_B, 1.0)
    u_B = fx * X_B[..., 0] / Zs + cx
    v_B = fy * X_B[..., 1] / Zs + cy
    I_Bw, bil_valid, _ = bilinear(B.I, u_B, v_B)
    W_Bp, _, taps = bilinear(B.W, u_B, v_B)
    all4 = bil_valid & (taps[0] > 0) & (taps[1] > 0) & (taps[2] > 0) & (taps[3] > 0)
    qB = np.stack([(u_B - cx) / fx, (v_B - cy) / fy, np.ones((h, w))], axis=-1)
    Xp_B = qB / np.where(all4, W_Bp, 1.0)[..., None]
    Zp = Xp_B @ R[2, :] + t[2]               # e_z^T (R X'_B + t)
    zp_pos = Zp > 0
    W_Bw = np.where(all4 & zp_pos, 1.0 / np.where(zp_pos, Zp, 1.0), 0.0)
    return dict(q=q, X_A=X_A, X_B=X_B, Z_B=Z_B, front=front, u_B=u_B, v_B=v_B,
                I_Bw=I_Bw, bil_valid=bil_valid, W_Bp=W_Bp, all4=all4, Zp=Zp, W_Bw=W_Bw,
                validA=validA, u=u, v=v)


# ----------------------------------------------------------------------------- robust statistics
def omega(x, nu):
    """Student-t IRLS weight w(x, nu) = (1/x) d rho/dx = (nu + 1)/(nu + x^2)
    (eq. logLikelihood_St with rho = (nu+1)/2 ln(nu + x^2))."""
    return (nu + 1.0) / (nu + np.asarray(x, dtype=np.float64) ** 2)


def location_scale(r, nu: float = 5.0, iters: int = 10, sigma_floor: float = 1e-12):
    """(mu, sigma) from the two likelihood equations with lagged weights
    ("Error distribution and robust optimisation"), reading R9."""
    r = np.asarray(r, dtype=np.float64)
    n = r.size
    if n == 0:
        return 0.0, 0.0
    mu = 0.0
    sigma = float(np.sqrt(np.mean(r * r)))
    for _ in range(iters):
        if sigma < sigma_floor:
            break
        wts = omega((r - mu) / sigma, nu)
        mu = float(np.sum(wts * r) / np.sum(wts))
        sigma = float(np.sqrt(np.sum(wts * (r - mu) ** 2) / n))
    return mu, sigma


def nu_equation(nu: float, x) -> float:
    """Left side of eq. robustnessValue: sum_i [-psi(nu/2) + ln(nu/2) + psi((nu+1)/2)
    - ln((nu+1)/2) + 1 + ln w(x_i, nu) - w(x_i, nu)], psi the digamma function."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    wts = omega(x, nu)
    const = -digamma(nu / 2.0) + np.log(nu / 2.0) + digamma((nu + 1.0) / 2.0) - np.log((nu + 1.0) / 2.0) + 1.0
    return float(n * const + np.sum(np.log(wts) - wts))


def estimate_nu(r, mu: float, sigma: float, lo: float = 2.0, hi: float = 10.0, steps: int = 20) -> float:
    """Bisection for nu on eq. robustnessValue with (mu, sigma) fixed, reading R10."""
    x = (np.asarray(r, dtype=np.float64) - mu) / sigma
    if nu_equation(hi, x) >= 0:
        return float(hi)
    if nu_equation(lo, x) <= 0:
        return float(lo)
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        if nu_equation(mid, x) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@dataclass
class AlignParams:
    """Alignment schedule and robust-estimation constants (``warp_mode``: "level"
    warps B at each level, "full" warps at level 0 and downsamples, reading R22)."""
    levels: int = 3
    iters: tuple = (5, 5, 10)          # per level, index 0 = finest (reading R12)
    scale_iters: int = 10              # reading R9
    bisect_steps: int = 20             # reading R10
    sample_cap: int = 19200            # N of the systematic sample
    estimate_nu: bool = True
    nu0: float = 5.0
    nu_lo: float = 2.0
    nu_hi: float = 10.0
    min_valid: int = 60                # reading R16
    sigma_floor: float = 1e-12
    warp_mode: str = "level"


def robust_params(rI, rW, P: AlignParams):
    """(mu, sigma, nu) for both channels from the sampled residuals.

    Returns dict(mu=[I, W], sigma=[I, W], nu=[I, W], ok=[I, W], n=[I, W])."""
    out = dict(mu=[0.0, 0.0], sigma=[0.0, 0.0], nu=[P.nu0, P.nu0], ok=[False, False],
               n=[int(np.size(rI)), int(np.size(rW))])
    for c, r in enumerate((rI, rW)):
        r = np.asarray(r, dtype=np.float64)
        if r.size == 0:
            continue
        mu, sigma = location_scale(r, P.nu0, P.scale_iters, P.sigma_floor)
        out["mu"][c], out["sigma"][c] = mu, sigma
        if sigma < P.sigma_floor:
            continue
        out["ok"][c] = True
        if P.estimate_nu:
            out["nu"][c] = estimate_nu(r, mu, sigma, P.nu_lo, P.nu_hi, P.bisect_steps)
    if P.estimate_nu and out["ok"][0] and out["ok"][1]:
        out["nu"][0] = max(out["nu"][0], out["nu"][1])
    return out


def sample_stride(w: int, h: int, cap: int = 19200) -> int:
    """Systematic-sample stride (reading R6)."""
    s = 1
    while -(-w // s) * -(-h // s) > cap:
        s += 1
    return s


# ----------------------------------------------------------------------------- one IRLS step
def downsample_valid(X, valid):
    """R1's reduction of a map with its own validity: each coarse pixel is the mean
    of its valid children, summed (a+b)+(c+d), and valid when one child is (reading R22)."""
    X = np.where(valid, np.asarray(X, dtype=np.float64), 0.0)
    h2, w2 = X.shape[0] // 2, X.shape[1] // 2
    kids = [(X[0:2 * h2:2, 0:2 * w2:2], valid[0:2 * h2:2, 0:2 * w2:2]),
            (X[0:2 * h2:2, 1:2 * w2:2], valid[0:2 * h2:2, 1:2 * w2:2]),
            (X[1:2 * h2:2, 0:2 * w2:2], valid[1:2 * h2:2, 0:2 * w2:2]),
            (X[1:2 * h2:2, 1:2 * w2:2], valid[1:2 * h2:2, 1:2 * w2:2])]
    n = kids[0][1].astype(np.float64) + kids[1][1] + kids[2][1] + kids[3][1]
    s = (kids[0][0] + kids[1][0]) + (kids[2][0] + kids[3][0])
    return np.where(n > 0, s / np.where(n > 0, n, 1.0), 0.0), n > 0


def warped_full_resolution(pyrA, pyrB, level: int, T):
    """The warped maps of "Iterative optimisation" read literally (reading R22): B
    warped towards A at level 0, then downsampled to ``level``.  Returns
    (I_B*, valid_I, W_B*, valid_W) at that level."""
    wp = inverse_geometric_warp(pyrA[0], pyrB[0], T)
    vI = wp["validA"] & wp["front"] & wp["bil_valid"]
    vW = vI & wp["all4"] & (wp["Zp"] > 0)
    I_s, W_s = np.where(vI, wp["I_Bw"], 0.0), np.where(vW, wp["W_Bw"], 0.0)
    for _ in range(level):
        I_s, vI = downsample_valid(I_s, vI)
        W_s, vW = downsample_valid(W_s, vW)
    return I_s, vI, W_s, vW


def eval_step(pyrA, pyrB, level: int, T, robust=None, P: AlignParams | None = None, grad_planes=None):
    """Residuals, Jacobians, weights and normal equations at one level and pose.

    Residuals r(p, 0) of eqs. res_int / res_depth; Jacobians of the same
    equations, J = g M(p) with M(p) = [I3 | -[X_A]x] (eq. DeltaX); weights of
    eq. minimisationIRLS; H = sum w J^T J and g = sum w J^T r(p, 0), so that the
    step solves H xi = -g.  ``robust`` = dict(mu, sigma, nu) per channel, or
    None to estimate it on the systematic sample.  ``grad_planes`` = (I, W) at
    this level whose gradients replace A's (the covariance iteration, reading
    R20); ``P.warp_mode`` "full" takes the warped maps of reading R22."""
    P = P or AlignParams()
    A, B = pyrA[level], pyrB[level]
    fx, fy, cx, cy = A.K
    h, w = A.W.shape
    wp = inverse_geometric_warp(A, B, T)
    if grad_planes is None:
        gIx, gIy, gWx, gWy, interior, gW_valid = gradients(A.I, A.W)
    else:
        gIx, gIy, gWx, gWy, interior, gW_valid = gradients(*grad_planes)
    if P.warp_mode == "full":
        I_s, vI, W_s, vW = warped_full_resolution(pyrA, pyrB, level, T)
        wp["I_Bw"], wp["W_Bw"] = I_s, W_s
        mask_I = wp["validA"] & interior & vI
        mask_W = mask_I & vW & gW_valid
    else:
        mask_I = wp["validA"] & interior & wp["front"] & wp["bil_valid"]
        mask_W = mask_I & wp["all4"] & gW_valid & (wp["Zp"] > 0)
    r_I = np.where(mask_I, wp["I_Bw"] - A.I, 0.0)
    r_W = np.where(mask_W, wp["W_Bw"] - A.W, 0.0)

    if robust is None:
        s = sample_stride(w, h, P.sample_cap)
        sm = (np.mod(wp["u"], s) == 0) & (np.mod(wp["v"], s) == 0)
        rob = robust_params(r_I[sm & mask_I], r_W[sm & mask_W], P)
    else:
        rob = dict(mu=list(robust["mu"]), sigma=list(robust["sigma"]), nu=list(robust["nu"]),
                   ok=[robust["sigma"][0] >= P.sigma_floor, robust["sigma"][1] >= P.sigma_floor],
                   n=[-1, -1])

    # (K - p e_z^T) per pixel; its last row is zero
    KP = np.zeros((h, w, 3, 3))
    KP[..., 0, 0] = fx
    KP[..., 0, 2] = cx - wp["u"]
    KP[..., 1, 1] = fy
    KP[..., 1, 2] = cy - wp["v"]
    gradI = np.stack([gIx, gIy, np.zeros((h, w))], axis=-1)
    gradW = np.stack([gWx, gWy, np.zeros((h, w))], axis=-1)
    ez = np.array([0.0, 0.0, 1.0])
    WA = A.W
    gI = WA[..., None] * np.einsum("hwi,hwij->hwj", gradI, KP)
    gW = WA[..., None] * (np.einsum("hwi,hwij->hwj", gradW, KP) + wp["W_Bw"][..., None] * ez)
    # M(p) = [I3 | -[X_A]x]
    X = wp["X_A"]
    M = np.zeros((h, w, 3, 6))
    M[..., 0, 0] = M[..., 1, 1] = M[..., 2, 2] = 1.0
    M[..., 0, 4], M[..., 0, 5] = X[..., 2], -X[..., 1]     # -[X]x
    M[..., 1, 3], M[..., 1, 5] = -X[..., 2], X[..., 0]
    M[..., 2, 3], M[..., 2, 4] = X[..., 1], -X[..., 0]
    J_I = np.einsum("hwi,hwij->hwj", gI, M)
    J_W = np.einsum("hwi,hwij->hwj", gW, M)

    # normal-vector weight lambda_n = n^T q / |q|, n = n_u / |n_u| (reading R8)
    Winv = 1.0 / np.where(WA > 0, WA, 1.0)
    n_u = Winv[..., None] * np.einsum("hwi,hwij->hwj", gradW, KP) + ez
    n_hat = n_u / np.linalg.norm(n_u, axis=-1, keepdims=True)
    q = wp["q"]
    lam = np.einsum("hwi,hwi->hw", n_hat, q) / np.linalg.norm(q, axis=-1)

    muI, muW = rob["mu"]
    sI, sW = rob["sigma"]
    nuI, nuW = rob["nu"]
    if rob["ok"][0]:
        w_I = omega((r_I - muI) / sI, nuI) / (sI * sI)
    else:
        w_I = np.zeros((h, w))
    if rob["ok"][1]:
        w_W = lam * omega((r_W - muW) / sW, nuW) / (sW * sW)
    else:
        w_W = np.zeros((h, w))
    w_I = np.where(mask_I, w_I, 0.0)
    w_W = np.where(mask_W, w_W, 0.0)

    H = np.einsum("hw,hwi,hwj->ij", w_I, J_I, J_I) + np.einsum("hw,hwi,hwj->ij", w_W, J_W, J_W)
    g = np.einsum("hw,hwi,hw->i", w_I, J_I, r_I) + np.einsum("hw,hwi,hw->i", w_W, J_W, r_W)
    cost = float(np.sum(w_I * r_I * r_I) + np.sum(w_W * r_W * r_W))
    return dict(r_I=r_I, r_W=r_W, mask_I=mask_I, mask_W=mask_W, H=H, g=g, cost=cost,
                n_valid=[int(mask_I.sum()), int(mask_W.sum())], robust=rob,
                w_I=w_I, w_W=w_W, lam=lam, J_I=J_I, J_W=J_W, warp=wp)


def solve_update(H, g, T, n_valid_total: int, min_valid: int):
    """Solve H xi = -g and apply T <- exp(xi)^-1 T ("Iterative optimisation").

    Returns (T_new, xi, ok); ok is False (T unchanged) for a degenerate step (R16)."""
    if n_valid_total < min_valid:
        return np.asarray(T, dtype=np.float64).copy(), np.zeros(6), False
    try:
        np.linalg.cholesky(H)
    except np.linalg.LinAlgError:
        return np.asarray(T, dtype=np.float64).copy(), np.zeros(6), False
    xi = np.linalg.solve(H, -np.asarray(g))
    return se3_inv(se3_exp(xi)) @ np.asarray(T, dtype=np.float64), xi, True


def align(pyrA, pyrB, T_init=None, P: AlignParams | None = None):
    """Coarse-to-fine IRLS Gauss-Newton alignment ("Iterative optimisation").

    Returns dict(T, H, g, robust, cost, n_valid, status, iters_done, trace)."""
    P = P or AlignParams()
    T = np.eye(4) if T_init is None else np.asarray(T_init, dtype=np.float64).copy()
    status = OK
    trace = []
    last = None
    done = 0
    for level in range(P.levels - 1, -1, -1):
        for _ in range(P.iters[level]):
            st = eval_step(pyrA, pyrB, level, T, None, P)
            T_new, xi, ok = solve_update(st["H"], st["g"], T, st["n_valid"][0] + st["n_valid"][1], P.min_valid)
            if not ok:
                status = DEGENERATE
            T = T_new
            done += 1
            last = st
            trace.append(dict(level=level, T=T.copy(), xi=xi, cost=st["cost"], robust=st["robust"],
                              n_valid=st["n_valid"], ok=ok))
    return dict(T=T, H=last["H"], g=last["g"], robust=last["robust"], cost=last["cost"],
                n_valid=last["n_valid"], status=status, iters_done=done, trace=trace)


# ----------------------------------------------------------------------------- keyframe fusion
def fuse(I_kf, W_kf, C_kf, I_k, W_k, K, T, sigma_W: float, fuse_intensity: bool = True):
    """Fuse frame k into the keyframe ("Keyframe fusion"), readings R13, R14.

    T = kf_T_k.  Each keyframe pixel with W_kf > 0 is warped into frame k with
    eq. 3d_registration; it passes when p_k is bilinear-valid with four valid W_k
    taps, the point lies in front of both cameras, and |W_k(p_k) - w_k| < 3 sigma_W
    (the visibility test of "Dense frame covisibility ratio").  Then
    W_kf <- (W_kf C_kf + C_k W_k*)/(C_kf + C_k), C_kf <- C_kf + C_k, with W_k* the
    transferred inverse depth and C_k = (dW_k*/dW_k(p_k))^-2.
    Returns new (I_kf, W_kf, C_kf, fused_mask) as float64 arrays."""
    I_kf = np.asarray(I_kf, dtype=np.float64)
    W_kf = np.asarray(W_kf, dtype=np.float64)
    C_kf = np.asarray(C_kf, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    # non-finite keyframe pixels and frame-k taps are not measurements (reading R19);
    # where the gate passes the keyframe values are the given ones
    A = Level(*measurement_planes(I_kf, W_kf), tuple(float(k) for k in K))
    B = Level(*measurement_planes(I_k, W_k), A.K)
    wp = inverse_geometric_warp(A, B, T)
    fx, fy, cx, cy = A.K
    w_B = 1.0 / np.where(wp["front"], wp["Z_B"], 1.0)
    gate = wp["validA"] & wp["front"] & wp["all4"] & (np.abs(wp["W_Bp"] - w_B) < 3.0 * sigma_W) & (wp["Zp"] > 0)
    W_star = wp["W_Bw"]
    qB = np.stack([(wp["u_B"] - cx) / fx, (wp["v_B"] - cy) / fy, np.ones_like(wp["u_B"])], axis=-1)
    a = qB @ R[2, :]                                  # e_z^T R K^-1 p_k
    Wk = np.where(gate, wp["W_Bp"], 1.0)
    dW = a / (a + t[2] * Wk) ** 2                     # d W_k* / d W_k(p_k)
    C_k = np.where(gate, 1.0 / np.where(gate, dW, 1.0) ** 2, 0.0)
    denom = C_kf + C_k
    W_new = np.where(gate, (W_kf * C_kf + C_k * W_star) / np.where(gate, denom, 1.0), W_kf)
    if fuse_intensity:
        I_new = np.where(gate, (I_kf * C_kf + C_k * wp["I_Bw"]) / np.where(gate, denom, 1.0), I_kf)
    else:
        I_new = I_kf.copy()
    C_new = np.where(gate, denom, C_kf)
    return I_new, W_new, C_new, gate



# ----------------------------------------------------------------------------- covariance of the estimate
@dataclass
class BilateralParams:
    """Bilateral filter of the covariance iteration (reading R20; the paper gives no values)."""
    radius: int = 2
    sigma_s: float = 1.5        # pixels
    sigma_r_I: float = 0.1      # intensity units
    sigma_r_W: float = 0.01     # inverse depth, 1/m


def bilateral_filter(I, W, F: BilateralParams):
    """Bilateral filter of {I_A, W_A} (reading R20), one output pixel at a time:
    out(p) = sum_q k(p, q) f(q) / sum_q k(p, q) over the window q = p + (dx, dy),
    |dx|, |dy| <= radius, inside the image, with
    k = exp(-(dx^2 + dy^2) / (2 sigma_s^2)) exp(-(f(p) - f(q))^2 / (2 sigma_r^2));
    for W only neighbours with W > 0 take part and a hole stays a hole."""
    I = np.asarray(I, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    h, w = I.shape
    r = int(F.radius)
    num_I = np.zeros((h, w)); den_I = np.zeros((h, w))
    num_W = np.zeros((h, w)); den_W = np.zeros((h, w))
    validW = W > 0
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            gs = np.exp(-(dx * dx + dy * dy) / (2.0 * F.sigma_s ** 2))
            # q = p + (dx, dy) for every p whose q lies inside the image
            ys, ye = max(0, -dy), min(h, h - dy)
            xs, xe = max(0, -dx), min(w, w - dx)
            P_I, Q_I = I[ys:ye, xs:xe], I[ys + dy:ye + dy, xs + dx:xe + dx]
            kI = gs * np.exp(-(P_I - Q_I) ** 2 / (2.0 * F.sigma_r_I ** 2))
            num_I[ys:ye, xs:xe] += kI * Q_I
            den_I[ys:ye, xs:xe] += kI
            P_W, Q_W = W[ys:ye, xs:xe], W[ys + dy:ye + dy, xs + dx:xe + dx]
            kW = np.where(validW[ys + dy:ye + dy, xs + dx:xe + dx],
                          gs * np.exp(-(P_W - Q_W) ** 2 / (2.0 * F.sigma_r_W ** 2)), 0.0)
            num_W[ys:ye, xs:xe] += kW * Q_W
            den_W[ys:ye, xs:xe] += kW
    I_f = num_I / den_I
    W_f = np.where(validW, num_W / np.where(validW, den_W, 1.0), 0.0)
    return I_f, W_f


def covariance(pyrA, pyrB, T, P: AlignParams | None = None, F: BilateralParams | None = None):
    """Covariance of the motion estimate ("Dense motion estimation", the paragraph
    after the update rule): one more iteration at the final pose T, not updating
    it, with {I_A, W_A} bilateral-filtered before their gradients are taken;
    Sigma = H_filt^-1 (reading R20).  Returns dict(H, Sigma, robust, n_valid, ok);
    ok is False (Sigma = 0) when H_filt is not positive definite (reading R16)."""
    P = P or AlignParams()
    F = F or BilateralParams()
    A0 = pyrA[0]
    I_f, W_f = bilateral_filter(A0.I, A0.W, F)
    st = eval_step(pyrA, pyrB, 0, T, None, P, grad_planes=(I_f, W_f))
    H = st["H"]
    ok = st["n_valid"][0] + st["n_valid"][1] >= P.min_valid
    try:
        np.linalg.cholesky(H)
    except np.linalg.LinAlgError:
        ok = False
    Sigma = np.linalg.inv(H) if ok else np.zeros((6, 6))
    return dict(H=H, Sigma=Sigma, robust=st["robust"], n_valid=st["n_valid"], ok=ok, step=st)


# ----------------------------------------------------------------------------- covisibility
def covisible_counts(A: Level, B: Level, T, sigma_W: float):
    """|S_V| and |S_H| of "Dense frame covisibility ratio" with A's pixels transferred
    into B by eq. 3d_registration, T = A_T_B (reading R21): p_B is read at its
    nearest pixel, which must lie in the image and hold a valid W_B within
    3 sigma_W of the transferred w_B = 1 / Z_B."""
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    fx, fy, cx, cy = A.K
    h, w = A.W.shape
    hb, wb = B.W.shape
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    validA = A.W > 0
    q = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones((h, w))], axis=-1)
    X_B = (q / np.where(validA, A.W, 1.0)[..., None] - t) @ R
    Z_B = X_B[..., 2]
    front = Z_B > 0
    Zs = np.where(front, Z_B, 1.0)
    xn = np.floor(fx * X_B[..., 0] / Zs + cx + 0.5)
    yn = np.floor(fy * X_B[..., 1] / Zs + cy + 0.5)
    inside = front & (xn >= 0) & (xn <= wb - 1) & (yn >= 0) & (yn <= hb - 1)
    Wn = B.W[np.where(inside, yn, 0).astype(np.int64), np.where(inside, xn, 0).astype(np.int64)]
    visible = validA & inside & (Wn > 0) & (np.abs(Wn - 1.0 / Zs) < 3.0 * sigma_W)
    return int(visible.sum()), int(validA.sum())


def covisibility_ratio(I_A, W_A, I_B, W_B, K, T, sigma_W: float):
    """vr = min(vr_AB, vr_BA), vr_AB = |S_V| / |S_H| (reading R21, R19 for the planes).
    Returns dict(vr, vr_AB, vr_BA, counts=((S_V, S_H) A->B, (S_V, S_H) B->A))."""
    K = tuple(float(k) for k in K)
    A = Level(*measurement_planes(I_A, W_A), K)
    B = Level(*measurement_planes(I_B, W_B), K)
    ab = covisible_counts(A, B, T, sigma_W)
    ba = covisible_counts(B, A, se3_inv(T), sigma_W)
    vr_ab = ab[0] / ab[1] if ab[1] else 0.0
    vr_ba = ba[0] / ba[1] if ba[1] else 0.0
    return dict(vr=min(vr_ab, vr_ba), vr_AB=vr_ab, vr_BA=vr_ba, counts=(ab, ba))


# ----------------------------------------------------------------------------- tracking front-end
def track_sequence(I_frames, W_frames, K, levels: int = 4, iters=(5, 5, 5, 10), kf_every: int | None = 20,
                   fuse_intensity: bool = True, n_frames: int | None = None, reduced: bool = False,
                   kf_covisibility: float | None = None):
    """Frame-to-keyframe tracking with fusion ("Camera tracking", "Keyframe fusion").

    Frame 0 initialises the keyframe (C_kf = 1).  Frame k is aligned to the
    keyframe from the constant-velocity guess kf_T_k(0) = kf_T_{k-1} (kf_T_{k-2})^-1
    kf_T_{k-1}; every ``kf_every`` frames the aligned frame becomes the new
    keyframe (reading R15), otherwise it is fused into the keyframe with the
    final sigma_W of its alignment (reading R14).  With ``kf_covisibility`` the
    switch happens instead when the covisibility ratio between the keyframe and
    the aligned frame falls below that value (0.7 in the paper; reading R21), and
    the ratios are returned under "covisibility".  With ``reduced`` the pyramids
    are those of the reduced-precision form (bfloat16 I, binary16 W per level;
    the keyframe planes themselves stay float).  Returns dict(T_world [n,4,4]
    camera-to-world with frame 0 at the identity, results (per-frame align
    dicts), keyframe=(I, W, C) at the end)."""
    P = AlignParams(levels=levels, iters=tuple(iters))
    n = len(I_frames) if n_frames is None else n_frames
    I_kf, W_kf = measurement_planes(I_frames[0], W_frames[0])       # reading R19
    C_kf = np.ones_like(W_kf)
    pyramid = build_pyramid_reduced if reduced else build_pyramid
    kfp = pyramid(I_kf, W_kf, K, levels)
    T1 = np.eye(4)
    T2 = np.eye(4)
    T_wkf = np.eye(4)
    T_world = [np.eye(4)]
    results = []
    covis = []
    for k in range(1, n):
        cur = pyramid(I_frames[k], W_frames[k], K, levels)
        T_init = se3_project(T1 @ se3_inv(T2) @ T1)
        r = align(kfp, cur, T_init, P)
        results.append(r)
        Tk = r["T"]
        T_world.append(T_wkf @ Tk)
        if kf_covisibility is not None:
            c = covisibility_ratio(I_kf, W_kf, I_frames[k], W_frames[k], K, Tk, r["robust"]["sigma"][1])
            covis.append(c["vr"])
            switch = c["vr"] < kf_covisibility
        else:
            switch = k % kf_every == 0
        if switch:
            T2 = se3_inv(Tk) @ T1
            T1 = np.eye(4)
            T_wkf = T_wkf @ Tk
            I_kf, W_kf = measurement_planes(I_frames[k], W_frames[k])
            C_kf = np.ones_like(W_kf)
        else:
            I_kf, W_kf, C_kf, _ = fuse(I_kf, W_kf, C_kf, I_frames[k], W_frames[k], K, Tk, r["robust"]["sigma"][1],
                                       fuse_intensity)
            T2 = T1
            T1 = Tk
        kfp = pyramid(I_kf, W_kf, K, levels)
    return dict(T_world=np.stack(T_world), results=results, keyframe=(I_kf, W_kf, C_kf), covisibility=covis)
