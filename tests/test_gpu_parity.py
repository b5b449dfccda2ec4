"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import (POSE_TOL, check_step, eval_step_both, gpu_pair, oracle_pair, pose_error)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402


@pytest.fixture(scope="module")
def pair0():
    return synth.make_pair(0)


@pytest.fixture(scope="module")
def pair640():
    return synth.make_pair(7, 640, 480, K=(525.0, 525.0, 319.5, 239.5))


# ----------------------------------------------------------------------------- pyramid
@pytest.mark.parametrize("shape", [(160, 120, 3), (640, 480, 4), (97, 75, 3)])
def test_pyramid_matches_oracle(shape):
    w, h, levels = shape
    rng = np.random.default_rng(w)
    I = rng.random((h, w)).astype(np.float32)
    W = rng.uniform(0.2, 2.0, (h, w)).astype(np.float32)
    W[rng.random((h, w)) < 0.2] = 0.0
    W[0, :3] = np.nan
    K = synth.pinhole(w, h)
    P = R.DevicePyramid(w, h, levels).build(torch.from_numpy(I).cuda(), torch.from_numpy(W).cuda(), K)
    Op = O.build_pyramid(I, W, K, levels)
    for l in range(levels):
        Ig, Wg = P.level_planes(l)
        assert Ig.shape == Op[l].I.shape
        assert np.array_equal(Wg > 0, Op[l].W > 0)                 # validity is exact
        assert np.allclose(Ig, Op[l].I, rtol=1e-6, atol=1e-7)
        assert np.allclose(Wg[Wg > 0], Op[l].W[Wg > 0], rtol=1e-6, atol=0)
        Lk = P.desc.lv[l].K
        assert (Lk.fx, Lk.fy, Lk.cx, Lk.cy) == O.level_intrinsics(K, l)


# ----------------------------------------------------------------------------- one step
FIXED = dict(mu=[0.001, -0.0002], sigma=[0.04, 0.004], nu=[5.0, 3.0])


@pytest.mark.parametrize("level", [0, 1, 2])
def test_eval_step_fixed_robust_c0(pair0, level):
    T = O.se3_exp([0.004, -0.003, 0.002, 0.003, -0.002, 0.004]) @ pair0["T_gt"]
    g, o, A = eval_step_both(pair0, level, T, FIXED)
    info = check_step(g, o, A, level)
    assert info["mask_mismatch"] <= 3


def _nu_tolerance(r, mu, sigma, nu):
    """How far the degrees of freedom may move when computed in FP32 (the kernel's
    precision) from a sample whose (mu, sigma) agree with the oracle's to 1e-5 sigma:
    nu is a root of f(nu) = n c(nu) + sum (ln w - w), so it moves by the change of the
    oracle's own root under mu -> mu + 1e-5 sigma and sigma -> (1 + 1e-5) sigma, plus
    an FP32 evaluation error of the sums, 64 eps_32 (sum |ln w| + sum w), over |f'(nu)|,
    plus the resolution of the 20 bisection halvings of [2, 10]."""
    lo, hi = 2.0, 10.0
    if nu <= lo or nu >= hi:
        return 1e-6
    dmu = abs(O.estimate_nu(r, mu + 1e-5 * sigma, sigma) - nu)
    dsig = abs(O.estimate_nu(r, mu, sigma * (1 + 1e-5)) - nu)
    x = (r - mu) / sigma
    w = O.omega(x, nu)
    h = 1e-4
    fprime = abs(O.nu_equation(nu + h, x) - O.nu_equation(nu - h, x)) / (2 * h)
    scale = np.sum(np.abs(np.log(w))) + np.sum(w)
    return dmu + dsig + 64 * 2.0 ** -24 * scale / fprime + 8.0 / 2 ** 20


@pytest.mark.parametrize("level", [0, 1, 2])
def test_eval_step_estimated_robust_c0(pair0, level):
    T = O.se3_exp([0.004, -0.003, 0.002, 0.003, -0.002, 0.004]) @ pair0["T_gt"]
    g, o, A = eval_step_both(pair0, level, T, None)
    rob = o["robust"]
    P = O.AlignParams()
    s = O.sample_stride(A[level].W.shape[1], A[level].W.shape[0])
    v, u = np.mgrid[0:A[level].W.shape[0], 0:A[level].W.shape[1]]
    sm = (u % s == 0) & (v % s == 0)
    own, tols = [], []
    for c, (r, m) in enumerate(((o["r_I"], o["mask_I"]), (o["r_W"], o["mask_W"]))):
        assert abs(g["mu"][c] - rob["mu"][c]) <= 1e-5 * rob["sigma"][c] + 1e-9
        assert abs(g["sigma"][c] - rob["sigma"][c]) <= 1e-5 * rob["sigma"][c]
        # each channel's own root (before nu_I <- max(nu_I, nu_W)) and its tolerance
        own.append(O.estimate_nu(r[sm & m], rob["mu"][c], rob["sigma"][c], P.nu_lo, P.nu_hi, P.bisect_steps))
        tols.append(_nu_tolerance(r[sm & m], rob["mu"][c], rob["sigma"][c], own[c]))
    for c in range(2):
        tol = tols[1] if (c == 0 and own[1] > own[0]) else tols[c]
        print(f"level {level} channel {c}: nu {rob['nu'][c]:.6f} gpu {g['nu'][c]:.6f} "
              f"|d| {abs(g['nu'][c] - rob['nu'][c]):.2e} tol {tol:.2e}")
        assert abs(g["nu"][c] - rob["nu"][c]) <= tol, (c, g["nu"][c], rob["nu"][c], tol)
        assert tol < 2e-3
    check_step(g, o, A, level)


def test_eval_step_at_identity_identical_frames_is_zero(pair0):
    p = dict(pair0)
    p["I_B"], p["W_B"] = p["I_A"], p["W_A"]
    g, o, A = eval_step_both(p, 0, np.eye(4), FIXED)
    assert np.abs(g["r_I"]).max() == 0.0 and np.abs(g["r_W"]).max() <= 1e-7
    # At T = I the CUDA path's pixel offset is exactly 0, so the bilinear taps are
    # (u..u+1, v..v+1) (the oracle's FP64 u_B may round just below u: every pixel
    # is at a floor decision and check_step accepts either side).
    W = p["W_A"]
    h, w = W.shape
    inner = np.zeros((h, w), bool)
    inner[1:-1, 1:-1] = True
    mI = inner & (W > 0)
    pos = W > 0
    taps = np.zeros((h, w), bool)
    taps[:-1, :-1] = pos[:-1, :-1] & pos[:-1, 1:] & pos[1:, :-1] & pos[1:, 1:]
    nb = np.zeros((h, w), bool)
    nb[1:-1, 1:-1] = pos[1:-1, :-2] & pos[1:-1, 2:] & pos[:-2, 1:-1] & pos[2:, 1:-1]
    assert np.array_equal(g["mask_I"], mI)
    assert np.array_equal(g["mask_W"], mI & taps & nb)
    # every pixel sits on a floor decision here, so H is compared in the other tests
    check_step(g, o, A, 0, check_normal_equations=False)


def test_eval_step_full_size_640(pair640):
    T = O.se3_exp([0.01, 0.004, -0.006, 0.004, 0.003, -0.002]) @ pair640["T_gt"]
    g, o, A = eval_step_both(pair640, 0, T, None, levels=4)
    check_step(g, o, A, 0)


# ----------------------------------------------------------------------------- alignment
def _align_gpu(pair, levels, iters, T_init=None, precision=0):
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels, precision)
    p = R.rgbid_default_params(levels=levels, iters=iters)
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T_init, p, ws, res)
    torch.cuda.synchronize()
    return R.parse_result(res)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 5, 8])
def test_align_c0_matches_oracle(seed):
    pair = synth.make_pair(seed)
    g = _align_gpu(pair, 3, (5, 5, 10))
    A, B = oracle_pair(pair, 3)
    o = O.align(A, B, None, O.AlignParams())
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    assert g["iters_done"] == 20 and g["status"] == o["status"]
    gr, gt = pose_error(g["T"], pair["T_gt"])
    assert gr < 2e-3 and gt < 2e-3


def test_align_640_matches_oracle(pair640):
    g = _align_gpu(pair640, 4, (5, 5, 5, 10))
    A, B = oracle_pair(pair640, 4)
    o = O.align(A, B, None, O.AlignParams(levels=4, iters=(5, 5, 5, 10)))
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)


def test_align_initial_guess_on_device(pair0):
    T0 = O.se3_exp([0.01, 0, 0, 0, 0.01, 0])
    g1 = _align_gpu(pair0, 3, (5, 5, 10), T_init=T0)
    g2 = _align_gpu(pair0, 3, (5, 5, 10), T_init=torch.from_numpy(T0.reshape(16).copy()).cuda())
    assert np.array_equal(g1["T"], g2["T"])
    A, B = oracle_pair(pair0, 3)
    o = O.align(A, B, T0, O.AlignParams())
    er, et = pose_error(g1["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL


def test_align_degenerate_reference_keeps_pose(pair0):
    p = dict(pair0)
    p["W_A"] = np.zeros_like(p["W_A"])
    T0 = O.se3_exp([0.01, 0, 0, 0, 0, 0])
    g = _align_gpu(p, 3, (5, 5, 10), T_init=T0)
    assert np.array_equal(g["T"], T0)
    assert g["status"] == R.ERR_DEGENERATE and g["iters_skipped"] == 20 and g["n_valid"] == [0, 0]


def test_align_is_deterministic(pair0):
    a = _align_gpu(pair0, 3, (5, 5, 10))
    b = _align_gpu(pair0, 3, (5, 5, 10))
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["H"], b["H"])


# ----------------------------------------------------------------------------- fusion
def _fuse_both(pair, T, sigma_W, fuse_intensity=True, T_host=None, sigma_host=None):
    dev = "cuda"
    I_kf = torch.from_numpy(pair["I_A"]).to(dev).clone()
    W_kf = torch.from_numpy(pair["W_A"]).to(dev).clone()
    C_kf = torch.ones_like(W_kf)
    I_k = torch.from_numpy(pair["I_B"]).to(dev)
    W_k = torch.from_numpy(pair["W_B"]).to(dev)
    R.rgbid_fuse_keyframe(I_kf, W_kf, C_kf, I_k, W_k, pair["K"], T, sigma_W, fuse_intensity)
    torch.cuda.synchronize()
    o = O.fuse(pair["I_A"], pair["W_A"], np.ones_like(pair["W_A"], dtype=np.float64), pair["I_B"], pair["W_B"],
               pair["K"], T if T_host is None else T_host, sigma_W if sigma_host is None else sigma_host,
               fuse_intensity)
    return (I_kf.cpu().numpy(), W_kf.cpu().numpy(), C_kf.cpu().numpy()), o


@pytest.mark.parametrize("seed", [0, 3])
def test_fuse_matches_oracle(seed):
    pair = synth.make_pair(seed)
    T = pair["T_gt"]
    (Ig, Wg, Cg), (Io, Wo, Co, gate) = _fuse_both(pair, T, 2e-3)
    A = O.Level(pair["I_A"].astype(np.float64), pair["W_A"].astype(np.float64), pair["K"])
    wp = O.inverse_geometric_warp(A, O.Level(pair["I_B"].astype(np.float64), pair["W_B"].astype(np.float64),
                                             pair["K"]), T)
    fused_g = Cg != 1.0
    mism = fused_g != gate
    if mism.any():
        # only where the gate quantity sits at its threshold or the warp at a floor decision
        w_B = 1.0 / np.where(wp["front"], wp["Z_B"], 1.0)
        margin = np.abs(np.abs(wp["W_Bp"] - w_B) - 3 * 2e-3)
        du = np.abs(wp["u_B"] - np.round(wp["u_B"]))
        dv = np.abs(wp["v_B"] - np.round(wp["v_B"]))
        ok = (margin < 1e-6) | (np.minimum(du, dv) < 1e-4)
        assert ok[mism].all()
    both = fused_g & gate
    assert both.sum() > 5000
    assert np.allclose(Wg[both], Wo[both], rtol=1e-5, atol=0)
    assert np.allclose(Ig[both], Io[both], rtol=0, atol=1e-5)
    assert np.allclose(Cg[both], Co[both], rtol=1e-5)
    untouched = ~fused_g & ~gate
    assert np.array_equal(Wg[untouched], pair["W_A"][untouched])


def test_fuse_params_from_device_match_host(pair0):
    T = pair0["T_gt"]
    (Ig, Wg, Cg), _ = _fuse_both(pair0, T, 2e-3)
    Td = torch.from_numpy(T.reshape(16).copy()).cuda()
    sd = torch.tensor([2e-3], dtype=torch.float64, device="cuda")
    (Ig2, Wg2, Cg2), _ = _fuse_both(pair0, Td, sd, T_host=T, sigma_host=2e-3)
    assert np.array_equal(Wg, Wg2) and np.array_equal(Ig, Ig2) and np.array_equal(Cg, Cg2)


def test_pose_helpers_on_device():
    rng = np.random.default_rng(3)
    T1 = synth.random_relative_pose(rng, 10, 0.2)
    T2 = synth.random_relative_pose(rng, 10, 0.2)
    a = torch.from_numpy(T1.reshape(16).copy()).cuda()
    b = torch.from_numpy(T2.reshape(16).copy()).cuda()
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    R.rgbid_predict_pose(a, b, out)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy().reshape(4, 4), T1 @ O.se3_inv(T2) @ T1, atol=1e-14)
    R.rgbid_compose_pose(a, True, b, out)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy().reshape(4, 4), O.se3_inv(T1) @ T2, atol=1e-14)


# ----------------------------------------------------------------------------- sequence
def test_tracking_sequence_prefix_matches_oracle():
    """Device-resident tracking front-end (constant-velocity guess, alignment,
    fusion, keyframe switch at frame 20) against the oracle's, frame by frame."""
    from paper_1807_08271_gb300.tracker import Tracker
    n = 23
    seq = synth.render_sequence(0, n_frames=n)
    I_all = torch.from_numpy(seq["I"]).cuda()
    W_all = torch.from_numpy(seq["W"]).cuda()
    trk = Tracker(640, 480, seq["K"], levels=4, iters=(5, 5, 5, 10), kf_every=20, max_frames=n)
    for k in range(n):
        trk.step(I_all[k], W_all[k])
    torch.cuda.synchronize()
    gT = trk.trajectory()
    o = O.track_sequence(seq["I"], seq["W"], seq["K"], levels=4, iters=(5, 5, 5, 10), kf_every=20)
    for k in range(1, n):
        er, et = pose_error(gT[k], o["T_world"][k])
        assert er <= POSE_TOL and et <= POSE_TOL, (k, er, et)
    truth = [np.linalg.inv(seq["T_wc"][0]) @ seq["T_wc"][k] for k in range(n)]
    assert max(pose_error(gT[k], truth[k])[0] for k in range(n)) < 2e-3
    # the fused keyframe (frame 20 onwards) matches too
    Ig, Wg, Cg = trk.I_kf.cpu().numpy(), trk.W_kf.cpu().numpy(), trk.C_kf.cpu().numpy()
    Io, Wo, Co = o["keyframe"]
    both = (Cg > 1) & (Co > 1)
    assert both.sum() > 0.5 * (Wo > 0).sum()
    assert np.allclose(Wg[both], Wo[both], rtol=1e-4)
    assert np.allclose(Ig[both], Io[both], atol=1e-4)


def test_tracking_graph_replay_equals_eager_enqueue():
    """The CUDA-graph form of the tracker's frame step (one replay per frame) gives
    the same bits as enqueueing every launch, across two keyframe switches."""
    from paper_1807_08271_gb300.tracker import Tracker
    n = 45
    seq = synth.render_sequence(1, n_frames=n)
    I_all = torch.from_numpy(seq["I"]).cuda()
    W_all = torch.from_numpy(seq["W"]).cuda()
    out = []
    for graphs in (False, True):
        trk = Tracker(640, 480, seq["K"], levels=4, iters=(5, 5, 5, 10), kf_every=20, max_frames=n, graphs=graphs)
        s = torch.cuda.Stream()
        for k in range(n):
            trk.step(I_all[k], W_all[k], s)
        torch.cuda.synchronize()
        out.append((trk.results.cpu().numpy(), trk.I_kf.cpu().numpy(), trk.W_kf.cpu().numpy(),
                    trk.C_kf.cpu().numpy(), trk.is_kf.copy()))
        if graphs:
            assert set(trk._graph) == {(False, 0), (True, 0)}
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_tracking_full_sequence_stays_on_ground_truth():
    """300 frames of the benchmark sequence: every frame's pose stays close to the
    ground truth (no drift from the constant-velocity composition)."""
    from paper_1807_08271_gb300.tracker import Tracker
    seq = synth.render_sequence(0, n_frames=300)
    I_all = torch.from_numpy(seq["I"]).cuda()
    W_all = torch.from_numpy(seq["W"]).cuda()
    trk = Tracker(640, 480, seq["K"], levels=4, iters=(5, 5, 5, 10), kf_every=20, max_frames=300)
    for k in range(300):
        trk.step(I_all[k], W_all[k])
    torch.cuda.synchronize()
    gT = trk.trajectory()
    errs = [pose_error(gT[k], np.linalg.inv(seq["T_wc"][0]) @ seq["T_wc"][k]) for k in range(1, 300)]
    assert max(e[0] for e in errs) < 5e-3 and max(e[1] for e in errs) < 2e-2
    assert all(r["status"] == R.OK for r in trk.frame_results())
