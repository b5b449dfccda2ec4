"""Failure detection without a GPU fault.

Non-finite input (NaN, +-inf in I or W) is injected on the host and must give
the oracle's answer (a non-finite pixel is a hole); a device wait with nothing
to wait for must run out of its clock64 budget, report, and leave the context
usable.  Nothing here faults, traps or hangs the GPU: every wait in the probe is
bounded, and no CTA writes to another's shared memory."""
import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import POSE_TOL, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402
from paper_1807_08271_gb300.batch import BatchAligner  # noqa: E402


def _inject(seed, pair, frac=0.01):
    """Copies of a pair's planes with about ``frac`` of the pixels of each kind made non-finite."""
    rng = np.random.default_rng(seed)
    out = {k: pair[k].copy() for k in ("I_A", "W_A", "I_B", "W_B")}
    for key, val in (("I_B", np.nan), ("W_B", np.inf), ("I_B", -np.inf), ("W_B", np.nan), ("W_A", np.nan),
                     ("I_A", np.inf), ("W_A", -np.inf)):
        m = rng.random(out[key].shape) < frac
        out[key][m] = val
    return out


def _pyr(I, W, K, levels, precision=R.PLANES_F32):
    h, w = I.shape
    return R.DevicePyramid(w, h, levels, precision).build(torch.from_numpy(I).cuda(), torch.from_numpy(W).cuda(), K)


@pytest.mark.parametrize("precision", [R.PLANES_F32, R.PLANES_BF16_F16])
def test_pyramid_of_nonfinite_input_matches_oracle(precision):
    rng = np.random.default_rng(11)
    h, w = 120, 160
    I = rng.random((h, w)).astype(np.float32)
    W = rng.uniform(0.2, 2.0, (h, w)).astype(np.float32)
    bad = rng.random((h, w))
    I[bad < 0.03] = np.nan
    I[(bad >= 0.03) & (bad < 0.05)] = np.inf
    W[(bad >= 0.05) & (bad < 0.08)] = np.nan
    W[(bad >= 0.08) & (bad < 0.10)] = np.inf
    W[(bad >= 0.10) & (bad < 0.11)] = -np.inf
    K = synth.pinhole(w, h)
    P = _pyr(I, W, K, 3, precision)
    Op = (O.build_pyramid_reduced if precision else O.build_pyramid)(I, W, K, 3)
    for l in range(3):
        Ig, Wg = P.level_planes(l)
        assert np.all(np.isfinite(Ig)) and np.all(np.isfinite(Wg))
        assert np.array_equal(Wg > 0, Op[l].W > 0)
        if precision == R.PLANES_F32:
            assert np.allclose(Ig, Op[l].I, rtol=1e-6, atol=1e-7)
            assert np.allclose(Wg[Wg > 0], Op[l].W[Wg > 0], rtol=1e-6, atol=0)
        else:
            # FP32 box means vs FP64 box means may round to neighbouring codes at ties
            dI, dW = Ig != Op[l].I, Wg != Op[l].W
            assert dI.mean() < 1e-3 and dW.mean() < 1e-3
            assert np.all(np.abs(Ig - Op[l].I)[dI] <= 2.0 ** -7 * np.abs(Op[l].I[dI]) + 1e-12)
            assert np.all(np.abs(Wg - Op[l].W)[dW] <= 2.0 ** -10 * np.abs(Op[l].W[dW]) + 1e-12)


def test_alignment_of_nonfinite_input_matches_oracle():
    pair = synth.make_pair(0)
    q = _inject(3, pair)
    PA, PB = _pyr(q["I_A"], q["W_A"], pair["K"], 3), _pyr(q["I_B"], q["W_B"], pair["K"], 3)
    p = R.rgbid_default_params()
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, ws, res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    o = O.align(O.build_pyramid(q["I_A"], q["W_A"], pair["K"], 3), O.build_pyramid(q["I_B"], q["W_B"], pair["K"], 3),
                None, O.AlignParams())
    assert g["status"] == o["status"] == R.OK and g["iters_done"] == o["iters_done"]
    assert np.all(np.isfinite(g["T"])) and np.all(np.isfinite(g["H"]))
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    # the batched form reads the same pyramids and gives the same pose
    B = BatchAligner([dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=3, iters=[5, 5, 10])])
    B.run()
    torch.cuda.synchronize()
    b = B.all_results()[0]
    assert b["status"] == R.OK
    er, et = pose_error(b["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)


def test_all_nonfinite_reference_is_degenerate_and_keeps_the_pose():
    pair = synth.make_pair(1)
    IA = np.full_like(pair["I_A"], np.nan)
    PA, PB = _pyr(IA, pair["W_A"], pair["K"], 3), _pyr(pair["I_B"], pair["W_B"], pair["K"], 3)
    T0 = O.se3_exp([0.01, 0, 0, 0, 0, 0])
    p = R.rgbid_default_params()
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T0, p, R.new_workspace(PA.desc, p), res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    assert g["status"] == R.ERR_DEGENERATE and g["iters_skipped"] == 20 and g["n_valid"] == [0, 0]
    assert np.array_equal(g["T"], T0)


def test_keyframe_init_and_fusion_of_nonfinite_frames_match_oracle():
    pair = synth.make_pair(3)
    q = _inject(5, pair, frac=0.02)
    dev = "cuda"
    I_kf, W_kf, C_kf = (torch.empty_like(torch.from_numpy(pair["I_A"])).to(dev) for _ in range(3))
    R.rgbid_init_keyframe(I_kf, W_kf, C_kf, torch.from_numpy(q["I_A"]).to(dev), torch.from_numpy(q["W_A"]).to(dev))
    torch.cuda.synchronize()
    Iw, Ww = O.measurement_planes(q["I_A"], q["W_A"])
    assert np.array_equal(I_kf.cpu().numpy(), Iw.astype(np.float32))
    assert np.array_equal(W_kf.cpu().numpy(), Ww.astype(np.float32))
    assert np.all(C_kf.cpu().numpy() == 1.0)
    T = pair["T_gt"]
    R.rgbid_fuse_keyframe(I_kf, W_kf, C_kf, torch.from_numpy(q["I_B"]).to(dev), torch.from_numpy(q["W_B"]).to(dev),
                          pair["K"], T, 2e-3, True)
    torch.cuda.synchronize()
    Ig, Wg, Cg = I_kf.cpu().numpy(), W_kf.cpu().numpy(), C_kf.cpu().numpy()
    Io, Wo, Co, gate = O.fuse(Iw, Ww, np.ones_like(Ww), q["I_B"], q["W_B"], pair["K"], T, 2e-3, True)
    assert np.all(np.isfinite(Ig)) and np.all(np.isfinite(Wg)) and np.all(np.isfinite(Cg))
    fused = Cg != 1.0
    mism = fused != gate
    if mism.any():
        # only where the gate quantity sits at its threshold or the warp at a floor decision
        wp = O.inverse_geometric_warp(O.Level(Iw, Ww, pair["K"]),
                                      O.Level(*O.measurement_planes(q["I_B"], q["W_B"]), pair["K"]), T)
        w_B = 1.0 / np.where(wp["front"], wp["Z_B"], 1.0)
        margin = np.abs(np.abs(wp["W_Bp"] - w_B) - 3 * 2e-3)
        du = np.abs(wp["u_B"] - np.round(wp["u_B"]))
        dv = np.abs(wp["v_B"] - np.round(wp["v_B"]))
        ok = (margin < 1e-6) | (np.minimum(du, dv) < 1e-4)
        assert ok[mism].all()
    both = fused & gate
    assert both.sum() > 3000
    assert np.allclose(Wg[both], Wo[both], rtol=1e-5, atol=0)
    assert np.allclose(Ig[both], Io[both], rtol=0, atol=1e-5)
    assert np.allclose(Cg[both], Co[both], rtol=1e-5)


def test_a_wait_with_nothing_to_wait_for_runs_out_and_reports():
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    R.rgbid_probe_wait_timeout(200_000, counter)            # ~0.1 ms at 2 GHz
    torch.cuda.synchronize()
    assert int(counter.item()) == 4                          # one expired wait per CTA of the cluster
    R.rgbid_probe_wait_timeout(0, counter)
    torch.cuda.synchronize()
    assert int(counter.item()) == 8
    # the context is still usable: a normal alignment runs and converges
    pair = synth.make_pair(2)
    PA, PB = _pyr(pair["I_A"], pair["W_A"], pair["K"], 3), _pyr(pair["I_B"], pair["W_B"], pair["K"], 3)
    p = R.rgbid_default_params()
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, R.new_workspace(PA.desc, p), res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    assert g["status"] == R.OK and g["iters_done"] == 20


def test_a_mailbox_wait_with_nothing_to_wait_for_gives_up_and_raises_the_flag():
    # the split level kernel's roles wait on workspace counters; a wait that runs out
    # raises the error flag and every later wait of the launch gives up at once
    import time
    scratch = torch.zeros(256, dtype=torch.int32, device="cuda")
    out = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    R.rgbid_probe_mailbox_timeout(200_000, scratch, out)     # ~0.1 ms at 2 GHz
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # (timeouts, first wait, second wait, error flag): the second wait did not spend its ~2 s budget
    assert tuple(int(v) for v in out.cpu()) == (1, 0, 0, 1)
    assert dt < 1.0
    assert int(scratch.abs().sum()) == 0                     # the mailbox is left clear
    out.fill_(-1)
    R.rgbid_probe_mailbox_timeout(0, scratch, out)
    torch.cuda.synchronize()
    assert tuple(int(v) for v in out.cpu()) == (1, 0, 0, 1)
    # the context is still usable: a 640x480 alignment, whose two finest levels run in
    # the split kernel, completes every iteration
    pair = synth.make_pair(3, width=640, height=480)
    PA, PB = _pyr(pair["I_A"], pair["W_A"], pair["K"], 4), _pyr(pair["I_B"], pair["W_B"], pair["K"], 4)
    p = R.rgbid_default_params(levels=4, iters=[5, 5, 5, 10])
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, R.new_workspace(PA.desc, p), res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    assert g["status"] == R.OK and g["iters_done"] == 25
