"""The literal "warp at full resolution, then downsample" mode
(RGBID_WARP_FULL_RESOLUTION; "Iterative optimisation": the maps of B warped
towards A are downsampled to the level of the current iteration; reading R22)
through the C ABI, against the FP64 oracle with warp_mode "full".

A level-l pixel's value is the mean over its level-0 descendants, so a mask
decision that FP32 may take either way at one descendant (its warp coordinate
within 1e-4 px of an integer) can move the level-l value; such level-l pixels
are excluded from the per-pixel comparison and counted."""
import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import H_TOL, POSE_TOL, RES_TOL, gpu_pair, near_threshold, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402

ROB = dict(mu=[0.002, -0.001], sigma=[0.03, 0.004], nu=[4.0, 6.0])


def _near_at_level(A, B, level, T):
    """Level-l pixels with a level-0 descendant whose decision sits at a threshold."""
    wp0 = O.inverse_geometric_warp(A[0], B[0], T)
    near = near_threshold(wp0)
    for _ in range(level):
        h2, w2 = near.shape[0] // 2, near.shape[1] // 2
        near = (near[0:2 * h2:2, 0:2 * w2:2] | near[0:2 * h2:2, 1:2 * w2:2]
                | near[1:2 * h2:2, 0:2 * w2:2] | near[1:2 * h2:2, 1:2 * w2:2])
    # and the pixel's own level-l neighbours do not matter: the gradients are A's
    return near


def _step(pair, levels, level, T, robust):
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels)
    p = R.rgbid_default_params(levels=levels)
    p.warp_mode = R.WARP_FULL_RESOLUTION
    ws = R.new_workspace(PA.desc, p)
    L = PA.desc.lv[level]
    n = L.width * L.height
    rI = torch.empty(n, dtype=torch.float32, device="cuda")
    rW = torch.empty_like(rI)
    mI = torch.empty(n, dtype=torch.uint8, device="cuda")
    mW = torch.empty_like(mI)
    res = R.result_tensor()
    rob = None if robust is None else [robust["mu"][0], robust["sigma"][0], robust["nu"][0],
                                       robust["mu"][1], robust["sigma"][1], robust["nu"][1]]
    R.rgbid_eval_step(PA.desc, PB.desc, level, T, rob, p, ws, rI, rW, mI, mW, res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    shape = (L.height, L.width)
    g.update(r_I=rI.cpu().numpy().reshape(shape), r_W=rW.cpu().numpy().reshape(shape),
             mask_I=mI.cpu().numpy().reshape(shape).astype(bool), mask_W=mW.cpu().numpy().reshape(shape).astype(bool))
    return g


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("estimate", [False, True])
def test_full_resolution_step_matches_the_oracle(level, estimate):
    pair = synth.make_pair(3)
    A = O.build_pyramid(pair["I_A"], pair["W_A"], pair["K"], 3)
    B = O.build_pyramid(pair["I_B"], pair["W_B"], pair["K"], 3)
    T = O.se3_exp([0.004, -0.002, 0.003, 0.002, -0.003, 0.001]) @ pair["T_gt"]
    rob = None if estimate else ROB
    g = _step(pair, 3, level, T, rob)
    o = O.eval_step(A, B, level, T, rob, O.AlignParams(warp_mode="full"))
    near = _near_at_level(A, B, level, T)
    for m in ("mask_I", "mask_W"):
        bad = (g[m] != o[m]) & ~near
        assert not bad.any(), (m, np.argwhere(bad)[:5].tolist())
    both_I = g["mask_I"] & o["mask_I"] & ~near
    both_W = g["mask_W"] & o["mask_W"] & ~near
    assert both_I.sum() > 0.5 * o["mask_I"].sum() and both_W.sum() > 0.3 * o["mask_W"].sum()
    eI = np.abs(g["r_I"] - o["r_I"])[both_I]
    assert (eI <= RES_TOL * np.maximum(np.abs(o["r_I"][both_I]), 1.0)).all(), eI.max()
    rangeW = float(A[level].W.max())
    eW = np.abs(g["r_W"] - o["r_W"])[both_W]
    assert (eW <= RES_TOL * np.maximum(np.abs(o["r_W"][both_W]), rangeW)).all(), eW.max()
    Ho = o["H"]
    d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
    assert (np.abs(g["H"] - Ho) <= H_TOL * d).all(), np.max(np.abs(g["H"] - Ho) / d)
    if estimate:
        for c in range(2):
            assert abs(g["sigma"][c] - o["robust"]["sigma"][c]) <= 1e-5 * o["robust"]["sigma"][c]


@pytest.mark.parametrize("shape", [(160, 120, 3, (5, 5, 10), None), (640, 480, 4, (5, 5, 5, 10), (525.0, 525.0, 319.5, 239.5))])
def test_full_resolution_alignment_matches_the_oracle(shape):
    w, h, levels, iters, K = shape
    pair = synth.make_pair(4, w, h, K=K)
    A = O.build_pyramid(pair["I_A"], pair["W_A"], pair["K"], levels)
    B = O.build_pyramid(pair["I_B"], pair["W_B"], pair["K"], levels)
    o = O.align(A, B, None, O.AlignParams(levels=levels, iters=iters, warp_mode="full"))
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels)
    p = R.rgbid_default_params(levels=levels, iters=iters)
    p.warp_mode = R.WARP_FULL_RESOLUTION
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, ws, res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    assert g["status"] == o["status"] and g["iters_done"] == o["iters_done"]
    # and it differs from the per-level warp, which is a different method
    p.warp_mode = R.WARP_PER_LEVEL
    res2 = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, R.new_workspace(PA.desc, p), res2)
    torch.cuda.synchronize()
    assert pose_error(R.parse_result(res2)["T"], g["T"])[0] > 1e-7


def test_batched_form_rejects_the_full_resolution_warp():
    p = R.rgbid_default_params()
    p.warp_mode = R.WARP_FULL_RESOLUTION
    ws = torch.zeros(R.rgbid_align_batched_workspace_bytes(), dtype=torch.uint8, device="cuda")
    items = torch.zeros(64, dtype=torch.uint8, device="cuda")
    code = R.lib().rgbid_align_batched(R._ptr(items), 0, R.PLANES_F32, __import__("ctypes").byref(p), None,
                                       R._ptr(ws), ws.numel(), None)
    assert code == R.ERR_UNSUPPORTED
