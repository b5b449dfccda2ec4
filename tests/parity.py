"""Helpers shared by the GPU parity tests: run one step or one alignment on
both the CUDA path (through the C ABI) and the FP64 oracle, and compare them
with the tolerances of the method:

* per-pixel residuals: |dr| <= 1e-5 max(|r|, range) with range 1 for I and
  max W_A for W;
* normal equations: |dH_ij| <= 1e-4 sqrt(H_ii H_jj) and, by Cauchy-Schwarz
  (|g_i| <= sqrt(H_ii cost)), |dg_i| <= 1e-4 sqrt(H_ii cost);
* masks: bit-exact except where the FP64 decision quantity lies within FP32
  rounding of its threshold (a warp coordinate within 1e-4 px of an integer,
  i.e. of a floor/bounds decision); such pixels are reported and counted;
* poses: <= 1e-5 rad and <= 1e-5 m.
"""
from __future__ import annotations

import numpy as np

import oracle as O

RES_TOL = 1e-5
H_TOL = 1e-4
POSE_TOL = 1e-5
NEAR_PX = 1e-4


def gpu_pair(pair, levels, precision=0):
    import torch
    from paper_1807_08271_gb300 import rgbid as R
    dev = "cuda"
    h, w = pair["I_A"].shape
    out = []
    for a, b in (("I_A", "W_A"), ("I_B", "W_B")):
        I = torch.from_numpy(pair[a]).to(dev)
        W = torch.from_numpy(pair[b]).to(dev)
        P = R.DevicePyramid(w, h, levels, precision).build(I, W, pair["K"])
        out.append((P, I, W))
    return out


def oracle_pair(pair, levels):
    A = O.build_pyramid(pair["I_A"], pair["W_A"], pair["K"], levels)
    B = O.build_pyramid(pair["I_B"], pair["W_B"], pair["K"], levels)
    return A, B


def near_threshold(wp) -> np.ndarray:
    """Pixels whose oracle warp coordinate is within NEAR_PX of an integer, or
    whose depth tests sit at zero: FP32 may decide them either way."""
    du = np.abs(wp["u_B"] - np.round(wp["u_B"]))
    dv = np.abs(wp["v_B"] - np.round(wp["v_B"]))
    return (np.minimum(du, dv) < NEAR_PX) | (np.abs(wp["Z_B"]) < 1e-6) | (np.abs(wp["Zp"]) < 1e-6)


def compare_masks(name, m_gpu, m_ora, near):
    bad = (m_gpu != m_ora)
    unexplained = bad & ~near
    assert not unexplained.any(), (f"{name}: {int(unexplained.sum())} mask mismatches away from any threshold "
                                   f"at {np.argwhere(unexplained)[:5].tolist()}")
    return int(bad.sum())


def eval_step_both(pair, level, T, robust=None, levels=3, precision=0, params=None, oracle_planes=None):
    import torch
    from paper_1807_08271_gb300 import rgbid as R
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels, precision)
    p = params or R.rgbid_default_params(levels=levels)
    ws = R.new_workspace(PA.desc, p)
    L = PA.desc.lv[level]
    n = L.width * L.height
    rI = torch.empty(n, dtype=torch.float32, device="cuda")
    rW = torch.empty_like(rI)
    mI = torch.empty(n, dtype=torch.uint8, device="cuda")
    mW = torch.empty_like(mI)
    res = R.result_tensor()
    rob_flat = None
    if robust is not None:
        rob_flat = [robust["mu"][0], robust["sigma"][0], robust["nu"][0],
                    robust["mu"][1], robust["sigma"][1], robust["nu"][1]]
    R.rgbid_eval_step(PA.desc, PB.desc, level, T, rob_flat, p, ws, rI, rW, mI, mW, res)
    torch.cuda.synchronize()
    g = R.parse_result(res)
    shape = (L.height, L.width)
    g.update(r_I=rI.cpu().numpy().reshape(shape), r_W=rW.cpu().numpy().reshape(shape),
             mask_I=mI.cpu().numpy().reshape(shape).astype(bool), mask_W=mW.cpu().numpy().reshape(shape).astype(bool))
    if oracle_planes is None:
        A, B = oracle_pair(pair, levels)
    else:
        A, B = oracle_planes
    P = O.AlignParams(levels=levels, iters=tuple(p.iters[:levels]))
    o = O.eval_step(A, B, level, T, robust, P)
    return g, o, A


def check_step(g, o, A, level, check_normal_equations=True):
    near = near_threshold(o["warp"])
    nI = compare_masks("mask_I", g["mask_I"], o["mask_I"], near)
    nW = compare_masks("mask_W", g["mask_W"], o["mask_W"], near)
    both_I = g["mask_I"] & o["mask_I"]
    both_W = g["mask_W"] & o["mask_W"]
    eI = np.abs(g["r_I"] - o["r_I"])[both_I]
    tolI = RES_TOL * np.maximum(np.abs(o["r_I"][both_I]), 1.0)
    assert (eI <= tolI).all(), f"r_I max err {eI.max():.3e}"
    rangeW = float(A[level].W.max())
    eW = np.abs(g["r_W"] - o["r_W"])[both_W]
    tolW = RES_TOL * np.maximum(np.abs(o["r_W"][both_W]), rangeW)
    assert (eW <= tolW).all(), f"r_W max err {eW.max():.3e}"
    assert g["n_valid"] == o["n_valid"] or (nI + nW) > 0
    if check_normal_equations:
        Hg, Ho = g["H"], o["H"]
        d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
        relH = np.abs(Hg - Ho) / d
        assert relH.max() <= H_TOL, f"H normalised err {relH.max():.3e}"
        gt = np.sqrt(np.diag(Ho) * o["cost"])
        relg = np.abs(g["g"] - o["g"]) / gt
        assert relg.max() <= H_TOL, f"g normalised err {relg.max():.3e}"
        assert abs(g["cost"] - o["cost"]) <= H_TOL * o["cost"]
    return dict(mask_mismatch=nI + nW, max_rI=float(eI.max(initial=0)), max_rW=float(eW.max(initial=0)))


def pose_error(T1, T2):
    E = O.se3_inv(np.asarray(T1)) @ np.asarray(T2)
    return float(np.linalg.norm(O.so3_log(E[:3, :3]))), float(np.linalg.norm(E[:3, 3]))
