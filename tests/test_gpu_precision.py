"""Reduced-precision form (bfloat16 I, binary16 W planes; FP32 residuals with
compensated partial sums; FP64 6x6 solve and update) against the FP64 oracle
on the same rounded planes, plus its storage error against the full-precision
oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import POSE_TOL, check_step, eval_step_both, gpu_pair, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402

BF = R.PLANES_BF16_F16


@pytest.mark.parametrize("shape", [(160, 120, 3), (640, 480, 4)])
def test_reduced_pyramid_matches_oracle(shape):
    w, h, levels = shape
    p = synth.make_pair(3, w, h)
    P = R.DevicePyramid(w, h, levels, BF).build(torch.from_numpy(p["I_A"]).cuda(), torch.from_numpy(p["W_A"]).cuda(),
                                                p["K"])
    Op = O.build_pyramid_reduced(p["I_A"], p["W_A"], p["K"], levels)
    for l in range(levels):
        Ig, Wg = P.level_planes(l)
        assert np.array_equal(Wg > 0, Op[l].W > 0)
        if l == 0:
            # the same float32 inputs rounded once: bit-exact
            assert np.array_equal(Ig, Op[l].I) and np.array_equal(Wg, Op[l].W)
        else:
            # FP32 box means vs FP64 box means may round to neighbouring codes at ties
            dI = Ig != Op[l].I
            dW = Wg != Op[l].W
            assert dI.mean() < 1e-3 and dW.mean() < 1e-3
            assert np.all(np.abs(Ig - Op[l].I)[dI] <= 2.0 ** -7 * np.abs(Op[l].I[dI]) + 1e-12)   # one bf16 ulp
            assert np.all(np.abs(Wg - Op[l].W)[dW] <= 2.0 ** -10 * np.abs(Op[l].W[dW]))


def test_reduced_eval_step_level0_matches_oracle_on_rounded_planes():
    pair = synth.make_pair(0)
    T = O.se3_exp([0.004, -0.003, 0.002, 0.003, -0.002, 0.004]) @ pair["T_gt"]
    planes = (O.build_pyramid_reduced(pair["I_A"], pair["W_A"], pair["K"], 3),
              O.build_pyramid_reduced(pair["I_B"], pair["W_B"], pair["K"], 3))
    g, o, A = eval_step_both(pair, 0, T, None, levels=3, precision=BF, oracle_planes=planes)
    check_step(g, o, A, 0)


def _align_gpu(pair, levels, iters, precision):
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels, precision)
    p = R.rgbid_default_params(levels=levels, iters=iters)
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, ws, res)
    torch.cuda.synchronize()
    return R.parse_result(res)


@pytest.mark.parametrize("seed", [0, 2, 5])
def test_reduced_alignment_matches_oracle_on_rounded_planes(seed):
    pair = synth.make_pair(seed)
    g = _align_gpu(pair, 3, (5, 5, 10), BF)
    A = O.build_pyramid_reduced(pair["I_A"], pair["W_A"], pair["K"], 3)
    B = O.build_pyramid_reduced(pair["I_B"], pair["W_B"], pair["K"], 3)
    o = O.align(A, B, None, O.AlignParams())
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    # storage error: the same alignment on the full-precision planes
    Af = O.build_pyramid(pair["I_A"], pair["W_A"], pair["K"], 3)
    Bf = O.build_pyramid(pair["I_B"], pair["W_B"], pair["K"], 3)
    of = O.align(Af, Bf, None, O.AlignParams())
    sr, st = pose_error(g["T"], of["T"])
    assert sr < 5e-4 and st < 5e-4


def test_reduced_alignment_640_matches_oracle_on_rounded_planes():
    pair = synth.make_pair(7, 640, 480, K=(525.0, 525.0, 319.5, 239.5))
    g = _align_gpu(pair, 4, (5, 5, 5, 10), BF)
    A = O.build_pyramid_reduced(pair["I_A"], pair["W_A"], pair["K"], 4)
    B = O.build_pyramid_reduced(pair["I_B"], pair["W_B"], pair["K"], 4)
    o = O.align(A, B, None, O.AlignParams(levels=4, iters=(5, 5, 5, 10)))
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
