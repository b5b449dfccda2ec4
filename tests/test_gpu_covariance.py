"""Covariance of the motion estimate (rgbid_covariance: one non-updating
iteration at the final pose with the reference bilateral-filtered before its
gradients are taken, Sigma = H_filt^-1; "Dense motion estimation") through the
C ABI, against the FP64 oracle (oracle.covariance) at the same pose."""
import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import H_TOL, gpu_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402

KINECT = (525.0, 525.0, 319.5, 239.5)


def _case(seed, w, h, levels, iters, reduced=False):
    pair = synth.make_pair(seed, w, h, K=None if w == 160 else KINECT)
    build = O.build_pyramid_reduced if reduced else O.build_pyramid
    A = build(pair["I_A"], pair["W_A"], pair["K"], levels)
    B = build(pair["I_B"], pair["W_B"], pair["K"], levels)
    P = O.AlignParams(levels=levels, iters=iters)
    T = O.align(A, B, None, P)["T"]
    return pair, A, B, P, T


def _gpu(pair, levels, iters, T, filt, reduced=False, T_dev=False):
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels, R.PLANES_BF16_F16 if reduced else R.PLANES_F32)
    p = R.rgbid_default_params(levels=levels, iters=iters)
    ws = R.new_covariance_workspace(PA.desc)
    res = R.result_tensor()
    sig = torch.zeros(36, dtype=torch.float64, device="cuda")
    Tin = torch.from_numpy(np.asarray(T, dtype=np.float64).reshape(16).copy()).cuda() if T_dev else T
    R.rgbid_covariance(PA.desc, PB.desc, Tin, p, filt, ws, res, sig)
    torch.cuda.synchronize()
    return R.parse_result(res), sig.cpu().numpy().reshape(6, 6), (PA, PB, p)


def _compare(g, S, o, F):
    Ho = o["H"]
    d = np.sqrt(np.outer(np.diag(Ho), np.diag(Ho)))
    assert (np.abs(g["H"] - Ho) <= H_TOL * d).all(), np.max(np.abs(g["H"] - Ho) / d)
    for c in range(2):
        assert g["n_valid"][c] == o["n_valid"][c] or abs(g["n_valid"][c] - o["n_valid"][c]) <= 2
        assert abs(g["sigma"][c] - o["robust"]["sigma"][c]) <= 1e-5 * o["robust"]["sigma"][c]
        # mu is the weighted mean of the fixed point: its weights move with sigma's
        # 1e-5 relative error, which moves mu by up to a few 1e-5 of sigma
        assert abs(g["mu"][c] - o["robust"]["mu"][c]) <= 3e-5 * o["robust"]["sigma"][c]
    # Sigma = H^-1: a normalised error of H of e moves Sigma by at most about cond(D H D) e
    Dm = np.diag(1.0 / np.sqrt(np.diag(Ho)))
    cond = np.linalg.cond(Dm @ Ho @ Dm)
    So = o["Sigma"]
    ds = np.sqrt(np.outer(np.diag(So), np.diag(So)))
    assert (np.abs(S - So) <= 2 * H_TOL * cond * ds).all(), (np.max(np.abs(S - So) / ds), cond)
    assert np.allclose(S @ g["H"], np.eye(6), atol=1e-8)


@pytest.mark.parametrize("shape", [(160, 120, 3, (5, 5, 10)), (640, 480, 4, (5, 5, 5, 10))])
def test_covariance_matches_the_oracle(shape):
    w, h, levels, iters = shape
    pair, A, B, P, T = _case(5, w, h, levels, iters)
    F = O.BilateralParams()
    o = O.covariance(A, B, T, P, F)
    g, S, _ = _gpu(pair, levels, iters, T, R.rgbid_default_bilateral())
    assert g["status"] == R.OK and o["ok"]
    _compare(g, S, o, F)
    # the filter lowers the information of the noisy reference
    assert np.trace(S) > np.trace(np.linalg.inv(O.eval_step(A, B, 0, T, None, P)["H"]))


def test_covariance_of_the_reduced_precision_planes_and_a_device_pose():
    pair, A, B, P, T = _case(6, 160, 120, 3, (5, 5, 10), reduced=True)
    F = O.BilateralParams(radius=3, sigma_s=2.0, sigma_r_I=0.05, sigma_r_W=0.02)
    o = O.covariance(A, B, T, P, F)
    g, S, _ = _gpu(pair, 3, (5, 5, 10), T, R.rgbid_default_bilateral(radius=3, sigma_s=2.0, sigma_r_I=0.05,
                                                                        sigma_r_W=0.02), reduced=True, T_dev=True)
    assert g["status"] == R.OK
    _compare(g, S, o, F)


def test_radius_zero_is_the_unfiltered_step_and_a_featureless_reference_is_degenerate():
    pair, A, B, P, T = _case(7, 160, 120, 3, (5, 5, 10))
    g, S, (PA, PB, p) = _gpu(pair, 3, (5, 5, 10), T, R.rgbid_default_bilateral(radius=0))
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_eval_step(PA.desc, PB.desc, 0, T, None, p, ws, None, None, None, None, res)
    torch.cuda.synchronize()
    e = R.parse_result(res)
    assert np.array_equal(g["H"], e["H"]) and np.array_equal(g["g"], e["g"])
    assert np.allclose(S, np.linalg.inv(e["H"]), rtol=1e-9, atol=0)
    # no inverse depth in the reference: no residual, no covariance
    I = torch.from_numpy(pair["I_A"]).cuda()
    Z = torch.zeros_like(I)
    PZ = R.DevicePyramid(160, 120, 3).build(I, Z, pair["K"])
    res2 = R.result_tensor()
    sig = torch.full((36,), 7.0, dtype=torch.float64, device="cuda")
    R.rgbid_covariance(PZ.desc, PB.desc, T, p, R.rgbid_default_bilateral(), R.new_covariance_workspace(PZ.desc),
                       res2, sig)
    torch.cuda.synchronize()
    assert R.parse_result(res2)["status"] == R.ERR_DEGENERATE
    assert not sig.cpu().numpy().any()
