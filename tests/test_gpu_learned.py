"""The learned initialiser in use: the device-side iteration schedule of
rgbid_align, and (with the committed trained weights) the gain of the learned
start over the plain alignment on held-out 640x480 pairs at equal accuracy."""
import os

import numpy as np
import pytest

from paper_1807_08271_gb300 import synth

from parity import pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402
from paper_1807_08271_gb300 import learned as Lm  # noqa: E402


def _pyr(pair, levels=4):
    dev = "cuda"
    PA = R.DevicePyramid(pair["width"], pair["height"], levels).build(torch.from_numpy(pair["I_A"]).to(dev),
                                                                     torch.from_numpy(pair["W_A"]).to(dev), pair["K"])
    PB = R.DevicePyramid(pair["width"], pair["height"], levels).build(torch.from_numpy(pair["I_B"]).to(dev),
                                                                     torch.from_numpy(pair["W_B"]).to(dev), pair["K"])
    return PA, PB


def test_device_level_schedule_matches_host_schedule():
    pair = synth.make_pair(3, 640, 480, K=(525.0, 525.0, 319.5, 239.5), max_angle_deg=4.0, max_trans=0.06)
    PA, PB = _pyr(pair)
    T0 = pair["T_gt"] @ synth.random_relative_pose(np.random.default_rng(1), 1.0, 0.01)
    # host schedule: the two finest levels only
    p_host = R.rgbid_default_params(levels=2, iters=[5, 4])
    ws = R.new_workspace(PA.desc, p_host)
    r_host = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T0, p_host, ws, r_host)
    # device schedule: all four levels launched, the two coarsest set to zero iterations on the device
    lv = torch.tensor([5, 4, 0, 0, 0, 0], dtype=torch.int32, device="cuda")
    p_dev = R.rgbid_default_params(levels=4, iters=[5, 5, 5, 10])
    p_dev.level_iters = lv.data_ptr()
    r_dev = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T0, p_dev, ws, r_dev)
    torch.cuda.synchronize()
    a, b = R.parse_result(r_host), R.parse_result(r_dev)
    assert a["iters_done"] == b["iters_done"] == 9
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["H"], b["H"])
    assert a["status"] == b["status"] == R.OK


def _weights():
    if not os.path.exists(Lm.WEIGHTS):
        pytest.skip("no trained weights in the package")
    return Lm.InitNet.load(Lm.WEIGHTS, max_batch=1024)


@pytest.fixture(scope="module")
def held_out():
    from paper_1807_08271_gb300.learned_train import EvalSet
    from paper_1807_08271_gb300.synth import gpu as G
    bank = G.TextureBank(4242, n=16)
    return EvalSet(777, 256, bank, 10.0, 0.15)


def _summary(ev, results):
    from paper_1807_08271_gb300.learned_train import pose_diff
    ok = ev.converged(results)
    err = [pose_diff(r["T"], T)[0] for r, T in zip(results, ev.T_gt)]
    return float(np.mean(ok)), float(np.median(err)), float(np.mean([r["iters_done"] for r in results]))


def test_learned_start_per_pair_is_faster_at_equal_accuracy(held_out):
    from paper_1807_08271_gb300.learned_train import evaluate_per_pair
    net = _weights()
    thr = net.meta["thresholds"]
    r = evaluate_per_pair(net, held_out, thr, held_out.n)
    p, q = r["plain"], r["learned"]
    assert q["converged_fraction"] >= p["converged_fraction"]
    assert q["median_rot_err_vs_truth_rad"] <= 1.5 * p["median_rot_err_vs_truth_rad"] + 1e-5
    assert q["mean_iterations"] <= p["mean_iterations"] - 8
    assert q["alignments_per_s"] >= 1.1 * p["alignments_per_s"], (q["alignments_per_s"], p["alignments_per_s"])


def test_learned_start_batched_is_faster_at_equal_accuracy(held_out):
    from paper_1807_08271_gb300.learned import LearnedPlanner
    from paper_1807_08271_gb300.learned_train import _sized
    net = _weights()
    thr = net.meta["thresholds"]
    res_p, ms_p, _ = held_out.run(None, reps=5)
    res_l, ms_l, B = held_out.run(lambda m, prec: LearnedPlanner(_sized(net, m), m, prec, thr), reps=5)
    cp, ep, ip = _summary(held_out, res_p)
    cl, el, il = _summary(held_out, res_l)
    assert cl >= cp and el <= 1.5 * ep + 1e-5 and il <= ip - 8
    assert ms_l < ms_p, (ms_l, ms_p)
    # pairs in no tier ran the plain alignment unchanged
    skipped = B.planner.skipped[:held_out.n].cpu().numpy()
    for slot in np.nonzero(skipped == 0)[0]:
        i = B.order[slot]
        assert np.array_equal(res_l[i]["T"], res_p[i]["T"])
