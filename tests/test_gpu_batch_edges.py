"""Edge cases of the batched alignment: degenerate schedules, tiny and ragged
images, duplicate and wrong-precision items, the empty batch, and a 640x480 pair
against the FP64 oracle directly."""
import ctypes

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


def _pyr(I, W, K, levels, precision=R.PLANES_F32):
    h, w = I.shape
    return R.DevicePyramid(w, h, levels, precision).build(torch.from_numpy(I).cuda(), torch.from_numpy(W).cuda(), K)


def _plain(PA, PB, T0, levels, iters, precision=R.PLANES_F32):
    p = R.rgbid_default_params(levels=levels, iters=iters)
    ws = R.new_workspace(PA.desc, p)
    r = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T0, p, ws, r)
    torch.cuda.synchronize()
    return R.parse_result(r)


def _crop_pair(seed, w, h):
    p = synth.make_pair(seed, 160, 120)
    K = p["K"]
    return (np.ascontiguousarray(p["I_A"][:h, :w]), np.ascontiguousarray(p["W_A"][:h, :w]),
            np.ascontiguousarray(p["I_B"][:h, :w]), np.ascontiguousarray(p["W_B"][:h, :w]), K, p["T_gt"])


def test_mixed_edge_items_match_the_per_pair_form():
    keep, items, expect = [], [], []
    # ragged 97x75 (tiles and samples with tails), 3 levels
    IA, WA, IB, WB, K, Tg = _crop_pair(1, 97, 75)
    PA, PB = _pyr(IA, WA, K, 3), _pyr(IB, WB, K, 3)
    keep += [PA, PB]
    items.append(dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=3, iters=[5, 5, 10]))
    expect.append(_plain(PA, PB, None, 3, [5, 5, 10]))
    # a tiny single-level pair rendered at 32x24 with its own (centred) intrinsics
    q = synth.make_pair(2, 32, 24)
    PA2, PB2 = _pyr(q["I_A"], q["W_A"], q["K"], 1), _pyr(q["I_B"], q["W_B"], q["K"], 1)
    keep += [PA2, PB2]
    items.append(dict(ref=PA2.desc, cur=PB2.desc, T_init=None, levels=1, iters=[4]))
    expect.append(_plain(PA2, PB2, None, 1, [4]))
    # no iterations at all: the start pose comes back unchanged
    T0 = synth.random_relative_pose(np.random.default_rng(3), 1.0, 0.01)
    items.append(dict(ref=PA.desc, cur=PB.desc, T_init=T0, levels=3, iters=[0, 0, 0]))
    expect.append(None)
    # the first item again: duplicate work gives the identical answer
    items.append(dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=3, iters=[5, 5, 10]))
    expect.append(expect[0])
    B = BatchAligner(items)
    B.run()
    torch.cuda.synchronize()
    res = B.all_results()
    for i in (0, 1, 3):
        assert res[i]["status"] == expect[i]["status"] and res[i]["iters_done"] == expect[i]["iters_done"], i
        er, et = pose_error(res[i]["T"], expect[i]["T"])
        assert er <= POSE_TOL and et <= POSE_TOL, (i, er, et)
    assert np.array_equal(res[0]["T"], res[3]["T"]) and np.array_equal(res[0]["H"], res[3]["H"])
    assert res[2]["iters_done"] == 0 and res[2]["status"] == R.OK
    assert np.array_equal(res[2]["T"], T0) and not np.any(res[2]["H"])


def test_wrong_precision_item_is_rejected_alone():
    p = synth.make_pair(4)
    PA, PB = _pyr(p["I_A"], p["W_A"], p["K"], 3), _pyr(p["I_B"], p["W_B"], p["K"], 3)
    QA = _pyr(p["I_A"], p["W_A"], p["K"], 3, R.PLANES_BF16_F16)
    good = dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=3, iters=[5, 5, 10])
    B = BatchAligner([good, good])
    # swap item 1's reference for a bf16 pyramid on the device (the host check would refuse it)
    table = (R.BatchItem * 2).from_buffer_copy(bytes(B.d_items.cpu().numpy()))
    table[1].ref = QA.desc
    B.d_items.copy_(torch.frombuffer(bytearray(bytes(table)), dtype=torch.uint8))
    B.run()
    torch.cuda.synchronize()
    res = B.all_results()
    bad = B.order[1]
    assert res[bad]["status"] == R.ERR_INVALID_ARG
    assert res[1 - bad]["status"] == R.OK and res[1 - bad]["iters_done"] == 20


def test_empty_batch_is_a_no_op():
    ws = torch.zeros(R.rgbid_align_batched_workspace_bytes(), dtype=torch.uint8, device="cuda")
    items = torch.zeros(8, dtype=torch.uint8, device="cuda")
    R.rgbid_align_batched(items, 0, R.PLANES_F32, R.rgbid_default_params(), None, ws)
    torch.cuda.synchronize()
    assert int(ws.sum()) == 0


def test_batched_640_pair_matches_the_oracle():
    pair = synth.make_pair(7, 640, 480, K=(525.0, 525.0, 319.5, 239.5))
    PA, PB = _pyr(pair["I_A"], pair["W_A"], pair["K"], 4), _pyr(pair["I_B"], pair["W_B"], pair["K"], 4)
    B = BatchAligner([dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=4, iters=[5, 5, 5, 10])])
    B.config = R.BatchConfig(16, 1, 0, 0)
    B.run()
    torch.cuda.synchronize()
    g = B.all_results()[0]
    A = O.build_pyramid(pair["I_A"], pair["W_A"], pair["K"], 4)
    Bo = O.build_pyramid(pair["I_B"], pair["W_B"], pair["K"], 4)
    o = O.align(A, Bo, None, O.AlignParams(levels=4, iters=(5, 5, 5, 10)))
    er, et = pose_error(g["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    assert g["iters_done"] == o["iters_done"] and g["status"] == o["status"]
