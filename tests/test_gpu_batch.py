"""Batched persistent alignment (rgbid_align_batched) against the per-pair
form (rgbid_align) and the FP64 oracle.

Both GPU forms evaluate the same per-pixel terms; they differ only in how the
sums are partitioned (cluster CTAs and tiles here, one block per tile there),
so their poses agree to FP32 summation-order effects (<= 1e-5 rad / 1e-5 m).
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import H_TOL, POSE_TOL, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402
from paper_1807_08271_gb300.batch import BatchAligner  # noqa: E402


def _pyramids(pair, levels, precision=R.PLANES_F32):
    w, h = pair["width"], pair["height"]
    out = []
    for I, W in ((pair["I_A"], pair["W_A"]), (pair["I_B"], pair["W_B"])):
        P = R.DevicePyramid(w, h, levels, precision).build(torch.from_numpy(I).cuda(), torch.from_numpy(W).cuda(),
                                                           pair["K"])
        out.append(P)
    return out


def _plain(PA, PB, T_init, levels, iters):
    p = R.rgbid_default_params(levels=levels, iters=iters)
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T_init, p, ws, res)
    torch.cuda.synchronize()
    return R.parse_result(res)


def _make(pairs, precision=R.PLANES_F32):
    keep, items = [], []
    for p in pairs:
        PA, PB = _pyramids(p, p["levels"], precision)
        keep += [PA, PB]
        items.append(dict(ref=PA.desc, cur=PB.desc, T_init=p["T_init"], levels=p["levels"], iters=p["iters"]))
    return keep, items


def _small_pairs(n=6, seed=11):
    rng = np.random.default_rng(seed)
    pairs = []
    for i in range(n):
        w, h = ((160, 120), (320, 240))[i % 2]
        p = synth.make_pair(int(rng.integers(1 << 30)), w, h, max_angle_deg=10.0, max_trans=0.2)
        p["T_init"] = p["T_gt"] @ synth.random_relative_pose(rng, 2.0, 0.03)
        p["levels"] = 3
        p["iters"] = [5, 5, 10]
        pairs.append(p)
    return pairs


@pytest.fixture(scope="module")
def small():
    pairs = _small_pairs()
    keep, items = _make(pairs)
    plain = [_plain(PA, PB, p["T_init"], p["levels"], p["iters"])
             for p, PA, PB in zip(pairs, keep[0::2], keep[1::2])]
    return pairs, keep, items, plain


def _close(a, b, tol=POSE_TOL):
    er, et = pose_error(a["T"], b["T"])
    assert er <= tol and et <= tol, (er, et)


def test_batched_matches_per_pair_alignment(small):
    pairs, keep, items, plain = small
    B = BatchAligner(items)
    B.run()
    torch.cuda.synchronize()
    for i, (g, q) in enumerate(zip(B.all_results(), plain)):
        assert g["status"] == q["status"] == R.OK, i
        assert g["iters_done"] == q["iters_done"] == sum(pairs[i]["iters"])
        _close(g, q)
        d = np.sqrt(np.outer(np.diag(q["H"]), np.diag(q["H"])))
        assert (np.abs(g["H"] - q["H"]) <= 10 * H_TOL * d).all(), i
        for c in range(2):
            assert abs(g["n_valid"][c] - q["n_valid"][c]) <= max(2, 1e-4 * q["n_valid"][c])
            assert abs(g["nu"][c] - q["nu"][c]) <= 1e-3 * q["nu"][c]
            assert abs(g["sigma"][c] - q["sigma"][c]) <= 1e-4 * q["sigma"][c]


@pytest.mark.parametrize("cluster", [4, 8, 16])
@pytest.mark.parametrize("rows", [1, 2, 4])
def test_every_launch_shape_agrees(small, cluster, rows):
    pairs, keep, items, plain = small
    B = BatchAligner(items)
    B.config = R.BatchConfig(cluster, rows, 0, 0)
    if R.rgbid_batch_resident_clusters(R.PLANES_F32, B.config) < 1:
        pytest.skip("shape does not fit on this device")
    B.run()
    torch.cuda.synchronize()
    for g, q in zip(B.all_results(), plain):
        assert g["status"] == R.OK
        _close(g, q)


def test_fewer_clusters_than_pairs_drain_the_queue(small):
    pairs, keep, items, plain = small
    B = BatchAligner(items)
    B.config = R.BatchConfig(8, 2, 1, 0)            # one cluster takes every pair in turn
    B.run()
    torch.cuda.synchronize()
    for g, q in zip(B.all_results(), plain):
        assert g["iters_done"] == q["iters_done"]
        _close(g, q)
    assert int(B.workspace.sum()) == 0                # the queue is left empty for the next batch


def test_deterministic_and_graph_replay(small):
    pairs, keep, items, plain = small
    B = BatchAligner(items)
    B.config = R.BatchConfig(8, 2, 0, 0)
    B.run()
    torch.cuda.synchronize()
    first = B.results.clone()
    B.results.zero_()
    B.capture()
    for _ in range(2):
        B.results.zero_()
        B.replay()
        torch.cuda.synchronize()
        assert torch.equal(B.results, first)        # same shape -> same sums in the same order
    # another cluster count changes which cluster runs which pair, not the arithmetic
    B2 = BatchAligner(items)
    B2.config = R.BatchConfig(8, 2, 2, 0)
    B2.run()
    torch.cuda.synchronize()
    assert torch.equal(B2.results, first)


def test_invalid_item_is_reported_and_the_rest_complete(small):
    pairs, keep, items, plain = small
    B = BatchAligner(items[:3])
    table = (R.BatchItem * 3).from_buffer_copy(bytes(B.d_items.cpu().numpy()))
    table[1].cur.lv[0].width += 2                   # A and B differ: rejected on the device
    B.d_items.copy_(torch.frombuffer(bytearray(bytes(table)), dtype=torch.uint8))
    B.run()
    torch.cuda.synchronize()
    res = B.all_results()
    bad = B.order[1]
    for i, r in enumerate(res):
        if i == bad:
            assert r["status"] == R.ERR_INVALID_ARG and r["iters_done"] == 0
        else:
            assert r["status"] == R.OK
            _close(r, plain[i])


def test_batched_matches_oracle_on_small_pairs(small):
    pairs, keep, items, plain = small
    B = BatchAligner(items[:2])
    B.run()
    torch.cuda.synchronize()
    for i, g in enumerate(B.all_results()):
        p = pairs[i]
        A = O.build_pyramid(p["I_A"], p["W_A"], p["K"], 3)
        Bp = O.build_pyramid(p["I_B"], p["W_B"], p["K"], 3)
        o = O.align(A, Bp, p["T_init"], O.AlignParams(levels=3, iters=(5, 5, 10)))
        er, et = pose_error(g["T"], o["T"])
        assert er <= POSE_TOL and et <= POSE_TOL, (i, er, et)


def test_reduced_precision_batch_matches_per_pair_form():
    pairs = _small_pairs(4, seed=5)
    keep, items = _make(pairs, R.PLANES_BF16_F16)
    B = BatchAligner(items, precision=R.PLANES_BF16_F16)
    B.run()
    torch.cuda.synchronize()
    for i, g in enumerate(B.all_results()):
        q = _plain(keep[2 * i], keep[2 * i + 1], pairs[i]["T_init"], 3, [5, 5, 10])
        assert g["status"] == R.OK
        _close(g, q)


@pytest.fixture(scope="module")
def loop_closure_batch():
    """64 pairs, 16 at each of 320x240, 640x480, 960x720 and 1280x960."""
    pairs = synth.make_batch(seed=0)
    keep, items = _make(pairs)
    return pairs, keep, items


def test_loop_closure_batch_matches_per_pair_form_and_truth(loop_closure_batch):
    pairs, keep, items = loop_closure_batch
    B = BatchAligner(items)
    cfg = B.tune(reps=2)
    assert cfg.cluster in (4, 8, 16) and cfg.rows_per_warp in (1, 2, 4) and cfg.n_clusters >= 1
    B.results.zero_()
    B.run()
    torch.cuda.synchronize()
    res = B.all_results()
    errs_truth = []
    for i, p in enumerate(pairs):
        q = _plain(keep[2 * i], keep[2 * i + 1], p["T_init"], p["levels"], p["iters"])
        assert res[i]["status"] == q["status"]
        _close(res[i], q)
        errs_truth.append(pose_error(res[i]["T"], p["T_gt"])[0])
    # the dense check recovers the ground truth from the perturbed seed
    assert np.median(errs_truth) < 2e-3 and np.max(errs_truth) < 2e-2, (np.median(errs_truth), np.max(errs_truth))


def test_loop_closure_batch_outruns_the_per_pair_form(loop_closure_batch):
    pairs, keep, items = loop_closure_batch
    B = BatchAligner(items)
    B.tune(reps=2)
    B.capture()
    B.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        B.replay()
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 3
    ps, wss, rs = [], [], []
    for p in pairs:
        pp = R.rgbid_default_params(levels=p["levels"], iters=p["iters"])
        ps.append(pp)
    for i in range(len(pairs)):
        wss.append(R.new_workspace(keep[2 * i].desc, ps[i]))
        rs.append(R.result_tensor())
    torch.cuda.synchronize()
    e0.record()
    for i, p in enumerate(pairs):
        R.rgbid_align(keep[2 * i].desc, keep[2 * i + 1].desc, p["T_init"], ps[i], wss[i], rs[i])
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1)
    assert t_batch < t_plain, (t_batch, t_plain)
