"""The 64-pair loop-closure batch (16 pairs each at 320x240, 640x480, 960x720
and 1280x960; up to 10 deg / 20 cm; perturbed ground-truth start) through the
batched persistent kernel and through the per-pair form, against the FP64
oracle's alignment of every pair, stored in tests/golden/c3_oracle_poses.json
and c3_oracle_poses_reduced.json (written by tests/golden/make_c3_oracle_poses.py).
Every pose within 1e-5 rad / 1e-5 m of the oracle's: with the launch shape the
autotuner picks for this batch and with every shape it can pick."""
import json
import os

import numpy as np
import pytest

from paper_1807_08271_gb300 import synth

from parity import POSE_TOL, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402
from paper_1807_08271_gb300.batch import BatchAligner  # noqa: E402

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def pairs():
    return synth.make_batch(seed=0, n=64)


def _setup(pairs, precision):
    keep, items = [], []
    for p in pairs:
        w, h = p["width"], p["height"]
        out = []
        for I, W in ((p["I_A"], p["W_A"]), (p["I_B"], p["W_B"])):
            out.append(R.DevicePyramid(w, h, p["levels"], precision).build(torch.from_numpy(I).cuda(),
                                                                          torch.from_numpy(W).cuda(), p["K"]))
        keep += out
        items.append(dict(ref=out[0].desc, cur=out[1].desc, T_init=p["T_init"], levels=p["levels"],
                          iters=p["iters"]))
    return keep, items


def _gold(reduced):
    name = "c3_oracle_poses_reduced.json" if reduced else "c3_oracle_poses.json"
    g = json.load(open(os.path.join(HERE, name)))["pairs"]
    return [np.array(g[str(i)]["T"]).reshape(4, 4) for i in range(len(g))], g


def _check(results, gold, label):
    errs = np.array([pose_error(r["T"], G) for r, G in zip(results, gold)])
    print(f"{label}: max {errs[:, 0].max():.2e} rad {errs[:, 1].max():.2e} m, "
          f"median {np.median(errs[:, 0]):.2e} rad")
    bad = np.argwhere((errs > POSE_TOL).any(axis=1)).ravel()
    assert bad.size == 0, f"{label}: pairs {bad.tolist()} at {errs[bad].tolist()}"
    return errs


@pytest.mark.parametrize("reduced", [False, True])
def test_autotuned_batch_matches_the_oracle_on_every_pair(pairs, reduced):
    prec = R.PLANES_BF16_F16 if reduced else R.PLANES_F32
    keep, items = _setup(pairs, prec)
    gold, g = _gold(reduced)
    B = BatchAligner(items, precision=prec)
    B.tune(reps=2)
    B.capture()
    for _ in range(2):
        B.replay()
    torch.cuda.synchronize()
    res = B.all_results()
    for r, p, i in zip(res, pairs, range(len(pairs))):
        assert r["status"] == g[str(i)]["status"] and r["iters_done"] == g[str(i)]["iters_done"], i
    _check(res, gold, f"batch {B.config.as_tuple()} {'reduced' if reduced else 'fp32'}")


@pytest.mark.parametrize("cluster", [4, 8, 16])
@pytest.mark.parametrize("rows", [1, 2, 4])
def test_every_batch_shape_matches_the_oracle(pairs, cluster, rows):
    keep, items = _setup(pairs, R.PLANES_F32)
    gold, _ = _gold(False)
    B = BatchAligner(items)
    resident = R.rgbid_batch_resident_clusters(R.PLANES_F32, R.BatchConfig(cluster, rows, 0, 0))
    if resident < 1:
        pytest.skip("shape does not fit on this device")
    for n_clusters in (0, max(1, resident // 2)):      # all or half of the resident clusters
        B.config = R.BatchConfig(cluster, rows, n_clusters, 0)
        B.run()
        torch.cuda.synchronize()
        _check(B.all_results(), gold, f"batch ({cluster}, {rows}, {n_clusters})")


@pytest.mark.parametrize("reduced", [False, True])
def test_per_pair_form_matches_the_oracle_on_every_pair(pairs, reduced):
    prec = R.PLANES_BF16_F16 if reduced else R.PLANES_F32
    keep, items = _setup(pairs, prec)
    gold, _ = _gold(reduced)
    res = []
    for p, it in zip(pairs, items):
        prm = R.rgbid_default_params(levels=p["levels"], iters=p["iters"])
        ws = R.new_workspace(it["ref"], prm)
        out = R.result_tensor()
        R.rgbid_align(it["ref"], it["cur"], p["T_init"], prm, ws, out)
        res.append(out)
    torch.cuda.synchronize()
    _check([R.parse_result(r) for r in res], gold, f"per pair {'reduced' if reduced else 'fp32'}")
