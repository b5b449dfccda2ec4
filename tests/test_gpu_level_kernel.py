"""The one-launch-per-level kernels of rgbid_align against the per-iteration
robust-scale and sweep kernels and the FP64 oracle: the persistent level kernel (a
level whose systematic sample is every pixel runs all its Gauss-Newton iterations in
one 16-CTA cluster launch) and the split kernel (a larger level: the cluster solves,
samples and estimates the robust parameters while helper CTAs of the same
cooperative launch evaluate every pixel).

Both paths evaluate the same steps ("Iterative optimisation", "Error
distribution and robust optimisation"); their FP32 sums run in another order,
so their poses agree far inside the oracle tolerance but not bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_1807_08271_gb300 import synth

from parity import POSE_TOL, gpu_pair, oracle_pair, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402

KINECT = (525.0, 525.0, 319.5, 239.5)
PATHS_TOL = 1e-6      # rad and m between the two paths (summation order only)


def _align(PA, PB, levels, iters, level_kernel, T_init=None, level_iters=None, timer=None):
    p = R.rgbid_default_params(levels=levels, iters=iters)
    p.no_level_kernel = 0 if level_kernel else 1
    if level_iters is not None:
        p.level_iters = level_iters.data_ptr()
    if timer is not None:
        timer.attach(p)
    ws = R.new_workspace(PA.desc, p)
    res = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, T_init, p, ws, res)
    torch.cuda.synchronize()
    return R.parse_result(res), p


@pytest.fixture(scope="module")
def pair640():
    return synth.make_pair(4, 640, 480, K=KINECT, max_angle_deg=4.0, max_trans=0.08)


def _both_paths(pair, levels, iters, precision=R.PLANES_F32, T_init=None):
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels, precision)
    a, pa = _align(PA, PB, levels, iters, True, T_init)
    b, pb = _align(PA, PB, levels, iters, False, T_init)
    return a, b, (PA, PB, pa, pb)


@pytest.mark.parametrize("precision", [R.PLANES_F32, R.PLANES_BF16_F16])
def test_level_kernel_matches_the_per_iteration_kernels_and_the_oracle(pair640, precision):
    a, b, (PA, _, pa, pb) = _both_paths(pair640, 4, (5, 5, 5, 10), precision)
    # one level-kernel launch (80x60) and one split launch (160x120, 320x240 and
    # 640x480 in turn) replace 2 x 25 per-iteration launches
    assert R.rgbid_align_launches(PA.desc, pa) == 2 + 2
    assert R.rgbid_align_launches(PA.desc, pb) == 2 + 2 * 25
    er, et = pose_error(a["T"], b["T"])
    assert er <= PATHS_TOL and et <= PATHS_TOL, (er, et)
    assert a["status"] == b["status"] == R.OK
    assert a["iters_done"] == b["iters_done"] == 25 and a["iters_skipped"] == b["iters_skipped"] == 0
    for c in range(2):
        assert abs(a["n_valid"][c] - b["n_valid"][c]) <= 2
        assert abs(a["sigma"][c] - b["sigma"][c]) <= 1e-4 * b["sigma"][c]
    if precision == R.PLANES_F32:
        A, B = oracle_pair(pair640, 4)
        o = O.align(A, B, None, O.AlignParams(levels=4, iters=(5, 5, 5, 10)))
        er, et = pose_error(a["T"], o["T"])
        assert er <= POSE_TOL and et <= POSE_TOL, (er, et)


@pytest.mark.parametrize("seed", [0, 6])
def test_every_level_in_one_launch(seed):
    """160x120: every level's sample is every pixel; the finest level runs in the split
    kernel (its sample at stride 1), the two coarser in the level kernel, then the
    closing launch."""
    pair = synth.make_pair(seed)
    T0 = O.se3_exp([0.004, -0.003, 0.002, 0.01, -0.006, 0.003])
    a, b, (PA, PB, pa, _) = _both_paths(pair, 3, (5, 5, 10), T_init=T0)
    assert R.rgbid_align_launches(PA.desc, pa) == 2 + 3
    lvl, spl = R.KernelTimer(R.KERNEL_LEVEL, 8), R.KernelTimer(R.KERNEL_SPLIT, 8)
    _align(PA, PB, 3, (5, 5, 10), True, T_init=T0, timer=lvl)
    _align(PA, PB, 3, (5, 5, 10), True, T_init=T0, timer=spl)
    assert (lvl.t.count, spl.t.count) == (2, 1)
    assert spl.t.units == 160 * 120 * 5
    er, et = pose_error(a["T"], b["T"])
    assert er <= PATHS_TOL and et <= PATHS_TOL, (er, et)
    A, B = oracle_pair(pair, 3)
    o = O.align(A, B, T0, O.AlignParams())
    er, et = pose_error(a["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    assert a["iters_done"] == 20 and a["status"] == o["status"]


def test_device_iteration_counts_in_the_level_kernel(pair640):
    """level_iters read on the device: the coarsest level skipped and the next cut to
    3 iterations gives the bits of the host schedule with those counts."""
    (PA, _, _), (PB, _, _) = gpu_pair(pair640, 4)
    counts = torch.tensor([5, 5, 3, 0], dtype=torch.int32, device="cuda")
    dev_sched, _ = _align(PA, PB, 4, (5, 5, 5, 10), True, level_iters=counts)
    host_sched, _ = _align(PA, PB, 4, (5, 5, 3, 0), True)
    assert np.array_equal(dev_sched["T"], host_sched["T"]) and np.array_equal(dev_sched["H"], host_sched["H"])
    assert dev_sched["iters_done"] == host_sched["iters_done"] == 13
    per_it, _ = _align(PA, PB, 4, (5, 5, 5, 10), False, level_iters=counts)
    er, et = pose_error(dev_sched["T"], per_it["T"])
    assert er <= PATHS_TOL and et <= PATHS_TOL, (er, et)
    # device counts that cut the split levels too
    counts2 = torch.tensor([2, 3, 5, 10], dtype=torch.int32, device="cuda")
    dev2, _ = _align(PA, PB, 4, (5, 5, 5, 10), True, level_iters=counts2)
    host2, _ = _align(PA, PB, 4, (2, 3, 5, 10), True)
    assert np.array_equal(dev2["T"], host2["T"]) and np.array_equal(dev2["H"], host2["H"])
    assert dev2["iters_done"] == 20


def test_level_kernel_timing_counts_its_launches_and_units(pair640):
    (PA, _, _), (PB, _, _) = gpu_pair(pair640, 4)
    timer = R.KernelTimer(R.KERNEL_LEVEL, 8)
    _align(PA, PB, 4, (5, 5, 5, 10), True, timer=timer)
    assert timer.t.count == 1
    assert timer.t.units == 80 * 60 * 10
    assert timer.total_ms() > 0.0
    split = R.KernelTimer(R.KERNEL_SPLIT, 8)
    _align(PA, PB, 4, (5, 5, 5, 10), True, timer=split)
    assert split.t.count == 1
    assert split.t.units == 640 * 480 * 5 + 320 * 240 * 5 + 160 * 120 * 5
    assert split.total_ms() > 0.0


def test_split_kernel_is_deterministic(pair640):
    (PA, _, _), (PB, _, _) = gpu_pair(pair640, 4)
    a, _ = _align(PA, PB, 4, (5, 5, 5, 10), True)
    b, _ = _align(PA, PB, 4, (5, 5, 5, 10), True)
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["H"], b["H"]) and np.array_equal(a["g"], b["g"])


def test_split_kernel_on_a_pyramid_with_few_sweep_blocks():
    """A 200x100 finest level (stride 2, 91 tiles): fewer sweep blocks than helper CTAs,
    so the workspace must hold a partial per helper."""
    K = (200.0, 200.0, 99.5, 49.5)
    pair = synth.make_pair(9, 200, 100, K=K, max_angle_deg=3.0, max_trans=0.05)
    a, b, (PA, _, pa, _) = _both_paths(pair, 2, (5, 10))
    assert R.rgbid_align_launches(PA.desc, pa) == 2 + 2
    er, et = pose_error(a["T"], b["T"])
    assert er <= PATHS_TOL and et <= PATHS_TOL, (er, et)
    A, B = oracle_pair(pair, 2)
    o = O.align(A, B, None, O.AlignParams(levels=2, iters=(5, 10)))
    er, et = pose_error(a["T"], o["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)


def test_a_level_without_measurements_is_degenerate_in_the_level_kernel():
    pair = synth.make_pair(2)
    p = dict(pair)
    p["W_A"] = np.zeros_like(p["W_A"])
    T0 = O.se3_exp([0.01, 0, 0, 0, 0, 0])
    a, b, _ = _both_paths(p, 3, (5, 5, 10), T_init=T0)
    for g in (a, b):
        assert np.array_equal(g["T"], T0)
        assert g["status"] == R.ERR_DEGENERATE and g["iters_skipped"] == 20 and g["n_valid"] == [0, 0]


def test_a_reference_without_measurements_is_degenerate_in_the_split_kernel(pair640):
    p = dict(pair640)
    p["W_A"] = np.zeros_like(p["W_A"])
    T0 = O.se3_exp([0.0, 0.01, 0, 0, 0, 0.002])
    a, b, _ = _both_paths(p, 4, (5, 5, 5, 10), T_init=T0)
    for g in (a, b):
        assert np.array_equal(g["T"], T0)
        assert g["status"] == R.ERR_DEGENERATE and g["iters_skipped"] == 25 and g["n_valid"] == [0, 0]
