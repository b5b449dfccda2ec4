"""The allocation-free alignment entry point, rgbid_align_noalloc.

Some callers cannot allocate device memory or keep a workspace (a real-time
loop under a no-allocation policy, a plugin whose host owns every device
allocation).  rgbid_align_noalloc serves them with a fixed scratch array inside
the library.  These checks call it through the C ABI twice in a row, on two
different frame pairs, and compare each result with rgbid_align's (which uses a
caller-owned workspace) within the alignment tolerances.  The file is named so
that pytest collects it last; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1807_08271_gb300 import synth

from parity import H_TOL, POSE_TOL, gpu_pair, pose_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402


def _both(pair, levels, iters):
    (PA, _, _), (PB, _, _) = gpu_pair(pair, levels)
    p = R.rgbid_default_params(levels=levels, iters=iters)
    ws = R.new_workspace(PA.desc, p)
    res_ws = R.result_tensor()
    res_na = R.result_tensor()
    R.rgbid_align(PA.desc, PB.desc, None, p, ws, res_ws)
    R.rgbid_align_noalloc(PA.desc, PB.desc, None, p, res_na)
    torch.cuda.synchronize()
    return R.parse_result(res_ws), R.parse_result(res_na)


def _close(a, b):
    er, et = pose_error(a["T"], b["T"])
    assert er <= POSE_TOL and et <= POSE_TOL, (er, et)
    d = np.sqrt(np.outer(np.diag(a["H"]), np.diag(a["H"])))
    assert (np.abs(a["H"] - b["H"]) <= H_TOL * d).all()
    assert a["n_valid"] == b["n_valid"] and a["status"] == b["status"] and a["iters_done"] == b["iters_done"]


def test_noalloc_matches_workspace_alignment_on_two_calls_in_a_row():
    first = synth.make_pair(2)
    second = synth.make_pair(7, 640, 480, K=(525.0, 525.0, 319.5, 239.5))
    a, b = _both(first, 3, (5, 5, 10))
    _close(a, b)
    c, d = _both(second, 4, (5, 5, 5, 10))
    _close(c, d)
    # the second call did not inherit the first call's state
    assert pose_error(b["T"], d["T"])[0] > 1e-4


def test_noalloc_rejects_a_reference_beyond_the_scratch_size():
    big = R.Pyramid()
    big.levels = 1
    big.precision = R.PLANES_F32
    big.lv[0].width, big.lv[0].height, big.lv[0].pitch = 4096, 4096, 4096
    big.lv[0].K = R.Intrinsics(3000.0, 3000.0, 2047.5, 2047.5)
    big.lv[0].IW = 256                      # never dereferenced: the size check comes first
    p = R.rgbid_default_params(levels=1, iters=(1,))
    code = R.lib().rgbid_align_noalloc(ctypes.byref(big), ctypes.byref(big), None, 0, ctypes.byref(p), None, None)
    assert code == R.ERR_WORKSPACE
