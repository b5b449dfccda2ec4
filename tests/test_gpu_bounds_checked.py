"""Every gather of the kernels stays inside its plane (the stand-in for a memory
checker, which this GPU pool does not offer): the GPU parity, edge-case and fault
tests run again in a child process against the bounds-checked build
(librgbid_checked.so, -DRGBID_BOUNDS_CHECK), whose kernels check every index they
gather from an image plane against the plane's allocation and count those outside
it; the count must be zero and the tests must pass there too."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the per-iteration and one-launch-per-level alignment paths, both plane precisions,
# ragged and non-finite inputs, the full-resolution warp, the covariance iteration,
# covisibility and fusion, the batched kernel's edge cases and the failure probes
MODULES = ["test_gpu_parity.py", "test_gpu_level_kernel.py", "test_gpu_precision.py", "test_gpu_warp_full.py",
           "test_gpu_covariance.py", "test_gpu_covisibility.py", "test_gpu_faults.py", "test_gpu_batch_edges.py"]


def test_gathers_stay_inside_their_planes(tmp_path):
    report = tmp_path / "violations.txt"
    env = dict(os.environ, RGBID_LIBRARY="checked", RGBID_BOUNDS_REPORT=str(report))
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
           *[os.path.join(ROOT, "tests", m) for m in MODULES]]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert report.exists(), r.stdout[-2000:]
    assert report.read_text().strip() == "0", f"out-of-plane gathers: {report.read_text()}"


def test_the_product_build_does_not_check():
    from paper_1807_08271_gb300 import rgbid as R
    if os.environ.get("RGBID_LIBRARY") == "checked":
        pytest.skip("running against the checked build")
    assert R.rgbid_debug_bounds_violations() is None
