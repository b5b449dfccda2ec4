"""The C ABI (include/rgbid.h): the library builds, loads, exports every declared
symbol, and the Python binding's structures have the header's layout.
No GPU is needed: nothing here launches a kernel."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rgbid.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rgbid_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def binding():
    from paper_1807_08271_gb300 import rgbid
    return rgbid


def test_library_exports_every_declared_symbol(binding):
    L = binding.lib()
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n
    assert sorted(n for n, _, _ in binding.SIGNATURES) == names


def test_struct_layouts_match_header(binding, tmp_path):
    src = tmp_path / "abi.c"
    src.write_text(f'''#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu\\n", sizeof(rgbid_intrinsics), sizeof(rgbid_level), sizeof(rgbid_pyramid),
         sizeof(rgbid_align_params), sizeof(rgbid_align_result));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(rgbid_level, IW), offsetof(rgbid_align_params, nu0),
         offsetof(rgbid_align_result, cost), offsetof(rgbid_align_result, status), sizeof(rgbid_timing),
         offsetof(rgbid_timing, units), offsetof(rgbid_align_params, timing));
  return 0;
}}''')
    exe = tmp_path / "abi"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    b = binding
    assert sizes[:5] == [ctypes.sizeof(b.Intrinsics), ctypes.sizeof(b.Level), ctypes.sizeof(b.Pyramid),
                         ctypes.sizeof(b.AlignParams), ctypes.sizeof(b.AlignResult)]
    assert sizes[5:] == [b.Level.IW.offset, b.AlignParams.nu0.offset, b.AlignResult.cost.offset,
                         b.AlignResult.status.offset, ctypes.sizeof(b.Timing), b.Timing.units.offset,
                         b.AlignParams.timing.offset]


def test_host_side_calls_without_a_gpu(binding):
    """Calls that only compute sizes or validate arguments run on the host."""
    b = binding
    assert b.rgbid_status_string(0) == "RGBID_OK"
    assert b.rgbid_status_string(4) == "RGBID_ERR_DEGENERATE"
    p = b.rgbid_default_params()
    assert (p.levels, list(p.iters)[:3], p.scale_iters, p.bisect_steps, p.sample_cap) == (3, [5, 5, 10], 10, 20, 19200)
    assert (p.nu0, p.nu_lo, p.nu_hi, p.estimate_nu) == (5.0, 2.0, 10.0, 1)
    n = b.rgbid_pyramid_bytes(640, 480, 4, b.PLANES_F32)
    assert n >= 8 * (640 * 480 + 320 * 240 + 160 * 120 + 80 * 60)
    assert b.rgbid_pyramid_bytes(640, 480, 4, b.PLANES_BF16_F16) < n
    assert b.rgbid_pyramid_bytes(640, 480, 7, b.PLANES_F32) == 0
    # argument validation rejects before touching the device
    L = b.lib()
    out = b.Pyramid()
    K = b.Intrinsics(525.0, 525.0, 319.5, 239.5)
    code = L.rgbid_build_pyramid(None, None, 640, 640, 480, K, 4, 0, None, 0, ctypes.byref(out), None)
    assert code == b.ERR_INVALID_ARG
    code = L.rgbid_align(None, None, None, 0, None, None, 0, None, None)
    assert code == b.ERR_INVALID_ARG
