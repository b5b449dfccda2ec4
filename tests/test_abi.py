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
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(rgbid_level, IW), offsetof(rgbid_align_params, nu0),
         offsetof(rgbid_align_result, cost), offsetof(rgbid_align_result, status), sizeof(rgbid_timing),
         offsetof(rgbid_timing, units), offsetof(rgbid_align_params, timing),
         offsetof(rgbid_align_params, level_iters));
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
                         b.AlignParams.timing.offset, b.AlignParams.level_iters.offset]


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


def test_batch_struct_layouts_match_header(binding, tmp_path):
    src = tmp_path / "abi_batch.c"
    src.write_text(f'''#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rgbid_batch_item), offsetof(rgbid_batch_item, cur),
         offsetof(rgbid_batch_item, T_init), offsetof(rgbid_batch_item, levels),
         offsetof(rgbid_batch_item, iters), offsetof(rgbid_batch_item, result), sizeof(rgbid_batch_config));
  return 0;
}}''')
    exe = tmp_path / "abi_batch"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    b = binding
    assert sizes == [ctypes.sizeof(b.BatchItem), b.BatchItem.cur.offset, b.BatchItem.T_init.offset,
                     b.BatchItem.levels.offset, b.BatchItem.iters.offset, b.BatchItem.result.offset,
                     ctypes.sizeof(b.BatchConfig)]


def _host_item(b, w=320, h=240, levels=3, precision=0):
    """A descriptor whose pointers are never dereferenced (host-side checks only)."""
    it = b.BatchItem()
    for pyr, base in ((it.ref, 0x10000000), (it.cur, 0x20000000)):
        pyr.levels, pyr.precision = levels, precision
        for l in range(levels):
            L = pyr.lv[l]
            L.width, L.height, L.pitch = w >> l, h >> l, ((w >> l) + 15) // 16 * 16
            f = 525.0 * w / 640 / (1 << l)
            L.K = b.Intrinsics(f, f, (w >> l) / 2.0 - 0.5, (h >> l) / 2.0 - 0.5)
            L.IW = base + 4096 * l
    it.levels = levels
    for l in range(levels):
        it.iters[l] = 5
    it.T_init[0] = it.T_init[5] = it.T_init[10] = it.T_init[15] = 1.0
    it.result = 0x30000000
    return it


def test_batch_item_checks_on_the_host(binding):
    b = binding
    assert b.rgbid_align_batched_workspace_bytes() == 256
    it = _host_item(b)
    assert b.rgbid_batch_check_item(it, b.PLANES_F32) == b.OK
    assert b.rgbid_batch_check_item(it, b.PLANES_BF16_F16) == b.ERR_INVALID_ARG   # precision mismatch
    assert b.rgbid_batch_check_item(it, 7) == b.ERR_UNSUPPORTED
    bad = _host_item(b)
    bad.cur.lv[1].width += 1                      # sizes differ between A and B
    assert b.rgbid_batch_check_item(bad, b.PLANES_F32) == b.ERR_INVALID_ARG
    bad = _host_item(b)
    bad.levels = 4                                # more levels than the pyramids hold
    assert b.rgbid_batch_check_item(bad, b.PLANES_F32) == b.ERR_INVALID_ARG
    bad = _host_item(b)
    bad.ref.lv[0].IW += 4                         # float2 planes need 8-byte alignment
    assert b.rgbid_batch_check_item(bad, b.PLANES_F32) == b.ERR_INVALID_ARG
    bad = _host_item(b)
    bad.cur.lv[2].K = b.Intrinsics(1.0, 1.0, 1.0, 1.0)
    assert b.rgbid_batch_check_item(bad, b.PLANES_F32) == b.ERR_INVALID_ARG
    bad = _host_item(b)
    bad.iters[0] = -1
    assert b.rgbid_batch_check_item(bad, b.PLANES_F32) == b.ERR_INVALID_ARG
    bad = _host_item(b)
    bad.result = None
    assert b.rgbid_batch_check_item(bad, b.PLANES_F32) == b.ERR_INVALID_ARG


def test_batched_call_rejects_bad_arguments_before_launching(binding):
    b = binding
    L = b.lib()
    p = b.rgbid_default_params()
    cfg = b.BatchConfig(5, 2, 0, 0)             # unsupported cluster size
    ws = ctypes.create_string_buffer(512)
    assert L.rgbid_align_batched(None, 1, 0, ctypes.byref(p), None, None, 0, None) == b.ERR_INVALID_ARG
    assert L.rgbid_align_batched(None, 0, 0, ctypes.byref(p), ctypes.byref(cfg), None, 0, None) == b.ERR_INVALID_ARG
    assert L.rgbid_align_batched(None, 0, 3, ctypes.byref(p), None, None, 0, None) == b.ERR_UNSUPPORTED
    p.bisect_steps = 99
    assert L.rgbid_align_batched(None, 0, 0, ctypes.byref(p), None, None, 0, None) == b.ERR_INVALID_ARG
    p = b.rgbid_default_params()
    assert L.rgbid_align_batched(None, 0, 0, ctypes.byref(p), None, None, 0, None) == b.ERR_WORKSPACE
    # an empty batch with a valid (host-memory stand-in) workspace enqueues nothing
    addr = (ctypes.addressof(ws) + 255) // 256 * 256
    assert L.rgbid_align_batched(None, 0, 0, ctypes.byref(p), None, ctypes.c_void_p(addr), 256, None) == b.OK
