"""The C ABI (include/rgbid.h): the library builds, loads, exports every declared
symbol, and the Python binding's structures have the header's layout.
No GPU is needed: nothing here launches a kernel."""
import ctypes
import os
import re
import subprocess

import numpy as np
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
  printf("%zu %zu %zu %zu %zu\\n", sizeof(rgbid_bilateral), offsetof(rgbid_bilateral, sigma_s),
         offsetof(rgbid_bilateral, sigma_r_W), offsetof(rgbid_align_params, warp_mode),
         offsetof(rgbid_align_params, no_level_kernel));
  return 0;
}}''')
    exe = tmp_path / "abi"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    b = binding
    assert sizes[:5] == [ctypes.sizeof(b.Intrinsics), ctypes.sizeof(b.Level), ctypes.sizeof(b.Pyramid),
                         ctypes.sizeof(b.AlignParams), ctypes.sizeof(b.AlignResult)]
    assert sizes[5:13] == [b.Level.IW.offset, b.AlignParams.nu0.offset, b.AlignResult.cost.offset,
                           b.AlignResult.status.offset, ctypes.sizeof(b.Timing), b.Timing.units.offset,
                           b.AlignParams.timing.offset, b.AlignParams.level_iters.offset]
    assert sizes[13:] == [ctypes.sizeof(b.Bilateral), b.Bilateral.sigma_s.offset, b.Bilateral.sigma_r_W.offset,
                          b.AlignParams.warp_mode.offset, b.AlignParams.no_level_kernel.offset]


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


def test_the_product_build_has_no_diagnostic_counters(binding):
    """The bounds-checked and phase-stamped builds are separate libraries; the product
    library answers their queries with RGBID_ERR_UNSUPPORTED without touching a device."""
    import os
    if os.environ.get("RGBID_LIBRARY") in ("checked", "phases"):
        pytest.skip("running against a diagnostic build")
    L = binding.lib()
    n = ctypes.c_ulonglong(7)
    assert L.rgbid_debug_bounds_violations(ctypes.byref(n)) == binding.ERR_UNSUPPORTED and n.value == 0
    assert L.rgbid_debug_bounds_violations(None) == binding.ERR_INVALID_ARG
    buf = (ctypes.c_longlong * (binding.MAX_LEVELS * 256))()
    assert L.rgbid_debug_phase_stamps(buf, len(buf)) == binding.ERR_UNSUPPORTED
    assert binding.rgbid_debug_bounds_violations() is None and binding.rgbid_debug_phase_stamps() is None
    from paper_1807_08271_gb300 import build
    with pytest.raises(ValueError):
        build.build(checked=True, phases=True)


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


def _no_device():
    """The pointer-check tests below pass made-up device addresses: they run only
    where no GPU exists, so a check that failed to reject could never reach a kernel."""
    try:
        import torch
        return not torch.cuda.is_available()
    except ImportError:  # pragma: no cover
        return True


@pytest.mark.skipif(not _no_device(), reason="made-up device addresses stay off machines with a GPU")
def test_misaligned_and_nonfinite_arguments_are_rejected_on_the_host(binding):
    b = binding
    L = b.lib()
    V = ctypes.c_void_p
    base = 0x7F0000000000                                  # 256-byte aligned stand-in addresses
    K = b.Intrinsics(131.25, 131.25, 79.5, 59.5)

    def pyr(iw, prec=b.PLANES_F32, K=K):
        P = b.Pyramid()
        P.levels, P.precision = 1, prec
        lv = P.lv[0]
        lv.width, lv.height, lv.pitch, lv.IW, lv.K = 160, 120, 160, iw, K
        return P

    p = b.rgbid_default_params(levels=1, iters=[3])
    ws, wsb = V(base + 0x100000), 1 << 24
    res = V(base + 0x200000)

    def align(A, B, T=None, on_dev=0, result=res, params=p):
        return L.rgbid_align(ctypes.byref(A), ctypes.byref(B), T, on_dev, ctypes.byref(params), ws, wsb, result, None)

    good = pyr(base)
    assert align(pyr(base + 4), good) == b.ERR_INVALID_ARG                   # f32 pixel is 8 bytes
    assert align(good, pyr(base + 4)) == b.ERR_INVALID_ARG
    assert align(pyr(base + 2, b.PLANES_BF16_F16), pyr(base, b.PLANES_BF16_F16)) == b.ERR_INVALID_ARG
    assert align(good, good, result=V(base + 0x200004)) == b.ERR_INVALID_ARG  # result record: 8 bytes
    assert align(good, good, T=V(base + 0x300004), on_dev=1) == b.ERR_INVALID_ARG
    q = b.rgbid_default_params(levels=1, iters=[3])
    q.level_iters = base + 0x400002
    assert align(good, good, params=q) == b.ERR_INVALID_ARG
    for bad in ((np.nan, 131.25, 79.5, 59.5), (131.25, np.inf, 79.5, 59.5), (131.25, 131.25, np.nan, 59.5),
                (131.25, 131.25, 79.5, -np.inf), (-1.0, 131.25, 79.5, 59.5)):
        Kb = b.Intrinsics(*bad)
        assert align(pyr(base, K=Kb), pyr(base, K=Kb)) == b.ERR_INVALID_ARG, bad
        out = b.Pyramid()
        assert L.rgbid_build_pyramid(V(base), V(base + 0x10000), 160, 160, 120, Kb, 1, 0, ws, wsb,
                                     ctypes.byref(out), None) == b.ERR_INVALID_ARG, bad
    # fusion, keyframe initialisation, pose helpers
    f = [V(base + i * 0x100000) for i in range(5)]
    T, s = V(base + 0x600000), V(base + 0x700000)
    assert L.rgbid_fuse_keyframe(V(base + 2), *f[1:3], 160, *f[3:5], 160, 160, 120, K, T, s, 1, 1, None) == \
        b.ERR_INVALID_ARG
    assert L.rgbid_fuse_keyframe(*f[:3], 160, *f[3:5], 160, 160, 120, K, V(base + 0x600004), s, 1, 1, None) == \
        b.ERR_INVALID_ARG
    assert L.rgbid_fuse_keyframe(*f[:3], 160, *f[3:5], 160, 160, 120, b.Intrinsics(131.25, 131.25, np.nan, 59.5),
                                 T, s, 1, 1, None) == b.ERR_INVALID_ARG
    assert L.rgbid_init_keyframe(*f[:3], 160, f[3], V(base + 0x400001), 160, 160, 120, None) == b.ERR_INVALID_ARG
    assert L.rgbid_predict_pose(T, V(base + 0x600004), s, None) == b.ERR_INVALID_ARG
    assert L.rgbid_compose_pose(T, 0, s, V(base + 0x800004), None) == b.ERR_INVALID_ARG
    # batched alignment and the network
    assert L.rgbid_align_batched(V(base + 4), 1, 0, ctypes.byref(p), None, ws, wsb, None) == b.ERR_INVALID_ARG
    nws = b.rgbid_net_workspace_bytes(4)
    assert L.rgbid_net_forward(V(base + 2), f[1], 4, f[2], ws, nws, None) == b.ERR_INVALID_ARG
    assert L.rgbid_net_backward(*f[:2], 4, V(base + 0x300002), f[3], ws, nws, None) == b.ERR_INVALID_ARG
    assert L.rgbid_net_loss(f[0], f[1], 4, f[2], V(base + 0x400002), None) == b.ERR_INVALID_ARG
    assert L.rgbid_net_adam(*f[:3], V(base + 0x400001), 1, 1e-3, 0.9, 0.999, 1e-8, None) == b.ERR_INVALID_ARG
    assert L.rgbid_net_inputs(V(base + 4), 1, 0, f[1], None) == b.ERR_INVALID_ARG
    assert L.rgbid_net_init(V(base + 2), 1, None) == b.ERR_INVALID_ARG
    assert L.rgbid_net_plan(f[0], 1, None, 0, V(base + 0x100004), f[2], None, None) == b.ERR_INVALID_ARG
    # covisibility, the keyframe decision and fusion-or-switch
    cnt, flag = V(base + 0x900000), V(base + 0xA00000)
    assert L.rgbid_covisibility(V(base + 2), *f[1:2], 160, *f[2:4], 160, 160, 120, K, T, s, 1, cnt, None,
                                None) == b.ERR_INVALID_ARG
    assert L.rgbid_covisibility(*f[:2], 160, *f[2:4], 160, 160, 120, K, T, s, 1, V(base + 0x900002), None,
                                None) == b.ERR_INVALID_ARG
    assert L.rgbid_covisibility(*f[:2], 160, *f[2:4], 160, 160, 120, b.Intrinsics(131.25, -1.0, 79.5, 59.5), T, s,
                                1, cnt, None, None) == b.ERR_INVALID_ARG
    assert L.rgbid_keyframe_decide(cnt, 1.5, T, f[0], f[1], flag, None, None) == b.ERR_INVALID_ARG
    assert L.rgbid_keyframe_decide(cnt, 0.7, T, f[0], f[0], flag, None, None) == b.ERR_INVALID_ARG
    assert L.rgbid_keyframe_decide(cnt, 0.7, T, f[0], f[1], V(base + 0xA00002), None, None) == b.ERR_INVALID_ARG
    assert L.rgbid_fuse_or_switch_keyframe(*f[:3], 160, *f[3:5], 160, 160, 120, K, T, s, 1, None, None) == \
        b.ERR_INVALID_ARG
    # the covariance iteration: filter values and workspace
    filt = b.rgbid_default_bilateral()
    d_sig = V(base + 0xB00000)

    def cov(A, B, F=filt, wsz=wsb, sigma=d_sig):
        return L.rgbid_covariance(ctypes.byref(A), ctypes.byref(B), T, 1, ctypes.byref(p), ctypes.byref(F), ws,
                                  wsz, res, sigma, None)
    assert cov(good, good, F=b.rgbid_default_bilateral(radius=6)) == b.ERR_INVALID_ARG
    assert cov(good, good, F=b.rgbid_default_bilateral(sigma_r_W=0.0)) == b.ERR_INVALID_ARG
    assert cov(good, good, F=b.rgbid_default_bilateral(sigma_s=np.inf)) == b.ERR_INVALID_ARG
    assert cov(good, good, sigma=V(base + 0xB00004)) == b.ERR_INVALID_ARG
    assert cov(good, good, wsz=b.lib().rgbid_covariance_workspace_bytes(ctypes.byref(good)) - 1) == b.ERR_WORKSPACE
    # the warp mode: unknown values are rejected, and the batched form takes the per-level warp only
    pw = b.rgbid_default_params(levels=1, iters=[3])
    pw.warp_mode = 2
    assert align(good, good, params=pw) == b.ERR_INVALID_ARG
    pw.warp_mode = b.WARP_FULL_RESOLUTION
    assert L.rgbid_align_batched(V(base), 1, 0, ctypes.byref(pw), None, ws, wsb, None) == b.ERR_UNSUPPORTED
    # the level-kernel switch takes 0 or 1
    pk = b.rgbid_default_params(levels=1, iters=[3])
    assert pk.no_level_kernel == 0
    pk.no_level_kernel = 2
    assert align(good, good, params=pk) == b.ERR_INVALID_ARG
    # the wait-timeout probe's own arguments
    assert L.rgbid_probe_wait_timeout(-1, f[0], None) == b.ERR_INVALID_ARG
    assert L.rgbid_probe_wait_timeout(1000, None, None) == b.ERR_INVALID_ARG
    # ... and the mailbox probe's (scratch too small, misaligned, NULL output, bad budget)
    assert L.rgbid_probe_mailbox_timeout(1000, f[0], 512, f[0], None) == b.ERR_INVALID_ARG
    assert L.rgbid_probe_mailbox_timeout(1000, V(base + 4), 1024, f[0], None) == b.ERR_INVALID_ARG
    assert L.rgbid_probe_mailbox_timeout(1000, f[0], 1024, None, None) == b.ERR_INVALID_ARG
    assert L.rgbid_probe_mailbox_timeout(-1, f[0], 1024, f[0], None) == b.ERR_INVALID_ARG


def test_nu_constant_series_matches_digamma(binding):
    """The host series of the degrees-of-freedom equation's constant part
    (psi((nu+1)/2) - psi(nu/2) + 1 + ln nu) against scipy's digamma."""
    from scipy.special import digamma
    # every interval the alignment accepts has (lo + hi)/(hi - lo) >= 1.4
    for lo, hi in ((2.0, 10.0), (2.0, 12.0), (1.0, 5.0), (3.0, 4.0)):
        g = np.array(binding.rgbid_nu_constant_series(lo, hi), dtype=np.float64)
        assert len(g) == 22
        nu = np.linspace(lo, hi, 997)
        tau = (nu - 0.5 * (lo + hi)) / (0.5 * (hi - lo))
        want = digamma(0.5 * (nu + 1)) - digamma(0.5 * nu) + 1 + np.log(nu)
        got = np.polynomial.chebyshev.chebval(tau, g)
        # float32 coefficients: a few ulps of the largest one
        assert np.abs(got - want).max() < 1e-6 * max(1.0, np.abs(g).max()), (lo, hi)
    assert binding.lib().rgbid_nu_constant_series(10.0, 2.0, (ctypes.c_float * 4)(), 4) == -binding.ERR_INVALID_ARG
    assert binding.lib().rgbid_nu_constant_series(1.5, 30.0, (ctypes.c_float * 4)(), 4) == -binding.ERR_UNSUPPORTED


def test_workspace_covers_the_largest_sweep_over_the_levels(binding):
    """The alignment workspace holds the state plus one 32-slot compensated pair per
    block of the largest sweep over the reference's levels (32-pixel-wide tiles of
    8 rows on levels under 250K pixels, 32 rows on larger ones), and at least one per
    helper CTA the split level kernel may launch (128).  Descriptor-only pyramids:
    nothing is read or launched."""
    b = binding

    def blocks(w, h):
        th = 32 if w * h >= 250000 else 8
        return ((w + 31) // 32) * ((h + th - 1) // th)

    for w0, h0, levels in ((640, 480, 4), (160, 120, 3), (97, 75, 3), (1280, 960, 5), (32, 24, 1)):
        P = b.Pyramid()
        P.levels, P.precision = levels, b.PLANES_F32
        w, h = w0, h0
        nb = 128
        for l in range(levels):
            P.lv[l].width, P.lv[l].height, P.lv[l].pitch = w, h, w
            nb = max(nb, blocks(w, h))
            w, h = w // 2, h // 2
        got = b.rgbid_align_workspace_bytes(P, b.rgbid_default_params(levels=levels, iters=[1] * levels))
        assert got >= nb * 32 * 8, (w0, h0, got, nb)
        assert got <= nb * 32 * 8 + 4096, (w0, h0, got, nb)   # the state header and alignment padding only
