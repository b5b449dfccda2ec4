"""The learned initialiser's kernels against the FP64 network oracle
(oracle/cnn_oracle.py): forward output, loss, parameter gradients, Adam, the
input packing from pyramids and the plan that turns proposals into items.

The GPU rounds stored tensors to bfloat16 where the oracle does and accumulates
in FP32 where the oracle is exact, so stored values can differ by one bfloat16
step where an FP32 sum lands next to a rounding boundary; the tolerances below
(relative to each tensor's norm) allow for that and nothing more."""
import ctypes

import numpy as np
import pytest

from oracle import cnn_oracle as C
from paper_1807_08271_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300 import rgbid as R  # noqa: E402
from paper_1807_08271_gb300.batch import BatchAligner  # noqa: E402
from paper_1807_08271_gb300.learned import InitNet, twist_of_pose  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(0)
    B = 3
    net = InitNet(max_batch=8, seed=3)
    x = C.round_bf16(rng.normal(size=(B, 60, 80, 4)) * 0.5)
    xd = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    t = rng.normal(size=(B, 6))
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    y = net.forward(xd, B).clone()
    R.rgbid_net_loss(net.y, td, B, net.dy, net.loss)
    R.rgbid_net_backward(net.params, xd, B, net.dy, net.grad, net.ws)
    torch.cuda.synchronize()
    p = net.params.cpu().numpy().astype(np.float64)
    yo, acts = C.forward(p, x)
    Lo, dyo = C.loss_and_grad(y.cpu().numpy().astype(np.float64), t)
    go = C.backward(p, acts, net.dy[:B].cpu().numpy().astype(np.float64))
    return dict(net=net, p=p, y=y.cpu().numpy(), yo=yo, L=float(net.loss.cpu()), Lo=Lo,
                dy=net.dy[:B].cpu().numpy(), dyo=dyo, g=net.grad.cpu().numpy(), go=go)


def test_init_is_he_uniform_with_zero_biases(case):
    p = case["p"]
    L = C.param_layout()
    for name, kind, kh, kw, ci, co in C.LAYERS:
        w_off, shape, b_off, nb = L[name]
        w = p[w_off:w_off + int(np.prod(shape))]
        bound = np.sqrt(6.0 / (kh * kw * ci))
        assert np.abs(w).max() <= bound and np.abs(w).max() > 0.9 * bound
        assert abs(w.mean()) < 0.05 * bound and abs(w.std() - bound / np.sqrt(3)) < 0.05 * bound
        assert np.all(p[b_off:b_off + nb] == 0)
    used = np.zeros(L["_total"], dtype=bool)
    for name, *_ in C.LAYERS:
        w_off, shape, b_off, nb = L[name]
        used[w_off:w_off + int(np.prod(shape))] = True
        used[b_off:b_off + nb] = True
    assert np.all(p[~used] == 0)


def test_forward_matches_oracle(case):
    assert _rel(case["y"], case["yo"]) < 3e-3


def test_loss_and_its_gradient_match_oracle(case):
    assert abs(case["L"] - case["Lo"]) <= 1e-5 * max(1.0, abs(case["Lo"]))
    assert _rel(case["dy"], case["dyo"]) < 1e-6


def test_parameter_gradients_match_oracle(case):
    L = C.param_layout()
    for name, *_ in C.LAYERS:
        w_off, shape, b_off, nb = L[name]
        n = int(np.prod(shape))
        assert _rel(case["g"][w_off:w_off + n], case["go"][w_off:w_off + n]) < 1e-2, name
        assert _rel(case["g"][b_off:b_off + nb], case["go"][b_off:b_off + nb]) < 1e-2, name
        cos = np.dot(case["g"][w_off:w_off + n], case["go"][w_off:w_off + n]) / (
            np.linalg.norm(case["g"][w_off:w_off + n]) * np.linalg.norm(case["go"][w_off:w_off + n]))
        assert cos > 0.9999, name


def test_adam_matches_oracle():
    rng = np.random.default_rng(1)
    P = R.rgbid_net_param_count()
    p = rng.normal(size=P)
    m = np.zeros(P)
    v = np.zeros(P)
    pd, md, vd = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (p, m, v))
    for t in range(1, 4):
        g = rng.normal(size=P)
        gd = torch.from_numpy(g.astype(np.float32)).cuda()
        R.rgbid_net_adam(pd, gd, md, vd, t, 1e-3)
        # the kernel's hyper-parameters are float32: give the oracle the same values
        p, m, v = C.adam_step(p, g.astype(np.float32).astype(np.float64), m, v, t, float(np.float32(1e-3)),
                              b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
    torch.cuda.synchronize()
    assert np.abs(pd.cpu().numpy() - p).max() < 1e-6
    assert _rel(md.cpu().numpy(), m) < 1e-6 and _rel(vd.cpu().numpy(), v) < 1e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_inputs_are_the_80x60_level_of_both_pyramids(precision):
    pair = synth.make_pair(4, 640, 480, K=(525.0, 525.0, 319.5, 239.5))
    dev = "cuda"
    PA = R.DevicePyramid(640, 480, 4, precision).build(torch.from_numpy(pair["I_A"]).to(dev),
                                                      torch.from_numpy(pair["W_A"]).to(dev), pair["K"])
    PB = R.DevicePyramid(640, 480, 4, precision).build(torch.from_numpy(pair["I_B"]).to(dev),
                                                      torch.from_numpy(pair["W_B"]).to(dev), pair["K"])
    B = BatchAligner([dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=4, iters=[5, 5, 5, 10])],
                     precision=precision)
    x = torch.zeros((1, 60, 80, 4), dtype=torch.bfloat16, device=dev)
    R.rgbid_net_inputs(B.d_items, 1, precision, x)
    torch.cuda.synchronize()
    IA, WA = PA.level_planes(3)
    IB, WB = PB.level_planes(3)
    want = C.input_stack(IA, WA, IB, WB)
    got = x[0].float().cpu().numpy().astype(np.float64)
    diff = got != want
    # the only admissible difference is the rounding of I - 0.5 in float32 before bfloat16
    assert diff.mean() < 1e-3
    assert np.all(np.abs(got - want)[diff] <= 2.0 ** -8 * np.abs(want[diff]) + 1e-12)


def test_plan_sets_start_pose_and_skips_levels_by_tier():
    dev = "cuda"
    pair = synth.make_pair(5, 640, 480, K=(525.0, 525.0, 319.5, 239.5))
    PA = R.DevicePyramid(640, 480, 4).build(torch.from_numpy(pair["I_A"]).to(dev),
                                           torch.from_numpy(pair["W_A"]).to(dev), pair["K"])
    PB = R.DevicePyramid(640, 480, 4).build(torch.from_numpy(pair["I_B"]).to(dev),
                                           torch.from_numpy(pair["W_B"]).to(dev), pair["K"])
    items = [dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=4, iters=[5, 5, 5, 10]) for _ in range(3)]
    B = BatchAligner(items)
    y = np.zeros((3, 7), dtype=np.float32)
    y[0, :6] = [0.3, -0.2, 0.1, 0.5, -0.4, 0.2]
    y[0, 6] = -6.0                                   # tier 2: skip two levels
    y[1, :6] = [-0.1, 0.2, 0.05, -0.3, 0.1, 0.4]
    y[1, 6] = -4.0                                   # tier 1: skip one level
    y[2, :6] = [0.1, 0.1, 0.1, 0.1, 0.1, 0.1]
    y[2, 6] = 0.0                                    # no tier: plain
    yd = torch.from_numpy(y).cuda()
    out = torch.zeros_like(B.d_items)
    skipped = torch.zeros(3, dtype=torch.int32, device=dev)
    R.rgbid_net_plan(yd, 3, [-3.0, -5.0], B.d_items, out, skipped)
    torch.cuda.synchronize()
    tab = (R.BatchItem * 3).from_buffer_copy(bytes(out.cpu().numpy()))
    src = (R.BatchItem * 3).from_buffer_copy(bytes(B.d_items.cpu().numpy()))
    assert skipped.cpu().tolist() == [2, 1, 0]
    for i, iters in ((0, [5, 5, 0, 0]), (1, [5, 5, 5, 0])):
        T = np.array(tab[i].T_init).reshape(4, 4)
        assert np.abs(T - C.pose_of(y[i, :6].astype(np.float64) * 0.1)).max() < 1e-12
        assert np.allclose(twist_of_pose(T), y[i, :6] * 0.1, atol=1e-12)
        assert list(tab[i].iters)[:4] == iters
    assert bytes(tab[2]) == bytes(src[2])


def test_training_lowers_the_loss_on_labelled_pairs():
    from paper_1807_08271_gb300.learned_train import label_chunk, train
    from paper_1807_08271_gb300.synth import gpu as G
    bank = G.TextureBank(11, n=8)
    x, lab, _, keep = label_chunk(5, 256, bank, R.PLANES_F32, 10.0, 0.15)
    assert keep.mean() > 0.9
    k = torch.from_numpy(np.nonzero(keep)[0]).cuda()
    X = x[k].contiguous()
    Y = torch.from_numpy((lab[keep] / R.NET_TWIST_SCALE).astype(np.float32)).cuda()
    net = InitNet(max_batch=64, seed=2)
    hist = train(net, X, Y, epochs=6, batch=64, lr=1e-3, seed=0, log=lambda m: None)
    assert hist[-1] < hist[0] - 0.5, hist


def test_no_tensor_core_wait_ran_out():
    # every GEMM above waited on its tcgen05 commits; none may have given up
    assert R.rgbid_net_wait_timeouts() == 0
