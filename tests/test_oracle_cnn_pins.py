"""Pins of the learned initialiser's FP64 oracle (oracle/cnn_oracle.py) against
definitions that do not depend on it: brute-force loops, scipy's correlation,
adjoint identities, central finite differences, the NLL's closed-form optimum
and a textbook property of Adam's first step.  CPU only."""
import numpy as np
import pytest
from scipy import signal

from oracle import cnn_oracle as C



def _brute_conv(x, W, b):
    B, H, Wd, Ci = x.shape
    Co = W.shape[3]
    Ho, Wo = (H - 1) // 2 + 1, (Wd - 1) // 2 + 1
    out = np.zeros((B, Ho, Wo, Co))
    for n in range(B):
        for i in range(Ho):
            for j in range(Wo):
                for o in range(Co):
                    acc = b[o]
                    for kh in range(3):
                        for kw in range(3):
                            y, xx = 2 * i + kh - 1, 2 * j + kw - 1
                            if 0 <= y < H and 0 <= xx < Wd:
                                for c in range(Ci):
                                    acc += x[n, y, xx, c] * W[kh, kw, c, o]
                    out[n, i, j, o] = acc
    return out


def test_conv_forward_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    for (H, Wd) in ((5, 7), (6, 8), (4, 5)):
        x = rng.normal(size=(2, H, Wd, 3))
        W = rng.normal(size=(3, 3, 3, 4))
        b = rng.normal(size=4)
        assert np.allclose(C.conv_forward(x, W, b), _brute_conv(x, W, b), atol=1e-12)


def test_conv_forward_matches_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 9, 12, 2))
    W = rng.normal(size=(3, 3, 2, 3))
    b = np.zeros(3)
    got = C.conv_forward(x, W, b)
    for o in range(3):
        ref = 0.0
        for c in range(2):
            xp = np.pad(x[0, :, :, c], 1)
            ref = ref + signal.correlate(xp, W[:, :, c, o], mode="valid")[::2, ::2]
        assert np.allclose(got[0, :, :, o], ref, atol=1e-12)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 7, 10, 5))
    W = rng.normal(size=(3, 3, 5, 6))
    g = rng.normal(size=(3, 4, 5, 6))
    dx, dW, db = C.conv_backward(x, W, g)
    zero = np.zeros(6)
    # linear in x: <conv(x), g> = <x, dx>;  linear in W: <conv_W(x), g> = <W, dW>
    assert np.isclose(np.sum(C.conv_forward(x, W, zero) * g), np.sum(x * dx), rtol=1e-12)
    assert np.isclose(np.sum(C.conv_forward(x, W, zero) * g), np.sum(W * dW), rtol=1e-12)
    assert np.allclose(db, g.sum(axis=(0, 1, 2)))


def test_layout_counts_and_alignment():
    L = C.param_layout()
    n = 0
    for name, kind, kh, kw, ci, co in C.LAYERS:
        w_off, shape, b_off, nb = L[name]
        assert w_off % C.ALIGN == 0 and b_off % C.ALIGN == 0
        assert int(np.prod(shape)) == kh * kw * ci * co and nb == co
        n += kh * kw * ci * co + co
    assert n == 395591
    assert L["_total"] >= n
    # the flattened c4 output feeds f1
    assert 64 * C.conv_out_size(C.conv_out_size(C.conv_out_size(C.conv_out_size(60)))) * \
        C.conv_out_size(C.conv_out_size(C.conv_out_size(C.conv_out_size(80)))) == 1280


def _small_params(rng):
    L = C.param_layout()
    p = np.zeros(L["_total"])
    for name, kind, kh, kw, ci, co in C.LAYERS:
        w_off, shape, b_off, nb = L[name]
        fan_in = kh * kw * ci
        p[w_off:w_off + int(np.prod(shape))] = rng.normal(size=int(np.prod(shape))) * np.sqrt(2.0 / fan_in)
        p[b_off:b_off + nb] = rng.normal(size=nb) * 0.1
    return p


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = _small_params(rng)
    x = rng.normal(size=(2, 60, 80, 4)) * 0.5
    t = rng.normal(size=(2, 6))

    def loss(pp):
        y, _ = C.forward(pp, x, rounding=False)
        return C.loss_and_grad(y, t)[0]

    y, acts = C.forward(p, x, rounding=False)
    _, dy = C.loss_and_grad(y, t)
    g = C.backward(p, acts, dy, rounding=False)
    L = C.param_layout()
    picks = []
    for name, *_ in C.LAYERS:
        w_off, shape, b_off, nb = L[name]
        picks += list(w_off + rng.choice(int(np.prod(shape)), 5, replace=False))
        picks += list(b_off + rng.choice(nb, 2, replace=False))
    for i in picks:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_nll_gradient_and_optimum():
    rng = np.random.default_rng(4)
    y = rng.normal(size=(3, 7))
    t = rng.normal(size=(3, 6))
    L, dy = C.loss_and_grad(y, t)
    for b in range(3):
        for j in range(7):
            h = 1e-6
            yp, ym = y.copy(), y.copy()
            yp[b, j] += h
            ym[b, j] -= h
            fd = (C.loss_and_grad(yp, t)[0] - C.loss_and_grad(ym, t)[0]) / (2 * h)
            assert abs(fd - dy[b, j]) < 1e-8
    # for fixed residuals the NLL is minimal at exp(s) = |d|^2 / 6 (the Gaussian variance MLE)
    d2 = ((y[:, :6] - t) ** 2).sum(axis=1)
    y2 = y.copy()
    y2[:, 6] = np.log(d2 / 6.0)
    _, dy2 = C.loss_and_grad(y2, t)
    assert np.allclose(dy2[:, 6], 0.0, atol=1e-12)
    assert C.loss_and_grad(np.concatenate([t, np.zeros((3, 1))], axis=1), t)[0] == 0.0


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(5)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = C.adam_step(p, g, np.zeros(100), np.zeros(100), 1, 1e-3, eps=1e-12)
    assert np.allclose(p - p1, 1e-3 * np.sign(g), rtol=1e-6)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_rounded_forward_stays_close_to_float64():
    rng = np.random.default_rng(6)
    p = _small_params(rng)
    x = rng.normal(size=(2, 60, 80, 4)) * 0.5
    y0, _ = C.forward(p, x, rounding=False)
    y1, acts = C.forward(p, x, rounding=True)
    assert np.abs(y1 - y0).max() <= 2e-2 * np.abs(y0).max()
    # stored activations are bfloat16 values
    for a in acts:
        assert np.array_equal(C.round_bf16(a), a)


def test_twist_pose_round_trip():
    rng = np.random.default_rng(7)
    for _ in range(5):
        tw = rng.normal(size=6) * 0.2
        assert np.allclose(C.twist_of(C.pose_of(tw)), tw, atol=1e-12)
