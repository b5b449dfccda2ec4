"""FP64 oracle of the learned initialiser's network.

TEST INFRASTRUCTURE ONLY (see the package header): the product never imports it.

The paper has no learned component; this network is the project's extension
that proposes the initial twist of a frame-to-keyframe alignment (and how far
to trust it) from the 80x60 pyramid level of both frames.  Definitions used:

Network (activations NHWC, batch first):
  x   [B, 60, 80, 4]   channels I_A - 0.5, W_A, I_B - 0.5, W_B of the 80x60 level
  c1  3x3 conv, stride 2, zero pad 1,  4 -> 32, ReLU   -> [B, 30, 40, 32]
  c2  3x3 conv, stride 2, zero pad 1, 32 -> 32, ReLU   -> [B, 15, 20, 32]
  c3  3x3 conv, stride 2, zero pad 1, 32 -> 64, ReLU   -> [B,  8, 10, 64]
  c4  3x3 conv, stride 2, zero pad 1, 64 -> 64, ReLU   -> [B,  4,  5, 64]
  f1  fully connected 1280 -> 256 (input = c4 flattened in NHWC order), ReLU
  f2  fully connected  256 -> 7:  y[0:6] = twist / TWIST_SCALE, y[6] = s
A convolution is the cross-correlation
  out[b, i, j, o] = bias[o] + sum_{kh, kw, c} x[b, 2i + kh - 1, 2j + kw - 1, c] W[kh, kw, c, o]
with x = 0 outside the image; a fully connected layer is out = x W + bias with
W stored [in, out].

Twist: translation first, then the rotation vector, of the decoupled pose
T = [exp([w]x), t; 0, 1] (the decoupled SE(3) map of "Preliminaries").

Loss per pair, averaged over the batch: the negative log-likelihood of an
isotropic Gaussian with variance exp(s) in the scaled twist units, constants
dropped:  L = 0.5 exp(-s) |y[0:6] - t|^2 + 3 s.

Optimiser: Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization",
2015, Algorithm 1) with bias correction.

Storage rounding (``rounding=True``): the input, the weights, every hidden
activation after ReLU, the loss gradient entering the network and every
back-propagated activation gradient are rounded to bfloat16 (nearest, ties to
even) where they are stored; sums are exact float64 here.  Biases, the output
y and all parameter gradients stay unrounded.  With ``rounding=False`` the
same functions are plain float64 (finite-difference pins use that).
"""
from __future__ import annotations

import numpy as np

from .rgbid_oracle import round_bf16

IN_H, IN_W, IN_C = 60, 80, 4
OUT = 7
TWIST_SCALE = 0.1          # metres and radians per network unit

# (name, kind, kh, kw, c_in, c_out); convolutions are 3x3, stride 2, pad 1
LAYERS = [
    ("c1", "conv", 3, 3, 4, 32),
    ("c2", "conv", 3, 3, 32, 32),
    ("c3", "conv", 3, 3, 32, 64),
    ("c4", "conv", 3, 3, 64, 64),
    ("f1", "fc", 1, 1, 1280, 256),
    ("f2", "fc", 1, 1, 256, OUT),
]
ALIGN = 64                 # every tensor starts on a multiple of 64 parameters


def _pad_to(n: int) -> int:
    return (n + ALIGN - 1) // ALIGN * ALIGN


def param_layout() -> dict:
    """name -> (W offset, W shape, bias offset, bias length); plus the total count."""
    off, out = 0, {}
    for name, kind, kh, kw, ci, co in LAYERS:
        shape = (kh, kw, ci, co) if kind == "conv" else (ci, co)
        w_off = off
        off = _pad_to(off + int(np.prod(shape)))
        b_off = off
        off = _pad_to(off + co)
        out[name] = (w_off, shape, b_off, co)
    out["_total"] = off
    return out


def unpack(params: np.ndarray) -> dict:
    L = param_layout()
    d = {}
    for name, kind, *_ in LAYERS:
        w_off, shape, b_off, n = L[name]
        d[name] = (params[w_off:w_off + int(np.prod(shape))].reshape(shape), params[b_off:b_off + n])
    return d


def _r(a, rounding):
    return round_bf16(a) if rounding else np.asarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- layers
def conv_out_size(n: int) -> int:
    return (n + 2 - 3) // 2 + 1


def conv_forward(x: np.ndarray, W: np.ndarray, bias: np.ndarray) -> np.ndarray:
    """3x3 stride-2 zero-pad-1 cross-correlation, NHWC (the definition above,
    written as a sum over the nine kernel taps of (pixels x c_in) @ (c_in x c_out))."""
    B, H, Wd, C = x.shape
    Ho, Wo = conv_out_size(H), conv_out_size(Wd)
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:H + 1, 1:Wd + 1, :] = x
    out = np.zeros((B, Ho, Wo, W.shape[3])) + bias
    for kh in range(3):
        for kw in range(3):
            patch = xp[:, kh:kh + 2 * Ho:2, kw:kw + 2 * Wo:2, :]       # x[b, 2i + kh - 1, 2j + kw - 1, :]
            out += patch @ W[kh, kw]
    return out


def conv_backward(x: np.ndarray, W: np.ndarray, g: np.ndarray):
    """Adjoint of conv_forward: (dL/dx, dL/dW, dL/dbias) given g = dL/dout."""
    B, H, Wd, C = x.shape
    Ho, Wo = g.shape[1], g.shape[2]
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:H + 1, 1:Wd + 1, :] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for kh in range(3):
        for kw in range(3):
            patch = xp[:, kh:kh + 2 * Ho:2, kw:kw + 2 * Wo:2, :]
            dW[kh, kw] = np.einsum("bijc,bijo->co", patch, g)
            dxp[:, kh:kh + 2 * Ho:2, kw:kw + 2 * Wo:2, :] += g @ W[kh, kw].T
    return dxp[:, 1:H + 1, 1:Wd + 1, :], dW, g.sum(axis=(0, 1, 2))


def relu(z):
    return np.maximum(z, 0.0)


# ----------------------------------------------------------------------------- network
def forward(params: np.ndarray, x: np.ndarray, rounding: bool = True):
    """y [B, 7] and the stored activations (for backward)."""
    P = unpack(params)
    a = _r(x, rounding)
    acts = [a]
    for name, kind, *_ in LAYERS:
        W, b = P[name]
        Wr = _r(W, rounding)
        if kind == "conv":
            z = conv_forward(a, Wr, b)
        else:
            z = a.reshape(a.shape[0], -1) @ Wr + b
        if name == "f2":
            return z, acts
        a = _r(relu(z), rounding)
        acts.append(a)
    raise AssertionError("unreachable")


def backward(params: np.ndarray, acts: list, dy: np.ndarray, rounding: bool = True) -> np.ndarray:
    """dL/dparams (flat, param_layout order) given dy = dL/dy and forward's activations."""
    P = unpack(params)
    L = param_layout()
    grad = np.zeros(L["_total"])
    g = _r(dy, rounding)                                   # gradient w.r.t. the current layer's output
    for li in range(len(LAYERS) - 1, -1, -1):
        name, kind, *_ = LAYERS[li]
        W, _ = P[name]
        Wr = _r(W, rounding)
        a_in = acts[li]
        w_off, shape, b_off, n = L[name]
        if kind == "conv":
            dx, dW, db = conv_backward(a_in, Wr, g)
        else:
            a2 = a_in.reshape(a_in.shape[0], -1)
            dW = a2.T @ g
            db = g.sum(axis=0)
            dx = (g @ Wr.T).reshape(a_in.shape)
        grad[w_off:w_off + dW.size] = dW.reshape(-1)
        grad[b_off:b_off + n] = db
        if li == 0:
            break
        # through the previous layer's ReLU: its stored output is > 0 exactly where it passed
        g = _r(dx, rounding) * (a_in > 0)
    return grad


def loss_and_grad(y: np.ndarray, t: np.ndarray):
    """Mean Gaussian NLL over the batch and dL/dy."""
    B = y.shape[0]
    s = y[:, 6]
    d = y[:, :6] - t
    e = np.exp(-s)
    sq = (d * d).sum(axis=1)
    L = float(np.mean(0.5 * e * sq + 3.0 * s))
    dy = np.zeros_like(y)
    dy[:, :6] = (e[:, None] * d) / B
    dy[:, 6] = (-0.5 * e * sq + 3.0) / B
    return L, dy


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Algorithm 1 of Kingma & Ba) on copies; returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------------------------- inputs and targets
def input_stack(I_A, W_A, I_B, W_B, rounding: bool = True) -> np.ndarray:
    """One network input [60, 80, 4] from the 80x60 level planes of A and B."""
    x = np.stack([np.asarray(I_A, np.float64) - 0.5, np.asarray(W_A, np.float64),
                  np.asarray(I_B, np.float64) - 0.5, np.asarray(W_B, np.float64)], axis=-1)
    return _r(x, rounding)


def twist_of(T: np.ndarray) -> np.ndarray:
    """(t, w) of the decoupled pose T = [exp([w]x), t; 0, 1]."""
    from .rgbid_oracle import so3_log
    T = np.asarray(T, dtype=np.float64)
    return np.concatenate([T[:3, 3], so3_log(T[:3, :3])])


def pose_of(twist) -> np.ndarray:
    from .rgbid_oracle import so3_exp
    tw = np.asarray(twist, dtype=np.float64)
    T = np.eye(4)
    T[:3, :3] = so3_exp(tw[3:])
    T[:3, 3] = tw[:3]
    return T
