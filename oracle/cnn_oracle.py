"""FP64 CPU oracle of the learned kernel proposal (TEST INFRASTRUCTURE).

The paper (Sections 4-5) recovers the kernels only by the GCD solve; the
proposal network is an addition whose shape is a reading: both blurred frames'
luma (channel mean), area-downsampled to S x S, then

    conv 3x3 stride 2 pad 1 (2 -> 32), ReLU
    conv 3x3 stride 2 pad 1 (32 -> 32), ReLU
    conv 3x3 stride 4 pad 1 (32 -> 32), ReLU
    conv 2x2 stride 1 pad 0 (32 -> 2)
    softmax over each output channel's (S/16 - 1)^2 logits -> K1, K2

so S = 256 gives two 15 x 15 kernels.  Training loss: mean squared error of
both kernels against the true ones; optimiser AdamW.  Everything here is plain
numpy in float64, written for checking by eye: direct sums, explicit
backward passes, no blocking or fusion.  Pinned in tests/test_cnn_pins.py by
finite differences, library correlation and closed forms.
"""
from __future__ import annotations

import numpy as np

LAYERS = (  # (c_in, c_out, k, stride, pad, relu)
    (2, 32, 3, 2, 1, True),
    (32, 32, 3, 2, 1, True),
    (32, 32, 3, 4, 1, True),
    (32, 2, 2, 1, 0, False),
)


def out_size(n: int, k: int, stride: int, pad: int) -> int:
    return (n + 2 * pad - k) // stride + 1


def kernel_side(S: int) -> int:
    """Side of the proposed kernels for an S x S input."""
    n = S
    for _, _, k, s, p, _ in LAYERS:
        n = out_size(n, k, s, p)
    return n


def area_matrix(n_in: int, n_out: int) -> np.ndarray:
    """(n_out, n_in) weights of area resampling: output cell i covers the input
    interval [i f, (i + 1) f), f = n_in / n_out, and averages the input over it
    (each input sample is a unit cell; partial overlaps weigh by length)."""
    f = n_in / n_out
    A = np.zeros((n_out, n_in))
    for i in range(n_out):
        a, b = i * f, (i + 1) * f
        for r in range(int(np.floor(a)), min(n_in, int(np.ceil(b)))):
            A[i, r] = (min(b, r + 1) - max(a, r)) / f
    return A


def network_input(b1: np.ndarray, b2: np.ndarray, S: int) -> np.ndarray:
    """(2, S, S): luma (channel mean) of each blurred frame, area-downsampled.
    b1, b2: (C, H_k, W_k) arrays."""
    out = []
    for b in (b1, b2):
        y = np.asarray(b, dtype=np.float64).mean(axis=0)
        out.append(area_matrix(y.shape[0], S) @ y @ area_matrix(y.shape[1], S).T)
    return np.stack(out)


def conv2d(x: np.ndarray, w: np.ndarray, bias: np.ndarray, stride: int, pad: int) -> np.ndarray:
    """Cross-correlation y[o, i, j] = bias[o] + sum_{c, u, v} w[o, c, u, v]
    x[c, i s - p + u, j s - p + v] (zero outside x)."""
    c_in, H, W = x.shape
    c_out, _, k, _ = w.shape
    Ho, Wo = out_size(H, k, stride, pad), out_size(W, k, stride, pad)
    xp = np.zeros((c_in, H + 2 * pad, W + 2 * pad))
    xp[:, pad:pad + H, pad:pad + W] = x
    y = np.zeros((c_out, Ho, Wo))
    for o in range(c_out):
        y[o] += bias[o]
        for c in range(c_in):
            for u in range(k):
                for v in range(k):
                    y[o] += w[o, c, u, v] * xp[c, u:u + stride * (Ho - 1) + 1:stride,
                                               v:v + stride * (Wo - 1) + 1:stride]
    return y


def conv2d_backward(x, w, dy, stride, pad):
    """Gradients (dx, dw, dbias) of conv2d for the upstream gradient dy."""
    c_in, H, W = x.shape
    c_out, _, k, _ = w.shape
    Ho, Wo = dy.shape[1:]
    xp = np.zeros((c_in, H + 2 * pad, W + 2 * pad))
    xp[:, pad:pad + H, pad:pad + W] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for o in range(c_out):
        for c in range(c_in):
            for u in range(k):
                for v in range(k):
                    sl = (c, slice(u, u + stride * (Ho - 1) + 1, stride),
                          slice(v, v + stride * (Wo - 1) + 1, stride))
                    dw[o, c, u, v] = np.sum(dy[o] * xp[sl])
                    dxp[sl] += w[o, c, u, v] * dy[o]
    db = dy.sum(axis=(1, 2))
    return dxp[:, pad:pad + H, pad:pad + W], dw, db


def bf16_round(x: np.ndarray) -> np.ndarray:
    """The values rounded first to float32, then to bfloat16 (8 significant
    bits, round to nearest, ties to even), returned as float64: the weights as
    the tensor-core products see them.  On the float32 bit pattern: add
    0x7FFF plus the lowest kept bit, clear the low 16 bits (finite inputs)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def softmax(z: np.ndarray) -> np.ndarray:
    e = np.exp(z - z.max())
    return e / e.sum()


def init_params(seed: int) -> list:
    """He-normal weights, zero biases, from a seeded generator."""
    rng = np.random.default_rng(seed)
    params = []
    for c_in, c_out, k, _, _, _ in LAYERS:
        std = np.sqrt(2.0 / (c_in * k * k))
        params.append([rng.normal(0.0, std, (c_out, c_in, k, k)), np.zeros(c_out)])
    return params


def forward(params, x: np.ndarray):
    """x: (2, S, S).  Returns (K (2, t, t), cache)."""
    acts = [x]
    pre = []
    h = x
    for (w, b), (_, _, _, s, p, relu) in zip(params, LAYERS):
        z = conv2d(h, w, b, s, p)
        pre.append(z)
        h = np.maximum(z, 0.0) if relu else z
        acts.append(h)
    t = h.shape[1]
    K = np.stack([softmax(h[c].ravel()).reshape(t, t) for c in range(2)])
    return K, (acts, pre, K)


def loss(K: np.ndarray, K_true: np.ndarray) -> float:
    """Mean squared error over both kernels' entries."""
    return float(np.mean((K - K_true) ** 2))


def backward(params, cache, K_true: np.ndarray):
    """Gradients of loss(forward(params, x), K_true) with respect to params."""
    acts, pre, K = cache
    g = 2.0 * (K - K_true) / K.size                  # dL/dK
    dz = np.stack([K[c] * (g[c] - np.sum(g[c] * K[c])) for c in range(2)])  # softmax backward
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, _ = params[li]
        _, _, _, s, p, relu = LAYERS[li]
        if relu:
            dz = dz * (pre[li] > 0)
        dx, dw, db = conv2d_backward(acts[li], w, dz, s, p)
        grads[li] = [dw, db]
        dz = dx
    return grads


def adamw_step(params, grads, state, step: int, lr: float, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-8, weight_decay: float = 1e-4):
    """Decoupled weight decay Adam (Loshchilov & Hutter): for each tensor,
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) - lr wd p.
    `step` counts from 1; state is a list like params of (m, v) pairs."""
    for li, (pw, gw) in enumerate(zip(params, grads)):
        for j in range(2):
            m, v = state[li][j]
            m[...] = beta1 * m + (1 - beta1) * gw[j]
            v[...] = beta2 * v + (1 - beta2) * gw[j] ** 2
            mh = m / (1 - beta1 ** step)
            vh = v / (1 - beta2 ** step)
            pw[j] -= lr * mh / (np.sqrt(vh) + eps) + lr * weight_decay * pw[j]


def adam_state(params) -> list:
    return [[(np.zeros_like(w), np.zeros_like(w)), (np.zeros_like(b), np.zeros_like(b))]
            for w, b in params]


def consistency_residual(b1: np.ndarray, b2: np.ndarray, k1: np.ndarray, k2: np.ndarray,
                         grid=None) -> float:
    """rho = ||B1 * K2 - B2 * K1|| / ||B1||, circular convolutions on the
    Ph x Pw deconvolution grid (each frame and kernel zero-padded there), the
    norms summed over channels.  Eq. 4 makes rho vanish for exact kernels of
    a noise-free pair; with wrap-around on both sides the identity still holds
    because circular convolution on a common grid is linear and commutative."""
    C = b1.shape[0]
    Ph, Pw = grid
    K1 = np.fft.fft2(k1, (Ph, Pw))
    K2 = np.fft.fft2(k2, (Ph, Pw))
    num = den = 0.0
    for c in range(C):
        B1 = np.fft.fft2(b1[c], (Ph, Pw))
        B2 = np.fft.fft2(b2[c], (Ph, Pw))
        r = np.fft.ifft2(B1 * K2 - B2 * K1).real
        num += float(np.sum(r * r))
        den += float(np.sum(np.asarray(b1[c], dtype=np.float64) ** 2))
    return float(np.sqrt(num / den))
