"""Pins of the learned-proposal oracle (oracle/cnn_oracle.py) against things
other than itself: scipy's correlation, finite differences, closed forms and
the Eq. 4 identity."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.signal

from oracle import cnn_oracle as cn
import oracle


def test_kernel_side():
    assert cn.kernel_side(256) == 15
    assert cn.kernel_side(64) == 3


def test_area_matrix_closed_forms():
    A = cn.area_matrix(12, 3)                      # integer factor 4: block means
    ref = np.zeros((3, 12))
    for i in range(3):
        ref[i, 4 * i:4 * i + 4] = 0.25
    np.testing.assert_allclose(A, ref, atol=1e-15)
    B = cn.area_matrix(1096, 256)                  # fractional factor
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-12)          # constants stay constant
    np.testing.assert_allclose(B.sum(axis=0) * (1096 / 256), 1.0, atol=1e-12)  # mass conserved
    # a linear ramp maps to the interval means (closed form)
    x = np.arange(1096, dtype=np.float64)
    f = 1096 / 256
    i = np.arange(256)
    # mean of the piecewise-constant ramp over [i f, (i+1) f): integrate floor
    def integral(a):
        n = np.floor(a)
        return n * (n - 1) / 2 + n * (a - n)
    want = (integral((i + 1) * f) - integral(i * f)) / f
    np.testing.assert_allclose(B @ x, want, rtol=1e-12)


def test_conv2d_matches_scipy_and_strides():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 17, 19))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cn.conv2d(x, w, b, 1, 0)
    for o in range(4):
        ref = b[o] + sum(scipy.signal.correlate2d(x[c], w[o, c], mode="valid") for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)
    # stride s with padding p == stride-1 result on the padded input, subsampled
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    for s in (2, 4):
        ys = cn.conv2d(x, w, b, s, 1)
        full = cn.conv2d(xp, w, b, 1, 0)
        np.testing.assert_allclose(ys, full[:, ::s, ::s][:, :ys.shape[1], :ys.shape[2]], rtol=1e-12)


def _fd(f, arr, idx, h=1e-6):
    old = arr[idx]
    arr[idx] = old + h
    fp = f()
    arr[idx] = old - h
    fm = f()
    arr[idx] = old
    return (fp - fm) / (2 * h)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 9, 11))
    w = rng.normal(size=(5, 3, 3, 3))
    b = rng.normal(size=5)
    for s, p in ((1, 0), (2, 1), (4, 1)):
        y = cn.conv2d(x, w, b, s, p)
        g = rng.normal(size=y.shape)
        f = lambda: float(np.sum(g * cn.conv2d(x, w, b, s, p)))
        dx, dw, db = cn.conv2d_backward(x, w, g, s, p)
        for idx in [(0, 0, 0), (2, 4, 5), (1, 8, 10)]:
            assert abs(_fd(f, x, idx) - dx[idx]) <= 1e-7 * max(1.0, abs(dx[idx]))
        for idx in [(0, 0, 0, 0), (4, 2, 1, 2), (3, 1, 2, 0)]:
            assert abs(_fd(f, w, idx) - dw[idx]) <= 1e-7 * max(1.0, abs(dw[idx]))
        assert abs(_fd(f, b, (3,)) - db[3]) <= 1e-7 * max(1.0, abs(db[3]))


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(3)
    params = cn.init_params(7)
    for w, b in params:
        b += rng.normal(0, 0.05, b.shape)          # biases off zero so every path is active
    x = rng.uniform(0, 1, size=(2, 64, 64))
    t = cn.kernel_side(64)
    Kt = rng.uniform(size=(2, t, t))
    Kt /= Kt.sum(axis=(1, 2), keepdims=True)
    K, cache = cn.forward(params, x)
    np.testing.assert_allclose(K.sum(axis=(1, 2)), 1.0, atol=1e-14)
    grads = cn.backward(params, cache, Kt)
    f = lambda: cn.loss(cn.forward(params, x)[0], Kt)
    checked = 0
    for li, idx in [(0, (3, 1, 2, 0)), (1, (10, 5, 1, 1)), (2, (7, 30, 0, 2)), (3, (1, 4, 1, 0)),
                    (0, (5, 0, 0, 1)), (3, (0, 31, 0, 1))]:
        num = _fd(f, params[li][0], idx, h=1e-6)
        ana = grads[li][0][idx]
        if abs(ana) < 1e-12 and abs(num) < 1e-12:
            continue
        assert abs(num - ana) <= 1e-6 * max(abs(ana), 1e-9) + 1e-12, (li, idx, num, ana)
        checked += 1
    for li in range(4):
        num = _fd(f, params[li][1], (1,), h=1e-6)
        ana = grads[li][1][1]
        assert abs(num - ana) <= 1e-6 * max(abs(ana), 1e-9) + 1e-12
    assert checked >= 4


def test_softmax_invariants():
    z = np.random.default_rng(4).normal(size=225) * 10
    p = cn.softmax(z)
    assert abs(p.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(cn.softmax(z + 123.0), p, rtol=1e-13)


def test_adamw_first_step_closed_form():
    params = [[np.array([[0.5, -1.0]]), np.array([0.25])]]
    grads = [[np.array([[0.2, -3.0]]), np.array([1e-3])]]
    state = cn.adam_state(params)
    lr, wd, eps = 1e-2, 0.1, 1e-8
    before = [params[0][0].copy(), params[0][1].copy()]
    cn.adamw_step(params, grads, state, 1, lr, weight_decay=wd, eps=eps)
    for j in range(2):
        g = grads[0][j]
        want = before[j] - lr * g / (np.abs(g) + eps) - lr * wd * before[j]
        np.testing.assert_allclose(params[0][j], want, rtol=1e-12)


def test_consistency_residual_eq4():
    rng = np.random.default_rng(5)
    lat = rng.uniform(size=(2, 20, 24))
    k1 = rng.uniform(size=(3, 3))
    k2 = rng.uniform(size=(5, 5))
    k1 /= k1.sum()
    k2 /= k2.sum()
    b1 = np.stack([oracle.blur_full(c, k1) for c in lat])
    b2 = np.stack([oracle.blur_full(c, k2) for c in lat])
    grid = (28, 30)
    assert cn.consistency_residual(b1, b2, k1, k2, grid) < 1e-13
    k1p = k1.copy()
    k1p[1, 1] += 1e-3
    assert cn.consistency_residual(b1, b2, k1p, k2, grid) > 1e-5


def test_bf16_round_pins():
    """bfloat16 rounding: representable values unchanged, ties to even in both
    directions, one ulp of 2^-7 at 1, signs and powers of two, and the CPU
    library's float32 -> bfloat16 conversion on a million random values."""
    import torch
    one = 1.0
    assert cn.bf16_round(np.array([one]))[0] == one
    assert cn.bf16_round(np.array([one + 2.0 ** -7]))[0] == one + 2.0 ** -7       # representable
    assert cn.bf16_round(np.array([one + 2.0 ** -8]))[0] == one                    # tie -> even (down)
    assert cn.bf16_round(np.array([one + 3 * 2.0 ** -8]))[0] == one + 2.0 ** -6   # tie -> even (up)
    assert cn.bf16_round(np.array([one + 2.0 ** -8 + 2.0 ** -20]))[0] == one + 2.0 ** -7   # above the tie
    assert cn.bf16_round(np.array([-(one + 2.0 ** -8 + 2.0 ** -20)]))[0] == -(one + 2.0 ** -7)
    for e in (-30, -1, 0, 5, 30):
        assert cn.bf16_round(np.array([2.0 ** e]))[0] == 2.0 ** e
    x = np.random.default_rng(5).normal(0, 1, 1_000_000) * np.exp(np.random.default_rng(6).uniform(-20, 20, 1_000_000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    assert np.array_equal(cn.bf16_round(x), ref)
    # at most half an ulp (2^-8 relative) from the float32 value
    f = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(cn.bf16_round(x) - f) <= 2.0 ** -8 * np.abs(f))
