"""Learned proposal kernels against the FP64 oracle.  The forward
convolutions run on the tensor cores with BF16 activations and the weights
rounded to BF16 (FP32 accumulation); the oracle takes the same rounded
weights (round to nearest even, oracle.cnn_oracle.bf16_round), so each
layer computed from the GPU's own previous activation differs from it only
by that layer's accumulation order and output rounding.  Also: the whole
forward pass, the loss gradient through the oracle's backward pass, the
AdamW update, and determinism.  The backward products run on the tensor
cores too, with the gradients and the weights rounded to BF16; the bias
gradients sum the unrounded gradients in FP32."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import cnn_oracle as cn
from tests._inputs import make_batch

pytestmark = pytest.mark.gpu


def _flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def _bf16(params):
    """The weights as the tensor-core products see them: each float32 weight
    rounded to BF16 by the oracle's rounding (biases stay float32)."""
    return [[cn.bf16_round(w), b.copy()] for w, b in params]


def _unflat(vec):
    out, o = [], 0
    for c_in, c_out, k, _, _, _ in cn.LAYERS:
        nw = c_out * c_in * k * k
        out.append([vec[o:o + nw].reshape(c_out, c_in, k, k).astype(np.float64),
                    vec[o + nw:o + nw + c_out].astype(np.float64)])
        o += nw + c_out
    return out


@pytest.fixture(scope="module")
def case(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1, k2, _, cfg = make_batch("video_480p", [0, 1], h=300, w=420, fast=True)
    dev = torch.device("cuda", 0)
    t1 = torch.tensor(b1, dtype=torch.float32, device=dev)
    t2 = torch.tensor(b2, dtype=torch.float32, device=dev)
    params = cn.init_params(11)
    rng = np.random.default_rng(12)
    for w, b in params:
        b += rng.normal(0, 0.05, b.shape)
    w = torch.tensor(_flat(params), dtype=torch.float32, device=dev)
    assert w.numel() == cbp.cbp_cnn_param_count()
    kt = rng.uniform(size=(2, 2, 15, 15))
    kt /= kt.sum(axis=(2, 3), keepdims=True)
    return dict(b1=b1.astype(np.float32).astype(np.float64), b2=b2.astype(np.float32).astype(np.float64),
                t1=t1, t2=t2, params=_unflat(w.cpu().numpy()), w=w, kt=kt,
                ktt=torch.tensor(kt, dtype=torch.float32, device=dev))


def test_layers_against_oracle(gpu_ctx, case):
    from paper_1203_4874_gb300 import cbp
    tr = cbp.cnn_trace_buffers(2, case["t1"].device)
    K = cbp.cbp_cnn_forward(gpu_ctx, case["t1"], case["t2"], case["w"], trace=tr)
    torch.cuda.synchronize()
    P = _bf16(case["params"])
    for f in range(2):
        # network input: area-downsampled luma; bfloat16 storage (8 bits of mantissa)
        x_ref = cn.network_input(case["b1"][f], case["b2"][f], 256)
        x = tr["input"][f].double().cpu().numpy()
        assert np.max(np.abs(x - x_ref)) <= 2 ** -8 * np.max(np.abs(x_ref)) + 1e-6
        # each layer from the GPU's previous activation
        prev = x
        for li in range(3):
            c_in, c_out, k, s, p, relu = cn.LAYERS[li]
            ref = np.maximum(cn.conv2d(prev, P[li][0], P[li][1], s, p), 0.0)
            got = tr["act"][li][f].double().cpu().numpy()
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(got - ref)) <= 2 ** -8 * scale + 1e-4 * scale, li
            prev = got
        _, _, k, s, p, _ = cn.LAYERS[3]
        z_ref = cn.conv2d(prev, P[3][0], P[3][1], s, p)
        z = tr["logits"][f].double().cpu().numpy()
        np.testing.assert_allclose(z, z_ref, rtol=1e-4, atol=1e-5 * np.max(np.abs(z_ref)))
        # softmax of the GPU logits
        for c in range(2):
            want = cn.softmax(z[c].ravel()).reshape(15, 15)
            np.testing.assert_allclose(K[f, c].double().cpu().numpy(), want, rtol=1e-5, atol=1e-8)
        # whole forward pass in FP64 with the rounded weights: the GPU differs by
        # its BF16 storage of activations
        K_ref, _ = cn.forward(P, x_ref)
        err = np.linalg.norm(K[f].double().cpu().numpy() - K_ref) / np.linalg.norm(K_ref)
        assert err < 2e-2, err


def test_gradient_and_adamw_against_oracle(gpu_ctx, case):
    from paper_1203_4874_gb300 import cbp
    dev = case["t1"].device
    P_count = cbp.cbp_cnn_param_count()
    w = case["w"].clone()
    m = torch.zeros(P_count, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    tr = cbp.cnn_trace_buffers(2, dev, grad=True)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    cbp.cbp_cnn_train_step(gpu_ctx, case["t1"], case["t2"], case["ktt"], w, m, v, step=1, lr=1e-3,
                           weight_decay=1e-2, loss=loss, trace=tr)
    torch.cuda.synchronize()
    P = case["params"]
    # oracle backward through the GPU's own activations (BF16 values as FP64)
    grads_ref = None
    losses = []
    for f in range(2):
        acts = [tr["input"][f].double().cpu().numpy()] + [a[f].double().cpu().numpy()
                                                         for a in tr["act"]]
        z = tr["logits"][f].double().cpu().numpy()
        Kf = np.stack([cn.softmax(z[c].ravel()).reshape(15, 15) for c in range(2)])
        acts.append(z)
        pre = acts[1:]                            # only signs of ReLU inputs are used
        g = cn.backward(P, (acts, pre, Kf), case["kt"][f])
        losses.append(cn.loss(Kf, case["kt"][f]))
        g = [[gw / 2.0, gb / 2.0] for gw, gb in g]  # batch mean over the two pairs
        grads_ref = g if grads_ref is None else [[a[0] + b[0], a[1] + b[1]] for a, b in zip(grads_ref, g)]
    assert abs(loss.item() - np.mean(losses)) <= 1e-5 * np.mean(losses)
    got = _unflat(tr["grad"].cpu().numpy())
    for li in range(4):
        for j in range(2):
            ref = grads_ref[li][j]
            # the last bias gradient is zero exactly (softmax is shift-invariant):
            # measure it against the layer's weight gradient
            scale = max(np.linalg.norm(ref), 1e-3 * np.linalg.norm(grads_ref[li][0]))
            rel = np.linalg.norm(got[li][j] - ref) / scale
            # each BF16 operand rounding is a relative error below 2^-9; the
            # first layer's gradient is at most seven roundings (three input-
            # gradient products with their gradient and weight operands, and
            # its own gradient operand) from the oracle's
            assert rel < 7 * 2.0 ** -9, (li, j, rel)
    # AdamW with the GPU gradient, in FP64
    state = cn.adam_state(P)
    P2 = [[a.copy(), b.copy()] for a, b in P]
    cn.adamw_step(P2, got, state, 1, 1e-3, weight_decay=1e-2)
    np.testing.assert_allclose(w.cpu().numpy(), _flat(P2), rtol=1e-5, atol=1e-7)


def test_train_step_deterministic(gpu_ctx, case):
    from paper_1203_4874_gb300 import cbp
    dev = case["t1"].device
    outs = []
    for _ in range(2):
        w = case["w"].clone()
        m = torch.zeros_like(w)
        v = torch.zeros_like(w)
        tr = cbp.cnn_trace_buffers(2, dev, grad=True)
        cbp.cbp_cnn_train_step(gpu_ctx, case["t1"], case["t2"], case["ktt"], w, m, v, step=1, lr=1e-3,
                               trace=tr)
        torch.cuda.synchronize()
        outs.append((w, tr["grad"]))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_weights_file_roundtrip(gpu_ctx, case, tmp_path):
    from paper_1203_4874_gb300 import cbp
    p = tmp_path / "w.bin"
    cbp.save_cnn_weights(p, case["w"])
    cbp.cbp_learned_load(gpu_ctx, p)
    a = cbp.cbp_cnn_forward(gpu_ctx, case["t1"], case["t2"], case["w"])
    b = cbp.cbp_cnn_forward(gpu_ctx, case["t1"], case["t2"], None)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTAFILE")
    with pytest.raises(cbp.CbpError):
        cbp.cbp_learned_load(gpu_ctx, bad)
