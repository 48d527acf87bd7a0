"""Learned path (proposal + consistency gate + fallback) through the C ABI:
the gate's rho against the oracle's residual of the same proposals, and the
two outcomes -- every pair rejected is the mixed path exactly, every pair
accepted is the proposal (and its deconvolution) exactly, a mix is each."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.signal
import torch

from cbp_synth.generators import _rng, blob_latent, draw_kernel_pair, gaussian_noise
from oracle import cnn_oracle as cn

pytestmark = pytest.mark.gpu

T = 15


def _pairs(n, h, w, sigma, seed):
    b1s, b2s = [], []
    for f in range(n):
        rng = _rng(seed + f)
        lat = blob_latent(rng, h, w, channels=3)
        k1, k2 = draw_kernel_pair(rng, T, T, T, "mixture")
        b1 = np.stack([scipy.signal.fftconvolve(c, k1) for c in lat])
        b2 = np.stack([scipy.signal.fftconvolve(c, k2) for c in lat])
        b1 = b1 + gaussian_noise(rng, b1.shape, sigma)
        b2 = b2 + gaussian_noise(rng, b2.shape, sigma)
        b1s.append(b1)
        b2s.append(b2)
    dev = torch.device("cuda", 0)
    return (torch.tensor(np.stack(b1s), dtype=torch.float32, device=dev),
            torch.tensor(np.stack(b2s), dtype=torch.float32, device=dev))


@pytest.fixture(scope="module")
def learned(gpu_ctx, tmp_path_factory):
    from paper_1203_4874_gb300 import cbp
    from paper_1203_4874_gb300.train_cnn import init_weights
    w = init_weights(21)
    p = tmp_path_factory.mktemp("w") / "w.bin"
    cbp.save_cnn_weights(p, w)
    cbp.cbp_learned_load(gpu_ctx, p)
    b1, b2 = _pairs(3, 120, 150, 1e-3, 4321)
    return dict(w=torch.from_numpy(w).cuda(), b1=b1, b2=b2)


def _run(cbp, ctx, b1, b2, path, accept_rho=1e-3, flags=0, k1=None, k2=None):
    prm = cbp.params(T, T, path=path, eps=1e-4, accept_rho=accept_rho, flags=flags)
    lat, k1, k2, d, st = cbp.cbp_deblur_pair(ctx, b1, b2, prm, k1=k1, k2=k2)
    torch.cuda.synchronize()
    return lat, k1, k2, list(d)


def test_gate_rho_matches_oracle(gpu_ctx, learned):
    from paper_1203_4874_gb300 import cbp
    b1, b2 = learned["b1"], learned["b2"]
    _, _, _, d = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=0.0)
    K = cbp.cbp_cnn_forward(gpu_ctx, b1, b2, learned["w"]).double().cpu().numpy()
    for f in range(b1.shape[0]):
        grid = (d[f].pad_h, d[f].pad_w)
        want = cn.consistency_residual(b1[f].double().cpu().numpy(), b2[f].double().cpu().numpy(),
                                       K[f, 0], K[f, 1], grid)
        assert abs(d[f].rho - want) <= 1e-4 * want, (d[f].rho, want)
        assert d[f].used_fallback == 1


def test_all_rejected_is_the_mixed_path(gpu_ctx, learned):
    from paper_1203_4874_gb300 import cbp
    b1, b2 = learned["b1"], learned["b2"]
    a = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=0.0)
    m = _run(cbp, gpu_ctx, b1, b2, "mixed")
    for x, y in zip(a[:3], m[:3]):
        assert torch.equal(x, y)


def test_all_accepted_is_the_proposal(gpu_ctx, learned):
    from paper_1203_4874_gb300 import cbp
    b1, b2 = learned["b1"], learned["b2"]
    lat, k1, k2, d = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=1e30)
    K = cbp.cbp_cnn_forward(gpu_ctx, b1, b2, learned["w"])
    torch.cuda.synchronize()
    assert torch.equal(k1, K[:, 0].contiguous()) and torch.equal(k2, K[:, 1].contiguous())
    assert all(x.used_fallback == 0 for x in d)
    ref = _run(cbp, gpu_ctx, b1, b2, "mixed", flags=cbp.CBP_FLAG_KERNELS_IN,
               k1=K[:, 0].contiguous(), k2=K[:, 1].contiguous())
    assert torch.equal(lat, ref[0])


def test_mixed_outcomes_per_pair(gpu_ctx, learned):
    from paper_1203_4874_gb300 import cbp
    b1, b2 = learned["b1"], learned["b2"]
    _, _, _, d = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=0.0)
    rhos = sorted(x.rho for x in d)
    thr = 0.5 * (rhos[0] + rhos[1])
    lat, k1, k2, dd = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=thr)
    acc = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=1e30)
    rej = _run(cbp, gpu_ctx, b1, b2, "learned", accept_rho=0.0)
    n_acc = 0
    for f in range(b1.shape[0]):
        src = acc if d[f].rho <= thr else rej
        n_acc += d[f].rho <= thr
        assert dd[f].used_fallback == (0 if d[f].rho <= thr else 1)
        assert torch.equal(k1[f], src[1][f]) and torch.equal(k2[f], src[2][f])
        assert torch.equal(lat[f], src[0][f])
    assert n_acc == 1


def test_learned_path_preconditions(built_lib):
    from paper_1203_4874_gb300 import cbp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    b1, b2 = _pairs(1, 40, 50, 0.0, 99)
    ctx = cbp.cbp_create(0, 0)
    try:
        prm = cbp.params(T, T, path="learned")
        lat, k1, k2, d, st = None, None, None, None, None
        with pytest.raises(cbp.CbpError) as e:          # no weights loaded
            cbp.cbp_deblur_pair(ctx, b1, b2, prm)
        assert e.value.status == cbp.CBP_ERR_INVALID_ARG
        with pytest.raises(cbp.CbpError) as e:          # the network proposes 15 x 15 kernels only
            cbp.cbp_workspace_size(b1, b2[..., :-2, :-2], cbp.params(T, T - 2, path="learned"))
        assert e.value.status == cbp.CBP_ERR_UNSUPPORTED
    finally:
        cbp.cbp_destroy(ctx)
