"""Runs small cases of every kernel family through the bounds-checked build
(started by tests/test_checks_gpu.py with CBP_LIBRARY=checks) and prints the
check words as one JSON line: the FP64 and mixed paths on the generic and the
1080p (in-register, fused) kernels, the learned path with its gate taking and
refusing the proposals, a training step, the size scan, the camera side and
the forward model."""
from __future__ import annotations

import json
import os
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1203_4874_gb300 import cbp  # noqa: E402
from tests._inputs import make_batch  # noqa: E402


def main():
    assert os.environ.get("CBP_LIBRARY") == "checks"
    ctx = cbp.cbp_create(0, 0)
    cbp.cbp_check_words(reset=True)
    dev = torch.device("cuda", 0)
    # generic kernels: 64 x 64 FP64 path, 480p mixed path
    for name, frames, path, t in (("single_64", [0], "fp64", (5, 5)), ("video_480p", [0, 1], "mixed", None)):
        b1, b2, k1, k2, _, cfg = make_batch(name, frames)
        t1, t2 = t or (k1.shape[-1], k2.shape[-1])
        cbp.cbp_deblur_pair(ctx, torch.from_numpy(b1).to(dev), torch.from_numpy(b2).to(dev),
                            cbp.params(t1, t2, path=path, eps=cfg.eps))
    # 1080p RGB float frames: in-register row passes, fused column pass, both paths
    b1, b2, k1, k2, _, cfg = make_batch("rgb_1080p", [0, 1])
    B1 = torch.from_numpy(b1).float().to(dev)
    B2 = torch.from_numpy(b2).float().to(dev)
    for path in ("mixed", "fp64"):
        cbp.cbp_deblur_pair(ctx, B1, B2, cbp.params(k1.shape[-1], k2.shape[-1], path=path, eps=cfg.eps))
    # learned path (15 x 15 kernels): every proposal taken, then the gate refusing them
    cbp.cbp_learned_load(ctx, ROOT / "paper_1203_4874_gb300" / "cnn_weights.bin")
    g = torch.Generator(device="cuda").manual_seed(1)
    L1 = torch.rand((2, 3, 1094, 1934), device=dev, generator=g)
    L2 = torch.rand((2, 3, 1094, 1934), device=dev, generator=g)
    for rho in (1e30, 1e-3):
        cbp.cbp_deblur_pair(ctx, L1, L2, cbp.params(15, 15, path="learned", eps=1e-4, accept_rho=rho))
    # a training step (forward and backward convolutions)
    P = cbp.cbp_cnn_param_count()
    w = torch.randn(P, device=dev, generator=g) * 0.05
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    kt = torch.rand((2, 2, 15, 15), device=dev, generator=g)
    kt /= kt.sum(dim=(2, 3), keepdim=True)
    cbp.cbp_cnn_train_step(ctx, L1[:, :1].contiguous(), L2[:, :1].contiguous(), kt, w, m, v, step=1, lr=1e-3)
    # size scan, camera side (coprime draws, forward blur, cascade)
    b1, b2, *_ = make_batch("video_480p", [0], noise=False)
    cbp.cbp_estimate_size(ctx, torch.from_numpy(b1).to(dev), torch.from_numpy(b2).to(dev), 5, 13, 1e-6)
    lat = torch.from_numpy(np.random.default_rng(2).uniform(size=(2, 3, 96, 128))).float().to(dev)
    cbp.cbp_encrypt(ctx, lat, 7, 5, seed=9, cascade=(3, 4))
    torch.cuda.synchronize()
    words = cbp.cbp_check_words()
    print(json.dumps({"words": words, "library": cbp.LIB_PATH.name}))
    cbp.cbp_destroy(ctx)


if __name__ == "__main__":
    main()
