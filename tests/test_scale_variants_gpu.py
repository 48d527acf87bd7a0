"""The scale-fix variants on the device against the oracle on the same
frames: the paper's k1-only pipeline (kernel 1's scale equations, B1 / K1,
Section 4) and the single-pass support-constrained fix (M > t).  Tolerances
as for the main path: FP64 kernels 1e-9, f64 latents 1e-9, f32 latents 1e-4,
mixed-path kernels 1e-3."""
import numpy as np
import pytest
import torch

import oracle
from tests._inputs import make_batch, rel

pytestmark = pytest.mark.gpu


def _run(ctx, b1, b2, t1, t2, path, eps, flags, m, dtype=torch.float64):
    from paper_1203_4874_gb300 import cbp
    B1 = torch.from_numpy(np.ascontiguousarray(b1)).to(dtype).cuda()
    B2 = torch.from_numpy(np.ascontiguousarray(b2)).to(dtype).cuda()
    n = B1.shape[0]
    K2 = torch.full((n, t2, t2), float("nan"), dtype=torch.float64, device="cuda")
    prm = cbp.params(t1, t2, m=m, path=path, eps=eps, flags=flags | cbp.CBP_FLAG_KERNELS_F64)
    lat, k1, k2, diag, _ = cbp.cbp_deblur_pair(ctx, B1, B2, prm, k2=K2)
    torch.cuda.synchronize()
    return lat.double().cpu().numpy(), k1.cpu().numpy(), k2.cpu().numpy(), diag


def test_k1_only_pipeline_64(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1, k2, lat, cfg = make_batch("single_64", [0], fast=False)
    g_lat, g_k1, g_k2, diag = _run(gpu_ctx, b1, b2, 5, 5, "fp64", 0.0, cbp.CBP_FLAG_K1_ONLY, 0)
    o = oracle.deblur_pair(b1[0], b2[0], 5, 5, eps=0.0, scale="k1")
    assert rel(g_k1[0], o["k1"]) <= 1e-9 and rel(g_k1[0], k1[0]) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-9
    assert np.all(np.isnan(g_k2))                 # kernel 2 is not written
    assert diag[0].status == 0


def test_support_scale_fix_64(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1, k2, lat, cfg = make_batch("single_64", [0], fast=False)
    g_lat, g_k1, g_k2, diag = _run(gpu_ctx, b1, b2, 5, 5, "fp64", 0.0, cbp.CBP_FLAG_SCALE_SUPPORT, 7)
    o = oracle.deblur_pair(b1[0], b2[0], 5, 5, m=7, eps=0.0, scale="support")
    assert rel(g_k1[0], o["k1"]) <= 1e-9 and rel(g_k2[0], o["k2"]) <= 1e-9
    assert rel(g_k1[0], k1[0]) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-9


@pytest.mark.parametrize("path,tol", [("fp64", 1e-9), ("mixed", 1e-3)])
def test_support_scale_fix_480p(gpu_ctx, path, tol):
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_, cfg = make_batch("video_480p", [3])
    g_lat, g_k1, g_k2, _ = _run(gpu_ctx, b1, b2, 9, 11, path, cfg.eps, cbp.CBP_FLAG_SCALE_SUPPORT, 13,
                                torch.float32)
    o = oracle.deblur_pair(b1[0], b2[0], 9, 11, m=13, eps=cfg.eps, scale="support")
    assert rel(g_k1[0], o["k1"]) <= tol and rel(g_k2[0], o["k2"]) <= tol
    if path == "fp64":
        assert rel(g_lat[0], o["latent"]) <= 1e-4


def test_k1_only_pipeline_480p(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_, cfg = make_batch("video_480p", [4])
    g_lat, g_k1, _, _ = _run(gpu_ctx, b1, b2, 9, 11, "fp64", cfg.eps, cbp.CBP_FLAG_K1_ONLY, 0,
                             torch.float32)
    o = oracle.deblur_pair(b1[0], b2[0], 9, 11, eps=cfg.eps, scale="k1")
    assert rel(g_k1[0], o["k1"]) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-4
