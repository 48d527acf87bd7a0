"""The allocation-free estimation entry point against the regular one.

cbp_estimate_kernels_noalloc exists for callers that may not allocate device
memory (a memory manager owns all allocations, or a real-time path must not
fail on one); it runs in a fixed device array inside the library.  Its
kernels must equal those of cbp_estimate_kernels within the FP64 path's
tolerance (relative L2 <= 1e-9) on both estimation paths -- the same kernels
run on the same inputs, only the workspace differs -- on two calls in a row
(the second call finds the first call's data in the shared array).  This file
is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from tests._inputs import make_batch, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_noalloc_matches_regular_entry_point_twice(gpu_ctx, path):
    from paper_1203_4874_gb300 import cbp
    results = []
    for frames, name in (([0, 1], "video_480p"), ([3], "video_480p")):
        b1, b2, *_, cfg = make_batch(name, frames, h=240, w=320)
        B1 = torch.from_numpy(b1).float().cuda()
        B2 = torch.from_numpy(b2).float().cuda()
        prm = cbp.params(cfg.t1, cfg.t2, path=path, eps=cfg.eps, flags=cbp.CBP_FLAG_KERNELS_F64)
        n = len(frames)
        k1 = torch.full((n, cfg.t1, cfg.t1), float("nan"), dtype=torch.float64, device="cuda")
        k2 = torch.full((n, cfg.t2, cfg.t2), float("nan"), dtype=torch.float64, device="cuda")
        diag, status = cbp.cbp_estimate_kernels_noalloc(B1, B2, prm, k1, k2)
        r1, r2, rdiag, _ = cbp.cbp_estimate_kernels(gpu_ctx, B1, B2, prm)
        torch.cuda.synchronize()
        assert status >= 0
        for i in range(n):
            assert rel(k1[i].cpu().numpy(), r1[i].cpu().numpy()) <= 1e-9
            assert rel(k2[i].cpu().numpy(), r2[i].cpu().numpy()) <= 1e-9
            assert diag[i].status == rdiag[i].status
        results.append(k1.cpu())
    assert not torch.equal(results[0][:1], results[1][:1])


def test_noalloc_rejects_oversized_problems(built_lib):
    from paper_1203_4874_gb300 import cbp
    big = cbp.cbp_frames(0x1000, 8, 3, 1094, 1934, cbp.CBP_F32, 0, 0, 0)
    big2 = cbp.cbp_frames(0x1000, 8, 3, 1096, 1936, cbp.CBP_F32, 0, 0, 0)
    prm = cbp.params(15, 17, path="fp64")
    s = cbp.lib().cbp_estimate_kernels_noalloc(ctypes.byref(big), ctypes.byref(big2),
                                               ctypes.byref(prm), ctypes.c_void_p(0x2000),
                                               ctypes.c_void_p(0x3000), None, None)
    assert s == cbp.CBP_ERR_UNSUPPORTED


def test_noalloc_one_1080p_rgb_pair(gpu_ctx):
    """The fixed array holds one 1080p RGB pair with 15x15 / 17x17 kernels on
    the mixed path (its largest estimation workspace): same kernels as the
    regular entry point."""
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_, cfg = make_batch("rgb_1080p", [2])
    B1 = torch.from_numpy(b1).float().cuda()
    B2 = torch.from_numpy(b2).float().cuda()
    prm = cbp.params(15, 17, path="mixed", eps=cfg.eps, flags=cbp.CBP_FLAG_KERNELS_F64)
    k1 = torch.full((1, 15, 15), float("nan"), dtype=torch.float64, device="cuda")
    k2 = torch.full((1, 17, 17), float("nan"), dtype=torch.float64, device="cuda")
    diag, status = cbp.cbp_estimate_kernels_noalloc(B1, B2, prm, k1, k2)
    r1, r2, rdiag, _ = cbp.cbp_estimate_kernels(gpu_ctx, B1, B2, prm)
    torch.cuda.synchronize()
    assert status >= 0
    assert rel(k1[0].cpu().numpy(), r1[0].cpu().numpy()) <= 1e-9
    assert rel(k2[0].cpu().numpy(), r2[0].cpu().numpy()) <= 1e-9
    assert diag[0].status == rdiag[0].status
