"""A chunked call's results do not depend on what ran before it on the same
context.  Calls that lay the context's workspace out differently (an
un-chunked batch, a kernel-size scan, another chunk count) run between two
identical chunked deblur calls; the outputs stay equal bit for bit.  The FFT
twiddle tables that a chunked call leaves in the workspace are reused only
while the layout is unchanged, and rebuilt otherwise."""
from __future__ import annotations

import pytest
import torch

from tests._inputs import make_batch

pytestmark = pytest.mark.gpu


def test_chunked_calls_unchanged_by_other_layouts(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_, cfg = make_batch("rgb_1080p", [0, 1])
    idx = [i % 2 for i in range(24)]
    B1 = torch.from_numpy(b1).float().cuda()[idx].contiguous()
    B2 = torch.from_numpy(b2).float().cuda()[idx].contiguous()
    prm = cbp.params(15, 17, path="mixed", eps=cfg.eps)

    def run(n=24):
        L, K1, K2, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1[:n], B2[:n], prm, diag=False)
        torch.cuda.synchronize()
        return L.clone(), K1.clone(), K2.clone()

    ref = run()
    again = run()                      # the same layout: the kept tables are used
    for x, y in zip(ref, again):
        assert torch.equal(x, y)
    run(3)                             # one chunk: another layout
    cbp.cbp_estimate_size(gpu_ctx, B1[:2], B2[:2])
    part = run(16)                     # two chunks
    after = run()
    for x, y in zip(ref, after):
        assert torch.equal(x, y)
    for x, y in zip(ref, part):        # and the two-chunk call's pairs agree too
        assert torch.equal(x[:16], y)
