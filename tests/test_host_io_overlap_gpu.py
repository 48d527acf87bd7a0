"""Host-I/O calls with CBP_FLAG_OVERLAP_CALLS: consecutive calls on one stream
overlap (a call's input copies wait only for the previous call's chunk to be
done with its buffers), and every call's results are bit for bit those of the
same call made alone.  Four calls, two input batches alternating, 24 pairs
each (three chunks), enqueued back to back without synchronising."""
from __future__ import annotations

import pytest
import torch

from tests._inputs import make_batch

pytestmark = pytest.mark.gpu


def test_overlapped_calls_match_calls_alone(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1, k2, _, cfg = make_batch("video_480p", [0, 1])
    B1 = torch.from_numpy(b1).float()
    B2 = torch.from_numpy(b2).float()
    orders = [[i % 2 for i in range(24)], [(i + 1) % 2 for i in range(24)]]
    ins = [(B1[o].contiguous().pin_memory(), B2[o].contiguous().pin_memory()) for o in orders]
    t1, t2 = k1.shape[-1], k2.shape[-1]
    n, c, h, w = ins[0][0].shape
    hh, ww = h - t1 + 1, w - t1 + 1

    def outs():
        return (torch.empty((n, c, hh, ww)).pin_memory(), torch.empty((n, t1, t1)).pin_memory(),
                torch.empty((n, t2, t2)).pin_memory())

    def call(x, o, flags):
        prm = cbp.params(t1, t2, path="mixed", eps=cfg.eps, flags=flags)
        cbp.cbp_deblur_pair(gpu_ctx, x[0], x[1], prm, k1=o[1], k2=o[2], latent=o[0], diag=False)

    plain = cbp.CBP_FLAG_HOST_IO
    ref = []
    for x in ins:
        o = outs()
        call(x, o, plain)
        torch.cuda.synchronize()
        ref.append(o)
    got = [outs() for _ in range(4)]
    for k in range(4):   # back to back: the second to fourth calls overlap their predecessors
        call(ins[k % 2], got[k], plain | cbp.CBP_FLAG_OVERLAP_CALLS)
    torch.cuda.synchronize()
    for k in range(4):
        for a, b in zip(got[k], ref[k % 2]):
            assert torch.equal(a, b), k
