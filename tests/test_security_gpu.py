"""Multi-level security (Section 3) on the device: LSB truncation of the
private stream against the oracle (bit-exact: both take the code's integer
decision in double precision from the same element values), and the blind
deblur of a truncated pair against the oracle on the very same truncated
frames (the FP64 path's kernel tolerance, 1e-9; f32 latent 1e-4)."""
import numpy as np
import pytest
import torch

import oracle
from tests._inputs import make_batch, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("bits,drop", [(16, 0), (16, 4), (12, 7), (8, 3)])
def test_truncation_bit_exact(gpu_ctx, dtype, bits, drop):
    from paper_1203_4874_gb300 import cbp
    rng = np.random.default_rng(bits * 31 + drop)
    x = rng.uniform(-0.1, 1.1, size=(3, 37, 53))
    top = (1 << bits) - 1
    x[0, 0, :10] = (np.arange(10) + 0.5) / top          # halfway codes
    x = torch.from_numpy(x).to(dtype)
    g = cbp.cbp_truncate_lsb(gpu_ctx, x.cuda(), bits, drop)
    torch.cuda.synchronize()
    ref = oracle.truncate_lsb(x.double().numpy(), bits, drop)
    ref = torch.from_numpy(ref).to(dtype)
    assert torch.equal(g.cpu(), ref)


def test_deblur_of_a_truncated_private_stream(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_, cfg = make_batch("video_480p", [2], h=120, w=160, noise=False)
    B1 = torch.from_numpy(b1).float().cuda()
    B2 = cbp.cbp_truncate_lsb(gpu_ctx, torch.from_numpy(b2).float().cuda().contiguous(), 16, 4)
    prm = cbp.params(9, 11, path="fp64", eps=cfg.eps, flags=cbp.CBP_FLAG_KERNELS_F64)
    lat, k1, k2, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1, B2, prm)
    torch.cuda.synchronize()
    o_b1 = b1[0].astype(np.float32).astype(np.float64)
    o_b2 = oracle.truncate_lsb(b2[0].astype(np.float32).astype(np.float64), 16, 4)
    o_b2 = o_b2.astype(np.float32).astype(np.float64)
    assert np.array_equal(B2.cpu().double().numpy()[0], o_b2)
    o = oracle.deblur_pair(o_b1, o_b2, 9, 11, eps=cfg.eps)
    assert rel(k1[0].cpu().numpy(), o["k1"]) <= 1e-9 and rel(k2[0].cpu().numpy(), o["k2"]) <= 1e-9
    assert rel(lat[0].double().cpu().numpy(), o["latent"]) <= 1e-4
