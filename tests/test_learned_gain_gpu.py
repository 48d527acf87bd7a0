"""What the trained proposal network gains, measured honestly on held-out
pairs of its training distribution (1080p blob latents, 15 x 15 mixture
kernels, noise sigma U[0, 2e-3], seed 8): its kernels against the true ones,
next to the untrained network and the uniform kernel (no network at all) and
next to the method without it (the GCD solve); and the gate on full
learned-path calls -- a proposal is taken only where its consistency residual
passes, else the result is the GCD solve's."""
from __future__ import annotations

from pathlib import Path

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

WEIGHTS = Path(__file__).resolve().parents[1] / "paper_1203_4874_gb300" / "cnn_weights.bin"


def _load(path):
    raw = path.read_bytes()
    assert raw[:8] == b"CBPCNN1\0"
    side, count = np.frombuffer(raw[8:16], dtype="<i4")
    return np.frombuffer(raw[16:], dtype="<f4", count=count).copy()


def test_trained_proposal_beats_references(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    from paper_1203_4874_gb300.train_cnn import evaluate, init_weights
    dev = torch.device("cuda", 0)
    trained = torch.from_numpy(_load(WEIGHTS)).to(dev)
    untrained = torch.from_numpy(init_weights(7)).to(dev)
    u = np.full((15, 15), 1.0 / 225)
    ev_t = evaluate(gpu_ctx, trained, dev, 64, 8, u)
    ev_u = evaluate(gpu_ctx, untrained, dev, 64, 8, u)
    # relative L2 error of the kernels, mean over 128 held-out kernels
    assert ev_t["proposal"] <= 0.95 * ev_t["uniform_kernel"], ev_t
    assert ev_t["proposal"] <= ev_u["proposal"] - 0.03, (ev_t, ev_u)


def test_gate_on_heldout_pairs(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    from paper_1203_4874_gb300.train_cnn import make_batch
    from cbp_synth.generators import _rng
    cbp.cbp_learned_load(gpu_ctx, WEIGHTS)
    dev = torch.device("cuda", 0)
    b1, b2, kt = make_batch(gpu_ctx, _rng(8_000_001), 4, dev, 77)
    prm = cbp.params(15, 15, path="learned", eps=1e-4, accept_rho=1e-3)
    lat, k1, k2, d, _ = cbp.cbp_deblur_pair(gpu_ctx, b1, b2, prm)
    ref = cbp.cbp_deblur_pair(gpu_ctx, b1, b2, cbp.params(15, 15, path="mixed", eps=1e-4))
    torch.cuda.synchronize()
    for f in range(4):
        assert np.isfinite(d[f].rho) and d[f].rho > 0
        accepted = d[f].rho <= 1e-3
        assert d[f].used_fallback == (0 if accepted else 1)
        if not accepted:
            assert torch.equal(k1[f], ref[1][f]) and torch.equal(k2[f], ref[2][f])


def test_network_against_the_gcd_path(gpu_ctx):
    """The comparison the method itself sets, on 8 held-out pairs: the kernels
    of the learned path with every proposal taken (the network alone) and of
    the GCD solve (the mixed path), both against the truth; and the solver time
    a taken proposal saves (the per-sample and scale solves of its pair exit at
    once)."""
    from paper_1203_4874_gb300 import cbp
    from paper_1203_4874_gb300.train_cnn import make_batch
    from cbp_synth.generators import _rng
    cbp.cbp_learned_load(gpu_ctx, WEIGHTS)
    dev = torch.device("cuda", 0)
    b1, b2, kt = make_batch(gpu_ctx, _rng(8_000_002), 8, dev, 78)

    def run(path, rho):
        prm = cbp.params(15, 15, path=path, eps=1e-4, accept_rho=rho)
        cbp.cbp_deblur_pair(gpu_ctx, b1, b2, prm)          # warm-up
        torch.cuda.synchronize()
        cbp.cbp_stage_times(gpu_ctx)
        cbp.cbp_profile(gpu_ctx, True)
        _, k1, k2, d, _ = cbp.cbp_deblur_pair(gpu_ctx, b1, b2, prm)
        torch.cuda.synchronize()
        cbp.cbp_profile(gpu_ctx, False)
        st = cbp.cbp_stage_times(gpu_ctx)
        g = torch.cat([k1.flatten(1), k2.flatten(1)], 1).double()
        t = kt.flatten(1).double()
        err = ((g - t).norm(dim=1) / t.norm(dim=1)).cpu().numpy()
        return err, st, d

    e_net, st_net, d_net = run("learned", 1e30)
    e_gcd, st_gcd, _ = run("mixed", 1e-3)
    assert all(x.used_fallback == 0 for x in d_net)
    solve = lambda st: st["sample_solve"][0] + st["scale_solve"][0]
    assert solve(st_net) < 0.2 * solve(st_gcd), (solve(st_net), solve(st_gcd))
    # Measured on these pairs: the network's kernels 0.70 .. 0.87 from the truth
    # on every pair; the GCD solve 0.026 on the least noisy pair and up to ~98
    # on noise-dominated ones.  The network gains robustness (a bounded error,
    # a lower median), not accuracy on clean pairs, where the GCD solve is
    # near-exact and the gate would reject the proposal.
    assert np.all(np.isfinite(e_net)) and np.all(np.isfinite(e_gcd))
    assert e_net.max() < 1.0 and e_net.max() < e_gcd.max(), (e_net, e_gcd)
    assert np.median(e_net) < np.median(e_gcd), (e_net, e_gcd)
    assert e_gcd.min() < 0.1 * e_net.min(), (e_net, e_gcd)
