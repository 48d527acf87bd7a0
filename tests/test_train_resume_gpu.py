"""Training resumed from a checkpoint ends where an uninterrupted run ends:
six steps straight against three steps, a checkpoint, a fresh state loaded
from it and three more steps (small frames, two pairs per batch).  The
batches come from the saved generator state and every kernel of a training
step is deterministic, so weights and moments agree bit for bit."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1203_4874_gb300 import train_cnn as tc

pytestmark = pytest.mark.gpu


def test_resume_matches_uninterrupted(gpu_ctx, tmp_path):
    dev = torch.device("cuda", 0)
    kw = dict(batch=2, lr0=1e-3, weight_decay=1e-4, h=120, w=200, log_every=1)
    full = tc.train(gpu_ctx, tc.new_state(5, 6, dev), dev, **kw)
    ck = tmp_path / "t.ckpt"
    part = tc.train(gpu_ctx, tc.new_state(5, 6, dev), dev, checkpoint=ck, checkpoint_every=3,
                    stop_after=3, **kw)
    assert part["step"] == 3
    resumed = tc.train(gpu_ctx, tc.load_checkpoint(ck, dev), dev, checkpoint=ck, **kw)
    assert resumed["step"] == full["step"] == 6
    for k in ("w", "m", "v"):
        assert torch.equal(resumed[k], full[k]), k
    assert np.array_equal(resumed["ksum"], full["ksum"])
    assert [e["loss"] for e in resumed["log"]] == [e["loss"] for e in full["log"]]
    assert not torch.equal(full["w"], tc.new_state(5, 6, dev)["w"])   # training moved the weights
    # the final checkpoint holds the finished state
    last = tc.load_checkpoint(ck, dev)
    assert last["step"] == 6 and torch.equal(last["w"], full["w"])
