"""Training checkpoints on the host: a saved state loads back equal (weights,
both AdamW moments, step and schedule length, kernel sum, log), the loaded
generator continues the saved one's stream, a file of another kind is
refused, and no temporary file is left behind."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1203_4874_gb300 import train_cnn as tc


def _state():
    st = tc.new_state(7, 40, torch.device("cpu"))
    g = np.random.default_rng(3)
    st["w"] = torch.from_numpy(g.normal(size=st["w"].numel()).astype(np.float32))
    st["m"] = torch.from_numpy(g.normal(size=st["w"].numel()).astype(np.float32))
    st["v"] = torch.from_numpy(g.uniform(size=st["w"].numel()).astype(np.float32))
    st["ksum"] = g.uniform(size=(tc.T, tc.T))
    st["rng"].normal(size=17)                     # a generator part-way through its stream
    st.update(step=12, log=[{"step": 10, "pairs": 320, "loss": 0.25, "lr": 1e-3, "seconds": 1.5}],
              seconds=2.0, data_seconds=0.5)
    return st


def test_checkpoint_roundtrip(tmp_path):
    st = _state()
    p = tmp_path / "train.ckpt"
    tc.save_checkpoint(p, st)
    assert not (tmp_path / "train.ckpt.tmp").exists()
    ld = tc.load_checkpoint(p, torch.device("cpu"))
    for k in ("w", "m", "v"):
        assert torch.equal(ld[k], st[k])
    assert np.array_equal(ld["ksum"], st["ksum"])
    assert (ld["step"], ld["steps"], ld["log"]) == (st["step"], st["steps"], st["log"])
    assert ld["seconds"] == st["seconds"] and ld["data_seconds"] == st["data_seconds"]
    # the next batches are drawn from the same point of the stream
    assert np.array_equal(ld["rng"].normal(size=50), st["rng"].normal(size=50))
    assert np.array_equal(ld["rng"].integers(0, 1 << 30, size=9), st["rng"].integers(0, 1 << 30, size=9))


def test_checkpoint_overwrite_and_refusal(tmp_path):
    st = _state()
    p = tmp_path / "train.ckpt"
    tc.save_checkpoint(p, st)
    st["step"] = 13
    tc.save_checkpoint(p, st)                     # replaced in place
    assert tc.load_checkpoint(p, torch.device("cpu"))["step"] == 13
    bad = tmp_path / "other.npz"
    with open(bad, "wb") as f:
        np.savez(f, w=np.zeros(3, np.float32), meta=np.frombuffer(b'{"magic": "x"}', dtype=np.uint8))
    with pytest.raises(ValueError):
        tc.load_checkpoint(bad, torch.device("cpu"))
