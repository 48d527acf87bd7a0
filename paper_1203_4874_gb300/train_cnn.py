"""Train the learned kernel proposal on the GPU.

Training pairs come from the library's own forward model (Eq. 1): a blob
latent at 1080 x 1920 (cbp_synth_latent), two 15 x 15 kernels of the
Gaussian + motion mixture family drawn on the host, full 2D convolution and
Gaussian noise with sigma drawn uniformly from [0, 2e-3] per pair
(cbp_forward_blur); the network sees both blurred frames and is trained on
the true kernels by the library's own forward/backward/AdamW kernels
(cbp_cnn_train_step).  Held-out pairs (seed 8) measure the proposal's error
against the true kernels next to two references that use no network: the
uniform kernel and the mean kernel of the training draws.

    python -m paper_1203_4874_gb300.train_cnn --pairs 200000 --out cnn_weights.bin

Checkpoints: with --checkpoint PATH the training state is written to PATH
every --checkpoint-every steps (and at the end): the weights, both AdamW
moments, the step and the schedule's length, the host generator's state, the
running sum of the training kernels and the log.  --resume continues from
PATH; since the batches are drawn from the saved generator state and the
device kernels are deterministic, a resumed run ends with the same weights,
bit for bit, as an uninterrupted one.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from pathlib import Path

import numpy as np
import torch

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

from cbp_synth.generators import _rng, blob_params, mixture_kernel  # noqa: E402
from paper_1203_4874_gb300 import cbp  # noqa: E402

H, W, T = 1080, 1920, cbp.CNN_T
SIGMA_MAX = 2e-3
CKPT_MAGIC = "cbp-cnn-train-1"


def init_weights(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    layers = ((2, 32, 3), (32, 32, 3), (32, 32, 3), (32, 2, 2))
    out = []
    for c_in, c_out, k in layers:
        out.append(rng.normal(0.0, math.sqrt(2.0 / (c_in * k * k)), c_out * c_in * k * k))
        out.append(np.zeros(c_out))
    return np.concatenate(out).astype(np.float32)


def make_batch(ctx, rng, n: int, device, seed: int, h: int = H, w: int = W):
    """n training pairs on the device: (b1, b2, true kernels [n][2][15][15])."""
    ks = np.stack([np.stack([mixture_kernel(rng, T), mixture_kernel(rng, T)]) for _ in range(n)])
    blobs = np.stack([blob_params(rng, h, w)[None] for _ in range(n)])
    sig = rng.uniform(0.0, SIGMA_MAX, size=n)
    lat = cbp.cbp_synth_latent(ctx, torch.from_numpy(blobs).to(device), n, 1, h, w, torch.float32,
                               0.05, seed)
    kt = torch.from_numpy(ks).to(device)
    b1 = torch.empty((n, 1, h + T - 1, w + T - 1), dtype=torch.float32, device=device)
    b2 = torch.empty_like(b1)
    for i in range(n):
        cbp.cbp_forward_blur(ctx, lat[i:i + 1], kt[i:i + 1, 0], float(sig[i]), 2 * (seed * n + i) + 1,
                             out=b1[i:i + 1])
        cbp.cbp_forward_blur(ctx, lat[i:i + 1], kt[i:i + 1, 1], float(sig[i]), 2 * (seed * n + i) + 2,
                             out=b2[i:i + 1])
    return b1, b2, kt.float()


def evaluate(ctx, weights, device, pairs: int, seed: int, mean_kernel: np.ndarray, batch: int = 32):
    """Mean relative L2 error of the proposals (and of the references)."""
    rng = _rng(seed)
    errs, uni, mean = [], [], []
    u = np.full((T, T), 1.0 / (T * T))
    for b0 in range(0, pairs, batch):
        n = min(batch, pairs - b0)
        b1, b2, kt = make_batch(ctx, rng, n, device, 10_000_000 + seed * 1000 + b0)
        k = cbp.cbp_cnn_forward(ctx, b1, b2, weights).double().cpu().numpy()
        t = kt.double().cpu().numpy()
        for i in range(n):
            for c in range(2):
                nt = np.linalg.norm(t[i, c])
                errs.append(np.linalg.norm(k[i, c] - t[i, c]) / nt)
                uni.append(np.linalg.norm(u - t[i, c]) / nt)
                mean.append(np.linalg.norm(mean_kernel - t[i, c]) / nt)
    return {"proposal": float(np.mean(errs)), "uniform_kernel": float(np.mean(uni)),
            "mean_kernel": float(np.mean(mean))}


def save_checkpoint(path, state: dict) -> None:
    """Write the training state (see the module docstring) to path, replacing
    it only once the new file is complete."""
    path = Path(path)
    meta = {"magic": CKPT_MAGIC, "step": state["step"], "steps": state["steps"],
            "rng": state["rng"].bit_generator.state, "log": state["log"],
            "seconds": state["seconds"], "data_seconds": state["data_seconds"]}
    tmp = path.with_name(path.name + ".tmp")
    with open(tmp, "wb") as f:
        np.savez(f, w=_host(state["w"]), m=_host(state["m"]), v=_host(state["v"]),
                 ksum=state["ksum"], meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8))
    os.replace(tmp, path)


def load_checkpoint(path, device) -> dict:
    """The training state written by save_checkpoint, tensors on device."""
    with np.load(path) as z:
        meta = json.loads(z["meta"].tobytes().decode())
        if meta.get("magic") != CKPT_MAGIC:
            raise ValueError(f"{path}: not a training checkpoint")
        rng = np.random.Generator(np.random.PCG64())
        rng.bit_generator.state = meta["rng"]
        return {"w": torch.from_numpy(z["w"].copy()).to(device), "m": torch.from_numpy(z["m"].copy()).to(device),
                "v": torch.from_numpy(z["v"].copy()).to(device), "ksum": z["ksum"].copy(),
                "step": int(meta["step"]), "steps": int(meta["steps"]), "rng": rng, "log": meta["log"],
                "seconds": float(meta["seconds"]), "data_seconds": float(meta["data_seconds"])}


def _host(t) -> np.ndarray:
    return (t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)).astype(np.float32)


def new_state(seed: int, steps: int, device) -> dict:
    P = cbp.cbp_cnn_param_count()
    return {"w": torch.from_numpy(init_weights(seed)).to(device),
            "m": torch.zeros(P, dtype=torch.float32, device=device),
            "v": torch.zeros(P, dtype=torch.float32, device=device),
            "ksum": np.zeros((T, T)), "step": 0, "steps": steps, "rng": _rng(seed), "log": [],
            "seconds": 0.0, "data_seconds": 0.0}


def train(ctx, state: dict, device, batch: int, lr0: float, weight_decay: float, h: int = H,
          w: int = W, log_every: int = 100, time_budget: float = 0.0, checkpoint=None,
          checkpoint_every: int = 0, stop_after: int = 0) -> dict:
    """Run training steps from state["step"] to state["steps"] (or stop_after
    steps of this call, if given), updating state in place."""
    loss = torch.zeros(1, dtype=torch.float32, device=device)
    t0 = time.time() - state["seconds"]
    done = 0
    while state["step"] < state["steps"] and not (stop_after and done >= stop_after):
        state["step"] += 1
        step, steps = state["step"], state["steps"]
        if step == 11 and time_budget > 0:
            per = (time.time() - t0) / 10
            state["steps"] = steps = max(step, min(steps, int(time_budget / per)))
        tg = time.time()
        b1, b2, kt = make_batch(ctx, state["rng"], batch, device, step, h, w)
        torch.cuda.synchronize()
        state["data_seconds"] += time.time() - tg
        state["ksum"] += kt.double().sum(dim=(0, 1)).cpu().numpy()
        lr = lr0 * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / steps))   # cosine decay
        cbp.cbp_cnn_train_step(ctx, b1, b2, kt, state["w"], state["m"], state["v"], step=step, lr=lr,
                               weight_decay=weight_decay, loss=loss)
        done += 1
        if step % log_every == 0 or step == steps:
            state["log"].append({"step": step, "pairs": step * batch, "loss": float(loss.item()),
                                 "lr": lr, "seconds": time.time() - t0})
            print(json.dumps(state["log"][-1]), flush=True)
        state["seconds"] = time.time() - t0
        if checkpoint and ((checkpoint_every and step % checkpoint_every == 0) or step == state["steps"]):
            torch.cuda.synchronize()
            save_checkpoint(checkpoint, state)
    torch.cuda.synchronize()
    return state


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=200_000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--weight-decay", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--eval-pairs", type=int, default=256)
    ap.add_argument("--eval-seed", type=int, default=8)
    ap.add_argument("--out", default=str(Path(__file__).with_name("cnn_weights.bin")))
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--time-budget", type=float, default=0.0,
                    help="seconds: after 10 steps, shorten the run to fit (0: no limit)")
    ap.add_argument("--checkpoint", default="", help="training-state file (written, or resumed)")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
    args = ap.parse_args()

    device = torch.device("cuda", 0)
    ctx = cbp.cbp_create(0, 0)
    if args.resume:
        state = load_checkpoint(args.checkpoint, device)
    else:
        state = new_state(args.seed, max(1, args.pairs // args.batch), device)
    state = train(ctx, state, device, args.batch, args.lr, args.weight_decay, log_every=args.log_every,
                  time_budget=args.time_budget, checkpoint=args.checkpoint or None,
                  checkpoint_every=args.checkpoint_every)
    w, steps = state["w"], state["steps"]
    w0 = torch.from_numpy(init_weights(args.seed)).to(device)
    mean_kernel = state["ksum"] / (2 * steps * args.batch)
    cbp.save_cnn_weights(args.out, w)
    ev_trained = evaluate(ctx, w, device, args.eval_pairs, args.eval_seed, mean_kernel)
    ev_init = evaluate(ctx, w0, device, args.eval_pairs, args.eval_seed, mean_kernel)
    summary = {"pairs": steps * args.batch, "batch": args.batch, "steps": steps,
               "train_seconds": state["seconds"], "data_seconds": state["data_seconds"],
               "final_loss": state["log"][-1]["loss"] if state["log"] else None,
               "heldout_rel_l2": {"trained": ev_trained, "untrained": ev_init["proposal"]},
               "out": str(args.out)}
    print(json.dumps(summary), flush=True)
    cbp.cbp_destroy(ctx)


if __name__ == "__main__":
    main()
