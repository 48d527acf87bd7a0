"""Benchmark: blind deblurring throughput of coprime blurred pairs at 1080p.

Workload (rgb_1080p): batches of 60 frame pairs, 1920x1080 RGB float32 latents
(20-blob generator), kernels 15x15 and 17x17 (Gaussian + random-walk motion
mixture, unit sum), full-convolution blur plus N(0, 1e-3^2) noise; the mixed
precision path.  One step = blind kernel estimation and dual-kernel
deconvolution of one batch of 60 pairs, one cbp_deblur_pair call.  Inputs are
synthesised on the device before timing (3.0 GB per batch, larger than L2, so
no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: one process per GPU (torchrun); each rank deblurs its own batch
(weak scaling, no data-path collective -- frame pairs are independent);
the host-side barrier and max-over-ranks timing use gloo.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "deblurred frame-pairs/s at 1080p (plain vs mixed/learned, kernel rel-err≤1e-3); p99 ms"
UNIT = "frame-pairs/s"
WORKLOAD = "rgb_1080p"
H, W, C, T1, T2, SIGMA, EPS = 1080, 1920, 3, 15, 17, 1e-3, 1e-4
H1, W1, H2, W2 = H + T1 - 1, W + T1 - 1, H + T2 - 1, W + T2 - 1
PH, PW = 1120, 1944          # smallest 7-smooth sizes >= 1096, 1936
PW2 = PW // 2 + 1
M = max(T1, T2)              # unit-circle samples (the default)
NS = M // 2 + 1              # samples solved per direction


def config(pairs, arm="mixed path (CUDA)"):
    return {"workload": f"{WORKLOAD}: {pairs} pairs/step, 1920x1080x3 f32, kernels 15x15 + 17x17 "
                        f"(Gaussian+motion mixture), noise sigma 1e-3, {arm}, eps 1e-4",
            "pairs_per_step": pairs, "fft_grid": [PH, PW],
            "l2": f"inputs {pairs * C * (H1 * W1 + H2 * W2) * 4 / 1e9:.2g} GB per step"
                  + ("; larger than L2, no flush between steps" if pairs * C * (H1 * W1 + H2 * W2) * 4 > 2e8
                     else "")}


# ----------------------------------------------------------- roofline data --
def algorithmic_bytes(stage: str, n: int) -> float | None:
    """Bytes a stage must move per launch in the three-pass design (f32 frames,
    complex64 spectra), for n pairs."""
    fr = n * C * (H1 * W1 + H2 * W2) * 4
    spec = n * C * (H1 + H2) * PW2 * 8
    khat = n * 2 * PH * PW2 * 8
    ihat = n * C * H * PW2 * 8
    lat = n * C * H * W * 4
    bins = n * C * M * (H1 + H2 + W1 + W2) * 8
    samples = n * C * NS * (H1 + H2 + W1 + W2) * 16 * 2   # double + float-float copies
    return {
        "eval": bins + samples,                    # fold bins -> samples
        "row_fft": fr + spec + bins,               # one read of the frames: folds + row FFTs
        # the fused column pass of this grid computes the kernel spectra itself:
        # row spectra in, deconvolved spectrum out (khat: the unfused pass's extra)
        "col_deconv": spec + ihat,
        "row_ifft": ihat + lat,
    }.get(stage)


def algorithmic_flops(stage: str, n: int) -> float | None:
    """Floating-point operations a compute-bound stage must do per launch, for
    n pairs, counted on the method's arithmetic (a complex multiply-add = 8):
    per solved sample (M/2 + 1 per direction) the 2 (t1 + t2) - 1 Toeplitz
    correlations over the channels' samples, and ~7 sweeps of parallel Jacobi
    on the (t1 + t2)-square Hermitian normal matrix (every rotation updates
    two rows and two columns of A and two columns of V)."""
    if stage != "sample_solve":
        return None
    nn = T1 + T2
    lags = 2 * nn - 1
    corr = NS * lags * C * (H1 + W1) * 8                  # both directions
    jacobi = 2 * NS * 7 * (nn - 1) * (nn // 2) * (3 * 2 * nn) * 8
    return float(n * (corr + jacobi))


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# The sources each stage's kernels are compiled from (the file, then the
# headers its kernels' code comes from).
_COMMON = ["cbp_common.cuh", "cbp_internal.h"]
STAGE_FILES = {"eval": ["cbp_eval.cu"] + _COMMON,
               "sample_solve": ["cbp_solve.cu", "cbp_tri.cuh", "cbp_ff.cuh"] + _COMMON,
               "scale_solve": ["cbp_solve.cu", "cbp_tri.cuh", "cbp_ff.cuh"] + _COMMON,
               "kernel_spectra": ["cbp_fft.cu", "cbp_dft.cuh"] + _COMMON,
               "row_fft": ["cbp_fft.cu", "cbp_dft.cuh"] + _COMMON,
               "col_deconv": ["cbp_colpass.cu", "cbp_dft.cuh"] + _COMMON,
               "row_ifft": ["cbp_fft.cu", "cbp_dft.cuh"] + _COMMON}


def source_hash(stage: str) -> str:
    h = hashlib.sha256()
    for name in STAGE_FILES[stage]:
        h.update((ROOT / "paper_1203_4874_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def measured_traffic(stage: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since it was captured."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    rec = json.loads(p.read_text()).get(stage)
    if not rec or rec.get("source_sha256_16") != source_hash(stage):
        return None
    return rec.get("dram_bytes_per_launch")


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.out = None
        self.skip = 0

    def start(self):
        """Start sampling every 100 ms; returns once the first sample is in, so
        that the timed region that follows is covered from its start."""
        self.skip = 0
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device)], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 10.0 and self.proc.poll() is None:
            if Path(self.out.name).read_text().strip():
                break
            time.sleep(0.02)

    def mark(self):
        """Samples taken before this call (warm-up) are not counted."""
        if self.proc:
            self.skip = len([l for l in Path(self.out.name).read_text().splitlines() if l.strip()])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = [l.split(",") for l in Path(self.out.name).read_text().splitlines() if l.strip()]
        rows = rows[max(0, self.skip - 1):]   # the sample just before the region, and those in it
        os.unlink(self.out.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ multi-rank ---
SEED_BASE = 1203000


def shard_seed(rank: int, n: int) -> int:
    """First input seed of a rank: rank r deblurs the pairs seeded
    SEED_BASE + r n ... SEED_BASE + (r + 1) n - 1, so the ranks' batches are
    disjoint and each rank's work is fixed as ranks are added (weak scaling)."""
    return SEED_BASE + rank * n


def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values (gloo all-reduce); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, n: int, steps: int, ms: float) -> float:
    """Whole-job pairs/s: every rank's n pairs per step over the slowest rank's time."""
    return world * n * steps / (ms / 1e3)


# ----------------------------------------------------------------- inputs ---
def make_inputs(ctx, n: int, seed0: int, device, t1: int = T1, t2: int = T2, keep: int = 0,
                sigma: float = SIGMA, h: int = H, w: int = W, c: int = C, family: str = "mixture"):
    """Kernels and blob parameters drawn on the host (cbp_synth), latents and
    blurred frames synthesised on the device by the library's forward model.
    keep > 0: also returns the true latents of the first `keep` pairs (host)."""
    import numpy as np
    import torch
    from cbp_synth.generators import _rng, blob_params, draw_kernel_pair
    from paper_1203_4874_gb300 import cbp

    k1s, k2s, blobs = [], [], []
    for f in range(n):
        rng = _rng(seed0 + f)
        blobs.append(np.stack([blob_params(rng, h, w) for _ in range(c)]))
        a, b = draw_kernel_pair(rng, t1, t2, max(t1, t2), family)
        k1s.append(a)
        k2s.append(b)
    k1 = torch.from_numpy(np.stack(k1s)).to(device)
    k2 = torch.from_numpy(np.stack(k2s)).to(device)
    bl = torch.from_numpy(np.stack(blobs)).to(device)
    lat = cbp.cbp_synth_latent(ctx, bl, n, c, h, w, torch.float32, 0.05, seed0)
    b1 = cbp.cbp_forward_blur(ctx, lat, k1, sigma, seed0 * 2 + 1)
    b2 = cbp.cbp_forward_blur(ctx, lat, k2, sigma, seed0 * 2 + 2)
    torch.cuda.synchronize()
    truth = lat[:keep].cpu() if keep else None
    del lat
    if keep:
        return b1, b2, k1, k2, truth
    return b1, b2, k1, k2


# ------------------------------------------------------------- serving ---
SERVE_RES = [(240, 320), (480, 640), (720, 1280), (1080, 1920)]
SERVE_SIZES = [7, 9, 11, 13, 15, 17]


def serving_bench(seconds: float, device, seed: int = 5150, cameras: int = 16, rate: float = 30.0,
                  pool: int = 4, budget_gb: float = 150.0):
    """Camera workload through the serving engine: `cameras` cameras, each with
    a resolution from SERVE_RES and odd kernel sizes in 7..17 drawn once, new
    kernels per frame (a pool of `pool` synthetic pairs per camera), Poisson
    arrivals at `rate` pairs/s per camera, grayscale f32, noise sigma 1e-3.
    One second of the same traffic warms the engine (graph captures) first."""
    import threading
    import numpy as np
    import torch
    from cbp_synth.generators import _rng, blob_params, draw_kernel_pair
    from paper_1203_4874_gb300 import cbp

    ctx = cbp.cbp_create(device.index or 0, int(budget_gb * 2**30))
    rng = _rng(seed)
    cams = []
    for cam in range(cameras):
        h, w = SERVE_RES[int(rng.integers(len(SERVE_RES)))]
        t1 = SERVE_SIZES[int(rng.integers(len(SERVE_SIZES)))]
        t2 = SERVE_SIZES[int(rng.integers(len(SERVE_SIZES)))]
        pairs = []
        for f in range(pool):
            r = _rng(seed * 1000 + cam * pool + f)
            a, b = draw_kernel_pair(r, t1, t2, max(t1, t2), "mixture")
            bl = torch.from_numpy(blob_params(r, h, w)[None, None]).to(device)
            lat = cbp.cbp_synth_latent(ctx, bl, 1, 1, h, w, torch.float32, 0.05, seed + cam * pool + f)
            k1 = torch.from_numpy(a[None]).to(device)
            k2 = torch.from_numpy(b[None]).to(device)
            b1 = cbp.cbp_forward_blur(ctx, lat, k1, SIGMA, 2 * (cam * pool + f) + 1)
            b2 = cbp.cbp_forward_blur(ctx, lat, k2, SIGMA, 2 * (cam * pool + f) + 2)
            pairs.append((b1, b2))
        prm = cbp.params(t1, t2, path="mixed", eps=EPS)
        cams.append({"h": h, "w": w, "t1": t1, "t2": t2, "pairs": pairs, "prm": prm})
    torch.cuda.synchronize()

    def trace(duration, seed_arr):
        r = np.random.default_rng(seed_arr)
        ev = []
        for cam in range(cameras):
            t = r.exponential(1.0 / rate)
            while t < duration:
                ev.append((t, cam))
                t += r.exponential(1.0 / rate)
        return sorted(ev)

    def run(events):
        outq, done, lock = [], threading.Event(), threading.Lock()
        statuses = []

        def poller():
            i = 0
            while True:
                with lock:
                    item = outq[i] if i < len(outq) else None
                if item is None:
                    if done.is_set():
                        with lock:
                            if i >= len(outq):
                                return
                    time.sleep(0.0002)
                    continue
                s, _ = cbp.cbp_stream_poll(ctx, item[0], -1)
                statuses.append(s)
                with lock:
                    outq[i] = None          # the request's buffers may go
                i += 1

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        count = [0] * cameras
        for t, cam in events:
            c = cams[cam]
            b1, b2 = c["pairs"][count[cam] % pool]
            count[cam] += 1
            k1 = torch.empty((1, c["t1"], c["t1"]), dtype=torch.float32, device=device)
            k2 = torch.empty((1, c["t2"], c["t2"]), dtype=torch.float32, device=device)
            lat = torch.empty((1, 1, c["h"], c["w"]), dtype=torch.float32, device=device)
            while time.perf_counter() - t0 < t:
                pass
            tk = cbp.cbp_stream_submit(ctx, b1, b2, c["prm"], k1, k2, lat)
            with lock:
                outq.append((tk, k1, k2, lat))
        done.set()
        th.join()
        return time.perf_counter() - t0, statuses

    run(trace(1.0, seed + 1))
    cbp.cbp_stream_stats(ctx, reset=True)
    events = trace(seconds, seed + 2)
    wall, statuses = run(events)
    st = cbp.cbp_stream_stats(ctx)
    cbp.cbp_destroy(ctx)
    ok = sum(1 for s in statuses if s >= 0)
    return {"workload": f"{cameras} cameras, resolutions {SERVE_RES}, odd kernel sizes 7..17, new kernels "
                        f"per frame, Poisson {rate:g} pairs/s per camera, grayscale f32, noise sigma 1e-3, "
                        f"mixed path, budget {budget_gb:g} GB",
            "seconds": seconds, "requests": len(events), "ok": ok, "value": ok / wall,
            "unit": "frame-pairs/s", "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "cameras": [{"h": c["h"], "w": c["w"], "t1": c["t1"], "t2": c["t2"]} for c in cams]}


# ---------------------------------------------------------- learned path --
def learned_bench(ctx, n: int, device, steps: int = 3) -> dict:
    """The learned kernel proposal at 1080p (both kernels 15 x 15, the
    network's output size; RGB f32, noise sigma 1e-3): the learned path
    (network, consistency gate fused into the proposal's deconvolution,
    GCD-solve fallback for rejected pairs) at the operating threshold
    accept_rho = 1e-3 and with every proposal accepted (accept_rho = 1e30: the
    path's cost without the fallback), against the mixed path (the method
    without the network) on the same pairs, each timed over `steps` calls
    after one warm-up call; per path the median kernel error against the truth."""
    import torch
    from paper_1203_4874_gb300 import cbp

    cbp.cbp_learned_load(ctx, ROOT / "paper_1203_4874_gb300" / "cnn_weights.bin")
    b1, b2, k1t, k2t = make_inputs(ctx, n, 4_000_000, device, 15, 15)
    lat = torch.empty((n, C, H, W), dtype=torch.float32, device=device)
    k1 = torch.empty((n, 15, 15), dtype=torch.float32, device=device)
    k2 = torch.empty_like(k1)
    out = {}
    for key, path, rho_max in (("learned", "learned", 1e-3), ("learned_all_accepted", "learned", 1e30),
                               ("mixed", "mixed", 1e-3)):
        prm = cbp.params(15, 15, path=path, eps=EPS, accept_rho=rho_max)
        d = None
        for i in range(steps + 1):
            if i == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            _, _, _, d, _ = cbp.cbp_deblur_pair(ctx, b1, b2, prm, k1=k1, k2=k2, latent=lat,
                                                diag=(i == steps))
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        err = sorted(_kerr(k1, k2, k1t, k2t))
        out[key] = {"value": n / dt, "ms_per_step": 1e3 * dt,
                    "kernel_rel_err_vs_truth_median": err[len(err) // 2]}
        # per-stage times of one unsplit call (stages one after another)
        cbp.cbp_stage_times(ctx)
        cbp.cbp_profile(ctx, True)
        cbp.cbp_deblur_pair(ctx, b1, b2, prm, k1=k1, k2=k2, latent=lat, diag=False)
        torch.cuda.synchronize()
        cbp.cbp_profile(ctx, False)
        out[key]["stage_ms"] = {k: round(v[0], 4) for k, v in cbp.cbp_stage_times(ctx).items() if v[1] > 0}
        if path == "learned":
            rho = [x.rho for x in d]
            out[key]["accepted"] = sum(1 for x in d if x.used_fallback == 0)
            out[key]["rho_median"] = float(sorted(rho)[len(rho) // 2])
    return {"workload": f"{n} pairs/step, 1920x1080x3 f32, both kernels 15x15 (mixture), noise sigma 1e-3, "
                        "trained weights (200k pairs)", "unit": UNIT, **out}


# ------------------------------------------------- the paper's other rows --
def _kerr(k1, k2, k1t, k2t):
    """Per-pair relative L2 error of both kernels against the truth."""
    import torch
    g = torch.cat([k1.flatten(1).double(), k2.flatten(1).double()], 1)
    t = torch.cat([k1t.flatten(1).double(), k2t.flatten(1).double()], 1)
    return ((g - t).norm(dim=1) / t.norm(dim=1)).cpu().tolist()


def _psnr_t(x, ref):
    import torch
    mse = ((x.double() - ref.double()) ** 2).flatten(1).mean(1)
    peak = ref.double().flatten(1).abs().max(1).values
    return (10 * torch.log10(peak * peak / mse)).cpu().tolist()


def _timed(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return 1e3 * (time.perf_counter() - t0) / reps


def size_estimation_bench(ctx, device, pairs: int = 4) -> dict:
    """Kernel-size estimation (Section 4-5's degree step) on the first pairs
    of the 1080p RGB workload, noise-free and at sigma 1e-3."""
    from paper_1203_4874_gb300 import cbp
    out = []
    for sg in (0.0, SIGMA):
        b1, b2, _, _ = make_inputs(ctx, pairs, 1203000, device, sigma=sg)
        res = {}
        ms = _timed(lambda: res.update(r=cbp.cbp_estimate_size(ctx, b1, b2, 5, 21)), reps=2)
        t1, t2, found, _ = res["r"]
        out.append({"sigma": sg, "t1": t1, "t2": t2, "found": found,
                    "recovered": sum(1 for a, b in zip(t1, t2) if (a, b) == (T1, T2)), "ms_per_call": ms})
        del b1, b2
    return {"workload": f"{pairs} pairs of {WORKLOAD}, true sizes {T1}/{T2}, candidates 5..21, tol 1e-6",
            "points": out}


def multilevel_bench(ctx, device, pairs: int = 4) -> dict:
    """Multi-level security (Section 3): the private stream with its `drop`
    least significant bits (of 16) removed, deblurred on the mixed path;
    480p grayscale, kernels 9 / 11, noise-free latents."""
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1t, k2t, truth = make_inputs(ctx, pairs, 4874, device, 9, 11, keep=pairs, sigma=0.0,
                                          h=480, w=640, c=1, family="uniform")
    truth = truth.to(device)
    out = []
    for drop in (0, 2, 4, 6, 8):
        b2t = cbp.cbp_truncate_lsb(ctx, b2, 16, drop)
        b1q = cbp.cbp_truncate_lsb(ctx, b1, 16, 0)          # the public stream at full resolution
        prm = cbp.params(9, 11, path="mixed", eps=EPS, flags=cbp.CBP_FLAG_KERNELS_F64)
        lat, k1, k2, _, _ = cbp.cbp_deblur_pair(ctx, b1q, b2t, prm)
        out.append({"drop_bits": drop, "kernel_rel_err_vs_truth": _kerr(k1, k2, k1t, k2t),
                    "latent_psnr_db": _psnr_t(lat, truth)})
    return {"workload": f"{pairs} pairs, 480x640 grayscale f32, kernels 9x9 + 11x11 (U[0,1]), noise-free, "
                        "16-bit codes, private stream truncated, mixed path", "points": out}


def camera_bench(ctx, device, n: int = 60, reps: int = 3) -> dict:
    """Encryption at camera rate (Section 3): per-frame coprime kernel pairs
    drawn and tested on the device, both streams blurred; then with the
    cascaded pair.  1080p RGB f32 latents resident on the device."""
    import torch
    from paper_1203_4874_gb300 import cbp
    lat = torch.rand((n, C, H, W), dtype=torch.float32, device=device)
    res = {}
    ms = _timed(lambda: res.update(o=cbp.cbp_encrypt(ctx, lat, T1, T2, seed=1, sigma=SIGMA)), reps)
    att = res["o"]["attempts"]
    del res["o"]
    ms_c = _timed(lambda: res.update(o=cbp.cbp_encrypt(ctx, lat, T1, T2, seed=1, sigma=SIGMA, cascade=(9, 11))),
                  reps)
    del res["o"]
    return {"workload": f"{n} frames 1920x1080x3 f32 per call, kernels {T1}x{T1} + {T2}x{T2} (U[0,1], "
                        "redrawn until coprime at every sample), sigma 1e-3; cascade 9x9 + 11x11",
            "unit": "frames/s", "pair": {"value": n / (ms / 1e3), "ms_per_call": ms},
            "pair_and_cascade": {"value": n / (ms_c / 1e3), "ms_per_call": ms_c},
            "redraws": sum(1 for a in att if a > 0), "failed": sum(1 for a in att if a < 0)}


def scale_variants_bench(ctx, device, pairs: int = 8) -> dict:
    """The scale fixes compared (Sections 4-5): two-order least squares with
    both kernels (the default), the paper's k1-only pipeline, and the
    single-pass support constraint (m = 13 > 11); 480p grayscale 9 / 11."""
    from paper_1203_4874_gb300 import cbp
    out = []
    for sg in (0.0, SIGMA):
        b1, b2, k1t, k2t = make_inputs(ctx, pairs, 4874, device, 9, 11, sigma=sg, h=480, w=640, c=1,
                                       family="uniform")
        row = {"sigma": sg}
        for name, m, flags in (("least_squares", 0, 0), ("k1_only", 0, cbp.CBP_FLAG_K1_ONLY),
                               ("support", 13, cbp.CBP_FLAG_SCALE_SUPPORT)):
            prm = cbp.params(9, 11, m=m, path="fp64", eps=EPS, flags=flags | cbp.CBP_FLAG_KERNELS_F64)
            res = {}
            ms = _timed(lambda: res.update(r=cbp.cbp_estimate_kernels(ctx, b1, b2, prm)), reps=2)
            k1, k2 = res["r"][0], res["r"][1]
            e1 = ((k1.flatten(1) - k1t.flatten(1)).norm(dim=1) / k1t.flatten(1).norm(dim=1)).cpu().tolist()
            row[name] = {"k1_rel_err_vs_truth": e1, "ms_per_call": ms}
            if name != "k1_only":
                row[name]["kernel_rel_err_vs_truth"] = _kerr(k1, k2, k1t, k2t)
        out.append(row)
    return {"workload": f"{pairs} pairs, 480x640 grayscale f32, kernels 9x9 + 11x11 (U[0,1]), FP64 path",
            "points": out}


# ------------------------------------------------------- CPU oracle sample --
def _rel(a, b):
    import numpy as np
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64))
                 / np.linalg.norm(np.asarray(b, np.float64)))


def _psnr(x, ref):
    import numpy as np
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    mse = float(np.mean((x - ref) ** 2))
    return 10.0 * np.log10(float(np.max(np.abs(ref))) ** 2 / mse) if mse > 0 else float("inf")


def cpu_worker(folder: str):
    """Time the FP64 oracle on the frames the GPU deblurred (saved in `folder`
    by the parent) and state, per pair, the errors of the GPU results against
    the oracle's and of both against the truth."""
    import numpy as np
    import oracle

    d = Path(folder)
    b1, b2 = np.load(d / "b1.npy", mmap_mode="r"), np.load(d / "b2.npy", mmap_mode="r")
    k1t, k2t = np.load(d / "k1_true.npy"), np.load(d / "k2_true.npy")
    lat_t = np.load(d / "latent_true.npy", mmap_mode="r")
    gk = {p: (np.load(d / f"k1_{p}.npy"), np.load(d / f"k2_{p}.npy")) for p in ("mixed", "fp64")}
    gl = {p: np.load(d / f"latent_{p}.npy", mmap_mode="r") for p in ("mixed", "fp64")}
    total, per = 0.0, []
    for f in range(b1.shape[0]):
        x1, x2 = np.asarray(b1[f], np.float64), np.asarray(b2[f], np.float64)
        t0 = time.perf_counter()
        o = oracle.deblur_pair(x1, x2, T1, T2, eps=EPS)
        total += time.perf_counter() - t0
        ok = np.concatenate([o["k1"].ravel(), o["k2"].ravel()])
        tk = np.concatenate([k1t[f].ravel(), k2t[f].ravel()])
        rec = {"pair": f, "kernel_vs_oracle": {}, "latent_vs_oracle": {}, "kernel_vs_truth": {},
               "latent_psnr_vs_truth_db": {}}
        for p in ("mixed", "fp64"):
            g = np.concatenate([gk[p][0][f].ravel(), gk[p][1][f].ravel()])
            rec["kernel_vs_oracle"][p] = _rel(g, ok)
            rec["latent_vs_oracle"][p] = _rel(gl[p][f], o["latent"])
            rec["kernel_vs_truth"][p] = _rel(g, tk)
            rec["latent_psnr_vs_truth_db"][p] = _psnr(gl[p][f], lat_t[f])
        rec["kernel_vs_truth"]["oracle"] = _rel(ok, tk)
        rec["latent_psnr_vs_truth_db"]["oracle"] = _psnr(o["latent"], lat_t[f])
        o1 = T1 // 2   # the blur centre: B1 shifted back by half the kernel
        rec["latent_psnr_vs_truth_db"]["blurred_b1"] = _psnr(np.asarray(b1[f])[:, o1:o1 + H, o1:o1 + W],
                                                             lat_t[f])
        per.append(rec)
    print(json.dumps({"pairs": int(b1.shape[0]), "seconds": total, "per_pair": per}))


def accuracy_sample(ctx, b1, b2, k1t, k2t, truth, k: int, folder: Path):
    """Deblur the first k pairs of the batch on both paths with double-precision
    kernel outputs and save them, the frames and the truth for the oracle leg."""
    import numpy as np
    import torch
    from paper_1203_4874_gb300 import cbp

    np.save(folder / "b1.npy", b1[:k].cpu().numpy())
    np.save(folder / "b2.npy", b2[:k].cpu().numpy())
    np.save(folder / "k1_true.npy", k1t[:k].cpu().numpy())
    np.save(folder / "k2_true.npy", k2t[:k].cpu().numpy())
    np.save(folder / "latent_true.npy", truth[:k].numpy())
    for path in ("mixed", "fp64"):
        prm = cbp.params(T1, T2, path=path, eps=EPS, flags=cbp.CBP_FLAG_KERNELS_F64)
        lat, g1, g2, _, _ = cbp.cbp_deblur_pair(ctx, b1[:k].contiguous(), b2[:k].contiguous(), prm)
        torch.cuda.synchronize()
        np.save(folder / f"k1_{path}.npy", g1.cpu().numpy())
        np.save(folder / f"k2_{path}.npy", g2.cpu().numpy())
        np.save(folder / f"latent_{path}.npy", lat.cpu().numpy())
        del lat


def cpu_baseline(folder: Path):
    """The oracle on the host cores (BLAS threads = core count) in a fresh
    process, on the pairs saved in `folder`: (cpu_baseline record, accuracy)."""
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    r = subprocess.run([sys.executable, str(Path(__file__).resolve()), "--cpu-worker", str(folder)],
                       capture_output=True, text=True, env=env, timeout=1800)
    line = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not line:
        return ({"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                 "sample": "failed: " + (r.stderr.strip().splitlines() or ["?"])[-1]}, None)
    d = json.loads(line[-1])
    base = {"value": d["pairs"] / d["seconds"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the first {d['pairs']} pairs of the GPU's own batch (device-synthesised "
                      f"{WORKLOAD} frames copied to the host), FP64 numpy oracle, estimation + "
                      f"deconvolution, BLAS threads = {cores}"}
    per = d["per_pair"]
    worst = lambda key, p: max(x[key][p] for x in per)
    acc = {
        "pairs": [x["pair"] for x in per],
        "kernel_rel_err_vs_oracle": {p: worst("kernel_vs_oracle", p) for p in ("mixed", "fp64")},
        "latent_rel_err_vs_oracle": {p: worst("latent_vs_oracle", p) for p in ("mixed", "fp64")},
        "kernel_rel_err_vs_truth": {p: worst("kernel_vs_truth", p) for p in ("mixed", "fp64", "oracle")},
        "bars": {"kernel_vs_oracle": {"mixed": 1e-3, "fp64": 1e-9}, "latent_vs_oracle": 1e-4},
        "per_pair": per,
        "note": "max over the sampled pairs; kernels relative L2 over both kernels, latents relative "
                "L2 over all channels; PSNR against the true latent (peak = its max)",
    }
    return base, acc


def noise_sweep(ctx, device, sigmas=(0.0, 1e-5, 1e-4, 1e-3), pairs: int = 4) -> dict:
    """Kernel error against the truth of the mixed path at 1080p RGB as the
    noise level grows: where the method's output means something."""
    import torch
    from paper_1203_4874_gb300 import cbp

    out = []
    for sg in sigmas:
        b1, b2, k1t, k2t = make_inputs(ctx, pairs, 1203000, device, sigma=sg)
        prm = cbp.params(T1, T2, path="mixed", eps=EPS, flags=cbp.CBP_FLAG_KERNELS_F64)
        k1, k2, d, _ = cbp.cbp_estimate_kernels(ctx, b1, b2, prm)
        torch.cuda.synchronize()
        g = torch.cat([k1.flatten(1), k2.flatten(1)], 1)
        t = torch.cat([k1t.flatten(1), k2t.flatten(1)], 1)
        e = ((g - t).norm(dim=1) / t.norm(dim=1)).cpu().tolist()
        out.append({"sigma": sg, "kernel_rel_err_vs_truth": e,
                    "gap_min": [x.gap_min for x in d]})
        del b1, b2
    return {"workload": f"first {pairs} pairs of {WORKLOAD} (seeds 1203000..), mixed path, eps 1e-4",
            "points": out}


def percentile(xs, q):
    """The q-th percentile of xs, linear interpolation between order statistics
    (numpy's default); with fewer than 100 samples p99 lies between the two
    largest."""
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


def reference_arm(args):
    """The oracle on the host cores: each step deblurs one pair of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ.setdefault(k, str(cores))
    import numpy as np
    import scipy.signal
    import oracle
    from cbp_synth import make_pair_inputs

    inputs = []
    for f in range(args.steps + args.warmup):
        inp = make_pair_inputs(WORKLOAD, f % 60)
        b1 = np.stack([scipy.signal.fftconvolve(ch, inp.k1) for ch in inp.latent]) + inp.noise1
        b2 = np.stack([scipy.signal.fftconvolve(ch, inp.k2) for ch in inp.latent]) + inp.noise2
        inputs.append((b1.astype(np.float32).astype(np.float64), b2.astype(np.float32).astype(np.float64)))
    for i in range(args.warmup):
        oracle.deblur_pair(*inputs[i], T1, T2, eps=EPS)
    times = []
    for i in range(args.warmup, args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.deblur_pair(*inputs[i], T1, T2, eps=EPS)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(1, "FP64 numpy oracle on the host cores"),
        "p50_ms": 1e3 * statistics.median(times), "p99_ms": 1e3 * percentile(times, 99),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"1 pair per step of {WORKLOAD}, FP64 numpy oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ main ----
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cbp", choices=["cbp", "reference"])
    ap.add_argument("--pairs", type=int, default=60)
    ap.add_argument("--cpu-pairs", type=int, default=12,
                    help="pairs of the GPU's batch the oracle deblurs on the host (timed, and "
                         "the errors of the GPU results against it)")
    ap.add_argument("--no-noise-sweep", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the size-estimation, multi-level, camera-side and scale-fix sections")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-path measurement")
    ap.add_argument("--serve-seconds", type=float, default=6.0,
                    help="seconds of the camera serving trace (0: skip)")
    ap.add_argument("--cpu-worker", default="")
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args.cpu_worker)
        return
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    import torch.distributed as dist
    from paper_1203_4874_gb300 import build, cbp

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = cbp.cbp_create(local, 0)
    n = args.pairs
    keep = min(args.cpu_pairs, n) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else 0
    inputs = make_inputs(ctx, n, shard_seed(rank, n), dev, keep=keep)
    b1, b2, k1_true, k2_true = inputs[:4]
    truth = inputs[4] if keep else None
    prm = cbp.params(T1, T2, path="mixed", eps=EPS)
    lat = torch.empty((n, C, H, W), dtype=torch.float32, device=dev)
    k1 = torch.empty((n, T1, T1), dtype=torch.float32, device=dev)
    k2 = torch.empty((n, T2, T2), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(p=prm):
        cbp.cbp_deblur_pair(ctx, b1, b2, p, k1=k1, k2=k2, latent=lat, diag=False, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    clocks = ClockSampler(local)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark()
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]

    # ---- stage breakdown: the same call with per-stage CUDA events; stages
    # then run one after another (no chunk overlap), so each stage's time is
    # its kernels' own duration ----
    prof_steps = min(args.steps, 3)
    cbp.cbp_stage_times(ctx)
    cbp.cbp_profile(ctx, True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    cbp.cbp_profile(ctx, False)
    stages = cbp.cbp_stage_times(ctx)
    elapsed_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), world)
    value = job_rate(world, n, args.steps, elapsed_ms)
    mixed_k1, mixed_k2 = k1.clone(), k2.clone()

    # ---- plain FP64 path on the same batch (comparison) ----
    prm64 = cbp.params(T1, T2, path="fp64", eps=EPS)
    step(prm64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.fp64_steps):
        step(prm64)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = max_over_ranks(e0.elapsed_time(e1), world) / max(args.fp64_steps, 1)
    rel = lambda a, b: ((a - b).flatten(1).norm(dim=1) / b.flatten(1).norm(dim=1)).max().item()
    kerr = max(rel(mixed_k1.double(), k1.double()), rel(mixed_k2.double(), k2.double()))

    # ---- end to end through the C ABI with host buffers ----
    b1h = b1.cpu().pin_memory()
    b2h = b2.cpu().pin_memory()
    lath = torch.empty((n, C, H, W), dtype=torch.float32).pin_memory()
    k1h = torch.empty((n, T1, T1), dtype=torch.float32).pin_memory()
    k2h = torch.empty((n, T2, T2), dtype=torch.float32).pin_memory()
    # consecutive steps overlap (one step's input copies beside the previous one's tail)
    prmh = cbp.params(T1, T2, path="mixed", eps=EPS, flags=cbp.CBP_FLAG_HOST_IO | cbp.CBP_FLAG_OVERLAP_CALLS)

    def step_h():
        cbp.cbp_deblur_pair(ctx, b1h, b2h, prmh, k1=k1h, k2=k2h, latent=lath, diag=False, stream=stream)

    step_h()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        step_h()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    e2e_value = job_rate(world, n, args.e2e_steps, e2e_ms)
    h2d = n * C * (H1 * W1 + H2 * W2) * 4
    d2h = n * C * H * W * 4 + n * (T1 * T1 + T2 * T2) * 4

    # ---- roofline of the dominant stage ----
    dom = max((s for s in stages if stages[s][1] > 0), key=lambda s: stages[s][0])
    dom_ms = stages[dom][0] / prof_steps
    alg = algorithmic_bytes(dom, n)
    peak, peak_kind = peaks()
    if alg is not None:
        achieved = alg / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg, "ms_per_launch": dom_ms,
                "traffic": measured_traffic(dom)}
    elif algorithmic_flops(dom, n) is not None:
        fl = algorithmic_flops(dom, n)
        achieved = fl / (dom_ms / 1e3) / 1e12
        mhz = clk.get("sm_mhz") or 2070.0
        pk = fp32_peak_tflops(mhz)
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk, "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz",
                "algorithmic_flops_per_launch": fl, "ms_per_launch": dom_ms, "traffic": None}
    else:
        roof = {"bound": "alu", "kernel": dom, "achieved": None, "peak": None, "unit": None,
                "frac": None, "ms_per_launch": dom_ms, "traffic": None}
    stage_ms = {s: round(stages[s][0] / prof_steps, 4) for s in stages if stages[s][1] > 0}
    # launches per step of the profiled (unsplit) call, times the library's
    # split of a call into up to 3 chunks of at least 8 pairs (each launches
    # the whole sequence)
    chunks = max(1, min(3, n // 8))
    launches = int(sum(v[1] for v in stages.values()) / prof_steps) * chunks * args.steps

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (eval/Gram/FFT) + f64 (solves)",
        "data": "synthetic (device forward model)", "config": config(n),
        "p50_ms": statistics.median(per_step), "p99_ms": percentile(per_step, 99),
        "plain_fp64": {"value": job_rate(world, n, 1, fp64_ms), "unit": UNIT, "ms_per_step": fp64_ms},
        "kernel_rel_err_mixed_vs_fp64": kerr,
        "roofline": roof, "stage_ms_per_step": stage_ms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0 and not args.no_learned:
        result["learned"] = learned_bench(ctx, n, dev)
    if rank == 0 and args.serve_seconds > 0:
        result["serving"] = serving_bench(args.serve_seconds, dev)
    if rank == 0 and not args.no_noise_sweep:
        result["noise_sweep"] = noise_sweep(ctx, dev)
    if rank == 0 and not args.no_extras:
        result["size_estimation"] = size_estimation_bench(ctx, dev)
        result["multilevel_security"] = multilevel_bench(ctx, dev)
        result["camera_side"] = camera_bench(ctx, dev)
        result["scale_variants"] = scale_variants_bench(ctx, dev)
    if keep:
        folder = Path(tempfile.mkdtemp(prefix="cbp_bench_"))
        try:
            accuracy_sample(ctx, b1, b2, k1_true, k2_true, truth, keep, folder)
            result["cpu_baseline"], acc = cpu_baseline(folder)
            if acc is not None:
                result["accuracy"] = acc
        finally:
            for f in folder.glob("*.npy"):
                f.unlink()
            folder.rmdir()
    cbp.cbp_destroy(ctx)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
