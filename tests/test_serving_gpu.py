"""A9 serving engine through the C ABI: results identical alone and in a mixed
batch (and equal to the synchronous call), admission under a small HBM
budget, poll semantics, concurrent submitters, statistics."""
from __future__ import annotations

import threading

import numpy as np
import pytest
import torch

from tests._inputs import make_batch

pytestmark = pytest.mark.gpu


def _pair(cfg_name, frame, h, w):
    b1, b2, _, _, _, cfg = make_batch(cfg_name, [frame], h=h, w=w, fast=True)
    dt = torch.float64 if cfg.frame_dtype == "f64" else torch.float32
    dev = torch.device("cuda", 0)
    return (torch.tensor(b1, dtype=dt, device=dev), torch.tensor(b2, dtype=dt, device=dev), cfg)


def _outputs(cbp, b1, cfg, prm, deblur=True):
    dev, dt = b1.device, b1.dtype
    k1 = torch.empty((1, prm.t1, prm.t1), dtype=dt, device=dev)
    k2 = torch.empty((1, prm.t2, prm.t2), dtype=dt, device=dev)
    lat = None
    if deblur:
        c, h1, w1 = b1.shape[-3:]
        lat = torch.empty((1, c, h1 - prm.t1 + 1, w1 - prm.t1 + 1), dtype=dt, device=dev)
    return k1, k2, lat


def _prm(cbp, cfg, path=None):
    return cbp.params(cfg.t1, cfg.t2, path=path or cfg.path, eps=cfg.eps)


def _submit(cbp, ctx, b1, b2, cfg, deblur=True, path=None):
    prm = _prm(cbp, cfg, path)
    k1, k2, lat = _outputs(cbp, b1, cfg, prm, deblur)
    t = cbp.cbp_stream_submit(ctx, b1, b2, prm, k1, k2, lat)
    return t, (k1, k2, lat)


def _wait(cbp, ctx, t):
    s, d = cbp.cbp_stream_poll(ctx, t, -1)
    assert s >= 0, cbp.status_string(s)
    return s, d


@pytest.mark.parametrize("path", [None, "mixed"])
def test_identical_alone_in_mix_and_sync(gpu_ctx, path):
    """Alone, in a mix of buckets, and from the synchronous call: the same
    result, bit for bit -- on each workload's own path and on the mixed path
    the serving benchmark runs."""
    from paper_1203_4874_gb300 import cbp
    a1, a2, cfg = _pair("video_480p", 0, 60, 80)
    b1, b2, _ = _pair("video_480p", 1, 60, 80)
    c1, c2, _ = _pair("video_480p", 2, 48, 64)       # another bucket
    d1, d2, _ = _pair("video_480p", 3, 60, 80)
    e1, e2, cfg64 = _pair("single_64", 0, None, None)  # float64 frames, another bucket
    ta, outa = _submit(cbp, gpu_ctx, a1, a2, cfg, path=path)
    _wait(cbp, gpu_ctx, ta)
    # the same request again, in a mix of buckets
    tickets = []
    for x1, x2, cf in ((b1, b2, cfg), (c1, c2, cfg), (a1, a2, cfg), (e1, e2, cfg64), (d1, d2, cfg)):
        tickets.append(_submit(cbp, gpu_ctx, x1, x2, cf, path=path))
    for t, _ in tickets:
        _wait(cbp, gpu_ctx, t)
    outa2 = tickets[2][1]
    for x, y in zip(outa, outa2):
        assert torch.equal(x, y)
    # and the synchronous call on the same pair
    lat, k1, k2, _, st = cbp.cbp_deblur_pair(gpu_ctx, a1, a2, _prm(cbp, cfg, path))
    torch.cuda.synchronize()
    assert st >= 0
    assert torch.equal(k1, outa[0]) and torch.equal(k2, outa[1]) and torch.equal(lat, outa[2])


def test_estimate_only_request(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    a1, a2, cfg = _pair("video_480p", 4, 60, 80)
    t, (k1, k2, _) = _submit(cbp, gpu_ctx, a1, a2, cfg, deblur=False)
    _wait(cbp, gpu_ctx, t)
    r1, r2, _, st = cbp.cbp_estimate_kernels(gpu_ctx, a1, a2, _prm(cbp, cfg))
    torch.cuda.synchronize()
    assert torch.equal(k1, r1) and torch.equal(k2, r2)


def test_poll_semantics(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    s, _ = cbp.cbp_stream_poll(gpu_ctx, 1 << 60, 0)
    assert s == cbp.CBP_ERR_INVALID_ARG
    pairs = [_pair("video_480p", 10 + i, 240, 320) for i in range(6)]
    subs = [_submit(cbp, gpu_ctx, x1, x2, cf) for x1, x2, cf in pairs]
    last = subs[-1][0]
    s, _ = cbp.cbp_stream_poll(gpu_ctx, last, 1)
    assert s in (cbp.CBP_ERR_TIMEOUT, cbp.CBP_OK, cbp.CBP_WARN_ILL_CONDITIONED)
    if s == cbp.CBP_ERR_TIMEOUT:
        s0, _ = cbp.cbp_stream_poll(gpu_ctx, last, 0)
        assert s0 in (cbp.CBP_ERR_BUSY, cbp.CBP_OK, cbp.CBP_WARN_ILL_CONDITIONED)
        if s0 == cbp.CBP_ERR_BUSY:
            _wait(cbp, gpu_ctx, last)
    for t, _ in subs[:-1]:
        _wait(cbp, gpu_ctx, t)
    # a released ticket is unknown
    s, _ = cbp.cbp_stream_poll(gpu_ctx, last, 0)
    assert s == cbp.CBP_ERR_INVALID_ARG


def test_concurrent_submitters(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    pairs = [_pair("video_480p", 20 + i, 60, 80) for i in range(4)]
    refs = []
    for x1, x2, cf in pairs:
        t, out = _submit(cbp, gpu_ctx, x1, x2, cf)
        _wait(cbp, gpu_ctx, t)
        refs.append(out)
    results = [[None] * 3 for _ in range(4)]
    errors = []

    def worker(w):
        try:
            subs = []
            for rep in range(3):
                x1, x2, cf = pairs[(w + rep) % 4]
                subs.append(((w + rep) % 4, rep, _submit(cbp, gpu_ctx, x1, x2, cf)))
            for idx, rep, (t, out) in subs:
                s, _ = cbp.cbp_stream_poll(gpu_ctx, t, -1)
                assert s >= 0
                results[w][rep] = (idx, out)
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for w in range(4):
        for idx, out in results[w]:
            for x, y in zip(out, refs[idx]):
                assert torch.equal(x, y)
    st = cbp.cbp_stream_stats(gpu_ctx)
    assert st["completed"] >= 12 and 0 < st["p50_ms"] <= st["p99_ms"]


def test_small_budget_admission(built_lib):
    from paper_1203_4874_gb300 import cbp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a1, a2, cfg = _pair("video_480p", 30, 60, 80)
    prm = _prm(cbp, cfg)
    one = cbp.cbp_workspace_size(a1, a2, prm)
    ctx = cbp.cbp_create(0, int(1.6 * one) + (1 << 16))
    try:
        pairs = [_pair("video_480p", 31 + i, 60, 80) for i in range(5)]
        subs = [_submit(cbp, ctx, x1, x2, cf) for x1, x2, cf in pairs]
        for t, _ in subs:
            s, _ = cbp.cbp_stream_poll(ctx, t, -1)
            assert s >= 0, cbp.status_string(s)
        # larger than the whole budget: refused, not queued forever
        big1, big2, cfgb = _pair("video_480p", 40, 240, 320)
        t, _ = _submit(cbp, ctx, big1, big2, cfgb)
        s, _ = cbp.cbp_stream_poll(ctx, t, -1)
        assert s == cbp.CBP_ERR_BUDGET
        assert cbp.cbp_stream_stats(ctx)["completed"] == 6
    finally:
        cbp.cbp_destroy(ctx)


def test_two_buckets_overlap_on_the_device(gpu_ctx):
    """Requests of two buckets submitted together run as two batches on two
    slot streams at once: their device intervals (CUDA events around each
    batch) overlap."""
    from paper_1203_4874_gb300 import cbp
    a1, a2, cfg = _pair("rgb_1080p", 0, 720, 1280)
    b1, b2, _ = _pair("rgb_1080p", 1, 540, 960)           # another bucket
    prm_a = cbp.params(cfg.t1, cfg.t2, path="mixed", eps=cfg.eps)
    # warm the engine (graph captures) so that both batches launch at once
    for x1, x2 in ((a1, a2), (b1, b2)):
        k1, k2, lat = _outputs(cbp, x1, cfg, prm_a)
        _wait(cbp, gpu_ctx, cbp.cbp_stream_submit(gpu_ctx, x1, x2, prm_a, k1, k2, lat))
    outs, tickets = [], []
    for x1, x2 in ((a1, a2), (b1, b2)):
        k1, k2, lat = _outputs(cbp, x1, cfg, prm_a)
        outs.append((k1, k2, lat))
        tickets.append(cbp.cbp_stream_submit(gpu_ctx, x1, x2, prm_a, k1, k2, lat))
    (_, da), (_, db) = (_wait(cbp, gpu_ctx, t) for t in tickets)
    assert 0 < da.gpu_start_ms < da.gpu_end_ms and 0 < db.gpu_start_ms < db.gpu_end_ms
    overlap = min(da.gpu_end_ms, db.gpu_end_ms) - max(da.gpu_start_ms, db.gpu_start_ms)
    assert overlap > 0, (da.gpu_start_ms, da.gpu_end_ms, db.gpu_start_ms, db.gpu_end_ms)
