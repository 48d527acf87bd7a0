"""The row passes' bulk-copy waits made to run out (checked build, started by
tests/test_timeout_gpu.py with CBP_LIBRARY=checks): every copy lands but no
barrier phase completes, so each bounded wait expires with nothing in flight.
Prints one JSON line: the per-pair statuses with the waits expiring, the
seconds the calls took, and whether the same calls afterwards, with the waits
restored, give the results of calls made before (the context stays usable)."""
from __future__ import annotations

import json
import os
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import torch  # noqa: E402

from paper_1203_4874_gb300 import cbp  # noqa: E402
from tests._inputs import make_batch  # noqa: E402


def main():
    assert os.environ.get("CBP_LIBRARY") == "checks"
    ctx = cbp.cbp_create(0, 0)
    dev = torch.device("cuda", 0)
    cases = []
    # generic row passes (480p) and the in-register ones (1080p RGB), mixed path
    for name, frames, cast in (("video_480p", [0, 1], None), ("rgb_1080p", [0], torch.float32)):
        b1, b2, k1, k2, _, cfg = make_batch(name, frames)
        B1, B2 = torch.from_numpy(b1).to(dev), torch.from_numpy(b2).to(dev)
        if cast is not None:
            B1, B2 = B1.to(cast), B2.to(cast)
        cases.append((name, B1, B2, cbp.params(k1.shape[-1], k2.shape[-1], path="mixed", eps=cfg.eps)))

    def run(B1, B2, prm):
        lat, K1, K2, d, _ = cbp.cbp_deblur_pair(ctx, B1, B2, prm)
        torch.cuda.synchronize()
        return lat.clone(), K1.clone(), K2.clone(), [x.status for x in d]

    before = [run(B1, B2, prm) for _, B1, B2, prm in cases]
    cbp.cbp_check_expire_waits(True)
    expired, seconds = [], []
    for _, B1, B2, prm in cases:
        t0 = time.time()
        expired.append(run(B1, B2, prm)[3])
        seconds.append(time.time() - t0)
    cbp.cbp_check_expire_waits(False)
    after = [run(B1, B2, prm) for _, B1, B2, prm in cases]
    same = all(torch.equal(a, b) for x, y in zip(before, after) for a, b in zip(x[:3], y[:3]))
    print(json.dumps({"cases": [c[0] for c in cases], "before": [b[3] for b in before],
                      "expired": expired, "after": [a[3] for a in after], "same_after": same,
                      "seconds": seconds, "timeout_status": cbp.CBP_ERR_TIMEOUT}))
    cbp.cbp_destroy(ctx)


if __name__ == "__main__":
    main()
