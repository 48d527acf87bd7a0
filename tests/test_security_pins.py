"""Pins of the oracle's multi-level security step (Section 3: lower clearance
levels lose the least significant bits of the private stream), checked
against what the definition fixes: the quantisation bound at full
resolution, the truncation bound and its sign, code multiples of 2^drop,
idempotence, monotonicity, clamping, and halfway values rounding to even."""
import numpy as np
import pytest

import oracle


def test_full_resolution_is_plain_quantisation():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=10000)
    q = oracle.truncate_lsb(x, 16, 0)
    assert np.max(np.abs(q - x)) <= 0.5 / 65535 + 1e-16


@pytest.mark.parametrize("drop", [1, 4, 8, 12])
def test_truncation_bound_codes_and_idempotence(drop):
    rng = np.random.default_rng(drop)
    x = rng.uniform(size=5000)
    full = oracle.truncate_lsb(x, 16, 0)
    t = oracle.truncate_lsb(x, 16, drop)
    # truncation only lowers the code, by less than 2^drop units
    assert np.all(t <= full + 1e-15)
    assert np.all(full - t <= ((1 << drop) - 1) / 65535 + 1e-15)
    codes = np.rint(t * 65535).astype(np.int64)
    assert np.all(codes % (1 << drop) == 0)
    assert np.array_equal(oracle.truncate_lsb(t, 16, drop), t)


def test_monotone_and_clamped():
    x = np.linspace(-0.5, 1.5, 20001)
    t = oracle.truncate_lsb(x, 12, 3)
    assert np.all(np.diff(t) >= 0)
    assert t[0] == 0.0 and t[-1] == 4088 / 4095     # code 4095 with its 3 low bits cleared


def test_halfway_values_round_to_even():
    top = 255.0
    x = np.array([0.5, 1.5, 2.5, 3.5]) / top
    assert np.array_equal(oracle.truncate_lsb(x, 8, 0) * top, [0.0, 2.0, 2.0, 4.0])
