"""The seeded input recipes (CPU): every generator is reproducible, keeps
keys in the user domain and has the shape, mix and distribution its
configuration states (batch sizes, delete fractions, deletes only of keys
inserted before, half-hit lookups, query widths for an expected result size,
Zipf ranks mapped by a bijection, Poisson arrivals and the request mix)."""

import math

import numpy as np
import pytest

from paper_1707_05354_gb300 import workload as W


def test_tiny_configuration_recipe():
    cfg = W.tiny()
    calls = cfg["calls"]
    assert cfg["b"] == 1024 and len(calls) == 16
    seen = set()
    for t, (kind, keys, vals, dele) in enumerate(calls):
        assert kind == "update" and len(keys) == 1024
        assert keys.max() < (1 << 20)
        n_del = int(dele.sum())
        assert n_del == (0 if t == 0 else 102)            # floor(0.1 b)
        assert np.all(vals[dele == 1] == 0)
        assert set(keys[dele == 1].tolist()) <= seen      # deletes hit earlier inserts
        seen |= set(keys[dele == 0].tolist())
    q = cfg["lookups"]
    assert len(q) == 65536 and np.isin(q, np.array(sorted(seen), np.uint32)).sum() >= 32768
    for k1, k2 in (cfg["count"], cfg["range"]):
        w = k2.astype(np.int64) - k1.astype(np.int64) + 1
        assert len(k1) == 16384 and w.min() >= 1 and w.max() <= 1024
    again = W.tiny()
    for a, b in zip(calls, again["calls"]):
        for x, y in zip(a[1:], b[1:]):
            np.testing.assert_array_equal(x, y)


def test_paper_scale_recipe_small():
    cfg = W.paper_scale(b=1024, batches=8, n_lookup=4096, n_count=512, n_range=512)
    assert cfg["width"] == int(round(8 * float(W.KEY_LIMIT) / (1024 * 8)))
    assert W.paper_scale()["width"] == 128                # L = 8 at 2^27 updates
    k3, v3 = cfg["batch"](3)
    k3b, _ = cfg["batch"](3)                              # any batch regenerates alone
    np.testing.assert_array_equal(k3, k3b)
    assert k3.max() < W.KEY_LIMIT and len(k3) == len(v3) == 1024
    ins = np.concatenate([cfg["batch"](t)[0] for t in range(8)])
    q = cfg["lookups"]()
    assert len(q) == 4096 and np.isin(q, ins).sum() >= 2048
    k1, k2 = cfg["count"]()
    assert np.all(k2.astype(np.int64) - k1.astype(np.int64) + 1 == cfg["width"])
    assert k2.max() < W.KEY_LIMIT


def test_zipf_keys_bijection_and_head_frequency():
    ranks = np.arange(1, 1 << 16, dtype=np.uint64)
    mapped = (ranks * np.uint64(0x9E3779B1)) % np.uint64(W.SWEEP_KEY_SPACE)
    assert len(np.unique(mapped)) == len(ranks)           # odd multiplier: distinct
    g = W.rng(5, 9)
    keys = W.zipf_keys(g, 200000)
    assert keys.max() < W.SWEEP_KEY_SPACE
    # the most frequent key is rank 1 (key 0x9E3779B1 mod 2^30), with mass
    # 1 / Z, Z = sum over r <= 2^30 of r^-1.1 = zeta(1.1) - (tail above 2^30,
    # about 2^-3 / 0.1 by the integral) = 10.5844 - 1.25 (ranks above the
    # bound are redrawn)
    vals, cnt = np.unique(keys, return_counts=True)
    top = vals[np.argmax(cnt)]
    assert int(top) == 0x9E3779B1 % W.SWEEP_KEY_SPACE
    z = 10.5844 - float(W.SWEEP_KEY_SPACE) ** -0.1 / 0.1
    assert abs(cnt.max() / len(keys) - 1 / z) < 0.003


@pytest.mark.parametrize("dist,frac", [("uniform", 0.25), ("zipf", 0.5)])
def test_sweep_updates_recipe(dist, frac):
    b, total = 512, 512 * 6
    calls = W.sweep_updates(11, b, total, frac, dist)
    assert len(calls) == total // b
    seen = set()
    for t, (_, keys, vals, dele) in enumerate(calls):
        assert len(keys) == b and keys.max() < W.SWEEP_KEY_SPACE
        assert int(dele.sum()) == (0 if t == 0 else int(round(b * frac)))
        assert set(keys[dele == 1].tolist()) <= seen
        assert np.all(vals[dele == 1] == 0)
        seen |= set(keys[dele == 0].tolist())
    assert W.sweep_width(8, 1 << 27) == int(round(8 * W.SWEEP_KEY_SPACE / (1 << 27)))


def test_serving_trace_and_pools_recipe():
    n, rate = 200000, 3.0e5
    kind, arrival, start, size = W.serving_trace(n_req=n, rate=rate, pool_n=1 << 20)
    frac = np.bincount(kind, minlength=5) / n
    np.testing.assert_allclose(frac, W.SERVING_MIX, atol=0.005)
    gaps = np.diff(arrival)
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1e6 / rate) / (1e6 / rate) < 0.01
    # exponential gaps: the standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02
    assert size.min() >= 1 and size.max() <= 1 << 16
    assert abs(np.log2(np.median(size)) - 8.0) < 0.1       # log-uniform on [0, 16]
    assert np.all(start.astype(np.int64) + size.astype(np.int64) <= 1 << 20)
    a, v, c = W.serving_pools(n=1 << 16, width=8)
    assert a.max() < W.KEY_LIMIT
    np.testing.assert_array_equal(c, np.minimum(a.astype(np.int64) + 7, W.KEY_LIMIT - 1).astype(np.uint32))
    assert len(v) == len(a) == 1 << 16
    assert math.isclose(sum(W.SERVING_MIX), 1.0)
