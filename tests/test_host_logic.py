"""Host-side logic that needs no GPU: the workload recipes, the batched
form's tuning table lookup and byte model, and the oracle on batched
workloads (every instance an independent dictionary)."""

import numpy as np
import pytest

import oracle
from paper_1707_05354_gb300 import workload

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_batched_sizes_log_uniform_integers():
    s = workload.batched_sizes()
    assert len(s) == 256
    assert s.min() >= 1 << 10 and s.max() <= 1 << 18
    # log-uniform: about an eighth of the instances per octave
    octs = np.floor(np.log2(s)).astype(int)
    counts = np.bincount(octs, minlength=19)[10:18]
    assert counts.min() > 10 and counts.max() < 60
    assert np.mean((s & (s - 1)) != 0) > 0.9   # not powers of two


def test_batched_workload_recipe():
    sizes = np.array([7, 100, 1000, 33], np.int64)
    wl = workload.BatchedWorkload(seed=5, sizes=sizes, rounds=4, delete_frac=0.2)
    wl2 = workload.BatchedWorkload(seed=5, sizes=sizes, rounds=4, delete_frac=0.2)
    seen = [set() for _ in sizes]
    for t in range(4):
        k, v, d, q = wl.round(t)
        k2, v2, d2, q2 = wl2.round(t)
        for a, b_ in ((k, k2), (v, v2), (d, d2), (q, q2)):
            np.testing.assert_array_equal(a, b_)       # seeded: reproducible
        assert len(k) == wl.total == sizes.sum()
        assert k.max() < workload.KEY_LIMIT
        for i, b in enumerate(sizes):
            s = slice(int(wl.off[i]), int(wl.off[i + 1]))
            ki, di = k[s], d[s]
            n_del = 0 if t == 0 else int(round(b * 0.2))
            assert int(di.sum()) == n_del
            assert np.all(v[s][di == 1] == 0)
            # deletes target keys inserted by earlier rounds of this instance
            assert set(ki[di == 1].tolist()) <= seen[i]
            seen[i] |= set(ki[di == 0].tolist())
            # half the lookups are inserted keys
            hits = np.isin(q[s], np.array(sorted(seen[i]), np.uint32))
            assert hits.sum() >= b // 2


def test_batched_workload_on_oracles():
    """Per instance, O1 (ordered map) and O2 (offline) agree on a batched
    workload with short batches padded as the batched form pads them."""
    sizes = np.array([5, 64, 300], np.int64)
    wl = workload.BatchedWorkload(seed=11, sizes=sizes, rounds=6)
    calls = {i: [] for i in range(len(sizes))}
    o1 = [oracle.MapOracle(int(b)) for b in sizes]
    for t in range(6):
        k, v, d, q = wl.round(t)
        for i, b in enumerate(sizes):
            s = slice(int(wl.off[i]), int(wl.off[i + 1]))
            c = ("update", k[s], v[s], d[s])
            calls[i].append(c)
            o1[i].call(*c)
    for i, b in enumerate(sizes):
        o2 = oracle.OfflineOracle.from_calls(calls[i], int(b))
        ek, ev = o1[i].items()
        np.testing.assert_array_equal(o2.keys, ek)
        np.testing.assert_array_equal(o2.vals, ev)


def test_tuning_table_lookup():
    from paper_1707_05354_gb300 import autotune
    table = {10: {"tile": 1024, "bin_log2": 2}, 11: {"tile": 1024, "bin_log2": 3},
             18: {"tile": 2048, "bin_log2": 5}}
    got = autotune.tuning_for([1, 1024, 1500, 3000, 1 << 18, 1 << 20], table)
    # below / above the table clamp to its ends; missing buckets use the default
    assert got == [(1024, 2), (1024, 2), (1024, 3), autotune.DEFAULT, (2048, 5), (2048, 5)]
    assert autotune.tuning_for([5, 6], {}) == [autotune.DEFAULT] * 2
    for t, e in autotune.CANDIDATES:
        assert t in (1024, 2048) and 1 <= e <= 6


def test_batched_byte_model():
    import bench
    # one instance, rounds 0..3: k = 0, 1, 0, 2; full levels after: 1, 1, 2, 1
    b = 100
    expect = 16 * b * (1 + 2 + 1 + 4) + b * (9 * 4 + 32 * (1 + 1 + 2 + 1))
    assert bench.batched_bytes([b], 4) == expect
    # the update bytes over R = 2^m rounds are (8m + 16) B per update
    m = 5
    upd = sum(16.0 * (1 << ((~r & (r + 1)).bit_length() - 1)) for r in range(1 << m))
    assert upd / (1 << m) == 8 * m + 16


def test_update_phase_roofline():
    import bench
    r = bench.update_roofline(1000.0, 128, 6786.9)
    assert r["bytes_per_update"] == 72.0                      # 8m + 16 at m = 7
    assert abs(r["achieved_GB/s"] - 72.0) < 1e-9              # 10^9 updates/s x 72 B
    assert abs(r["frac"] - 72.0 / 6786.9) < 1e-12
    assert abs(r["roofline_M_updates_per_s"] - 6786.9e3 / 72.0) < 1e-6
    for m in range(0, 9):
        assert bench.update_roofline(1.0, 1 << m, 1.0)["bytes_per_update"] == 8 * m + 16
    # not a power of two: batches 0..2 fold into levels 0, 1, 0
    assert bench.update_roofline(1.0, 3, 1.0)["bytes_per_update"] == (16 + 32 + 16) / 3


def test_tuning_cache_round_trip(tmp_path, monkeypatch):
    """load_or_tune reads a cached table (keys back to ints), and on a
    missing or corrupt cache tunes once and writes the cache it then reads."""
    import json
    from paper_1707_05354_gb300 import autotune
    path = tmp_path / "multi_tuning_test.json"
    monkeypatch.setattr(autotune, "cache_path", lambda device=0: str(path))
    calls = []

    def fake_tune(device=0, verbose=False):
        calls.append(device)
        return {12: {"tile": 1024, "bin_log2": 4, "ms": {}}, 16: {"tile": 2048, "bin_log2": 2, "ms": {}}}

    monkeypatch.setattr(autotune, "tune", fake_tune)
    path.write_text("{not json")
    t1 = autotune.load_or_tune()
    assert calls == [0] and sorted(t1) == [12, 16]
    t2 = autotune.load_or_tune()                                  # from the cache now
    assert calls == [0] and t2 == {12: t1[12], 16: t1[16]}
    assert json.loads(path.read_text())["buckets"]["12"]["tile"] == 1024
    assert autotune.tuning_for([3000, 1 << 16, 1 << 20], t2) == [(1024, 4), (2048, 2), (2048, 2)]
    autotune.load_or_tune(retune=True)
    assert calls == [0, 0]
