"""Parity of the CUDA path with the CPU oracle (needs a GPU).

Every comparison is exact (integer work): level contents against the
structural oracle S, query answers against the ordered-map oracle O1 (or the
offline oracle O2 at full size).  All calls go through the C ABI via the
ctypes binding.
"""

import numpy as np
import pytest

import oracle
from paper_1707_05354_gb300 import workload
from tests.walkthrough import parse

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g(lsm_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lsm_lib


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def assert_levels(lsm, s):
    lv = lsm.levels()
    assert lsm.r == s.r
    for i in range(40):
        ekv, ev = s.level(i)
        if len(ekv):
            assert i in lv, "level %d missing" % i
            np.testing.assert_array_equal(lv[i][0], ekv, err_msg="keys of level %d" % i)
            np.testing.assert_array_equal(lv[i][1], ev, err_msg="values of level %d" % i)
        else:
            assert i not in lv


def assert_queries(lsm, o1, q, k1, k2):
    val, found = lsm.lookup(q)
    ev, ef = o1.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))
    off, rk, rv = lsm.range(k1, k2)
    eo, ek, evv = o1.range(k1, k2)
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), eo)
    np.testing.assert_array_equal(u32(rk), ek)
    np.testing.assert_array_equal(u32(rv), evv)


# ------------------------------------------------------------------ golden --
def test_walkthrough_on_gpu(g):
    b, steps = parse("fig1_walkthrough.txt")
    lsm = g.LSM(b, 64 * b)
    for st in steps:
        if st[0] == "op":
            _, kind, keys, vals, dels = st
            lsm.call(kind, keys, vals, dels)
        elif st[0] == "cleanup":
            lsm.cleanup()
        elif st[0] == "r":
            assert lsm.r == st[1]
        elif st[0] == "level":
            lv = lsm.levels()
            if st[2] is None:
                assert st[1] not in lv
            else:
                np.testing.assert_array_equal(lv[st[1]][0], st[2])
                np.testing.assert_array_equal(lv[st[1]][1], st[3])
        elif st[0] == "lookup":
            val, found = lsm.lookup(st[1])
            np.testing.assert_array_equal(found.cpu().numpy(), st[3])
            np.testing.assert_array_equal(u32(val), st[2])
        elif st[0] == "count":
            _, k1, k2, n = st
            assert int(u32(lsm.count([k1], [min(k2, 2**32 - 1)]))[0]) == n
        elif st[0] == "range":
            _, k1, k2, pairs = st
            off, rk, rv = lsm.range([k1], [min(k2, 2**32 - 1)])
            assert list(zip(u32(rk).tolist(), u32(rv).tolist())) == pairs
    assert lsm.device_errors() == 0


# -------------------------------------------------------------------- sort --
@pytest.mark.parametrize("n", [1, 2, 31, 4095, 4096, 4097, 12345, 1 << 16, (1 << 20) - 3, 1 << 20, 3 << 20])
def test_sort_pairs_matches_stable_sort(g, n):
    lsm = g.LSM(max(n, 1), max(n, 1))
    rng = np.random.default_rng(n)
    if n % 2:
        keys = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    else:  # many duplicates: stability matters
        keys = rng.integers(0, 50, size=n).astype(np.uint32) * np.uint32(0x01010101)
    vals = np.arange(n, dtype=np.uint32)
    kd, vd = g.as_device_u32(keys, 0), g.as_device_u32(vals, 0)
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    g.lsm_sort_pairs(lsm.h, kd.data_ptr(), vd.data_ptr(), ko.data_ptr(), vo.data_ptr(), n,
                     torch.cuda.current_stream().cuda_stream)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(u32(ko), keys[order])
    np.testing.assert_array_equal(u32(vo), vals[order])


@pytest.mark.parametrize("dist", ["dup4", "sub_bin_skew", "one_bucket_spread", "hot_key"])
def test_sort_pairs_key_distributions(g, dist):
    """Stability and order for the bucket sort's paths: keys that repeat
    about 4 times each (ties inside the counting pass's sub-bins), buckets
    whose keys crowd a few sub-bins (the pass-by-pass path), every key in
    one top-byte bucket of at most 5120 elements spread over its low bits,
    and one key holding 40 % of the input beside uniform keys (its bucket,
    far above shared memory, is sorted through the spill area)."""
    n = 1 << 20
    rng = np.random.default_rng(7)
    if dist == "hot_key":
        keys = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
        keys[rng.random(n) < 0.4] = np.uint32(0x9E3779B1)
    elif dist == "dup4":
        keys = (rng.integers(0, 1 << 18, size=n).astype(np.uint64) * np.uint64(16411) % np.uint64(1 << 32))
        keys = keys.astype(np.uint32)
    elif dist == "sub_bin_skew":
        # random top byte and low 12 bits, few distinct values in bits 12..23
        top = rng.integers(0, 256, size=n).astype(np.uint32) << np.uint32(24)
        mid = (rng.integers(0, 3, size=n).astype(np.uint32) * np.uint32(1111)) << np.uint32(12)
        keys = top | mid | rng.integers(0, 4096, size=n).astype(np.uint32)
    else:
        n = 5000
        keys = (np.uint32(0x5A) << np.uint32(24)) | rng.integers(0, 1 << 24, size=n).astype(np.uint32)
    lsm = g.LSM(n, n)
    vals = np.arange(n, dtype=np.uint32)
    kd, vd = g.as_device_u32(keys, 0), g.as_device_u32(vals, 0)
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    g.lsm_sort_pairs(lsm.h, kd.data_ptr(), vd.data_ptr(), ko.data_ptr(), vo.data_ptr(), n,
                     torch.cuda.current_stream().cuda_stream)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(u32(ko), keys[order])
    np.testing.assert_array_equal(u32(vo), vals[order])


# ------------------------------------------------------ configuration tiny --
def test_tiny_configuration_bit_exact(g):
    cfg = workload.tiny()
    b = cfg["b"]
    lsm = g.LSM(b, 64 * b)
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    for kind, k, v, d in cfg["calls"]:
        lsm.call(kind, k, v, d)
        o1.call(kind, k, v, d)
        s.call(kind, k, v, d)
        assert_levels(lsm, s)
    k1, k2 = cfg["count"]
    val, found = lsm.lookup(cfg["lookups"])
    ev, ef = o1.lookup(cfg["lookups"])
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))
    r1, r2 = cfg["range"]
    off, rk, rv = lsm.range(r1, r2)
    eo, ek, evv = o1.range(r1, r2)
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), eo)
    np.testing.assert_array_equal(u32(rk), ek)
    np.testing.assert_array_equal(u32(rv), evv)
    lsm.set_lookup_mode(g.LOOKUP_SORTED)
    val2, found2 = lsm.lookup(cfg["lookups"])
    np.testing.assert_array_equal(found2.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val2), ev)
    lsm.cleanup()
    s.cleanup()
    assert_levels(lsm, s)
    assert_queries(lsm, o1, cfg["lookups"][:5000], k1[:3000], k2[:3000])
    assert lsm.device_errors() == 0


# ------------------------------------------------------- random, many b ---
def random_calls(rng, b, ncalls, key_space):
    calls = []
    for _ in range(ncalls):
        kind = rng.choice(["insert", "delete", "update", "insert"])
        n = int(rng.integers(1, b + 1)) if kind == "update" else int(rng.integers(1, 3 * b + 1))
        keys = rng.integers(0, key_space, size=n).astype(np.uint32)
        vals = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
        dels = (rng.random(n) < 0.3).astype(np.uint8)
        calls.append((kind, keys, vals, dels))
    return calls


@pytest.mark.parametrize("b,key_space,ncalls", [(1, 8, 40), (2, 16, 40), (3, 30, 30), (5, 50, 30),
                                                 (17, 200, 25), (100, 3000, 20), (1000, 1 << 20, 12),
                                                 (3000, 1 << 12, 12), (4096, (1 << 31) - 1, 10),
                                                 (1 << 14, 1 << 20, 6)])
def test_random_logs_bit_exact(g, b, key_space, ncalls):
    rng = np.random.default_rng(b * 7919 + key_space)
    calls = random_calls(rng, b, ncalls, min(key_space, (1 << 31) - 1))
    nb = sum(-(-len(c[1]) // b) if c[0] != "update" else 1 for c in calls)
    lsm = g.LSM(b, (nb + 2) * b)
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    ks = min(key_space, (1 << 31) - 1)
    q = np.concatenate([rng.integers(0, ks, size=2000), [0, ks - 1, (1 << 31) - 2, (1 << 31) - 1, 2**32 - 1]])
    q = q.astype(np.uint32)
    k1 = rng.integers(0, ks, size=500).astype(np.uint32)
    k2 = (k1.astype(np.int64) + rng.integers(-3, max(4, ks // 50), size=500)).clip(0, 2**32 - 1).astype(np.uint32)
    for i, c in enumerate(calls):
        lsm.call(*c)
        o1.call(*c)
        s.call(*c)
        if i % 4 == 3 or i == len(calls) - 1:
            assert_levels(lsm, s)
            assert_queries(lsm, o1, q, k1, k2)
    lsm.cleanup()
    s.cleanup()
    assert_levels(lsm, s)
    assert_queries(lsm, o1, q, k1, k2)
    more = random_calls(rng, b, 3, ks)
    for c in more:
        lsm.call(*c)
        o1.call(*c)
        s.call(*c)
    assert_levels(lsm, s)
    assert_queries(lsm, o1, q, k1, k2)
    assert lsm.device_errors() == 0


def test_deep_fold_many_sources(g):
    """Folds of up to 9 sources over many tiles, b not a multiple of 32."""
    b = 1000
    lsm = g.LSM(b, 600 * b)
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    rng = np.random.default_rng(5)
    for t in range(511):
        keys = rng.integers(0, 1 << 16, size=b).astype(np.uint32)  # heavy duplication
        vals = np.full(b, t, np.uint32)
        dels = (rng.random(b) < 0.05).astype(np.uint8)
        lsm.update(keys, vals, dels)
        o1.call("update", keys, vals, dels)
        s.call("update", keys, vals, dels)
        if t in (6, 62, 255, 510):
            assert_levels(lsm, s)
    q = rng.integers(0, 1 << 16, size=20000).astype(np.uint32)
    k1 = rng.integers(0, 1 << 16, size=2000).astype(np.uint32)
    assert_queries(lsm, o1, q, k1, k1 + 40)
    lsm.set_lookup_mode(g.LOOKUP_SORTED)
    assert_queries(lsm, o1, q, k1, k1 + 40)
    assert lsm.device_errors() == 0


def test_wide_count_range_queries(g):
    """Queries whose windows hold hundreds to thousands of elements (the
    warp-per-query path: the interval cut into 32 key sub-intervals) mixed
    with narrow ones in one call, over several levels with stale versions and
    tombstones; intervals reaching past the key domain and empty ones."""
    b = 4096
    lsm = g.LSM(b, 64 * b)
    o1 = oracle.MapOracle(b)
    rng = np.random.default_rng(77)
    for t in range(23):                     # r = 23: levels 0, 1, 2, 4
        keys = rng.integers(0, 1 << 14, size=b).astype(np.uint32)
        vals = rng.integers(0, 1 << 32, size=b, dtype=np.uint64).astype(np.uint32)
        dels = (rng.random(b) < 0.2).astype(np.uint8)
        lsm.update(keys, vals, dels)
        o1.call("update", keys, vals, dels)
    n = 3000
    k1 = rng.integers(0, 1 << 14, size=n).astype(np.uint32)
    w = np.where(rng.random(n) < 0.5, rng.integers(1, 16, size=n), rng.integers(64, 1 << 14, size=n))
    k2 = (k1.astype(np.int64) + w).clip(0, 2**32 - 1).astype(np.uint32)
    k1[:3] = [0, 0, 5000]
    k2[:3] = [2**32 - 1, (1 << 31) - 1, 4000]   # whole domain, past the key domain, empty
    assert_queries(lsm, o1, k1[:10], k1, k2)
    np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))
    assert int(u32(lsm.count(k1[:1], k2[:1]))[0]) == len(o1.items()[0])
    assert lsm.device_errors() == 0


# ------------------------------------------------------ checkpoint / resume --
@pytest.mark.parametrize("b,ncalls", [(100, 13), (4096, 11)])
def test_checkpoint_resume(g, b, ncalls):
    """lsm_save / lsm_load: a dictionary restored from a checkpoint into a
    fresh handle (same b, more room) has the same levels bit for bit and
    answers like the oracle; further batches and a cleanup on both the
    original and the restored one keep them identical."""
    calls = workload.sweep_updates(1707053521, b, ncalls * b, 0.25, "uniform")
    lsm = g.LSM(b, 16 * b)
    s = oracle.StructuralOracle(b)
    o1 = oracle.MapOracle(b)
    for c in calls[:-2]:
        lsm.call(*c)
        s.call(*c)
        o1.call(*c)
    r, hk, hv = lsm.save()
    assert r == lsm.r and len(hk) == r * b
    lsm2 = g.LSM(b, 40 * b)
    lsm2.load(r, hk, hv)
    assert lsm2.r == r
    assert_levels(lsm2, s)
    rng = np.random.default_rng(b)
    ins = np.concatenate([c[1][c[3] == 0] for c in calls])
    q = workload.lookup_queries(9, ins, 4096, workload.SWEEP_KEY_SPACE)
    k1 = rng.integers(0, workload.SWEEP_KEY_SPACE, size=1024).astype(np.uint32)
    k2 = (k1 + rng.integers(0, 1 << 24, size=1024)).astype(np.uint32)
    assert_queries(lsm2, o1, q, k1, k2)
    for c in calls[-2:]:
        lsm.call(*c)
        lsm2.call(*c)
        s.call(*c)
    assert_levels(lsm, s)
    assert_levels(lsm2, s)
    lsm2.cleanup()
    s.cleanup()
    assert_levels(lsm2, s)
    # errors: a handle that is not empty, another b, too few levels
    with pytest.raises(g.LSMError):
        lsm2.load(r, hk, hv)
    with pytest.raises(g.LSMError) as e:
        g.LSM(b + 1, 40 * b).load(r, hk, hv, b=b)
    assert e.value.status == g.LSM_ERR_ARG
    with pytest.raises(g.LSMError) as e:
        g.LSM(b, b).load(r, hk, hv)
    assert e.value.status == g.LSM_ERR_FULL
    assert lsm.device_errors() == 0 and lsm2.device_errors() == 0


# ------------------------------------------------------ deferred key check --
@pytest.mark.parametrize("b", [64, 5000])
def test_deferred_key_check(g, b):
    """LSM_OPT_KEY_CHECK = 1: update calls do not wait for the key check; a
    batch holding a bad key is applied as b placebo tombstones (key 2^31 - 1,
    which no query sees): the levels equal the oracle's for the same log with
    that batch replaced by b deletes of key 2^31 - 1, every query answers as
    if the batch had never been issued, the device error word records the bad
    key, and cleanup drops the placebos."""
    rng = np.random.default_rng(b)
    calls = workload.sweep_updates(1707053511, b, 9 * b, 0.25, "uniform")
    lsm = g.LSM(b, 16 * b)
    g.lsm_set_option(lsm.h, g.LSM_OPT_KEY_CHECK, 1)
    assert g.lsm_get_option(lsm.h, g.LSM_OPT_KEY_CHECK) == 1
    s = oracle.StructuralOracle(b)
    o1 = oracle.MapOracle(b)
    placebo = np.full(b, (1 << 31) - 1, np.uint32)
    for i, c in enumerate(calls):
        if i in (3, 6):
            kind, keys, vals, dele = c
            keys = keys.copy()
            keys[rng.integers(0, len(keys))] = np.uint32(2**31 + 5 if i == 3 else 2**32 - 1)
            lsm.call(kind, keys, vals, dele)          # returns at once, no error
            s.call("delete", placebo)                 # what the batch becomes
            continue
        lsm.call(*c)
        s.call(*c)
        o1.call(*c)
    assert lsm.r == len(calls)
    assert_levels(lsm, s)
    ins = np.concatenate([c[1][c[3] == 0] for c in calls])
    q = np.concatenate([workload.lookup_queries(5, ins, 2048, workload.SWEEP_KEY_SPACE),
                        np.array([(1 << 31) - 1, 2**31 + 5], np.uint32)])
    k1 = rng.integers(0, workload.SWEEP_KEY_SPACE, size=1024).astype(np.uint32)
    k2 = (k1 + rng.integers(0, 1 << 22, size=1024)).astype(np.uint32)
    k1[:2], k2[:2] = 0, 2**32 - 1
    assert_queries(lsm, o1, q, k1, k2)
    assert lsm.device_errors() & 1                   # the bad keys were recorded
    lsm.cleanup()
    s.cleanup()
    assert_levels(lsm, s)
    assert_queries(lsm, o1, q, k1, k2)
    # back to the synchronous check: the same bad batch is refused
    g.lsm_set_option(lsm.h, g.LSM_OPT_KEY_CHECK, 0)
    r = lsm.r
    with pytest.raises(g.LSMError) as e:
        lsm.insert(np.array([1, 2**31], np.uint32), np.array([1, 2], np.uint32))
    assert e.value.status == g.LSM_ERR_KEY_RANGE and lsm.r == r
    assert lsm.device_errors() == 0


# ------------------------------------------------------------------- edges --
def test_edges(g):
    b = 64
    lsm = g.LSM(b, 3 * b)    # two levels: room for 3 batches
    empty_q = np.array([0, 5, (1 << 31) - 2], np.uint32)
    val, found = lsm.lookup(empty_q)
    assert not found.cpu().numpy().any() and not u32(val).any()
    assert not u32(lsm.count([0], [2**32 - 1])).any()
    off, rk, rv = lsm.range([0, 10], [100, 5])
    assert off.cpu().numpy().tolist() == [0, 0, 0] and rk.numel() == 0
    lsm.cleanup()                                    # empty: no-op
    assert lsm.r == 0
    lsm.insert(np.zeros(0, np.uint32), np.zeros(0, np.uint32))  # n = 0: no-op
    assert lsm.r == 0
    # key out of range: error, nothing applied
    with pytest.raises(g.LSMError) as e:
        lsm.insert(np.array([1, (1 << 31) - 1], np.uint32), np.array([1, 2], np.uint32))
    assert e.value.status == g.LSM_ERR_KEY_RANGE
    assert lsm.r == 0
    lsm.insert(np.arange(b, dtype=np.uint32), np.arange(b, dtype=np.uint32))
    assert lsm.r == 1
    before = lsm.levels()
    for bad in ([2**32 - 1], [5, 2**31]):
        with pytest.raises(g.LSMError):
            lsm.delete(np.array(bad, np.uint32))
    with pytest.raises(g.LSMError):   # multi-batch call: checked as a whole
        keys = np.arange(3 * b, dtype=np.uint32)
        keys[2 * b + 5] = 2**31 + 7
        lsm.insert(keys, keys)
    assert lsm.r == 1
    after = lsm.levels()
    assert before.keys() == after.keys()
    np.testing.assert_array_equal(before[0][0], after[0][0])
    # capacity: 3 batches fit, the 4th does not
    lsm.insert(np.arange(b, dtype=np.uint32) + 1000, np.ones(b, np.uint32))
    lsm.insert(np.arange(b, dtype=np.uint32) + 2000, np.ones(b, np.uint32))
    assert lsm.r == 3
    with pytest.raises(g.LSMError) as e:
        lsm.insert(np.arange(b, dtype=np.uint32), np.ones(b, np.uint32))
    assert e.value.status == g.LSM_ERR_FULL
    assert lsm.r == 3
    # update batch larger than b is an argument error
    with pytest.raises(g.LSMError) as e:
        lsm.update(np.arange(b + 1, dtype=np.uint32), np.zeros(b + 1, np.uint32), np.zeros(b + 1, np.uint8))
    assert e.value.status == g.LSM_ERR_ARG
    # range with too small a buffer: LSM_ERR_CAPACITY with offsets and total
    a = g.as_device_u32([0], 0)
    z = g.as_device_u32([100000], 0)
    offs = torch.empty(2, dtype=torch.int64, device=0)
    ok = torch.empty(4, dtype=torch.int32, device=0)
    s, total = g.lsm_range(lsm.h, a.data_ptr(), z.data_ptr(), 1, offs.data_ptr(), ok.data_ptr(),
                           ok.data_ptr(), 4, torch.cuda.current_stream().cuda_stream)
    assert s == g.LSM_ERR_CAPACITY and total == 3 * b
    assert offs.cpu().numpy().tolist() == [0, 3 * b]
    off, rk, rv = lsm.range([0], [100000], capacity=4)   # retries with the reported total
    assert rk.numel() == 3 * b
    # delete everything, then cleanup -> empty
    lsm2 = g.LSM(b, 8 * b)
    lsm2.insert(np.arange(b, dtype=np.uint32), np.arange(b, dtype=np.uint32))
    lsm2.delete(np.arange(b, dtype=np.uint32))
    lsm2.cleanup()
    assert lsm2.r == 0
    assert not u32(lsm2.count([0], [2**31])).any()
    lsm2.insert(np.array([7], np.uint32), np.array([70], np.uint32))  # padded single op
    assert lsm2.r == 1
    val, found = lsm2.lookup([7, 8])
    assert found.cpu().numpy().tolist() == [1, 0] and u32(val).tolist() == [70, 0]
    assert lsm.device_errors() == 0 and lsm2.device_errors() == 0


def test_max_user_key_and_lookup_mode_agreement(g):
    b = 256
    lsm = g.LSM(b, 16 * b)
    keys = np.array([(1 << 31) - 2, 0, 1, (1 << 30)] * (b // 4), np.uint32)
    vals = np.arange(b, dtype=np.uint32)
    lsm.insert(keys, vals)
    o1 = oracle.MapOracle(b)
    o1.call("insert", keys, vals)
    q = np.array([(1 << 31) - 2, (1 << 31) - 1, 2**32 - 1, 0, 1, 2, 1 << 30], np.uint32)
    for mode in (g.LOOKUP_DIRECT, g.LOOKUP_SORTED, g.LOOKUP_AUTO):
        lsm.set_lookup_mode(mode)
        val, found = lsm.lookup(q)
        ev, ef = o1.lookup(q)
        np.testing.assert_array_equal(found.cpu().numpy(), ef)
        np.testing.assert_array_equal(u32(val), ev)
    assert u32(lsm.count([0], [2**32 - 1])).tolist() == [4]


@pytest.mark.parametrize("b,key_space,nb", [(1, 4, 30), (7, 6, 20), (64, 40, 25), (1000, 300, 12), (4096, 2000, 6)])
def test_ordered_update_batches(g, b, key_space, nb):
    """lsm_update_batch_ordered: the ops of a batch take effect in input
    order (the last op on a key decides, a delete then an insert leaves the
    key inserted), i.e. the batch equals applying its ops one by one to the
    ordered map.  The levels equal those of the plain update batch whose ops
    were pre-resolved to the last op on each key (written out with numpy)."""
    rs = np.random.default_rng(b * 31 + key_space)
    lsm = g.LSM(b, nb * b + b)
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    for t in range(nb):
        n = int(rs.integers(1, b + 1))
        keys = rs.integers(0, key_space, size=n).astype(np.uint32)
        vals = rs.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        dele = (rs.random(n) < 0.4).astype(np.uint8)
        lsm.update_ordered(keys, vals, dele)
        for i in range(n):   # one op at a time
            o1.apply_batch(keys[i:i + 1], vals[i:i + 1], dele[i:i + 1])
        # the same batch pre-resolved: every op a copy of the last op on its key
        last = {}
        for i in range(n):
            last[int(keys[i])] = i
        w = np.array([last[int(k)] for k in keys], np.int64)
        s.call("update", keys[w], vals[w], dele[w])
    assert_levels(lsm, s)
    q = np.arange(key_space + 3, dtype=np.uint32)
    val, found = lsm.lookup(q)
    ev, ef = o1.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    k1 = np.zeros(1, np.uint32)
    k2 = np.full(1, key_space, np.uint32)
    np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))


@pytest.mark.parametrize("case", ["few", "one_bucket_chunked", "almost_full", "pad_key_smallest"])
def test_short_batch_padding(g, case):
    """A short batch is padded with copies of its last op (one run of equal
    key variables, placed before the real elements of that key variable):
    the bucket sort writes the run at its place without sorting it.  Cases:
    a handful of ops; a bucket of real elements too large for shared memory
    (the run is opened inside the chunked path's output); b - 1 ops; the
    padded key smaller than every other key."""
    b = 1 << 16
    rng = np.random.default_rng(len(case))
    lsm = g.LSM(b, 8 * b)
    s = oracle.StructuralOracle(b)
    o1 = oracle.MapOracle(b)
    seen = []
    for t in range(5):
        if case == "few":
            n = 5
            keys = rng.integers(0, 1 << 31, size=n).astype(np.uint32) % np.uint32(0x7FFFFFFE)
        elif case == "one_bucket_chunked":
            n = 6000
            keys = (np.uint32(0x21) << np.uint32(23)) | rng.integers(0, 1 << 12, size=n).astype(np.uint32)
        elif case == "almost_full":
            n = b - 1
            keys = rng.integers(0, 0x7FFFFFFE, size=n).astype(np.uint32)
        else:
            n = 300
            keys = rng.integers(1000, 0x7FFFFFFE, size=n).astype(np.uint32)
            keys[-1] = np.uint32(t)     # the padded op has the smallest key
        vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        dele = (rng.random(n) < 0.3).astype(np.uint8)
        lsm.update(keys, vals, dele)
        s.call("update", keys, vals, dele)
        o1.call("update", keys, vals, dele)
        seen.append(keys)
        assert_levels(lsm, s)
    q = np.concatenate(seen + [rng.integers(0, 0x7FFFFFFE, size=1000).astype(np.uint32)])
    val, found = lsm.lookup(q)
    ev, ef = o1.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    # count / range windows over the long runs of padded copies
    k1 = np.concatenate([q[:2000] - np.minimum(q[:2000], 3), np.zeros(2, np.uint32)])
    k2 = np.concatenate([q[:2000] + 3, np.full(2, 0x7FFFFFFE, np.uint32)])
    np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))
    off, rk, rv = lsm.range(k1, k2)
    eo, ek, evv = o1.range(k1, k2)
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), eo)
    np.testing.assert_array_equal(u32(rk), ek)
    np.testing.assert_array_equal(u32(rv), evv)
    assert lsm.device_errors() == 0


@pytest.mark.parametrize("b,n,key_space", [(1024, 1, 100), (1024, 5000, 3000), (1000, 77777, 1 << 20),
                                           (1 << 16, (3 << 20) + 5, 1 << 21)])
def test_bulk_build(g, b, n, key_space):
    """lsm_bulk_build equals inserting the pairs and cleaning up: the same
    level layout as the oracle's insert + cleanup (sorted live pairs over the
    set bits of ceil(n'/b), placebos after them) and the same answers; the
    largest case sorts more than 2^20 pairs (the pass-by-pass sort)."""
    rng = np.random.default_rng(n)
    keys = rng.integers(0, key_space, size=n).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    lsm = g.LSM(b, n + 2 * b)
    lsm.bulk_build(keys, vals)
    s = oracle.StructuralOracle(b)
    s.call("insert", keys, vals)
    s.cleanup()
    assert_levels(lsm, s)
    o1 = oracle.MapOracle(b)
    o1.call("insert", keys, vals)
    q = np.concatenate([keys[:4096], rng.integers(0, key_space + 10, size=4096).astype(np.uint32)])
    val, found = lsm.lookup(q)
    ev, ef = o1.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    k1 = rng.integers(0, key_space, size=2048).astype(np.uint32)
    k2 = (k1 + rng.integers(0, 64, size=2048)).astype(np.uint32)
    np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))
    with pytest.raises(g.LSMError):
        lsm.bulk_build(keys[:10], vals[:10])   # only into an empty dictionary
    assert lsm.device_errors() == 0


@pytest.mark.parametrize("b,key_space,ncalls,cleanup", [(1, 12, 30, False), (7, 40, 25, False),
                                                        (64, 500, 30, True), (1000, 5000, 20, False)])
def test_successor_predecessor(g, b, key_space, ncalls, cleanup):
    """Order-based neighbour queries against the ordered-map oracle, on logs
    with deletes and overwrites (several versions of a key across levels,
    deleted keys to skip), after a cleanup (placebos at the end), and at the
    edges of the key domain."""
    rng = np.random.default_rng(b * 7 + key_space)
    lsm = g.LSM(b, (ncalls + 2) * b)
    o1 = oracle.MapOracle(b)
    for _ in range(ncalls):
        n = int(rng.integers(1, b + 1))
        keys = rng.integers(0, key_space, size=n).astype(np.uint32)
        vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        dele = (rng.random(n) < 0.35).astype(np.uint8)
        lsm.update(keys, vals, dele)
        o1.call("update", keys, vals, dele)
    if cleanup:
        lsm.cleanup()
    q = np.concatenate([np.arange(key_space + 2, dtype=np.uint32),
                        np.array([0, 0x7FFFFFFE, 0x7FFFFFFF, 0xFFFFFFFF], np.uint32)])
    for succ in (True, False):
        k, v, f = lsm.neighbor(q, successor=succ)
        ek, ev, ef = o1.neighbor(q, successor=succ)
        np.testing.assert_array_equal(f.cpu().numpy(), ef)
        np.testing.assert_array_equal(u32(k), ek)
        np.testing.assert_array_equal(u32(v), ev)
    assert lsm.device_errors() == 0


def test_profile_one_group(g):
    """lsm_profile(h, 2 + group) brackets that group alone; 1 brackets every
    group; out-of-range codes are refused.  The levels are the same either
    way (profiling only adds events)."""
    b = 4096
    rng = np.random.default_rng(11)
    batches = [(rng.integers(0, 1 << 20, size=b).astype(np.uint32),
                rng.integers(0, 1 << 32, size=b, dtype=np.uint64).astype(np.uint32)) for _ in range(7)]
    lsm = g.LSM(b, 8 * b)
    g.lsm_profile(lsm.h, "merge")
    for k, v in batches:
        lsm.insert(k, v)
    prof = g.lsm_profile_read(lsm.h)
    assert prof["merge"]["launches"] == 3          # the batches at r = 1, 3, 5 fold (k = 1, 2, 1)
    assert all(prof[n]["launches"] == 0 for n in g.PROF_GROUPS if n != "merge")
    assert prof["merge"]["ms"] > 0
    g.lsm_profile(lsm.h, True)
    lsm.insert(*batches[0])
    prof = g.lsm_profile_read(lsm.h)                # r = 7: a fold into level 3
    assert [prof[n]["launches"] for n in ("sort", "partition", "merge")] == [1, 1, 1]
    g.lsm_profile(lsm.h, False)
    for bad in (-1, 2 + len(g.PROF_GROUPS)):
        with pytest.raises(g.LSMError):
            g._check(g._lib.lsm_profile(lsm.h, bad), "lsm_profile")
    s = oracle.StructuralOracle(b)
    for k, v in batches + [batches[0]]:
        s.call("insert", k, v)
    assert_levels(lsm, s)
