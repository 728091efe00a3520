"""Pins of the CPU oracle against things other than itself (no GPU).

* the hand-derived walkthrough of Fig. 1 / §III-A / §IV-E (tests/golden),
* each batch-semantics rule of §III-A on a hand-written scenario,
* the brute-force answer straight from the op log (oracle.brute) on thousands
  of random tiny logs,
* closed forms (inserts of distinct keys only: count = keys in the interval),
* the building invariants of §III-D and the binary-counter property of §III-B
  on the structural model's levels,
* O1 <-> O2 <-> S agreement, and cleanup invariance (§III-F).
"""

import numpy as np
import pytest

import oracle
from oracle import brute
from tests.walkthrough import levels_lookup, parse

MAXK = (1 << 31) - 2


def _levels_newest_first(s, upto=40):
    return [s.level(i) for i in range(upto) if len(s.level(i)[0])]


# ---------------------------------------------------------------- golden --
def test_walkthrough_on_oracles():
    b, steps = parse("fig1_walkthrough.txt")
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    log = []  # list of batches for the brute force
    for st in steps:
        if st[0] == "op":
            _, kind, keys, vals, dels = st
            o1.call(kind, keys, vals, dels)
            s.call(kind, keys, vals, dels)
            for k, v, d in oracle.split_call(kind, keys, vals, b, dels):
                n = len(k)
                log.append([(int(k[min(i, n - 1)]), int(v[min(i, n - 1)]), int(d[min(i, n - 1)])) for i in range(b)])
        elif st[0] == "cleanup":
            s.cleanup()
        elif st[0] == "r":
            assert s.r == st[1]
        elif st[0] == "level":
            kv, v = s.level(st[1])
            if st[2] is None:
                assert len(kv) == 0
            else:
                np.testing.assert_array_equal(kv, st[2])
                np.testing.assert_array_equal(v, st[3])
        elif st[0] == "lookup":
            val, found = o1.lookup(st[1])
            np.testing.assert_array_equal(found, st[3])
            np.testing.assert_array_equal(val, st[2])
            lv = _levels_newest_first(s)
            for q, ev, ef in zip(st[1], st[2], st[3]):
                assert levels_lookup(lv, int(q)) == (int(ef), int(ev))
                assert brute.state_of(log, int(q)) == (bool(ef), int(ev))
        elif st[0] == "count":
            _, k1, k2, n = st
            assert int(o1.count([k1], [min(k2, 0xFFFFFFFF)])[0]) == n
            assert brute.count(log, k1, k2) == n
        elif st[0] == "range":
            _, k1, k2, pairs = st
            off, keys, vals = o1.range([k1], [min(k2, 0xFFFFFFFF)])
            assert list(zip(keys.tolist(), vals.tolist())) == pairs
            assert brute.range_query(log, k1, k2) == pairs


# ------------------------------------------------------------ §III-A rules --
def _run(b, calls):
    o1 = oracle.MapOracle(b)
    for kind, k, v, d in calls:
        o1.call(kind, np.array(k, np.uint32), None if v is None else np.array(v, np.uint32),
                None if d is None else np.array(d, np.uint8))
    return o1


def test_rule3_latest_batch_wins():
    o1 = _run(2, [("insert", [5, 6], [1, 2], None), ("insert", [5, 7], [3, 4], None)])
    val, found = o1.lookup([5, 6, 7])
    assert found.tolist() == [1, 1, 1] and val.tolist() == [3, 2, 4]


def test_rule4_last_insert_in_batch_wins():
    o1 = _run(4, [("insert", [9, 9, 9, 1], [10, 20, 30, 40], None)])
    assert o1.lookup([9])[0].tolist() == [30]


def test_rule5_delete_removes_all_and_repeats_are_one():
    o1 = _run(3, [("insert", [4, 5, 6], [1, 1, 1], None), ("insert", [4, 8, 9], [2, 2, 2], None),
                  ("delete", [4, 4, 4], None, None)])
    assert o1.lookup([4])[1].tolist() == [0]
    assert o1.count([0], [100]).tolist() == [4]


@pytest.mark.parametrize("order", [[0, 1], [1, 0]])
def test_rule6_insert_and_delete_in_one_batch_is_deleted(order):
    keys, vals, dels = np.array([7, 7]), np.array([5, 0]), np.array([0, 1])
    o1 = _run(2, [("insert", [7, 8], [1, 1], None),
                  ("update", keys[order], vals[order], dels[order])])
    assert o1.lookup([7])[1].tolist() == [0]
    assert o1.lookup([8])[0].tolist() == [1]


def test_deleted_then_reinserted_key_returns():
    o1 = _run(1, [("insert", [3], [1], None), ("delete", [3], None, None), ("insert", [3], [9], None)])
    assert o1.lookup([3])[0].tolist() == [9] and o1.lookup([3])[1].tolist() == [1]


# ---------------------------------------------------------- random tiny logs --
def _random_calls(g, b, ncalls, key_space=16):
    calls = []
    for _ in range(ncalls):
        kind = g.choice(["insert", "delete", "update"])
        if kind == "update":
            n = int(g.integers(1, b + 1))
        else:
            n = int(g.integers(1, 3 * b + 1))
        keys = g.integers(0, key_space, size=n).astype(np.uint32)
        vals = g.integers(0, 1000, size=n).astype(np.uint32)
        dels = (g.random(n) < 0.3).astype(np.uint8)
        calls.append((kind, keys, vals, dels))
    return calls


def _log_of(calls, b):
    log = []
    for kind, k, v, d in calls:
        for kk, vv, dd in oracle.split_call(kind, k, v, b, d):
            n = len(kk)
            log.append([(int(kk[min(i, n - 1)]), int(vv[min(i, n - 1)]), int(dd[min(i, n - 1)]))
                        for i in range(b)])
    return log


@pytest.mark.parametrize("b", [1, 2, 3, 4, 8])
def test_map_oracle_vs_brute_force(b):
    g = np.random.default_rng(1000 + b)
    for trial in range(60):
        calls = _random_calls(g, b, int(g.integers(1, 12)))
        o1 = oracle.MapOracle(b)
        for c in calls:
            o1.call(*c)
        log = _log_of(calls, b)
        q = np.arange(18, dtype=np.uint32)
        val, found = o1.lookup(q)
        for i, qq in enumerate(q):
            assert brute.state_of(log, int(qq)) == (bool(found[i]), int(val[i]))
        k1 = g.integers(0, 18, size=20).astype(np.uint32)
        k2 = g.integers(0, 18, size=20).astype(np.uint32)
        cnt = o1.count(k1, k2)
        off, rk, rv = o1.range(k1, k2)
        for i in range(20):
            assert int(cnt[i]) == brute.count_by_enumeration(log, int(k1[i]), int(k2[i]))
            ref = brute.range_query(log, int(k1[i]), int(k2[i]))
            got = list(zip(rk[off[i]:off[i + 1]].tolist(), rv[off[i]:off[i + 1]].tolist()))
            assert got == ref
        # successor / predecessor: the nearest live key on each side, checked
        # by testing every key the log mentions (and the closed form on an
        # enumerated key range)
        qn = np.concatenate([np.arange(19, dtype=np.uint32), np.array([0x7FFFFFFF, 0xFFFFFFFF], np.uint32)])
        for succ in (True, False):
            nk, nv, nf = o1.neighbor(qn, successor=succ)
            for i, qq in enumerate(qn.tolist()):
                ref = brute.neighbor(log, qq, successor=succ)
                assert (ref is not None) == bool(nf[i])
                if ref is not None:
                    assert (int(nk[i]), int(nv[i])) == ref
                    live = [k for k in range(18) if brute.state_of(log, k)[0]]
                    side = [k for k in live if (k >= qq if succ else k <= qq)]
                    assert int(nk[i]) == (min(side) if succ else max(side))


@pytest.mark.parametrize("b", [1, 2, 3, 5, 8])
def test_structural_oracle_invariants_and_queries(b):
    g = np.random.default_rng(2000 + b)
    for trial in range(25):
        calls = _random_calls(g, b, int(g.integers(1, 16)), key_space=24)
        s = oracle.StructuralOracle(b)
        o1 = oracle.MapOracle(b)
        for c in calls:
            s.call(*c)
            o1.call(*c)
        r = s.r
        lv = []
        for i in range(40):
            kv, v, bt = s.level(i, with_batch=True)
            # §III-B: level i is full (b * 2^i elements) iff bit i of r is set
            assert len(kv) == (b << i if (r >> i) & 1 else 0)
            if not len(kv):
                continue
            key = kv >> 1
            assert np.all(np.diff(key.astype(np.int64)) >= 0)            # invariant 1
            same = key[1:] == key[:-1]
            assert np.all(bt[1:][same] <= bt[:-1][same])                  # invariant 2
            tie = same & (bt[1:] == bt[:-1])
            assert np.all((kv[1:] & 1)[tie] >= (kv[:-1] & 1)[tie])         # invariant 3
            lv.append((kv, v))
        assert sum(len(x[0]) for x in lv) == r * b
        for q in range(26):
            exp_v, exp_f = o1.lookup([q])
            assert levels_lookup(lv, q) == (int(exp_f[0]), int(exp_v[0]))


def test_offline_oracle_matches_map_oracle():
    g = np.random.default_rng(7)
    for b in (4, 16, 64):
        calls = _random_calls(g, b, 40, key_space=500)
        o1 = oracle.MapOracle(b)
        for c in calls:
            o1.call(*c)
        o2 = oracle.OfflineOracle.from_calls(calls, b)
        k, v = o1.items()
        np.testing.assert_array_equal(o2.keys, k)
        np.testing.assert_array_equal(o2.vals, v)
        q = g.integers(0, 520, size=300).astype(np.uint32)
        for a, c in zip(o1.lookup(q), o2.lookup(q)):
            np.testing.assert_array_equal(a, c)
        k1 = g.integers(0, 520, size=200).astype(np.uint32)
        k2 = (k1 + g.integers(-5, 60, size=200)).clip(0, 2**32 - 1).astype(np.uint32)
        np.testing.assert_array_equal(o1.count(k1, k2), o2.count(k1, k2))
        for a, c in zip(o1.range(k1, k2), o2.range(k1, k2)):
            np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("dist,frac", [("uniform", 0.25), ("zipf", 0.5)])
def test_oracles_agree_on_sweep_recipe(dist, frac):
    """The config-3 recipe at a small size (mixed batches, deletes of earlier
    inserts, Zipf-skewed keys with heavy repeats): O1, O2, S and brute force
    give the same live set and the same query answers."""
    from paper_1707_05354_gb300 import workload as W
    b = 64
    calls = W.sweep_updates(3, b, 12 * b, frac, dist)
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    for c in calls:
        o1.call(*c)
        s.call(*c)
    o2 = oracle.OfflineOracle.from_calls(calls, b)
    k, v = o1.items()
    np.testing.assert_array_equal(o2.keys, k)
    np.testing.assert_array_equal(o2.vals, v)
    g = np.random.default_rng(1)
    ks = np.concatenate([c[1] for c in calls])
    q = np.concatenate([ks[g.integers(0, len(ks), size=200)], g.integers(0, 1 << 30, size=100)]).astype(np.uint32)
    ev, ef = o1.lookup(q)
    for a, c in zip((ev, ef), o2.lookup(q)):
        np.testing.assert_array_equal(a, c)
    # brute force from the raw log, and the lookup rule of §III-D on S's levels
    log = [list(zip(c[1].tolist(), c[2].tolist(), c[3].tolist())) for c in calls]
    levels = [s.level(i) for i in range(12)]
    for i, qq in enumerate(q.tolist()):
        assert brute.state_of(log, qq) == (bool(ef[i]), int(ev[i]))
        assert levels_lookup(levels, qq) == (int(ef[i]), int(ev[i]))
    k1 = np.sort(ks[g.integers(0, len(ks), size=100)])
    k2 = (k1.astype(np.int64) + g.integers(0, 1 << 24, size=100)).clip(0, (1 << 31) - 2).astype(np.uint32)
    np.testing.assert_array_equal(o1.count(k1, k2), o2.count(k1, k2))
    for a, c in zip(o1.range(k1, k2), o2.range(k1, k2)):
        np.testing.assert_array_equal(a, c)


# ------------------------------------------------------------ closed forms --
def test_closed_form_distinct_inserts():
    g = np.random.default_rng(11)
    keys = g.choice(1 << 20, size=5000, replace=False).astype(np.uint32)
    vals = g.integers(0, 2**32, size=5000, dtype=np.uint64).astype(np.uint32)
    o1 = oracle.MapOracle(256)
    o1.call("insert", keys, vals)
    val, found = o1.lookup(keys)
    assert found.all() and np.array_equal(val, vals)
    k1 = g.integers(0, 1 << 20, size=500).astype(np.uint32)
    k2 = (k1.astype(np.int64) + g.integers(0, 5000, size=500)).astype(np.uint32)
    exp = np.array([np.count_nonzero((keys >= a) & (keys <= c)) for a, c in zip(k1, k2)])
    np.testing.assert_array_equal(o1.count(k1, k2), exp)
    o1.call("delete", keys)
    assert o1.size() == 0 and not o1.count([0], [2**31]).any()


def test_key_bounds_and_clamp():
    o1 = _run(2, [("insert", [MAXK, 0], [5, 6], None)])
    assert o1.count([0], [0xFFFFFFFF]).tolist() == [2]
    assert o1.count([MAXK], [MAXK]).tolist() == [1]
    assert o1.count([5], [4]).tolist() == [0]
    assert o1.lookup([MAXK + 1, 0xFFFFFFFF])[1].tolist() == [0, 0]


# ----------------------------------------------------------------- cleanup --
@pytest.mark.parametrize("b", [1, 3, 4, 7])
def test_cleanup_model(b):
    g = np.random.default_rng(3000 + b)
    for trial in range(20):
        calls = _random_calls(g, b, int(g.integers(1, 14)), key_space=30)
        s = oracle.StructuralOracle(b)
        o1 = oracle.MapOracle(b)
        for c in calls:
            s.call(*c)
            o1.call(*c)
        s.cleanup()
        n_live = o1.size()
        r2 = -(-n_live // b)
        assert s.r == r2
        flat_kv = np.concatenate([s.level(i)[0] for i in range(40)])
        flat_v = np.concatenate([s.level(i)[1] for i in range(40)])
        k, v = o1.items()
        pad = r2 * b - n_live
        assert 0 <= pad < b or (n_live == 0 and pad == 0)
        np.testing.assert_array_equal(flat_kv[:n_live], (k << 1) | 1)
        np.testing.assert_array_equal(flat_v[:n_live], v)
        assert np.all(flat_kv[n_live:] == oracle.PLACEBO_KV) and not flat_v[n_live:].any()
        lv = _levels_newest_first(s)
        for q in range(32):
            ev, ef = o1.lookup([q])
            assert levels_lookup(lv, q) == (int(ef[0]), int(ev[0]))
        # further batches keep working after a cleanup
        more = _random_calls(g, b, 3, key_space=30)
        for c in more:
            s.call(*c)
            o1.call(*c)
        lv = _levels_newest_first(s)
        for q in range(32):
            ev, ef = o1.lookup([q])
            assert levels_lookup(lv, q) == (int(ef[0]), int(ev[0]))


# ------------------------------------------------- single-level closed form --
@pytest.mark.parametrize("b,nb", [(1, 8), (3, 4), (4, 16), (16, 32), (5, 2)])
def test_single_level_closed_form_matches_structural_replay(b, nb):
    """With 2^m resident batches all elements sit in level m (§III-B); the
    closed form (key asc, batch desc, tombstone first, later op first) must
    equal the literal cascade of Fig. 2(a) / Fig. 3."""
    g = np.random.default_rng(77 + b * nb)
    calls = []
    for _ in range(nb):
        n = int(g.integers(1, b + 1))
        calls.append(("update", g.integers(0, 6 * b, size=n).astype(np.uint32),
                      g.integers(0, 1000, size=n).astype(np.uint32), (g.random(n) < 0.3).astype(np.uint8)))
    s = oracle.StructuralOracle(b)
    for c in calls:
        s.call(*c)
    m = nb.bit_length() - 1
    kv, v = oracle.single_level(calls, b)
    ekv, ev = s.level(m)
    np.testing.assert_array_equal(kv, ekv)
    np.testing.assert_array_equal(v, ev)
