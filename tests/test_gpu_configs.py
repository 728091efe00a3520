"""Parity at the benchmark's full size and on the sweep recipe (needs a GPU).

* paper-scale: b = 2^20, 128 insert batches (2^27 updates), exactly the
  workload bench.py times, through the same C-ABI calls.  The single full
  level (r = 128) is compared bit for bit with the oracle's closed form;
  all 2^24 lookups and a sample of 2^18 count and 2^18 range queries with the
  offline oracle O2; then cleanup, and the rebuilt levels and lookups again.
* sweep: the configuration-3 recipe (batches with 25 % / 50 % deletes of
  earlier keys, uniform or Zipf(1.1) keys over 2^30, range widths for 8 and
  64 expected results) at sizes the structural oracle replays quickly; levels
  bit-exact after every few batches, queries against O1, cleanup at the end.
"""

import numpy as np
import pytest

import oracle
from paper_1707_05354_gb300 import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g(lsm_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lsm_lib


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_paper_scale_full_size(g):
    cfg = workload.paper_scale()
    b, nb = cfg["b"], cfg["batches"]
    keys = np.empty(nb * b, np.uint32)
    vals = np.empty(nb * b, np.uint32)
    for t in range(nb):
        keys[t * b:(t + 1) * b], vals[t * b:(t + 1) * b] = cfg["batch"](t)
    dk, dv = g.as_device_u32(keys, 0), g.as_device_u32(vals, 0)
    lsm = g.LSM(b, nb * b)
    st = torch.cuda.current_stream().cuda_stream
    for t in range(nb):
        g.lsm_insert_batch(lsm.h, dk.data_ptr() + 4 * t * b, dv.data_ptr() + 4 * t * b, b, st)
    torch.cuda.synchronize()
    assert lsm.r == nb
    calls = [("insert", keys[t * b:(t + 1) * b], vals[t * b:(t + 1) * b], None) for t in range(nb)]

    lv = lsm.levels()
    assert list(lv) == [7]
    ekv, ev = oracle.single_level(calls, b)
    np.testing.assert_array_equal(lv[7][0], ekv)
    np.testing.assert_array_equal(lv[7][1], ev)
    del lv, ekv, ev

    o2 = oracle.OfflineOracle.from_calls(calls, b)
    q = cfg["lookups"](inserted_keys=keys)
    for mode in (g.LOOKUP_DIRECT, g.LOOKUP_SORTED):
        lsm.set_lookup_mode(mode)
        val, found = lsm.lookup(q)
        ev, ef = o2.lookup(q)
        np.testing.assert_array_equal(found.cpu().numpy(), ef)
        np.testing.assert_array_equal(u32(val), ev)
    c1, c2 = cfg["count"]()
    r1, r2 = cfg["range"]()
    c1, c2, r1, r2 = c1[:1 << 18], c2[:1 << 18], r1[:1 << 18], r2[:1 << 18]
    np.testing.assert_array_equal(u32(lsm.count(c1, c2)), o2.count(c1, c2))
    off, rk, rv = lsm.range(r1, r2)
    eo, ek, evv = o2.range(r1, r2)
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), eo)
    np.testing.assert_array_equal(u32(rk), ek)
    np.testing.assert_array_equal(u32(rv), evv)

    lsm.cleanup()
    n_live = o2.size()
    assert lsm.r == -(-n_live // b)
    lv = lsm.levels()
    flat_k = np.concatenate([lv[i][0] for i in sorted(lv)])
    flat_v = np.concatenate([lv[i][1] for i in sorted(lv)])
    np.testing.assert_array_equal(flat_k[:n_live], (o2.keys << 1) | 1)
    np.testing.assert_array_equal(flat_v[:n_live], o2.vals)
    assert np.all(flat_k[n_live:] == oracle.PLACEBO_KV)
    lsm.set_lookup_mode(g.LOOKUP_DIRECT)
    val, found = lsm.lookup(q[:1 << 22])
    ev, ef = o2.lookup(q[:1 << 22])
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    assert lsm.device_errors() == 0


@pytest.mark.parametrize("b_log2,total_log2,delete_frac,dist", [
    (10, 16, 0.25, "uniform"), (10, 16, 0.5, "zipf"), (12, 18, 0.5, "uniform"), (12, 18, 0.25, "zipf"),
    (8, 15, 0.0, "zipf")])
def test_sweep_recipe_bit_exact(g, b_log2, total_log2, delete_frac, dist):
    b = 1 << b_log2
    calls = workload.sweep_updates(1707053503 + b_log2, b, 1 << total_log2, delete_frac, dist)
    lsm = g.LSM(b, len(calls) * b)
    o1 = oracle.MapOracle(b)
    s = oracle.StructuralOracle(b)
    for i, c in enumerate(calls):
        lsm.call(*c)
        o1.call(*c)
        s.call(*c)
        if i % 7 == 6 or i == len(calls) - 1:
            lv = lsm.levels()
            assert lsm.r == s.r
            for lvl in range(40):
                ekv, ev = s.level(lvl)
                if len(ekv):
                    np.testing.assert_array_equal(lv[lvl][0], ekv)
                    np.testing.assert_array_equal(lv[lvl][1], ev)
    rng = np.random.default_rng(b_log2)
    ins = np.concatenate([c[1][c[3] == 0] for c in calls])
    q = workload.lookup_queries(11, ins, 1 << 14, workload.SWEEP_KEY_SPACE)
    for L in (8, 64):
        w = workload.sweep_width(L, o1.size())
        k1 = rng.integers(0, workload.SWEEP_KEY_SPACE - w, size=4096).astype(np.uint32)
        k2 = (k1 + w - 1).astype(np.uint32)
        np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o1.count(k1, k2))
        off, rk, rv = lsm.range(k1, k2)
        eo, ek, evv = o1.range(k1, k2)
        np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), eo)
        np.testing.assert_array_equal(u32(rk), ek)
        np.testing.assert_array_equal(u32(rv), evv)
    val, found = lsm.lookup(q)
    ev, ef = o1.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    lsm.cleanup()
    s.cleanup()
    lv = lsm.levels()
    assert lsm.r == s.r
    for lvl in range(40):
        ekv, ev2 = s.level(lvl)
        if len(ekv):
            np.testing.assert_array_equal(lv[lvl][0], ekv)
            np.testing.assert_array_equal(lv[lvl][1], ev2)
    val, found = lsm.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    assert lsm.device_errors() == 0
