"""The serving engine: every request's result equals running it alone
against the ordered-map oracle O1 at its linearisation point.

The server reports, per request, the sequence number of the group it was
admitted in.  The oracle replays the requests in that order (requests of
one update group in their admission order, each applied as one batch: a
request holds one kind of op, so batch and one-by-one application agree)
and answers every retrieval on the state it reaches; lookups, counts and
range results must match bit for bit.  A small key space makes requests
collide on keys, so coalesced update batches mix inserts and deletes of the
same keys (the ordered batch must keep arrival order).  Covered: the
continuous and the fixed policy, a budget so small that cleanups run and
update groups get refused, and real-time order (a request that completed
before another arrived is linearised before it).
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


def replay_and_check(g, b, pools, preload, trace, out):
    a, pv, c = pools
    kind, arrival, start, size = trace
    o1 = oracle.MapOracle(b)
    if preload is not None:
        o1.call("insert", preload[0], preload[1])
    order = np.lexsort((np.arange(len(kind)), out["order"]))
    checked = 0
    for i in order:
        s, m = int(start[i]), int(size[i])
        k = int(kind[i])
        o = int(out["res_off"][i])
        if k in (g.REQ_INSERT, g.REQ_DELETE):
            if out["status"][i] != g.LSM_OK:
                assert out["status"][i] == g.LSM_ERR_BUDGET
                continue
            if k == g.REQ_INSERT:
                o1.apply_batch(a[s:s + m], pv[s:s + m], np.zeros(m, np.uint8))
            else:
                o1.apply_batch(a[s:s + m], np.zeros(m, np.uint32), np.ones(m, np.uint8))
            continue
        assert out["status"][i] == g.LSM_OK
        if k == g.REQ_LOOKUP:
            ev, ef = o1.lookup(a[s:s + m])
            np.testing.assert_array_equal(out["found"][o:o + m], ef, err_msg="lookup request %d" % i)
            np.testing.assert_array_equal(out["val"][o:o + m], ev, err_msg="lookup request %d" % i)
        elif k == g.REQ_COUNT:
            np.testing.assert_array_equal(out["val"][o:o + m], o1.count(a[s:s + m], c[s:s + m]),
                                          err_msg="count request %d" % i)
        else:
            eo, ek, evv = o1.range(a[s:s + m], c[s:s + m])
            cnt = np.diff(eo.astype(np.int64))
            np.testing.assert_array_equal(out["val"][o:o + m], cnt, err_msg="range request %d" % i)
            for t in range(m):
                rs = int(out["range_start"][o + t])
                n_t = int(cnt[t])
                np.testing.assert_array_equal(out["rk"][rs:rs + n_t], ek[int(eo[t]):int(eo[t + 1])])
                np.testing.assert_array_equal(out["rv"][rs:rs + n_t], evv[int(eo[t]):int(eo[t + 1])])
        checked += 1
    return checked


def real_time_order_holds(out, arrival):
    """If request A completed before request B arrived, A's group was
    admitted before B's: order(A) < order(B)."""
    done, order = out["done_us"], out["order"].astype(np.int64)
    idx = np.argsort(done)
    # for every B, all A with done(A) < arrival(B) have order(A) < order(B):
    # compare B's order with the max order among requests done before it arrived
    done_sorted = done[idx]
    prefix_max = np.maximum.accumulate(order[idx])
    pos = np.searchsorted(done_sorted, arrival, side="left")
    ok = np.ones(len(arrival), bool)
    has = pos > 0
    ok[has] = prefix_max[pos[has] - 1] < order[has]
    return bool(ok.all())


def small_setup(seed, n_req, key_space, rate, size_hi_log2=8.0):
    pools = workload.serving_pools(seed=seed, n=1 << 15, key_space=key_space, width=64)
    trace = workload.serving_trace(seed=seed, n_req=n_req, rate=rate, pool_n=1 << 15, size_hi_log2=size_hi_log2)
    g_ = workload.rng(seed, 3, 99)
    pre = (workload.u32(g_, 4096, 0, key_space), workload.u32(g_, 4096))
    return pools, trace, pre


@pytest.mark.parametrize("policy,slots", [(0, 3), (1, 1), (0, 1)])
def test_serving_linearisable(g, policy, slots):
    b = 1024
    pools, trace, pre = small_setup(1707053505 + policy + 10 * slots, 3000, 1 << 14, 6.0e4)
    srv = g.Server(b, 1 << 30, flush_us=300.0, group_keys=4096, slots=slots, range_cap=1 << 18, policy=policy)
    srv.set_pool(*pools)
    srv.preload(*pre)
    out = srv.run(*trace, keep_results=True)
    assert (out["status"] == g.LSM_OK).all()
    assert out["update_batches"] > 0 and out["retrieval_groups"] > 0
    n = replay_and_check(g, b, pools, pre, trace, out)
    assert n > 1000
    assert real_time_order_holds(out, trace[1])
    # groups really coalesced requests
    assert out["update_batches"] + out["retrieval_groups"] < len(trace[0])


def test_serving_large_groups_sorted(g):
    """Requests that arrive almost at once form retrieval groups of tens of
    thousands of keys, which the server processes in key order (sorted
    lookups, counts and ranges with their positions)."""
    b = 1 << 15
    pools, trace, pre = small_setup(1707053577, 3000, 1 << 14, 1.0e7, size_hi_log2=12.0)
    srv = g.Server(b, 1 << 31, flush_us=2000.0, group_keys=1 << 17, slots=2, range_cap=1 << 21)
    srv.set_pool(*pools)
    srv.preload(*pre)
    out = srv.run(*trace, keep_results=True)
    assert (out["status"] == g.LSM_OK).all()
    sizes = trace[3].astype(np.int64)
    assert out["retrieval_groups"] < 200 and sizes[trace[0] >= 2].sum() > (1 << 17)
    replay_and_check(g, b, pools, pre, trace, out)
    assert real_time_order_holds(out, trace[1])


def test_serving_budget_cleanup_and_refusal(g):
    """A budget that leaves the dictionary few levels: cleanups run, and
    update groups are refused while the live data fills every level; the
    refused requests change nothing."""
    b = 1024
    pools, trace, pre = small_setup(1707053555, 2500, 1 << 14, 8.0e4)
    # the smallest budget that still gives a few levels
    lv = None
    for budget in [(64 << 20) + (k << 17) for k in range(1, 64)]:
        try:
            srv = g.Server(b, budget, flush_us=200.0, group_keys=2048, slots=2, range_cap=1 << 12)
        except g.LSMError:
            continue
        lv = srv.stats()["levels"]
        if lv >= 3:
            break
        srv.close()
    assert lv is not None and 3 <= lv <= 5
    srv.set_pool(*pools)
    srv.preload(*pre)
    out = srv.run(*trace, keep_results=True)
    assert out["cleanups"] >= 1
    replay_and_check(g, b, pools, pre, trace, out)
    assert real_time_order_holds(out, trace[1])
