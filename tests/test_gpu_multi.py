"""Parity of the batched form (many dictionaries per round) with the oracle.

Every instance of a multi handle must hold exactly what a separate dictionary
with the same batch size would hold after the same batches: its levels are
compared bit for bit with the structural oracle S and its lookups with the
ordered-map oracle O1 (or the offline oracle O2 at the full configuration
size).  Covered: uneven batch sizes (not powers of two, a batch of 1), short
and empty batches, every merge tile / prefix-index resolution the tuner can
pick, graph replay vs plain launches, per-instance refusals (bad key, count
> b, full) leaving the other instances untouched, custom query offsets.
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


def inst_call(wl, keys, vals, dele, i, n=None):
    s = int(wl.off[i])
    b = int(wl.sizes[i])
    n = b if n is None else n
    return ("update", keys[s:s + n], vals[s:s + n], dele[s:s + n])


def check_levels(m, s_oracles, idx):
    for i in idx:
        lv = m.levels(i)
        s = s_oracles[i]
        assert m.stats(i)["r"] == s.r, i
        for lvl in range(16):
            ekv, ev = s.level(lvl)
            if len(ekv):
                np.testing.assert_array_equal(lv[lvl][0], ekv, err_msg="inst %d level %d" % (i, lvl))
                np.testing.assert_array_equal(lv[lvl][1], ev, err_msg="inst %d level %d" % (i, lvl))
            else:
                assert lvl not in lv


@pytest.mark.parametrize("tile,bin_log2,graph", [(2048, 3, True), (1024, 2, True), (2048, 5, False),
                                                 (1024, 6, True)])
def test_multi_rounds_bit_exact(g, tile, bin_log2, graph):
    sizes = workload.batched_sizes(seed=17 + bin_log2, n_inst=24, lo_log2=5, hi_log2=12)
    sizes[0] = 1            # a batch of one
    sizes[1] = 4096         # exactly one sort tile
    sizes[2] = 4097         # a ragged second tile
    wl = workload.BatchedWorkload(seed=99, sizes=sizes, rounds=11)
    m = g.MultiLSM(list(sizes), max_batches=15, tuning=[(tile, bin_log2)] * len(sizes))
    m.set_graph(graph)
    s_or = [oracle.StructuralOracle(int(b)) for b in sizes]
    o1 = [oracle.MapOracle(int(b)) for b in sizes]
    for t in range(wl.rounds):
        keys, vals, dele, q = wl.round(t)
        m.update(keys, vals, dele)
        status, flags = m.sync()
        assert status == g.LSM_OK and not any(flags)
        for i in range(wl.n):
            c = inst_call(wl, keys, vals, dele, i)
            s_or[i].call(*c)
            o1[i].call(*c)
        if t in (0, 1, 2, 5, 7, 10):
            check_levels(m, s_or, range(wl.n))
        val, found = m.lookup(q, wl.off)
        torch.cuda.synchronize()
        val, found = u32(val), found.cpu().numpy()
        for i in range(wl.n):
            s = slice(int(wl.off[i]), int(wl.off[i + 1]))
            ev, ef = o1[i].lookup(q[s])
            np.testing.assert_array_equal(found[s], ef, err_msg="round %d inst %d" % (t, i))
            np.testing.assert_array_equal(val[s], ev, err_msg="round %d inst %d" % (t, i))


def test_multi_round_graph_matches_separate_calls(g):
    """lsm_multi_round (update + lookup in one replay) == update then lookup."""
    sizes = workload.batched_sizes(seed=5, n_inst=12, lo_log2=6, hi_log2=13)
    wl_a = workload.BatchedWorkload(seed=7, sizes=sizes, rounds=6)
    ma = g.MultiLSM(list(sizes), max_batches=8)
    mb = g.MultiLSM(list(sizes), max_batches=8)
    st = torch.cuda.current_stream().cuda_stream
    n = wl_a.total
    dk = torch.empty(n, dtype=torch.int32, device=0)
    dv = torch.empty(n, dtype=torch.int32, device=0)
    dd = torch.empty(n, dtype=torch.uint8, device=0)
    dq = torch.empty(n, dtype=torch.int32, device=0)
    off = torch.as_tensor(wl_a.off, dtype=torch.int64).to(0)
    val = torch.empty(n, dtype=torch.int32, device=0)
    fnd = torch.empty(n, dtype=torch.uint8, device=0)
    for t in range(wl_a.rounds):
        keys, vals, dele, q = wl_a.round(t)
        dk.copy_(torch.from_numpy(keys.view(np.int32)))
        dv.copy_(torch.from_numpy(vals.view(np.int32)))
        dd.copy_(torch.from_numpy(dele))
        dq.copy_(torch.from_numpy(q.view(np.int32)))
        # same buffers every round: the captured graph is replayed
        g.lsm_multi_round(ma.h, dk.data_ptr(), dv.data_ptr(), dd.data_ptr(), None, dq.data_ptr(),
                          off.data_ptr(), n, val.data_ptr(), fnd.data_ptr(), st)
        mb.update(keys, vals, dele)
        vb, fb = mb.lookup(q, wl_a.off)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u32(val), u32(vb))
        np.testing.assert_array_equal(fnd.cpu().numpy(), fb.cpu().numpy())
    assert g.lsm_multi_get_option(ma.h, g.LSM_MULTI_OPT_GRAPH_KERNELS) >= 8
    for i in range(wl_a.n):
        la, lb = ma.levels(i), mb.levels(i)
        assert la.keys() == lb.keys()
        for l in la:
            np.testing.assert_array_equal(la[l][0], lb[l][0])
            np.testing.assert_array_equal(la[l][1], lb[l][1])


def test_multi_partial_empty_and_refused_batches(g):
    sizes = np.array([300, 1000, 77, 4100, 2048, 513], np.int64)
    n = len(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)])
    m = g.MultiLSM(list(sizes), max_batches=3)
    s_or = [oracle.StructuralOracle(int(b)) for b in sizes]
    o1 = [oracle.MapOracle(int(b)) for b in sizes]
    rs = np.random.default_rng(3)
    for t in range(6):
        keys = rs.integers(0, 5000, size=off[-1]).astype(np.uint32)
        vals = rs.integers(0, 1 << 32, size=off[-1], dtype=np.uint64).astype(np.uint32)
        dele = (rs.random(off[-1]) < 0.3).astype(np.uint8)
        counts = np.array([rs.integers(0, b + 1) for b in sizes], np.uint32)
        counts[t % n] = 0                       # no batch for one instance
        bad = (t + 2) % n
        if t in (1, 4):                         # an out-of-range key refuses that instance only
            keys[off[bad] + max(0, int(counts[bad]) - 1)] = 0x7FFFFFFF
            counts[bad] = max(1, counts[bad])
        over = (t + 3) % n
        if t == 2:
            counts[over] = sizes[over] + 1      # more ops than b: refused
        m.update(keys, vals, dele, counts)
        status, flags = m.sync()
        expect = [0] * n
        for i in range(n):
            c = int(counts[i])
            if c == 0:
                continue
            if t == 2 and i == over:
                expect[i] = g.MULTI_FLAG_ARG
                continue
            if t in (1, 4) and i == bad:
                expect[i] = g.MULTI_FLAG_BAD_KEY
                continue
            if s_or[i].r >= 3:                   # capacity: 3 batches (levels 0, 1)
                expect[i] = g.MULTI_FLAG_FULL
                continue
            call = ("update", keys[off[i]:off[i] + c], vals[off[i]:off[i] + c], dele[off[i]:off[i] + c])
            s_or[i].call(*call)
            o1[i].call(*call)
        assert flags == expect, (t, flags, expect)
        assert (status == g.LSM_OK) == (not any(expect))
        check_levels(m, s_or, range(n))
    # uneven query counts per instance, one instance with none
    qn = np.array([5, 0, 700, 1, 64, 3000], np.int64)
    qoff = np.concatenate([[0], np.cumsum(qn)])
    q = rs.integers(0, 6000, size=qoff[-1]).astype(np.uint32)
    q[-1] = 0xFFFFFFFF                          # out of the key domain: absent
    val, found = m.lookup(q, qoff)
    torch.cuda.synchronize()
    val, found = u32(val), found.cpu().numpy()
    for i in range(n):
        s = slice(int(qoff[i]), int(qoff[i + 1]))
        ev, ef = o1[i].lookup(q[s])
        np.testing.assert_array_equal(found[s], ef)
        np.testing.assert_array_equal(val[s], ev)


def test_multi_reset(g):
    sizes = [100, 2000, 33]
    m = g.MultiLSM(sizes, max_batches=4)
    tot = sum(sizes)
    keys = np.arange(tot, dtype=np.uint32)
    m.update(keys, keys)
    assert m.sync()[0] == g.LSM_OK
    assert m.stats(1)["r"] == 1
    m.reset()
    assert all(m.stats(i)["r"] == 0 for i in range(3))
    val, found = m.lookup(keys, [0, 100, 2100, tot])
    torch.cuda.synchronize()
    assert found.sum().item() == 0
    m.update(keys[::-1].copy(), keys)
    assert m.sync()[0] == g.LSM_OK
    s = oracle.StructuralOracle(2000)
    s.call("update", keys[::-1][100:2100], keys[100:2100], np.zeros(2000, np.uint8))
    np.testing.assert_array_equal(m.levels(1)[0][0], s.level(0)[0])


@pytest.mark.slow
def test_multi_config_full_size(g):
    """The full batched configuration (256 instances, b log-uniform in
    [2^10, 2^18], 32 rounds, 20 % deletes): a sample of instances checked
    bit for bit (levels vs S) and by lookups (vs O2) after the last round,
    every instance's lookups of the last round vs O2 for the sample."""
    wl = workload.BatchedWorkload()
    m = g.MultiLSM(list(wl.sizes), max_batches=wl.rounds)
    sample = sorted(set([0, 1, int(np.argmin(wl.sizes)), int(np.argmax(wl.sizes))] + list(range(7, wl.n, 37))))
    calls = {i: [] for i in sample}
    q = None
    for t in range(wl.rounds):
        keys, vals, dele, q = wl.round(t)
        m.update(keys, vals, dele)
        for i in sample:
            calls[i].append(inst_call(wl, keys, vals, dele, i))
    status, flags = m.sync()
    assert status == g.LSM_OK and not any(flags)
    val, found = m.lookup(q, wl.off)
    torch.cuda.synchronize()
    val, found = u32(val), found.cpu().numpy()
    for i in sample:
        b = int(wl.sizes[i])
        assert m.stats(i)["r"] == wl.rounds
        lv = m.levels(i)
        assert list(lv) == [5]
        ekv, ev = oracle.single_level(calls[i], b)
        np.testing.assert_array_equal(lv[5][0], ekv)
        np.testing.assert_array_equal(lv[5][1], ev)
        o2 = oracle.OfflineOracle.from_calls(calls[i], b)
        s = slice(int(wl.off[i]), int(wl.off[i + 1]))
        ev, ef = o2.lookup(q[s])
        np.testing.assert_array_equal(found[s], ef)
        np.testing.assert_array_equal(val[s], ev)
