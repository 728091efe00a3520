"""Configuration 3 (update/delete sweep) at the sizes bench.py times (needs a GPU).

The sweep line of bench.py draws its inputs on the device
(``workload.sweep_batches_device``: 2^28 updates per point, uniform or
Zipf(1.1) keys over 2^30, a fraction of deletes of earlier inserts).  Here the
same inputs, from the same generator and seed, go through the same C-ABI
calls (``lsm_update_batch`` once per batch); then they are copied back and
replayed by the CPU oracles:

* the single full level (2^28 / b batches, a power of two) bit for bit against
  the closed form of one level (every resident batch, newest first, §III-B);
* 2^20 lookups (half drawn from the inserted keys) and 2^18 count and 2^18
  range queries at expected result sizes 8 and 512 against the offline
  oracle O2, before and after cleanup;
* after cleanup, the levels against O2's live set (§IV-E: sorted live pairs
  over the set bits of r' = ceil(n'/b), placebos after them).

Two points: b = 2^16 with Zipf keys and 50 % deletes (4096 batches: the hot
keys' buckets exceed shared memory, so the batch sort takes its chunked
path), and b = 2^24 with uniform keys and 25 % deletes (16 batches above the
bucket sort's limit: the radix-sort path).
"""

import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_1707_05354_gb300 import workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g(lsm_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lsm_lib


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def check_queries(g, lsm, o2, q, rng):
    val, found = lsm.lookup(q)
    ev, ef = o2.lookup(q)
    np.testing.assert_array_equal(found.cpu().numpy(), ef)
    np.testing.assert_array_equal(u32(val), ev)
    for L in (8, 512):
        w = workload.sweep_width(L, o2.size())
        k1 = rng.integers(0, workload.SWEEP_KEY_SPACE - w, size=1 << 18).astype(np.uint32)
        k2 = (k1 + w - 1).astype(np.uint32)
        np.testing.assert_array_equal(u32(lsm.count(k1, k2)), o2.count(k1, k2))
        off, rk, rv = lsm.range(k1, k2, capacity=int(1.3 * L * len(k1)) + (1 << 20))
        eo, ek, evv = o2.range(k1, k2)
        np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), eo)
        np.testing.assert_array_equal(u32(rk), ek)
        np.testing.assert_array_equal(u32(rv), evv)


@pytest.mark.parametrize("b_log2,frac,dist", [(16, 0.5, "zipf"), (24, 0.25, "uniform")])
def test_sweep_point_full_size(g, b_log2, frac, dist):
    total = 1 << 28
    b = 1 << b_log2
    nb = total // b
    dev = torch.device("cuda", 0)
    keys, vals, dele = workload.sweep_batches_device(torch, dev, b, nb, frac, dist,
                                                     workload.sweep_device_seed(b_log2, frac))
    lsm = g.LSM(b, total)
    st = torch.cuda.current_stream().cuda_stream
    kp, vp, dp = keys.data_ptr(), vals.data_ptr(), dele.data_ptr()
    for t in range(nb):
        g.lsm_update_batch(lsm.h, kp + 4 * t * b, vp + 4 * t * b, dp + t * b, b, st)
    torch.cuda.synchronize()
    assert lsm.r == nb
    hk, hv, hd = u32(keys), u32(vals), dele.cpu().numpy()
    del keys, vals, dele
    torch.cuda.empty_cache()

    calls = [("update", hk[t * b:(t + 1) * b], hv[t * b:(t + 1) * b], hd[t * b:(t + 1) * b]) for t in range(nb)]
    batch = np.repeat(np.arange(nb, dtype=np.uint32), b)
    # the two oracles run at once (ctypes releases the interpreter lock)
    with cf.ThreadPoolExecutor(2) as ex:
        f_level = ex.submit(oracle.single_level, calls, b)
        f_o2 = ex.submit(oracle.OfflineOracle, hk, hv, hd, batch)
        lv = lsm.levels()
        assert list(lv) == [nb.bit_length() - 1]
        ekv, ev = f_level.result()
        np.testing.assert_array_equal(lv[nb.bit_length() - 1][0], ekv)
        np.testing.assert_array_equal(lv[nb.bit_length() - 1][1], ev)
        del lv, ekv, ev
        o2 = f_o2.result()
    del batch, calls

    ins = hk[hd == 0]
    q = workload.lookup_queries(1707053503 + b_log2, ins, 1 << 20, workload.SWEEP_KEY_SPACE)
    del ins, hk, hv, hd
    rng = np.random.default_rng(b_log2)
    check_queries(g, lsm, o2, q, rng)

    lsm.cleanup()
    n_live = o2.size()
    assert lsm.r == -(-n_live // b)
    lv = lsm.levels()
    flat_k = np.concatenate([lv[i][0] for i in sorted(lv)])
    flat_v = np.concatenate([lv[i][1] for i in sorted(lv)])
    del lv
    np.testing.assert_array_equal(flat_k[:n_live], (o2.keys << 1) | 1)
    np.testing.assert_array_equal(flat_v[:n_live], o2.vals)
    assert np.all(flat_k[n_live:] == oracle.PLACEBO_KV)
    del flat_k, flat_v
    check_queries(g, lsm, o2, q, np.random.default_rng(b_log2 + 1))
    assert lsm.device_errors() == 0
    lsm.close()
