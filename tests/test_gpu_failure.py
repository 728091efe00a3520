"""Error paths of the failure design, driven without faulting a GPU (needs a GPU).

* A device wait that runs out: ``lsm_debug_wait_flag`` spins, with the bounded
  spin every wait of the library uses, on a device word nothing writes.  The
  wait must give up after its limit and report LSM_ERR_TIMEOUT, and the
  context must stay usable; the same wait on a word that is set returns at
  once.
* Allocation failures: ``lsm_debug_fail_allocs`` makes the library's next
  allocations fail on the host.  ``lsm_create`` and ``lsm_multi_create``, failing
  at each of their allocations in turn, must return LSM_ERR_OOM and leak
  nothing; ``lsm_cleanup`` and ``lsm_bulk_build``, failing at each of theirs,
  must return LSM_ERR_OOM and leave the dictionary as it was (all or nothing),
  and succeed once the failures are disarmed.
"""

import time

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
    yield lsm_lib
    lsm_lib.lsm_debug_fail_allocs(0, 0)


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def snapshot(lsm):
    lv = lsm.levels()
    return lsm.r, {i: (k.copy(), v.copy()) for i, (k, v) in lv.items()}


def assert_same(lsm, snap):
    r, lv = snap
    assert lsm.r == r
    now = lsm.levels()
    assert sorted(now) == sorted(lv)
    for i in lv:
        np.testing.assert_array_equal(now[i][0], lv[i][0])
        np.testing.assert_array_equal(now[i][1], lv[i][1])


def test_device_wait_gives_up_and_context_survives(g):
    st = torch.cuda.current_stream().cuda_stream
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    limit_ns = 200_000_000
    t = time.perf_counter()
    s = g.lsm_debug_wait_flag(flag.data_ptr(), status.data_ptr(), limit_ns, st)
    waited = time.perf_counter() - t
    assert s == g.LSM_ERR_TIMEOUT
    assert int(status.item()) & 2           # the library's timeout bit
    assert 0.2 <= waited < 5.0
    flag.fill_(1)
    assert g.lsm_debug_wait_flag(flag.data_ptr(), status.data_ptr(), limit_ns, st) == g.LSM_OK
    assert int(status.item()) == 0
    # the context still works: a sort through the library after the timeout
    n = 5000
    keys = np.random.default_rng(1).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    kd = g.as_device_u32(keys, 0)
    vd = g.as_device_u32(np.arange(n, dtype=np.uint32), 0)
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    g.lsm_sort_pairs_noalloc(kd.data_ptr(), vd.data_ptr(), ko.data_ptr(), vo.data_ptr(), n, st)
    np.testing.assert_array_equal(u32(ko), np.sort(keys))
    with pytest.raises(g.LSMError):
        g.lsm_debug_wait_flag(flag.data_ptr(), status.data_ptr(), 0, st)


def _fails_then_works(g, make, max_allocs=64):
    """make() at every allocation index failing in turn; returns how many
    allocations it needs."""
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(max_allocs):
        g.lsm_debug_fail_allocs(k, 1)
        try:
            obj = make()
        except g.LSMError as e:
            assert e.status == g.LSM_ERR_OOM, (k, e.status)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert abs(free1 - free0) < (4 << 20), (k, free0, free1)   # nothing leaked
            continue
        g.lsm_debug_fail_allocs(0, 0)
        obj.close()
        assert k >= 3, "a create needs several allocations"
        return k
    raise AssertionError("never succeeded")


def test_create_fails_cleanly_at_every_allocation(g):
    _fails_then_works(g, lambda: g.LSM(1 << 20, 1 << 24))


def test_multi_create_fails_cleanly_at_every_allocation(g):
    _fails_then_works(g, lambda: g.MultiLSM([1000, 3000, 70000], max_batches=4))


def test_cleanup_out_of_memory_changes_nothing(g):
    b = 1 << 12
    calls = workload.sweep_updates(17, b, 11 * b, 0.25, "uniform")
    lsm = g.LSM(b, 16 * b)
    for c in calls:
        lsm.call(*c)
    snap = snapshot(lsm)
    q = np.random.default_rng(3).integers(0, workload.SWEEP_KEY_SPACE, size=4096).astype(np.uint32)
    val0, found0 = lsm.lookup(q)
    for k in range(3):   # the first cleanup allocates its scratch: three buffers
        g.lsm_debug_fail_allocs(k, 1)
        with pytest.raises(g.LSMError) as e:
            lsm.cleanup()
        assert e.value.status == g.LSM_ERR_OOM
        g.lsm_debug_fail_allocs(0, 0)
        assert_same(lsm, snap)
        val, found = lsm.lookup(q)
        np.testing.assert_array_equal(u32(val), u32(val0))
        np.testing.assert_array_equal(found.cpu().numpy(), found0.cpu().numpy())
    lsm.cleanup()
    s = oracle.StructuralOracle(b)
    for c in calls:
        s.call(*c)
    s.cleanup()
    assert lsm.r == s.r
    lv = lsm.levels()
    for i in range(20):
        ekv, ev = s.level(i)
        if len(ekv):
            np.testing.assert_array_equal(lv[i][0], ekv)
            np.testing.assert_array_equal(lv[i][1], ev)
    assert lsm.device_errors() == 0


@pytest.mark.parametrize("n", [30000, 3 << 20])
def test_bulk_build_out_of_memory_changes_nothing(g, n):
    b = 1 << 14
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 24, size=n).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    lsm = g.LSM(b, n + 2 * b)
    failed = 0
    for k in range(16):
        g.lsm_debug_fail_allocs(k, 1)
        try:
            lsm.bulk_build(keys, vals)
        except g.LSMError as e:
            assert e.status == g.LSM_ERR_OOM
            g.lsm_debug_fail_allocs(0, 0)
            assert lsm.r == 0 and lsm.levels() == {}
            failed += 1
            continue
        g.lsm_debug_fail_allocs(0, 0)
        break
    assert failed >= 4   # its own buffers, then the rebuild's scratch
    s = oracle.StructuralOracle(b)
    s.call("insert", keys, vals)
    s.cleanup()
    assert lsm.r == s.r
    lv = lsm.levels()
    for i in range(20):
        ekv, ev = s.level(i)
        if len(ekv):
            np.testing.assert_array_equal(lv[i][0], ekv)
            np.testing.assert_array_equal(lv[i][1], ev)
    assert lsm.device_errors() == 0
