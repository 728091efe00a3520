"""The allocation-free sort entry point against the handle-based one (GPU).

lsm_sort_pairs_noalloc serves callers that must not allocate device memory
while they run -- a process whose device memory all comes from its own pool,
or a latency-bound loop that cannot wait on cudaMalloc/cudaFree.  It takes
its scratch from a fixed array inside the library instead of a handle.  Here
it must give the same output as lsm_sort_pairs (integer keys: bit for bit)
on two calls in a row, which also shows that the shared array carries nothing
over from one call to the next; its output must equal numpy's stable sort;
a call after the first one on a device must leave the device's free memory
unchanged; and it must refuse sizes above its limit.

Kept in a file of its own, named to be collected after every other test.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g(lsm_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lsm_lib


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32).copy()).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_handle_sort_on_two_calls(g):
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        (300_001, lambda r, n: r.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)),
        (g.SORT_NOALLOC_MAX_PAIRS, lambda r, n: (r.integers(0, 40, size=n) * 0x01010101).astype(np.uint32)),
    ]
    lsm = g.LSM(g.SORT_NOALLOC_MAX_PAIRS, g.SORT_NOALLOC_MAX_PAIRS)
    for call, (n, draw) in enumerate(cases):
        rng = np.random.default_rng(4242 + call)
        keys = draw(rng, n)
        vals = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
        kd, vd = _dev(keys), _dev(vals)
        ref_k, ref_v = torch.empty_like(kd), torch.empty_like(vd)
        out_k, out_v = torch.full_like(kd, -1), torch.full_like(vd, -1)
        g.lsm_sort_pairs(lsm.h, kd.data_ptr(), vd.data_ptr(), ref_k.data_ptr(), ref_v.data_ptr(), n, stream)
        g.lsm_sort_pairs_noalloc(kd.data_ptr(), vd.data_ptr(), out_k.data_ptr(), out_v.data_ptr(), n, stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(_u32(out_k), _u32(ref_k))
        np.testing.assert_array_equal(_u32(out_v), _u32(ref_v))
        order = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(_u32(out_k), keys[order])
        np.testing.assert_array_equal(_u32(out_v), vals[order])
    lsm.close()


def test_noalloc_sort_allocates_no_device_memory(g):
    """After a first call on the device (which looks up the array's address),
    further calls leave the device's free memory exactly where it was."""
    stream = torch.cuda.current_stream().cuda_stream
    n = 1 << 20
    rng = np.random.default_rng(99)
    keys = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    kd, vd = _dev(keys), _dev(np.arange(n, dtype=np.uint32))
    out_k, out_v = torch.empty_like(kd), torch.empty_like(vd)
    g.lsm_sort_pairs_noalloc(kd.data_ptr(), vd.data_ptr(), out_k.data_ptr(), out_v.data_ptr(), n, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        g.lsm_sort_pairs_noalloc(kd.data_ptr(), vd.data_ptr(), out_k.data_ptr(), out_v.data_ptr(), n, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_array_equal(_u32(out_k), np.sort(keys))


def test_noalloc_sort_refuses_sizes_above_its_limit(g):
    n = g.SORT_NOALLOC_MAX_PAIRS + 1
    with pytest.raises(g.LSMError) as e:
        g.lsm_sort_pairs_noalloc(1, 1, 1, 1, n, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == g.LSM_ERR_CAPACITY
