"""ctypes binding of libgpulsm.so (the C ABI in include/gpulsm.h).

Argument marshalling only: every step of every operation runs in the CUDA
kernels of the library.  Importing this module loads the library and raises
``ImportError`` when it has not been built (``paper_1707_05354_gb300.build``);
there is no CPU fallback.

Two layers:
  * module functions with the C names (``lsm_create``, ``lsm_insert_batch``,
    ...) taking raw device pointers (ints) and a stream handle, raising
    :class:`LSMError` on any status but LSM_OK;
  * :class:`LSM`, a convenience wrapper over torch CUDA tensors (uint32 data
    travels in int32 tensors, bit for bit).
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpulsm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libgpulsm.so is not built: run `python -m paper_1707_05354_gb300.build` "
                      "(or __graft_entry__.build()) on a machine with the CUDA toolkit")

_lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "LSM_OK", 1: "LSM_ERR_ARG", 2: "LSM_ERR_KEY_RANGE", 3: "LSM_ERR_FULL", 4: "LSM_ERR_OOM",
          5: "LSM_ERR_BUDGET", 6: "LSM_ERR_CAPACITY", 7: "LSM_ERR_CUDA", 8: "LSM_ERR_TIMEOUT"}
LSM_OK, LSM_ERR_ARG, LSM_ERR_KEY_RANGE, LSM_ERR_FULL = 0, 1, 2, 3
LSM_ERR_OOM, LSM_ERR_BUDGET, LSM_ERR_CAPACITY, LSM_ERR_CUDA, LSM_ERR_TIMEOUT = 4, 5, 6, 7, 8
LSM_OPT_LOOKUP_MODE, LSM_OPT_DEVICE_ERROR, LSM_OPT_KERNEL_LAUNCHES, LSM_OPT_KEY_CHECK = 1, 2, 3, 4
LOOKUP_AUTO, LOOKUP_DIRECT, LOOKUP_SORTED = 0, 1, 2
LSM_MULTI_OPT_GRAPH, LSM_MULTI_OPT_GRAPH_KERNELS, LSM_MULTI_OPT_DEVICE_BYTES = 1, 2, 3
REQ_INSERT, REQ_DELETE, REQ_LOOKUP, REQ_COUNT, REQ_RANGE = 0, 1, 2, 3, 4
SERVE_CONTINUOUS, SERVE_FIXED = 0, 1
MULTI_FLAG_BAD_KEY, MULTI_FLAG_ARG, MULTI_FLAG_FULL = 1, 8, 16
PROF_GROUPS = ("sort", "partition", "merge", "lookup", "count", "emit", "cleanup")


class MultiTuning(ctypes.Structure):
    """lsm_multi_tuning: merge tile (1024 | 2048) and prefix-index bin_log2."""
    _fields_ = [("tile", ctypes.c_uint32), ("bin_log2", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    """lsm_server_config."""
    _fields_ = [("b", ctypes.c_uint32), ("hbm_budget", ctypes.c_uint64), ("flush_us", ctypes.c_double),
                ("group_keys", ctypes.c_uint32), ("slots", ctypes.c_uint32), ("range_cap", ctypes.c_uint32),
                ("policy", ctypes.c_int), ("device", ctypes.c_int)]


class Trace(ctypes.Structure):
    """lsm_trace."""
    _fields_ = [("n", ctypes.c_uint64), ("kind", ctypes.c_void_p), ("arrival_us", ctypes.c_void_p),
                ("start", ctypes.c_void_p), ("size", ctypes.c_void_p)]


class TraceResult(ctypes.Structure):
    """lsm_trace_result."""
    _fields_ = [("done_us", ctypes.c_void_p), ("status", ctypes.c_void_p), ("order", ctypes.c_void_p),
                ("res_off", ctypes.c_void_p), ("val", ctypes.c_void_p), ("found", ctypes.c_void_p),
                ("range_start", ctypes.c_void_p), ("rk", ctypes.c_void_p), ("rv", ctypes.c_void_p),
                ("range_cap", ctypes.c_uint64), ("range_total", ctypes.c_uint64),
                ("update_batches", ctypes.c_uint64), ("padded_ops", ctypes.c_uint64),
                ("retrieval_groups", ctypes.c_uint64), ("cleanups", ctypes.c_uint64), ("refused", ctypes.c_uint64),
                ("wall_us", ctypes.c_double), ("host_admit_update_us", ctypes.c_double),
                ("host_admit_retrieval_us", ctypes.c_double), ("host_range_us", ctypes.c_double),
                ("host_complete_us", ctypes.c_double), ("host_cleanup_us", ctypes.c_double),
                ("host_sleep_us", ctypes.c_double), ("gpu_update_ms", ctypes.c_double),
                ("gpu_retrieval_ms", ctypes.c_double), ("gpu_prep_ms", ctypes.c_double),
                ("gpu_lookup_ms", ctypes.c_double), ("gpu_count_ms", ctypes.c_double),
                ("gpu_range_ms", ctypes.c_double), ("gpu_emit_ms", ctypes.c_double)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


_vp, _u64, _u32, _i32, _i64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int64
_SIGS = {
    "lsm_status_str": ([_i32], ctypes.c_char_p),
    "lsm_create": ([ctypes.POINTER(_vp), _u32, _u64, _i32], _i32),
    "lsm_destroy": ([_vp], None),
    "lsm_insert_batch": ([_vp, _vp, _vp, _u64, _vp], _i32),
    "lsm_delete_batch": ([_vp, _vp, _u64, _vp], _i32),
    "lsm_update_batch": ([_vp, _vp, _vp, _vp, _u64, _vp], _i32),
    "lsm_update_batch_ordered": ([_vp, _vp, _vp, _vp, _u64, _vp], _i32),
    "lsm_lookup": ([_vp, _vp, _u64, _vp, _vp, _vp], _i32),
    "lsm_count": ([_vp, _vp, _vp, _u64, _vp, _vp], _i32),
    "lsm_successor": ([_vp, _vp, _u64, _vp, _vp, _vp, _vp], _i32),
    "lsm_predecessor": ([_vp, _vp, _u64, _vp, _vp, _vp, _vp], _i32),
    "lsm_range": ([_vp, _vp, _vp, _u64, _vp, _vp, _vp, _u64, ctypes.POINTER(_u64), _vp], _i32),
    "lsm_cleanup": ([_vp, _vp], _i32),
    "lsm_bulk_build": ([_vp, _vp, _vp, _u64, _vp], _i32),
    "lsm_stats": ([_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u32),
                   ctypes.POINTER(_u32)], _i32),
    "lsm_level_offset": ([_vp, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u64)], _i32),
    "lsm_dump_levels": ([_vp, _vp, _vp, _vp], _i32),
    "lsm_capacity": ([_vp], _u64),
    "lsm_sort_pairs": ([_vp, _vp, _vp, _vp, _vp, _u64, _vp], _i32),
    "lsm_set_option": ([_vp, _i32, _i64], _i32),
    "lsm_get_option": ([_vp, _i32, ctypes.POINTER(_i64)], _i32),
    "lsm_reset": ([_vp], _i32),
    "lsm_stream_wait": ([_vp, _vp], _i32),
    "lsm_profile": ([_vp, _i32], _i32),
    "lsm_profile_read": ([_vp, ctypes.POINTER(ProfileEntry)], _i32),
    "lsm_sort_pairs_noalloc": ([_vp, _vp, _vp, _vp, _u64, _vp], _i32),
    "lsm_debug_fail_allocs": ([_u64, _u64], _i32),
    "lsm_save": ([_vp, _vp, _vp, _u64, _vp, _vp], _i32),
    "lsm_load": ([_vp, _vp, _vp, _u64, _u32, _vp], _i32),
    "lsm_debug_wait_flag": ([_vp, _vp, _u64, _vp], _i32),
    "lsm_multi_create": ([ctypes.POINTER(_vp), _u32, _vp, _u32, _vp, _i32], _i32),
    "lsm_multi_destroy": ([_vp], None),
    "lsm_multi_update": ([_vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "lsm_multi_lookup": ([_vp, _vp, _vp, _u64, _vp, _vp, _vp], _i32),
    "lsm_multi_round": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp], _i32),
    "lsm_multi_sync": ([_vp, _vp, _vp], _i32),
    "lsm_multi_stats": ([_vp, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u32), ctypes.POINTER(_u64)], _i32),
    "lsm_multi_layout": ([_vp, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u32), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(_u32)], _i32),
    "lsm_multi_dump_levels": ([_vp, _u32, _vp, _vp], _i32),
    "lsm_multi_reset": ([_vp, _vp], _i32),
    "lsm_multi_set_option": ([_vp, _i32, _i64], _i32),
    "lsm_server_create": ([ctypes.POINTER(_vp), ctypes.POINTER(ServerConfig)], _i32),
    "lsm_server_destroy": ([_vp], None),
    "lsm_server_set_pool": ([_vp, _vp, _vp, _vp, _u64], _i32),
    "lsm_server_preload": ([_vp, _vp, _vp, _u64], _i32),
    "lsm_server_run": ([_vp, ctypes.POINTER(Trace), ctypes.POINTER(TraceResult)], _i32),
    "lsm_server_stats": ([_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u32),
                          ctypes.POINTER(_u64)], _i32),
    "lsm_server_dict": ([_vp], _vp),
    "lsm_multi_get_option": ([_vp, _i32, ctypes.POINTER(_i64)], _i32),
}
SORT_NOALLOC_MAX_PAIRS = 1 << 20
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class LSMError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s%s" % (where + ": " if where else "", STATUS.get(status, status)))


def _check(status, where):
    if status != LSM_OK:
        raise LSMError(status, where)
    return status


def lsm_status_str(s):
    return _lib.lsm_status_str(s).decode()


def lsm_create(b, max_elements, device=0):
    h = _vp()
    _check(_lib.lsm_create(ctypes.byref(h), b, max_elements, device), "lsm_create")
    return h.value


def lsm_destroy(h):
    _lib.lsm_destroy(h)


def lsm_insert_batch(h, d_keys, d_vals, n, stream=None):
    return _check(_lib.lsm_insert_batch(h, d_keys, d_vals, n, stream), "lsm_insert_batch")


def lsm_delete_batch(h, d_keys, n, stream=None):
    return _check(_lib.lsm_delete_batch(h, d_keys, n, stream), "lsm_delete_batch")


def lsm_update_batch(h, d_keys, d_vals, d_is_delete, n, stream=None):
    return _check(_lib.lsm_update_batch(h, d_keys, d_vals, d_is_delete, n, stream), "lsm_update_batch")


def lsm_update_batch_ordered(h, d_keys, d_vals, d_is_delete, n, stream=None):
    return _check(_lib.lsm_update_batch_ordered(h, d_keys, d_vals, d_is_delete, n, stream),
                  "lsm_update_batch_ordered")


def lsm_lookup(h, d_q, nq, d_val, d_found, stream=None):
    return _check(_lib.lsm_lookup(h, d_q, nq, d_val, d_found, stream), "lsm_lookup")


def lsm_successor(h, d_q, nq, d_key, d_val, d_found, stream=None):
    return _check(_lib.lsm_successor(h, d_q, nq, d_key, d_val, d_found, stream), "lsm_successor")


def lsm_predecessor(h, d_q, nq, d_key, d_val, d_found, stream=None):
    return _check(_lib.lsm_predecessor(h, d_q, nq, d_key, d_val, d_found, stream), "lsm_predecessor")


def lsm_count(h, d_k1, d_k2, nq, d_count, stream=None):
    return _check(_lib.lsm_count(h, d_k1, d_k2, nq, d_count, stream), "lsm_count")


def lsm_range(h, d_k1, d_k2, nq, d_offsets, d_keys, d_vals, capacity, stream=None):
    """Returns (status, total); LSM_ERR_CAPACITY is returned, not raised."""
    total = _u64(0)
    s = _lib.lsm_range(h, d_k1, d_k2, nq, d_offsets, d_keys, d_vals, capacity, ctypes.byref(total), stream)
    if s not in (LSM_OK, LSM_ERR_CAPACITY):
        raise LSMError(s, "lsm_range")
    return s, total.value


def lsm_cleanup(h, stream=None):
    return _check(_lib.lsm_cleanup(h, stream), "lsm_cleanup")


def lsm_bulk_build(h, d_keys, d_vals, n, stream=None):
    return _check(_lib.lsm_bulk_build(h, d_keys, d_vals, n, stream), "lsm_bulk_build")


def lsm_stats(h):
    r, res, b, lv = _u64(), _u64(), _u32(), _u32()
    _check(_lib.lsm_stats(h, ctypes.byref(r), ctypes.byref(res), ctypes.byref(b), ctypes.byref(lv)), "lsm_stats")
    return dict(r=r.value, resident=res.value, b=b.value, levels=lv.value)


def lsm_level_offset(h, i):
    off, size = _u64(), _u64()
    _check(_lib.lsm_level_offset(h, i, ctypes.byref(off), ctypes.byref(size)), "lsm_level_offset")
    return off.value, size.value


def lsm_capacity(h):
    return _lib.lsm_capacity(h)


def lsm_dump_levels(h, h_keys, h_vals, stream=None):
    return _check(_lib.lsm_dump_levels(h, h_keys, h_vals, stream), "lsm_dump_levels")


def lsm_sort_pairs(h, d_kin, d_vin, d_kout, d_vout, n, stream=None):
    return _check(_lib.lsm_sort_pairs(h, d_kin, d_vin, d_kout, d_vout, n, stream), "lsm_sort_pairs")


def lsm_set_option(h, opt, value):
    return _check(_lib.lsm_set_option(h, opt, value), "lsm_set_option")


def lsm_get_option(h, opt):
    v = _i64()
    _check(_lib.lsm_get_option(h, opt, ctypes.byref(v)), "lsm_get_option")
    return v.value


def lsm_sort_pairs_noalloc(d_kin, d_vin, d_kout, d_vout, n, stream=None):
    """Allocation-free sort (no handle); raises LSMError(LSM_ERR_CAPACITY) for
    n > SORT_NOALLOC_MAX_PAIRS."""
    return _check(_lib.lsm_sort_pairs_noalloc(d_kin, d_vin, d_kout, d_vout, n, stream),
                  "lsm_sort_pairs_noalloc")


def lsm_debug_fail_allocs(skip, count):
    """Fault injection: after `skip` more library allocations succeed, the
    next `count` fail (the calls needing them return LSM_ERR_OOM); (0, 0)
    disarms."""
    return _check(_lib.lsm_debug_fail_allocs(skip, count), "lsm_debug_fail_allocs")


def lsm_debug_wait_flag(d_flag, d_status, limit_ns, stream=None):
    """Fault injection: a bounded device wait on *d_flag != 0; returns the
    status code (LSM_OK or LSM_ERR_TIMEOUT) instead of raising."""
    s = _lib.lsm_debug_wait_flag(d_flag, d_status, limit_ns, stream)
    if s not in (LSM_OK, LSM_ERR_TIMEOUT):
        raise LSMError(s, "lsm_debug_wait_flag")
    return s


def lsm_reset(h):
    return _check(_lib.lsm_reset(h), "lsm_reset")


def lsm_stream_wait(h, stream=None):
    return _check(_lib.lsm_stream_wait(h, stream), "lsm_stream_wait")


def lsm_profile(h, enable):
    """enable: False / True (every group), or one group's name (that group alone)."""
    if isinstance(enable, str):
        code = 2 + PROF_GROUPS.index(enable)
    else:
        code = 1 if enable else 0
    return _check(_lib.lsm_profile(h, code), "lsm_profile")


def lsm_profile_read(h):
    """{group name: dict(launches, ms, bytes)} accumulated since lsm_profile(h, 1)."""
    arr = (ProfileEntry * len(PROF_GROUPS))()
    _check(_lib.lsm_profile_read(h, arr), "lsm_profile_read")
    return {n: dict(launches=int(e.launches), ms=float(e.ms), bytes=float(e.bytes))
            for n, e in zip(PROF_GROUPS, arr)}


# batched form ----------------------------------------------------------
def lsm_multi_create(b_list, max_batches, tuning=None, device=0):
    """b_list: batch size per instance; tuning: None or [(tile, bin_log2)] per instance."""
    n = len(b_list)
    bs = (_u32 * n)(*[int(x) for x in b_list])
    tun = None
    if tuning is not None:
        tun = (MultiTuning * n)(*[MultiTuning(int(t), int(e)) for t, e in tuning])
    h = _vp()
    _check(_lib.lsm_multi_create(ctypes.byref(h), n, bs, max_batches, tun, device), "lsm_multi_create")
    return h.value


def lsm_multi_destroy(h):
    _lib.lsm_multi_destroy(h)


def lsm_multi_update(h, d_keys, d_vals, d_is_delete, d_counts, stream=None):
    return _check(_lib.lsm_multi_update(h, d_keys, d_vals, d_is_delete, d_counts, stream), "lsm_multi_update")


def lsm_multi_lookup(h, d_q, d_qoff, nq, d_val, d_found, stream=None):
    return _check(_lib.lsm_multi_lookup(h, d_q, d_qoff, nq, d_val, d_found, stream), "lsm_multi_lookup")


def lsm_multi_round(h, d_keys, d_vals, d_is_delete, d_counts, d_q, d_qoff, nq, d_val, d_found, stream=None):
    return _check(_lib.lsm_multi_round(h, d_keys, d_vals, d_is_delete, d_counts, d_q, d_qoff, nq, d_val,
                                       d_found, stream), "lsm_multi_round")


def lsm_multi_sync(h, stream=None, n_flags=0):
    """Returns (status, per-instance flags as a list or None); never raises on
    the round errors it reports."""
    flags = (_u32 * n_flags)() if n_flags else None
    s = _lib.lsm_multi_sync(h, stream, flags)
    if s in (LSM_ERR_CUDA, LSM_ERR_OOM):
        raise LSMError(s, "lsm_multi_sync")
    return s, (list(flags) if flags is not None else None)


def lsm_multi_stats(h, i):
    r, b, res = _u64(), _u32(), _u64()
    _check(_lib.lsm_multi_stats(h, i, ctypes.byref(r), ctypes.byref(b), ctypes.byref(res)), "lsm_multi_stats")
    return dict(r=r.value, b=b.value, resident=res.value)


def lsm_multi_layout(h, i):
    off, tile, fs, lv = _u64(), _u32(), ctypes.c_int32(), _u32()
    _check(_lib.lsm_multi_layout(h, i, ctypes.byref(off), ctypes.byref(tile), ctypes.byref(fs), ctypes.byref(lv)),
           "lsm_multi_layout")
    return dict(in_off=off.value, tile=tile.value, fence_shift0=fs.value, levels=lv.value)


def lsm_multi_dump_levels(h, i, h_keys, h_vals):
    return _check(_lib.lsm_multi_dump_levels(h, i, h_keys, h_vals), "lsm_multi_dump_levels")


def lsm_multi_reset(h, stream=None):
    return _check(_lib.lsm_multi_reset(h, stream), "lsm_multi_reset")


def lsm_multi_set_option(h, opt, value):
    return _check(_lib.lsm_multi_set_option(h, opt, value), "lsm_multi_set_option")


def lsm_multi_get_option(h, opt):
    v = _i64()
    _check(_lib.lsm_multi_get_option(h, opt, ctypes.byref(v)), "lsm_multi_get_option")
    return v.value


# serving form ----------------------------------------------------------
def lsm_server_create(b, hbm_budget, flush_us=200.0, group_keys=1 << 20, slots=3, range_cap=1 << 25,
                      policy=0, device=0):
    cfg = ServerConfig(b, hbm_budget, flush_us, group_keys, slots, range_cap, policy, device)
    h = _vp()
    _check(_lib.lsm_server_create(ctypes.byref(h), ctypes.byref(cfg)), "lsm_server_create")
    return h.value


def lsm_server_destroy(h):
    _lib.lsm_server_destroy(h)


def lsm_server_set_pool(h, d_a, d_b, d_c, n):
    return _check(_lib.lsm_server_set_pool(h, d_a, d_b, d_c, n), "lsm_server_set_pool")


def lsm_server_preload(h, d_keys, d_vals, n):
    return _check(_lib.lsm_server_preload(h, d_keys, d_vals, n), "lsm_server_preload")


def lsm_server_run(h, trace, result):
    return _check(_lib.lsm_server_run(h, ctypes.byref(trace), ctypes.byref(result)), "lsm_server_run")


def lsm_server_stats(h):
    r, res, lv, by = _u64(), _u64(), _u32(), _u64()
    _check(_lib.lsm_server_stats(h, ctypes.byref(r), ctypes.byref(res), ctypes.byref(lv), ctypes.byref(by)),
           "lsm_server_stats")
    return dict(r=r.value, resident=res.value, levels=lv.value, device_bytes=by.value)


def lsm_server_dict(h):
    return _lib.lsm_server_dict(h)


def kernel_launches():
    """Kernels launched by the library in this process (all handles)."""
    v = _i64()
    _check(_lib.lsm_get_option(None, LSM_OPT_KERNEL_LAUNCHES, ctypes.byref(v)), "lsm_get_option")
    return v.value


# --------------------------------------------------------------------------
# torch convenience layer
# --------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(device):
    return _torch().cuda.current_stream(device).cuda_stream


def as_device_u32(a, device):
    """numpy uint32 (or any int array) -> int32 CUDA tensor with the same bits."""
    import numpy as np
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.to(device=device).contiguous()
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32)
    return torch.from_numpy(arr.copy()).to(device)


def as_device_u8(a, device):
    import numpy as np
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.uint8).contiguous()
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint8)).copy()).to(device)


def to_numpy_u32(t):
    import numpy as np
    return t.cpu().numpy().view(np.uint32)


class LSM:
    """A GPU LSM dictionary on one CUDA device (batch size b)."""

    def __init__(self, b, max_elements, device=0):
        self.device = device
        self.b = b
        self.h = lsm_create(b, max_elements, device)

    def close(self):
        if self.h:
            lsm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # updates -------------------------------------------------------------
    def insert(self, keys, vals):
        k, v = as_device_u32(keys, self.device), as_device_u32(vals, self.device)
        lsm_insert_batch(self.h, _ptr(k), _ptr(v), k.numel(), _stream(self.device))

    def delete(self, keys):
        k = as_device_u32(keys, self.device)
        lsm_delete_batch(self.h, _ptr(k), k.numel(), _stream(self.device))

    def update(self, keys, vals, is_delete):
        k, v = as_device_u32(keys, self.device), as_device_u32(vals, self.device)
        d = as_device_u8(is_delete, self.device)
        lsm_update_batch(self.h, _ptr(k), _ptr(v), _ptr(d), k.numel(), _stream(self.device))

    def update_ordered(self, keys, vals, is_delete):
        k, v = as_device_u32(keys, self.device), as_device_u32(vals, self.device)
        d = as_device_u8(is_delete, self.device)
        lsm_update_batch_ordered(self.h, _ptr(k), _ptr(v), _ptr(d), k.numel(), _stream(self.device))

    def call(self, kind, keys, vals=None, is_delete=None):
        if kind == "insert":
            self.insert(keys, vals)
        elif kind == "delete":
            self.delete(keys)
        elif kind == "update":
            self.update(keys, vals, is_delete)
        else:
            raise ValueError(kind)

    def cleanup(self):
        lsm_cleanup(self.h, _stream(self.device))

    def bulk_build(self, keys, vals):
        k, v = as_device_u32(keys, self.device), as_device_u32(vals, self.device)
        lsm_bulk_build(self.h, _ptr(k), _ptr(v), k.numel(), _stream(self.device))

    # queries -------------------------------------------------------------
    def lookup(self, q):
        torch = _torch()
        qd = as_device_u32(q, self.device)
        n = qd.numel()
        val = torch.empty(n, dtype=torch.int32, device=self.device)
        found = torch.empty(n, dtype=torch.uint8, device=self.device)
        lsm_lookup(self.h, _ptr(qd), n, _ptr(val), _ptr(found), _stream(self.device))
        return val, found

    def neighbor(self, q, successor=True):
        """(key, value, found) of each query's successor or predecessor."""
        torch = _torch()
        qd = as_device_u32(q, self.device)
        n = qd.numel()
        key = torch.empty(n, dtype=torch.int32, device=self.device)
        val = torch.empty(n, dtype=torch.int32, device=self.device)
        found = torch.empty(n, dtype=torch.uint8, device=self.device)
        fn = lsm_successor if successor else lsm_predecessor
        fn(self.h, _ptr(qd), n, _ptr(key), _ptr(val), _ptr(found), _stream(self.device))
        return key, val, found

    def count(self, k1, k2):
        torch = _torch()
        a, z = as_device_u32(k1, self.device), as_device_u32(k2, self.device)
        out = torch.empty(a.numel(), dtype=torch.int32, device=self.device)
        lsm_count(self.h, _ptr(a), _ptr(z), a.numel(), _ptr(out), _stream(self.device))
        return out

    def range(self, k1, k2, capacity=None):
        """(offsets int64[nq+1], keys int32[total], vals int32[total]); grows
        the output buffers and retries once on LSM_ERR_CAPACITY."""
        torch = _torch()
        a, z = as_device_u32(k1, self.device), as_device_u32(k2, self.device)
        nq = a.numel()
        off = torch.empty(nq + 1, dtype=torch.int64, device=self.device)
        cap = max(1, capacity if capacity is not None else 8 * nq)
        for _ in range(2):
            ok = torch.empty(cap, dtype=torch.int32, device=self.device)
            ov = torch.empty(cap, dtype=torch.int32, device=self.device)
            s, total = lsm_range(self.h, _ptr(a), _ptr(z), nq, _ptr(off), _ptr(ok), _ptr(ov), cap,
                                 _stream(self.device))
            if s == LSM_OK:
                return off, ok[:total], ov[:total]
            cap = max(1, total)
        raise LSMError(LSM_ERR_CAPACITY, "range")

    # state ---------------------------------------------------------------
    def stats(self):
        return lsm_stats(self.h)

    @property
    def r(self):
        return self.stats()["r"]

    def levels(self):
        """Host copy of every full level: {i: (key variables, values)} as uint32."""
        import numpy as np
        cap = lsm_capacity(self.h)
        hk = np.zeros(cap, np.uint32)
        hv = np.zeros(cap, np.uint32)
        lsm_dump_levels(self.h, hk.ctypes.data, hv.ctypes.data, _stream(self.device))
        r = self.r
        out = {}
        for i in range(self.stats()["levels"]):
            if (r >> i) & 1:
                off, size = lsm_level_offset(self.h, i)
                out[i] = (hk[off:off + size].copy(), hv[off:off + size].copy())
        return out

    def save(self):
        """Checkpoint: (r, key variables, values) of the full levels in
        ascending level order, as host uint32 arrays (lsm_save)."""
        import numpy as np
        st = self.stats()
        n = st["r"] * st["b"]
        hk = np.empty(max(1, n), np.uint32)
        hv = np.empty(max(1, n), np.uint32)
        r = _u64()
        _check(_lib.lsm_save(self.h, hk.ctypes.data, hv.ctypes.data, n, ctypes.byref(r), _stream(self.device)),
               "lsm_save")
        return r.value, hk[:n], hv[:n]

    def load(self, r, keys, vals, b=None):
        """Resume from a checkpoint (lsm_load) of a dictionary with batch size
        b (default: this handle's; another b is refused)."""
        import numpy as np
        hk = np.ascontiguousarray(keys, dtype=np.uint32)
        hv = np.ascontiguousarray(vals, dtype=np.uint32)
        _check(_lib.lsm_load(self.h, hk.ctypes.data, hv.ctypes.data, r, self.b if b is None else b,
                             _stream(self.device)), "lsm_load")
        _torch().cuda.synchronize(self.device)   # the host arrays may be freed after the call returns

    def set_lookup_mode(self, mode):
        lsm_set_option(self.h, LSM_OPT_LOOKUP_MODE, mode)

    def device_errors(self):
        return lsm_get_option(self.h, LSM_OPT_DEVICE_ERROR)


class MultiLSM:
    """n independent GPU LSMs with batch sizes b_list, advanced a round at a
    time (lsm_multi_*).  Batches of a round are laid out back to back in
    instance order (instance i at offset sum(b_list[:i]))."""

    def __init__(self, b_list, max_batches, tuning=None, device=0):
        import numpy as np
        self.device = device
        self.b = np.asarray(b_list, dtype=np.int64)
        self.n = len(b_list)
        self.in_off = np.concatenate([[0], np.cumsum(self.b)])
        self.h = lsm_multi_create(b_list, max_batches, tuning, device)

    def close(self):
        if self.h:
            lsm_multi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, keys, vals, is_delete=None, counts=None):
        """keys/vals: sum(b) entries (instance i's ops first in its slot);
        counts: ops per instance (None = full batches).  Asynchronous; call
        sync() for errors."""
        k, v = as_device_u32(keys, self.device), as_device_u32(vals, self.device)
        d = None if is_delete is None else as_device_u8(is_delete, self.device)
        c = None if counts is None else as_device_u32(counts, self.device)
        self._keep = (k, v, d, c)
        lsm_multi_update(self.h, _ptr(k), _ptr(v), _ptr(d), _ptr(c), _stream(self.device))

    def lookup(self, q, qoff):
        torch = _torch()
        qd = as_device_u32(q, self.device)
        off = torch.as_tensor(qoff, dtype=torch.int64).to(self.device)
        n = qd.numel()
        val = torch.empty(n, dtype=torch.int32, device=self.device)
        found = torch.empty(n, dtype=torch.uint8, device=self.device)
        lsm_multi_lookup(self.h, _ptr(qd), _ptr(off), n, _ptr(val), _ptr(found), _stream(self.device))
        return val, found

    def sync(self):
        return lsm_multi_sync(self.h, _stream(self.device), self.n)

    def stats(self, i):
        return lsm_multi_stats(self.h, i)

    def levels(self, i):
        """Full levels of instance i: {l: (key variables, values)} as uint32."""
        import numpy as np
        st = self.stats(i)
        r, b = st["r"], st["b"]
        hk = np.zeros(max(1, r * b), np.uint32)
        hv = np.zeros(max(1, r * b), np.uint32)
        lsm_multi_dump_levels(self.h, i, hk.ctypes.data, hv.ctypes.data)
        out, pos = {}, 0
        for l in range(32):
            if (r >> l) & 1:
                n = b << l
                out[l] = (hk[pos:pos + n].copy(), hv[pos:pos + n].copy())
                pos += n
        return out

    def reset(self):
        lsm_multi_reset(self.h, _stream(self.device))

    def set_graph(self, on):
        lsm_multi_set_option(self.h, LSM_MULTI_OPT_GRAPH, 1 if on else 0)


class Server:
    """Serving engine (lsm_server_*) over one dictionary of batch size b.

    ``pools``: (a, b, c) device tensors (int32 bits of u32) of equal length;
    ``run(kind, arrival_us, start, size, keep_results)`` replays a trace and
    returns a dict of per-request numpy arrays (done_us, status, order, and,
    with keep_results, the results)."""

    def __init__(self, b, hbm_budget, flush_us=200.0, group_keys=1 << 20, slots=3, range_cap=1 << 25,
                 policy=SERVE_CONTINUOUS, device=0):
        self.device = device
        self.h = lsm_server_create(b, hbm_budget, flush_us, group_keys, slots, range_cap, policy, device)
        self._pools = None

    def close(self):
        if self.h:
            lsm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_pool(self, a, b, c):
        self._pools = tuple(as_device_u32(x, self.device) for x in (a, b, c))
        pa, pb, pc = self._pools
        lsm_server_set_pool(self.h, _ptr(pa), _ptr(pb), _ptr(pc), pa.numel())

    def preload(self, keys, vals):
        k, v = as_device_u32(keys, self.device), as_device_u32(vals, self.device)
        lsm_server_preload(self.h, _ptr(k), _ptr(v), k.numel())

    def stats(self):
        return lsm_server_stats(self.h)

    def run(self, kind, arrival_us, start, size, keep_results=False, range_cap=None):
        import numpy as np
        n = len(kind)
        kind = np.ascontiguousarray(kind, np.uint8)
        arr = np.ascontiguousarray(arrival_us, np.float64)
        start = np.ascontiguousarray(start, np.uint64)
        size = np.ascontiguousarray(size, np.uint32)
        tr = Trace(n, kind.ctypes.data, arr.ctypes.data, start.ctypes.data, size.ctypes.data)
        out = dict(done_us=np.zeros(n, np.float64), status=np.zeros(n, np.int32), order=np.zeros(n, np.uint64))
        res = TraceResult()
        res.done_us, res.status, res.order = (out["done_us"].ctypes.data, out["status"].ctypes.data,
                                              out["order"].ctypes.data)
        if keep_results:
            off = np.concatenate([[0], np.cumsum(size.astype(np.uint64))]).astype(np.uint64)
            tot = int(off[-1])
            out["res_off"] = off[:-1].copy()
            out["val"] = np.zeros(max(1, tot), np.uint32)
            out["found"] = np.zeros(max(1, tot), np.uint8)
            out["range_start"] = np.zeros(max(1, tot), np.uint64)
            cap = int(range_cap if range_cap is not None else 16 * tot)
            out["rk"] = np.zeros(max(1, cap), np.uint32)
            out["rv"] = np.zeros(max(1, cap), np.uint32)
            res.res_off, res.val, res.found = (out["res_off"].ctypes.data, out["val"].ctypes.data,
                                               out["found"].ctypes.data)
            res.range_start, res.rk, res.rv = (out["range_start"].ctypes.data, out["rk"].ctypes.data,
                                               out["rv"].ctypes.data)
            res.range_cap = cap
        lsm_server_run(self.h, tr, res)
        out.update(range_total=res.range_total, update_batches=res.update_batches, padded_ops=res.padded_ops,
                   retrieval_groups=res.retrieval_groups, cleanups=res.cleanups, refused=res.refused,
                   wall_us=res.wall_us,
                   time_split={k: getattr(res, k) for k in (
                       "host_admit_update_us", "host_admit_retrieval_us", "host_range_us", "host_complete_us",
                       "host_cleanup_us", "host_sleep_us", "gpu_update_ms", "gpu_retrieval_ms", "gpu_prep_ms",
                       "gpu_lookup_ms", "gpu_count_ms", "gpu_range_ms", "gpu_emit_ms")})
        return out
