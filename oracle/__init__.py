"""CPU oracle for the GPU LSM dictionary (arXiv 1707.05354).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The product library never
imports, links or calls it, and it imports nothing from the product library.

Contents
--------
``MapOracle``         O1: the dictionary of §I-B as a ``std::map``, updated one
                      batch at a time under the semantics of §III-A.
``StructuralOracle``  S: the level arrays of Fig. 2(a) / Fig. 3 replayed with
                      ``std::stable_sort`` and ``std::merge``, plus the cleanup
                      of §III-F / §IV-E; gives the exact expected level contents.
``OfflineOracle``     O2: the live dictionary computed once from the whole log
                      (sort by key, newest batch first), queried with
                      ``numpy.searchsorted``; for logs too large for O1.
``brute``             B: answers straight from the operation log (tiny inputs).

The C++ source is ``lsm_oracle.cpp`` next to this file; :func:`build` compiles it
with g++ (plain ``-O2``, no architecture flags) into ``liblsm_oracle.so``.

API-level call semantics mirrored here (the library's boundary contract):
an insert or delete call of n ops is applied as ceil(n / b) consecutive batches
of b ops, the last one padded; an update (mixed) call is one batch of n <= b.
"""

import ctypes
import os
import subprocess

import numpy as np

from . import brute  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsm_oracle.cpp")
_LIB = os.path.join(_HERE, "liblsm_oracle.so")

MAX_USER_KEY = (1 << 31) - 2
PLACEBO_KV = 0xFFFFFFFE

_lib = None


def build(force=False):
    """Compile the oracle's C++ into liblsm_oracle.so (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    lib.o1_new.restype = vp
    lib.o1_free.argtypes = [vp]
    lib.o1_apply_batch.argtypes = [vp, vp, vp, vp, u64]
    lib.o1_size.argtypes = [vp]
    lib.o1_size.restype = u64
    lib.o1_dump.argtypes = [vp, vp, vp]
    lib.o1_lookup.argtypes = [vp, vp, u64, vp, vp]
    lib.o1_count.argtypes = [vp, vp, vp, u64, vp]
    lib.o1_range.argtypes = [vp, vp, vp, u64, vp, vp, vp]
    lib.o1_neighbor.argtypes = [vp, vp, u64, ctypes.c_int, vp, vp, vp]
    lib.s_new.argtypes = [ctypes.c_uint32]
    lib.s_new.restype = vp
    lib.s_free.argtypes = [vp]
    lib.s_apply_batch.argtypes = [vp, vp, vp, vp, u64]
    lib.s_cleanup_all.argtypes = [vp]
    lib.s_r.argtypes = [vp]
    lib.s_r.restype = u64
    lib.s_level_size.argtypes = [vp, i32]
    lib.s_level_size.restype = u64
    lib.s_level.argtypes = [vp, i32, vp, vp, vp]
    lib.o2_build.argtypes = [vp, vp, vp, vp, u64, vp, vp]
    lib.o2_build.restype = u64
    lib.o2_single_level.argtypes = [vp, vp, vp, vp, u64, vp, vp]
    _lib = lib
    return lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def split_call(kind, keys, vals, b, is_delete=None):
    """Batches (keys, vals, is_del) that one API call of ``kind`` applies.

    ``insert``/``delete``: ceil(n/b) consecutive chunks of at most b ops.
    ``update``: one batch of n <= b mixed ops.
    """
    keys = _u32(keys)
    n = len(keys)
    if kind == "update":
        assert n <= b
        return [(keys, _u32(vals), _u8(is_delete))]
    out = []
    for s in range(0, n, b):
        k = keys[s:s + b]
        if kind == "insert":
            out.append((k, _u32(vals[s:s + b]), np.zeros(len(k), np.uint8)))
        elif kind == "delete":
            out.append((k, np.zeros(len(k), np.uint32), np.ones(len(k), np.uint8)))
        else:
            raise ValueError(kind)
    return out


class MapOracle:
    """O1: ordered map, one batch at a time (§I-B, §III-A)."""

    def __init__(self, b):
        self.b = int(b)
        self._lib = _load()
        self._h = self._lib.o1_new()

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.o1_free(self._h)
            self._h = None

    def apply_batch(self, keys, vals, is_del):
        keys, vals, is_del = _u32(keys), _u32(vals), _u8(is_del)
        if len(keys) == 0:
            return
        self._lib.o1_apply_batch(self._h, _p(keys), _p(vals), _p(is_del), len(keys))

    def call(self, kind, keys, vals=None, is_delete=None):
        for k, v, d in split_call(kind, keys, vals, self.b, is_delete):
            self.apply_batch(k, v, d)

    def size(self):
        return int(self._lib.o1_size(self._h))

    def items(self):
        n = self.size()
        k = np.empty(n, np.uint32)
        v = np.empty(n, np.uint32)
        self._lib.o1_dump(self._h, _p(k), _p(v))
        return k, v

    def lookup(self, q):
        q = _u32(q)
        val = np.empty(len(q), np.uint32)
        found = np.empty(len(q), np.uint8)
        self._lib.o1_lookup(self._h, _p(q), len(q), _p(val), _p(found))
        return val, found

    def count(self, k1, k2):
        k1, k2 = _u32(k1), _u32(k2)
        out = np.empty(len(k1), np.uint32)
        self._lib.o1_count(self._h, _p(k1), _p(k2), len(k1), _p(out))
        return out

    def neighbor(self, q, successor=True):
        """(key, value, found) of the successor (smallest live key >= q) or
        predecessor (largest live key <= q) of every query."""
        q = _u32(q)
        key = np.empty(len(q), np.uint32)
        val = np.empty(len(q), np.uint32)
        found = np.empty(len(q), np.uint8)
        self._lib.o1_neighbor(self._h, _p(q), len(q), 1 if successor else 0, _p(key), _p(val), _p(found))
        return key, val, found

    def range(self, k1, k2):
        k1, k2 = _u32(k1), _u32(k2)
        nq = len(k1)
        off = np.empty(nq + 1, np.uint64)
        self._lib.o1_range(self._h, _p(k1), _p(k2), nq, _p(off), None, None)
        total = int(off[nq])
        keys = np.empty(total, np.uint32)
        vals = np.empty(total, np.uint32)
        self._lib.o1_range(self._h, _p(k1), _p(k2), nq, _p(off), _p(keys), _p(vals))
        return off, keys, vals


class StructuralOracle:
    """S: exact level contents of Fig. 2(a) / Fig. 3 and of cleanup (§IV-E)."""

    def __init__(self, b):
        self.b = int(b)
        self._lib = _load()
        self._h = self._lib.s_new(self.b)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.s_free(self._h)
            self._h = None

    def apply_batch(self, keys, vals, is_del):
        keys, vals, is_del = _u32(keys), _u32(vals), _u8(is_del)
        assert 1 <= len(keys) <= self.b
        self._lib.s_apply_batch(self._h, _p(keys), _p(vals), _p(is_del), len(keys))

    def call(self, kind, keys, vals=None, is_delete=None):
        for k, v, d in split_call(kind, keys, vals, self.b, is_delete):
            self.apply_batch(k, v, d)

    def cleanup(self):
        self._lib.s_cleanup_all(self._h)

    @property
    def r(self):
        return int(self._lib.s_r(self._h))

    def level(self, i, with_batch=False):
        """(key variables, values[, batch numbers]) of level i; empty if not full."""
        n = int(self._lib.s_level_size(self._h, i))
        kv = np.empty(n, np.uint32)
        v = np.empty(n, np.uint32)
        bt = np.empty(n, np.uint32)
        if n:
            self._lib.s_level(self._h, i, _p(kv), _p(v), _p(bt))
        return (kv, v, bt) if with_batch else (kv, v)


class OfflineOracle:
    """O2: live dictionary from the whole log at once, queried by bisection."""

    def __init__(self, keys, vals, is_del, batch):
        lib = _load()
        keys, vals, is_del, batch = _u32(keys), _u32(vals), _u8(is_del), _u32(batch)
        n = len(keys)
        ok = np.empty(n, np.uint32)
        ov = np.empty(n, np.uint32)
        m = int(lib.o2_build(_p(keys), _p(vals), _p(is_del), _p(batch), n, _p(ok), _p(ov)))
        self.keys = ok[:m].copy()
        self.vals = ov[:m].copy()

    @classmethod
    def from_calls(cls, calls, b):
        """calls: list of (kind, keys, vals, is_delete) applied in order."""
        ks, vs, ds, bs = [], [], [], []
        t = 0
        for kind, keys, vals, is_delete in calls:
            for k, v, d in split_call(kind, keys, vals, b, is_delete):
                ks.append(k)
                vs.append(v)
                ds.append(d)
                bs.append(np.full(len(k), t, np.uint32))
                t += 1
        cat = (lambda xs, dt: np.concatenate(xs) if xs else np.zeros(0, dt))
        return cls(cat(ks, np.uint32), cat(vs, np.uint32), cat(ds, np.uint8),
                   cat(bs, np.uint32))

    def size(self):
        return len(self.keys)

    def lookup(self, q):
        q = _u32(q)
        val = np.zeros(len(q), np.uint32)
        found = np.zeros(len(q), np.uint8)
        if len(self.keys):
            i = np.searchsorted(self.keys, q, side="left")
            ic = np.minimum(i, len(self.keys) - 1)
            hit = (i < len(self.keys)) & (self.keys[ic] == q)
            val[hit] = self.vals[ic[hit]]
            found[hit] = 1
        return val, found

    def _bounds(self, k1, k2):
        k1 = _u32(k1).astype(np.int64)
        k2 = np.minimum(_u32(k2).astype(np.int64), MAX_USER_KEY)
        lo = np.searchsorted(self.keys, k1, side="left")
        hi = np.searchsorted(self.keys, k2, side="right")
        hi = np.where(k1 > k2, lo, np.maximum(hi, lo))
        return lo, hi

    def count(self, k1, k2):
        lo, hi = self._bounds(k1, k2)
        return (hi - lo).astype(np.uint32)

    def range(self, k1, k2):
        lo, hi = self._bounds(k1, k2)
        cnt = (hi - lo).astype(np.int64)
        off = np.zeros(len(cnt) + 1, np.int64)
        np.cumsum(cnt, out=off[1:])
        total = int(off[-1])
        idx = np.arange(total, dtype=np.int64) + np.repeat(lo - off[:-1], cnt)
        return off.astype(np.uint64), self.keys[idx], self.vals[idx]


def single_level(calls, b):
    """Closed-form contents of the one full level when the number of resident
    batches is a power of two (and no cleanup happened): (key variables,
    values) sorted by key, newer batch first, tombstone first, later op first.
    ``calls`` as for OfflineOracle.from_calls; short batches are padded."""
    lib = _load()
    ks, vs, ds, bs = [], [], [], []
    t = 0
    for kind, keys, vals, is_delete in calls:
        for k, v, d in split_call(kind, keys, vals, b, is_delete):
            n = len(k)
            idx = np.minimum(np.arange(b), n - 1)   # pad with copies of op n-1
            ks.append(k[idx])
            vs.append(v[idx])
            ds.append(d[idx])
            bs.append(np.full(b, t, np.uint32))
            t += 1
    assert t and (t & (t - 1)) == 0, "resident batches must be a power of two"
    keys, vals = _u32(np.concatenate(ks)), _u32(np.concatenate(vs))
    dels, bt = _u8(np.concatenate(ds)), _u32(np.concatenate(bs))
    n = len(keys)
    kv = np.empty(n, np.uint32)
    v = np.empty(n, np.uint32)
    lib.o2_single_level(_p(keys), _p(vals), _p(dels), _p(bt), n, _p(kv), _p(v))
    return kv, v
