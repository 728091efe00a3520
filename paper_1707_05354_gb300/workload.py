"""Seeded synthetic workloads for the GPU LSM (no dictionary arithmetic here).

Both the CUDA path and the CPU oracle are fed from these generators; the module
only draws random keys, values, operation kinds and query bounds.  Every array
comes from ``numpy.random.Generator(PCG64(SeedSequence([seed, stream, index])))``
so a batch can be regenerated on its own without replaying the ones before it.

The recipes follow the paper's workloads (§V: uniformly random 32-bit values,
31-bit keys, batches of b updates, lookups with hits and misses, count/range
queries of a given expected result size L) at the sizes of the benchmark
configurations.  Keys always stay below 2^31 - 1, which the dictionary reserves.

A *call* is a tuple ``(kind, keys, vals, is_delete)`` with kind in
{"insert", "delete", "update"}; ``update`` carries a per-op delete flag.
"""

import numpy as np

KEY_LIMIT = (1 << 31) - 1          # user keys are in [0, KEY_LIMIT)
_STREAM_UPDATE, _STREAM_QUERY, _STREAM_MISC = 1, 2, 3


def rng(seed, stream, index=0):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream, index])))


def u32(g, n, lo=0, hi=1 << 32):
    return g.integers(lo, hi, size=n, dtype=np.uint64).astype(np.uint32)


# --------------------------------------------------------------------------
# Configuration "tiny": b = 1024, 16 mixed batches, then queries.
# --------------------------------------------------------------------------
def tiny_updates(seed=1707053501, b=1024, batches=16, key_space=1 << 20, delete_frac=0.1):
    """Mixed update calls: batch 0 all inserts; later batches floor(0.1 b)
    deletes of keys inserted by earlier batches, shuffled among inserts."""
    calls = []
    inserted = []
    for t in range(batches):
        g = rng(seed, _STREAM_UPDATE, t)
        n_del = 0 if t == 0 else int(b * delete_frac)
        n_ins = b - n_del
        ins_k = u32(g, n_ins, 0, key_space)
        ins_v = u32(g, n_ins)
        if n_del:
            hist = np.concatenate(inserted)
            del_k = hist[g.integers(0, len(hist), size=n_del)]
        else:
            del_k = np.zeros(0, np.uint32)
        keys = np.concatenate([ins_k, del_k]).astype(np.uint32)
        vals = np.concatenate([ins_v, np.zeros(n_del, np.uint32)]).astype(np.uint32)
        is_del = np.concatenate([np.zeros(n_ins, np.uint8), np.ones(n_del, np.uint8)])
        perm = g.permutation(b)
        calls.append(("update", keys[perm], vals[perm], is_del[perm]))
        inserted.append(ins_k)
    return calls


def lookup_queries(seed, inserted_keys, nq, key_space):
    """Half drawn from the inserted keys, half uniform over the key space."""
    g = rng(seed, _STREAM_QUERY, 0)
    half = nq // 2
    hits = inserted_keys[g.integers(0, len(inserted_keys), size=half)]
    rand = u32(g, nq - half, 0, key_space)
    q = np.concatenate([hits, rand]).astype(np.uint32)
    return q[g.permutation(nq)]


def range_queries(seed, nq, key_space, width_lo, width_hi, stream_index=1):
    """k1 uniform, width uniform in [width_lo, width_hi], k2 = k1 + width - 1."""
    g = rng(seed, _STREAM_QUERY, stream_index)
    w = g.integers(width_lo, width_hi + 1, size=nq, dtype=np.int64)
    k1 = g.integers(0, key_space, size=nq, dtype=np.int64)
    k2 = np.minimum(k1 + w - 1, KEY_LIMIT - 1)
    return k1.astype(np.uint32), k2.astype(np.uint32)


def tiny(seed=1707053501):
    """Configuration 1 (b = 1024): 16 mixed batches, 65,536 lookups,
    16,384 count and 16,384 range queries of width U[1, 1024]."""
    b, ks = 1024, 1 << 20
    calls = tiny_updates(seed, b=b, key_space=ks)
    ins = np.concatenate([c[1][c[3] == 0] for c in calls])
    return dict(
        b=b, calls=calls,
        lookups=lookup_queries(seed, ins, 65536, ks),
        count=range_queries(seed, 16384, ks, 1, 1024, 1),
        range=range_queries(seed, 16384, ks, 1, 1024, 2),
    )


# --------------------------------------------------------------------------
# Configuration "paper-scale": b = 2^20, 128 insert batches of 31-bit keys.
# --------------------------------------------------------------------------
def paper_batch(seed, t, b):
    """Insert batch t: keys uniform in [0, 2^31 - 1), values uniform u32."""
    g = rng(seed, _STREAM_UPDATE, t)
    return u32(g, b, 0, KEY_LIMIT), u32(g, b)


def paper_scale(seed=1707053502, b=1 << 20, batches=128, n_lookup=1 << 24,
                n_count=1 << 22, n_range=1 << 22, expected_result=8):
    """Configuration 2.  Batches are produced lazily by ``batch(t)``.

    Count/range width W = round(L * 2^31 / (b * batches)) so that a query over
    uniformly spread live keys expects L results (L = 8 gives W = 128)."""
    width = max(1, int(round(expected_result * float(KEY_LIMIT) / (b * batches))))

    def batch(t):
        return paper_batch(seed, t, b)

    def lookups(inserted_keys=None):
        g = rng(seed, _STREAM_QUERY, 0)
        half = n_lookup // 2
        # hits: keys of randomly chosen (batch, position) pairs, regenerated
        # batch by batch so the 2^27 keys never need to be held at once.
        if inserted_keys is None:
            src_t = g.integers(0, batches, size=half)
            src_i = g.integers(0, b, size=half)
            hits = np.empty(half, np.uint32)
            for t in np.unique(src_t):
                sel = src_t == t
                hits[sel] = batch(int(t))[0][src_i[sel]]
        else:
            hits = inserted_keys[g.integers(0, len(inserted_keys), size=half)]
        rand = u32(g, n_lookup - half, 0, KEY_LIMIT)
        q = np.concatenate([hits, rand]).astype(np.uint32)
        return q[g.permutation(n_lookup)]

    return dict(
        b=b, batches=batches, width=width, batch=batch, lookups=lookups,
        count=lambda: range_queries(seed, n_count, KEY_LIMIT - width, width, width, 1),
        range=lambda: range_queries(seed, n_range, KEY_LIMIT - width, width, width, 2),
    )


# --------------------------------------------------------------------------
# Configuration "sweep": b = 2^16 .. 2^24 at ~2^28 updates, deletes, Zipf.
# --------------------------------------------------------------------------
ZIPF_S = 1.1
SWEEP_KEY_SPACE = 1 << 30


def zipf_keys(g, n, key_space=SWEEP_KEY_SPACE, s=ZIPF_S):
    """Zipf(s) ranks in [1, key_space] (numpy's unbounded sampler, redrawn
    above the bound), mapped to keys by the bijection rank * 0x9E3779B1 mod
    key_space (an odd multiplier, so distinct ranks give distinct keys)."""
    out = np.empty(0, np.int64)
    while len(out) < n:
        z = g.zipf(s, size=2 * (n - len(out)) + 16)
        out = np.concatenate([out, z[z <= key_space][: n - len(out)]])
    return ((out.astype(np.uint64) * np.uint64(0x9E3779B1)) % np.uint64(key_space)).astype(np.uint32)


def sweep_updates(seed, b, total, delete_frac, dist):
    """Calls of configuration 3: total/b update batches; batch 0 all inserts,
    later ones delete_frac of deletes of keys inserted earlier (uniform over
    the inserted history), shuffled among the inserts."""
    calls = []
    history = []
    hist_len = 0
    for t in range(total // b):
        g = rng(seed, _STREAM_UPDATE, t)
        n_del = 0 if t == 0 else int(round(b * delete_frac))
        n_ins = b - n_del
        ins_k = (zipf_keys(g, n_ins) if dist == "zipf" else u32(g, n_ins, 0, SWEEP_KEY_SPACE))
        ins_v = u32(g, n_ins)
        if n_del:
            idx = g.integers(0, hist_len, size=n_del)
            allk = np.concatenate(history) if len(history) > 1 else history[0]
            history = [allk]
            del_k = allk[idx]
        else:
            del_k = np.zeros(0, np.uint32)
        keys = np.concatenate([ins_k, del_k]).astype(np.uint32)
        vals = np.concatenate([ins_v, np.zeros(n_del, np.uint32)]).astype(np.uint32)
        is_del = np.concatenate([np.zeros(n_ins, np.uint8), np.ones(n_del, np.uint8)])
        perm = g.permutation(b)
        calls.append(("update", keys[perm], vals[perm], is_del[perm]))
        history.append(ins_k)
        hist_len += n_ins
    return calls


def sweep_width(expected_result, n_estimate, key_space=SWEEP_KEY_SPACE):
    """Query width giving `expected_result` hits at uniform density n/key_space."""
    return max(1, int(round(expected_result * key_space / max(1, n_estimate))))
