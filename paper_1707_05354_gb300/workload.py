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


def sweep_device_seed(b_log2, delete_frac):
    """Seed of the device-drawn sweep point (b = 2^b_log2, delete fraction)."""
    return 1707053503 + b_log2 * 10 + int(delete_frac * 4)


def sweep_batches_device(torch, dev, b, nb, frac, dist, seed):
    """The sweep recipe drawn on the device (the inputs bench.py times): keys
    uniform in [0, 2^30) or Zipf(1.1) over ranks 1 .. 2^30 (inverse transform
    of the continuous power law, ranks mapped to keys by rank * 0x9E3779B1 mod
    2^30); batch 0 all inserts, later batches round(frac * b) deletes of keys
    drawn uniformly from the earlier inserts, shuffled among the inserts."""
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    space = 1 << 30
    keys = torch.empty(nb * b, dtype=torch.int64, device=dev)
    dele = torch.zeros(nb * b, dtype=torch.uint8, device=dev)
    vals = torch.randint(0, 1 << 31, (nb * b,), device=dev, dtype=torch.int64, generator=gen).to(torch.int32)
    inserted = torch.empty(nb * b, dtype=torch.int64, device=dev)
    n_ins_total = 0
    for t in range(nb):
        n_del = 0 if t == 0 else int(round(b * frac))
        n_ins = b - n_del
        if dist == "zipf":
            u = torch.rand(n_ins, device=dev, dtype=torch.float64, generator=gen)
            a = 1.0 - 1.1
            rank = torch.floor(((float(space) ** a - 1.0) * u + 1.0) ** (1.0 / a)).clamp_(1, space).to(torch.int64)
            ins = (rank * 0x9E3779B1) % space
        else:
            ins = torch.randint(0, space, (n_ins,), device=dev, dtype=torch.int64, generator=gen)
        if n_del:
            idx = torch.randint(0, n_ins_total, (n_del,), device=dev, dtype=torch.int64, generator=gen)
            batch = torch.cat([ins, inserted[idx]])
            flags = torch.cat([torch.zeros(n_ins, dtype=torch.uint8, device=dev),
                               torch.ones(n_del, dtype=torch.uint8, device=dev)])
            perm = torch.randperm(b, device=dev, generator=gen)
            batch, flags = batch[perm], flags[perm]
        else:
            batch, flags = ins, torch.zeros(b, dtype=torch.uint8, device=dev)
        keys[t * b:(t + 1) * b] = batch
        dele[t * b:(t + 1) * b] = flags
        inserted[n_ins_total:n_ins_total + n_ins] = ins
        n_ins_total += n_ins
    return keys.to(torch.int32), vals, dele


# --------------------------------------------------------------------------
# Configuration "batched": many dictionaries with uneven batch sizes.
# --------------------------------------------------------------------------
BATCHED_SEED = 1707053504


def batched_sizes(seed=BATCHED_SEED, n_inst=256, lo_log2=10, hi_log2=18):
    """Batch size per instance: round(2^U[lo, hi]) (log-uniform integers)."""
    g = rng(seed, _STREAM_MISC, 0)
    return np.rint(np.exp2(g.uniform(lo_log2, hi_log2, size=n_inst))).astype(np.int64)


class BatchedWorkload:
    """Configuration 4: rounds of one update batch and b_i lookups per
    instance.  Round 0 inserts b_i fresh keys; later rounds delete
    round(delete_frac * b_i) keys drawn uniformly from the instance's earlier
    inserts and insert fresh keys for the rest, shuffled.  Keys uniform in
    [0, 2^31 - 1), values uniform u32.  Lookups: half drawn from the
    instance's inserts so far, half uniform.

    Arrays of a round hold instance i's entries at [off[i], off[i] + b_i)."""

    def __init__(self, seed=BATCHED_SEED, n_inst=256, rounds=32, delete_frac=0.2, lo_log2=10, hi_log2=18,
                 sizes=None):
        self.seed = seed
        self.sizes = (np.asarray(sizes, np.int64) if sizes is not None
                      else batched_sizes(seed, n_inst, lo_log2, hi_log2))
        self.n = len(self.sizes)
        self.rounds = rounds
        self.delete_frac = delete_frac
        self.off = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.total = int(self.off[-1])
        self._hist = [[] for _ in range(self.n)]
        self._hlen = [[] for _ in range(self.n)]

    def round(self, t):
        """(keys, vals, is_delete, queries) of round t; rounds must be drawn
        in order 0, 1, 2, ... (deletes sample the earlier rounds)."""
        keys = np.empty(self.total, np.uint32)
        vals = np.empty(self.total, np.uint32)
        dele = np.empty(self.total, np.uint8)
        q = np.empty(self.total, np.uint32)
        for i in range(self.n):
            b = int(self.sizes[i])
            g = rng(self.seed, _STREAM_UPDATE, t * 65536 + i)
            n_del = 0 if t == 0 else int(round(b * self.delete_frac))
            n_ins = b - n_del
            ins_k = u32(g, n_ins, 0, KEY_LIMIT)
            ins_v = u32(g, n_ins)
            if n_del:
                cum = np.cumsum(self._hlen[i])
                idx = g.integers(0, int(cum[-1]), size=n_del)
                which = np.searchsorted(cum, idx, side="right")
                start = np.concatenate([[0], cum[:-1]])
                del_k = np.empty(n_del, np.uint32)
                for w in np.unique(which):
                    sel = which == w
                    del_k[sel] = self._hist[i][w][idx[sel] - start[w]]
            else:
                del_k = np.zeros(0, np.uint32)
            kk = np.concatenate([ins_k, del_k])
            vv = np.concatenate([ins_v, np.zeros(n_del, np.uint32)])
            dd = np.concatenate([np.zeros(n_ins, np.uint8), np.ones(n_del, np.uint8)])
            perm = g.permutation(b)
            s = slice(int(self.off[i]), int(self.off[i]) + b)
            keys[s], vals[s], dele[s] = kk[perm], vv[perm], dd[perm]
            self._hist[i].append(ins_k)
            self._hlen[i].append(n_ins)
            gq = rng(self.seed, _STREAM_QUERY, t * 65536 + i)
            half = b // 2
            cum = np.cumsum(self._hlen[i])
            idx = gq.integers(0, int(cum[-1]), size=half)
            which = np.searchsorted(cum, idx, side="right")
            start = np.concatenate([[0], cum[:-1]])
            hits = np.empty(half, np.uint32)
            for w in np.unique(which):
                sel = which == w
                hits[sel] = self._hist[i][w][idx[sel] - start[w]]
            qq = np.concatenate([hits, u32(gq, b - half, 0, KEY_LIMIT)])
            q[s] = qq[gq.permutation(b)]
        return keys, vals, dele, q


# --------------------------------------------------------------------------
# Configuration "serving": a Poisson stream of mixed requests.
# --------------------------------------------------------------------------
SERVING_SEED = 1707053505
SERVING_MIX = (0.40, 0.10, 0.35, 0.05, 0.10)   # insert, delete, lookup, count, range


def serving_pools(seed=SERVING_SEED, n=1 << 26, key_space=KEY_LIMIT, width=8):
    """Payload pools: a = keys uniform in [0, key_space) (update and lookup
    keys, count/range lower bounds), b = values uniform u32, c = a + width - 1
    (count/range upper bounds, clamped below 2^31 - 1)."""
    g = rng(seed, _STREAM_MISC, 1)
    a = u32(g, n, 0, key_space)
    b = u32(g, n)
    c = np.minimum(a.astype(np.int64) + width - 1, KEY_LIMIT - 1).astype(np.uint32)
    return a, b, c


def serving_trace(seed=SERVING_SEED, n_req=10 ** 6, rate=3.0e5, pool_n=1 << 26, size_lo_log2=0.0,
                  size_hi_log2=16.0, mix=SERVING_MIX):
    """Requests of configuration 5: Poisson arrivals at `rate` per second
    (exponential gaps, microseconds), kinds drawn with probabilities `mix`
    (insert, delete, lookup, count, range), sizes round(2^U[lo, hi]) keys,
    each request a window of that many consecutive pool entries starting at
    a uniform position."""
    g = rng(seed, _STREAM_QUERY, 7)
    gaps = g.exponential(1e6 / rate, size=n_req)
    arrival = np.cumsum(gaps) - gaps[0]
    kind = g.choice(5, size=n_req, p=np.asarray(mix) / np.sum(mix)).astype(np.uint8)
    size = np.rint(np.exp2(g.uniform(size_lo_log2, size_hi_log2, size=n_req))).astype(np.int64)
    size = np.maximum(size, 1)
    start = (g.random(n_req) * (pool_n - size + 1)).astype(np.int64)
    return kind, arrival, start.astype(np.uint64), size.astype(np.uint32)
