"""Autotuner of the batched form's per-instance shapes.

Two shapes of the batched form (lsm_multi_*) depend on an instance's batch
size b and are picked per bucket round(log2 b):

  tile      output elements per merge work item (1024 or 2048): smaller tiles
            give the persistent merge more items to balance when instances are
            small, larger ones amortise the per-item co-rank search and setup;
  bin_log2  resolution of every level's prefix index, about 2^bin_log2
            elements per bin: the fan-out of the first step of each search
            (lookups and the merge partition).  Finer tables cost more bytes to
            write at every fold, coarser ones leave longer binary searches.

For each bucket the tuner times a few rounds (update batch + b lookups per
instance, one graph replay each) of a multi handle whose instances all have
b = 2^bucket, for every candidate pair, and keeps the fastest.  The result is
cached as JSON per device name.  Timing uses CUDA events on the stream the
rounds run on; the inputs are random keys drawn on the device (the tuner
measures speed only; correctness is the tests' job).
"""

import json
import os
import time

CANDIDATES = tuple((t, e) for t in (1024, 2048) for e in (2, 3, 4, 5))
DEFAULT = (2048, 3)
BUCKETS = tuple(range(10, 19))
_HERE = os.path.dirname(os.path.abspath(__file__))


def bucket_of(b):
    import math
    return int(round(math.log2(max(1, int(b)))))


def cache_path(device=0):
    import torch
    name = torch.cuda.get_device_name(device).replace(" ", "_").replace("/", "_")
    return os.path.join(_HERE, "_build", "multi_tuning_%s.json" % name)


def _time_candidate(G, torch, b, n_inst, rounds, tile, e, device, reps):
    st = torch.cuda.current_stream(device)
    sp = st.cuda_stream
    m = G.MultiLSM([b] * n_inst, max_batches=rounds, tuning=[(tile, e)] * n_inst, device=device)
    tot = b * n_inst
    gen = torch.Generator(device=device)
    gen.manual_seed(1707053599)
    keys = [torch.randint(0, (1 << 31) - 1, (tot,), device=device, dtype=torch.int64, generator=gen)
            .to(torch.int32) for _ in range(rounds)]
    vals = torch.zeros(tot, dtype=torch.int32, device=device)
    off = torch.arange(n_inst + 1, dtype=torch.int64, device=device) * b
    val = torch.empty(tot, dtype=torch.int32, device=device)
    fnd = torch.empty(tot, dtype=torch.uint8, device=device)

    def run():
        m.reset()
        for t in range(rounds):
            G.lsm_multi_round(m.h, keys[t].data_ptr(), vals.data_ptr(), None, None, keys[t].data_ptr(),
                              off.data_ptr(), tot, val.data_ptr(), fnd.data_ptr(), sp)

    run()  # capture the graphs
    best = None
    for _ in range(reps):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        a.record(st)
        run()
        z.record(st)
        z.synchronize()
        ms = a.elapsed_time(z)
        best = ms if best is None else min(best, ms)
    status, _ = m.sync()
    m.close()
    if status != G.LSM_OK:
        raise RuntimeError("tuning round failed: %s" % G.STATUS.get(status, status))
    return best


def tune(device=0, buckets=BUCKETS, rounds=8, elements=1 << 22, reps=3, verbose=False):
    """{bucket: {"tile", "bin_log2", "ms": {candidate: ms}}} measured now."""
    import torch
    from . import gpulsm as G
    out = {}
    for q in buckets:
        b = 1 << q
        n_inst = min(256, max(1, elements // b))
        times = {}
        for tile, e in CANDIDATES:
            times["%d/%d" % (tile, e)] = _time_candidate(G, torch, b, n_inst, rounds, tile, e, device, reps)
        best = min(times, key=times.get)
        t, e = (int(x) for x in best.split("/"))
        out[q] = {"tile": t, "bin_log2": e, "ms": times}
        if verbose:
            print("bucket 2^%d: %s  %s" % (q, best, {k: round(v, 3) for k, v in times.items()}), flush=True)
    return out


def load_or_tune(device=0, retune=False, verbose=False):
    """Cached table for this device (tuned and written on first use)."""
    path = cache_path(device)
    if not retune:
        try:
            with open(path) as f:
                return {int(k): v for k, v in json.load(f)["buckets"].items()}
        except (OSError, ValueError, KeyError):
            pass
    t0 = time.time()
    table = tune(device=device, verbose=verbose)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"buckets": {str(k): v for k, v in table.items()}, "seconds": time.time() - t0}, f, indent=1)
    return table


def tuning_for(sizes, table):
    """Per-instance (tile, bin_log2) for batch sizes `sizes` from a table."""
    out = []
    for b in sizes:
        q = min(max(bucket_of(b), min(table)), max(table)) if table else None
        ent = table.get(q) if table else None
        out.append((ent["tile"], ent["bin_log2"]) if ent else DEFAULT)
    return out
