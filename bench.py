#!/usr/bin/env python3
"""Benchmark of the GPU LSM on the paper-scale workload (b = 2^20).

One step = one pass of the whole path over the workload, inputs resident in
HBM: reset the dictionary, insert 128 batches of b = 2^20 uniformly random
31-bit keys with u32 values (2^27 updates, sort + cascade fold per batch),
2^24 lookups (half drawn from the inserted keys), 2^22 count and 2^22 range
queries of width 128 (8 expected results), and a cleanup.  The headline value
is M updates/s over the insert phase; lookups/s and the other phases are
reported beside it.  The insert inputs (1 GiB) are larger than L2, so no L2
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpulsm|reference]

Under torchrun (N > 1) every rank runs an independent replica (the method has
no cross-dictionary exchange): weak scaling, value summed over ranks, time
the max over ranks.  `--impl reference` times the CPU oracle (std::map
dictionary) on a bounded sample of the same workload, rank 0 only.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M updates/s and M lookups/s at b=2^20 (GB300), % of HBM roofline"
SEED = 1707053502
PAPER_UPDATE_RATE_B20 = 354.1  # M updates/s, harmonic mean over r at b=2^20, n=2^27 (Table II, K40c)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpulsm", choices=["gpulsm", "reference"])
    p.add_argument("--b-log2", type=int, default=20)
    p.add_argument("--batches", type=int, default=128)
    p.add_argument("--lookups-log2", type=int, default=24)
    p.add_argument("--queries-log2", type=int, default=22)
    p.add_argument("--lookup-mode", type=int, default=0, help="0 auto, 1 direct, 2 sorted")
    p.add_argument("--key-check", default="sync", choices=["sync", "deferred"],
                   help="paper/sweep: update calls wait for the key check (sync) or not (deferred)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="paper", choices=["paper", "batched", "serving", "sweep"],
                   help="paper: b=2^20 plain dictionary (default); batched: 256 dictionaries per round; "
                        "serving: a Poisson stream of mixed requests through the serving engine")
    p.add_argument("--requests", type=int, default=10 ** 6, help="serving: requests in the trace")
    p.add_argument("--sweep-b", default="16,18,20,22,24", help="sweep: log2 of the batch sizes")
    p.add_argument("--sweep-total-log2", type=int, default=28, help="sweep: updates per point")
    p.add_argument("--rate", type=float, default=3.0e5, help="serving: arrivals per second")
    p.add_argument("--rate2", type=float, default=6.0e5, help="serving: a second, heavier load point (0: none)")
    p.add_argument("--flush-us", type=float, default=1000.0, help="serving: longest wait of a partial batch")
    p.add_argument("--preload-log2", type=int, default=28, help="serving: dictionary size before the stream")
    p.add_argument("--preload-batches", type=int, default=0,
                   help="serving: preload this many batches of b instead of 2^preload-log2 keys")
    p.add_argument("--budget-gb", type=float, default=64.0, help="serving: HBM admission budget (GiB)")
    p.add_argument("--instances", type=int, default=256)
    p.add_argument("--rounds", type=int, default=32)
    p.add_argument("--no-plain", action="store_true", help="batched: skip the per-instance plain-call arm")
    p.add_argument("--no-tune", action="store_true", help="batched: default shapes instead of the tuner's")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def paper_config(args, world):
    """The `config` of the paper-scale line (both arms)."""
    b, nb = 1 << args.b_log2, args.batches
    return {"workload": "paper-scale plain LSM: b=2^%d, %d insert batches (2^%d updates), 2^%d lookups "
                        "(half hits), 2^%d count + 2^%d range queries (expected 8 results), cleanup"
                        % (args.b_log2, nb, int(np.log2(nb * b)), args.lookups_log2, args.queries_log2,
                           args.queries_log2),
            "b": b, "batches": nb, "lookup_mode": args.lookup_mode, "key_check": args.key_check,
            "l2": "inputs larger than L2 (1 GiB of updates per step), no flush",
            "parallelism": "replicas" if world > 1 else "single GPU"}


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth, for context beside the measured copy peak


def update_roofline(upd_rate_m, nb, peak_gbs):
    """Whole insert phase against the HBM roofline: a batch folding into
    level k = ffz(r) moves 16 * 2^k * b bytes (read the batch and levels
    0..k-1, write level k), so nb batches from r = 0 move
    sum_r 16 * 2^ffz(r) bytes per batch element (72 B at nb = 128)."""
    bpu = sum(16.0 * (1 << ((~r & (r + 1)).bit_length() - 1)) for r in range(nb)) / nb
    gbs = upd_rate_m * 1e6 * bpu / 1e9
    return {"bytes_per_update": bpu, "achieved_GB/s": gbs, "frac": gbs / peak_gbs,
            "frac_of_nominal": gbs / NOMINAL_HBM_GBS, "nominal_GB/s": NOMINAL_HBM_GBS,
            "roofline_M_updates_per_s": peak_gbs * 1e9 / bpu / 1e6}


def max_over_ranks(vec, device, world):
    """Element-wise maximum of a list of floats over all ranks of the
    process group (the timed quantities: the slowest rank defines each)."""
    if world <= 1:
        return list(vec)
    import torch
    import torch.distributed as dist
    t = torch.tensor(vec, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def workload_arrays(args):
    from paper_1707_05354_gb300 import workload
    b = 1 << args.b_log2
    cfg = workload.paper_scale(seed=SEED, b=b, batches=args.batches, n_lookup=1 << args.lookups_log2,
                               n_count=1 << args.queries_log2, n_range=1 << args.queries_log2)
    keys = np.empty(args.batches * b, np.uint32)
    vals = np.empty(args.batches * b, np.uint32)
    for t in range(args.batches):
        keys[t * b:(t + 1) * b], vals[t * b:(t + 1) * b] = cfg["batch"](t)
    q = cfg["lookups"](inserted_keys=keys)
    c1, c2 = cfg["count"]()
    r1, r2 = cfg["range"]()
    return cfg, keys, vals, q, (c1, c2), (r1, r2)


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic():
    """Per-element DRAM traffic of each kernel from the committed ncu summary."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------ CPU oracle --
def oracle_sample(keys, vals, q, b, n_batches, n_lookups):
    """Time the std::map oracle on the first n_batches batches and n_lookups
    lookups of the workload; returns (M updates/s, M lookups/s, seconds)."""
    import oracle
    o1 = oracle.MapOracle(b)
    zeros = np.zeros(b, np.uint8)
    t0 = time.perf_counter()
    for t in range(n_batches):
        o1.apply_batch(keys[t * b:(t + 1) * b], vals[t * b:(t + 1) * b], zeros)
    t1 = time.perf_counter()
    o1.lookup(q[:n_lookups])
    t2 = time.perf_counter()
    return n_batches * b / (t1 - t0) / 1e6, n_lookups / (t2 - t1) / 1e6, t2 - t0


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cfg, keys, vals, q, _, _ = workload_arrays(args)
    b = cfg["b"]
    n_batches, n_lookups = 2, 1 << 20   # a bounded sample of the workload per step
    rates, lrates, secs = [], [], []
    for i in range(args.warmup + args.steps):
        u, l, s = oracle_sample(keys, vals, q, b, n_batches, n_lookups)
        if i >= args.warmup:
            rates.append(u)
            lrates.append(l)
            secs.append(s)
    value = statistics.median(rates)
    sample = ("per step: a fresh std::map, the first %d of %d insert batches (b=2^%d, %d updates) and %d "
              "lookups of the workload" % (n_batches, args.batches, args.b_log2, n_batches * b, n_lookups))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "M updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_UPDATE_RATE_B20,
        "dtype": "u32", "data": "synthetic (seeded uniform 31-bit keys, u32 values)",
        "config": paper_config(args, 1),
        "lookups": {"value": statistics.median(lrates), "unit": "M lookups/s"},
        "cpu_baseline": {"value": value, "unit": "M updates/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "M updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU ---
def run_gpu(args):
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1707_05354_gb300 import gpulsm as G

    cfg, keys, vals, q, (c1, c2), (r1, r2) = workload_arrays(args)
    b, nb = cfg["b"], args.batches
    n_upd, nq, ncq = nb * b, len(q), len(c1)
    st = torch.cuda.current_stream(dev)
    sp = st.cuda_stream

    def dev_u32(a):
        return torch.from_numpy(a.view(np.int32)).to(dev)

    d_keys, d_vals = dev_u32(keys), dev_u32(vals)
    d_q, d_c1, d_c2, d_r1, d_r2 = dev_u32(q), dev_u32(c1), dev_u32(c2), dev_u32(r1), dev_u32(r2)
    o_val = torch.empty(nq, dtype=torch.int32, device=dev)
    o_found = torch.empty(nq, dtype=torch.uint8, device=dev)
    o_cnt = torch.empty(ncq, dtype=torch.int32, device=dev)
    o_off = torch.empty(len(r1) + 1, dtype=torch.int64, device=dev)
    cap = 4 * 8 * len(r1)
    o_rk = torch.empty(cap, dtype=torch.int32, device=dev)
    o_rv = torch.empty(cap, dtype=torch.int32, device=dev)

    h = G.lsm_create(b, n_upd, local)
    G.lsm_set_option(h, G.LSM_OPT_LOOKUP_MODE, args.lookup_mode)
    G.lsm_set_option(h, G.LSM_OPT_KEY_CHECK, 1 if args.key_check == "deferred" else 0)
    kp, vp = d_keys.data_ptr(), d_vals.data_ptr()
    phases = ("update", "lookup", "count", "range", "cleanup")

    def step(ev):
        G.lsm_reset(h)
        ev[0].record(st)
        for t in range(nb):
            G.lsm_insert_batch(h, kp + 4 * t * b, vp + 4 * t * b, b, sp)
        G.lsm_stream_wait(h, sp)   # the last folds run on the handle's internal stream
        ev[1].record(st)
        G.lsm_lookup(h, d_q.data_ptr(), nq, o_val.data_ptr(), o_found.data_ptr(), sp)
        ev[2].record(st)
        G.lsm_count(h, d_c1.data_ptr(), d_c2.data_ptr(), ncq, o_cnt.data_ptr(), sp)
        ev[3].record(st)
        s, total = G.lsm_range(h, d_r1.data_ptr(), d_r2.data_ptr(), len(r1), o_off.data_ptr(),
                               o_rk.data_ptr(), o_rv.data_ptr(), cap, sp)
        assert s == G.LSM_OK, "range output capacity"
        ev[4].record(st)
        G.lsm_cleanup(h, sp)
        ev[5].record(st)
        return total

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for _ in range(args.warmup):
        step(mk())
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    # The timed steps bracket only the merge launches with events (the
    # roofline's kernel, timed live); an event between two kernels ends their
    # launch overlap, so bracketing every group would slow the timed steps.
    # The table of all groups comes from one more, untimed step.
    G.lsm_profile(h, "merge")
    launches0 = G.kernel_launches()
    evs = [mk() for _ in range(args.steps)]
    barrier()
    t_wall0 = time.perf_counter()
    totals = [step(ev) for ev in evs]
    barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = G.kernel_launches() - launches0
    prof_timed = G.lsm_profile_read(h)
    G.lsm_profile(h, True)
    step(mk())
    prof = G.lsm_profile_read(h)
    G.lsm_profile(h, 0)
    clocks = sampler.stop()
    ph = {p: 0.0 for p in phases}
    for ev in evs:
        for i, p in enumerate(phases):
            ph[p] += ev[i].elapsed_time(ev[i + 1]) / 1000.0
    step_s = sum(ev[0].elapsed_time(ev[5]) for ev in evs) / 1000.0
    found_frac = float(o_found.float().mean().item())

    # correctness spot check of this run's final state against the oracle
    # is left to the tests; here only the device error word is checked
    errs = G.lsm_get_option(h, G.LSM_OPT_DEVICE_ERROR)
    assert errs == 0, "device error bits %d" % errs

    # max over ranks of the timed quantities
    vec = max_over_ranks([ph[p] for p in phases] + [step_s, t_wall], dev, world)
    ph = dict(zip(phases, vec[:5]))
    step_s, t_wall = vec[5], vec[6]
    K = args.steps
    upd_rate = world * K * n_upd / ph["update"] / 1e6
    look_rate = world * K * nq / ph["lookup"] / 1e6

    # Roofline of the dominant kernel: fold_merge, the kernel with the largest
    # device-time share in the launch list of this workload (the "sort" group
    # is two kernels; the larger, bucket_sort, has about three quarters of the
    # merge's share).  Every group's fraction is reported beside it.
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    dom = "merge"
    d = prof_timed[dom]
    achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9 if d["ms"] > 0 else 0.0
    tr = ncu_traffic().get(dom)
    traffic = None
    if tr and tr.get("bytes_per_unit") and d["launches"]:
        units_per_launch = d["bytes"] / d["launches"] / tr.get("algorithmic_bytes_per_unit", 16.0)
        traffic = tr["bytes_per_unit"] * units_per_launch
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "traffic": traffic, "peak_source": peak_kind,
                "launches": d["launches"], "avg_launch_ms": d["ms"] / max(1, d["launches"]),
                "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"])}
    groups = {g: {"launches": v["launches"], "ms": round(v["ms"], 4),
                  "GB/s": (v["bytes"] / (v["ms"] / 1000) / 1e9) if v["ms"] > 0 and v["bytes"] else None}
              for g, v in prof.items()}
    for g in groups.values():
        g["frac"] = g["GB/s"] / hbm if g["GB/s"] else None

    # Worst case of the lookups: r = 2^m - 1 (m levels full), where a miss
    # probes every level; the timed r = 2^m state holds one level (the
    # sorted-array layout).
    wl = []
    wl_found = 0.0
    for _ in range(3):
        G.lsm_reset(h)
        for t in range(nb - 1):
            G.lsm_insert_batch(h, kp + 4 * t * b, vp + 4 * t * b, b, sp)
        G.lsm_stream_wait(h, sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        G.lsm_lookup(h, d_q.data_ptr(), nq, o_val.data_ptr(), o_found.data_ptr(), sp)
        e1.record(st)
        e1.synchronize()
        wl.append(nq / (e0.elapsed_time(e1) / 1000.0) / 1e6)
        wl_found = float(o_found.float().mean().item())
    lookups_worst = {"value": world * statistics.median(wl), "unit": "M lookups/s", "r": nb - 1,
                     "levels": bin(nb - 1).count("1"), "found_fraction": wl_found}

    # Per-batch rates over r (each insert timed alone: the stream drained
    # before it, its fold joined after it), as the paper tabulates min / max
    # beside the mean; grouped by k = ffz(r), the level the batch folds into.
    G.lsm_reset(h)
    per_k = {}
    for t in range(nb):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        G.lsm_insert_batch(h, kp + 4 * t * b, vp + 4 * t * b, b, sp)
        G.lsm_stream_wait(h, sp)
        e1.record(st)
        e1.synchronize()
        k = (~t & (t + 1)).bit_length() - 1
        per_k.setdefault(k, []).append(e0.elapsed_time(e1))
    all_ms = [x for v in per_k.values() for x in v]
    per_batch = {"min_M_updates_per_s": b / (max(all_ms) / 1000.0) / 1e6,
                 "max_M_updates_per_s": b / (min(all_ms) / 1000.0) / 1e6,
                 "mean_M_updates_per_s": nb * b / (sum(all_ms) / 1000.0) / 1e6,
                 "ms_by_k": {str(k): round(statistics.median(v), 4) for k, v in sorted(per_k.items())},
                 "note": "each batch alone (stream drained before, fold joined after): no sort/fold overlap"}

    # Bulk build (the paper's build-from-scratch figure, §V-A): the step's
    # insert pairs sorted and laid out in one call on an empty dictionary;
    # the call allocates its sort buffers, inside the timed region.
    bb = []
    for _ in range(3):
        G.lsm_reset(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        G.lsm_bulk_build(h, kp, vp, n_upd, sp)
        e1.record(st)
        e1.synchronize()
        bb.append(e0.elapsed_time(e1))
    bulk = {"value": world * n_upd / (statistics.median(bb) / 1000.0) / 1e6, "unit": "M pairs/s",
            "ms": round(statistics.median(bb), 3), "pairs": n_upd, "r": G.lsm_stats(h)["r"],
            "note": "lsm_bulk_build of the step's insert pairs into an empty dictionary (a sort of all pairs, "
                    "then cleanup's compaction and distribution into the levels of ceil(n'/b)); median of 3"}

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, G, h, torch, dev, keys, vals, q, c1, c2, r1, r2, world)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        nbs, nls = 8, 1 << 21
        u, l, s = oracle_sample(keys, vals, q, b, nbs, nls)
        cpu = {"value": u, "unit": "M updates/s", "cores": 1, "kind": "oracle",
               "lookups_M_per_s": l, "seconds": s,
               "sample": "std::map oracle, single thread: the first %d of %d insert batches (%d updates) "
                         "then %d lookups of the workload" % (nbs, nb, nbs * b, nls)}

    G.lsm_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": upd_rate, "unit": "M updates/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1000.0 * step_s / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": upd_rate / PAPER_UPDATE_RATE_B20, "dtype": "u32",
            "data": "synthetic (seeded uniform 31-bit keys, u32 values; PCG64)",
            "config": paper_config(args, world),
            "lookups": {"value": look_rate, "unit": "M lookups/s", "found_fraction": found_frac,
                        "r": nb, "levels": bin(nb).count("1")},
            "lookups_worst_case": lookups_worst,
            "per_batch": per_batch,
            "bulk_build": bulk,
            "phases_ms_per_step": {p: 1000.0 * ph[p] / K for p in phases},
            "rates": {"count_M_per_s": world * K * ncq / ph["count"] / 1e6,
                      "range_M_per_s": world * K * len(r1) / ph["range"] / 1e6,
                      "cleanup_M_elements_per_s": world * K * n_upd / ph["cleanup"] / 1e6,
                      "range_results_per_step": int(totals[-1])},
            "kernel_groups": groups,
            "kernel_groups_note": "one more untimed step with every group bracketed by events; the timed steps "
                                  "bracket only the merge launches (the roofline's kernel)",
            "roofline": roofline,
            "update_phase_roofline": update_roofline(upd_rate / world, nb, hbm),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wall_s_timed": t_wall,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_e2e(args, G, h, torch, dev, keys, vals, q, c1, c2, r1, r2, world):
    """Same step through the C ABI, inputs copied from pinned host memory
    inside the timed region (a copy stream stages the batches in four
    device buffers, up to three ahead of the inserts) and
    every result read back to the host."""
    b, nb = 1 << args.b_log2, args.batches
    pin = lambda a: torch.from_numpy(a.view(np.int32)).pin_memory()
    hk, hv, hq = pin(keys), pin(vals), pin(q)
    hc1, hc2, hr1, hr2 = pin(c1), pin(c2), pin(r1), pin(r2)
    st = torch.cuda.current_stream(dev)
    cs = torch.cuda.Stream(dev)
    sp = st.cuda_stream
    G4 = 4  # batches per copy: two device staging groups of four batches, one group ahead of the inserts
    gbuf = [(torch.empty(G4 * b, dtype=torch.int32, device=dev), torch.empty(G4 * b, dtype=torch.int32, device=dev))
            for _ in range(2)]
    dq = torch.empty(len(q), dtype=torch.int32, device=dev)
    dc1, dc2 = torch.empty_like(dq[:len(c1)]), torch.empty_like(dq[:len(c1)])
    dr1, dr2 = torch.empty_like(dq[:len(r1)]), torch.empty_like(dq[:len(r1)])
    o_val = torch.empty(len(q), dtype=torch.int32, device=dev)
    o_found = torch.empty(len(q), dtype=torch.uint8, device=dev)
    o_cnt = torch.empty(len(c1), dtype=torch.int32, device=dev)
    o_off = torch.empty(len(r1) + 1, dtype=torch.int64, device=dev)
    cap = 4 * 8 * len(r1)
    o_rk = torch.empty(cap, dtype=torch.int32, device=dev)
    o_rv = torch.empty(cap, dtype=torch.int32, device=dev)
    h_val = torch.empty(len(q), dtype=torch.int32).pin_memory()
    h_found = torch.empty(len(q), dtype=torch.uint8).pin_memory()
    h_cnt = torch.empty(len(c1), dtype=torch.int32).pin_memory()
    h_off = torch.empty(len(r1) + 1, dtype=torch.int64).pin_memory()
    h_rk = torch.empty(cap, dtype=torch.int32).pin_memory()
    h_rv = torch.empty(cap, dtype=torch.int32).pin_memory()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    looked, counted_in = torch.cuda.Event(), torch.cuda.Event()

    ngroups = (nb + G4 - 1) // G4

    def issue_group(g):
        # batches 4g .. 4g + 3 into staging group g % 2 in one copy per array,
        # once the inserts of group g - 2 (whose sorts read it) are done
        j = g % 2
        lo = g * G4 * b
        n = min(G4 * b, nb * b - lo)
        with torch.cuda.stream(cs):
            if g >= 2:
                cs.wait_event(consumed[j])
            gbuf[j][0][:n].copy_(hk[lo:lo + n], non_blocking=True)
            gbuf[j][1][:n].copy_(hv[lo:lo + n], non_blocking=True)
            copied[j].record(cs)

    def step():
        G.lsm_reset(h)
        t0 = time.perf_counter()
        # the copies run a group (four batches) ahead of the inserts, a few
        # host calls per four batches: with the default key check an insert
        # call returns once its batch is sorted, so host work between two
        # inserts leaves the device waiting
        issue_group(0)
        for g in range(ngroups):
            j = g % 2
            if g + 1 < ngroups:
                issue_group(g + 1)
            st.wait_event(copied[j])
            for u in range(min(G4, nb - g * G4)):
                G.lsm_insert_batch(h, gbuf[j][0].data_ptr() + 4 * u * b, gbuf[j][1].data_ptr() + 4 * u * b, b, sp)
            consumed[j].record(st)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        # the count's inputs go up while the lookups run, the lookups'
        # results come back while the count runs (copy stream)
        dq.copy_(hq, non_blocking=True)
        G.lsm_lookup(h, dq.data_ptr(), len(q), o_val.data_ptr(), o_found.data_ptr(), sp)
        looked.record(st)
        with torch.cuda.stream(cs):
            dc1.copy_(hc1, non_blocking=True)
            dc2.copy_(hc2, non_blocking=True)
            counted_in.record(cs)
            cs.wait_event(looked)
            h_val.copy_(o_val, non_blocking=True)
            h_found.copy_(o_found, non_blocking=True)
        st.wait_event(counted_in)
        G.lsm_count(h, dc1.data_ptr(), dc2.data_ptr(), len(c1), o_cnt.data_ptr(), sp)
        h_cnt.copy_(o_cnt, non_blocking=True)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        dr1.copy_(hr1, non_blocking=True)
        dr2.copy_(hr2, non_blocking=True)
        s, total = G.lsm_range(h, dr1.data_ptr(), dr2.data_ptr(), len(r1), o_off.data_ptr(), o_rk.data_ptr(),
                               o_rv.data_ptr(), cap, sp)
        h_off.copy_(o_off, non_blocking=True)
        h_rk[:total].copy_(o_rk[:total], non_blocking=True)
        h_rv[:total].copy_(o_rv[:total], non_blocking=True)
        G.lsm_cleanup(h, sp)
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        return t1 - t0, t2 - t1, t3 - t0, total

    for _ in range(max(1, args.warmup)):
        step()
    K = max(1, args.steps // 2)
    res = [step() for _ in range(K)]
    upd_s = sum(r[0] for r in res)
    look_s = sum(r[1] for r in res)
    tot = res[-1][3]
    h2d = nb * b * 8 + len(q) * 4 + len(c1) * 8 + len(r1) * 8
    d2h = len(q) * 5 + len(c1) * 4 + (len(r1) + 1) * 8 + tot * 8
    return {"value": world * K * nb * b / upd_s / 1e6, "unit": "M updates/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "lookup_and_count_M_per_s": world * K * (len(q) + len(c1)) / look_s / 1e6,
            "ms_per_step": 1000.0 * sum(r[2] for r in res) / K, "steps": K,
            "note": "wall clock on the host around each phase; update batches copied from pinned memory on a "
                    "second stream, four batches per copy, one group ahead of the inserts, into two staging groups"}


# ----------------------------------------------------------- batched form --
BATCHED_METRIC = "M updates/s of the batched form (256 dictionaries, b log-uniform in [2^10, 2^18])"


def batched_rounds(args):
    from paper_1707_05354_gb300 import workload
    wl = workload.BatchedWorkload(n_inst=args.instances, rounds=args.rounds)
    return wl, [wl.round(t) for t in range(wl.rounds)]


def batched_bytes(sizes, rounds):
    """Algorithmic bytes of one pass over all rounds: per instance and round
    16 * 2^k * b for the update (k = ffz(r)) and, for its b lookups, 9 B per
    query plus 32 B per full level probed (upper bound: every full level)."""
    tot = 0.0
    for r in range(rounds):
        k = (~r & (r + 1)).bit_length() - 1
        levels = bin(r + 1).count("1")
        for b in sizes:
            tot += 16.0 * (1 << k) * b + b * (9.0 + 32.0 * levels)
    return tot


def run_batched(args):
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1707_05354_gb300 import autotune
    from paper_1707_05354_gb300 import gpulsm as G

    wl, rounds = batched_rounds(args)
    sizes = [int(x) for x in wl.sizes]
    tot, R = wl.total, wl.rounds
    st = torch.cuda.current_stream(dev)
    sp = st.cuda_stream

    def dev_u32(a):
        return torch.from_numpy(a.view(np.int32)).to(dev)

    dk = [dev_u32(r[0]) for r in rounds]
    dv = [dev_u32(r[1]) for r in rounds]
    dd = [torch.from_numpy(r[2]).to(dev) for r in rounds]
    dq = [dev_u32(r[3]) for r in rounds]
    off = torch.as_tensor(wl.off, dtype=torch.int64).to(dev)
    o_val = torch.empty(tot, dtype=torch.int32, device=dev)
    o_fnd = torch.empty(tot, dtype=torch.uint8, device=dev)

    table = {} if args.no_tune else autotune.load_or_tune(local)
    tuning = autotune.tuning_for(sizes, table)
    m = G.MultiLSM(sizes, max_batches=R, tuning=tuning, device=local)

    def step_multi():
        m.reset()
        for t in range(R):
            G.lsm_multi_round(m.h, dk[t].data_ptr(), dv[t].data_ptr(), dd[t].data_ptr(), None, dq[t].data_ptr(),
                              off.data_ptr(), tot, o_val.data_ptr(), o_fnd.data_ptr(), sp)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(steps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            z.record(st)
            evs.append((a, z))
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(z) / 1000.0 for a, z in evs]

    for _ in range(args.warmup):
        step_multi()
    status, flags = m.sync()
    assert status == G.LSM_OK and not any(flags), "batched round error %s" % status
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    l0 = G.kernel_launches()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.synchronize(dev)
        dist.barrier()
    secs = timed(step_multi, args.steps, 0)
    launches = G.kernel_launches() - l0
    clocks = sampler.stop()
    status, _ = m.sync()
    assert status == G.LSM_OK
    per_round_kernels = G.lsm_multi_get_option(m.h, G.LSM_MULTI_OPT_GRAPH_KERNELS)
    mult_s = max_over_ranks([statistics.median(secs)], dev, world)[0]

    # the same rounds as separate per-instance plain calls (one handle each)
    plain = None
    if not args.no_plain:
        hs = [G.lsm_create(b, b * R, local) for b in sizes]
        vo = [int(x) for x in wl.off]

        def step_plain():
            for h in hs:
                G.lsm_reset(h)
            for t in range(R):
                kp, vp, dp, qp = dk[t].data_ptr(), dv[t].data_ptr(), dd[t].data_ptr(), dq[t].data_ptr()
                for i, h in enumerate(hs):
                    o = vo[i]
                    G.lsm_update_batch(h, kp + 4 * o, vp + 4 * o, dp + o, sizes[i], sp)
                    G.lsm_lookup(h, qp + 4 * o, sizes[i], o_val.data_ptr() + 4 * o, o_fnd.data_ptr() + o, sp)

        psecs = timed(step_plain, max(1, min(args.steps, 3)), 1)
        for h in hs:
            G.lsm_destroy(h)
        p_s = statistics.median(psecs)
        plain = {"value": R * tot / p_s / 1e6, "unit": "M updates/s", "ms_per_step": 1000 * p_s,
                 "speedup_of_batched": p_s / mult_s,
                 "what": "one plain handle per dictionary; per round and dictionary lsm_update_batch + "
                         "lsm_lookup (each update waits for its key check, as the plain API does)"}

    # end to end: each round's inputs copied from pinned host memory, results
    # read back.  The copies run on a copy stream one round ahead into two
    # device staging sets; a round starts with a device-to-device copy of its
    # set into the fixed buffers its graph was captured on, and its results
    # go back through two staging sets the same way, so the host link works
    # while the previous or next round runs.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hk = [pin(r[0].view(np.int32)) for r in rounds]
        hv = [pin(r[1].view(np.int32)) for r in rounds]
        hd = [pin(r[2]) for r in rounds]
        hq = [pin(r[3].view(np.int32)) for r in rounds]
        bk, bv = torch.empty(tot, dtype=torch.int32, device=dev), torch.empty(tot, dtype=torch.int32, device=dev)
        bd, bq = torch.empty(tot, dtype=torch.uint8, device=dev), torch.empty(tot, dtype=torch.int32, device=dev)
        sin = [(torch.empty_like(bk), torch.empty_like(bv), torch.empty_like(bd), torch.empty_like(bq))
               for _ in range(2)]
        sout = [(torch.empty_like(o_val), torch.empty_like(o_fnd)) for _ in range(2)]
        hval = torch.empty(tot, dtype=torch.int32).pin_memory()
        hfnd = torch.empty(tot, dtype=torch.uint8).pin_memory()
        cs = torch.cuda.Stream(dev)
        st_ = torch.cuda.current_stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]      # staging set j holds round t's inputs
        ev_taken = [torch.cuda.Event() for _ in range(2)]   # round t copied set j into the fixed buffers
        ev_res = [torch.cuda.Event() for _ in range(2)]     # round t's results in output set j
        ev_read = [torch.cuda.Event() for _ in range(2)]    # output set j read back to the host

        def load(t):
            j = t % 2
            with torch.cuda.stream(cs):
                if t >= 2:
                    cs.wait_event(ev_taken[j])
                for d, h in zip(sin[j], (hk[t], hv[t], hd[t], hq[t])):
                    d.copy_(h, non_blocking=True)
                ev_in[j].record(cs)

        def step_e2e():
            m.reset()
            load(0)
            for t in range(R):
                j = t % 2
                if t + 1 < R:
                    load(t + 1)
                st_.wait_event(ev_in[j])
                for d, sset in zip((bk, bv, bd, bq), sin[j]):
                    d.copy_(sset, non_blocking=True)
                ev_taken[j].record(st_)
                G.lsm_multi_round(m.h, bk.data_ptr(), bv.data_ptr(), bd.data_ptr(), None, bq.data_ptr(),
                                  off.data_ptr(), tot, o_val.data_ptr(), o_fnd.data_ptr(), sp)
                if t >= 2:
                    st_.wait_event(ev_read[j])
                sout[j][0].copy_(o_val, non_blocking=True)
                sout[j][1].copy_(o_fnd, non_blocking=True)
                ev_res[j].record(st_)
                with torch.cuda.stream(cs):
                    cs.wait_event(ev_res[j])
                    hval.copy_(sout[j][0], non_blocking=True)
                    hfnd.copy_(sout[j][1], non_blocking=True)
                    ev_read[j].record(cs)
            torch.cuda.synchronize(dev)

        for _ in range(max(1, args.warmup)):
            step_e2e()
        K = max(1, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(K):
            step_e2e()
        e_s = (time.perf_counter() - t0) / K
        e2e = {"value": R * tot / e_s / 1e6, "unit": "M updates/s", "h2d_bytes_per_step": R * tot * 13,
               "d2h_bytes_per_step": R * tot * 5, "ms_per_step": 1000 * e_s, "steps": K,
               "note": "wall clock per pass of all rounds; per round the update batch and queries are copied "
                       "from pinned host memory (on a copy stream, one round ahead, through two device staging "
                       "sets) and the lookup results read back the same way"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        n_done = 0
        o1s = [oracle.MapOracle(b) for b in sizes]
        for t in range(min(R, 4)):
            k, v, d, q = rounds[t]
            for i, b in enumerate(sizes):
                s = slice(int(wl.off[i]), int(wl.off[i + 1]))
                o1s[i].apply_batch(k[s], v[s], d[s])
                o1s[i].lookup(q[s])
            n_done += tot
        c_s = time.perf_counter() - t0
        cpu = {"value": n_done / c_s / 1e6, "unit": "M updates/s", "cores": 1, "kind": "oracle",
               "seconds": c_s, "sample": "std::map oracle per dictionary, single thread: the first %d rounds "
                                         "(update batch + lookups of every dictionary)" % min(R, 4)}

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    abytes = batched_bytes(sizes, R)
    achieved = abytes / mult_s / 1e9
    m.close()
    value = world * R * tot / mult_s / 1e6
    if rank == 0:
        line = {
            "metric": BATCHED_METRIC, "value": value, "unit": "M updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * mult_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded: b_i = round(2^U[10,18]), uniform 31-bit keys, 20% deletes of earlier "
                    "keys, half-hit lookups; PCG64)",
            "config": {"workload": "batched form: %d dictionaries, %d rounds of one update batch (b_i ops) and b_i "
                                   "lookups each; %d updates per round" % (wl.n, R, tot),
                       "instances": wl.n, "rounds": R, "updates_per_round": tot,
                       "b_min": min(sizes), "b_max": max(sizes),
                       "l2": "inputs larger than L2 (%.0f MB of updates per step), no flush" % (R * tot * 9 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "lookups": {"value": world * R * tot / mult_s / 1e6, "unit": "M lookups/s",
                        "note": "lookups run in the same graph replay as the updates; value and lookups share "
                                "the round time"},
            "ms_per_round": 1000 * mult_s / R,
            "plain_calls": plain,
            "tuning": {"table": {str(k): [v["tile"], v["bin_log2"]] for k, v in table.items()},
                       "default": list(autotune.DEFAULT)},
            "roofline": {"bound": "hbm", "kernel": "whole round (one graph replay)", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "peak_source": peak_kind, "algorithmic_bytes_per_step": abytes},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "graph_kernels_per_round": per_round_kernels, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- serving --
SERVING_METRIC = "serving: M keys/s and p50/p99 request latency (mixed stream, 64 GB HBM budget)"


def latency_stats(out, arrival, kind=None):
    """p50 / p99 / mean / max latency; with `kind`, the same for the update
    requests (insert, delete) and the retrievals (lookup, count, range)."""
    lat = (out["done_us"] - arrival) / 1000.0
    st = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
          "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}
    if kind is not None:
        for name, sel in (("updates", kind <= 1), ("retrievals", kind >= 2)):
            if sel.any():
                st[name] = {"p50_ms": float(np.percentile(lat[sel], 50)), "p99_ms": float(np.percentile(lat[sel], 99))}
    return st


def run_serving(args):
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1707_05354_gb300 import gpulsm as G
    from paper_1707_05354_gb300 import workload

    b = 1 << args.b_log2
    pool_n = 1 << 26
    pa, pb, pc = workload.serving_pools(n=pool_n)
    traces = {r: workload.serving_trace(n_req=args.requests, rate=r, pool_n=pool_n)
              for r in [args.rate] + ([args.rate2] if args.rate2 else [])}
    kind, arrival, start, size = traces[args.rate]
    wk, wa, ws, wz = workload.serving_trace(seed=workload.SERVING_SEED + 1, n_req=max(1000, args.requests // 100),
                                            rate=args.rate, pool_n=pool_n)
    keys_total = int(size.astype(np.int64).sum())
    # preload: uniform keys drawn on the device (setup, not timed), in chunks
    npre = args.preload_batches * b if args.preload_batches else 1 << args.preload_log2

    def preload(srv):
        gen = torch.Generator(device=dev)
        gen.manual_seed(workload.SERVING_SEED)
        done_ = 0
        while done_ < npre:
            m = min(1 << 26, npre - done_)
            k = torch.randint(0, (1 << 31) - 1, (m,), device=dev, dtype=torch.int64, generator=gen).to(torch.int32)
            v = torch.randint(0, 1 << 31, (m,), device=dev, dtype=torch.int64, generator=gen).to(torch.int32)
            srv.preload(k, v)
            done_ += m

    budget = int(args.budget_gb * (1 << 30))
    results = {}
    clocks = None
    launches = 0
    for rate, (t_kind, t_arr, t_start, t_size) in traces.items():
        res = {}
        t_keys = int(t_size.astype(np.int64).sum())
        for name, policy in (("continuous", G.SERVE_CONTINUOUS), ("fixed", G.SERVE_FIXED)):
            srv = G.Server(b, budget, flush_us=args.flush_us, group_keys=1 << 20, slots=3, range_cap=1 << 25,
                           policy=policy, device=local)
            srv.set_pool(pa, pb, pc)
            preload(srv)
            for _ in range(max(1, args.warmup)):
                srv.run(wk, wa, ws, wz)       # warm-up: a short trace of the same mix
            st0 = srv.stats()
            first = rate == args.rate and name == "continuous"
            sampler = ClockSampler(local) if first else None
            if sampler:
                sampler.start()
                time.sleep(0.3)
            l0 = G.kernel_launches()
            out = srv.run(t_kind, t_arr, t_start, t_size)
            if first:
                launches = G.kernel_launches() - l0
                clocks = sampler.stop()
            st1 = srv.stats()
            wall_s = out["wall_us"] / 1e6
            res[name] = dict(latency=latency_stats(out, t_arr, t_kind), requests_per_s=len(t_kind) / wall_s,
                             M_keys_per_s=t_keys / wall_s / 1e6, wall_s=wall_s,
                             arrivals_s=float(t_arr[-1]) / 1e6,
                             update_batches=int(out["update_batches"]), padded_ops=int(out["padded_ops"]),
                             retrieval_groups=int(out["retrieval_groups"]), cleanups=int(out["cleanups"]),
                             refused=int(out["refused"]), range_results=int(out["range_total"]),
                             time_split=out["time_split"],
                             levels=st0["levels"], device_bytes=st0["device_bytes"],
                             resident_before=st0["resident"], resident_after=st1["resident"],
                             all_ok=bool((out["status"] == 0).all()))
            print("serving %s at %.0f/s: %s" % (name, rate, json.dumps(res[name])), file=sys.stderr, flush=True)
            srv.close()
            del srv
            torch.cuda.synchronize(dev)
        results[rate] = res
    res = results[args.rate]
    c = res["continuous"]
    span_s = float(arrival[-1]) / 1e6
    if rank == 0:
        line = {
            "metric": SERVING_METRIC, "value": c["M_keys_per_s"], "unit": "M keys/s", "n_gpus": world,
            "steps": 1, "warmup": max(1, args.warmup), "ms_per_step": 1000 * c["wall_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded Poisson arrivals, kinds 40/10/35/5/10 %%, sizes round(2^U[0,16]) keys; "
                    "payload windows of device-resident pools of 2^26 uniform keys; preload %d uniform keys)"
                    % npre,
            "config": {"workload": "serving: %d requests at %.0f/s (%.2f s of arrivals, %d keys), b=2^%d, "
                                   "%.0f GiB HBM budget, flush %.0f us, 3 slots"
                                   % (len(kind), args.rate, span_s, keys_total, args.b_log2, args.budget_gb,
                                      args.flush_us),
                       "requests": len(kind), "rate_per_s": args.rate, "b": b, "budget_gib": args.budget_gb,
                       "l2": "payload pools (768 MB) and dictionary (>= 2 GB) larger than L2",
                       "parallelism": "single GPU"},
            "latency_ms": {"p50": c["latency"]["p50_ms"], "p99": c["latency"]["p99_ms"]},
            "continuous": c, "fixed_batching": res["fixed"],
            "vs_fixed": {"p50_ratio": res["fixed"]["latency"]["p50_ms"] / max(1e-9, c["latency"]["p50_ms"]),
                         "p99_ratio": res["fixed"]["latency"]["p99_ms"] / max(1e-9, c["latency"]["p99_ms"]),
                         "throughput_ratio": c["M_keys_per_s"] / max(1e-9, res["fixed"]["M_keys_per_s"])},
            "heavier_load": ({"rate_per_s": args.rate2, "continuous": results[args.rate2]["continuous"],
                              "fixed_batching": results[args.rate2]["fixed"]} if args.rate2 else None),
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": c["M_keys_per_s"], "unit": "M keys/s", "h2d_bytes_per_step": 21 * len(kind),
                    "d2h_bytes_per_step": None,
                    "note": "the serving loop itself is end to end: request descriptors go host to device per "
                            "group, results come back to pinned host memory before a request completes"},
            "gpu_launches": int(launches), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ sweep --
SWEEP_METRIC = "M updates/s over the update/delete sweep (b = 2^16 .. 2^24, ~2^28 updates per point)"


def run_sweep(args):
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1707_05354_gb300 import gpulsm as G
    from paper_1707_05354_gb300 import workload
    st = torch.cuda.current_stream(dev)
    sp = st.cuda_stream
    total = 1 << args.sweep_total_log2
    nq = 1 << 22
    points = []
    for bl in [int(x) for x in args.sweep_b.split(",")]:
        b = 1 << bl
        nb = total // b
        for dist in ("uniform", "zipf"):
            for frac in (0.0, 0.25, 0.5):
                keys, vals, dele = workload.sweep_batches_device(torch, dev, b, nb, frac, dist,
                                                                 workload.sweep_device_seed(bl, frac))
                h = G.lsm_create(b, total, local)
                G.lsm_set_option(h, G.LSM_OPT_KEY_CHECK, 1 if args.key_check == "deferred" else 0)
                kp, vp, dp = keys.data_ptr(), vals.data_ptr(), dele.data_ptr()

                def updates():
                    G.lsm_reset(h)
                    for t in range(nb):
                        G.lsm_update_batch(h, kp + 4 * t * b, vp + 4 * t * b, dp + t * b, b, sp)
                    G.lsm_stream_wait(h, sp)

                updates()  # warm-up pass
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                a.record(st)
                updates()
                z.record(st)
                z.synchronize()
                upd_s = a.elapsed_time(z) / 1000.0
                # live keys (for the query widths): counts over 2^16 slices of the key space
                lo = torch.arange(1 << 16, device=dev, dtype=torch.int64) << 14
                hi = (lo + (1 << 14) - 1).to(torch.int32)
                lo = lo.to(torch.int32)
                cnt = torch.empty(1 << 16, dtype=torch.int32, device=dev)
                G.lsm_count(h, lo.data_ptr(), hi.data_ptr(), 1 << 16, cnt.data_ptr(), sp)
                n_live = max(1, int(cnt.to(torch.int64).sum().item()))
                ranges = {}
                gen = torch.Generator(device=dev)
                gen.manual_seed(bl)
                for L in (8, 64, 512):
                    w = max(1, int(round(L * (1 << 30) / n_live)))
                    k1 = torch.randint(0, (1 << 30) - w, (nq,), device=dev, dtype=torch.int64, generator=gen)
                    k2 = (k1 + w - 1).to(torch.int32)
                    k1 = k1.to(torch.int32)
                    off = torch.empty(nq + 1, dtype=torch.int64, device=dev)
                    capq = int(1.3 * L * nq) + (1 << 20)
                    rk = torch.empty(capq, dtype=torch.int32, device=dev)
                    rv = torch.empty(capq, dtype=torch.int32, device=dev)
                    c = torch.empty(nq, dtype=torch.int32, device=dev)
                    for rep in range(2):
                        torch.cuda.synchronize(dev)
                        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                        e0.record(st)
                        G.lsm_count(h, k1.data_ptr(), k2.data_ptr(), nq, c.data_ptr(), sp)
                        e1.record(st)
                        s_, tot = G.lsm_range(h, k1.data_ptr(), k2.data_ptr(), nq, off.data_ptr(), rk.data_ptr(),
                                              rv.data_ptr(), capq, sp)
                        e2.record(st)
                        e2.synchronize()
                    ranges[str(L)] = {"width": w, "count_M_per_s": nq / (e0.elapsed_time(e1) / 1000) / 1e6,
                                      "range_M_per_s": nq / (e1.elapsed_time(e2) / 1000) / 1e6,
                                      "results": int(tot), "status": int(s_)}
                resident = G.lsm_stats(h)["resident"]
                torch.cuda.synchronize(dev)
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(st)
                G.lsm_cleanup(h, sp)
                c1.record(st)
                c1.synchronize()
                clean_ms = c0.elapsed_time(c1)
                r_after = G.lsm_stats(h)["r"]
                errs = G.lsm_get_option(h, G.LSM_OPT_DEVICE_ERROR)
                G.lsm_destroy(h)
                m = nb.bit_length() - 1
                pt = {"b_log2": bl, "dist": dist, "delete_frac": frac, "batches": nb,
                      "M_updates_per_s": nb * b / upd_s / 1e6, "update_ms": 1000 * upd_s,
                      "algorithmic_B_per_update": 8 * m + 16,
                      "hbm_frac": (8 * m + 16) * nb * b / upd_s / 1e9 / float(measured_peaks()[0]["hbm_gbs"]),
                      "live_keys": n_live, "ranges": ranges, "cleanup_ms": clean_ms,
                      "cleanup_G_elements_per_s": resident / (clean_ms / 1000) / 1e9, "r_after_cleanup": r_after,
                      "device_errors": errs}
                points.append(pt)
                print("sweep point: %s" % json.dumps(pt), file=sys.stderr, flush=True)
                del keys, vals, dele
                torch.cuda.empty_cache()
    rates = [p["M_updates_per_s"] for p in points]
    geo = float(np.exp(np.mean(np.log(rates))))
    if rank == 0:
        line = {"metric": SWEEP_METRIC, "value": geo, "unit": "M updates/s (geometric mean over points)",
                "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": sum(p["update_ms"] for p in points),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic, drawn on the device (uniform keys over 2^30 or Zipf(1.1) by inverse transform; "
                        "deletes of earlier inserted keys)",
                "config": {"workload": "update/delete sweep: b = 2^%s, 2^%d updates per point, delete fraction "
                                       "0/25/50%%, uniform or Zipf(1.1) keys; 2^22 count and range queries at "
                                       "expected sizes 8/64/512; cleanup" % (args.sweep_b, args.sweep_total_log2),
                           "key_check": args.key_check, "l2": "inputs larger than L2", "parallelism": "single GPU"},
                "points": points, "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
