"""The benchmark's GPU arms (paper scale, batched and serving forms),
dry-run on the CPU: the library binding and torch's CUDA calls replaced by
stand-ins that do no work, so that the Python around the timed region
(argument handling, phase timing, the roofline, per-batch and worst-case
figures, the end-to-end leg, the oracle baseline and the JSON line) runs
without a GPU.  The numbers it prints mean nothing; the tests check that
each arm prints its line once, with the contract's shape."""

import contextlib
import json
import sys
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class FakeEvent:
    _clock = 0.0

    def __init__(self, *a, **k):
        self.t = 0.0

    def record(self, stream=None):
        FakeEvent._clock += 0.25
        self.t = FakeEvent._clock

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return max(other.t - self.t, 1e-3)


class FakeStream:
    cuda_stream = 0

    def __init__(self, *a, **k):
        pass

    def wait_event(self, ev):
        pass


def fake_library(real):
    """A stand-in for the ctypes binding: the real constants, calls that do
    nothing but count themselves as launches, and a profiler that reports
    ten launches, 1 ms and 1 GB for every kernel group."""
    g = types.SimpleNamespace()
    for name in dir(real):
        if name.startswith(("LSM_", "PROF_", "SERVE_", "REQ_")):
            setattr(g, name, getattr(real, name))
    state = {"launches": 0}

    def launch(*a, **k):
        state["launches"] += 1
        return 0

    for name in ("lsm_set_option", "lsm_reset", "lsm_insert_batch", "lsm_stream_wait", "lsm_lookup",
                 "lsm_count", "lsm_cleanup", "lsm_profile", "lsm_destroy", "lsm_bulk_build"):
        setattr(g, name, launch)
    g.lsm_stats = lambda h: dict(r=1, resident=1, b=1, levels=1)
    g.lsm_create = lambda b, n, dev=0: 1
    g.lsm_range = lambda h, k1, k2, nq, off, rk, rv, cap, s=None: (real.LSM_OK, min(cap, 8 * nq))
    g.lsm_get_option = lambda h, opt: 0
    g.kernel_launches = lambda: state["launches"]
    g.lsm_profile_read = lambda h: {n: dict(launches=10, ms=1.0, bytes=1e9) for n in real.PROF_GROUPS}
    g.lsm_update_batch = launch
    g.lsm_multi_round = launch
    g.lsm_multi_get_option = lambda h, opt: 8

    class MultiLSM:
        def __init__(self, sizes, max_batches, tuning=None, device=0):
            assert len(tuning) == len(sizes)
            self.h, self.n = 2, len(sizes)

        def reset(self):
            launch()

        def sync(self):
            return real.LSM_OK, [0] * self.n

        def close(self):
            pass

    g.MultiLSM = MultiLSM

    class Server:
        def __init__(self, b, budget, **kw):
            self.b = b

        def set_pool(self, a, v, c):
            self.pool = len(a)

        def preload(self, k, v):
            launch()

        def run(self, kind, arrival, start, size, keep_results=False):
            launch()
            n = len(kind)
            return {"wall_us": float(arrival[-1]) + 500.0, "done_us": arrival.astype(float) + 100.0,
                    "status": np.zeros(n, np.int32), "update_batches": 3,
                    "padded_ops": 0, "retrieval_groups": 5, "cleanups": 0, "refused": 0, "range_total": 7,
                    "time_split": {"host_admission_s": 0.0}}

        def stats(self):
            return {"levels": 11, "device_bytes": 1 << 30, "resident": 1 << 20}

        def close(self):
            pass

    g.Server = Server
    return g


@pytest.fixture
def dry_gpu(monkeypatch, lsm_lib):
    cpu = torch.device("cpu")
    monkeypatch.setattr(torch, "device", lambda *a, **k: cpu)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: FakeStream())
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    pkg = sys.modules["paper_1707_05354_gb300"]
    monkeypatch.setattr(pkg, "gpulsm", fake_library(lsm_lib), raising=False)
    monkeypatch.setitem(sys.modules, "paper_1707_05354_gb300.gpulsm", pkg.gpulsm)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)


def test_gpu_arm_prints_the_contract_line(dry_gpu, monkeypatch, capsys):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "4", "--warmup", "3", "--b-log2", "10",
                                      "--batches", "8", "--lookups-log2", "12", "--queries-log2", "10"])
    assert bench.run_gpu(bench.parse_args()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks", "update_phase_roofline", "lookups", "per_batch"):
        assert key in line, key
    assert line["metric"] == bench.METRIC and line["unit"] == "M updates/s"
    assert line["steps"] == 4 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["config"]["b"] == 1024 and line["config"]["batches"] == 8 and "workload" in line["config"]
    rf = line["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["kernel"] == "merge"
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-12
    assert rf["achieved"] == pytest.approx(1e9 / 1e-3 / 1e9)          # 1 GB in 1 ms (the stand-in profile)
    assert line["update_phase_roofline"]["bytes_per_update"] == 8 * 3 + 16   # 8 batches: m = 3
    assert line["gpu_launches"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    e2e = line["e2e"]
    assert e2e["unit"] == line["unit"] and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] == 8 * 1024 * 8 + 4096 * 4 + 1024 * 8 + 1024 * 8


def test_batched_arm_prints_the_contract_line(dry_gpu, monkeypatch, capsys):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "batched", "--steps", "2", "--warmup", "3",
                                      "--instances", "3", "--rounds", "4", "--no-tune"])
    assert bench.run_batched(bench.parse_args()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches",
                "plain_calls", "tuning"):
        assert key in line, key
    assert line["metric"] == bench.BATCHED_METRIC
    assert line["config"]["instances"] == 3 and line["config"]["rounds"] == 4
    tot = line["config"]["updates_per_round"]
    assert line["e2e"]["h2d_bytes_per_step"] == 4 * tot * 13
    assert line["roofline"]["algorithmic_bytes_per_step"] > 16 * tot
    assert line["cpu_baseline"]["kind"] == "oracle" and line["plain_calls"]["value"] > 0


def test_serving_arm_prints_the_contract_line(dry_gpu, monkeypatch, capsys):
    import bench
    from paper_1707_05354_gb300 import workload
    real_pools = workload.serving_pools
    monkeypatch.setattr(workload, "serving_pools", lambda n=0, **k: real_pools(n=1 << 12, **k))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "serving", "--requests", "2000", "--b-log2", "10",
                                      "--preload-batches", "2", "--warmup", "1"])
    assert bench.run_serving(bench.parse_args()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "latency_ms", "continuous", "fixed_batching", "vs_fixed",
                "heavier_load", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["metric"] == bench.SERVING_METRIC and line["config"]["requests"] == 2000
    assert line["latency_ms"]["p50"] == pytest.approx(0.1)                 # done = arrival + 100 us
    assert line["e2e"]["h2d_bytes_per_step"] == 21 * 2000
    assert line["heavier_load"]["rate_per_s"] == 6.0e5
    assert np.isfinite(line["value"]) and line["value"] > 0
