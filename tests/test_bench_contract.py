"""The JSON line of ``bench.py --impl reference`` (the oracle timed on the host cores,
no GPU needed): one line, the same metric and workload as the GPU arm, and the keys
the measurement contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.CONFIG["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_timed_calls_are_queued_before_any_read_back():
    """bench.queued_times records every event pair and issues every call before the one
    synchronisation that precedes the first read-back, and drops the first ``skip``."""
    sys.path.insert(0, ROOT)
    import bench

    log = []

    class Ev:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self):
            self.t = len(log)
            log.append("record")

        def elapsed_time(self, other):
            assert "sync" in log, "read back before the synchronisation"
            return float(other.t - self.t)

    class Cuda:
        Event = Ev

        @staticmethod
        def synchronize():
            log.append("sync")

    class FakeTorch:
        cuda = Cuda

    class Flush:
        def fill_(self, v):
            log.append("flush")

    times = bench.queued_times(FakeTorch, lambda k: log.append(f"step{k}"), 5, Flush(), skip=2)
    assert log.count("sync") == 1 and log[-1] == "sync"
    assert [x for x in log if x.startswith("step")] == [f"step{k}" for k in range(5)]
    assert len(times) == 3 and all(t == 2.0 for t in times)  # record, step, record: the flush sits outside
