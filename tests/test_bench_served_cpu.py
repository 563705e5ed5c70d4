"""Host logic of bench.py's served-mix leg, on CPU: the client loop, the
latency bookkeeping (overall and for requests of at most 10^4 outputs) and the
plain one-request-at-a-time form, driven by a fake server that completes
requests in submission order with a latency proportional to their length."""
import sys
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from conftest import ROOT  # noqa: E402

sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeServer:
    def __init__(self, **kw):
        self.kw = kw
        self.pending, self.done = [], {}
        self.next_id = 1
        self.batches = 0

    def submit(self, v, m, dt, seed, jump, n):
        rid = self.next_id
        self.next_id += 1
        self.pending.append((rid, n))
        return rid

    def wait(self, rid):
        self.next_done(0)

    def next_done(self, timeout_us):
        if not self.pending:
            time.sleep(min(timeout_us, 1000) / 1e6)
            return None
        rid, n = self.pending.pop(0)
        self.done[rid] = n
        self.batches += 1
        return rid

    def poll(self, rid):
        return (2, None, 4 * self.done[rid], 1e-9 * self.done[rid])

    # batched forms
    @staticmethod
    def requests(rows):
        return list(rows)

    def submit_many(self, rows, first, count):
        return np.array([self.submit(*rows[first + k]) for k in range(count)], np.uint64)

    def next_done_many(self, timeout_us, cap):
        ids, lat = [], []
        rid = self.next_done(timeout_us)
        while rid is not None and len(ids) < cap:
            ids.append(rid)
            lat.append(self.poll(rid)[3])
            rid = self.next_done(0) if len(ids) < cap else None
        return np.array(ids, np.uint64), np.full(len(ids), 2, np.int32), np.array(lat)

    def release_many(self, ids):
        for rid in ids.tolist():
            self.release(rid)

    def release(self, rid):
        self.done.pop(rid, None)

    def stats(self):
        return {"batches": self.batches, "peak_output_bytes": 0, "host_launch_s": 0.0,
                "init_gpu_s": 0.0, "batch_gpu_s": 0.0, "express_batches": 0, "express_completed": 0,
                "queued_s": 0.0, "running_s": 0.0, "express_queued_s": 0.0, "express_running_s": 0.0,
                "express_init_gpu_s": 0.0, "express_batch_gpu_s": 0.0}

    def close(self):
        pass


class FakeGenerator:
    made = []

    def __init__(self, v, m, seeds, jumps):
        FakeGenerator.made.append((v, m, seeds, jumps))

    def generate(self, n, dt):
        return n

    def close(self):
        pass


class FakeVmt:
    Server = FakeServer
    VGenerator = FakeGenerator


class FakeStream:
    def synchronize(self):
        pass


@pytest.fixture
def no_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: FakeStream())


@pytest.mark.parametrize("client", ["batched", "single"])
def test_served_leg_reports_overall_and_small_request_latency(no_cuda, client):
    FakeGenerator.made.clear()
    requests, plain = 300, 40
    r = bench.run_served(FakeVmt, requests, 2.0e4, plain, client)
    assert r["batched"]["client"] == client
    tr = bench.I.request_trace(requests, rate_per_s=2.0e4)
    small = tr["n"] <= bench.SMALL_N
    b = r["batched"]
    assert r["requests"] == requests
    assert b["small_n_requests"] == int(small.sum()) > 0
    # the fake's latency is 1 ns per output, plus the submit lag (under a few ms)
    assert b["small_n_p50_ms"] is not None and b["small_n_p50_ms"] < b["p50_ms"]
    assert b["p99_ms"] >= b["p50_ms"] > 0
    p = r["plain"]
    assert p["requests"] == plain and len(FakeGenerator.made) == plain
    assert p["small_n_requests"] == int(small[:plain].sum())
    assert (p["small_n_p50_ms"] is None) == (p["small_n_requests"] == 0)
    assert p["throughput_GBps"] > 0


def test_percentiles_of_empty_sets_are_null():
    assert bench._ms([], 50) is None
    assert bench._ms([0.002, 0.004, 0.006], 50) == pytest.approx(4.0)
    assert np.isclose(bench._pct([1.0, 2.0, 3.0, 4.0], 50), 2.5)
