"""Host logic of the serving loop that needs no GPU: the admission rule, the
initial capacities and the latency summaries (paper_2212_09807_gb300/serve.py)."""
import numpy as np

from paper_2212_09807_gb300 import serve

GB = 1e9


class J:
    """A waiting request as the admission rule sees it: its name, size class and bytes."""

    def __init__(self, name, gb, large=False):
        self.name, self.bytes, self.large = name, gb * GB, large

    def __repr__(self):
        return self.name


def admit(waiting, n_running=0, large_running=False, used_gb=0.0, budget_gb=100.0, max_jobs=8):
    out = serve.admission(waiting, n_running, large_running, used_gb * GB, budget_gb * GB, max_jobs,
                          lambda j: j.large, lambda j: j.bytes)
    return [j.name for j in out]


def test_first_fit_in_arrival_order_within_the_budget():
    w = [J("a", 30), J("b", 50), J("c", 40), J("d", 10)]
    assert admit(w, used_gb=0) == ["a", "b", "d"]                 # c would exceed 100 GB; d still fits
    assert admit(w, n_running=1, used_gb=70) == ["a"]             # 70 + 30 = 100 fits exactly; nothing else


def test_a_request_larger_than_the_budget_runs_alone():
    w = [J("huge", 300), J("small", 1)]
    assert admit(w) == ["huge"]                                   # nothing on the GPU: admitted anyway
    assert admit(w, n_running=1, used_gb=5) == ["small"]          # otherwise it waits


def test_the_job_limit():
    w = [J(str(i), 1) for i in range(10)]
    assert admit(w, max_jobs=4) == ["0", "1", "2", "3"]
    assert admit(w, n_running=3, used_gb=3, max_jobs=4) == ["0"]
    assert admit(w, n_running=4, used_gb=4, max_jobs=4) == []


def test_large_requests_one_at_a_time_in_arrival_order():
    w = [J("L1", 20, True), J("s", 1), J("L2", 20, True)]
    assert admit(w) == ["L1", "s"]                                # the second large one waits for the first
    assert admit(w, n_running=1, large_running=True, used_gb=20) == ["s"]
    # a large request waiting for the budget holds back the large ones behind it, not the small ones
    w = [J("L1", 90, True), J("L2", 10, True), J("s", 5)]
    assert admit(w, n_running=1, used_gb=20) == ["s"]
    assert admit(w, n_running=0) == ["L1", "s"]


def test_initial_capacities_grow_with_the_event():
    a, b = serve._caps(1000), serve._caps(100000)
    assert all(x < y for x, y in zip(a, b))
    assert serve._caps(1000, 2.0) == tuple(int(2.0 * (m * 1000 + 10000)) for m in (30, 0.8, 4))


def test_latency_summary_and_bootstrap_spread():
    rng = np.random.default_rng(0)
    res = []
    for i in range(200):
        arr = 0.01 * i
        lat = rng.exponential(0.05) + (1.0 if i % 10 == 0 else 0.0)
        res.append(serve.Result(i, "spill" if i % 10 == 0 else "nu", 1000, arr, arr, arr + lat, [0, 0, 0, 0], {}))
    s = serve.summarize(res)
    lat = np.array([r.latency for r in res]) * 1e3
    assert s["requests"] == 200
    assert s["latency_ms"]["p99"] == float(np.percentile(lat, 99))
    lo, hi = s["latency_ms"]["p99_spread"]
    assert lo <= s["latency_ms"]["p99"] <= hi
    assert s["latency_ms_spill"]["n"] == 20 and s["latency_ms_nu"]["n"] == 180
    assert s["latency_ms_spill"]["p50"] > 900 > s["latency_ms_nu"]["p99"]
    span = max(r.done for r in res) - min(r.arrival for r in res)
    assert abs(s["segments_per_s"] - 200 * 1000 / span) < 1e-6 * s["segments_per_s"]
