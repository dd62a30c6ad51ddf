"""Serving form: requests admitted while others run, overlapping on the GPU,
give each the result they give alone (run_plain: one sim_event per request).
FP32 form: hits and currents bit for bit.  Tensor-core form: hits-bearing
pixels identical, currents within 1e-5 of each pixel's peak (its pixel groups
are formed per current slice)."""
import numpy as np
import pytest

from paper_2212_09807_gb300 import serve
from synth import events, params

from gpu_harness import lut_pair

pytestmark = pytest.mark.gpu


def _requests(cfg):
    reqs = []
    sizes = [40, 3000, 25, 60, 0, 35, 80, 1500]
    for i, n in enumerate(sizes):
        seg = events.scatter_event(cfg, 500 + i, n, max_len=0.7)
        reqs.append(serve.Request(rid=i, event_id=1000 + 7 * i, seg=seg, arrival=0.002 * i,
                                  kind="large" if n >= 1500 else "small"))
    return reqs


def _by_rid(results):
    return {r.rid: r for r in results}


def _check_same(mix, alone, exact):
    for rid, a in alone.items():
        m = mix[rid]
        assert m.counts[1] == a.counts[1] and m.counts[0] == a.counts[0]
        assert np.array_equal(m.active, a.active)
        if exact:
            assert np.array_equal(m.current, a.current), rid
            assert m.counts == a.counts
            for k in a.hits:
                assert np.array_equal(m.hits[k], a.hits[k]), (rid, k)
        elif a.counts[1]:
            scale = np.maximum(np.abs(a.current).max(axis=1, keepdims=True), 1e-30)
            assert float((np.abs(m.current - a.current) / scale).max()) <= 1e-5, rid


@pytest.mark.parametrize("precision", [0, 2])
def test_serving_results_equal_alone(precision):
    cfg = params.small_config(precision=precision)
    lut_dev, _ = lut_pair(cfg)
    reqs = _requests(cfg)
    srv = serve.Server(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], hbm_budget=64e9,
                       slice_pixels=256, max_jobs=6, keep_current=True)
    mix = _by_rid(srv.run(reqs))
    alone = _by_rid(serve.run_plain(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"],
                                    [serve.Request(r.rid, r.event_id, r.seg, 0.0, r.kind) for r in reqs],
                                    keep_current=True))
    assert set(mix) == set(alone) == {r.rid for r in reqs}
    # the work overlapped: some request was admitted before an earlier-admitted one finished
    spans = sorted((m.admitted, m.done) for m in mix.values())
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    _check_same(mix, alone, exact=(precision == 0))
    assert sum(a.counts[2] for a in alone.values()) > 20          # the events make hits


def test_serving_under_a_small_budget_admits_one_at_a_time():
    cfg = params.small_config()
    lut_dev, _ = lut_pair(cfg)
    reqs = _requests(cfg)[:4]
    srv = serve.Server(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], hbm_budget=1.0,
                       slice_pixels=256, max_jobs=4, keep_current=True)
    mix = _by_rid(srv.run(reqs))
    spans = sorted((m.admitted, m.done) for m in mix.values())
    assert all(spans[i + 1][0] >= spans[i][1] for i in range(len(spans) - 1))
    alone = _by_rid(serve.run_plain(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"],
                                    [serve.Request(r.rid, r.event_id, r.seg, 0.0, r.kind) for r in reqs],
                                    keep_current=True))
    _check_same(mix, alone, exact=True)
    s = serve.summarize(list(mix.values()))
    assert s["requests"] == 4 and s["latency_ms"]["p99"] >= s["latency_ms"]["p50"] > 0
