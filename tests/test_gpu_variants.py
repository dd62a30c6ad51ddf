"""Variants of the path (beyond the default configuration), on the GPU:
  * FP64 running charge of the front end (``fp64_charge``) over a long
    readout window: the digitised CSA charge against the oracle's FP64 front
    end fed the same FP32 current;
  * disabled channels (``disabled_pixels``): those pixels produce no hits and
    every other pixel's hits are unchanged."""
import numpy as np
import pytest
import torch

import oracle
from synth import events, params

from gpu_harness import Steps, compare_pixel_hits, hits_of_pixel, lut_pair

pytestmark = pytest.mark.gpu


def _long_window_case(fp64):
    cfg = params.small_config(n_ticks=20000, fp64_charge=fp64)
    seg = events.scatter_event(cfg, 77, 40, max_len=0.7, t_range=(0.0, 1800.0))   # arrivals over 2 ms
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=9).all()
    return cfg, st, oracle.Oracle(cfg, params.LUT, lut64)


def test_fp64_running_charge_long_window():
    worst = {}
    for fp64 in (0, 1):
        cfg, st, o = _long_window_case(fp64)
        m, cur, h = st.maps_np(), st.current_np(), st.hits_np()
        band = 0.05
        dq, n_cmp, n_hit_pix, n_tied = [0.0], 0, 0, 0
        for i, p in enumerate(m["active"]):
            ref = o.electronics(int(p), cur[i].astype(np.float64), event_id=9, band=band)
            g = hits_of_pixel(h, int(p))
            n_hit_pix += bool(len(ref["t_cross"]) or len(g["t_cross"]))
            n_tied += ref["tie_tick"] >= 0
            ok, nc = compare_pixel_hits(g, ref, 976.5625)
            assert ok, (fp64, p)
            n_cmp += nc
            if nc:
                dq.append(float(np.abs(g["q"][:nc].astype(np.float64) - ref["q"][:nc]).max()))
        assert n_cmp > 20 and n_tied <= max(1, 0.02 * n_hit_pix)
        worst[fp64] = max(dq)
    print(f"long window: max |q_gpu - q_oracle| FP32 sum {worst[0]:.3e} e-, FP64 sum {worst[1]:.3e} e-")
    assert worst[1] <= 2e-3            # FP32 noise normals and FP32 rounding of the stored charge only
    assert worst[1] <= worst[0]


def test_disabled_pixels_have_no_hits():
    cfg = params.small_config()
    seg = events.scatter_event(cfg, 101, 60, max_len=0.6)
    lut_dev, _ = lut_pair(cfg)
    base = Steps(cfg, seg, lut_dev, event_id=5).all()
    m, h0 = base.maps_np(), base.hits_np()
    hit_pix = np.unique(h0["pixel"])
    assert len(hit_pix) > 10
    off = hit_pix[::3]                                  # disable a third of the hit-bearing pixels
    words = np.zeros((params.geometry(cfg)["n_pixels"] + 31) // 32, dtype=np.uint32)
    np.bitwise_or.at(words, off // 32, (np.uint32(1) << (off % 32).astype(np.uint32)))
    mask = torch.as_tensor(words.view(np.int32), device="cuda")
    st = Steps(dict(cfg, disabled_pixels=mask), seg, lut_dev, event_id=5).all()
    h1 = st.hits_np()
    assert not np.isin(h1["pixel"], off).any()
    keep = ~np.isin(h0["pixel"], off)
    for k in ("pixel", "t_cross", "t_adc", "adc", "q"):
        assert np.array_equal(h1[k], h0[k][keep]), k
    assert np.array_equal(st.current_np(), base.current_np())   # currents are still computed


@pytest.mark.parametrize("precision", [0, 2])
def test_per_point_drift_against_oracle(precision):
    """Per-point lifetime and widths (short lifetime: 60 us): the map (up to
    pixels at the radius within FP32 rounding) and every pixel's current
    against the oracle, in both current forms."""
    from gpu_harness import current_errors
    cfg = params.small_config(per_point_drift=1, lifetime_us=60.0, precision=precision)
    seg = events.scatter_event(cfg, 311, 60, max_len=1.5)
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=4).quench_drift().pixel_map().induced_current()
    m, cur = st.maps_np(), st.current_np()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    g = st.drifted_np()
    np.testing.assert_allclose(g["sigma_T"], d["sigma_T"], rtol=2e-6, atol=1e-30)   # farther end's width
    ref_pix, _, _, _ = o.pixel_map(seg, d)
    assert len(set(m["active"].tolist()) ^ set(ref_pix)) <= 2
    ref = np.array([o.pixel_current(seg, d, int(p), m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]], event_id=4)
                    for i, p in enumerate(m["active"])])     # the same segment lists on both sides
    sig = np.abs(ref).sum(-1) >= 1.0
    rel, qrel = current_errors(cur[sig], ref[sig])
    print(f"per-point drift, precision {precision}: pixels {sig.sum()} rel max {rel.max():.2e} q max {qrel.max():.2e}")
    assert rel.max() <= (1e-4 if precision == 0 else 1e-3)
    # the variant is visible: per-segment drift distributes the charge differently along the
    # segments (the totals agree to second order), compared on the pixels both maps hold
    cfg0 = dict(cfg, per_point_drift=0)
    st0 = Steps(cfg0, seg, lut_dev, event_id=4).quench_drift().pixel_map().induced_current()
    a0 = st0.maps_np()["active"]
    common, i1, i0 = np.intersect1d(m["active"], a0, return_indices=True)
    diff = np.abs(cur[i1] - st0.current_np()[i0]).max() / np.abs(cur[i1]).max()
    assert diff > 1e-3, diff


@pytest.mark.parametrize("precision", [0, 2])
def test_nearest_lookup_against_oracle(precision):
    """Nearest-bin lookup: every pixel against the oracle.  A point whose
    nearest-node or nearest-tick rounding lies within 1e-3 (bins, ticks) of
    its half-way point may round the other way in FP32: each such point may
    move its charge q to another table row, so the allowed difference is the
    form's tolerance plus 2 q max|R| per tied point (counted by the oracle)."""
    cfg = params.small_config(nearest_lut=1, precision=precision)
    seg = events.scatter_event(cfg, 411, 50, max_len=0.8)
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=6).quench_drift().pixel_map().induced_current()
    m, cur = st.maps_np(), st.current_np()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    rmax = float(np.abs(lut64).max())
    tol = 1e-4 if precision == 0 else 1e-3
    n_ties_total, checked = 0, 0
    for i, p in enumerate(m["active"]):
        segs = m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]]
        ref, n_ties = o.pixel_current(seg, d, int(p), segs, event_id=6, tie_band=1e-3)
        if np.abs(ref).sum() < 1.0:
            continue
        qmax = max(d["Qa"][s] / d["n_samples"][s] for s in segs if d["n_samples"][s] > 0)
        bound = tol * np.abs(ref).max() + n_ties * 2 * qmax * rmax
        assert np.abs(cur[i] - ref).max() <= bound, (p, n_ties)
        n_ties_total += n_ties
        checked += 1
    print(f"nearest lookup, precision {precision}: pixels {checked}, tied points {n_ties_total}")
    assert checked > 100
