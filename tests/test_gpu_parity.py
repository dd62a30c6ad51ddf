"""GPU parity of every step of the CUDA path against the FP64 oracle, called
through the C ABI.

Tolerances (stated once, used below):
  * Q_a, t_drift, sigma_T, sigma_L: FP32 evaluation of closed forms, rtol 2e-6;
    anode and point count N: exact (decided in FP64 on both sides);
  * pixel map: set-equal, except pairs whose oracle distance margin is within
    1e-5 cm of the map radius (FP32 geometry on the GPU);
  * current (FP32 form on the CUDA cores): per pixel ||I_gpu - I_ref||_inf <= 1e-4 ||I_ref||_inf
    (hard; faint neighbour pixels whose bipolar current nearly cancels reach ~1e-4)
    with the median <= 1e-6; every prefix sum of each pixel's current
    (the charge integrated by each tick) within 1e-5 of the pixel's largest one
    plus 2e-6 of the event's peak pixel charge (gpu_harness.prefix_charge_ok:
    the floor covers pixels fed through small interpolation weights, whose
    absolute error follows the FP32 rounding of their neighbours' points);
  * hits: bit-exact pixel, t_cross, t_adc and ADC code up to the oracle's first
    tie (a threshold or ADC decision within the band of its threshold); the
    tied pixels, picked by the oracle's trace alone, number at most
    gpu_harness.tie_cap of the oracle's tie probabilities.  End to end the band
    is gpu_harness.BAND[0] = 0.2 e- (the FP32 form's charge error at the
    decisions); on the GPU's own current 0.05 e- (FP32 scan and noise
    rounding, ~1e-3 e-).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import sim
from synth import events, params, response

from gpu_harness import (BAND, Steps, compare_pixel_hits, current_errors, hits_of_pixel, lut_pair, prefix_charge_ok,
                         tie_cap)

pytestmark = pytest.mark.gpu

MAP_BAND = 1e-5
CUR_HARD, CUR_MED, Q_TOL = 1e-4, 1e-6, 1e-5


def _edge_segments(cfg):
    """Degenerate cases appended to the random events: zero length, midpoint
    outside, on the cathode, exactly 10 um long, a long diagonal, near a tile
    corner and on the detector edge."""
    g = params.geometry(cfg)
    D = g["drift"]
    rows = [
        (5.0, 5.0, 10.0, 0.0, 5.0, 5.0, 10.0, 0.0, 1.0),
        (-3.0, 5.0, 10.0, 0.0, -2.5, 5.0, 10.0, 0.0, 1.0),
        (8.0, 9.0, D - 0.05, 0.0, 8.2, 9.1, D + 0.05, 0.0, 0.3),
        (12.0, 13.0, 20.0, 0.0, 12.001, 13.0, 20.0, 0.0, 0.002),
        (10.0, 10.0, 5.0, 0.0, 10.7, 10.6, 6.0, 0.0, 2.5),
        (31.0, 31.0, 40.0, 1.0, 31.1, 31.05, 40.3, 1.0, 0.5),
        (0.05, 0.1, 3.0, 0.0, 0.4, 0.2, 3.2, 0.0, 0.6),
    ]
    a = np.asarray(rows, dtype=np.float32)
    return {k: a[:, i] for i, k in enumerate(events.COLS)}


def _event(cfg, seed, n, max_len=0.6, t_range=(0.0, 0.0)):
    seg = events.scatter_event(cfg, seed, n, max_len=max_len, t_range=t_range)
    e = _edge_segments(cfg)
    return {k: np.concatenate([seg[k], e[k]]).astype(np.float32) for k in events.COLS}


@pytest.fixture(scope="module")
def small():
    cfg = params.small_config()
    seg = _event(cfg, 101, 60)
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=5).all()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    return dict(cfg=cfg, seg=seg, st=st, o=o, d=o.quench_drift(seg), lut_dev=lut_dev, lut64=lut64)


@pytest.mark.parametrize("model", [0, 1])
def test_quench_drift(model):
    cfg = params.small_config(recomb_model=model)
    seg = _event(cfg, 7 + model, 300)
    lut_dev, _ = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev).quench_drift()
    g = st.drifted_np()
    d = oracle.Oracle(cfg, params.LUT).quench_drift(seg)
    assert np.array_equal(g["anode"], d["anode"])
    assert np.array_equal(g["n_samples"], d["n_samples"])
    for k in ("Qa", "t_drift", "sigma_T", "sigma_L"):
        np.testing.assert_allclose(g[k], d[k], rtol=2e-6, atol=1e-30, err_msg=k)
    assert (d["anode"] < 0).sum() >= 2   # degenerate segments present and inactive


def test_recombination_closed_form_values_gpu():
    """Q_R / Q_0 of the GPU's quench step at 2.1, 5, 10 and 20 MeV/cm against the
    hand-evaluated closed forms of Eq. (birks) / Eq. (box) (tests/golden), to
    1e-5.  R is recovered from the outputs as Q_a e^(t_drift/tau) W_ion / dE."""
    import os
    rows = []
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", "recombination_closed_form.txt")):
        f = ln.split("#")[0].split()
        if f:
            rows.append((f[0], float(f[1]), float(f[2])))
    for model, name in ((0, "birks"), (1, "box")):
        cfg = params.small_config(recomb_model=model)
        ref = [(d, r) for m, d, r in rows if m == name]
        a = np.asarray([(5.0, 5.0, 3.0, 0.0, 5.5, 5.0, 3.0, 0.0, 0.5 * d) for d, _ in ref], dtype=np.float32)
        seg = {k: np.ascontiguousarray(a[:, i]) for i, k in enumerate(events.COLS)}
        lut_dev, _ = lut_pair(cfg)
        g = Steps(cfg, seg, lut_dev).quench_drift().drifted_np()
        assert np.all(g["anode"] >= 0)
        R = (g["Qa"].astype(np.float64) * np.exp(g["t_drift"].astype(np.float64) / np.float64(np.float32(cfg["lifetime_us"])))
             * np.float64(np.float32(cfg["w_ion_MeV"])) / seg["dE"].astype(np.float64))
        np.testing.assert_allclose(R, [r for _, r in ref], rtol=1e-5, atol=0, err_msg=name)


def test_pixel_map(small):
    st, o, seg, d = small["st"], small["o"], small["seg"], small["d"]
    m = st.maps_np()
    n = len(seg["x0"])
    seen_ties = 0
    for s in range(n):
        gpu = set(m["seg_ids"][m["seg_off"][s]:m["seg_off"][s + 1]].tolist())
        ids, mg = o.map_segment(seg, d, s)
        ref = set(ids.tolist())
        for p in ref - gpu:
            assert mg[list(ids).index(p)] < MAP_BAND, (s, p)
            seen_ties += 1
        for p in gpu - ref:
            assert o.pair_margin(seg, d, s, p) > -MAP_BAND, (s, p)
            seen_ties += 1
    assert seen_ties <= 2
    act = m["active"]
    assert np.all(np.diff(act) > 0)                         # increasing pixel ids
    assert set(act.tolist()) == set(m["seg_ids"].tolist())
    for i, p in enumerate(act):
        lst = m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]]
        assert np.all(np.diff(lst) > 0)                     # segment order fixed
        assert all(p in m["seg_ids"][m["seg_off"][s]:m["seg_off"][s + 1]] for s in lst)


def _current_parity(cfg, seg, lut_dev, lut64, event_id=0, lut_par=None, frac=1.0):
    lut_par = lut_par or params.LUT
    st = Steps(cfg, seg, lut_dev, event_id=event_id, lut_par=lut_par).quench_drift().pixel_map().induced_current()
    m = st.maps_np()
    cur = st.current_np()
    o = oracle.Oracle(cfg, lut_par, lut64)
    d = o.quench_drift(seg)
    idx = np.arange(len(m["active"]))
    if frac < 1.0:
        idx = np.random.default_rng(0).choice(idx, max(8, int(frac * len(idx))), replace=False)
    refs = []
    for i in idx:
        segs = m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]]
        refs.append(o.pixel_current(seg, d, int(m["active"][i]), segs, event_id=event_id))
    ref = np.array(refs)
    rel, qrel = current_errors(cur[idx], ref)
    big = np.abs(ref).max(axis=1) > 0
    q_ok, q_worst = prefix_charge_ok(cur[idx], ref, Q_TOL)
    return rel[big], qrel[big], ref, q_ok, q_worst


def test_induced_current_all_pixels(small):
    rel, qrel, ref, q_ok, q_worst = _current_parity(small["cfg"], small["seg"], small["lut_dev"], small["lut64"],
                                                    event_id=5)
    assert len(rel) > 200
    print(f"all pixels: rel max {rel.max():.2e} med {np.median(rel):.2e}, prefix-charge worst {q_worst:.2e}")
    assert rel.max() <= CUR_HARD, rel.max()
    assert np.median(rel) <= CUR_MED, np.median(rel)
    assert q_ok, q_worst


def test_term_by_term_form_all_pixels(small):
    """precision 3, the FP32 term-by-term gather (each record's bilinear and
    linear table reads summed per tick, no regrouping by table node): every
    pixel against the oracle at the FP32 tolerances of the first build of
    this form (max 1e-4, median 1e-5, prefix charge 1e-5 plus the floor)."""
    cfg = dict(small["cfg"], precision=3)
    rel, qrel, ref, q_ok, q_worst = _current_parity(cfg, small["seg"], small["lut_dev"], small["lut64"], event_id=5)
    print(f"term by term: rel max {rel.max():.2e} med {np.median(rel):.2e}, prefix-charge worst {q_worst:.2e}")
    assert len(rel) > 200
    assert rel.max() <= 1e-4, rel.max()
    assert np.median(rel) <= 1e-5, np.median(rel)
    assert q_ok, q_worst


@pytest.mark.parametrize("case", ["M4", "ragged_window", "box_shifted", "bipolar"])
def test_induced_current_variants(case):
    over, lut_kw, tr = {}, {}, (0.0, 0.0)
    if case == "M4":
        over = dict(mc_per_sample=4)
    elif case == "ragged_window":
        over = dict(n_ticks=2500, t_window0_us=-37.3)           # two tick chunks, ragged tail
    elif case == "box_shifted":
        over = dict(recomb_model=1, t_window0_us=3.05)
        tr = (0.0, 9.0)
    elif case == "bipolar":
        lut_kw = dict(bipolar=0.5)
    cfg = params.small_config(**over)
    seg = _event(cfg, 300 + len(case), 25, t_range=tr)
    lut_dev, lut64 = lut_pair(cfg, **lut_kw)
    rel, qrel, _, q_ok, q_worst = _current_parity(cfg, seg, lut_dev, lut64, event_id=11)
    print(f"{case}: rel max {rel.max():.2e} med {np.median(rel):.2e}, prefix-charge worst {q_worst:.2e}")
    assert rel.max() <= CUR_HARD, rel.max()
    assert np.median(rel) <= CUR_MED
    if case != "bipolar":                  # bipolar pixels can integrate to ~0
        assert q_ok, q_worst


def test_electronics_bit_exact_on_same_current(small):
    """Same FP32 current into both front ends: hits must agree up to ties."""
    st, o, cfg = small["st"], small["o"], small["cfg"]
    m = st.maps_np()
    cur = st.current_np()
    h = st.hits_np()
    band = 0.05                        # electrons; FP32 scan vs FP64 sum differ by ~1e-3 e-
    n_hit_pix, n_tied, n_cmp, p_ties = 0, 0, 0, []
    for i, p in enumerate(m["active"]):
        ref = o.electronics(int(p), cur[i].astype(np.float64), event_id=5, band=band)
        g = hits_of_pixel(h, int(p))
        if len(ref["t_cross"]) or len(g["t_cross"]):
            n_hit_pix += 1
            p_ties.append(ref["p_tie"])
        if ref["tie_tick"] >= 0:
            n_tied += 1
        ok, nc = compare_pixel_hits(g, ref, 976.5625)
        assert ok, (p, ref, g)
        n_cmp += nc
        mref = ref["t_adc"] < (ref["tie_tick"] if ref["tie_tick"] >= 0 else 1 << 30)
        np.testing.assert_allclose(g["q"][: mref.sum()], ref["q"][mref], rtol=1e-5, atol=0.05)
    assert n_cmp > 20
    assert n_tied <= tie_cap(p_ties)


def test_electronics_closed_form_gpu():
    """Noise off, constant current per pixel: first crossing, ADC code and period."""
    cfg = params.small_config(sigma_reset_e=0.0, sigma_disc_e=0.0, sigma_unc_e=0.0, n_ticks=1000)
    c = sim.make_config(cfg)
    dev = torch.device("cuda:0")
    iv = np.array([37.0, 333.0, 1250.5, 4999.0, 7000.0, 10.0], dtype=np.float32)
    P = len(iv)
    cur = torch.as_tensor(np.repeat(iv[:, None], 1000, axis=1), device=dev)
    active = torch.arange(P, dtype=torch.int32, device=dev) * 7
    hits = sim.Hits(10000, dev)
    ws = torch.zeros((sim.workspace_size(c, 0, 0, P) + 7) // 8, dtype=torch.int64, device=dev)
    counts = ws[:4]
    counts[1] = P
    sim.sim_electronics(c, 0, active, cur, counts, hits, ws)     # event id 0
    torch.cuda.synchronize()
    n = int(counts[2])
    h = hits.to_numpy(n)
    for j, i in enumerate(iv):
        g = hits_of_pixel(h, 7 * j)
        n_up = int(np.ceil(np.float32(5000.0) / i))
        t1 = n_up - 1
        if t1 + 16 >= 1000:
            assert len(g["t_cross"]) == 0
            continue
        assert g["t_cross"][0] == t1 and g["t_adc"][0] == t1 + 16
        assert g["adc"][0] == min(255, int(np.floor(np.float32((t1 + 17) * i) / np.float32(976.5625))))
        assert np.all(np.diff(g["t_cross"]) == 16 + n_up)


def test_electronics_adc_range_gpu():
    """Noise off: a current far above the ADC range saturates every code at
    2^8 - 1, and a charge that crossed the threshold and is negative when the
    ADC samples it (a bipolar current) digitises as 0; hits bit-exact with
    the oracle's front end on the same current."""
    cfg = params.small_config(sigma_reset_e=0.0, sigma_disc_e=0.0, sigma_unc_e=0.0, n_ticks=1000)
    c = sim.make_config(cfg)
    dev = torch.device("cuda:0")
    I = np.zeros((2, 1000), np.float32)
    I[0, :] = 1.0e6                                   # ~1000 ADC counts' worth per tick
    I[1, 10] = 5010.0                                  # crosses the 5000 e- threshold at tick 10
    I[1, 11] = -20000.0                                # negative at the ADC tick (10 + 16)
    P = 2
    cur = torch.as_tensor(I, device=dev)
    active = torch.tensor([3, 11], dtype=torch.int32, device=dev)
    hits = sim.Hits(10000, dev)
    ws = torch.zeros((sim.workspace_size(c, 0, 0, P) + 7) // 8, dtype=torch.int64, device=dev)
    counts = ws[:4]
    counts[1] = P
    sim.sim_electronics(c, 0, active, cur, counts, hits, ws)
    torch.cuda.synchronize()
    h = hits.to_numpy(int(counts[2]))
    o = oracle.Oracle(cfg, params.LUT)
    for row, pid in enumerate((3, 11)):
        g = hits_of_pixel(h, pid)
        r = o.electronics(pid, I[row].astype(np.float64), event_id=0)
        assert len(g["t_cross"]) == len(r["t_cross"]) > 0
        for k in ("t_cross", "t_adc", "adc"):
            assert np.array_equal(g[k], r[k]), (pid, k)
        assert np.allclose(g["q"], r["q"], rtol=1e-6)
    assert np.all(hits_of_pixel(h, 3)["adc"] == 255)
    assert list(hits_of_pixel(h, 11)["adc"]) == [0]


def test_event_matches_steps_and_is_deterministic(small):
    cfg, seg, lut_dev = small["cfg"], small["seg"], small["lut_dev"]
    st = small["st"]
    run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], len(seg["x0"]),
                          st.pair_cap, st.pix_cap, st.hit_cap)
    S = sim.Segments.from_numpy(seg, 5)
    outs = []
    for _ in range(2):
        run.enqueue(S)
        torch.cuda.synchronize()
        n_pairs, n_pix, n_hits, status = run.counts()
        assert status == 0
        outs.append((run.current(S.n, n_pix).cpu().numpy().copy(), run.hits.to_numpy(n_hits)))
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in outs[0][1]:
        assert np.array_equal(outs[0][1][k], outs[1][1][k])
    assert np.array_equal(outs[0][0], st.current_np())
    hs = st.hits_np()
    for k in hs:
        assert np.array_equal(hs[k], outs[0][1][k])


def test_event_hits_against_oracle_end_to_end(small):
    """Oracle current (FP64) into the oracle front end vs the GPU event."""
    st, o, seg, d = small["st"], small["o"], small["seg"], small["d"]
    m = st.maps_np()
    h = st.hits_np()
    band = BAND[0]
    n_hit_pix = n_tied = n_cmp = 0
    p_ties = []
    for i, p in enumerate(m["active"]):
        segs = m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]]
        I = o.pixel_current(seg, d, int(p), segs, event_id=5)
        ref = o.electronics(int(p), I, event_id=5, band=band)
        g = hits_of_pixel(h, int(p))
        if len(ref["t_cross"]) or len(g["t_cross"]):
            n_hit_pix += 1
            p_ties.append(ref["p_tie"])
        if ref["tie_tick"] >= 0:
            n_tied += 1
        ok, nc = compare_pixel_hits(g, ref, 976.5625)
        assert ok, (p, ref, g)
        n_cmp += nc
    assert n_cmp > 20
    assert n_tied <= tie_cap(p_ties)


def test_capacity_overflow_then_retry():
    cfg = params.small_config()
    seg = _event(cfg, 77, 40)
    lut_dev, _ = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, pair_cap=50, pix_cap=2000, hit_cap=5).all()
    n_pairs, n_pix, n_hits, status = st.count_values()
    assert status & sim.SIM_STATUS_PAIR_OVERFLOW and n_pairs > 50
    st2 = Steps(cfg, seg, lut_dev, pair_cap=n_pairs, pix_cap=10, hit_cap=5).all()
    _, n_pix2, _, status2 = st2.count_values()
    assert status2 & sim.SIM_STATUS_PIXEL_OVERFLOW and n_pix2 > 10
    st3 = Steps(cfg, seg, lut_dev, pair_cap=n_pairs, pix_cap=n_pix2, hit_cap=5).all()
    _, _, n_hits3, status3 = st3.count_values()
    assert status3 == (sim.SIM_STATUS_HIT_OVERFLOW if n_hits3 > 5 else 0)
    st4 = Steps(cfg, seg, lut_dev, pair_cap=n_pairs, pix_cap=n_pix2, hit_cap=max(n_hits3, 1)).all()
    assert st4.count_values()[3] == 0
    assert st4.count_values()[2] == n_hits3


def test_empty_and_all_inactive_events():
    cfg = params.small_config()
    lut_dev, _ = lut_pair(cfg)
    empty = {k: np.zeros(0, np.float32) for k in events.COLS}
    st = Steps(cfg, empty, lut_dev, pair_cap=16, pix_cap=16).all()
    assert st.count_values() == [0, 0, 0, 0]
    outside = _edge_segments(cfg)
    outside = {k: v[:2] for k, v in outside.items()}          # zero length + outside
    st = Steps(cfg, outside, lut_dev, pair_cap=16, pix_cap=16).all()
    assert st.count_values() == [0, 0, 0, 0]
