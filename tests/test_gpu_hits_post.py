"""GPU parity of the steps after the front end, through the C ABI: per-hit
charge truth (sim_hit_truth), hits -> 3-D points (sim_hit_points) and dQ/dx
along a known track (sim_track_dqdx), against the FP64 oracle.

Tolerances:
  * truth: each listed segment's charge within 2e-5 of the hit's summed
    |charge| plus 1e-2 e- (FP32 sums of the same terms as the FP32 current,
    through FP32 running sums of the table rows, ~1e-6 relative); the signal
    charge likewise; every segment whose oracle |charge| exceeds the GPU's
    smallest listed one by more than that tolerance is listed;
  * points: bit-exact (FP64 arithmetic on both sides in the same order,
    rounded to FP32);
  * dQ/dx: piece counts exact, piece charges within 2^-17 e- per point (the
    fixed-point rounding).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import sim
from synth import events, params

from gpu_harness import Steps, lut_pair

pytestmark = pytest.mark.gpu

K = 5


def _truth_run(st, k=K, max_cells=64):
    cum = sim.sim_response_cumulative(st.resp)
    tr = sim.Truth(st.hit_cap, k, max_cells=max_cells)      # small: the first call overflows and is retried
    sim.sim_hit_truth(st.cfg, st.seg, st.dr, st.resp, cum, st.active, st.pix_seg_off, st.pix_seg_ids, st.counts,
                      st.pix_cap, st.hits, tr)
    torch.cuda.synchronize()
    cells, runs, units, status = tr.counts()
    assert status == 0 and runs > 0 and units >= runs and cells > 64
    return tr


def _check_truth(o, seg, d, m, h, tr, n_hits, event_id, max_pixels=None, rng=None):
    segs_g = tr.segment[: n_hits * tr.k].cpu().numpy().reshape(n_hits, tr.k)
    q_g = tr.q[: n_hits * tr.k].cpu().numpy().reshape(n_hits, tr.k)
    sig_g = tr.q_signal[:n_hits].cpu().numpy()
    k0_g = tr.tick_first[:n_hits].cpu().numpy()
    pix = np.unique(h["pixel"])
    if max_pixels is not None and len(pix) > max_pixels:
        pix = rng.choice(pix, max_pixels, replace=False)
    n_cmp = 0
    for p in pix.tolist():
        hi = np.nonzero(h["pixel"] == p)[0]
        i = int(np.searchsorted(m["active"], p))
        segs = m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]]
        Q, qs, k0, _ = o.hit_truth(seg, d, p, segs, h["t_cross"][hi], h["t_adc"][hi], event_id=event_id)
        for r, hh in enumerate(hi.tolist()):
            tol = 2e-5 * np.abs(Q[r]).sum() + 1e-2
            assert k0_g[hh] == k0[r]
            assert abs(sig_g[hh] - qs[r]) <= tol, (p, hh, sig_g[hh], qs[r])
            ref = dict(zip(segs.tolist(), Q[r].tolist()))
            listed = [s for s in segs_g[hh].tolist() if s >= 0]
            assert len(listed) >= min(tr.k, int((np.abs(Q[r]) > tol).sum()))
            for s, v in zip(listed, q_g[hh][: len(listed)].tolist()):
                assert abs(v - ref[s]) <= tol, (p, hh, s, v, ref[s])
            floor = abs(q_g[hh][len(listed) - 1]) if len(listed) == tr.k else 0.0
            for s, v in ref.items():
                if abs(v) > floor + tol and v != 0.0:
                    assert s in listed, (p, hh, s, v, listed)
            n_cmp += 1
    return n_cmp


@pytest.mark.parametrize("case", ["plain", "periodic", "M2", "nearest", "per_point"])
def test_hit_truth_against_oracle(case):
    over = dict(thr_e=3000.0)
    if case == "periodic":
        over["periodic_reset_ticks"] = 150
    elif case == "M2":
        over["mc_per_sample"] = 2
    elif case == "nearest":
        over["nearest_lut"] = 1
    elif case == "per_point":
        over["per_point_drift"] = 1
    cfg = params.small_config(**over)
    seg = events.scatter_event(cfg, 404, 40, max_len=0.6)
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=9).all()
    m, h = st.maps_np(), st.hits_np()
    n_hits = len(h["pixel"])
    assert n_hits > 10
    tr = _truth_run(st)
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    n = _check_truth(o, seg, d, m, h, tr, n_hits, 9)
    assert n == n_hits
    t = tr.to_numpy(n_hits)                      # fractions of the listed segments in each hit's signal
    ok = np.abs(t["q_signal"]) > 1.0
    assert np.allclose(t["fraction"][ok] * t["q_signal"][ok, None], t["q"][ok], rtol=1e-6, atol=1e-6)
    if case != "bipolar":
        assert np.all(t["fraction"][ok].sum(axis=1) <= 1.0 + 1e-5)


def test_hit_truth_module_event_sampled_and_signal_sums():
    """The module event at full size: sampled hit pixels against the oracle;
    every hit's signal equals its interval sum of the FP32 current."""
    cfg = params.module_config()
    seg = events.module_event(cfg, seed=params.BASE["seed"] + 1)
    lut_dev, lut64 = lut_pair(cfg)
    n = len(seg["x0"])
    st = Steps(cfg, seg, lut_dev, event_id=1, pair_cap=40 * n, pix_cap=4 * n, hit_cap=4 * n).all()
    m, h = st.maps_np(), st.hits_np()
    n_hits = len(h["pixel"])
    tr = _truth_run(st, k=8)
    cur = st.current_np()
    sig = tr.q_signal[:n_hits].cpu().numpy()
    k0 = tr.tick_first[:n_hits].cpu().numpy()
    idx = np.searchsorted(m["active"], h["pixel"])
    cs = np.concatenate([np.zeros((len(cur), 1)), np.cumsum(cur.astype(np.float64), axis=1)], axis=1)
    want = cs[idx, h["t_adc"] + 1] - cs[idx, k0]
    scale = np.abs(cur[idx]).sum(axis=1)
    rel = np.abs(sig - want) / np.maximum(scale, 1.0)
    print(f"signal vs current interval sums: max rel {rel.max():.2e}, median {np.median(rel):.2e}")
    # both are FP32 sums of the same terms in different orders; the FP32 current is good to 1e-4 per pixel
    assert np.all(np.abs(sig - want) <= 1e-4 * scale + 1e-2)
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    n_cmp = _check_truth(o, seg, d, m, h, tr, n_hits, 1, max_pixels=6, rng=np.random.default_rng(4))
    assert n_cmp >= 6


def test_hit_points_bit_exact():
    cfg = params.module_config(t_window0_us=-3.3)
    cfg["n_tpc"] = 2
    seg = events.module_event(cfg, seed=params.BASE["seed"] + 1)
    lut_dev, _ = lut_pair(cfg)
    n = len(seg["x0"])
    st = Steps(cfg, seg, lut_dev, event_id=1, pair_cap=40 * n, pix_cap=4 * n, hit_cap=4 * n).all()
    h = st.hits_np()
    nh = len(h["pixel"])
    assert nh > 1000
    dev = torch.device("cuda:0")
    x, y, z = (torch.empty(st.hit_cap, dtype=torch.float32, device=dev) for _ in range(3))
    t_ev = torch.tensor([0.7], dtype=torch.float32, device=dev)
    sim.sim_hit_points(st.cfg, st.hits, x, y, z, t_event=t_ev)
    torch.cuda.synchronize()
    o = oracle.Oracle(cfg, params.LUT)
    ref = o.hit_points(h["pixel"], h["t_cross"], t_event=float(np.float32(0.7))).astype(np.float32)
    got = np.stack([x[:nh].cpu().numpy(), y[:nh].cpu().numpy(), z[:nh].cpu().numpy()], axis=1)
    assert np.array_equal(got, ref)
    assert set(np.unique((h["pixel"] // (70 * 70 * 20)) % 2).tolist()) == {0, 1}      # both TPCs present


def test_track_dqdx_on_the_tile_muon():
    """dQ/dx of the configuration-1 muon's hits along its generating line, in
    1 cm pieces: counts exact, charges to the fixed-point rounding."""
    cfg = params.tile_config(thr_e=3000.0)
    seg = events.tile_muon(cfg, params.BASE["seed"])
    lut_dev, _ = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=0).all()
    h = st.hits_np()
    nh = len(h["pixel"])
    assert nh > 20
    dev = torch.device("cuda:0")
    x, y, z = (torch.empty(st.hit_cap, dtype=torch.float32, device=dev) for _ in range(3))
    sim.sim_hit_points(st.cfg, st.hits, x, y, z)
    a = np.array([seg["x0"][0], seg["y0"][0], seg["z0"][0]], np.float64)
    b = np.array([seg["x1"][-1], seg["y1"][-1], seg["z1"][-1]], np.float64)
    u = (b - a) / np.linalg.norm(b - a)
    n_pieces = int(np.ceil(np.linalg.norm(b - a))) + 1
    dq = torch.empty(n_pieces, dtype=torch.float64, device=dev)
    cnt = torch.empty(n_pieces, dtype=torch.int32, device=dev)
    sim.sim_track_dqdx(x, y, z, st.hits.q, st.hits.n_out, a, u, 1.0, n_pieces, 1.0, dq, cnt)
    torch.cuda.synchronize()
    P = np.stack([x[:nh].cpu().numpy(), y[:nh].cpu().numpy(), z[:nh].cpu().numpy()], axis=1).astype(np.float64)
    ref_dq, ref_cnt, _ = oracle.Oracle.track_dqdx(P, h["q"].astype(np.float64), a, u, 1.0, n_pieces, 1.0)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert np.all(np.abs(dq.cpu().numpy() - ref_dq) <= ref_cnt * 2.0 ** -17 + 1e-9)
    d = np.linalg.norm(np.cross(P - a, u), axis=1)
    print(f"hits {nh}, within 1 cm of the line {ref_cnt.sum()}, median distance {np.median(d):.3f} cm")
    assert ref_cnt.sum() > 0.3 * nh


def test_hit_truth_and_points_of_a_batch_equal_the_events_alone():
    """Truth and 3-D points of a batch of events: each event's hits carry the
    truth of the event alone (segment indices offset by the event's first
    segment) and the same points (its own event time)."""
    cfg = params.small_config(thr_e=3000.0)
    lut_dev, _ = lut_pair(cfg)
    evs = [events.scatter_event(cfg, 70 + i, n, max_len=0.6) for i, n in enumerate((30, 0, 45))]
    ids = [4, 9, 13]
    det_px = params.geometry(cfg)["n_pixels"]
    dev = torch.device("cuda:0")

    def truth_and_points(seg, max_events, t_ev):
        n = max(seg.n, 1)
        run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], n, 64 * n, 40 * n,
                              200000, max_events=max_events)
        run.enqueue(seg)
        torch.cuda.synchronize()
        c = run.counts()
        assert c[3] == 0
        v = run.view(seg.n)
        A = sim._alias
        tr = sim.Truth(run.hits.capacity, 4, device=dev)
        sim.sim_hit_truth(run.cfg, seg, sim.Drifted.wrap(v.dr), run.resp, sim.sim_response_cumulative(run.resp),
                          A(v.active_pixels, run.max_pixels, torch.int32, dev),
                          A(v.pix_seg_off, run.max_pixels + 1, torch.int32, dev),
                          A(v.pix_seg_ids, run.max_pairs, torch.int32, dev), run.ws[:6], run.max_pixels, run.hits, tr)
        x, y, z = (torch.empty(run.hits.capacity, dtype=torch.float32, device=dev) for _ in range(3))
        sim.sim_hit_points(run.cfg, run.hits, x, y, z, t_event=t_ev)
        torch.cuda.synchronize()
        nh = c[2]
        h = run.hits.to_numpy(nh)
        return (h, tr.segment[: nh * 4].cpu().numpy().reshape(nh, 4), tr.q[: nh * 4].cpu().numpy().reshape(nh, 4),
                tr.q_signal[:nh].cpu().numpy(), np.stack([x[:nh].cpu().numpy(), y[:nh].cpu().numpy(),
                                                          z[:nh].cpu().numpy()], 1))

    t0s = [0.25, 0.0, 1.5]
    batch = sim.Segments.batch_from_numpy(evs, ids)
    hb, sb, qb, sigb, pb = truth_and_points(batch, len(evs), torch.tensor(t0s, dtype=torch.float32, device=dev))
    first = np.concatenate([[0], np.cumsum([len(e["x0"]) for e in evs])])
    n_cmp = 0
    for e, (ev, i) in enumerate(zip(evs, ids)):
        if len(ev["x0"]) == 0:
            continue
        ha, sa, qa, siga, pa = truth_and_points(sim.Segments.from_numpy(ev, i), 0,
                                                torch.tensor([t0s[e]], dtype=torch.float32, device=dev))
        m = hb["pixel"] // det_px == e
        assert np.array_equal(hb["pixel"][m] - e * det_px, ha["pixel"])
        assert np.array_equal(sb[m], np.where(sa >= 0, sa + first[e], -1))
        assert np.array_equal(qb[m], qa) and np.array_equal(sigb[m], siga)
        assert np.array_equal(pb[m], pa)
        n_cmp += int(m.sum())
    assert n_cmp > 5
