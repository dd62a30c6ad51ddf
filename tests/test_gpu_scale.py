"""Parity at full size, in the benchmark's launch configuration (one sim_event
call per event): the one-module neutrino interaction (~2e4 segments) on EVERY
active pixel, and the 35-module beam spill (~1.2e6 segments) on 2000 random
active pixels plus every active pixel of its densest tile, for the FP32
and the FP16 tensor-core forms of the current, against the FP64 oracle's own
map, currents and front end (the oracle shares its many pixels among the host
cores; nothing it computes comes from the GPU).

Checks and tolerances:
  * map: the active-pixel sets of the whole event are equal and each sampled
    pixel's segment list is equal, except pairs whose distance margin is
    within MAP_BAND of the map radius (FP32 geometry);
  * currents, per pixel: FP32 ||I - I_ref||_inf <= 2e-5 ||I_ref||_inf (median
    <= 1e-6); every prefix sum of the current (the charge the front end has
    integrated by each tick) within 1e-5 of the pixel's largest one plus a
    floor of 2e-6 of the event's peak pixel charge.  The floor covers pixels
    whose charge comes through small interpolation weights from their
    brighter neighbours' points: their absolute error follows from the FP32
    rounding of those points' positions, which scales with the charge density
    of the event, not with the pixel's own charge.  FP16: the tensor-core
    tolerances (||.||_2 <= 5e-4, ||.||_inf <= 1e-3 of the pixel's, prefix
    sums within 2e-4 plus the same floor; the whole sample within 2e-4);
  * hits: pixel, crossing tick, ADC tick and code bit-exact on every pixel up
    to the oracle's first tie: a discriminator or ADC decision of the oracle's
    own trace within BAND electrons of its threshold.  The band is what each
    form's charge error at the decisions needs: FP32 0.2 e- (4e-5 of the
    threshold; measured mismatches at 0.05 e-), FP16 1 e- (the tensor cores'
    truncating FP32 accumulation leaves ~4e-5 of a dense pixel's charge;
    measured mismatches at 0.5 e-).  Which pixels a band cuts is decided by
    the oracle alone, so the cut cannot hide a GPU error; its size is bounded
    by the oracle's own expectation under the noise model (p_tie of each
    trace): tied pixels <= sum p_tie + 4 sqrt(sum p_tie (1 - p_tie)) + 2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import serve, sim
from synth import events, params, response

from gpu_harness import BAND, tie_cap

pytestmark = pytest.mark.gpu

MAP_BAND = 1e-5
FLOOR = 2e-6                                   # of the event's peak pixel charge


def _tiles(cfg, pix):
    npx = cfg["tiles_x"] * cfg["px_per_tile"] * cfg["tiles_y"] * cfg["px_per_tile"]
    nxp = cfg["tiles_x"] * cfg["px_per_tile"]
    an, rem = pix // npx, pix % npx
    iy, ix = rem // nxp, rem % nxp
    return (an * cfg["tiles_y"] + iy // cfg["px_per_tile"]) * cfg["tiles_x"] + ix // cfg["px_per_tile"]


@pytest.fixture(scope="module", params=["module", "spill"])
def ref(request):
    """The oracle's side of one workload: quench + drift, its map of every
    segment, the sampled pixels' currents and their front end at each band."""
    if request.param == "module":
        cfg = params.module_config()
        seg, eid = events.module_event(cfg, params.BASE["seed"] + 1), 1
    else:
        cfg = params.spill_config()
        seg, eid = events.spill_event(cfg, params.BASE["seed"] + 2), 3
    pad = response.pad_rows(response.lut_for(cfg, params.LUT))
    o = oracle.Oracle(cfg, params.LUT, pad[..., : params.LUT["nt"]].astype(np.float64))
    d = o.quench_drift(seg)
    m = o.map_event(seg, d)
    P = len(m["pixels"])
    if request.param == "module":
        idx = np.arange(P)                                          # every active pixel
    else:
        tl = _tiles(cfg, m["pixels"])
        u, c = np.unique(tl, return_counts=True)
        rnd = np.random.default_rng(7).choice(P, 2000, replace=False)
        idx = np.unique(np.concatenate([rnd, np.nonzero(tl == u[c.argmax()])[0]]))
    pix = m["pixels"][idx]
    lens = m["off"][idx + 1] - m["off"][idx]
    off = np.concatenate([[0], np.cumsum(lens)])
    segs = np.concatenate([m["segs"][m["off"][i]:m["off"][i + 1]] for i in idx])
    I = o.pixel_currents(seg, d, pix, off, segs, event_id=eid)
    hits = {b: o.electronics_many(pix, I, event_id=eid, band=b) for b in set(BAND.values())}
    return dict(name=request.param, cfg=cfg, seg=seg, eid=eid, lut=pad, o=o, d=d, m=m, pix=pix, off=off, segs=segs,
                I=I, hits=hits)


def _run(cfg, lut_dev, seg, eid):
    n = len(seg["x0"])
    caps = serve._caps(n)
    while True:
        run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], n, *caps)
        run.enqueue(sim.Segments.from_numpy(seg, eid))
        torch.cuda.synchronize()
        c = run.counts()
        if c[3] == 0:
            return run, c
        caps = (max(caps[0], 2 * c[0]), max(caps[1], 2 * c[1]), max(caps[2], 2 * c[2]))
        del run
        torch.cuda.empty_cache()


def _map_checks(r, act, goff, gids, pos):
    o, seg, d, m = r["o"], r["seg"], r["d"], r["m"]
    only_gpu = np.setdiff1d(act, m["pixels"])
    only_ora = np.setdiff1d(m["pixels"], act)
    for p in only_ora.tolist():                                   # every pair of it is a boundary case
        i = int(np.searchsorted(m["pixels"], p))
        assert np.all(m["margin"][m["off"][i]:m["off"][i + 1]] < MAP_BAND), p
    for p in only_gpu.tolist():
        i = int(np.searchsorted(act, p))
        for s in gids[goff[i]:goff[i + 1]].tolist():
            assert o.pair_margin(seg, d, s, p) > -MAP_BAND, (p, s)
    n_diff = 0
    for j, i in enumerate(pos.tolist()):
        g = gids[goff[i]:goff[i + 1]]
        e = r["segs"][r["off"][j]:r["off"][j + 1]]
        if len(g) == len(e) and np.array_equal(np.sort(g), e):
            continue
        for s in set(g.tolist()) ^ set(e.tolist()):
            assert abs(o.pair_margin(seg, d, s, int(act[i]))) < MAP_BAND, (int(act[i]), s)
            n_diff += 1
    return len(only_gpu) + len(only_ora), n_diff


def _current_checks(precision, I, R, label):
    q_ref = np.cumsum(R, axis=1)
    scale = np.abs(q_ref).max(axis=1)
    peak = scale.max()
    cum = np.abs(np.cumsum(I - R, axis=1)).max(axis=1)
    lim_q = (1e-5 if precision == 0 else 2e-4) * scale + FLOOR * peak
    bad = np.nonzero(cum > lim_q)[0]
    assert len(bad) == 0, (label, bad[:5], cum[bad[:5]], scale[bad[:5]])
    sig = scale >= 1.0
    d = I[sig] - R[sig]
    inf = np.abs(d).max(axis=1) / np.abs(R[sig]).max(axis=1)
    if precision == 0:
        assert inf.max() <= 2e-5, (label, inf.max())
        assert np.median(inf) <= 1e-6, (label, np.median(inf))
    else:
        l2 = np.linalg.norm(d, axis=1) / np.linalg.norm(R[sig], axis=1)
        assert l2.max() <= 5e-4 and inf.max() <= 1e-3, (label, l2.max(), inf.max())
        assert np.linalg.norm(I - R) <= 2e-4 * np.linalg.norm(R), label
    print(f"{label}: {len(I)} pixels, inf max {inf.max():.2e} med {np.median(inf):.2e}, "
          f"prefix-charge err max {np.max(cum / np.maximum(scale, 1e-300)):.2e} of the pixel's, "
          f"{cum.max() / peak:.2e} of the peak")


def _hit_checks(r, precision, gh, label):
    band = BAND[precision]
    refs = r["hits"][band]
    hp = gh["pixel"]
    n_hit_pix = n_tied = n_cmp = n_tot = 0
    p_ties = []
    for j, p in enumerate(r["pix"].tolist()):
        e = refs[j]
        lo, hi = np.searchsorted(hp, p), np.searchsorted(hp, p, side="right")
        if len(e["t_cross"]) == 0 and hi == lo:
            continue
        n_hit_pix += 1
        p_ties.append(e["p_tie"])
        tie = e["tie_tick"]
        lim = tie if tie >= 0 else 1 << 30
        n_tied += tie >= 0
        rm = (e["t_adc"] < lim) & (e["t_cross"] < lim)
        g = {k: v[lo:hi] for k, v in gh.items()}
        gm = (g["t_adc"] < lim) & (g["t_cross"] < lim)
        same = (rm.sum() == gm.sum() and np.array_equal(e["t_cross"][rm], g["t_cross"][gm])
                and np.array_equal(e["t_adc"][rm], g["t_adc"][gm])
                and np.array_equal(e["adc"][rm], g["adc"][gm].astype(np.int64)))
        assert same, (label, p, e, g)
        n_cmp += int(rm.sum())
        n_tot += len(e["t_cross"])
    cap = tie_cap(p_ties)
    print(f"{label}: band {band} e-: {n_hit_pix} hit pixels, {n_tied} tied ({n_tied / max(n_hit_pix, 1):.2%}; "
          f"expected {sum(p_ties):.1f}, cap {cap:.1f}), hits compared {n_cmp} of {n_tot}")
    assert n_hit_pix > 1000 and n_cmp > 0.8 * n_tot
    assert n_tied <= cap, (label, n_tied, cap)


@pytest.mark.parametrize("precision", [0, 2])
def test_full_size_event_against_oracle(ref, precision):
    r = ref
    cfg = dict(r["cfg"], precision=precision)
    lut_dev = torch.as_tensor(r["lut"], device="cuda")
    seg, n = r["seg"], len(r["seg"]["x0"])
    run, (n_pairs, n_pix, n_hits, _) = _run(cfg, lut_dev, seg, r["eid"])
    label = f"{r['name']} precision {precision}"
    act = run.active_pixels(n, n_pix).cpu().numpy()
    goff, gids = (t.cpu().numpy() for t in run.csr(n, n_pix, n_pairs))
    pos = np.searchsorted(act, r["pix"])
    assert np.all(pos < n_pix) and np.array_equal(act[pos], r["pix"]), "sampled pixel not active on the GPU"
    n_set, n_list = _map_checks(r, act, goff, gids, pos)
    print(f"{label}: {n} segments, {n_pix} active pixels, map differences {n_set} pixels / {n_list} pairs")
    I = run.current(n, n_pix)[torch.as_tensor(pos, device="cuda")].cpu().numpy().astype(np.float64)
    _current_checks(precision, I, r["I"], label)
    gh = run.hits.to_numpy(min(n_hits, run.hits.capacity))
    assert n_hits <= run.hits.capacity
    _hit_checks(r, precision, gh, label)
    del run
    torch.cuda.empty_cache()


def test_fp32_form_in_short_record_chunks(ref):
    """The FP32 form with chunks of 4096 records (tc_record_chunk): the module
    event's dense pixels then take several chunks each (a pixel's records are
    generated, binned and applied chunk by chunk, the generation resuming
    where the full chunk stopped); every pixel against the same oracle, with
    the same tolerances."""
    if ref["name"] != "module":
        pytest.skip("module event only")
    r = ref
    cfg = dict(r["cfg"], precision=0, tc_record_chunk=4096)
    lut_dev = torch.as_tensor(r["lut"], device="cuda")
    seg, n = r["seg"], len(r["seg"]["x0"])
    run, (n_pairs, n_pix, n_hits, _) = _run(cfg, lut_dev, seg, r["eid"])
    act = run.active_pixels(n, n_pix).cpu().numpy()
    pos = np.searchsorted(act, r["pix"])
    assert np.all(pos < n_pix) and np.array_equal(act[pos], r["pix"])
    # candidate points of the densest pixels: several times a chunk (about half become records)
    ns = r["d"]["n_samples"].astype(np.int64) * int(cfg["mc_per_sample"])
    cand = np.array([ns[r["segs"][r["off"][j]:r["off"][j + 1]]].sum() for j in range(len(r["pix"]))])
    assert (cand > 4 * 4096).sum() > 100, cand.max()
    I = run.current(n, n_pix)[torch.as_tensor(pos, device="cuda")].cpu().numpy().astype(np.float64)
    _current_checks(0, I, r["I"], "module precision 0, 4096-record chunks")
    gh = run.hits.to_numpy(min(n_hits, run.hits.capacity))
    _hit_checks(r, 0, gh, "module precision 0, 4096-record chunks")
    del run
    torch.cuda.empty_cache()
