"""GPU parity of the tensor-core form of the induced-current step
(sim_config.precision 1 = BF16, 2 = FP16 operands, FP32 accumulation in
tensor memory) against the FP64 oracle, called through the C ABI.

The tensor-core form sums exactly the terms of the FP32 form; it
differs by the rounding of the charge tiles and of the table to the operand
type (relative 2^-11 for FP16, 2^-8 for BF16, per operand) and by the
fixed-point accumulation of the charge tiles (2^-12 e-).  Tolerances:
  * every pixel whose reference integrated |current| is at least 1 e- (pixels
    below carry nothing a discriminator at thousands of electrons can see):
      FP16: ||I - I_ref||_2 <= 5e-4 ||I_ref||_2, ||.||_inf <= 1e-3 ||I_ref||_inf,
            integrated charge within 5e-4;
      BF16: 1e-2, 3e-2 and 1e-2;
  * the whole event, all pixels: ||I - I_ref||_F <= 2e-4 ||I_ref||_F (FP16),
    1e-2 (BF16), and max |I - I_ref| <= the same fraction of max |I_ref|.
(Measured: FP16 ~1.6e-4 worst pixel, ~2e-5 event-wide, on the module event;
the tensor cores' FP32 accumulation truncates, which the kernel bounds by
adding its accumulators into the output every 64 table nodes.)
The results of a call are bitwise reproducible (integer tile accumulation,
fixed MMA order per pixel group).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import sim
from synth import events, params

from gpu_harness import Steps, lut_pair

pytestmark = pytest.mark.gpu

TOL = {2: dict(l2=5e-4, inf=1e-3, q=5e-4, event=2e-4), 1: dict(l2=1e-2, inf=3e-2, q=1e-2, event=1e-2)}
Q_MIN = 1.0          # e-: pixels with less integrated |current| are not compared one by one


def _norm_errors(I, ref):
    """Per-pixel relative errors over significant pixels and the event-level ones."""
    d = I - ref
    sig = np.abs(ref).sum(axis=-1) >= Q_MIN
    l2 = np.linalg.norm(d[sig], axis=-1) / np.linalg.norm(ref[sig], axis=-1)
    inf = np.abs(d[sig]).max(axis=-1) / np.abs(ref[sig]).max(axis=-1)
    q = np.abs(d[sig].sum(-1)) / np.abs(ref[sig]).sum(-1)
    ev = dict(fro=float(np.linalg.norm(d) / np.linalg.norm(ref)), max=float(np.abs(d).max() / np.abs(ref).max()))
    return l2, inf, q, ev


def _check(errs, t, label, charge=True):
    l2, inf, q, ev = errs
    print(f"{label}: pixels {len(l2)} l2 max {l2.max():.2e} med {np.median(l2):.2e} inf max {inf.max():.2e} "
          f"q max {q.max():.2e} event fro {ev['fro']:.2e} max {ev['max']:.2e}")
    assert len(l2) > 0
    assert l2.max() <= t["l2"] and inf.max() <= t["inf"]
    if charge:
        assert q.max() <= t["q"]
    assert ev["fro"] <= t["event"] and ev["max"] <= t["event"]


def _tc_vs_oracle(cfg, seg, lut_par=None, event_id=0, frac=1.0, **lut_kw):
    lut_par = lut_par or params.LUT
    lut_dev, lut64 = lut_pair(cfg, lut_par, **lut_kw)
    st = Steps(cfg, seg, lut_dev, event_id=event_id, lut_par=lut_par).quench_drift().pixel_map().induced_current()
    m = st.maps_np()
    cur = st.current_np()
    o = oracle.Oracle(cfg, lut_par, lut64)
    d = o.quench_drift(seg)
    idx = np.arange(len(m["active"]))
    if frac < 1.0:
        idx = np.random.default_rng(0).choice(idx, max(8, int(frac * len(idx))), replace=False)
    ref = np.array([o.pixel_current(seg, d, int(m["active"][i]), m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]],
                                    event_id=event_id) for i in idx])
    return _norm_errors(cur[idx], ref), st


def _event(cfg, seed, n, t_range=(0.0, 0.0)):
    return events.scatter_event(cfg, seed, n, max_len=0.6, t_range=t_range)


@pytest.mark.parametrize("precision", [2, 1])
def test_tensor_core_all_pixels(precision):
    cfg = params.small_config(precision=precision)
    errs, st = _tc_vs_oracle(cfg, _event(cfg, 101, 60), event_id=5)
    assert len(errs[0]) > 200
    _check(errs, TOL[precision], f"precision {precision}")


@pytest.mark.parametrize("case", ["M4", "two_passes_ragged", "bipolar", "box_shifted"])
def test_tensor_core_variants(case):
    over, lut_kw, tr = {}, {}, (0.0, 0.0)
    if case == "M4":
        over = dict(mc_per_sample=4)
    elif case == "two_passes_ragged":
        over = dict(n_ticks=2500, t_window0_us=-37.3)        # two tick passes, ragged tail
    elif case == "bipolar":
        lut_kw = dict(bipolar=0.5)
    elif case == "box_shifted":
        over = dict(recomb_model=1, t_window0_us=3.05)
        tr = (0.0, 9.0)
    cfg = params.small_config(precision=2, **over)
    errs, _ = _tc_vs_oracle(cfg, _event(cfg, 300 + len(case), 25, tr), event_id=11, **lut_kw)
    _check(errs, TOL[2], case, charge=(case != "bipolar"))     # bipolar pixels can integrate to ~0


def _module_run(precision, seg, lut_dev):
    cfg = params.module_config(precision=precision)
    n = len(seg["x0"])
    run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], n, 40 * n, 4 * n, 4 * n)
    run.enqueue(sim.Segments.from_numpy(seg, 1))
    torch.cuda.synchronize()
    n_pairs, n_pix, n_hits, status = run.counts()
    assert status == 0
    return run, n, n_pix


def test_tensor_core_module_event_against_direct_and_oracle():
    """The ~20k-segment module event at full size (several record chunks per
    pixel group): every pixel against the FP32 form, sampled pixels
    against the oracle, and bitwise reproducibility of the call."""
    cfg = params.module_config()
    seg = events.module_event(cfg, seed=params.BASE["seed"] + 1)
    lut_dev, lut64 = lut_pair(cfg)
    run0, n, n_pix = _module_run(0, seg, lut_dev)
    direct = run0.current(n, n_pix).cpu().numpy()
    act = run0.active_pixels(n, n_pix).cpu().numpy()
    del run0
    run2, _, n_pix2 = _module_run(2, seg, lut_dev)
    assert n_pix2 == n_pix
    tc = run2.current(n, n_pix).cpu().numpy().copy()
    errs = _norm_errors(tc, direct)
    sig = np.abs(direct).sum(-1) >= Q_MIN
    for w in np.argsort(errs[0])[-3:]:
        r = direct[sig][w]
        print(f"  worst module pixel: l2 {errs[0][w]:.2e} inf {errs[1][w]:.2e} peak {np.abs(r).max():.3e} "
              f"sum {r.sum():.3e}")
    _check(errs, TOL[2], "module FP16 vs direct")
    # oracle on sampled pixels
    off, ids = run2.csr(n, n_pix, run2.counts()[0])
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    for i in np.random.default_rng(3).choice(n_pix, 6, replace=False):
        ref = o.pixel_current(seg, d, int(act[i]), ids[off[i]:off[i + 1]], event_id=1)
        if np.abs(ref).sum() < Q_MIN:
            continue
        l2, inf, _, _ = _norm_errors(tc[i][None], ref[None])
        assert l2[0] <= TOL[2]["l2"] and inf[0] <= TOL[2]["inf"], (i, l2, inf)
    # the same call again: bitwise identical
    run2.enqueue(sim.Segments.from_numpy(seg, 1))
    torch.cuda.synchronize()
    assert np.array_equal(run2.current(n, n_pix).cpu().numpy(), tc)


def test_tensor_core_event_hits_against_oracle():
    """Hits of the whole path with the FP16 tensor-core current against the
    oracle (FP64 current, FP64 front end): bit-exact pixel, crossing tick, ADC
    tick and code up to the oracle's first decision within the FP16 band
    (gpu_harness.BAND: 1 e-, the CSA charge error the FP16 form leaves at its
    decisions); the tied pixels, chosen by the oracle's trace alone, number at
    most what its tie probabilities predict (gpu_harness.tie_cap)."""
    from gpu_harness import BAND, compare_pixel_hits, hits_of_pixel, tie_cap
    cfg = params.small_config(precision=2)
    seg = _event(cfg, 101, 60)
    lut_dev, lut64 = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=5).all()
    m = st.maps_np()
    h = st.hits_np()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    band = BAND[2]
    n_hit_pix = n_tied = n_cmp = 0
    p_ties = []
    for i, p in enumerate(m["active"]):
        I = o.pixel_current(seg, d, int(p), m["pix_ids"][m["pix_off"][i]:m["pix_off"][i + 1]], event_id=5)
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
    print(f"hits compared {n_cmp}, hit pixels {n_hit_pix}, tied {n_tied}, expected {sum(p_ties):.2f}")
    assert n_cmp > 20
    assert n_tied <= tie_cap(p_ties)
