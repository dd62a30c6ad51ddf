"""The 35-module beam spill (~1.2e6 segments, 50 interactions + 100 rock
muons, t0 spread over 10 us) at full size through sim_event, FP32 direct and
FP16 tensor-core forms: sampled active pixels against the oracle (segment
list and current), and the two forms against each other on every pixel."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import serve, sim
from synth import events, params

from gpu_harness import lut_pair

pytestmark = pytest.mark.gpu

MAP_BAND, CUR_HARD = 1e-5, 1e-4


def _run(cfg, lut_dev, seg):
    n = len(seg["x0"])
    caps = serve._caps(n)
    while True:
        run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], n, *caps)
        run.enqueue(sim.Segments.from_numpy(seg, 3))
        torch.cuda.synchronize()
        c = run.counts()
        if c[3] == 0:
            return run, c
        caps = (max(caps[0], 2 * c[0]), max(caps[1], 2 * c[1]), max(caps[2], 2 * c[2]))
        del run
        torch.cuda.empty_cache()


def test_spill_sampled_pixels_both_forms():
    cfg = params.spill_config()
    seg = events.spill_event(cfg, params.BASE["seed"] + 2)
    n = len(seg["x0"])
    lut_dev, lut64 = lut_pair(cfg)
    run, (n_pairs, n_pix, n_hits, _) = _run(cfg, lut_dev, seg)
    assert n > 1_000_000 and n_pix > 100_000 and n_hits > 1000
    act = run.active_pixels(n, n_pix).cpu().numpy()
    off, ids = run.csr(n, n_pix, n_pairs)
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    cur0 = run.current(n, n_pix).cpu().numpy()
    del run
    torch.cuda.empty_cache()
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    for i in np.random.default_rng(5).choice(n_pix, 5, replace=False):
        p = int(act[i])
        segs, _ = o.segments_for_pixel(seg, d, p)
        for s in set(segs.tolist()) ^ set(ids[off[i]:off[i + 1]].tolist()):
            assert abs(o.pair_margin(seg, d, s, p)) < MAP_BAND
        ref = o.pixel_current(seg, d, p, ids[off[i]:off[i + 1]], event_id=3)
        err = np.abs(cur0[i] - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= CUR_HARD, (p, err)
    run2, (p2, n_pix2, h2, _) = _run(params.spill_config(precision=2), lut_dev, seg)
    assert n_pix2 == n_pix and p2 == n_pairs
    cur2 = run2.current(n, n_pix).cpu().numpy()
    sig = np.abs(cur0).sum(-1) >= 1.0
    d2 = cur2[sig] - cur0[sig]
    l2 = np.linalg.norm(d2, axis=-1) / np.linalg.norm(cur0[sig], axis=-1)
    ev = float(np.linalg.norm(cur2 - cur0) / np.linalg.norm(cur0))
    print(f"spill FP16 vs FP32: pixels {sig.sum()} l2 max {l2.max():.2e} med {np.median(l2):.2e} event {ev:.2e}")
    assert l2.max() <= 5e-4 and ev <= 2e-4
