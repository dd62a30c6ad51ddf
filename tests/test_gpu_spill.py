"""The 35-module beam spill (~1.2e6 segments, 50 interactions + 100 rock
muons, t0 spread over 10 us) at full size through sim_event: the FP16
tensor-core form against the FP32 form on every active pixel (the
oracle comparison of both forms, on a sample, is tests/test_gpu_scale.py)."""
import numpy as np
import pytest
import torch

from paper_2212_09807_gb300 import serve, sim
from synth import events, params

from gpu_harness import lut_pair

pytestmark = pytest.mark.gpu


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
    lut_dev, _ = lut_pair(cfg)
    run, (n_pairs, n_pix, n_hits, _) = _run(cfg, lut_dev, seg)
    assert n > 1_000_000 and n_pix > 100_000 and n_hits > 1000
    cur0 = run.current(n, n_pix).cpu().numpy()
    del run
    torch.cuda.empty_cache()
    run2, (p2, n_pix2, h2, _) = _run(params.spill_config(precision=2), lut_dev, seg)
    assert n_pix2 == n_pix and p2 == n_pairs
    cur2 = run2.current(n, n_pix).cpu().numpy()
    sig = np.abs(cur0).sum(-1) >= 1.0
    d2 = cur2[sig] - cur0[sig]
    l2 = np.linalg.norm(d2, axis=-1) / np.linalg.norm(cur0[sig], axis=-1)
    ev = float(np.linalg.norm(cur2 - cur0) / np.linalg.norm(cur0))
    print(f"spill FP16 vs FP32: pixels {sig.sum()} l2 max {l2.max():.2e} med {np.median(l2):.2e} event {ev:.2e}")
    assert l2.max() <= 5e-4 and ev <= 2e-4
