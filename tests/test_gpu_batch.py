"""Batched events: several events in one call give, for every event, exactly
the currents and hits the event gives alone (random numbers are keyed by the
event id and the event-local segment index; pixel ids of a batch are virtual:
slot * detector_pixels + pixel id)."""
import numpy as np
import pytest
import torch

from paper_2212_09807_gb300 import sim
from synth import events, params

from gpu_harness import lut_pair

pytestmark = pytest.mark.gpu


def _run(cfg, lut_dev, segs, n_seg, max_events=0):
    run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], n_seg, 64 * n_seg,
                          40 * n_seg, 200000, max_events=max_events)
    run.enqueue(segs)
    torch.cuda.synchronize()
    n_pairs, n_pix, n_hits, status = run.counts()
    assert status == 0
    return (run.active_pixels(segs.n, n_pix).cpu().numpy().copy(), run.current(segs.n, n_pix).cpu().numpy().copy(),
            run.hits.to_numpy(n_hits))


def test_batch_equals_events_alone():
    cfg = params.small_config()
    lut_dev, _ = lut_pair(cfg)
    evs = [events.scatter_event(cfg, 40 + i, n, max_len=0.7) for i, n in enumerate((30, 1, 55, 0, 12))]
    ids = [11, 7, (1 << 40) + 3, 5, 99]
    det_px = params.geometry(cfg)["n_pixels"]
    alone = [_run(cfg, lut_dev, sim.Segments.from_numpy(e, i), max(1, len(e["x0"])))
             for e, i in zip(evs, ids)]
    batch = sim.Segments.batch_from_numpy(evs, ids)
    act, cur, hits = _run(cfg, lut_dev, batch, batch.n, max_events=len(evs))
    slot = act // det_px
    for e, (a1, c1, h1) in enumerate(alone):
        m = slot == e
        assert np.array_equal(act[m] - e * det_px, a1)
        assert np.array_equal(cur[m], c1)                      # bitwise
        hm = hits["pixel"] // det_px == e
        assert np.array_equal(hits["pixel"][hm] - e * det_px, h1["pixel"])
        for k in ("t_cross", "t_adc", "adc", "q"):
            assert np.array_equal(hits[k][hm], h1[k]), k
    assert len(act) == sum(len(a) for a, _, _ in alone)


def test_batch_rejects_inconsistent_arguments():
    cfg = params.small_config()
    lut_dev, _ = lut_pair(cfg)
    e = events.scatter_event(cfg, 1, 5)
    segs = sim.Segments.from_numpy(e, 1)
    segs.n_events = 2                     # event arrays missing
    run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], 8, 512, 256, 1000,
                          max_events=2)
    with pytest.raises(sim.SimError) as err:
        run.enqueue(segs)
    assert err.value.code == -1


def test_batch_tensor_core_form_matches_events_alone():
    """The FP16 tensor-core form in a batch: same active pixels; currents equal
    to the event alone up to the accumulation rounding (pixel groups, hence
    the 64-node accumulation windows, differ between the two runs)."""
    cfg = params.small_config(precision=2)
    lut_dev, _ = lut_pair(cfg)
    evs = [events.scatter_event(cfg, 60 + i, n, max_len=0.7) for i, n in enumerate((40, 3, 25))]
    ids = [21, 8, 77]
    det_px = params.geometry(cfg)["n_pixels"]
    alone = [_run(cfg, lut_dev, sim.Segments.from_numpy(e, i), max(1, len(e["x0"]))) for e, i in zip(evs, ids)]
    batch = sim.Segments.batch_from_numpy(evs, ids)
    act, cur, _ = _run(cfg, lut_dev, batch, batch.n, max_events=len(evs))
    slot = act // det_px
    worst = 0.0
    for e, (a1, c1, _) in enumerate(alone):
        m = slot == e
        assert np.array_equal(act[m] - e * det_px, a1)
        scale = np.maximum(np.abs(c1).max(axis=1, keepdims=True), 1e-30)
        worst = max(worst, float((np.abs(cur[m] - c1) / scale).max()))
    assert worst <= 1e-5, worst
