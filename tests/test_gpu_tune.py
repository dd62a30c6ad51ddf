"""The scheduling shapes picked by the autotuner change the speed, not the
results: the FP32 form is bitwise the same for every number of CTAs per SM,
the tensor-core form agrees across work-plan targets and record chunks to its
accumulation rounding; the autotuner returns one of its candidates."""
import numpy as np
import pytest
import torch

from paper_2212_09807_gb300 import sim, tune
from synth import events, params

from gpu_harness import lut_pair

pytestmark = pytest.mark.gpu


def _currents(cfg, lut_dev, seg, n):
    run = sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], n, 64 * n, 40 * n, 200000)
    S = sim.Segments.from_numpy(seg, 3)
    run.enqueue(S)
    torch.cuda.synchronize()
    c = run.counts()
    assert c[3] == 0
    return run.current(n, c[1]).cpu().numpy().copy(), run.hits.to_numpy(c[2])


def test_direct_form_is_bitwise_independent_of_ctas_per_sm():
    cfg = params.small_config(precision=0)
    lut_dev, _ = lut_pair(cfg)
    seg = events.scatter_event(cfg, 31, 50, max_len=0.7)
    n = len(seg["x0"])
    ref, href = _currents(cfg, lut_dev, seg, n)
    for k in (1, 2):
        cur, h = _currents(dict(cfg, direct_ctas_per_sm=k), lut_dev, seg, n)
        assert np.array_equal(cur, ref)
        assert all(np.array_equal(h[x], href[x]) for x in h)


def test_tensor_core_form_across_shapes():
    cfg = params.small_config(precision=2)
    lut_dev, _ = lut_pair(cfg)
    seg = events.scatter_event(cfg, 32, 60, max_len=0.7)
    n = len(seg["x0"])
    ref, _ = _currents(cfg, lut_dev, seg, n)
    scale = np.abs(ref).max()
    for u, r in ((1, 1 << 12), (8, 1 << 16), (16, 1 << 18), (2, 1 << 20)):
        cur, _ = _currents(dict(cfg, tc_units_per_sm=u, tc_record_chunk=r), lut_dev, seg, n)
        assert np.abs(cur - ref).max() <= 1e-6 * scale, (u, r)


def test_autotune_returns_a_candidate():
    cfg = params.small_config(precision=2)
    lut_dev, _ = lut_pair(cfg)
    seg = events.scatter_event(cfg, 33, 40, max_len=0.7)
    n = len(seg["x0"])
    S = sim.Segments.from_numpy(seg, 3)
    chosen, table = tune.autotune(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], S,
                                  (64 * n, 40 * n, 200000), reps=1)
    assert chosen in tune.candidates(2) and len(table) == len(tune.candidates(2))
    assert all(ms > 0 for _, ms in table)
