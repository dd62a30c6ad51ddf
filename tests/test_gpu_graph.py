"""The event step captured once in a CUDA graph (sim.GraphRunner) and
replayed for events of other sizes and ids gives bitwise the hits of direct
sim_event calls (the padding segments are inactive and the real segments'
random numbers are keyed by their own indices)."""
import numpy as np
import pytest
import torch

from paper_2212_09807_gb300 import sim
from synth import events, params

from gpu_harness import lut_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 2])
def test_graph_replay_matches_direct_calls(precision):
    cfg = params.small_config(precision=precision)
    lut_dev, _ = lut_pair(cfg)
    evs = [events.scatter_event(cfg, 900 + i, n, max_len=0.6) for i, n in enumerate((40, 15, 60))]
    cap = max(len(e["x0"]) for e in evs) + 7
    mk = lambda: sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], cap,   # noqa: E731
                                 64 * cap, 40 * cap, 200000)
    direct, graphed = mk(), mk()
    g = sim.GraphRunner(graphed)
    for i, e in enumerate(evs):
        eid = 77 + 3 * i
        seg = sim.Segments.from_numpy(e, eid)
        direct.enqueue(seg)
        torch.cuda.synchronize()
        cd = direct.counts()
        g.load(seg.cols, seg.n, eid)
        g.replay()
        torch.cuda.synchronize()
        cg = graphed.counts()
        assert cd[3] == 0 and cg[3] == 0
        assert cd[:3] == cg[:3], (cd, cg)
        hd, hg = direct.hits.to_numpy(cd[2]), graphed.hits.to_numpy(cg[2])
        for k in hd:
            assert np.array_equal(hd[k], hg[k]), k
        assert cd[2] > 0


def test_batch_graph_replay_matches_direct_batches():
    """A batch of events captured once (sim.BatchGraphRunner: event offsets
    and ids in device memory, fixed capacities) and replayed for two other
    batches, one with fewer events than its slots: the hits equal those of
    the same batches called directly, bit for bit (FP32 form)."""
    cfg = params.small_config(precision=0)
    lut_dev, _ = lut_pair(cfg)
    batches = []
    for b, sizes in enumerate(((30, 12, 45, 20), (50, 8, 33))):
        evs = [events.scatter_event(cfg, 950 + 10 * b + i, n, max_len=0.6) for i, n in enumerate(sizes)]
        ids = [3000 + 10 * b + i for i in range(len(evs))]
        batches.append(sim.Segments.batch_from_numpy(evs, ids))
    E = 4
    cap = max(bt.n for bt in batches) + 11
    mk = lambda: sim.EventRunner(cfg, lut_dev, params.LUT["nt"], params.LUT["bins_per_pitch"], cap,   # noqa: E731
                                 64 * cap, 40 * cap, 200000, max_events=E)
    direct, graphed = mk(), mk()
    g = sim.BatchGraphRunner(graphed)
    for bt in batches:
        direct.enqueue(bt)
        torch.cuda.synchronize()
        cd = direct.counts()
        g.load(bt)
        g.replay()
        torch.cuda.synchronize()
        cg = graphed.counts()
        assert cd[3] == 0 and cg[3] == 0
        assert cd[:3] == cg[:3], (cd, cg)
        hd, hg = direct.hits.to_numpy(cd[2]), graphed.hits.to_numpy(cg[2])
        for k in hd:
            assert np.array_equal(hd[k], hg[k]), k
        assert cd[2] > 0
