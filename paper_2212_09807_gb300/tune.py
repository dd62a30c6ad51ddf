"""Autotuner of the induced-current step's scheduling shapes.

The results of the path do not depend on these shapes (the tensor-core forms
up to their accumulation rounding), only its speed does:
  * tensor-core forms (precision 1, 2): ``tc_units_per_sm``, the work plan's
    target of work units per SM (heavy 32-pixel groups are cut by table-node
    ranges into units of about total / (units x SMs) work), and
    ``tc_record_chunk``, the records a CTA generates and sorts per chunk before
    its node loop;
  * FP32 form (precision 0): ``direct_ctas_per_sm``.
``autotune`` times every candidate on a sample of the workload (one event,
or a batch of events, already on the device) with CUDA events, after one
untimed run that sizes the buffers, and returns the fastest.  It runs all
candidates on one runner (the workspace is sized for the largest scratch
need) by changing the call's configuration between runs.
"""
from __future__ import annotations

import itertools

from . import sim

TC_UNITS = (1, 2, 4, 8)
TC_CHUNKS = (1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20)
DIRECT_CTAS = (2, 3, 4)


def candidates(precision: int) -> list[dict]:
    if precision == 0:
        return [dict(direct_ctas_per_sm=c) for c in DIRECT_CTAS]
    return [dict(tc_units_per_sm=u, tc_record_chunk=r) for u, r in itertools.product(TC_UNITS, TC_CHUNKS)]


def autotune(cfg: dict, lut, nt: int, bins_per_pitch: int, seg: sim.Segments, caps, reps: int = 2,
             device="cuda", cands: list[dict] | None = None):
    """Times each candidate on `seg` (a single event or a batch) and returns
    (best candidate dict, [(candidate, best ms), ...]).  `caps` = (pairs,
    pixels, hits) capacities that fit the sample."""
    import torch
    cands = cands if cands is not None else candidates(int(cfg.get("precision", 0)))
    # workspace for the largest scratch: the most units per SM and the longest record chunk
    big = dict(cfg)
    for k in ("tc_units_per_sm", "tc_record_chunk"):
        big[k] = max(int(c.get(k, 0)) for c in cands)
    run = sim.EventRunner(big, lut, nt, bins_per_pitch, seg.n, *caps, device=device,
                          max_events=max(seg.n_events, 0))
    table = []
    for cand in cands:
        for k, v in cand.items():
            setattr(run.cfg, k, int(v))
        run.enqueue(seg)                         # untimed: lazy loading, caches
        torch.cuda.synchronize()
        if run.counts()[3] != 0:
            raise RuntimeError("autotune: the sample does not fit the given capacities")
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run.enqueue(seg)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        table.append((dict(cand), best))
    del run
    torch.cuda.empty_cache()
    chosen = min(table, key=lambda t: t[1])[0]
    return chosen, table
