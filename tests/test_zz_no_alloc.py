"""The allocation-free pixel map against the workspace-based one.

Some callers cannot call cudaMalloc while they process events: services that
reserve their whole device-memory budget at start-up and must not allocate in
their event loop, or code embedded in a host framework whose allocator owns
every device buffer.  sim_pixel_map_noalloc serves them by keeping its
scratch in a fixed array inside the library.  The map is integer work, so its
output must equal sim_pixel_map's bit for bit, and it must keep doing so on
consecutive calls, which all reuse the same scratch array.

This file is collected last on purpose; it passes alone in a fresh process
and after the other GPU tests.
"""
import numpy as np
import pytest
import torch

from paper_2212_09807_gb300 import sim
from synth import events, params

from gpu_harness import Steps, lut_pair

pytestmark = pytest.mark.gpu


def _read(counts, seg_off, seg_ids, active, pix_off, pix_ids):
    torch.cuda.synchronize()
    n_pairs, n_pix, _, status = [int(x) for x in counts.cpu().tolist()]
    return dict(counts=(n_pairs, n_pix, status), seg_off=seg_off.cpu().numpy(),
                seg_ids=seg_ids[:n_pairs].cpu().numpy(), active=active[:n_pix].cpu().numpy(),
                pix_off=pix_off[: n_pix + 1].cpu().numpy(), pix_ids=pix_ids[:n_pairs].cpu().numpy())


def test_noalloc_map_equals_workspace_map_on_two_calls_in_a_row():
    cfg = params.small_config()
    lut_dev, _ = lut_pair(cfg)
    dev = torch.device("cuda:0")
    for seed, n in ((11, 300), (12, 120)):
        seg = events.scatter_event(cfg, seed, n, max_len=0.8)
        st = Steps(cfg, seg, lut_dev, event_id=seed).quench_drift().pixel_map()
        ref = _read(st.counts, st.seg_pix_off, st.seg_pix_ids, st.active, st.pix_seg_off, st.pix_seg_ids)
        assert ref["counts"][2] == 0 and ref["counts"][1] > 0
        i32 = dict(dtype=torch.int32, device=dev)
        seg_off = torch.full((st.n + 1,), -7, **i32)
        seg_ids = torch.full((st.pair_cap,), -7, **i32)
        active = torch.full((st.pix_cap,), -7, **i32)
        pix_off = torch.full((st.pix_cap + 1,), -7, **i32)
        pix_ids = torch.full((st.pair_cap,), -7, **i32)
        counts = torch.full((4,), -7, dtype=torch.int64, device=dev)
        sim.sim_pixel_map_noalloc(st.cfg, st.seg, st.dr, st.resp, seg_off, seg_ids, active, pix_off, pix_ids,
                                  counts)
        got = _read(counts, seg_off, seg_ids, active, pix_off, pix_ids)
        assert got["counts"] == ref["counts"]
        for k in ("seg_off", "seg_ids", "active", "pix_off", "pix_ids"):
            assert np.array_equal(got[k], ref[k]), k


def test_noalloc_map_rejects_detectors_beyond_its_scratch():
    cfg = params.spill_config()            # 35 modules: 6.86 M pixels need ~55 MB of scratch
    lut_dev, _ = lut_pair(params.small_config())
    seg = events.scatter_event(cfg, 3, 10)
    st = Steps(cfg, seg, lut_dev, pair_cap=64, pix_cap=64).quench_drift()
    counts = torch.zeros(4, dtype=torch.int64, device="cuda:0")
    with pytest.raises(sim.SimError) as e:
        sim.sim_pixel_map_noalloc(st.cfg, st.seg, st.dr, st.resp, st.seg_pix_off, st.seg_pix_ids, st.active,
                                  st.pix_seg_off, st.pix_seg_ids, counts)
    assert e.value.code == -2
