"""Edge cases of the entry points after the front end and of the light path,
through the C ABI: empty inputs and degenerate cases."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import sim
from synth import events, light, params

from gpu_harness import Steps, lut_pair

pytestmark = pytest.mark.gpu
KEYS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")


def _seg(rows):
    a = np.asarray(rows, dtype=np.float32).reshape(-1, 9)
    return {k: np.ascontiguousarray(a[:, i]) for i, k in enumerate(KEYS)}


def test_light_path_without_segments_is_noise_and_pedestal():
    """No deposits: the photocurrent is zero, the waveform is the noise plus
    the pedestal, equal to the oracle's electronics of a zero count."""
    cfg = params.small_config()
    L = dict(light.LIGHT)
    tab = light.tables(cfg, L)
    dev = torch.device("cuda:0")
    T = 2048
    lt = sim.Light(L, tab, 0.0, T, dev)
    c = sim.make_config(cfg)
    seg = sim.Segments({k: torch.empty(0, dtype=torch.float32, device=dev) for k in KEYS}, 5)
    dr = sim.Drifted(0, dev)
    ndt = lt.n_det_total(c)
    ws = torch.empty((sim.light_workspace_size(c, lt, 0) + 7) // 8, dtype=torch.int64, device=dev)
    wave = torch.empty(ndt * lt.n_samples, dtype=torch.uint16, device=dev)
    sim.sim_light_event(c, lt, seg, dr, wave, ws)
    pe = torch.empty(ndt * T, dtype=torch.int64, device=dev)
    sim.sim_light_photocurrent(c, lt, seg, dr, None, None, None, pe)
    S = torch.empty(ndt * T, dtype=torch.float32, device=dev)
    sim.sim_light_scintillation(c, lt, pe, S)
    torch.cuda.synchronize()
    assert int(pe.abs().sum().item()) == 0 and float(S.abs().sum().item()) == 0.0
    w = wave.cpu().numpy().reshape(ndt, -1).astype(np.int32)
    lo = oracle.LightOracle(cfg, L, tab, 0.0, T)
    for det in (0, ndt - 1):
        _, vs, code, mg = lo.electronics(np.zeros(T), det, 5)
        ok = mg > 1e-3
        assert np.array_equal(w[det][ok], code[ok])
        assert abs(w[det].mean() - L["pedestal"]) < 1.0


def test_light_segment_outside_the_window_adds_nothing():
    """A deposit arriving after the window: no photocurrent in the window."""
    cfg = params.small_config()
    L = dict(light.LIGHT)
    tab = light.tables(cfg, L)
    dev = torch.device("cuda:0")
    lt = sim.Light(L, tab, 0.0, 1024, dev)
    c = sim.make_config(cfg)
    seg = sim.Segments.from_numpy(_seg([(10, 10, 5, 50.0, 10.3, 10, 5, 50.0, 1.0)]), 1, dev)
    dr = sim.Drifted(1, dev)
    sim.sim_quench_drift(c, seg, dr)
    npe = torch.empty(lt.n_det, dtype=torch.float32, device=dev)
    tick = torch.empty(1, dtype=torch.int32, device=dev)
    vox = torch.empty(1, dtype=torch.int32, device=dev)
    pe = torch.empty(lt.n_det_total(c) * 1024, dtype=torch.int64, device=dev)
    sim.sim_light_yield(c, lt, seg, dr, npe, tick, vox)
    sim.sim_light_photocurrent(c, lt, seg, dr, npe, tick, vox, pe)
    torch.cuda.synchronize()
    assert float(npe.sum().item()) > 0 and int(tick.item()) > 1024
    assert int(pe.abs().sum().item()) == 0


def test_truth_points_and_dqdx_without_hits():
    """An event whose charge stays below threshold: no hits; truth, points and
    dQ/dx run on zero hits and leave zeros."""
    cfg = params.small_config(thr_e=1.0e9)
    seg = events.scatter_event(cfg, 5, 10, max_len=0.4)
    lut_dev, _ = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=2).all()
    assert st.count_values()[2] == 0
    tr = sim.Truth(st.hit_cap, 3, max_cells=16)
    sim.sim_hit_truth(st.cfg, st.seg, st.dr, st.resp, sim.sim_response_cumulative(st.resp), st.active,
                      st.pix_seg_off, st.pix_seg_ids, st.counts, st.pix_cap, st.hits, tr)
    assert tr.counts() == [0, 0, 0, 0]
    dev = torch.device("cuda:0")
    x, y, z = (torch.zeros(st.hit_cap, dtype=torch.float32, device=dev) for _ in range(3))
    sim.sim_hit_points(st.cfg, st.hits, x, y, z)
    dq = torch.full((4,), 7.0, dtype=torch.float64, device=dev)
    cnt = torch.full((4,), 7, dtype=torch.int32, device=dev)
    sim.sim_track_dqdx(x, y, z, st.hits.q, st.hits.n_out, (0, 0, 0), (1, 0, 0), 1.0, 4, 1.0, dq, cnt)
    torch.cuda.synchronize()
    assert float(x.abs().sum().item()) == 0.0
    assert np.all(dq.cpu().numpy() == 0.0) and np.all(cnt.cpu().numpy() == 0)


def test_truth_with_zero_capacity_is_a_no_op():
    cfg = params.small_config()
    seg = events.scatter_event(cfg, 6, 20, max_len=0.6)
    lut_dev, _ = lut_pair(cfg)
    st = Steps(cfg, seg, lut_dev, event_id=2).all()
    tr = sim.Truth(0, 2, max_cells=16)
    sim.sim_hit_truth(st.cfg, st.seg, st.dr, st.resp, sim.sim_response_cumulative(st.resp), st.active,
                      st.pix_seg_off, st.pix_seg_ids, st.counts, st.pix_cap, st.hits, tr)
    assert tr.counts()[3] == 0
