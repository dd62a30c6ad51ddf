"""GPU parity of the light path (Sec. 4) through the C ABI against the FP64
oracle.

Each step is checked on the GPU's own input to that step (so that its
arithmetic alone is compared), and the chain end to end:
  * yield: voxel and tick bit-exact (FP32 decisions on both sides),
    photoelectrons within 1e-6 relative;
  * photocurrent: within 2^-17 p.e. per term (the fixed-point rounding) plus
    1e-6 relative;
  * scintillation: within 2e-5 of the row's maximum (FP32 recurrences,
    FP64 carries);
  * fluctuation: Poisson counts bit-exact (the same FP64 decisions; ticks whose
    decision lies within 1e-12 of its threshold are excluded), normal draws
    within 1e-5 relative;
  * electronics: the analog waveform within 2e-4 ADC + 1e-5 relative, ADC codes
    bit-exact except samples within 1e-3 ADC + 2e-6 |v| of a rounding
    boundary.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_09807_gb300 import sim
from synth import events, light, params

pytestmark = pytest.mark.gpu


class LightRun:
    def __init__(self, cfg, seg, L=None, t_start=-0.05, n_ticks=4096, event_id=3):
        self.L = L or dict(light.LIGHT)
        self.cfg = cfg
        self.tab = light.tables(cfg, self.L)
        dev = torch.device("cuda:0")
        self.light = sim.Light(self.L, self.tab, t_start, n_ticks, dev)
        self.c = sim.make_config(cfg)
        self.seg = sim.Segments.from_numpy(seg, event_id, dev)
        self.event_id = event_id
        n = self.seg.n
        self.dr = sim.Drifted(n, dev)
        sim.sim_quench_drift(self.c, self.seg, self.dr)
        nd = self.light.n_det
        ndt = self.light.n_det_total(self.c)
        self.ndt = ndt
        self.npe = torch.empty(max(n, 1) * nd, dtype=torch.float32, device=dev)
        self.tick = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        self.vox = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        self.pe = torch.empty(ndt * n_ticks, dtype=torch.int64, device=dev)
        self.S = torch.empty(ndt * n_ticks, dtype=torch.float32, device=dev)
        self.obs = torch.empty(ndt * n_ticks, dtype=torch.float32, device=dev)
        self.V = torch.empty(ndt * n_ticks, dtype=torch.float32, device=dev)
        self.wave = torch.empty(ndt * self.light.n_samples, dtype=torch.uint16, device=dev)
        self.T = n_ticks

    def run(self):
        c, lt = self.c, self.light
        sim.sim_light_yield(c, lt, self.seg, self.dr, self.npe, self.tick, self.vox)
        sim.sim_light_photocurrent(c, lt, self.seg, self.dr, self.npe, self.tick, self.vox, self.pe)
        sim.sim_light_scintillation(c, lt, self.pe, self.S)
        sim.sim_light_fluctuate(c, lt, self.event_id, self.S, self.obs)
        sim.sim_light_electronics(c, lt, self.event_id, self.obs, self.V, self.wave)
        torch.cuda.synchronize()
        return self

    def np(self):
        n, nd, T = self.seg.n, self.light.n_det, self.T
        return dict(npe=self.npe[: n * nd].cpu().numpy().reshape(n, nd), tick=self.tick[:n].cpu().numpy(),
                    vox=self.vox[:n].cpu().numpy(), anode=self.dr.anode.cpu().numpy(),
                    pe=self.pe.cpu().numpy().reshape(self.ndt, T).astype(np.float64) / 65536.0,
                    S=self.S.cpu().numpy().reshape(self.ndt, T), obs=self.obs.cpu().numpy().reshape(self.ndt, T),
                    V=self.V.cpu().numpy().reshape(self.ndt, T),
                    wave=self.wave.cpu().numpy().reshape(self.ndt, -1).astype(np.int32))


def _check_steps(cfg, seg, lr, g, dets, lo):
    o = oracle.Oracle(cfg, params.LUT)
    d = o.quench_drift(seg)
    npe, tick, vox = lo.segments(seg, d)
    act = d["anode"] >= 0
    assert np.array_equal(g["vox"][act], vox[act]) and np.array_equal(g["tick"][act], tick[act])
    assert np.allclose(g["npe"], npe, rtol=1e-6, atol=1e-9 * max(1.0, npe.max()))
    # light truth: mean arrival time per (segment, photosensor)
    n = lr.seg.n
    t_arr = torch.empty(max(n, 1) * lr.light.n_det, dtype=torch.float32, device="cuda:0")
    sim.sim_light_truth(lr.c, lr.light, n, lr.tick, lr.vox, t_arr)
    torch.cuda.synchronize()
    ref_t = lo.truth(tick, vox)
    got_t = t_arr[: n * lr.light.n_det].cpu().numpy().reshape(n, -1)
    assert np.allclose(got_t, ref_t, rtol=1e-6, atol=1e-6)
    nd = lr.light.n_det
    n_cmp = n_pois = 0
    for det in dets:
        k = det % nd
        # photocurrent on the GPU's yield
        I = lo.photocurrent(g["npe"].astype(np.float64), g["tick"], g["vox"], g["anode"], det)
        n_terms = int(((g["anode"] == det // nd) & (g["vox"] >= 0)).sum()) * lr.L["nt"]
        assert np.all(np.abs(g["pe"][det] - I) <= n_terms * 2.0 ** -17 + 1e-6 * np.abs(I).max() + 1e-12)
        # end to end: the oracle's own yield
        I2 = lo.photocurrent(npe, tick, vox, d["anode"], det)
        assert np.allclose(g["pe"][det], I2, rtol=0, atol=1e-5 * max(1.0, np.abs(I2).max()))
        # scintillation on the GPU's photocurrent
        S = lo.scintillation(g["pe"][det])
        assert np.all(np.abs(g["S"][det] - S) <= 2e-5 * max(np.abs(S).max(), 1e-3))
        # fluctuation on the GPU's scintillation
        n, mg = lo.fluctuate(g["S"][det].astype(np.float64), det, lr.event_id)
        lam = g["S"][det].astype(np.float64) * float(np.float32(lr.L["tick_us"]))
        pois = (lam <= 30.0) & (mg > 1e-12)
        assert np.array_equal(g["obs"][det][pois], n[pois]), np.nonzero(g["obs"][det][pois] != n[pois])
        nrm = lam > 30.0
        assert np.allclose(g["obs"][det][nrm], n[nrm], rtol=1e-5)
        n_pois += int(pois.sum())
        # electronics on the GPU's counts
        V, vs, code, cm = lo.electronics(g["obs"][det].astype(np.float64), det, lr.event_id)
        assert np.all(np.abs(g["V"][det] - V) <= 2e-4 + 1e-5 * np.abs(V))
        ok = cm > 1e-3 + 2e-6 * np.abs(vs)
        assert np.array_equal(g["wave"][det][ok], code[ok])
        assert ok.mean() > 0.99
        n_cmp += len(code)
    return n_cmp, n_pois


def test_light_path_small_event_against_oracle():
    cfg = params.small_config()
    seg = events.scatter_event(cfg, 77, 60, max_len=0.8, t_range=(0.0, 1.5))
    lr = LightRun(cfg, seg).run()
    g = lr.np()
    lo = oracle.LightOracle(cfg, lr.L, lr.tab, -0.05, lr.T)
    assert lr.light.n_samples == lo.n_samples
    assert g["pe"].sum(axis=1).max() > 50.0                       # real light reached the detectors
    dets = np.argsort(-g["pe"].sum(axis=1))[:4].tolist() + [1]
    n_cmp, n_pois = _check_steps(cfg, seg, lr, g, dets, lo)
    assert n_pois > 10000


def test_light_path_large_means_and_short_scintillation():
    """Large deposits (normal branch above 30 p.e. per tick) and a slow time
    constant short enough for the truncation to act inside the window."""
    cfg = params.small_config()
    seg = events.scatter_event(cfg, 78, 40, max_len=1.0, t_range=(0.0, 0.5))
    seg["dE"] = (seg["dE"] * 60.0).astype(np.float32)
    L = dict(light.LIGHT, tau_slow_us=0.4, eff=0.2)
    lr = LightRun(cfg, seg, L=L, n_ticks=6000).run()
    g = lr.np()
    lo = oracle.LightOracle(cfg, lr.L, lr.tab, -0.05, lr.T)
    assert lo.n_trunc == 2000
    lam = g["S"] * float(np.float32(L["tick_us"]))
    assert (lam > 30.0).sum() > 100
    dets = np.argsort(-g["pe"].sum(axis=1))[:3].tolist()
    _check_steps(cfg, seg, lr, g, dets, lo)


def test_light_module_event_sampled_and_reproducible():
    """The module event (~2e4 segments, 32 photosensors) at its full window:
    sampled photosensors step by step against the oracle, the whole path
    through sim_light_event bitwise equal to the steps, twice."""
    cfg = params.module_config()
    seg = events.module_event(cfg, seed=params.BASE["seed"] + 1)
    t0, T = light.window(float(seg["t0"].min()), float(seg["t1"].max()))
    lr = LightRun(cfg, seg, t_start=t0, n_ticks=T, event_id=1).run()
    g = lr.np()
    lo = oracle.LightOracle(cfg, lr.L, lr.tab, t0, T)
    dets = np.argsort(-g["pe"].sum(axis=1))[:2].tolist()
    _check_steps(cfg, seg, lr, g, dets, lo)
    ws = torch.empty((sim.light_workspace_size(lr.c, lr.light, lr.seg.n) + 7) // 8, dtype=torch.int64,
                     device="cuda:0")
    for _ in range(2):
        wave = torch.empty_like(lr.wave)
        sim.sim_light_event(lr.c, lr.light, lr.seg, lr.dr, wave, ws)
        torch.cuda.synchronize()
        assert torch.equal(wave, lr.wave)


def test_light_path_window_edges():
    """Light that starts on the window's first tick (the scintillation sum's
    u = t term) in a window of 16 k + 1 ticks, whose last digitiser sample
    falls on the last tick (read without a neighbour): step by step against
    the oracle."""
    cfg = params.small_config()
    seg = events.scatter_event(cfg, 79, 30, max_len=0.8)
    seg["t0"][:] = np.float32(-0.05 + 0.0004)           # 0.4 ns after the window start: tick 0
    seg["t1"][:] = np.float32(-0.05 + 0.0004)
    lr = LightRun(cfg, seg, n_ticks=4097).run()
    g = lr.np()
    lo = oracle.LightOracle(cfg, lr.L, lr.tab, -0.05, lr.T)
    assert lr.light.n_samples == lo.n_samples == 257           # the last sample at tick 4096
    act = g["anode"] >= 0
    assert np.all(g["tick"][act] == 0)
    assert g["pe"][:, 0].max() > 1.0                            # light on the first tick
    dets = np.argsort(-g["pe"][:, 0])[:3].tolist()
    _check_steps(cfg, seg, lr, g, dets, lo)
