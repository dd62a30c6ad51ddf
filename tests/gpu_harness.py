"""Helpers of the GPU parity tests: run each step of the CUDA path through the
C ABI (via the binding) and collect numpy results; compare with the oracle."""
from __future__ import annotations

import numpy as np
import torch

from paper_2212_09807_gb300 import sim
from synth import params, response


def device():
    return torch.device("cuda:0")


def lut_pair(cfg, lut_par=None, **kw):
    """(FP32 padded device table, FP64 copy of the same FP32 values for the oracle)."""
    lut_par = lut_par or params.LUT
    lut64 = response.lut_for(cfg, lut_par, **kw)
    pad = response.pad_rows(lut64)
    oracle_lut = pad[..., : lut_par["nt"]].astype(np.float64)
    return torch.as_tensor(pad, device=device()), oracle_lut


class Steps:
    """Runs a1..a5 one entry point at a time and keeps every intermediate."""

    def __init__(self, cfg: dict, seg: dict, lut_dev, event_id=0, pair_cap=None, pix_cap=None,
                 hit_cap=None, lut_par=None):
        lut_par = lut_par or params.LUT
        dev = device()
        self.cfg_dict = cfg
        self.cfg = sim.make_config(cfg)
        self.seg = sim.Segments.from_numpy(seg, event_id, dev)
        self.n = self.seg.n
        self.resp = sim.Response(lut_dev, lut_par["nt"], lut_par["bins_per_pitch"])
        self.dr = sim.Drifted(self.n, dev)
        n = self.n
        self.pair_cap = pair_cap if pair_cap is not None else max(64, 64 * n)
        self.pix_cap = pix_cap if pix_cap is not None else max(64, 40 * n)
        self.hit_cap = hit_cap if hit_cap is not None else 200000
        i32 = dict(dtype=torch.int32, device=dev)
        self.seg_pix_off = torch.zeros(n + 1, **i32)
        self.seg_pix_ids = torch.zeros(max(self.pair_cap, 1), **i32)
        self.active = torch.zeros(max(self.pix_cap, 1), **i32)
        self.pix_seg_off = torch.zeros(self.pix_cap + 1, **i32)
        self.pix_seg_ids = torch.zeros(max(self.pair_cap, 1), **i32)
        wsb = sim.workspace_size(self.cfg, n, self.pair_cap, self.pix_cap)
        self.ws = torch.zeros((wsb + 7) // 8, dtype=torch.int64, device=dev)
        self.counts = self.ws[:4]
        self.current = torch.zeros(self.pix_cap, int(cfg["n_ticks"]), dtype=torch.float32, device=dev)
        self.hits = sim.Hits(self.hit_cap, dev)
        self.event_id = event_id

    def quench_drift(self):
        sim.sim_quench_drift(self.cfg, self.seg, self.dr)
        return self

    def pixel_map(self):
        sim.sim_pixel_map(self.cfg, self.seg, self.dr, self.resp, self.seg_pix_off, self.seg_pix_ids[: self.pair_cap],
                          self.active[: self.pix_cap], self.pix_seg_off, self.pix_seg_ids, self.ws)
        return self

    def induced_current(self):
        sim.sim_induced_current(self.cfg, self.seg, self.dr, self.resp, self.active, self.pix_seg_off,
                                self.pix_seg_ids, self.counts, self.current[: self.pix_cap], self.ws)
        return self

    def electronics(self):
        sim.sim_electronics(self.cfg, self.seg, self.active, self.current[: self.pix_cap], self.counts,
                            self.hits, self.ws)
        return self

    def all(self):
        return self.quench_drift().pixel_map().induced_current().electronics()

    # -- readback -------------------------------------------------------
    def drifted_np(self):
        torch.cuda.synchronize()
        return {k: getattr(self.dr, k).cpu().numpy() for k in ("Qa", "t_drift", "sigma_T", "sigma_L", "anode",
                                                                "n_samples")}

    def count_values(self):
        torch.cuda.synchronize()
        return [int(x) for x in self.counts.cpu().tolist()]

    def maps_np(self):
        n_pairs, n_pix, _, status = self.count_values()
        assert status == 0, status
        return dict(seg_off=self.seg_pix_off.cpu().numpy(), seg_ids=self.seg_pix_ids[:n_pairs].cpu().numpy(),
                    active=self.active[:n_pix].cpu().numpy(), pix_off=self.pix_seg_off[: n_pix + 1].cpu().numpy(),
                    pix_ids=self.pix_seg_ids[:n_pairs].cpu().numpy())

    def current_np(self):
        n_pix = self.count_values()[1]
        return self.current[:n_pix].cpu().numpy()

    def hits_np(self):
        n_hits = self.count_values()[2]
        return self.hits.to_numpy(min(n_hits, self.hit_cap))


# Tie band (electrons) of the end-to-end hit comparison, per current form: the
# charge error each form leaves at the front end's decisions (FP32: a
# few 1e-2 e- on the densest pixels; FP16 tensor cores: ~0.5 e-, from their
# truncating FP32 accumulation).  Mismatches were measured at 0.05 e- (FP32)
# and 0.5 e- (FP16) on the full-size module event and spill, none above.
BAND = {0: 0.2, 2: 1.0}


def tie_cap(p_ties):
    """Largest number of tied pixels a band may cut, from the oracle's own tie
    probabilities (p_tie of each hit pixel's trace): their expected number
    plus four binomial standard deviations plus two."""
    p = np.asarray(p_ties, dtype=np.float64)
    return float(p.sum() + 4.0 * np.sqrt((p * (1.0 - p)).sum()) + 2.0)


def prefix_charge_ok(I_gpu, I_ref, rel, floor_frac=2e-6):
    """Every prefix sum of each pixel's current (the charge integrated by each
    tick) within rel of the pixel's largest one plus floor_frac of the peak
    pixel charge; returns (ok, worst relative error)."""
    q_ref = np.cumsum(I_ref, axis=-1)
    scale = np.abs(q_ref).max(axis=-1)
    cum = np.abs(np.cumsum(np.asarray(I_gpu, np.float64) - I_ref, axis=-1)).max(axis=-1)
    ok = bool(np.all(cum <= rel * scale + floor_frac * scale.max()))
    return ok, float(np.max(cum / np.maximum(scale, 1e-300)))


def current_errors(I_gpu, I_ref):
    """Per-pixel relative infinity-norm error and relative error of the integrated charge."""
    num = np.abs(I_gpu - I_ref).max(axis=-1)
    den = np.maximum(np.abs(I_ref).max(axis=-1), 1e-300)
    qg, qr = I_gpu.sum(axis=-1), I_ref.sum(axis=-1)
    return num / den, np.abs(qg - qr) / np.maximum(np.abs(qr), 1e-300)


def hits_of_pixel(h, pid):
    m = h["pixel"] == pid
    return {k: v[m] for k, v in h.items()}


def compare_pixel_hits(g, ref, lsb_e):
    """Hits of one pixel, GPU vs oracle, up to the oracle's first tie.

    Returns (ok, n_compared).  Hits whose crossing or ADC tick is at or after
    the oracle's tie tick are not compared (everything after a tie differs).
    """
    tie = ref["tie_tick"]
    lim = tie if tie >= 0 else 1 << 30
    rm = (ref["t_adc"] < lim) & (ref["t_cross"] < lim)
    gm = (g["t_adc"] < lim) & (g["t_cross"] < lim)
    rt = ref["t_cross"][rm]
    if len(rt) != int(gm.sum()):
        return False, 0
    same = (np.array_equal(rt, g["t_cross"][gm]) and np.array_equal(ref["t_adc"][rm], g["t_adc"][gm])
            and np.array_equal(ref["adc"][rm], g["adc"][gm].astype(np.int64)))
    return same, len(rt)
