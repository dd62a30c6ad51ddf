#!/usr/bin/env python
"""Benchmark of the GB300 charge-readout path (arXiv:2212.09807, Sec. 3).

One step = the whole hot path (quench+drift, pixel map, induced current,
electronics) over one synthetic event resident in HBM.  Default workload: one
detector module (2 TPCs, 2 anodes of 4x5 tiles of 70x70 pixels) with one
neutrino-like interaction of ~20k segments.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only (independent events per rank, no data-path
collective); the barrier and the max over ranks of the timed region use
torch.distributed.  ``--impl reference`` times the FP64 CPU oracle (the only
reference this project has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import events, params, response  # noqa: E402

# kernels per step: 1 quench/drift + 14 pixel map + 6 electronics, plus the induced current:
# 1 (FP32 direct) or 13 (tensor cores: work plan 4 + two 3-kernel scans, table unfolding 1,
# contraction 1, reduction of split groups 1)
KERNELS_PER_STEP = {0: 22, 1: 34, 2: 34}
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["module", "tile", "spill"], default="module")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--precision", type=int, choices=[0, 1, 2], default=2,
                    help="induced-current form of the headline: 0 FP32 direct, 1 BF16 / 2 FP16 tensor cores")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the other induced-current forms")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-vs-plain request stream")
    ap.add_argument("--no-post", action="store_true", help="skip timing truth, hit points and dQ/dx")
    ap.add_argument("--no-light", action="store_true", help="skip timing the light path")
    ap.add_argument("--no-tune", action="store_true",
                    help="time the headline event with the default scheduling shapes instead of autotuned ones")
    ap.add_argument("--serving-requests", type=int, default=15, help="requests per load point")
    ap.add_argument("--batched-events", type=int, default=32)
    ap.add_argument("--batched-hi", type=float, default=1.0e4, help="largest event of the batched comparison")
    return ap.parse_args()


def workload(name):
    seed = params.BASE["seed"]
    if name == "tile":
        cfg = params.tile_config()
        seg = events.tile_muon(cfg, seed)
        desc = "tile_muon_200seg: 1 TPC, 1 tile 70x70 px, one 100 cm muon of 200 x 0.5 cm segments"
    elif name == "spill":
        cfg = params.spill_config()
        seg = events.spill_event(cfg, seed + 2)
        desc = "spill_35mod: 7x5 modules, 50 interactions + 100 rock muons, t0 ~ U[0,10us]"
    else:
        cfg = params.module_config()
        seg = events.module_event(cfg, seed + 1)
        desc = ("module_nu_20k: 1 module, 2 TPCs, anodes of 4x5 tiles of 70x70 px (196k px), "
                "one interaction of ~20k segments (muon + protons + EM cloud)")
    return cfg, seg, desc


def dist():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, pg=None, device="cpu") -> float:
    """Largest value of x over the job's ranks (x itself without a process group)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, slowest_s: float) -> float:
    """Whole-job rate of replicas (weak scaling): the units all ranks processed
    over the slowest rank's time."""
    return world * units_per_rank / slowest_s


def replica_event_id(rank: int) -> int:
    """Event id of a rank's replica: the same synthetic event, its own random numbers."""
    return rank


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "power_w_max": float(max(power)) if power else None, "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def stored_traffic(kernel_file: str):
    """DRAM bytes per launch from a committed ncu summary, if taken on this exact source."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except OSError:
        return None
    src = open(os.path.join(ROOT, "paper_2212_09807_gb300", "csrc", kernel_file), "rb").read()
    ent = t.get(kernel_file)
    if not ent or ent.get("src_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return ent.get("dram_bytes_per_launch_full")


# ------------------------------------------------------------------ oracle ---

def oracle_sample(cfg, seg, lut64, rng, n_pix=6):
    """Times the FP64 oracle on a bounded sample of one event and scales it to
    the whole event: quench+drift and the (box-restricted brute-force) pixel map
    of every segment are run in full; current + electronics of ``n_pix`` random
    active pixels are timed and scaled by the event's active-pixel count.
    Returns (estimated whole-event seconds, sample description)."""
    import oracle
    o = oracle.Oracle(cfg, params.LUT, lut64)
    t0 = time.perf_counter()
    d = o.quench_drift(seg)
    pix, _, _, _ = o.pixel_map(seg, d)
    t_map = time.perf_counter() - t0
    keys = np.array(sorted(pix))
    pick = rng.choice(keys, min(n_pix, len(keys)), replace=False)
    t0 = time.perf_counter()
    for p in pick:
        I = o.pixel_current(seg, d, int(p), pix[int(p)])
        o.electronics(int(p), I)
    t_pix = (time.perf_counter() - t0) / len(pick)
    est = t_map + t_pix * len(keys)
    desc = (f"oracle, 1 thread: quench+drift and pixel map of all {len(seg['x0'])} segments in full, "
            f"current+electronics timed on {len(pick)} random active pixels and scaled to all "
            f"{len(keys)} active pixels")
    return est, desc


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return
    cfg, seg, desc = workload(args.workload)
    lut64 = response.pad_rows(response.lut_for(cfg, params.LUT))[..., : params.LUT["nt"]].astype(np.float64)
    S = len(seg["x0"])
    rng = np.random.default_rng(0)
    ests = []
    t_start = time.perf_counter()
    for i in range(args.warmup + args.steps):
        est, sdesc = oracle_sample(cfg, seg, lut64, rng, n_pix=3)
        if i >= args.warmup:
            ests.append(est)
    wall = time.perf_counter() - t_start
    v = S / float(np.mean(ests))
    print(json.dumps({
        "impl": "reference", "metric": "segments/s", "value": v, "unit": "segments/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic", "config": {"workload": desc, "segments": S},
        "cpu_baseline": {"value": v, "unit": "segments/s", "cores": 1, "kind": "oracle", "sample": sdesc},
        "e2e": {"value": v, "unit": "segments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall, "vs_baseline": None,
    }))


# --------------------------------------------------------------------- ours ---

def batched_vs_plain(cfg, lut, dev, n_events=32, lo=1.0e3, hi=1.0e4, reps=2):
    """The same events run one sim_event call each (plain) and as one batch;
    segments/s of both and the per-event latencies of the plain form (each
    event's own device time) against the batch's completion time."""
    import torch
    from paper_2212_09807_gb300 import sim
    evs = events.batch_events(cfg, params.BASE["seed"] + 4, n_events, lo, hi)
    sizes = [len(e["x0"]) for e in evs]
    total, big = sum(sizes), max(sizes)
    ids = list(range(1000, 1000 + n_events))
    from paper_2212_09807_gb300 import serve
    singles = [sim.Segments.from_numpy(e, i, dev) for e, i in zip(evs, ids)]
    batch = sim.Segments.batch_from_numpy(evs, ids, dev)

    def fitted(n, caps, runs, max_events=0):
        """Runner whose capacities fit every event of `runs` (untimed sizing pass)."""
        while True:
            r = sim.EventRunner(cfg, lut, params.LUT["nt"], params.LUT["bins_per_pitch"], n, *caps, device=dev,
                                max_events=max_events)
            worst = [0, 0, 0]
            for sg in runs:
                r.enqueue(sg)
                torch.cuda.synchronize()
                c = r.counts()
                if c[3] != 0:
                    worst = [max(w, x) for w, x in zip(worst, c[:3])]
            if worst == [0, 0, 0]:
                return r
            caps = tuple(max(a, 2 * w) for a, w in zip(caps, worst))
            del r
            torch.cuda.empty_cache()

    plain = fitted(big, serve._caps(big), singles)
    # autotuned scheduling shapes for the batched call, timed on a batch of the first 16 events (untimed here)
    from paper_2212_09807_gb300 import tune
    ns = min(16, n_events)
    sample = sim.Segments.batch_from_numpy(evs[:ns], ids[:ns], dev)
    s_tot = sum(sizes[:ns])
    probe = fitted(s_tot, serve._caps(s_tot), [sample], max_events=ns)
    s_caps = (probe.max_pairs, probe.max_pixels, probe.hits.capacity)
    del probe
    chosen, table = tune.autotune(cfg, lut, params.LUT["nt"], params.LUT["bins_per_pitch"], sample, s_caps,
                                  device=dev)
    tuned_cfg = dict(cfg, **chosen)
    cfg_keep = cfg
    cfg = tuned_cfg
    batch_run = fitted(total, serve._caps(total), [batch], max_events=n_events)
    cfg = cfg_keep
    best_plain, best_batch, lat = None, None, None
    for _ in range(reps):
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(n_events + 1)]
        marks[0].record()
        for k, sg in enumerate(singles):
            plain.enqueue(sg)
            marks[k + 1].record()
        torch.cuda.synchronize()
        t_plain = marks[0].elapsed_time(marks[-1])
        per = [marks[k].elapsed_time(marks[k + 1]) for k in range(n_events)]
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        batch_run.enqueue(batch)
        b1.record()
        torch.cuda.synchronize()
        t_batch = b0.elapsed_time(b1)
        if best_plain is None or t_plain < best_plain:
            best_plain, lat = t_plain, per
        best_batch = t_batch if best_batch is None else min(best_batch, t_batch)
    assert batch_run.counts()[3] == 0
    # the plain loop again, each event a replay of one CUDA graph of the whole step (sim.GraphRunner)
    g = sim.GraphRunner(plain)
    best_graph, glat = None, None
    for _ in range(reps):
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(n_events + 1)]
        marks[0].record()
        for k, sg in enumerate(singles):
            g.load(sg.cols, sg.n, sg.event_id)
            g.replay()
            marks[k + 1].record()
        torch.cuda.synchronize()
        t_graph = marks[0].elapsed_time(marks[-1])
        if best_graph is None or t_graph < best_graph:
            best_graph, glat = t_graph, [marks[k].elapsed_time(marks[k + 1]) for k in range(n_events)]
    assert plain.counts()[3] == 0
    return {"events": n_events, "segments": total, "sizes": f"log-uniform [{lo:.0f}, {hi:.0f}] segments",
            "plain_segments_per_s": total / (best_plain / 1e3), "batched_segments_per_s": total / (best_batch / 1e3),
            "graph_segments_per_s": total / (best_graph / 1e3),
            "plain_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "graph_latency_ms": {"p50": float(np.percentile(glat, 50)), "p99": float(np.percentile(glat, 99))},
            "batched_completion_ms": best_batch,
            "tuning": {"sample": f"batch of the first {ns} events", "chosen": chosen,
                       "candidates_ms": [[c, round(ms, 3)] for c, ms in table]}}



FORMS = {0: ("fp32_direct", "f32"), 1: ("bf16_tensor", "bf16"), 2: ("fp16_tensor", "f16")}


def time_form(cfg, seg, lut, dev, precision, steps, warmup, rank):
    """Times `steps` whole-path steps (the four entry points, one by one, each
    bracketed by CUDA events on the current stream) with the induced-current
    form `precision`, after `warmup` untimed steps and with L2 flushed before
    every step.  Returns (runner, per-step-and-entry ms array, counts)."""
    import torch
    from paper_2212_09807_gb300 import sim
    cfg = dict(cfg, precision=precision)
    S = len(seg["x0"])
    T = int(cfg["n_ticks"])
    caps = [40 * S, 4 * S, 4 * S]
    while True:                         # capacities: grow until the event fits (untimed sizing pass)
        run = sim.EventRunner(cfg, lut, params.LUT["nt"], params.LUT["bins_per_pitch"], S, *caps, device=dev)
        segs = sim.Segments.from_numpy(seg, event_id=rank, device=dev)
        run.enqueue(segs)
        torch.cuda.synchronize()
        n_pairs, n_pix, n_hits, status = run.counts()
        if status == 0:
            break
        caps = [max(caps[0], 2 * n_pairs), max(caps[1], 2 * n_pix), max(caps[2], 2 * n_hits)]
        del run
        torch.cuda.empty_cache()
    v = run.view(S)
    A = sim._alias
    dr = sim.Drifted.wrap(v.dr)
    seg_pix_off = A(v.seg_pix_off, S + 1, torch.int32, dev)
    seg_pix_ids = A(v.seg_pix_ids, run.max_pairs, torch.int32, dev)
    active = A(v.active_pixels, run.max_pixels, torch.int32, dev)
    pix_seg_off = A(v.pix_seg_off, run.max_pixels + 1, torch.int32, dev)
    pix_seg_ids = A(v.pix_seg_ids, run.max_pairs, torch.int32, dev)
    current = A(v.current, run.max_pixels * T, torch.float32, dev).view(run.max_pixels, T)
    counts = run.ws[:4]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)   # 256 MB > L2

    def step(evs):
        evs[0].record()
        sim.sim_quench_drift(run.cfg, segs, dr)
        evs[1].record()
        sim.sim_pixel_map(run.cfg, segs, dr, run.resp, seg_pix_off, seg_pix_ids, active, pix_seg_off,
                          pix_seg_ids, run.ws)
        evs[2].record()
        sim.sim_induced_current(run.cfg, segs, dr, run.resp, active, pix_seg_off, pix_seg_ids, counts, current,
                                run.ws)
        evs[3].record()
        sim.sim_electronics(run.cfg, segs, active, current, counts, run.hits, run.ws)
        evs[4].record()

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(5)]  # noqa: E731
    for _ in range(warmup):
        flush.zero_()
        step(mk())
    torch.cuda.synchronize()
    all_evs = []
    for _ in range(steps):
        flush.zero_()                  # outside the timed intervals: every step starts with a cold L2
        e = mk()
        step(e)
        all_evs.append(e)
    torch.cuda.synchronize()
    per = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in all_evs])   # ms
    counts_now = run.counts()
    assert counts_now[3] == 0
    run.segs = segs
    return run, per, counts_now


def step_rooflines(per, S, n_pairs, n_pix, T):
    """The other steps of the path against their bounds (per-step CUDA-event means):
    quench + drift 36 B in + 88 B out per segment (HBM); electronics 4 B of
    current per pixel-tick read (HBM; its Philox noise makes it ALU-heavy); the
    pixel map as pairs per second (latency of its sort, not bandwidth)."""
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    q_ms, m_ms, e_ms = (float(per[:, i].mean()) for i in (0, 1, 3))
    q = 124.0 * S / (q_ms / 1e3) / 1e9
    e = 4.0 * n_pix * T / (e_ms / 1e3) / 1e9
    return {"quench_drift": {"bound": "hbm", "bytes_per_segment": 124, "achieved": q, "peak": hbm, "unit": "GB/s",
                             "frac": q / hbm},
            "electronics": {"bound": "hbm", "bytes_per_pixel_tick": 4, "achieved": e, "peak": hbm, "unit": "GB/s",
                            "frac": e / hbm},
            "pixel_map": {"pairs": n_pairs, "pairs_per_s": n_pairs / (m_ms / 1e3)}}


def post_hit_steps(run, cfg, dev, reps=5):
    """Times the steps after the front end on the event held by `run` (its last
    sim_event): per-hit charge truth (5 entries per hit), hits -> 3-D points and
    dQ/dx in 1 cm pieces along a line through the detector (L2 flushed before
    each launch; CUDA events on the launching stream)."""
    import torch
    from paper_2212_09807_gb300 import sim
    S = run.segs.n
    n_pairs, n_pix, n_hits, status = run.counts()
    assert status == 0
    v = run.view(S)
    A = sim._alias
    dr = sim.Drifted.wrap(v.dr)
    active = A(v.active_pixels, run.max_pixels, torch.int32, dev)
    pix_seg_off = A(v.pix_seg_off, run.max_pixels + 1, torch.int32, dev)
    pix_seg_ids = A(v.pix_seg_ids, run.max_pairs, torch.int32, dev)
    counts = run.ws[:6]
    cum = sim.sim_response_cumulative(run.resp)
    tr = sim.Truth(run.hits.capacity, 5, device=dev)
    cap = run.hits.capacity
    x, y, z = (torch.empty(cap, dtype=torch.float32, device=dev) for _ in range(3))
    g = params.geometry(cfg)
    o = (0.0, g["y_max"] / 2, g["z_max"] / 2)
    n_pieces = int(np.ceil(g["x_max"])) + 1
    dq = torch.empty(n_pieces, dtype=torch.float64, device=dev)
    cnt = torch.empty(n_pieces, dtype=torch.int32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    calls = {
        # warm-up calls size the cell capacity (a synchronising retry); timed calls do not retry
        "hit_truth": lambda retry=False: sim.sim_hit_truth(run.cfg, run.segs, dr, run.resp, cum, active,
                                                           pix_seg_off, pix_seg_ids, counts, run.max_pixels,
                                                           run.hits, tr, retry=retry),
        "hit_points": lambda: sim.sim_hit_points(run.cfg, run.hits, x, y, z),
        "track_dqdx": lambda: sim.sim_track_dqdx(x, y, z, run.hits.q, run.hits.n_out, o, (1.0, 0.0, 0.0), 1.0,
                                                 n_pieces, 1.0e4, dq, cnt),
    }
    out = {}
    for name, f in calls.items():
        for _ in range(2):
            f(retry=True) if name == "hit_truth" else f()
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[name] = {"ms": float(np.mean(ms)), "hits": n_hits, "hits_per_s": n_hits / (float(np.mean(ms)) / 1e3)}
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    for name, per_hit in (("hit_points", 20), ("track_dqdx", 16)):
        gbs = per_hit * n_hits / (out[name]["ms"] / 1e3) / 1e9
        out[name]["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                 "bytes_per_hit": per_hit}
    out["hit_truth"]["k"] = 5
    cells, runs, units, status = tr.counts()
    assert status == 0
    out["hit_truth"].update({"hit_pixels": runs, "units": units, "cells": cells})
    out["track_dqdx"]["points_in_pieces"] = int(cnt.sum().item())
    return out


def light_path(dev, names=("module", "spill"), reps=5):
    """Times the light path (Sec. 4) on the segments of a workload: each entry
    point (yield, photocurrent, scintillation, fluctuation, electronics) with
    CUDA events on the launching stream, L2 flushed before every pass, and the
    whole path through sim_light_event."""
    import torch
    from paper_2212_09807_gb300 import sim
    from synth import light
    out = {}
    props = torch.cuda.get_device_properties(dev)
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    sm_mhz = measured_peaks().get("sm_max_mhz", 2070.0)
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12      # TFLOP/s, FMA lanes x clock
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    for name in names:
        cfg, seg, desc = workload(name)
        L = dict(light.LIGHT)
        tab = light.tables(cfg, L)
        t0, T = light.window(float(seg["t0"].min()), float(seg["t1"].max()))
        lt = sim.Light(L, tab, t0, T, dev)
        c = sim.make_config(cfg)
        segs = sim.Segments.from_numpy(seg, 1, dev)
        n = segs.n
        dr = sim.Drifted(n, dev)
        sim.sim_quench_drift(c, segs, dr)
        ndt = lt.n_det_total(c)
        f32 = dict(dtype=torch.float32, device=dev)
        npe = torch.empty(n * lt.n_det, **f32)
        tick = torch.empty(n, dtype=torch.int32, device=dev)
        vox = torch.empty(n, dtype=torch.int32, device=dev)
        pe = torch.empty(ndt * T, dtype=torch.int64, device=dev)
        S, obs, V = (torch.empty(ndt * T, **f32) for _ in range(3))
        wave = torch.empty(ndt * lt.n_samples, dtype=torch.uint16, device=dev)
        calls = [("yield", lambda: sim.sim_light_yield(c, lt, segs, dr, npe, tick, vox)),
                 ("photocurrent", lambda: sim.sim_light_photocurrent(c, lt, segs, dr, npe, tick, vox, pe)),
                 ("scintillation", lambda: sim.sim_light_scintillation(c, lt, pe, S)),
                 ("fluctuate", lambda: sim.sim_light_fluctuate(c, lt, 1, S, obs)),
                 ("electronics", lambda: sim.sim_light_electronics(c, lt, 1, obs, V, wave))]
        ws = torch.empty((sim.light_workspace_size(c, lt, n) + 7) // 8, dtype=torch.int64, device=dev)
        wave2 = torch.empty_like(wave)
        for _ in range(2):
            for _, f in calls:
                f()
            sim.sim_light_event(c, lt, segs, dr, wave2, ws)
        torch.cuda.synchronize()
        per = np.zeros((reps, len(calls)))
        whole = []
        for r in range(reps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)]
            ev[0].record()
            for i, (_, f) in enumerate(calls):
                f()
                ev[i + 1].record()
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sim.sim_light_event(c, lt, segs, dr, wave2, ws)
            e1.record()
            torch.cuda.synchronize()
            per[r] = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(calls))]
            whole.append(e0.elapsed_time(e1))
        assert torch.equal(wave, wave2)
        ms = {k: float(per[:, i].mean()) for i, (k, _) in enumerate(calls)}
        ticks = ndt * T
        act = int((dr.anode >= 0).sum().item())
        terms = act * lt.n_det * L["nt"]
        rl = {
            "scintillation": {"bound": "hbm", "bytes_per_tick": 20,
                              "achieved": 20 * ticks / (ms["scintillation"] / 1e3) / 1e9, "peak": hbm,
                              "unit": "GB/s"},
            "fluctuate": {"bound": "hbm", "bytes_per_tick": 8,
                          "achieved": 8 * ticks / (ms["fluctuate"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s"},
            "electronics": {"bound": "alu", "flop_per_tick": 2 * L["n_resp"],
                            "achieved": 2 * L["n_resp"] * ticks / (ms["electronics"] / 1e3) / 1e12,
                            "peak": fp32_peak, "unit": "TFLOP/s",
                            "peak_note": "FP32 FMA lanes x SMs x max SM clock (derived, not measured)"},
            "photocurrent": {"terms": terms, "terms_per_s": terms / (ms["photocurrent"] / 1e3)},
        }
        for v in rl.values():
            if "peak" in v:
                v["frac"] = v["achieved"] / v["peak"]
        out[name] = {"workload": desc, "segments": n, "photosensors": ndt, "ticks": T,
                     "window_us": [t0, t0 + T * float(np.float32(L["tick_us"]))], "samples": lt.n_samples,
                     "ms": ms, "ms_whole_path": float(np.mean(whole)),
                     "segments_per_s": n / (float(np.mean(whole)) / 1e3), "roofline": rl}
        del npe, pe, S, obs, V, wave, wave2, ws
        torch.cuda.empty_cache()
    return out


def form_roofline(run, cfg, precision, a4_s, props, sm_mhz, dev):
    """Roofline of the induced-current kernel of one form: FP32 direct against
    the FP32 FMA peak; tensor-core forms against the measured dense 16-bit
    tensor peak (dense MMA work counted on the device), with the algorithmic
    (useful) work also stated."""
    import torch
    from paper_2212_09807_gb300 import sim
    S = run.max_segments
    dn = run.view(S)
    A = sim._alias
    ns = A(dn.dr.n_samples, S, torch.int32, dev).cpu().numpy().astype(np.int64)
    an = A(dn.dr.anode, S, torch.int32, dev).cpu().numpy()
    samples = int(ns[an >= 0].sum()) * int(cfg["mc_per_sample"])
    L = params.LUT["nt"]
    w_alg = 2.0 * 9 * L * samples                       # flop per launch (9 pixels per point)
    useful = w_alg / a4_s / 1e12
    if precision == 0:
        peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        return {"bound": "alu", "achieved": useful, "peak": peak, "unit": "TFLOP/s", "frac": useful / peak,
                "traffic": stored_traffic("induced_current.cu"), "kernel": "k_induced_current",
                "peak_note": f"FP32 FMA: {props.multi_processor_count} SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz",
                "work_note": "2 flop x 9 pixels x 1950 table ticks per (point, perturbation)"}, samples
    n_mma = int(run.ws[4].item())
    nnz = int(run.ws[5].item())
    L = params.LUT["nt"]
    dense = 2.0 * 128 * 32 * 16 * n_mma / a4_s / 1e12
    useful_q = 2.0 * nnz * L / a4_s / 1e12
    tpk = measured_peaks().get("bf16_tflops_sustained") or 1700.0
    return {"bound": "tensor", "achieved": dense, "peak": tpk, "unit": "TFLOP/s", "frac": dense / tpk,
            "traffic": stored_traffic("induced_current_tc.cu"), "kernel": "k_induced_current_tc",
            "mma_per_launch": n_mma, "nnz_charge_cells": nnz,
            "useful_achieved": useful_q, "useful_frac": useful_q / tpk,
            "per_point_achieved": useful,
            "peak_note": "measured dense bf16 sustained (kernel timed inside a step), of measured; fp16 has the "
                         "same nominal rate",
            "work_note": "dense: 2 x 128 x 32 x 16 flop per MMA (counted on the device); useful: 2 flop x "
                         "nnz(Q) x 1950 table ticks (nonzero binned-charge cells, counted on the device); "
                         "per_point: 2 flop x 9 pixels x 1950 ticks per (point, perturbation)"}, samples


SLICE = 32768        # active pixels per current launch of a large request (serving form)


def serving_vs_plain(precision, dev, n_requests=12, loads=(0.5, 0.7, 0.9), seed_off=20):
    """Serving form against the plain per-event form on the same Poisson
    request streams: 80 % single interactions (~2e4 segments) and 20 % whole
    spills (~1.2e6 segments) on the 35-module detector; the arrival rate is
    each of `loads` times the plain form's capacity (measured on one request
    of each kind first)."""
    import torch
    from paper_2212_09807_gb300 import serve
    cfg = params.spill_config(precision=precision)
    lut = torch.as_tensor(response.pad_rows(response.lut_for(cfg, params.LUT)), device=dev)
    nt, bpp = params.LUT["nt"], params.LUT["bins_per_pitch"]
    seed = params.BASE["seed"] + seed_off
    inter = [events.module_event(cfg, seed + i) for i in range(4)]
    spill = events.spill_event(cfg, seed + 9)
    # service times of the plain form, one request of each kind (after a warm-up one)
    probe = [serve.Request(0, 1, inter[0], 0.0, "interaction"), serve.Request(1, 2, inter[1], 0.0, "interaction"),
             serve.Request(2, 3, spill, 0.0, "spill")]
    res = serve.run_plain(cfg, lut, nt, bpp, probe, device=dev)
    t_int = res[1].done - res[1].admitted
    t_sp = res[2].done - res[2].admitted
    mean_service = 0.8 * t_int + 0.2 * t_sp
    out = []
    for li, load in enumerate(loads):
        rate = load / mean_service
        rng = np.random.default_rng(seed + li)
        n_sp = max(1, round(0.2 * n_requests))                 # exactly 20 % spills, at random positions
        kinds = rng.permutation(np.arange(n_requests) < n_sp)
        t, reqs = 0.0, []
        for i in range(n_requests):
            t += rng.exponential(1.0 / rate)
            if kinds[i]:
                reqs.append(serve.Request(i, 5000 + i, spill, t, "spill"))
            else:
                reqs.append(serve.Request(i, 5000 + i, inter[i % len(inter)], t, "interaction"))
        plain = serve.summarize(serve.run_plain(cfg, lut, nt, bpp, reqs, device=dev))
        torch.cuda.empty_cache()
        srv = serve.Server(cfg, lut, nt, bpp, hbm_budget=120e9, slice_pixels=SLICE, max_jobs=8, device=dev)
        serving = serve.summarize(srv.run(reqs))
        del srv
        torch.cuda.empty_cache()
        out.append({"load": load, "rate_per_s": rate, "plain": plain, "serving": serving})
    return {"requests_per_load": n_requests, "mix": "80% interactions (~2e4 segments), 20% spills (~1.2e6 "
            "segments), 35-module detector", "plain_service_ms": {"interaction": t_int * 1e3, "spill": t_sp * 1e3},
            "hbm_budget_gb": 120, "slice_pixels": SLICE, "loads": out}


def run_ours(args):
    import torch
    from paper_2212_09807_gb300 import sim

    world, rank, local = dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
        pg = tdist
    cfg, seg, desc = workload(args.workload)
    cfg["precision"] = args.precision
    S = len(seg["x0"])
    T = int(cfg["n_ticks"])
    L = params.LUT["nt"]
    lut64 = response.lut_for(cfg, params.LUT)
    lut_pad = response.pad_rows(lut64)
    lut = torch.as_tensor(lut_pad, device=dev)
    props = torch.cuda.get_device_properties(dev)

    # the other forms of the induced-current step, timed on the same event first (untimed for the headline)
    forms = {}
    if not args.no_forms:
        for prec in (0, 1, 2):
            if prec == args.precision:
                continue
            r2, per2, c2 = time_form(cfg, seg, lut, dev, prec, max(3, args.steps // 2), args.warmup, rank)
            sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
            rl, _ = form_roofline(r2, cfg, prec, float(per2[:, 2].mean()) / 1e3, props, sm_max, dev)
            forms[FORMS[prec][0]] = {"dtype": FORMS[prec][1], "ms_per_step": float(per2.sum(axis=1).mean()),
                                     "segments_per_s": S / (float(per2.sum(axis=1).mean()) / 1e3),
                                     "induced_current_ms": float(per2[:, 2].mean()), "roofline": rl}
            del r2
            torch.cuda.empty_cache()

    # scheduling shapes of the induced-current step for this event, picked by the autotuner (untimed);
    # results do not depend on them beyond the tensor-core forms' accumulation rounding
    tuned = None
    if not args.no_tune:
        from paper_2212_09807_gb300 import tune
        segs_dev = sim.Segments.from_numpy(seg, event_id=replica_event_id(rank), device=dev)
        tuned, _ = tune.autotune(cfg, lut, L, params.LUT["bins_per_pitch"], segs_dev, (40 * S, 4 * S, 4 * S),
                                 reps=2, device=dev)
        cfg = dict(cfg, **tuned)
        del segs_dev
        torch.cuda.empty_cache()

    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    clk = ClockSampler(gpu_id)
    clk.start()
    time.sleep(0.15)
    run, per, (n_pairs, n_pix, n_hits, status) = time_form(cfg, seg, lut, dev, args.precision, args.steps,
                                                           args.warmup, replica_event_id(rank))
    clocks = clk.stop()
    step_ms = per.sum(axis=1)
    total_ms = float(step_ms.sum())
    total_ms = max_over_ranks(total_ms, pg, dev)
    value = job_rate(world, S * args.steps, total_ms / 1e3)
    a45_ms = max_over_ranks(float(per[:, 2:].sum()), pg, dev)
    pix_ticks = job_rate(world, n_pix * T * args.steps, a45_ms / 1e3)
    sm_mhz = clocks.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
    roofline, samples = form_roofline(run, cfg, args.precision, float(per[:, 2].mean()) / 1e3, props, sm_mhz, dev)
    forms[FORMS[args.precision][0]] = {"dtype": FORMS[args.precision][1], "ms_per_step": total_ms / args.steps,
                                       "segments_per_s": value / world,
                                       "induced_current_ms": float(per[:, 2].mean()), "roofline": roofline}

    # end to end through the public API: pinned host segments in, hits out
    io = sim.EventIO(run)
    host = {k: torch.as_tensor(np.ascontiguousarray(seg[k], dtype=np.float32)).pin_memory() for k in seg}
    for _ in range(max(1, args.warmup)):
        io.simulate(host, S, replica_event_id(rank))
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(args.steps):
        _, _, hb, db = io.simulate(host, S, replica_event_id(rank))
        h2d, d2h = hb, db
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, pg, dev)
    e2e = {"value": job_rate(world, S * args.steps, e2e_s), "unit": "segments/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}
    post = post_hit_steps(run, cfg, dev) if not args.no_post else None
    del run, io
    torch.cuda.empty_cache()
    light_res = light_path(dev) if not args.no_light else None
    torch.cuda.empty_cache()

    batched = (batched_vs_plain(cfg, lut, dev, args.batched_events, 1.0e3, args.batched_hi,
                                reps=1 if args.batched_events > 64 else 2) if not args.no_batched else None)
    serving = serving_vs_plain(args.precision, dev, args.serving_requests) if not args.no_serving else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        lut_or = lut_pad[..., :L].astype(np.float64)
        est, sdesc = oracle_sample(cfg, seg, lut_or, np.random.default_rng(0), n_pix=8)
        cpu = {"value": S / est, "unit": "segments/s", "cores": 1, "kind": "oracle", "sample": sdesc}

    if rank == 0:
        print(json.dumps({
            "metric": "segments/s", "value": value, "unit": "segments/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": FORMS[args.precision][1], "data": "synthetic",
            "config": {"workload": desc, "segments": S, "active_pixels": n_pix, "pairs": n_pairs,
                       "hits": n_hits, "n_ticks": T, "points": samples, "parallelism": f"replicas{world}",
                       "induced_current_form": FORMS[args.precision][0] + " (FP32 accumulation)",
                       "scheduling": tuned if tuned is not None else "defaults",
                       "l2": "flushed (256 MB write) before every timed step"},
            "pixel_ticks_per_s": pix_ticks,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "step_breakdown_ms": {"quench_drift": float(per[:, 0].mean()), "pixel_map": float(per[:, 1].mean()),
                                  "induced_current": float(per[:, 2].mean()),
                                  "electronics": float(per[:, 3].mean())},
            "roofline": roofline, "step_rooflines": step_rooflines(per, S, n_pairs, n_pix, T),
            "forms": forms, "cpu_baseline": cpu, "e2e": e2e, "batched": batched,
            "serving": serving, "after_front_end": post, "light": light_res,
            "gpu_launches": KERNELS_PER_STEP[args.precision] * args.steps, "clocks": clocks,
        }))
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
