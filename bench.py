#!/usr/bin/env python
"""Benchmark of the GB300 charge-readout path (arXiv:2212.09807, Sec. 3).

One step = the whole hot path (quench+drift, pixel map, induced current,
electronics) over one synthetic event resident in HBM.  Default workload: the
largest single-GPU configuration, a beam spill on a 7x5 array of detector
modules (35 modules, 6.86 M pixels): 50 neutrino-like interactions plus 100
rock muons, ~1.2e6 segments, t0 spread over 10 us.  The one-module
interaction (~2e4 segments) is timed beside it.  Prints one JSON line.

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
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import events, params, response  # noqa: E402

# kernels per step: 1 quench/drift + 14 pixel map + 6 electronics, plus the induced current:
# 3 (FP32: work classes, queue order, sum) or 15 (tensor cores: work plan 5 + two 3-kernel
# scans, table rounding 1, table unfolding 1, contraction 1, reduction of split groups 1)
KERNELS_PER_STEP = {0: 24, 1: 36, 2: 36, 3: 22}
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["module", "tile", "spill"], default="spill")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--precision", type=int, choices=[0, 1, 2, 3], default=2,
                    help="induced-current form of the headline: 0 FP32 (node-binned cells), 1 BF16 / 2 FP16 "
                         "tensor cores, 3 FP32 term by term")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the other induced-current forms")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-vs-plain request stream")
    ap.add_argument("--no-post", action="store_true", help="skip timing truth, hit points and dQ/dx")
    ap.add_argument("--no-light", action="store_true", help="skip timing the light path")
    ap.add_argument("--no-tune", action="store_true",
                    help="time the headline event with the default scheduling shapes instead of autotuned ones")
    ap.add_argument("--serving-requests", type=int, default=60, help="requests per load point")
    ap.add_argument("--serving-loads", default="0.7",
                    help="comma-separated arrival rates as fractions of the plain form's capacity")
    ap.add_argument("--batched-events", type=int, default=256)
    ap.add_argument("--batched-hi", type=float, default=2.0e5, help="largest event of the batched comparison")
    ap.add_argument("--batched-subbatches", type=int, default=4,
                    help="graph-captured sub-batches the batched events are cut into")
    ap.add_argument("--form-steps", type=int, default=2, help="timed steps of each non-headline current form")
    ap.add_argument("--cpu-pixels", type=int, default=1024,
                    help="active pixels of the CPU baseline's timed sample")
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
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median and largest SM clock, largest power and the throttle reasons
        seen in nvidia-smi lines of the query Q (CSV, no header, no units).  A
        sample's reasons count even when its clocks or power do not parse."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons, power = [], [], set(), []
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
            try:
                clk, clk_max = float(f[1]), float(f[2])
            except ValueError:
                continue
            sm.append(clk)
            mx.append(clk_max)
            try:
                power.append(float(f[3]))
            except ValueError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": sorted(reasons) + ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "power_w_max": float(max(power)) if power else None, "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def code_sha256(src: str) -> str:
    """SHA-256 of a CUDA source with its comments removed and blank space
    collapsed: the key of a stored measurement, which a comment edit leaves
    valid and any change to the code invalidates."""
    s = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    s = re.sub(r"//[^\n]*", " ", s)
    s = " ".join(s.split())
    return hashlib.sha256(s.encode()).hexdigest()


def stored_traffic(kernel_file: str, workload_key: str):
    """DRAM bytes per launch from a committed ncu summary of this kernel on this
    workload (entry "<file>@<workload>"), if taken on this source's code."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except OSError:
        return None
    src = open(os.path.join(ROOT, "paper_2212_09807_gb300", "csrc", kernel_file)).read()
    ent = t.get(f"{kernel_file}@{workload_key}")
    if not ent or ent.get("code_sha256") != code_sha256(src):
        return None
    return ent.get("dram_bytes_per_launch_full")


# ------------------------------------------------------------------ oracle ---

def oracle_sample(cfg, seg, lut64, rng, n_pix=1024):
    """Times the FP64 oracle on a bounded sample of one event and scales it to
    the whole event: quench+drift and the pixel map of every segment run in
    full (one thread); current + front end of ``n_pix`` random active pixels
    run on all host cores (the oracle's OpenMP many-pixel functions) and are
    scaled by the event's active-pixel count.  Returns (estimated whole-event
    seconds, host threads used, sample description)."""
    import oracle
    o = oracle.Oracle(cfg, params.LUT, lut64)
    t0 = time.perf_counter()
    d = o.quench_drift(seg)
    m = o.map_event(seg, d)
    t_map = time.perf_counter() - t0
    P = len(m["pixels"])
    idx = np.sort(rng.choice(P, min(n_pix, P), replace=False))
    pix = m["pixels"][idx]
    off = np.concatenate([[0], np.cumsum(m["off"][idx + 1] - m["off"][idx])])
    segs = np.concatenate([m["segs"][m["off"][i]:m["off"][i + 1]] for i in idx])
    t0 = time.perf_counter()
    I = o.pixel_currents(seg, d, pix, off, segs)
    o.electronics_many(pix, I)
    t_pix = (time.perf_counter() - t0) / len(idx)
    threads = o.threads()
    est = t_map + t_pix * P
    desc = (f"FP64 oracle: quench+drift and pixel map of all {len(seg['x0'])} segments in full (1 thread); "
            f"current + front end of {len(idx)} random active pixels on {threads} host threads (OpenMP), "
            f"scaled to all {P} active pixels")
    return est, threads, desc


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
        est, threads, sdesc = oracle_sample(cfg, seg, lut64, rng, n_pix=128)
        if i >= args.warmup:
            ests.append(est)
    wall = time.perf_counter() - t_start
    v = S / float(np.mean(ests))
    print(json.dumps({
        "impl": "reference", "metric": "segments/s", "value": v, "unit": "segments/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic", "config": {"workload": desc, "segments": S},
        "cpu_baseline": {"value": v, "unit": "segments/s", "cores": threads, "kind": "oracle", "sample": sdesc},
        "e2e": {"value": v, "unit": "segments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall, "vs_baseline": None,
    }))


# --------------------------------------------------------------------- ours ---

def batched_vs_plain(cfg, lut, dev, n_events=256, lo=1.0e3, hi=2.0e5, n_sub=4):
    """Batched events (256 interactions with segment counts log-uniform in
    [1e3, 2e5], all waiting at t = 0) run two ways on the same GPU:
      * plain: one sim_event call per event, in order;
      * batched: the events cut into ``n_sub`` sub-batches of consecutive
        events, each a replay of one CUDA graph of the batched sim_event
        (sim.BatchGraphRunner: capacities of the largest sub-batch, event
        offsets and ids in device memory), scheduling shapes autotuned on a
        batch of the first 16 events.
    Reports segments/s of both, every event's completion time from the common
    start (its own call's end, or its sub-batch's replay end: p50 / p99), and
    the plain form's per-event device times.  Inputs are resident on the
    device before the timed region."""
    import torch
    from paper_2212_09807_gb300 import serve, sim, tune
    evs = events.batch_events(cfg, params.BASE["seed"] + 4, n_events, lo, hi)
    sizes = [len(e["x0"]) for e in evs]
    total, big = sum(sizes), max(sizes)
    ids = list(range(1000, 1000 + n_events))
    singles = [sim.Segments.from_numpy(e, i, dev) for e, i in zip(evs, ids)]
    per = -(-n_events // n_sub)
    subs = [(evs[k:k + per], ids[k:k + per]) for k in range(0, n_events, per)]
    sub_segs = [sim.Segments.batch_from_numpy(e, i, dev) for e, i in subs]

    def fitted(cfg_, n, caps, runs, max_events=0):
        """Runner whose capacities fit every event (or batch) of `runs` (untimed sizing pass)."""
        while True:
            r = sim.EventRunner(cfg_, lut, params.LUT["nt"], params.LUT["bins_per_pitch"], n, *caps, device=dev,
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

    # plain: the sizing pass is also the warm-up
    plain = fitted(cfg, big, serve._caps(big), singles)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(n_events + 1)]
    marks[0].record()
    for k, sg in enumerate(singles):
        plain.enqueue(sg)
        marks[k + 1].record()
    torch.cuda.synchronize()
    assert plain.counts()[3] == 0
    t_plain = marks[0].elapsed_time(marks[-1])
    plain_done = [marks[0].elapsed_time(marks[k + 1]) for k in range(n_events)]
    plain_service = [marks[k].elapsed_time(marks[k + 1]) for k in range(n_events)]
    del plain
    torch.cuda.empty_cache()

    # batched: shapes tuned on a sample batch, runner sized on every sub-batch, one graph replayed per sub-batch
    ns = min(16, n_events)
    sample = sim.Segments.batch_from_numpy(evs[:ns], ids[:ns], dev)
    s_tot = sum(sizes[:ns])
    probe = fitted(cfg, s_tot, serve._caps(s_tot), [sample], max_events=ns)
    s_caps = (probe.max_pairs, probe.max_pixels, probe.hits.capacity)
    del probe
    cands = None if int(cfg.get("precision", 0)) == 0 else [
        dict(tc_units_per_sm=u, tc_record_chunk=c) for u in (2, 4) for c in (1 << 19, 1 << 20)]
    chosen, table = tune.autotune(cfg, lut, params.LUT["nt"], params.LUT["bins_per_pitch"], sample, s_caps,
                                  reps=1, device=dev, cands=cands)
    bcfg = dict(cfg, **chosen)
    nmax = max(sg.n for sg in sub_segs)
    runner = fitted(bcfg, nmax, serve._caps(nmax), sub_segs, max_events=per)
    g = sim.BatchGraphRunner(runner)
    for sg in sub_segs[:1]:                       # one untimed replay
        g.load(sg)
        g.replay()
    torch.cuda.synchronize()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(len(sub_segs) + 1)]
    marks[0].record()
    for k, sg in enumerate(sub_segs):
        g.load(sg)
        g.replay()
        marks[k + 1].record()
    torch.cuda.synchronize()
    assert runner.counts()[3] == 0
    t_batch = marks[0].elapsed_time(marks[-1])
    batch_done = []
    for k, (e, _) in enumerate(subs):
        batch_done += [marks[0].elapsed_time(marks[k + 1])] * len(e)
    del g, runner
    torch.cuda.empty_cache()
    pct = lambda v, q: float(np.percentile(v, q))          # noqa: E731
    return {"events": n_events, "segments": total, "sizes": f"log-uniform [{lo:.0f}, {hi:.0f}] segments",
            "arrival": "all events waiting at t = 0; completion times from the common start",
            "plain_segments_per_s": total / (t_plain / 1e3),
            "graph_batched_segments_per_s": total / (t_batch / 1e3),
            "plain_completion_ms": {"p50": pct(plain_done, 50), "p99": pct(plain_done, 99)},
            "batched_completion_ms": {"p50": pct(batch_done, 50), "p99": pct(batch_done, 99)},
            "plain_service_ms": {"p50": pct(plain_service, 50), "p99": pct(plain_service, 99)},
            "subbatches": len(subs), "events_per_subbatch": per,
            "subbatch_ms": [marks[k].elapsed_time(marks[k + 1]) for k in range(len(subs))],
            "total_ms": {"plain": t_plain, "graph_batched": t_batch},
            "tuning": {"sample": f"batch of the first {ns} events", "chosen": chosen,
                       "candidates_ms": [[c, round(ms, 3)] for c, ms in table]}}


FORMS = {0: ("fp32_cells", "f32"), 1: ("bf16_tensor", "bf16"), 2: ("fp16_tensor", "f16"), 3: ("fp32_terms", "f32")}


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
    from paper_2212_09807_gb300 import serve
    caps = list(serve._caps(S))
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


def form_roofline(run, cfg, precision, a4_s, fp32_peak, dev, wl_key=""):
    """Roofline of the induced-current kernel of one form: achieved = the
    algorithmic work 2 flop x nnz(Q) x L (one multiply-add per nonzero
    binned-charge cell and table tick, cells counted on the device) over the
    call's time.  FP32 form: against the measured FP32 FMA rate
    (sim_probe_fma).  Tensor-core forms: against the measured dense 16-bit
    tensor peak; the dense MMA work (zeros inside the issued tiles included)
    is given beside it.  per_point: 2 flop per (point, pixel within the
    table's reach, table tick), the count of the term-by-term sum."""
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
    per_point = w_alg / a4_s / 1e12
    n_mma = int(run.ws[4].item())
    nnz = int(run.ws[5].item())
    useful = 2.0 * nnz * L / a4_s / 1e12
    work_note = ("achieved: 2 flop x nnz(Q) x 1950 table ticks (nonzero binned-charge cells Q[p, node, tick], "
                 "counted on the device); per_point: 2 flop x 9 pixels x 1950 ticks per (point, perturbation)")
    timing = {"duration_ms": a4_s * 1e3,
              "duration_note": "mean CUDA-event time of the sim_induced_current call on its stream over the timed "
                               "steps: the kernel plus the form's small preparation launches, so achieved is a "
                               "lower bound of the kernel's own rate"}
    if precision == 3:                                  # term by term: the per-point count is its work
        return {"bound": "alu", "achieved": per_point, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": per_point / fp32_peak, "traffic": None, "kernel": "k_induced_current_terms",
                "peak_note": "FP32 FMA rate measured on this GPU by sim_probe_fma (independent FMA chains), "
                             "of measured",
                "work_note": "2 flop x 9 pixels x 1950 table ticks per (point, perturbation)", **timing}, samples
    if precision == 0:
        return {"bound": "alu", "achieved": useful, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": useful / fp32_peak, "traffic": stored_traffic("induced_current.cu", wl_key),
                "kernel": "k_induced_current", "nnz_charge_cells": nnz, "per_point_achieved": per_point,
                "peak_note": "FP32 FMA rate measured on this GPU by sim_probe_fma (independent FMA chains), "
                             "of measured",
                "work_note": work_note, **timing}, samples
    dense = 2.0 * 128 * 32 * 16 * n_mma / a4_s / 1e12
    tpk = measured_peaks().get("bf16_tflops_sustained") or 1700.0
    return {"bound": "tensor", "achieved": useful, "peak": tpk, "unit": "TFLOP/s", "frac": useful / tpk,
            "traffic": stored_traffic("induced_current_tc.cu", wl_key), "kernel": "k_induced_current_tc",
            "nnz_charge_cells": nnz, "mma_per_launch": n_mma,
            "dense_achieved": dense, "dense_frac": dense / tpk, "per_point_achieved": per_point,
            "peak_note": "measured dense bf16 sustained (kernel timed inside a step), of measured; fp16 has the "
                         "same nominal rate",
            "work_note": work_note + "; dense: 2 x 128 x 32 x 16 flop per issued MMA", **timing}, samples


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


def timed_event(cfg, seg, lut, dev, precision, steps, warmup, event_id, fp32_peak, wl_key=""):
    """time_form plus the derived per-step numbers and the kernel roofline."""
    run, per, (n_pairs, n_pix, n_hits, _) = time_form(cfg, seg, lut, dev, precision, steps, warmup, event_id)
    S, T = len(seg["x0"]), int(cfg["n_ticks"])
    step_ms = per.sum(axis=1)
    rl, samples = form_roofline(run, dict(cfg, precision=precision), precision, float(per[:, 2].mean()) / 1e3,
                                fp32_peak, dev, wl_key)
    out = {"dtype": FORMS[precision][1], "ms_per_step": float(step_ms.mean()),
           "segments_per_s": S / (float(step_ms.mean()) / 1e3), "induced_current_ms": float(per[:, 2].mean()),
           "roofline": rl}
    info = dict(S=S, T=T, n_pairs=n_pairs, n_pix=n_pix, n_hits=n_hits, samples=samples, step_ms=step_ms)
    return run, per, out, info


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
    fp32_peak = sim.fma_peak_tflops(dev)           # measured FP32 FMA rate, TFLOP/s
    wall = {}                                      # wall seconds of each section (untimed parts included)
    t_sec = time.perf_counter()

    def lap(name):
        nonlocal t_sec
        now = time.perf_counter()
        wall[name] = round(now - t_sec, 1)
        t_sec = now

    # the other forms of the induced-current step, timed on the same event first (untimed for the headline)
    forms = {}
    if not args.no_forms:
        for prec in (0, 1, 2):
            if prec == args.precision:
                continue
            r2, _, out2, _ = timed_event(cfg, seg, lut, dev, prec, args.form_steps, 1, rank, fp32_peak,
                                         desc.split(":")[0])
            forms[FORMS[prec][0]] = dict(out2, steps=args.form_steps, warmup=1)
            del r2
            torch.cuda.empty_cache()
    lap("forms")

    # scheduling shapes of the induced-current step for this event, picked by the autotuner (untimed);
    # results do not depend on them beyond the tensor-core forms' accumulation rounding.  A large event
    # is tuned over a few candidates with one repetition each.
    tuned = None
    if not args.no_tune:
        from paper_2212_09807_gb300 import serve, tune
        segs_dev = sim.Segments.from_numpy(seg, event_id=replica_event_id(rank), device=dev)
        big = S > 200000
        cands = None
        if big and args.precision != 0:
            cands = [dict(tc_units_per_sm=u, tc_record_chunk=c) for u, c in ((1, 1 << 20), (2, 1 << 20), (2, 1 << 18))]
        tuned, _ = tune.autotune(cfg, lut, L, params.LUT["bins_per_pitch"], segs_dev, serve._caps(S, 1.2),
                                 reps=1 if big else 2, device=dev, cands=cands)
        cfg = dict(cfg, **tuned)
        del segs_dev
        torch.cuda.empty_cache()
    lap("tune")

    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    clk = ClockSampler(gpu_id)
    clk.start()
    time.sleep(0.15)
    run, per, head, info = timed_event(cfg, seg, lut, dev, args.precision, args.steps, args.warmup,
                                       replica_event_id(rank), fp32_peak, desc.split(":")[0])
    clocks = clk.stop()
    lap("headline")
    n_pairs, n_pix, n_hits, samples, step_ms = (info[k] for k in ("n_pairs", "n_pix", "n_hits", "samples",
                                                                   "step_ms"))
    total_ms = max_over_ranks(float(step_ms.sum()), pg, dev)
    value = job_rate(world, S * args.steps, total_ms / 1e3)
    a45_ms = max_over_ranks(float(per[:, 2:].sum()), pg, dev)
    pix_ticks = job_rate(world, n_pix * T * args.steps, a45_ms / 1e3)
    roofline = head["roofline"]
    forms[FORMS[args.precision][0]] = dict(head, steps=args.steps, warmup=args.warmup)

    # end to end through the public API: pinned host segments in, hits out
    io = sim.EventIO(run)
    host = {k: torch.as_tensor(np.ascontiguousarray(seg[k], dtype=np.float32)).pin_memory() for k in seg}
    for _ in range(max(1, min(args.warmup, 2))):
        io.simulate(host, S, replica_event_id(rank))
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    e2e_steps = max(2, min(4, args.steps))
    for _ in range(e2e_steps):
        _, _, hb, db = io.simulate(host, S, replica_event_id(rank))
        h2d, d2h = hb, db
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, pg, dev)
    e2e = {"value": job_rate(world, S * e2e_steps, e2e_s), "unit": "segments/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps}
    del run, io
    torch.cuda.empty_cache()
    lap("e2e")

    # the one-module interaction beside the headline, with the steps after the front end on its hits
    module = None
    post = None
    if args.workload != "module":
        mcfg, mseg, mdesc = workload("module")
        mcfg["precision"] = args.precision
        mlut = torch.as_tensor(response.pad_rows(response.lut_for(mcfg, params.LUT)), device=dev)
        mrun, mper, mout, minfo = timed_event(mcfg, mseg, mlut, dev, args.precision, 10, 3, replica_event_id(rank),
                                              fp32_peak, mdesc.split(":")[0])
        module = dict(mout, workload=mdesc, segments=minfo["S"], active_pixels=minfo["n_pix"],
                      hits=minfo["n_hits"], steps=10, warmup=3, scheduling="defaults",
                      step_breakdown_ms={k: float(mper[:, i].mean()) for i, k in
                                         enumerate(("quench_drift", "pixel_map", "induced_current", "electronics"))})
        post = post_hit_steps(mrun, mcfg, dev) if not args.no_post else None
        del mrun
        torch.cuda.empty_cache()
    lap("module_event")
    light_res = light_path(dev) if not args.no_light else None
    torch.cuda.empty_cache()
    lap("light")

    bcfg = params.module_config(precision=args.precision)
    blut = torch.as_tensor(response.pad_rows(response.lut_for(bcfg, params.LUT)), device=dev)
    batched = (batched_vs_plain(bcfg, blut, dev, args.batched_events, 1.0e3, args.batched_hi,
                                args.batched_subbatches) if not args.no_batched else None)
    lap("batched")
    loads = tuple(float(x) for x in args.serving_loads.split(",") if x)
    serving = serving_vs_plain(args.precision, dev, args.serving_requests, loads) if not args.no_serving else None
    lap("serving")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        lut_or = lut_pad[..., :L].astype(np.float64)
        est, threads, sdesc = oracle_sample(cfg, seg, lut_or, np.random.default_rng(0), n_pix=args.cpu_pixels)
        cpu = {"value": S / est, "unit": "segments/s", "cores": threads, "kind": "oracle", "sample": sdesc}
    lap("cpu_baseline")

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
            "fp32_fma_peak_tflops": fp32_peak,
            "forms": forms, "module_event": module, "cpu_baseline": cpu, "e2e": e2e, "batched": batched,
            "serving": serving, "after_front_end": post, "light": light_res,
            "gpu_launches": KERNELS_PER_STEP[args.precision] * args.steps, "clocks": clocks,
            "section_wall_s": wall,
        }))
    if pg:
        pg.destroy_process_group()


def check_ranks(gpus: int, world: int):
    """--gpus N runs as N ranks, one per GPU, started by a launcher that sets
    WORLD_SIZE (torch.distributed.run); a mismatch is an error, not a
    silent single-GPU run."""
    if gpus != world:
        raise SystemExit(f"bench.py --gpus {gpus} needs {gpus} ranks, found WORLD_SIZE={world}: launch it with "
                         f"python -m torch.distributed.run --nnodes=1 --nproc-per-node {gpus} "
                         f"--master-addr 127.0.0.1 --master-port <port> bench.py --gpus {gpus} ...")


def main():
    args = parse()
    check_ranks(args.gpus, dist()[0])
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
