"""Serving form of the charge-readout path: a continuous-batching request loop.

Requests (events of very uneven size: single interactions of ~2e4 segments,
whole beam spills of ~1e6) arrive over time.  A request is admitted as soon
as its device memory fits in the HBM budget beside the requests already on
the GPU; admitted requests run concurrently on their own CUDA streams, so
work that arrives while others are running overlaps with them on the device:

* a request whose active pixels fit one slice runs as one ``sim_event`` on a
  high-priority stream;
* a larger request runs step by step on a low-priority stream, its current
  step cut into slices of ``slice_pixels`` active pixels
  (``sim_induced_current_range``), at most two slices queued at a time, so the
  kernels of requests admitted meanwhile are scheduled between its slices
  instead of behind its whole current step.  Large requests run one at a
  time, in arrival order.

Each request's results are those of the request alone: its random numbers
are keyed by its event id and its own segment indices, and every pixel's
current is computed by one launch in the same summation order whether or not
the step is sliced (bit for bit with the FP32 form; within the stated
tolerance with the tensor-core form, whose pixel groups are formed per slice).

``run_plain`` is the reference form: the same requests, one ``sim_event`` at
a time in arrival order on one stream.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import sim


@dataclasses.dataclass
class Request:
    rid: int
    event_id: int
    seg: dict                       # host FP32 columns (numpy or pinned torch)
    arrival: float = 0.0            # seconds from the start of the run
    kind: str = ""

    @property
    def n(self) -> int:
        return int(len(self.seg["x0"]))


@dataclasses.dataclass
class Result:
    rid: int
    kind: str
    n: int
    arrival: float
    admitted: float
    done: float
    counts: list
    hits: dict
    current: object = None          # numpy [pixels][ticks] when kept

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def _caps(n: int, factor: float = 1.0):
    """Initial (pairs, pixels, hits) capacities of an event of n segments; an
    overflow (reported in the status word) is retried with the sizes it reports."""
    return (int(factor * (30 * n + 10000)), int(factor * (0.8 * n + 10000)), int(factor * (4 * n + 10000)))


class _Job:
    def __init__(self, server, req: Request, caps=None):
        self.s, self.req = server, req
        self.caps = caps or _caps(req.n)
        self.bytes = server.job_bytes(req.n, self.caps)
        self.state = "waiting"
        self.admitted = None
        self.events = []

    # -- device side -------------------------------------------------------
    def start(self, stream, now):
        import torch
        s, n = self.s, self.req.n
        self.stream, self.admitted = stream, now
        with torch.cuda.stream(stream):
            pairs, pixels, hits = self.caps
            self.run = sim.EventRunner(s.cfg_dict, s.lut, s.nt, s.bpp, max(n, 1), pairs, pixels, hits,
                                       device=s.device)
            self.cols = {k: torch.empty(max(n, 1), dtype=torch.float32, device=s.device) for k in sim.Segments.KEYS}
            for k in sim.Segments.KEYS:
                src = self.req.seg[k]
                if not isinstance(src, torch.Tensor):
                    src = torch.as_tensor(np.ascontiguousarray(src, dtype=np.float32)).pin_memory()
                self.cols[k][:n].copy_(src[:n], non_blocking=True)
            self.segs = sim.Segments({k: self.cols[k][:n] for k in sim.Segments.KEYS}, self.req.event_id)
            self.host_counts = torch.zeros(4, dtype=torch.int64).pin_memory()
            self.sliced = s.is_large(n)
            if not self.sliced:
                self.run.enqueue(self.segs, stream)
                self._read_counts("counted")
            else:
                v = self.run.view(n)
                A = sim._alias
                dev = s.device
                self.dr = sim.Drifted.wrap(v.dr)
                self.act = A(v.active_pixels, self.run.max_pixels, torch.int32, dev)
                self.off = A(v.pix_seg_off, self.run.max_pixels + 1, torch.int32, dev)
                self.ids = A(v.pix_seg_ids, self.run.max_pairs, torch.int32, dev)
                self.cur = A(v.current, self.run.max_pixels * s.T, torch.float32, dev).view(self.run.max_pixels, s.T)
                sim.sim_quench_drift(self.run.cfg, self.segs, self.dr, stream)
                sim.sim_pixel_map(self.run.cfg, self.segs, self.dr, self.run.resp,
                                  A(v.seg_pix_off, n + 1, torch.int32, dev),
                                  A(v.seg_pix_ids, self.run.max_pairs, torch.int32, dev), self.act, self.off,
                                  self.ids, self.run.ws, stream)
                self._read_counts("mapped")

    def _read_counts(self, next_state):
        import torch
        with torch.cuda.stream(self.stream):
            self.host_counts.copy_(self.run.ws[:4], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.events = [ev]
        self.state = next_state

    def _slice(self, b, e):
        import torch
        sim.sim_induced_current_range(self.run.cfg, self.segs, self.dr, self.run.resp, self.act, self.off, self.ids,
                                      self.run.ws[:4], b, e, self.cur, self.run.ws, self.stream)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self.events.append(ev)

    def step(self, now):
        """Advances the job's state machine; returns True when it finished."""
        import torch
        if any(not ev.query() for ev in self.events[:1]):
            return False
        if self.state == "mapped":
            counts = [int(x) for x in self.host_counts.tolist()]
            if counts[3] != 0:
                return self._overflow(counts)
            self.npix = counts[1]
            self.next_b = 0
            self.events = []
            self.state = "slicing"
        if self.state == "slicing":
            self.events = [ev for ev in self.events if not ev.query()]
            while len(self.events) < 2 and self.next_b < self.npix:
                e = min(self.npix, self.next_b + self.s.slice_pixels)
                self._slice(self.next_b, e)
                self.next_b = e
            if self.next_b < self.npix or self.events:
                return False
            with torch.cuda.stream(self.stream):
                sim.sim_electronics(self.run.cfg, self.segs, self.act, self.cur, self.run.ws[:4], self.run.hits,
                                    self.run.ws, self.stream)
            self._read_counts("counted")
            return False
        if self.state == "counted":
            counts = [int(x) for x in self.host_counts.tolist()]
            if counts[3] != 0:
                return self._overflow(counts)
            self.counts = counts
            nh = min(counts[2], self.run.hits.capacity)
            with torch.cuda.stream(self.stream):
                self.host_hits = {}
                for k in ("pixel", "t_cross", "t_adc", "adc", "q"):
                    src = getattr(self.run.hits, k)[:nh]
                    dst = torch.empty(max(nh, 1), dtype=src.dtype).pin_memory()[:nh]
                    dst.copy_(src, non_blocking=True)
                    self.host_hits[k] = dst
                if self.s.keep_current:
                    cur = self.run.current(self.req.n, counts[1])
                    self.host_cur = torch.empty(cur.shape, dtype=cur.dtype).pin_memory()
                    self.host_cur.copy_(cur, non_blocking=True)
                    act = self.run.active_pixels(self.req.n, counts[1])
                    self.host_act = torch.empty(act.shape, dtype=act.dtype).pin_memory()
                    self.host_act.copy_(act, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.stream)
            self.events = [ev]
            self.state = "reading"
            return False
        if self.state == "reading":
            self.result = Result(self.req.rid, self.req.kind, self.req.n, self.req.arrival, self.admitted, now,
                                 self.counts, {k: v.numpy().copy() for k, v in self.host_hits.items()})
            if self.s.keep_current:
                self.result.current = self.host_cur.numpy().copy()
                self.result.active = self.host_act.numpy().copy()
            self.state = "done"
            self.free()
            return True
        return False

    def _overflow(self, counts):
        """Capacity overflow: restart with the sizes the device reported."""
        pairs, pixels, hits = self.caps
        self.caps = (max(pairs, 2 * counts[0]), max(pixels, 2 * counts[1]), max(hits, 2 * counts[2]))
        stream, adm = self.stream, self.admitted
        self.free()
        self.s.used += self.s.job_bytes(self.req.n, self.caps) - self.bytes
        self.bytes = self.s.job_bytes(self.req.n, self.caps)
        self.start(stream, adm)
        return False

    def free(self):
        for k in ("run", "cols", "segs", "dr", "act", "off", "ids", "cur"):
            if hasattr(self, k):
                delattr(self, k)


def admission(waiting: list, n_running: int, large_running: bool, used: float, budget: float, max_jobs: int,
              is_large, nbytes) -> list:
    """The requests of `waiting` (in arrival order) to start in this turn of
    the loop: first fit in arrival order within the HBM budget (`used` bytes
    held, `nbytes(job)` more for each) and the job limit; a request that fits
    no budget starts when nothing else is on the GPU.  Large requests
    (`is_large(job)`) run one at a time and in arrival order: none starts
    while one runs, and one that waits (for the budget) holds back the large
    requests behind it.  Small requests may pass waiting ones."""
    start = []
    hold_large = large_running
    for job in waiting:
        on_gpu = n_running + len(start)
        if on_gpu >= max_jobs:
            break
        large = bool(is_large(job))
        if large and hold_large:
            continue
        b = float(nbytes(job))
        if used + b > budget and on_gpu > 0:
            hold_large = hold_large or large
            continue
        start.append(job)
        used += b
        hold_large = hold_large or large
    return start


class Server:
    """Continuous-batching request loop over one GPU (see the module docstring).

    hbm_budget: bytes of device memory the admitted requests may hold together.
    slice_pixels: active pixels per current launch of a large request.
    max_jobs: requests on the GPU at once."""

    def __init__(self, cfg: dict, lut_padded, lut_nt: int, bins_per_pitch: int, hbm_budget: float = 120e9,
                 slice_pixels: int = 16384, max_jobs: int = 8, keep_current: bool = False, device="cuda"):
        import torch
        self.cfg_dict, self.lut, self.nt, self.bpp = cfg, lut_padded, lut_nt, bins_per_pitch
        self.cfg = sim.make_config(cfg)
        self.T = int(cfg["n_ticks"])
        self.budget, self.slice_pixels, self.max_jobs = float(hbm_budget), int(slice_pixels), int(max_jobs)
        self.keep_current = keep_current
        self.device = torch.device(device)
        self.hi = [torch.cuda.Stream(device=self.device, priority=-1) for _ in range(max_jobs)]
        self.lo = [torch.cuda.Stream(device=self.device, priority=0) for _ in range(max_jobs)]
        self.used = 0.0

    def is_large(self, n: int) -> bool:
        """Runs step by step with a sliced current step: more active pixels
        expected (about one per two segments) than one slice."""
        return 0.5 * n > self.slice_pixels

    def job_bytes(self, n, caps):
        pairs, pixels, hits = caps
        return (sim.workspace_size(self.cfg, max(n, 1), pairs, pixels) + 36 * max(n, 1) + 17 * hits)

    def run(self, requests: list, poll_s: float = 2e-4) -> list:
        """Serves `requests` (sorted by arrival time, seconds from now); returns
        their Results in completion order."""
        import torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        waiting, running, results = [], [], []
        nxt = 0
        free_hi, free_lo = list(self.hi), list(self.lo)
        t0 = time.perf_counter()
        while nxt < len(reqs) or waiting or running:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                waiting.append(_Job(self, reqs[nxt]))
                nxt += 1
            # admission (see `admission`; two large requests sharing the GPU would both finish late)
            large_running = any(self.is_large(j.req.n) for j in running)
            for job in admission(waiting, len(running), large_running, self.used, self.budget, self.max_jobs,
                                 lambda j: self.is_large(j.req.n), lambda j: j.bytes):
                pool = free_lo if self.is_large(job.req.n) else free_hi
                stream = pool.pop()
                job.pool = pool
                self.used += job.bytes
                job.start(stream, now)
                waiting.remove(job)
                running.append(job)
            progressed = False
            for job in list(running):
                if job.step(time.perf_counter() - t0):
                    running.remove(job)
                    job.pool.append(job.stream)
                    self.used -= job.bytes
                    results.append(job.result)
                    progressed = True
            if not progressed:
                if not running and waiting == [] and nxt < len(reqs):
                    time.sleep(max(0.0, min(reqs[nxt].arrival - now, 0.01)))
                else:
                    time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        return results


def run_plain(cfg: dict, lut_padded, lut_nt: int, bins_per_pitch: int, requests: list, keep_current=False,
              device="cuda") -> list:
    """Reference form: one ``sim_event`` per request, whole, in arrival order,
    on one stream (a request waits for every earlier one)."""
    import torch
    reqs = sorted(requests, key=lambda r: r.arrival)
    results = []
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        adm = time.perf_counter() - t0
        caps = _caps(r.n)
        while True:
            run = sim.EventRunner(cfg, lut_padded, lut_nt, bins_per_pitch, max(r.n, 1), *caps, device=device)
            io = sim.EventIO(run)
            host = {k: (r.seg[k] if isinstance(r.seg[k], torch.Tensor)
                        else torch.as_tensor(np.ascontiguousarray(r.seg[k], dtype=np.float32)).pin_memory())
                    for k in sim.Segments.KEYS}
            hits, counts, _, _ = io.simulate(host, r.n, r.event_id)
            if counts[3] == 0:
                break
            caps = (max(caps[0], 2 * counts[0]), max(caps[1], 2 * counts[1]), max(caps[2], 2 * counts[2]))
            del run, io
        res = Result(r.rid, r.kind, r.n, r.arrival, adm, time.perf_counter() - t0, counts,
                     {k: v.numpy().copy() for k, v in hits.items()})
        if keep_current:
            res.current = run.current(r.n, counts[1]).cpu().numpy().copy()
            res.active = run.active_pixels(r.n, counts[1]).cpu().numpy().copy()
        results.append(res)
        del run, io
    return results


def percentile_spread(lat, q: float, n_boot: int = 2000, seed: int = 0):
    """[5 %, 95 %] interval of the q-th percentile of ``lat`` over bootstrap
    resamples of the requests (the spread of a percentile of a finite stream)."""
    lat = np.asarray(lat, dtype=np.float64)
    rng = np.random.default_rng(seed)
    qs = np.percentile(lat[rng.integers(0, len(lat), (n_boot, len(lat)))], q, axis=1)
    return [float(np.percentile(qs, 5)), float(np.percentile(qs, 95))]


def summarize(results: list, t_first: float = 0.0) -> dict:
    """p50/p99 latency (ms) overall (with the bootstrap spread of each) and per
    kind; sustained segments/s."""
    lat = np.array([r.latency for r in results]) * 1e3
    out = {"requests": len(results), "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                                     "p99": float(np.percentile(lat, 99)),
                                                     "p50_spread": percentile_spread(lat, 50),
                                                     "p99_spread": percentile_spread(lat, 99)}}
    for kind in sorted({r.kind for r in results}):
        lk = np.array([r.latency for r in results if r.kind == kind]) * 1e3
        out[f"latency_ms_{kind}"] = {"p50": float(np.percentile(lk, 50)), "p99": float(np.percentile(lk, 99)),
                                     "n": int(len(lk))}
    span = max(r.done for r in results) - min(min(r.arrival for r in results), t_first)
    out["segments_per_s"] = float(sum(r.n for r in results) / span)
    return out
