"""Python binding of the C ABI in include/sim.h (argument marshalling only).

Torch provides device memory and streams; every step of the simulation runs
in the sm_103a kernels of ``libsim.so``.  The functions keep the C names
(``sim_quench_drift``, ``sim_pixel_map``, ``sim_induced_current``,
``sim_electronics``, ``sim_event``) and take torch CUDA tensors.  If the
library has not been built, :func:`lib` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsim.so")

SIM_OK = 0
SIM_STATUS_PAIR_OVERFLOW = 1
SIM_STATUS_PIXEL_OVERFLOW = 2
SIM_STATUS_HIT_OVERFLOW = 4
SIM_STATUS_TICK_RANGE = 8
SIM_STATUS_TIMEOUT = 16
ANCHOR_BYTES = 64

_lib = None


class SimError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().sim_strerror(code).decode()
        if code == -3:
            msg += f" (cudaError {lib().sim_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{code}]")
        self.code = code


class SimConfig(C.Structure):
    _fields_ = [
        ("n_mod_x", C.c_int32), ("n_mod_y", C.c_int32), ("n_tpc", C.c_int32),
        ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("px_per_tile", C.c_int32),
        ("pitch_cm", C.c_float), ("drift_len_cm", C.c_float),
        ("recomb_model", C.c_int32),
        ("birks_Ab", C.c_float), ("birks_kb", C.c_float), ("box_alpha", C.c_float),
        ("box_beta", C.c_float), ("efield_kV_cm", C.c_float), ("lar_density_g_cm3", C.c_float),
        ("w_ion_MeV", C.c_float),
        ("vdrift_cm_us", C.c_float), ("lifetime_us", C.c_float), ("diff_long_cm2_s", C.c_float),
        ("diff_tran_cm2_s", C.c_float),
        ("sample_step_cm", C.c_float), ("mc_per_sample", C.c_int32), ("diff_clip_sigma", C.c_float),
        ("tick_us", C.c_float), ("n_ticks", C.c_int32), ("t_window0_us", C.c_float),
        ("thr_e", C.c_float), ("sigma_reset_e", C.c_float), ("sigma_disc_e", C.c_float),
        ("sigma_unc_e", C.c_float), ("gain_e_per_mV", C.c_float), ("adc_lsb_mV", C.c_float),
        ("hold_ticks", C.c_int32), ("min_adc_interval_ticks", C.c_int32),
        ("periodic_reset_ticks", C.c_int32), ("adc_bits", C.c_int32),
        ("seed", C.c_uint64),
        ("precision", C.c_int32), ("fp64_charge", C.c_int32), ("disabled_pixels", C.c_void_p),
        ("per_point_drift", C.c_int32), ("nearest_lut", C.c_int32),
        ("tc_units_per_sm", C.c_int32), ("tc_record_chunk", C.c_int32), ("direct_ctas_per_sm", C.c_int32),
        ("wait_spin_limit", C.c_int32),
    ]


_P = C.c_void_p


class SimSegments(C.Structure):
    _fields_ = [(k, _P) for k in ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")] + [
        ("n", C.c_int64), ("event_id", C.c_uint64), ("event_offsets", _P), ("event_ids", _P),
        ("n_events", C.c_int64)]


class SimResponse(C.Structure):
    _fields_ = [("lut", _P), ("nb", C.c_int32), ("nt", C.c_int32), ("ld", C.c_int32),
                ("bins_per_pitch", C.c_int32)]


class SimDrifted(C.Structure):
    _fields_ = [(k, _P) for k in ("Qa", "t_drift", "sigma_T", "sigma_L", "anode", "n_samples", "anchors")]


class SimHits(C.Structure):
    _fields_ = [(k, _P) for k in ("pixel", "t_cross", "t_adc", "adc", "q")] + [
        ("capacity", C.c_int64), ("n_out", _P)]


class SimTruth(C.Structure):
    _fields_ = [("k", C.c_int32), ("segment", _P), ("q", _P), ("q_signal", _P), ("tick_first", _P),
                ("capacity", C.c_int64)]


class SimLightConfig(C.Structure):
    _fields_ = [(k, _P) for k in ("vis", "tdist", "eff", "gain", "resp", "noise_amp")] + \
               [(k, C.c_int32) for k in ("nvx", "nvy", "nvz", "n_det", "nt", "n_resp", "noise_block", "adc_bits")] + \
               [("vox_cm", C.c_float), ("w_ph_MeV", C.c_float), ("tick_us", C.c_float), ("t_start_us", C.c_float),
                ("n_ticks", C.c_int32), ("pad0", C.c_int32)] + \
               [(k, C.c_float) for k in ("fast_frac", "tau_fast_us", "tau_slow_us", "trunc_taus", "poisson_max_mean",
                                         "sample_us", "pedestal_adc")]


class SimEventView(C.Structure):
    _fields_ = [("dr", SimDrifted)] + [(k, _P) for k in (
        "seg_pix_off", "seg_pix_ids", "active_pixels", "pix_seg_off", "pix_seg_ids", "current", "counts")]


def lib():
    """The compiled library; raises when it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        cp = C.POINTER
        L.sim_strerror.restype = C.c_char_p
        L.sim_strerror.argtypes = [C.c_int]
        L.sim_last_cuda_error.restype = C.c_int
        L.sim_abi_sizes.argtypes = [cp(C.c_int64)]
        L.sim_workspace_size.argtypes = [cp(SimConfig), C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                         cp(C.c_size_t)]
        L.sim_workspace_counts.restype = C.c_void_p
        L.sim_workspace_counts.argtypes = [_P]
        L.sim_quench_drift.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimDrifted), _P]
        L.sim_pixel_map.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimDrifted), cp(SimResponse),
                                    _P, _P, C.c_int64, _P, _P, _P, C.c_int64, _P, C.c_size_t, _P]
        L.sim_induced_current.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimDrifted), cp(SimResponse),
                                          _P, _P, _P, _P, C.c_int64, _P, _P, C.c_size_t, _P]
        L.sim_induced_current_range.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimDrifted), cp(SimResponse),
                                                _P, _P, _P, _P, C.c_int64, C.c_int64, C.c_int64, _P, _P,
                                                C.c_size_t, _P]
        L.sim_electronics.argtypes = [cp(SimConfig), cp(SimSegments), _P, _P, _P, C.c_int64, cp(SimHits),
                                      _P, C.c_size_t, _P]
        L.sim_event.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimResponse), C.c_int64, C.c_int64,
                                cp(SimHits), _P, C.c_size_t, _P]
        L.sim_event_view_of.argtypes = [cp(SimConfig), C.c_int64, C.c_int64, C.c_int64, C.c_int64, _P,
                                        C.c_size_t, cp(SimEventView)]
        L.sim_probe_fma.argtypes = [C.c_int64, C.c_int32, _P, cp(C.c_double), _P]
        L.sim_pixel_map_noalloc.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimDrifted), cp(SimResponse),
                                            _P, _P, C.c_int64, _P, _P, _P, C.c_int64, _P, _P]
        L.sim_response_cumulative.argtypes = [cp(SimResponse), _P, _P]
        L.sim_hit_truth_workspace_size.argtypes = [C.c_int64, C.c_int64, cp(C.c_size_t)]
        L.sim_hit_truth.argtypes = [cp(SimConfig), cp(SimSegments), cp(SimDrifted), cp(SimResponse), _P, _P, _P,
                                    _P, _P, C.c_int64, cp(SimHits), cp(SimTruth), C.c_int64, _P, C.c_size_t, _P]
        L.sim_hit_points.argtypes = [cp(SimConfig), cp(SimHits), _P, _P, _P, _P, _P]
        L.sim_track_dqdx.argtypes = [_P, _P, _P, _P, _P, C.c_int64, cp(C.c_double), cp(C.c_double), C.c_double,
                                     C.c_int32, C.c_double, _P, _P, _P]
        L.sim_light_n_samples.argtypes = [cp(SimLightConfig), cp(C.c_int64)]
        L.sim_light_yield.argtypes = [cp(SimConfig), cp(SimLightConfig), cp(SimSegments), cp(SimDrifted), _P, _P, _P,
                                      _P]
        L.sim_light_photocurrent.argtypes = [cp(SimConfig), cp(SimLightConfig), cp(SimSegments), cp(SimDrifted), _P,
                                             _P, _P, _P, _P]
        L.sim_light_scintillation.argtypes = [cp(SimConfig), cp(SimLightConfig), _P, _P, _P]
        L.sim_light_fluctuate.argtypes = [cp(SimConfig), cp(SimLightConfig), C.c_uint64, _P, _P, _P]
        L.sim_light_electronics.argtypes = [cp(SimConfig), cp(SimLightConfig), C.c_uint64, _P, _P, _P, _P]
        L.sim_light_truth.argtypes = [cp(SimConfig), cp(SimLightConfig), C.c_int64, _P, _P, _P, _P]
        L.sim_light_workspace_size.argtypes = [cp(SimConfig), cp(SimLightConfig), C.c_int64, cp(C.c_size_t)]
        L.sim_light_event.argtypes = [cp(SimConfig), cp(SimLightConfig), cp(SimSegments), cp(SimDrifted), _P, _P,
                                      C.c_size_t, _P]
        for f in ("sim_light_n_samples", "sim_light_yield", "sim_light_photocurrent", "sim_light_scintillation",
                  "sim_light_fluctuate", "sim_light_electronics", "sim_light_workspace_size", "sim_light_event",
                  "sim_light_truth"):
            getattr(L, f).restype = C.c_int
        for f in ("sim_workspace_size", "sim_quench_drift", "sim_pixel_map", "sim_induced_current",
                  "sim_induced_current_range", "sim_electronics", "sim_event", "sim_event_view_of",
                  "sim_pixel_map_noalloc", "sim_probe_fma", "sim_response_cumulative", "sim_hit_truth_workspace_size", "sim_hit_truth", "sim_hit_points",
                  "sim_track_dqdx"):
            getattr(L, f).restype = C.c_int
        sizes = (C.c_int64 * 5)()
        L.sim_abi_sizes(sizes)
        exp = [C.sizeof(SimConfig), C.sizeof(SimSegments), C.sizeof(SimResponse), C.sizeof(SimDrifted),
               C.sizeof(SimHits)]
        if list(sizes) != exp:
            raise RuntimeError(f"ABI struct size mismatch: library {list(sizes)} vs binding {exp}")
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != SIM_OK:
        raise SimError(code, where)


def make_config(cfg: dict) -> SimConfig:
    """sim_config from a parameter dict (floats rounded to FP32 by ctypes)."""
    c = SimConfig()
    for name, ct in SimConfig._fields_:
        if name == "disabled_pixels":       # optional CUDA tensor (int32/uint32 words) or None
            m = cfg.get(name)
            c.disabled_pixels = None if m is None else int(m.data_ptr())
            continue
        v = cfg.get(name, 0) if name in ("precision", "fp64_charge", "per_point_drift", "nearest_lut", "tc_units_per_sm",
                                         "tc_record_chunk", "direct_ctas_per_sm", "wait_spin_limit") else cfg[name]
        setattr(c, name, int(v) & 0xFFFFFFFFFFFFFFFF if name == "seed" else (float(v) if ct is C.c_float else int(v)))
    return c


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Segments:
    """Segment columns as FP32 CUDA tensors (x0, y0, z0, t0, x1, y1, z1, t1, dE).

    One event (``event_id``) or, with ``offsets`` (int64 [n_events + 1]) and
    ``ids`` (uint64 as int64 [n_events]) CUDA tensors, a batch of events."""

    KEYS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")

    def __init__(self, cols: dict, event_id: int = 0, offsets=None, ids=None):
        self.cols = cols
        self.n = int(cols["x0"].numel())
        self.event_id = int(event_id)
        self.offsets, self.ids = offsets, ids
        self.n_events = 0 if offsets is None else int(offsets.numel()) - 1

    @classmethod
    def from_numpy(cls, seg: dict, event_id: int = 0, device="cuda"):
        import torch
        return cls({k: torch.as_tensor(np.ascontiguousarray(seg[k], dtype=np.float32), device=device)
                    for k in cls.KEYS}, event_id)

    @classmethod
    def batch_from_numpy(cls, events: list, event_ids: list, device="cuda"):
        """Concatenate per-event segment dicts into one batch."""
        import torch
        cols = {k: torch.as_tensor(np.ascontiguousarray(np.concatenate([e[k] for e in events]), dtype=np.float32),
                                   device=device) for k in cls.KEYS}
        off = np.zeros(len(events) + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(e["x0"]) for e in events])
        ids = np.asarray([int(i) for i in event_ids], dtype=np.uint64).view(np.int64)
        return cls(cols, 0, torch.as_tensor(off, device=device), torch.as_tensor(ids, device=device))

    def struct(self) -> SimSegments:
        s = SimSegments()
        for k in self.KEYS:
            setattr(s, k, _ptr(self.cols[k]))
        s.n = self.n
        s.event_id = self.event_id
        s.event_offsets = _ptr(self.offsets)
        s.event_ids = _ptr(self.ids)
        s.n_events = self.n_events
        return s


class Response:
    """Response table as a CUDA FP32 tensor [nb][nb][ld]."""

    def __init__(self, lut_padded, nt: int, bins_per_pitch: int):
        self.t = lut_padded
        self.nb = int(lut_padded.shape[0])
        self.ld = int(lut_padded.shape[2])
        self.nt = int(nt)
        self.bpp = int(bins_per_pitch)

    def struct(self) -> SimResponse:
        r = SimResponse()
        r.lut = _ptr(self.t)
        r.nb, r.nt, r.ld, r.bins_per_pitch = self.nb, self.nt, self.ld, self.bpp
        return r


class Drifted:
    """Outputs of sim_quench_drift."""

    def __init__(self, n: int, device="cuda"):
        import torch
        f = dict(dtype=torch.float32, device=device)
        i = dict(dtype=torch.int32, device=device)
        m = max(n, 1)                      # never a null pointer, even for an empty event
        self.Qa, self.t_drift = torch.empty(m, **f)[:n], torch.empty(m, **f)[:n]
        self.sigma_T, self.sigma_L = torch.empty(m, **f)[:n], torch.empty(m, **f)[:n]
        self.anode, self.n_samples = torch.empty(m, **i)[:n], torch.empty(m, **i)[:n]
        self.anchors = torch.empty(m * ANCHOR_BYTES // 4, **f)

    @classmethod
    def wrap(cls, sd: SimDrifted):
        d = cls.__new__(cls)
        d._s = sd
        return d

    def struct(self) -> SimDrifted:
        if hasattr(self, "_s"):
            return self._s
        d = SimDrifted()
        for k in ("Qa", "t_drift", "sigma_T", "sigma_L", "anode", "n_samples", "anchors"):
            setattr(d, k, _ptr(getattr(self, k)))
        return d


class Hits:
    """Hit list buffers of a given capacity."""

    def __init__(self, capacity: int, device="cuda"):
        import torch
        self.capacity = int(capacity)
        n = max(self.capacity, 1)
        self.pixel = torch.empty(n, dtype=torch.int32, device=device)
        self.t_cross = torch.empty(n, dtype=torch.int32, device=device)
        self.t_adc = torch.empty(n, dtype=torch.int32, device=device)
        self.adc = torch.empty(n, dtype=torch.uint8, device=device)
        self.q = torch.empty(n, dtype=torch.float32, device=device)
        self.n_out = torch.zeros(1, dtype=torch.int64, device=device)

    def struct(self) -> SimHits:
        h = SimHits()
        for k in ("pixel", "t_cross", "t_adc", "adc", "q"):
            setattr(h, k, _ptr(getattr(self, k)))
        h.capacity = self.capacity
        h.n_out = _ptr(self.n_out)
        return h

    def to_numpy(self, n: int) -> dict:
        return {k: getattr(self, k)[:n].cpu().numpy() for k in ("pixel", "t_cross", "t_adc", "adc", "q")}


def workspace_size(cfg: SimConfig, max_segments: int, max_pairs: int, max_pixels: int, max_events: int = 0) -> int:
    b = C.c_size_t()
    _check(lib().sim_workspace_size(C.byref(cfg), max_events, max_segments, max_pairs, max_pixels, C.byref(b)),
           "sim_workspace_size")
    return int(b.value)


# ------------------------------------------------------------ C entry points --

def sim_quench_drift(cfg: SimConfig, seg: Segments, out: Drifted, stream=None):
    s, d = seg.struct(), out.struct()
    _check(lib().sim_quench_drift(C.byref(cfg), C.byref(s), C.byref(d), _stream(stream)), "sim_quench_drift")


def sim_pixel_map(cfg: SimConfig, seg: Segments, dr: Drifted, resp: Response, seg_pix_off, seg_pix_ids,
                  active_pixels, pix_seg_off, pix_seg_ids, ws, stream=None):
    s, d, r = seg.struct(), dr.struct(), resp.struct()
    _check(lib().sim_pixel_map(C.byref(cfg), C.byref(s), C.byref(d), C.byref(r), _ptr(seg_pix_off),
                               _ptr(seg_pix_ids), int(seg_pix_ids.numel()), _ptr(active_pixels),
                               _ptr(pix_seg_off), _ptr(pix_seg_ids), int(active_pixels.numel()),
                               _ptr(ws), int(ws.numel() * ws.element_size()), _stream(stream)),
           "sim_pixel_map")


def sim_pixel_map_noalloc(cfg: SimConfig, seg: Segments, dr: Drifted, resp: Response, seg_pix_off, seg_pix_ids,
                          active_pixels, pix_seg_off, pix_seg_ids, counts, stream=None):
    """sim_pixel_map without a workspace: for callers that cannot allocate
    device memory when they map an event (scratch lives in the library)."""
    s, d, r = seg.struct(), dr.struct(), resp.struct()
    _check(lib().sim_pixel_map_noalloc(C.byref(cfg), C.byref(s), C.byref(d), C.byref(r), _ptr(seg_pix_off),
                                       _ptr(seg_pix_ids), int(seg_pix_ids.numel()), _ptr(active_pixels),
                                       _ptr(pix_seg_off), _ptr(pix_seg_ids), int(active_pixels.numel()),
                                       _ptr(counts), _stream(stream)), "sim_pixel_map_noalloc")


def sim_induced_current(cfg: SimConfig, seg: Segments, dr: Drifted, resp: Response, active_pixels,
                        pix_seg_off, pix_seg_ids, counts, current, ws, stream=None):
    s, d, r = seg.struct(), dr.struct(), resp.struct()
    pix_cap = int(current.shape[0])
    _check(lib().sim_induced_current(C.byref(cfg), C.byref(s), C.byref(d), C.byref(r), _ptr(active_pixels),
                                     _ptr(pix_seg_off), _ptr(pix_seg_ids), _ptr(counts), pix_cap,
                                     _ptr(current), _ptr(ws), int(ws.numel() * ws.element_size()),
                                     _stream(stream)), "sim_induced_current")


def sim_induced_current_range(cfg: SimConfig, seg: Segments, dr: Drifted, resp: Response, active_pixels,
                              pix_seg_off, pix_seg_ids, counts, pix_begin: int, pix_end: int, current, ws,
                              stream=None):
    s, d, r = seg.struct(), dr.struct(), resp.struct()
    pix_cap = int(current.shape[0])
    _check(lib().sim_induced_current_range(C.byref(cfg), C.byref(s), C.byref(d), C.byref(r), _ptr(active_pixels),
                                           _ptr(pix_seg_off), _ptr(pix_seg_ids), _ptr(counts), int(pix_begin),
                                           int(pix_end), pix_cap, _ptr(current), _ptr(ws),
                                           int(ws.numel() * ws.element_size()), _stream(stream)),
           "sim_induced_current_range")


def sim_electronics(cfg: SimConfig, events, active_pixels, current, counts, hits: Hits, ws, stream=None):
    """``events``: the Segments (or a plain event id) whose event ids key the noise."""
    h = hits.struct()
    ev = events.struct() if isinstance(events, Segments) else SimSegments(n=0, event_id=int(events))
    pix_cap = int(current.shape[0])
    _check(lib().sim_electronics(C.byref(cfg), C.byref(ev), _ptr(active_pixels), _ptr(current), _ptr(counts),
                                 pix_cap, C.byref(h), _ptr(ws), int(ws.numel() * ws.element_size()),
                                 _stream(stream)), "sim_electronics")


def sim_event(cfg: SimConfig, seg: Segments, resp: Response, max_pairs: int, max_pixels: int, hits: Hits, ws,
              stream=None):
    s, r, h = seg.struct(), resp.struct(), hits.struct()
    _check(lib().sim_event(C.byref(cfg), C.byref(s), C.byref(r), int(max_pairs), int(max_pixels), C.byref(h),
                           _ptr(ws), int(ws.numel() * ws.element_size()), _stream(stream)), "sim_event")


def fma_peak_tflops(device=None, iters: int = 16384, reps: int = 7) -> float:
    """Measured FP32 FMA rate of the device (TFLOP/s): the median of `reps`
    timed launches (~16 ms each) of sim_probe_fma with 8 CTAs of 256 threads
    per SM, after one untimed launch."""
    import torch
    dev = torch.device("cuda") if device is None else torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * sms
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    flops = C.c_double()
    times = []
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(lib().sim_probe_fma(blocks, iters, _ptr(sink), C.byref(flops), _stream(None)), "sim_probe_fma")
        e1.record()
        torch.cuda.synchronize()
        if r > 0:                                  # the first launch warms up
            times.append(e0.elapsed_time(e1))
    return flops.value / (float(np.median(times)) / 1e3) / 1e12


def sim_response_cumulative(resp: Response, stream=None):
    """Running sums of the table rows as corner quads ([nb][nb][ld][4]), for sim_hit_truth."""
    import torch
    cum = torch.zeros(*resp.t.shape, 4, dtype=torch.float32, device=resp.t.device)
    r = resp.struct()
    _check(lib().sim_response_cumulative(C.byref(r), _ptr(cum), _stream(stream)), "sim_response_cumulative")
    return cum


class Truth:
    """Per-hit charge truth buffers (k entries per hit) and the call's workspace.

    ``max_cells`` bounds the sum over hit pixels of hits x mapped segments;
    :func:`sim_hit_truth` grows it (and retries) when the device reports more."""

    def __init__(self, capacity: int, k: int = 5, max_cells: int = 1 << 20, device="cuda"):
        import torch
        self.capacity, self.k = int(capacity), int(k)
        self.device = device
        n = max(self.capacity, 1)
        self.segment = torch.empty(n * self.k, dtype=torch.int32, device=device)
        self.q = torch.empty(n * self.k, dtype=torch.float32, device=device)
        self.q_signal = torch.empty(n, dtype=torch.float32, device=device)
        self.tick_first = torch.empty(n, dtype=torch.int32, device=device)
        self.reserve(max_cells)

    def reserve(self, max_cells: int):
        import torch
        self.max_cells = int(max_cells)
        b = C.c_size_t()
        _check(lib().sim_hit_truth_workspace_size(self.capacity, self.max_cells, C.byref(b)),
               "sim_hit_truth_workspace_size")
        self.ws = torch.empty((int(b.value) + 7) // 8, dtype=torch.int64, device=self.device)

    def counts(self):
        """(cells needed, runs, units, status) of the last call, after the stream has run."""
        return [int(x) for x in self.ws[:4].cpu().tolist()]

    def to_numpy(self, n_hits: int) -> dict:
        """segment [n, k], q [n, k], q_signal [n], tick_first [n] and the fraction
        of each listed segment in its hit's signal (q / q_signal; 0 where the
        signal is 0) for the first n_hits hits."""
        n = int(n_hits)
        seg = self.segment[: n * self.k].cpu().numpy().reshape(n, self.k)
        q = self.q[: n * self.k].cpu().numpy().reshape(n, self.k)
        sig = self.q_signal[:n].cpu().numpy()
        with np.errstate(divide="ignore", invalid="ignore"):
            frac = np.where(sig[:, None] != 0, q / sig[:, None], 0.0)
        return dict(segment=seg, q=q, q_signal=sig, tick_first=self.tick_first[:n].cpu().numpy(), fraction=frac)

    def struct(self) -> SimTruth:
        t = SimTruth()
        t.k, t.capacity = self.k, self.capacity
        t.segment, t.q, t.q_signal, t.tick_first = (_ptr(self.segment), _ptr(self.q), _ptr(self.q_signal),
                                                    _ptr(self.tick_first))
        return t


def sim_hit_truth(cfg: SimConfig, seg: Segments, dr: Drifted, resp: Response, cum, active_pixels, pix_seg_off,
                  pix_seg_ids, counts, pix_cap: int, hits: Hits, out: Truth, stream=None, retry: bool = True):
    """Enqueues the truth step; with ``retry`` it synchronises, and re-runs with a
    larger cell capacity when the device reports more cells than ``out.max_cells``."""
    import torch
    s, d, r, h, t = seg.struct(), dr.struct(), resp.struct(), hits.struct(), out.struct()
    for _ in range(2):
        _check(lib().sim_hit_truth(C.byref(cfg), C.byref(s), C.byref(d), C.byref(r), _ptr(cum),
                                   _ptr(active_pixels), _ptr(pix_seg_off), _ptr(pix_seg_ids), _ptr(counts),
                                   int(pix_cap), C.byref(h), C.byref(t), out.max_cells, _ptr(out.ws),
                                   int(out.ws.numel() * 8), _stream(stream)), "sim_hit_truth")
        if not retry:
            return
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        cells, _, _, status = out.counts()
        if status == 0:
            return
        out.reserve(max(2 * out.max_cells, cells + cells // 4))
    raise RuntimeError("sim_hit_truth: cell capacity still too small")


def sim_hit_points(cfg: SimConfig, hits: Hits, x, y, z, t_event=None, stream=None):
    h = hits.struct()
    _check(lib().sim_hit_points(C.byref(cfg), C.byref(h), _ptr(t_event), _ptr(x), _ptr(y), _ptr(z),
                                _stream(stream)), "sim_hit_points")


def sim_track_dqdx(x, y, z, q, n_points, origin, direction, piece_cm: float, n_pieces: int, r_max_cm: float,
                   dq, count, stream=None):
    """``n_points``: device int64 tensor holding the number of points; dq FP64 and count int32 [n_pieces]."""
    o = (C.c_double * 3)(*[float(v) for v in origin])
    u = (C.c_double * 3)(*[float(v) for v in direction])
    _check(lib().sim_track_dqdx(_ptr(x), _ptr(y), _ptr(z), _ptr(q), _ptr(n_points), int(x.numel()), o, u,
                                float(piece_cm), int(n_pieces), float(r_max_cm), _ptr(dq), _ptr(count),
                                _stream(stream)), "sim_track_dqdx")


def sim_event_view_of(cfg: SimConfig, n_segments: int, max_pairs: int, max_pixels: int, ws,
                      max_events: int = 0) -> SimEventView:
    v = SimEventView()
    _check(lib().sim_event_view_of(C.byref(cfg), int(max_events), int(n_segments), int(max_pairs), int(max_pixels),
                                   _ptr(ws),
                                   int(ws.numel() * ws.element_size()), C.byref(v)), "sim_event_view_of")
    return v


# ------------------------------------------------------------ convenience --

def _alias(ptr, n, dtype, device):
    """A torch tensor aliasing ``n`` elements of device memory at ``ptr`` (no copy)."""
    import torch
    elem = torch.tensor([], dtype=dtype).element_size()
    typestr = {torch.float32: "<f4", torch.int32: "<i4", torch.int64: "<i8", torch.uint8: "|u1"}[dtype]

    class _CAI:
        __cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                    "version": 2, "strides": None}

    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    t = torch.as_tensor(_CAI(), device=device)
    assert t.element_size() == elem
    return t


class EventRunner:
    """Allocates the workspace and hit buffers once and runs sim_event on events.

    ``max_pairs`` / ``max_pixels`` / ``max_hits`` bound one event; on a
    capacity overflow ``run`` reports it (status bits) and the caller grows
    the runner.
    """

    def __init__(self, cfg: dict, lut_padded, lut_nt: int, bins_per_pitch: int, max_segments: int,
                 max_pairs: int, max_pixels: int, max_hits: int, device="cuda", max_events: int = 0):
        import torch
        self.cfg_dict = cfg
        self.cfg = make_config(cfg)
        self.resp = Response(lut_padded, lut_nt, bins_per_pitch)
        self.max_segments, self.max_pairs, self.max_pixels = int(max_segments), int(max_pairs), int(max_pixels)
        self.max_events = int(max_events)
        self.ws_bytes = workspace_size(self.cfg, self.max_segments, self.max_pairs, self.max_pixels,
                                       self.max_events)
        self.ws = torch.empty((self.ws_bytes + 7) // 8, dtype=torch.int64, device=device)
        self.hits = Hits(max_hits, device)
        self.device = device

    def view(self, n_segments: int) -> SimEventView:
        return sim_event_view_of(self.cfg, n_segments, self.max_pairs, self.max_pixels, self.ws, self.max_events)

    def enqueue(self, seg: Segments, stream=None):
        if seg.n > self.max_segments:
            raise ValueError("event larger than the runner's max_segments")
        if seg.n_events > max(self.max_events, 1):
            raise ValueError("batch larger than the runner's max_events")
        sim_event(self.cfg, seg, self.resp, self.max_pairs, self.max_pixels, self.hits, self.ws, stream)

    def counts(self):
        """(pairs, pixels, hits, status) after the stream has run."""
        return [int(x) for x in self.ws[:4].cpu().tolist()]

    def current(self, n_segments: int, n_pixels: int):
        import torch
        v = self.view(n_segments)
        T = int(self.cfg.n_ticks)
        return _alias(v.current, n_pixels * T, torch.float32, self.ws.device).view(n_pixels, T)

    def active_pixels(self, n_segments: int, n_pixels: int):
        import torch
        v = self.view(n_segments)
        return _alias(v.active_pixels, n_pixels, torch.int32, self.ws.device)

    def csr(self, n_segments: int, n_pixels: int, n_pairs: int):
        import torch
        v = self.view(n_segments)
        off = _alias(v.pix_seg_off, n_pixels + 1, torch.int32, self.ws.device)
        ids = _alias(v.pix_seg_ids, n_pairs, torch.int32, self.ws.device)
        return off, ids


class EventIO:
    """End-to-end use of :class:`EventRunner`: pinned host segments in, hits out.

    ``simulate`` copies one event's segment columns from pinned host memory
    to the device, runs sim_event and reads the hit list back to the host.
    """

    def __init__(self, runner: EventRunner):
        import torch
        self.r = runner
        n = runner.max_segments
        self.dev_cols = {k: torch.empty(n, dtype=torch.float32, device=runner.device) for k in Segments.KEYS}
        self.host_counts = torch.zeros(4, dtype=torch.int64).pin_memory()
        cap = runner.hits.capacity
        self.host_hits = {k: torch.empty(max(cap, 1), dtype=getattr(runner.hits, k).dtype).pin_memory()
                          for k in ("pixel", "t_cross", "t_adc", "adc", "q")}

    def simulate(self, host_cols: dict, n: int, event_id: int = 0, stream=None):
        """Returns (hits dict of host tensors, counts, h2d_bytes, d2h_bytes)."""
        import torch
        for k in Segments.KEYS:
            self.dev_cols[k][:n].copy_(host_cols[k][:n], non_blocking=True)
        seg = Segments({k: self.dev_cols[k][:n] for k in Segments.KEYS}, event_id)
        self.r.enqueue(seg, stream)
        self.host_counts.copy_(self.r.ws[:4], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        counts = [int(x) for x in self.host_counts.tolist()]
        nh = min(counts[2], self.r.hits.capacity)
        d2h = 32
        out = {}
        for k, t in self.host_hits.items():
            src = getattr(self.r.hits, k)[:nh]
            t[:nh].copy_(src, non_blocking=True)
            out[k] = t[:nh]
            d2h += nh * src.element_size()
        torch.cuda.current_stream().synchronize()
        return out, counts, 9 * 4 * n, d2h


# ------------------------------------------------------------------ light --

class Light:
    """Light-path configuration with its tables on the device (Sec. 4).

    ``params``: the light parameters (synth.light.LIGHT layout); ``tables``:
    FP32 numpy tables (vis, tdist, eff, gain, resp, noise); the window is
    [t_start_us, t_start_us + n_ticks * tick_us)."""

    def __init__(self, params: dict, tables: dict, t_start_us: float, n_ticks: int, device="cuda"):
        import torch
        self.t = {k: torch.as_tensor(np.ascontiguousarray(v, dtype=np.float32), device=device)
                  for k, v in tables.items()}
        nvx, nvy, nvz, nd, nt = tables["tdist"].shape
        c = SimLightConfig()
        c.vis, c.tdist, c.eff, c.gain = (_ptr(self.t[k]) for k in ("vis", "tdist", "eff", "gain"))
        c.resp, c.noise_amp = _ptr(self.t["resp"]), _ptr(self.t["noise"])
        c.nvx, c.nvy, c.nvz, c.n_det, c.nt = nvx, nvy, nvz, nd, nt
        c.n_resp, c.noise_block, c.adc_bits = len(tables["resp"]), int(params["noise_block"]), int(params["adc_bits"])
        c.vox_cm, c.w_ph_MeV, c.tick_us = params["vox_cm"], params["w_ph_MeV"], params["tick_us"]
        c.t_start_us, c.n_ticks = float(t_start_us), int(n_ticks)
        c.fast_frac, c.tau_fast_us, c.tau_slow_us = params["fast_frac"], params["tau_fast_us"], params["tau_slow_us"]
        c.trunc_taus, c.poisson_max_mean = params["trunc_taus"], params["poisson_max_mean"]
        c.sample_us, c.pedestal_adc = params["sample_us"], params["pedestal"]
        self.c = c
        self.n_det = nd
        self.n_ticks = int(n_ticks)
        ns = C.c_int64()
        _check(lib().sim_light_n_samples(C.byref(c), C.byref(ns)), "sim_light_n_samples")
        self.n_samples = int(ns.value)

    def n_det_total(self, cfg: SimConfig) -> int:
        return cfg.n_mod_x * cfg.n_mod_y * cfg.n_tpc * self.n_det


def sim_light_yield(cfg: SimConfig, light: Light, seg: Segments, dr: Drifted, npe, tick, vox, stream=None):
    s, d = seg.struct(), dr.struct()
    _check(lib().sim_light_yield(C.byref(cfg), C.byref(light.c), C.byref(s), C.byref(d), _ptr(npe), _ptr(tick),
                                 _ptr(vox), _stream(stream)), "sim_light_yield")


def sim_light_photocurrent(cfg: SimConfig, light: Light, seg: Segments, dr: Drifted, npe, tick, vox, pe_fix,
                           stream=None):
    s, d = seg.struct(), dr.struct()
    _check(lib().sim_light_photocurrent(C.byref(cfg), C.byref(light.c), C.byref(s), C.byref(d), _ptr(npe),
                                        _ptr(tick), _ptr(vox), _ptr(pe_fix), _stream(stream)),
           "sim_light_photocurrent")


def sim_light_scintillation(cfg: SimConfig, light: Light, pe_fix, scint, stream=None):
    _check(lib().sim_light_scintillation(C.byref(cfg), C.byref(light.c), _ptr(pe_fix), _ptr(scint),
                                         _stream(stream)), "sim_light_scintillation")


def sim_light_fluctuate(cfg: SimConfig, light: Light, event_id: int, scint, pe_obs, stream=None):
    _check(lib().sim_light_fluctuate(C.byref(cfg), C.byref(light.c), int(event_id), _ptr(scint), _ptr(pe_obs),
                                     _stream(stream)), "sim_light_fluctuate")


def sim_light_electronics(cfg: SimConfig, light: Light, event_id: int, pe_obs, v, wave, stream=None):
    _check(lib().sim_light_electronics(C.byref(cfg), C.byref(light.c), int(event_id), _ptr(pe_obs), _ptr(v),
                                       _ptr(wave), _stream(stream)), "sim_light_electronics")


def sim_light_truth(cfg: SimConfig, light: Light, n_segments: int, tick, vox, t_arrival, stream=None):
    _check(lib().sim_light_truth(C.byref(cfg), C.byref(light.c), int(n_segments), _ptr(tick), _ptr(vox),
                                 _ptr(t_arrival), _stream(stream)), "sim_light_truth")


def light_workspace_size(cfg: SimConfig, light: Light, n_segments: int) -> int:
    b = C.c_size_t()
    _check(lib().sim_light_workspace_size(C.byref(cfg), C.byref(light.c), int(n_segments), C.byref(b)),
           "sim_light_workspace_size")
    return int(b.value)


def sim_light_event(cfg: SimConfig, light: Light, seg: Segments, dr: Drifted, wave, ws, stream=None):
    s, d = seg.struct(), dr.struct()
    _check(lib().sim_light_event(C.byref(cfg), C.byref(light.c), C.byref(s), C.byref(d), _ptr(wave), _ptr(ws),
                                 int(ws.numel() * ws.element_size()), _stream(stream)), "sim_light_event")


class GraphRunner:
    """One event step (sim_event) captured once in a CUDA graph and replayed.

    The graph is recorded at a fixed segment capacity with the batch form of
    sim_segments (one event slot whose id is read from device memory), so that
    any event of up to ``max_segments`` segments and any event id replay the
    same graph: the event's columns are copied into the graph's input buffers
    and the rest is filled with inactive segments (zero length: no charge, no
    pixels), which leaves the results of the real segments unchanged (their
    random numbers are keyed by their own indices).  Replaying skips the ~30
    kernel launches of a step, which matters for small events."""

    FILL = dict(x0=-1.0e4, y0=-1.0e4, z0=-1.0e4, t0=0.0, x1=-1.0e4, y1=-1.0e4, z1=-1.0e4, t1=0.0, dE=0.0)

    def __init__(self, runner: EventRunner, stream=None):
        import torch
        self.r = runner
        dev = runner.device
        n = runner.max_segments
        self.cols = {k: torch.full((n,), self.FILL[k], dtype=torch.float32, device=dev) for k in Segments.KEYS}
        self.fill = {k: v.clone() for k, v in self.cols.items()}          # padding source (device copies only)
        self.offsets = torch.tensor([0, n], dtype=torch.int64, device=dev)
        self.ids = torch.zeros(1, dtype=torch.int64, device=dev)
        self.ids_host = torch.zeros(64, dtype=torch.int64).pin_memory()   # ring of pinned id slots
        self.k = 0
        self.seg = Segments(self.cols, 0, self.offsets, self.ids)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        # warm up on the capture stream (lazy module loading, attributes), then capture
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            runner.enqueue(self.seg, self.stream)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            runner.enqueue(self.seg, self.stream)
        self.stream.synchronize()

    def load(self, cols: dict, n: int, event_id: int):
        """Enqueues the copies of an event (device or pinned host columns, n
        segments) and of its id into the graph's inputs (copies only, no kernels)."""
        if n > self.r.max_segments:
            raise ValueError("event larger than the graph's capacity")
        N = self.r.max_segments
        for k in Segments.KEYS:
            if n > 0:
                self.cols[k][:n].copy_(cols[k][:n], non_blocking=True)
            if n < N:
                self.cols[k][n:].copy_(self.fill[k][n:], non_blocking=True)
        slot = self.ids_host[self.k % 64: self.k % 64 + 1]
        self.k += 1
        slot.fill_(int(np.uint64(event_id & 0xFFFFFFFFFFFFFFFF).astype(np.int64)))
        self.ids.copy_(slot, non_blocking=True)

    def replay(self):
        """Runs the captured step after the work already on the current stream (the
        inputs' copies); the current stream then waits for it."""
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        torch.cuda.current_stream().wait_stream(self.stream)


class BatchGraphRunner:
    """A batch of events (sim_segments with ``max_events`` slots) through
    sim_event, captured once in a CUDA graph at fixed capacities and replayed
    for any batch of up to ``max_events`` events and ``runner.max_segments``
    segments.

    The event offsets and ids live in device memory, so a replay reads the
    batch that ``load`` copied into the graph's inputs: the events' columns
    (device tensors), then inactive padding segments (zero length: no
    charge, no pixels) up to the capacity, owned by the last slot; unused
    slots are empty.  Every event's results are those of the same batch
    called directly (its random numbers are keyed by its own id and
    event-local segment index).  ``runner`` must have been built with
    ``max_events`` slots and capacities that fit every batch it will run."""

    FILL = GraphRunner.FILL

    def __init__(self, runner: EventRunner, stream=None):
        import torch
        if runner.max_events < 1:
            raise ValueError("the runner needs max_events >= 1 for a batch graph")
        self.r = runner
        dev = runner.device
        n, E = runner.max_segments, runner.max_events
        self.E = E
        self.cols = {k: torch.full((n,), self.FILL[k], dtype=torch.float32, device=dev) for k in Segments.KEYS}
        self.fill = {k: v.clone() for k, v in self.cols.items()}
        self.offsets = torch.zeros(E + 1, dtype=torch.int64, device=dev)
        self.offsets[-1] = n
        self.ids = torch.zeros(E, dtype=torch.int64, device=dev)
        self.seg = Segments(self.cols, 0, self.offsets, self.ids)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            runner.enqueue(self.seg, self.stream)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            runner.enqueue(self.seg, self.stream)
        self.stream.synchronize()

    def load(self, batch: Segments):
        """Enqueues device copies of a batch (a Segments with n_events >= 1)
        into the graph's inputs on the current stream (copies only)."""
        N = self.r.max_segments
        n, e = batch.n, batch.n_events
        if n > N or e > self.E or e < 1:
            raise ValueError("batch outside the graph's capacities")
        for k in Segments.KEYS:
            if n > 0:
                self.cols[k][:n].copy_(batch.cols[k][:n], non_blocking=True)
            if n < N:
                self.cols[k][n:].copy_(self.fill[k][n:], non_blocking=True)
        self.offsets[: e + 1].copy_(batch.offsets[: e + 1], non_blocking=True)
        if e < self.E:
            self.offsets[e + 1:].fill_(n)
        self.offsets[self.E:].fill_(N)                 # the padding belongs to the last slot
        self.ids[:e].copy_(batch.ids[:e], non_blocking=True)
        if e < self.E:
            self.ids[e:].fill_(0)

    def replay(self):
        """Runs the captured batch after the work already on the current stream
        (the inputs' copies); the current stream then waits for it."""
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        torch.cuda.current_stream().wait_stream(self.stream)
