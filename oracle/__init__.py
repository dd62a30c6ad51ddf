"""FP64 CPU oracle of the pixelated-LArTPC simulation (arXiv:2212.09807: the
charge path of Sec. 3, the light path of Sec. 4, and the per-hit steps after
the front end).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the CUDA path.  The arithmetic lives in
``larsim_oracle.c`` (plain C, FP64); this module builds it with gcc and
marshals numpy arrays through ctypes.  Parity pins: see tests/test_oracle_*.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "larsim_oracle.c")
LIB = os.path.join(HERE, "liblarsim_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (IEEE order kept: no FMA contraction).

    With OpenMP when the compiler has it (the many-pixel functions then share
    their independent pixels among the host cores); without, they run on one
    thread and give the same results."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall"]
        try:
            subprocess.check_call(base + ["-fopenmp", SRC, "-o", tmp, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + [SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Cfg(C.Structure):
    _fields_ = [
        ("n_mod_x", C.c_int32), ("n_mod_y", C.c_int32), ("n_tpc", C.c_int32),
        ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("px_per_tile", C.c_int32),
        ("pitch", C.c_double), ("drift_len", C.c_double),
        ("recomb_model", C.c_int32),
        ("Ab", C.c_double), ("kb", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
        ("efield", C.c_double), ("density", C.c_double), ("w_ion", C.c_double),
        ("vdrift", C.c_double), ("lifetime", C.c_double), ("DL", C.c_double), ("DT", C.c_double),
        ("step", C.c_double), ("M", C.c_int32), ("clip", C.c_double),
        ("tick", C.c_double), ("n_ticks", C.c_int32), ("t_w0", C.c_double),
        ("thr", C.c_double), ("s_reset", C.c_double), ("s_disc", C.c_double),
        ("s_unc", C.c_double), ("gain", C.c_double), ("lsb_mV", C.c_double),
        ("hold", C.c_int32), ("min_int", C.c_int32), ("periodic", C.c_int32),
        ("adc_bits", C.c_int32),
        ("seed", C.c_uint64),
        ("nb", C.c_int32), ("nt", C.c_int32), ("bins_per_pitch", C.c_int32), ("per_point", C.c_int32),
        ("nearest", C.c_int32), ("pad2", C.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        f32p, f64p, i32p, i64p, u32p = (P(C.c_float), P(C.c_double), P(C.c_int32),
                                        P(C.c_int64), P(C.c_uint32))
        L.ora_cfg_size.restype = C.c_size_t
        L.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.ora_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_uint32, f64p]
        L.ora_recomb.argtypes = [P(_Cfg), C.c_double]
        L.ora_recomb.restype = C.c_double
        L.ora_quench_drift.argtypes = [P(_Cfg), C.c_int64] + [f32p] * 9 + [f64p] * 8 + [i32p, i32p]
        L.ora_cheb_distance.argtypes = [C.c_double] * 6
        L.ora_cheb_distance.restype = C.c_double
        L.ora_map_radius.argtypes = [P(_Cfg), C.c_double]
        L.ora_map_radius.restype = C.c_double
        L.ora_map_segment.argtypes = [P(_Cfg), C.c_float, C.c_float, C.c_float, C.c_float,
                                      C.c_double, C.c_int32, i32p, f64p, C.c_int64]
        L.ora_map_segment.restype = C.c_int64
        L.ora_map_segment_box.argtypes = L.ora_map_segment.argtypes
        L.ora_map_segment_box.restype = C.c_int64
        L.ora_pair_margin.argtypes = [P(_Cfg), C.c_float, C.c_float, C.c_float, C.c_float,
                                      C.c_double, C.c_int32, C.c_int32]
        L.ora_pair_margin.restype = C.c_double
        L.ora_pixel_current.argtypes = ([P(_Cfg), f64p] + [f32p] * 8 + [f64p] * 4
                                        + [i32p, i32p, C.c_uint64, C.c_int32, i64p, C.c_int64, f64p, C.c_double,
                                           C.POINTER(C.c_int64)])
        L.ora_electronics.argtypes = [P(_Cfg), C.c_uint64, C.c_int32, f64p, C.c_int64,
                                      i32p, i32p, i32p, f64p, C.c_double, i32p, f64p]
        L.ora_electronics.restype = C.c_int64
        L.ora_hit_intervals.argtypes = [P(_Cfg), C.c_int64, i32p, i32p, i32p, i32p]
        L.ora_hit_point.argtypes = [P(_Cfg), C.c_int32, C.c_int32, C.c_double, f64p]
        L.ora_track_dqdx.argtypes = [C.c_int64, f64p, f64p, f64p, f64p, f64p, f64p, C.c_double, C.c_int32,
                                     C.c_double, f64p, i64p, f64p]
        L.ora_threads.argtypes = [C.c_int]
        L.ora_threads.restype = C.c_int
        L.ora_map_event.argtypes = [P(_Cfg), C.c_int64] + [f32p] * 4 + [f64p, i32p, C.c_int64, i64p, i32p, f64p]
        L.ora_map_event.restype = C.c_int64
        L.ora_pixel_currents_many.argtypes = ([P(_Cfg), f64p] + [f32p] * 8 + [f64p] * 4
                                              + [i32p, i32p, C.c_uint64, C.c_int64, i32p, i64p, i64p, f64p, C.c_int])
        L.ora_electronics_many.argtypes = [P(_Cfg), C.c_uint64, C.c_int64, i32p, f64p, f64p, C.c_int64, i32p, i32p,
                                           i32p, f64p, i64p, i32p, f64p, C.c_int]
        assert L.ora_cfg_size() == C.sizeof(_Cfg), "oracle config struct mismatch"
        _lib = L
    return _lib


def _f32(v):
    return float(np.float32(v))


def make_cfg(cfg: dict, lut_par: dict) -> _Cfg:
    """Oracle configuration: FP32 configuration values widened to FP64."""
    c = _Cfg()
    for k in ("n_mod_x", "n_mod_y", "n_tpc", "tiles_x", "tiles_y", "px_per_tile"):
        setattr(c, k, int(cfg[k]))
    c.pitch = _f32(cfg["pitch_cm"])
    c.drift_len = _f32(cfg["drift_len_cm"])
    c.recomb_model = int(cfg["recomb_model"])
    c.Ab, c.kb = _f32(cfg["birks_Ab"]), _f32(cfg["birks_kb"])
    c.alpha, c.beta = _f32(cfg["box_alpha"]), _f32(cfg["box_beta"])
    c.efield, c.density = _f32(cfg["efield_kV_cm"]), _f32(cfg["lar_density_g_cm3"])
    c.w_ion = _f32(cfg["w_ion_MeV"])
    c.vdrift, c.lifetime = _f32(cfg["vdrift_cm_us"]), _f32(cfg["lifetime_us"])
    c.DL, c.DT = _f32(cfg["diff_long_cm2_s"]), _f32(cfg["diff_tran_cm2_s"])
    c.step, c.M, c.clip = _f32(cfg["sample_step_cm"]), int(cfg["mc_per_sample"]), _f32(cfg["diff_clip_sigma"])
    c.tick, c.n_ticks, c.t_w0 = _f32(cfg["tick_us"]), int(cfg["n_ticks"]), _f32(cfg["t_window0_us"])
    c.thr, c.s_reset = _f32(cfg["thr_e"]), _f32(cfg["sigma_reset_e"])
    c.s_disc, c.s_unc = _f32(cfg["sigma_disc_e"]), _f32(cfg["sigma_unc_e"])
    c.gain, c.lsb_mV = _f32(cfg["gain_e_per_mV"]), _f32(cfg["adc_lsb_mV"])
    c.hold, c.min_int = int(cfg["hold_ticks"]), int(cfg["min_adc_interval_ticks"])
    c.periodic, c.adc_bits = int(cfg["periodic_reset_ticks"]), int(cfg["adc_bits"])
    c.seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF
    c.nb, c.nt, c.bins_per_pitch = int(lut_par["nb"]), int(lut_par["nt"]), int(lut_par["bins_per_pitch"])
    c.per_point = int(cfg.get("per_point_drift", 0))
    c.nearest = int(cfg.get("nearest_lut", 0))
    return c


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block for a 4-word counter and a 2-word key."""
    L = lib()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    L.ora_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def normals(seed, event_id, c0, c1, c2, c3=0):
    L = lib()
    o = np.zeros(4)
    L.ora_normals(seed, event_id, c0, c1, c2, c3, _p(o, C.c_double))
    return o


class Oracle:
    """Per-step oracle for one configuration and response table."""

    def __init__(self, cfg: dict, lut_par: dict, lut: np.ndarray | None = None):
        self.L = lib()
        self.cfg = cfg
        self.c = make_cfg(cfg, lut_par)
        self.nb = int(lut_par["nb"])
        self.nt = int(lut_par["nt"])
        if lut is not None:
            lut = np.ascontiguousarray(np.asarray(lut, dtype=np.float64)[..., : self.nt])
            assert lut.shape == (self.nb, self.nb, self.nt)
        self.lut = lut
        self.npx_x = cfg["tiles_x"] * cfg["px_per_tile"]
        self.npx_y = cfg["tiles_y"] * cfg["px_per_tile"]
        self.n_anodes = cfg["n_mod_x"] * cfg["n_mod_y"] * cfg["n_tpc"]

    # -- steps 1-2 ---------------------------------------------------------
    def recomb(self, dedx: float) -> float:
        return self.L.ora_recomb(C.byref(self.c), float(dedx))

    def quench_drift(self, seg: dict) -> dict:
        n = len(seg["x0"])
        cols = [np.ascontiguousarray(seg[k], dtype=np.float32)
                for k in ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")]
        names = ("dx", "dedx", "R", "QR", "Qa", "t_drift", "sigma_T", "sigma_L")
        out = {k: np.zeros(n) for k in names}
        out["anode"] = np.zeros(n, dtype=np.int32)
        out["n_samples"] = np.zeros(n, dtype=np.int32)
        self.L.ora_quench_drift(C.byref(self.c), n, *[_p(a, C.c_float) for a in cols],
                                *[_p(out[k], C.c_double) for k in names],
                                _p(out["anode"], C.c_int32), _p(out["n_samples"], C.c_int32))
        out["_seg"] = cols
        return out

    # -- step 3 ------------------------------------------------------------
    def map_radius(self, sigma_T: float) -> float:
        return self.L.ora_map_radius(C.byref(self.c), float(sigma_T))

    def map_segment(self, seg: dict, dr: dict, s: int, box: bool = True):
        """(ids, margins) of the pixels segment s is mapped to (brute force over
        the whole anode, or over the segment's widened bounding box)."""
        fn = self.L.ora_map_segment_box if box else self.L.ora_map_segment
        cap = 4096
        while True:
            ids = np.zeros(cap, dtype=np.int32)
            mg = np.zeros(cap)
            n = fn(C.byref(self.c), float(seg["x0"][s]), float(seg["y0"][s]),
                                       float(seg["x1"][s]), float(seg["y1"][s]),
                                       float(dr["sigma_T"][s]), int(dr["anode"][s]),
                                       _p(ids, C.c_int32), _p(mg, C.c_double), cap)
            if n <= cap:
                return ids[:n].copy(), mg[:n].copy()
            cap = int(n)

    def pair_margin(self, seg, dr, s, pixel) -> float:
        return self.L.ora_pair_margin(C.byref(self.c), float(seg["x0"][s]), float(seg["y0"][s]),
                                      float(seg["x1"][s]), float(seg["y1"][s]),
                                      float(dr["sigma_T"][s]), int(dr["anode"][s]), int(pixel))

    def pixel_map(self, seg: dict, dr: dict):
        """Brute-force map of every segment: returns (pixel -> sorted segment list, pairs, margins)."""
        pix = {}
        pairs_s, pairs_p, margins = [], [], []
        for s in range(len(seg["x0"])):
            if dr["anode"][s] < 0:
                continue
            ids, mg = self.map_segment(seg, dr, s)
            for p, m in zip(ids.tolist(), mg.tolist()):
                pix.setdefault(p, []).append(s)
                pairs_s.append(s)
                pairs_p.append(p)
                margins.append(m)
        return pix, np.array(pairs_s, dtype=np.int64), np.array(pairs_p, dtype=np.int64), np.array(margins)

    def segments_for_pixel(self, seg: dict, dr: dict, pixel: int):
        """Segments mapped to one pixel and their margins (brute force over segments)."""
        out, mg = [], []
        for s in np.nonzero(dr["anode"] >= 0)[0].tolist():
            m = self.pair_margin(seg, dr, s, pixel)
            if m >= 0:
                out.append(s)
                mg.append(m)
        return np.array(out, dtype=np.int64), np.array(mg)

    def map_event(self, seg: dict, dr: dict) -> dict:
        """The map of every segment (ora_map_event) as both CSR directions:
        ``pixels`` (mapped pixel ids, increasing), ``off``/``segs`` (each
        pixel's segments, increasing) and ``margin`` (R_map - d of each entry)."""
        cols = dr["_seg"]
        n = len(cols[0])
        sT = np.ascontiguousarray(dr["sigma_T"], dtype=np.float64)
        an = np.ascontiguousarray(dr["anode"], dtype=np.int32)
        cap = max(1024, 64 * n)
        while True:
            ps = np.zeros(cap, np.int64)
            pp = np.zeros(cap, np.int32)
            pm = np.zeros(cap)
            m = self.L.ora_map_event(C.byref(self.c), n, _p(cols[0], C.c_float), _p(cols[1], C.c_float),
                                     _p(cols[4], C.c_float), _p(cols[5], C.c_float), _p(sT, C.c_double),
                                     _p(an, C.c_int32), cap, _p(ps, C.c_int64), _p(pp, C.c_int32),
                                     _p(pm, C.c_double))
            if m <= cap:
                break
            cap = int(m)
        ps, pp, pm = ps[:m], pp[:m], pm[:m]
        order = np.argsort(pp, kind="stable")            # segments stay increasing within a pixel
        pix_sorted = pp[order]
        pixels, start = np.unique(pix_sorted, return_index=True)
        off = np.append(start, m).astype(np.int64)
        return dict(pixels=pixels.astype(np.int32), off=off, segs=ps[order], margin=pm[order])

    @staticmethod
    def threads(n_threads: int = 0) -> int:
        """Host threads the many-pixel functions use (0 = all cores)."""
        return int(lib().ora_threads(int(n_threads)))

    def pixel_currents(self, seg: dict, dr: dict, pixels, off, segs, event_id: int = 0, n_threads: int = 0):
        """Currents [n, n_ticks] of many pixels: pixel pixels[i] with segment
        list segs[off[i]:off[i+1]], each exactly as pixel_current computes it."""
        assert self.lut is not None
        cols = dr["_seg"]
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        off = np.ascontiguousarray(off, dtype=np.int64)
        segs = np.ascontiguousarray(segs, dtype=np.int64)
        assert len(off) == len(pixels) + 1
        I = np.zeros((len(pixels), int(self.c.n_ticks)))
        self.L.ora_pixel_currents_many(C.byref(self.c), _p(self.lut, C.c_double),
                                       *[_p(a, C.c_float) for a in cols[:8]],
                                       _p(dr["Qa"], C.c_double), _p(dr["t_drift"], C.c_double),
                                       _p(dr["sigma_T"], C.c_double), _p(dr["sigma_L"], C.c_double),
                                       _p(dr["anode"], C.c_int32), _p(dr["n_samples"], C.c_int32), event_id,
                                       len(pixels), _p(pixels, C.c_int32), _p(off, C.c_int64), _p(segs, C.c_int64),
                                       _p(I, C.c_double), int(n_threads))
        return I

    def electronics_many(self, pixels, I, event_id: int = 0, band=None, n_threads: int = 0):
        """Front end of many pixels (row i of I is pixel pixels[i]'s current),
        each exactly as electronics computes it; band: one tie band per pixel
        (or a scalar).  Returns a list of per-pixel dicts like electronics."""
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        n = len(pixels)
        I = np.ascontiguousarray(I, dtype=np.float64)
        assert I.shape == (n, int(self.c.n_ticks))
        bnd = np.ascontiguousarray(np.broadcast_to(np.asarray(0.0 if band is None else band, np.float64), (n,)))
        cap = int(self.c.n_ticks)
        tc = np.zeros((n, cap), np.int32)
        ta = np.zeros((n, cap), np.int32)
        ad = np.zeros((n, cap), np.int32)
        qv = np.zeros((n, cap))
        nh = np.zeros(n, np.int64)
        tie = np.zeros(n, np.int32)
        pt = np.zeros(n)
        self.L.ora_electronics_many(C.byref(self.c), event_id, n, _p(pixels, C.c_int32), _p(I, C.c_double),
                                    _p(bnd, C.c_double), cap, _p(tc, C.c_int32), _p(ta, C.c_int32),
                                    _p(ad, C.c_int32), _p(qv, C.c_double), _p(nh, C.c_int64), _p(tie, C.c_int32),
                                    _p(pt, C.c_double), int(n_threads))
        return [dict(t_cross=tc[i, :nh[i]].copy(), t_adc=ta[i, :nh[i]].copy(), adc=ad[i, :nh[i]].copy(),
                     q=qv[i, :nh[i]].copy(), tie_tick=int(tie[i]), p_tie=float(pt[i])) for i in range(n)]

    # -- step 4 ------------------------------------------------------------
    def pixel_current(self, seg: dict, dr: dict, pixel: int, segs, event_id: int = 0,
                      lut: np.ndarray | None = None, tie_band: float | None = None):
        """Current of one pixel; with tie_band (nearest-bin lookup): also the
        number of points with a rounding within tie_band of its half-way point."""
        lut = self.lut if lut is None else np.ascontiguousarray(np.asarray(lut, np.float64)[..., : self.nt])
        assert lut is not None
        cols = dr["_seg"]
        segs = np.ascontiguousarray(segs, dtype=np.int64)
        I = np.zeros(int(self.c.n_ticks))
        nt_ = C.c_int64(0)
        self.L.ora_pixel_current(C.byref(self.c), _p(lut, C.c_double),
                                 *[_p(a, C.c_float) for a in cols[:8]],
                                 _p(dr["Qa"], C.c_double), _p(dr["t_drift"], C.c_double),
                                 _p(dr["sigma_T"], C.c_double),
                                 _p(dr["sigma_L"], C.c_double), _p(dr["anode"], C.c_int32),
                                 _p(dr["n_samples"], C.c_int32), event_id, int(pixel),
                                 _p(segs, C.c_int64), len(segs), _p(I, C.c_double),
                                 float(tie_band or 0.0), C.byref(nt_))
        return (I, int(nt_.value)) if tie_band is not None else I

    # -- step 5 ------------------------------------------------------------
    def electronics(self, pixel: int, I: np.ndarray, event_id: int = 0, band: float = 0.0) -> dict:
        I = np.ascontiguousarray(I, dtype=np.float64)
        assert len(I) == self.c.n_ticks
        cap = self.c.n_ticks
        tc = np.zeros(cap, np.int32)
        ta = np.zeros(cap, np.int32)
        ad = np.zeros(cap, np.int32)
        qv = np.zeros(cap)
        tie = np.zeros(1, np.int32)
        pt = np.zeros(1)
        n = self.L.ora_electronics(C.byref(self.c), event_id, int(pixel), _p(I, C.c_double), cap,
                                   _p(tc, C.c_int32), _p(ta, C.c_int32), _p(ad, C.c_int32),
                                   _p(qv, C.c_double), float(band), _p(tie, C.c_int32), _p(pt, C.c_double))
        return dict(t_cross=tc[:n].copy(), t_adc=ta[:n].copy(), adc=ad[:n].copy(),
                    q=qv[:n].copy(), tie_tick=int(tie[0]), p_tie=float(pt[0]))

    # -- after step 5: per-hit charge truth, 3-D points, dQ/dx --------------
    def hit_intervals(self, t_cross, t_adc):
        """[k0, k1] tick interval each hit of one pixel digitises (Sec. 3.4)."""
        tc = np.ascontiguousarray(t_cross, dtype=np.int32)
        ta = np.ascontiguousarray(t_adc, dtype=np.int32)
        k0 = np.zeros(len(tc), np.int32)
        k1 = np.zeros(len(tc), np.int32)
        self.L.ora_hit_intervals(C.byref(self.c), len(tc), _p(tc, C.c_int32), _p(ta, C.c_int32),
                                 _p(k0, C.c_int32), _p(k1, C.c_int32))
        return k0, k1

    def hit_truth(self, seg: dict, dr: dict, pixel: int, segs, t_cross, t_adc, event_id: int = 0):
        """Charge each mapped segment induced in each hit's interval.

        Returns (Q [n_hits, n_segs] electrons, q_signal [n_hits], k0, k1):
        Q[h, j] = sum over the interval of hit h of the current of segment
        segs[j] alone (Eq. (current) restricted to one segment); q_signal is
        the interval sum of the pixel's whole current."""
        segs = np.asarray(segs, dtype=np.int64)
        k0, k1 = self.hit_intervals(t_cross, t_adc)
        cs = np.zeros((len(segs), int(self.c.n_ticks) + 1))
        for j, s in enumerate(segs.tolist()):
            cs[j, 1:] = np.cumsum(self.pixel_current(seg, dr, pixel, [s], event_id=event_id))
        full = np.concatenate([[0.0], np.cumsum(self.pixel_current(seg, dr, pixel, segs, event_id=event_id))])
        Q = cs[:, k1 + 1].T - cs[:, k0].T
        return Q, full[k1 + 1] - full[k0], k0, k1

    def hit_points(self, pixel, t_cross, t_event: float = 0.0):
        """(x, y, z) [n, 3] of hits (Sec. 6): pixel centre, inverse of Eq. (drift)."""
        out = np.zeros((len(pixel), 3))
        for i, (p, k) in enumerate(zip(np.asarray(pixel).tolist(), np.asarray(t_cross).tolist())):
            self.L.ora_hit_point(C.byref(self.c), int(p), int(k), float(t_event), _p(out[i], C.c_double))
        return out

    @staticmethod
    def track_dqdx(points, q, origin, direction, dx: float, n_bins: int, r_max: float):
        """(dq [n_bins], count [n_bins], margin [n]) of points along a known straight track (Sec. 6)."""
        L = lib()
        P = np.ascontiguousarray(points, dtype=np.float64)
        x, y, z = (np.ascontiguousarray(P[:, i]) for i in range(3))
        qq = np.ascontiguousarray(q, dtype=np.float64)
        o = np.ascontiguousarray(origin, dtype=np.float64)
        u = np.ascontiguousarray(direction, dtype=np.float64)
        dq = np.zeros(n_bins)
        cnt = np.zeros(n_bins, np.int64)
        mg = np.zeros(len(qq))
        L.ora_track_dqdx(len(qq), _p(x, C.c_double), _p(y, C.c_double), _p(z, C.c_double), _p(qq, C.c_double),
                         _p(o, C.c_double), _p(u, C.c_double), float(dx), int(n_bins), float(r_max),
                         _p(dq, C.c_double), _p(cnt, C.c_int64), _p(mg, C.c_double))
        return dq, cnt, mg


# ================================================================= light ==

class _Light(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("nvx", "nvy", "nvz", "n_det", "nt", "n_ticks", "n_trunc", "n_resp",
                                         "noise_block", "adc_bits")] + \
               [(k, C.c_double) for k in ("vox", "w_ph", "tick", "t_start", "fast_frac", "tau_fast", "tau_slow",
                                          "poisson_max", "sample", "pedestal")]


def light_derived(L: dict, n_ticks: int):
    """(n_trunc, ratio, n_samples) of a light configuration: the truncation of
    the scintillation sum (trunc_taus tau_slow in ticks, rounded), the
    sampling period in ticks and the number of samples of the window."""
    tick = _f32(L["tick_us"])
    n_trunc = int(np.floor(_f32(L["trunc_taus"]) * _f32(L["tau_slow_us"]) / tick + 0.5))
    ratio = _f32(L["sample_us"]) / tick
    n_samples = int(np.floor((n_ticks - 1) / ratio)) + 1
    return n_trunc, ratio, n_samples


class LightOracle:
    """FP64 oracle of the light path (Sec. 4) for one configuration, light
    parameters, FP32 tables (synth.light.tables) and time window."""

    def __init__(self, cfg: dict, L: dict, tab: dict, t_start_us: float, n_ticks: int):
        self.lib = lib()
        f64p, i32p, f32p = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_float)
        self.lib.ora_light_size.restype = C.c_size_t
        assert self.lib.ora_light_size() == C.sizeof(_Light)
        self.lib.ora_light_segment.argtypes = [C.POINTER(_Cfg), C.POINTER(_Light), f32p, C.c_double, C.c_int32,
                                               f64p, f64p, f64p, i32p, i32p]
        self.lib.ora_light_segment.restype = C.c_int
        self.lib.ora_light_photocurrent.argtypes = [C.POINTER(_Light), C.c_int64, f64p, i32p, i32p, i32p, f64p,
                                                    C.c_int32, C.c_int32, f64p]
        self.lib.ora_light_scintillation.argtypes = [C.POINTER(_Light), f64p, f64p]
        self.lib.ora_light_fluctuate.argtypes = [C.POINTER(_Cfg), C.POINTER(_Light), C.c_uint64, C.c_int32, f64p,
                                                 f64p, f64p]
        self.lib.ora_light_electronics.argtypes = [C.POINTER(_Cfg), C.POINTER(_Light), C.c_uint64, C.c_int32,
                                                   C.c_double, f64p, f64p, f64p, C.c_double, C.c_int32, f64p, f64p,
                                                   i32p, f64p]
        self.lib.ora_light_truth.argtypes = [C.POINTER(_Light), C.c_int64, i32p, i32p, f64p, f64p]
        self.c = make_cfg(cfg, dict(nb=1, nt=1, bins_per_pitch=1))
        l = _Light()
        nvx, nvy, nvz, nd, nt = tab["tdist"].shape
        l.nvx, l.nvy, l.nvz, l.n_det, l.nt = nvx, nvy, nvz, nd, nt
        l.n_ticks = int(n_ticks)
        self.n_trunc, self.ratio, self.n_samples = light_derived(L, n_ticks)
        l.n_trunc = self.n_trunc
        l.n_resp = len(tab["resp"])
        l.noise_block = int(L["noise_block"])
        l.adc_bits = int(L["adc_bits"])
        l.vox, l.w_ph, l.tick = _f32(L["vox_cm"]), _f32(L["w_ph_MeV"]), _f32(L["tick_us"])
        l.t_start = _f32(t_start_us)
        l.fast_frac, l.tau_fast, l.tau_slow = _f32(L["fast_frac"]), _f32(L["tau_fast_us"]), _f32(L["tau_slow_us"])
        l.poisson_max, l.sample, l.pedestal = _f32(L["poisson_max_mean"]), _f32(L["sample_us"]), _f32(L["pedestal"])
        self.l = l
        self.n_det = nd
        self.vis = np.ascontiguousarray(tab["vis"].reshape(-1), dtype=np.float64)
        self.tdist = np.ascontiguousarray(tab["tdist"].reshape(-1), dtype=np.float64)
        self.eff = np.ascontiguousarray(tab["eff"], dtype=np.float64)
        self.gain = np.ascontiguousarray(tab["gain"], dtype=np.float64)
        self.resp = np.ascontiguousarray(tab["resp"], dtype=np.float64)
        self.amp = np.ascontiguousarray(tab["noise"], dtype=np.float64)

    def segments(self, seg: dict, dr: dict):
        """(npe [n, n_det], tick [n], vox [n]) of every segment (Sec. 4.1)."""
        n = len(seg["x0"])
        cols = np.stack([np.asarray(seg[k], dtype=np.float32) for k in
                         ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")], axis=1)
        cols = np.ascontiguousarray(cols)
        npe = np.zeros((n, self.n_det))
        tick = np.zeros(n, np.int32)
        vox = np.zeros(n, np.int32)
        for j in range(n):
            row = np.zeros(self.n_det)
            t = C.c_int32()
            v = C.c_int32()
            self.lib.ora_light_segment(C.byref(self.c), C.byref(self.l), _p(cols[j], C.c_float),
                                       float(dr["QR"][j]), int(dr["anode"][j]), _p(self.vis, C.c_double),
                                       _p(self.eff, C.c_double), _p(row, C.c_double), C.byref(t), C.byref(v))
            npe[j] = row
            tick[j] = t.value
            vox[j] = v.value
        return npe, tick, vox

    def photocurrent(self, npe, tick, vox, anode, det: int):
        """Expected photoelectrons per tick of global photosensor det (Sec. 4.2)."""
        npe = np.ascontiguousarray(npe, dtype=np.float64)
        tick = np.ascontiguousarray(tick, dtype=np.int32)
        vox = np.ascontiguousarray(vox, dtype=np.int32)
        anode = np.ascontiguousarray(anode, dtype=np.int32)
        I = np.zeros(self.l.n_ticks)
        self.lib.ora_light_photocurrent(C.byref(self.l), len(tick), _p(npe, C.c_double), _p(tick, C.c_int32),
                                        _p(vox, C.c_int32), _p(anode, C.c_int32), _p(self.tdist, C.c_double),
                                        det // self.n_det, det % self.n_det, _p(I, C.c_double))
        return I

    def truth(self, tick, vox):
        """Mean arrival time (us) of each segment's photoelectrons at each photosensor (Sec. 4.4)."""
        tick = np.ascontiguousarray(tick, dtype=np.int32)
        vox = np.ascontiguousarray(vox, dtype=np.int32)
        out = np.zeros((len(tick), self.n_det))
        self.lib.ora_light_truth(C.byref(self.l), len(tick), _p(tick, C.c_int32), _p(vox, C.c_int32),
                                 _p(self.tdist, C.c_double), _p(out, C.c_double))
        return out

    def scintillation(self, I):
        I = np.ascontiguousarray(I, dtype=np.float64)
        S = np.zeros(self.l.n_ticks)
        self.lib.ora_light_scintillation(C.byref(self.l), _p(I, C.c_double), _p(S, C.c_double))
        return S

    def fluctuate(self, S, det: int, event_id: int = 0):
        S = np.ascontiguousarray(S, dtype=np.float64)
        n = np.zeros(self.l.n_ticks)
        mg = np.zeros(self.l.n_ticks)
        self.lib.ora_light_fluctuate(C.byref(self.c), C.byref(self.l), event_id, int(det), _p(S, C.c_double),
                                     _p(n, C.c_double), _p(mg, C.c_double))
        return n, mg

    def electronics(self, n, det: int, event_id: int = 0):
        """(V [n_ticks], samples, ADC codes, code margins) of global photosensor det."""
        n = np.ascontiguousarray(n, dtype=np.float64)
        T = self.l.n_ticks
        V = np.zeros(T)
        vs = np.zeros(self.n_samples)
        code = np.zeros(self.n_samples, np.int32)
        mg = np.zeros(self.n_samples)
        self.lib.ora_light_electronics(C.byref(self.c), C.byref(self.l), event_id, int(det),
                                       float(self.gain[det % self.n_det]), _p(n, C.c_double),
                                       _p(self.resp, C.c_double), _p(self.amp, C.c_double), float(self.ratio),
                                       self.n_samples, _p(V, C.c_double), _p(vs, C.c_double), _p(code, C.c_int32),
                                       _p(mg, C.c_double))
        return V, vs, code, mg
