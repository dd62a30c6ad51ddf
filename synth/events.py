"""Seeded synthetic energy-deposit segments S_i = (r_s, r_e, E).

The paper feeds larnd-sim with edep-sim (Geant4) segments (Sec. 2): short
straight pieces of particle trails with 4-vector end points and the deposited
energy.  Neither edep-sim nor its inputs exist here, so these generators
produce segments with the shapes, sizes and dE/dx distributions of the
paper's workloads: straight muons of 0.5 cm steps with Landau-like (Moyal)
dE/dx, short highly-ionising protons, and an EM-shower-like cloud of short
segments.  Units: cm, us, MeV.  Segments are returned as a dict of FP32
structure-of-arrays columns x0, y0, z0, t0, x1, y1, z1, t1, dE.

Generators split segments at the cathode and at module boundaries (a segment
is attributed to one drift volume by its midpoint).  Nothing here computes a
step of the simulated method.
"""
from __future__ import annotations

import numpy as np

from .params import geometry

C_CM_US = 2.99792458e4  # speed of light, cm/us
COLS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")


def moyal_dedx(rng, n, mpv=2.1, lo=None, hi=50.0):
    """Moyal-distributed dE/dx (mode ``mpv``, width 0.1*mpv), clamped."""
    z = rng.standard_normal(n)
    lam = -np.log(np.maximum(z * z, 1e-300))
    v = mpv + 0.1 * mpv * lam
    return np.clip(v, 0.5 * mpv if lo is None else lo, hi)


def isotropic(rng, n=None):
    """Unit vectors uniform on the sphere."""
    shape = (3,) if n is None else (n, 3)
    v = rng.standard_normal(shape)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def straight_track(start, direction, length, step, dedx, t0=0.0):
    """Segments of a straight track cut every ``step`` cm (last one shorter).

    ``dedx`` is a scalar or an array with one value per segment.
    """
    n = max(1, int(np.ceil(length / step - 1e-9)))
    s = np.minimum(np.arange(n + 1, dtype=np.float64) * step, length)
    d = np.asarray(direction, dtype=np.float64)
    p = np.asarray(start, dtype=np.float64)[None, :] + s[:, None] * d[None, :]
    t = t0 + s / C_CM_US
    seg_len = np.diff(s)
    dedx = np.broadcast_to(np.asarray(dedx, dtype=np.float64), (n,))
    return dict(x0=p[:-1, 0], y0=p[:-1, 1], z0=p[:-1, 2], t0=t[:-1],
                x1=p[1:, 0], y1=p[1:, 1], z1=p[1:, 2], t1=t[1:], dE=dedx * seg_len)


def concat(parts):
    return {k: np.concatenate([np.asarray(p[k], dtype=np.float64) for p in parts]) for k in COLS}


def split_at_planes(seg, planes):
    """Split segments crossing axis-aligned planes [(axis, value), ...].

    Energy is shared in proportion to length, time linearly.
    """
    seg = {k: np.asarray(v, dtype=np.float64) for k, v in seg.items()}
    ax = {"x": ("x0", "x1"), "y": ("y0", "y1"), "z": ("z0", "z1")}
    for axis, val in planes:
        a0, a1 = ax[axis]
        c0 = seg[a0] - val
        c1 = seg[a1] - val
        cross = (c0 * c1) < 0
        if not np.any(cross):
            continue
        idx = np.nonzero(cross)[0]
        f = c0[idx] / (c0[idx] - c1[idx])
        mid = {}
        for a, b in (("x0", "x1"), ("y0", "y1"), ("z0", "z1"), ("t0", "t1")):
            mid[a] = seg[a][idx] + f * (seg[b][idx] - seg[a][idx])
        second = {k: seg[k][idx].copy() for k in COLS}
        for a, b in (("x0", "x1"), ("y0", "y1"), ("z0", "z1"), ("t0", "t1")):
            second[a] = mid[a]
            seg[b][idx] = mid[a]
        second["dE"] = seg["dE"][idx] * (1.0 - f)
        seg["dE"][idx] = seg["dE"][idx] * f
        # keep the two halves adjacent: insert the second half after the first
        order = np.arange(len(seg["x0"]) + len(idx))
        out = {}
        pos = idx + np.arange(1, len(idx) + 1)
        keep = np.ones(len(order), dtype=bool)
        keep[pos] = False
        for k in COLS:
            col = np.empty(len(order), dtype=np.float64)
            col[keep] = seg[k]
            col[pos] = second[k]
            out[k] = col
        seg = out
    return seg


def boundary_planes(cfg):
    g = geometry(cfg)
    planes = [("z", g["drift"] * k) for k in range(1, cfg["n_tpc"])]
    planes += [("x", g["mod_w"] * k) for k in range(1, cfg["n_mod_x"])]
    planes += [("y", g["mod_h"] * k) for k in range(1, cfg["n_mod_y"])]
    return planes


def to_f32(seg):
    return {k: np.ascontiguousarray(np.asarray(seg[k], dtype=np.float32)) for k in COLS}


def tile_muon(cfg, seed, n_seg=200, step=0.5, mpv=2.1):
    """A straight muon of ``n_seg`` x ``step`` cm, centred in the volume, isotropic direction."""
    rng = np.random.default_rng(seed)
    g = geometry(cfg)
    centre = np.array([g["x_max"] / 2, g["y_max"] / 2, g["z_max"] / 2])
    d = isotropic(rng)
    length = n_seg * step
    start = centre - 0.5 * length * d
    seg = straight_track(start, d, length, step, moyal_dedx(rng, n_seg, mpv))
    return to_f32(split_at_planes(seg, boundary_planes(cfg)))


def interaction(cfg, rng, n_target=20000, vertex=None, t0=0.0, mpv=2.1):
    """Neutrino-like interaction: one long muon, 3-6 protons, an EM-like cloud.

    The cloud fills the segment count up to about ``n_target``.
    """
    g = geometry(cfg)
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([g["x_max"], g["y_max"], g["z_max"]])
    if vertex is None:
        vertex = lo + (hi - lo) * (0.2 + 0.6 * rng.random(3))
    parts = []
    # muon of ~150 cm at 0.5 cm steps
    mu_len = rng.uniform(120.0, 180.0)
    n_mu = int(np.ceil(mu_len / 0.5))
    parts.append(straight_track(vertex, isotropic(rng), mu_len, 0.5,
                                moyal_dedx(rng, n_mu, mpv), t0))
    # 3-6 protons, 3-20 cm at 0.1 cm steps, dE/dx 5-20 MeV/cm
    for _ in range(int(rng.integers(3, 7))):
        L = rng.uniform(3.0, 20.0)
        n = int(np.ceil(L / 0.1))
        parts.append(straight_track(vertex, isotropic(rng), L, 0.1,
                                    rng.uniform(5.0, 20.0, n), t0))
    n_done = sum(len(p["x0"]) for p in parts)
    n_em = max(0, n_target - n_done)
    if n_em:
        axis = isotropic(rng)
        # two directions orthogonal to the shower axis
        tmp = np.array([1.0, 0.0, 0.0]) if abs(axis[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        e1 = np.cross(axis, tmp)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(axis, e1)
        centre = vertex + 20.0 * axis
        pos = (centre[None, :] + rng.normal(0.0, 15.0, n_em)[:, None] * axis[None, :]
               + rng.normal(0.0, 3.0, n_em)[:, None] * e1[None, :]
               + rng.normal(0.0, 3.0, n_em)[:, None] * e2[None, :])
        L = np.exp(rng.uniform(np.log(0.1), np.log(1.0), n_em))
        d = isotropic(rng, n_em)
        p1 = pos + L[:, None] * d
        ts = t0 + np.linalg.norm(pos - vertex[None, :], axis=1) / C_CM_US
        parts.append(dict(x0=pos[:, 0], y0=pos[:, 1], z0=pos[:, 2], t0=ts,
                          x1=p1[:, 0], y1=p1[:, 1], z1=p1[:, 2], t1=ts + L / C_CM_US,
                          dE=moyal_dedx(rng, n_em, mpv) * L))
    return concat(parts)


def module_event(cfg, seed, n_target=20000):
    """One interaction of ~``n_target`` segments in one module (t0 = 0)."""
    rng = np.random.default_rng(seed)
    seg = interaction(cfg, rng, n_target)
    return to_f32(split_at_planes(seg, boundary_planes(cfg)))


def batch_events(cfg, seed, n_events, lo=1.0e3, hi=2.0e5):
    """``n_events`` interactions with segment counts log-uniform in [lo, hi]
    (the module-event mixture scaled by its size), each split at the cathode."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_events)).astype(np.int64)
    out = []
    for n in sizes:
        seg = interaction(cfg, rng, int(n))
        out.append(to_f32(split_at_planes(seg, boundary_planes(cfg))))
    return out


def rock_muon(cfg, rng, t0):
    """A straight muon crossing the whole module array, mostly along x."""
    g = geometry(cfg)
    d = np.array([1.0, rng.normal(0, 0.15), rng.normal(0, 0.15)])
    d /= np.linalg.norm(d)
    y = rng.uniform(0.05, 0.95) * g["y_max"]
    z = rng.uniform(0.05, 0.95) * g["z_max"]
    start = np.array([-1.0, y, z])
    length = (g["x_max"] + 2.0) / d[0]
    n = int(np.ceil(length / 0.5))
    return straight_track(start, d, length, 0.5, moyal_dedx(rng, n, 2.1), t0)


def spill_event(cfg, seed, n_interactions=50, n_rock=100, n_per=20000, t_spill_us=10.0):
    """A beam spill: ``n_interactions`` interactions plus ``n_rock`` rock muons, t0 ~ U[0, t_spill]."""
    rng = np.random.default_rng(seed)
    g = geometry(cfg)
    parts = []
    for _ in range(n_interactions):
        vtx = np.array([g["x_max"], g["y_max"], g["z_max"]]) * (0.05 + 0.9 * rng.random(3))
        parts.append(interaction(cfg, rng, n_per, vertex=vtx, t0=rng.uniform(0, t_spill_us)))
    for _ in range(n_rock):
        parts.append(rock_muon(cfg, rng, rng.uniform(0, t_spill_us)))
    return to_f32(split_at_planes(concat(parts), boundary_planes(cfg)))


def scatter_event(cfg, seed, n_seg, max_len=1.0, mpv=2.1, t_range=(0.0, 0.0)):
    """``n_seg`` independent short segments spread over the whole detector.

    Used by parity tests: many anodes, tiles and drift distances at once.
    """
    rng = np.random.default_rng(seed)
    g = geometry(cfg)
    pos = rng.random((n_seg, 3)) * np.array([g["x_max"], g["y_max"], g["z_max"]])
    L = np.exp(rng.uniform(np.log(0.02), np.log(max_len), n_seg))
    d = isotropic(rng, n_seg)
    p1 = pos + L[:, None] * d
    t0 = rng.uniform(t_range[0], t_range[1], n_seg) if t_range[1] > t_range[0] else np.zeros(n_seg)
    seg = dict(x0=pos[:, 0], y0=pos[:, 1], z0=pos[:, 2], t0=t0,
               x1=p1[:, 0], y1=p1[:, 1], z1=p1[:, 2], t1=t0 + L / C_CM_US,
               dE=moyal_dedx(rng, n_seg, mpv) * L)
    return to_f32(split_at_planes(seg, boundary_planes(cfg)))


def n_segments(seg) -> int:
    return int(len(seg["x0"]))
