"""Pins of the oracle's steps after the front end: the interval of ticks a
hit digitises and the per-segment charge truth built on it (Sec. 3.4 with the
truth scheme of Sec. 4.4 applied to the charge readout), hits -> 3-D points
(Sec. 6, inverse of Eq. (drift)) and dQ/dx along a known straight track.

Each pin ties the oracle function to something other than itself: the front
end's own CSA charge, the response table row of a point charge, the drift
time of ora_quench_drift, the pixel map, and closed forms.
"""
import numpy as np
import pytest

import oracle
from synth import events, params, response

KEYS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")


def _seg(rows):
    a = np.asarray(rows, dtype=np.float32)
    return {k: np.ascontiguousarray(a[:, i]) for i, k in enumerate(KEYS)}


def _quiet(**over):
    c = params.tile_config(sigma_reset_e=0.0, sigma_disc_e=0.0, sigma_unc_e=0.0, n_ticks=2000)
    c.update(over)
    return c


@pytest.mark.parametrize("periodic", [0, 97, 400])
def test_intervals_hold_the_csa_charge(periodic):
    """Noise off: a hit's digitised charge is exactly the current summed over
    its interval (the CSA charge since its last reset)."""
    cfg = _quiet(periodic_reset_ticks=periodic)
    o = oracle.Oracle(cfg, params.LUT)
    rng = np.random.default_rng(7 + periodic)
    I = np.zeros(2000)
    for c in rng.integers(0, 1900, 25):
        I[c:c + 60] += rng.random(60) * rng.choice([40.0, 400.0])
    r = o.electronics(4321, I)
    assert len(r["t_cross"]) >= 5
    k0, k1 = o.hit_intervals(r["t_cross"], r["t_adc"])
    cs = np.concatenate([[0.0], np.cumsum(I)])
    got = cs[k1 + 1] - cs[k0]
    assert np.allclose(got, r["q"], rtol=1e-12, atol=1e-9)
    assert np.all(k0 <= r["t_cross"]) and np.all(k1 == r["t_adc"])
    if periodic:
        # some interval must start at a periodic reset rather than after a hit
        after_hit = np.concatenate([[0], r["t_adc"][:-1] + 1])
        assert np.any(k0 != after_hit)


def test_truth_sums_to_the_signal_and_the_csa_charge():
    """Per-segment charges of each hit add up to the interval sum of the
    pixel's whole current (linearity of Eq. (current)); with the front-end
    noise off that sum is the hit's digitised charge."""
    cfg = params.small_config(sigma_reset_e=0.0, sigma_disc_e=0.0, sigma_unc_e=0.0, thr_e=2000.0)
    seg = events.scatter_event(cfg, 11, 12, max_len=0.6)
    lut64 = response.lut_for(cfg, params.LUT)
    o = oracle.Oracle(cfg, params.LUT, lut64)
    d = o.quench_drift(seg)
    pix, _, _, _ = o.pixel_map(seg, d)
    n_checked = 0
    for p, segs in sorted(pix.items()):
        I = o.pixel_current(seg, d, p, segs, event_id=3)
        r = o.electronics(p, I, event_id=3)
        if len(r["t_cross"]) == 0:
            continue
        Q, qs, k0, k1 = o.hit_truth(seg, d, p, segs, r["t_cross"], r["t_adc"], event_id=3)
        assert Q.shape == (len(r["t_cross"]), len(segs))
        assert np.allclose(Q.sum(axis=1), qs, rtol=1e-10, atol=1e-7)
        assert np.allclose(qs, r["q"], rtol=1e-10, atol=1e-6)
        n_checked += len(qs)
        if n_checked > 12:
            break
    assert n_checked > 3


def test_truth_of_point_charges_is_a_table_row_sum():
    """Two point charges on one pixel at different depths (exact binary
    geometry, sigma = 0): the charge each puts in an interval is its Q_a times
    the sum of the table row over the ticks of the interval."""
    cfg = dict(params.tile_config(pitch_cm=0.46875, vdrift_cm_us=0.125, tick_us=0.125,
                                  diff_long_cm2_s=0.0, diff_tran_cm2_s=0.0, n_ticks=256, lifetime_us=1e9))
    lut_par = dict(nb=45, nt=64, bins_per_pitch=30, z0_cm=0.1)
    rng = np.random.default_rng(5)
    lut = rng.random((45, 45, 64))
    o = oracle.Oracle(cfg, lut_par, lut)
    p, h = 0.46875, 0.46875 / 30
    xc, yc = 10.5 * p, 20.5 * p
    pts = [((3, 8), 1.0), ((20, 2), 3.0)]           # (node offset (bx, by), depth cm)
    rows = []
    for (bx, by), z in pts:
        x, y = xc + (bx + 0.5) * h, yc - (by + 0.5) * h
        rows.append((x, y, z - 2 ** -12, 0.0, x, y, z + 2 ** -12, 0.0, 1.0))
    seg = _seg(rows)
    d = o.quench_drift(seg)
    pixel = 20 * 70 + 10
    t_cross = np.array([40, 120, 170], np.int32)
    t_adc = np.array([70, 150, 200], np.int32)
    Q, qs, k0, k1 = o.hit_truth(seg, d, pixel, [0, 1], t_cross, t_adc)
    assert list(k0) == [0, 71, 151] and list(k1) == [70, 150, 200]
    for j, ((bx, by), z) in enumerate(pts):
        A = int(z / 0.125 / 0.125)                  # arrival tick
        for hh in range(3):
            ks = np.arange(k0[hh], k1[hh] + 1)
            jj = ks - A + 64 - 1
            ok = (jj >= 0) & (jj < 64)
            exp = d["Qa"][j] * lut[bx, by, jj[ok]].sum()
            assert Q[hh, j] == pytest.approx(exp, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("tpc", [0, 1])
def test_hit_point_inverts_the_drift(tpc):
    """A point charge at depth z0 and time t0 arrives at t0 + t_drift
    (ora_quench_drift); the hit point at that tick has z = z0 and the x-y of
    the pixel containing the charge (the pixel map's nearest pixel)."""
    cfg = dict(params.tile_config(pitch_cm=0.46875, vdrift_cm_us=0.125, tick_us=0.125, n_ticks=4096,
                                  diff_long_cm2_s=0.0, diff_tran_cm2_s=0.0, lifetime_us=1e9,
                                  t_window0_us=-2.0))
    cfg["n_tpc"] = 2
    o = oracle.Oracle(cfg, params.LUT)
    D = float(np.float32(cfg["drift_len_cm"]))
    rng = np.random.default_rng(31 + tpc)
    for _ in range(6):
        x0 = float(rng.uniform(3, 28))
        y0 = float(rng.uniform(3, 28))
        depth = float(rng.integers(8, 200)) * 0.125 * 0.125          # drift a whole number of ticks
        z0 = depth if tpc == 0 else 2 * D - depth
        t0 = float(rng.integers(0, 40)) * 0.125
        seg = _seg([(x0, y0, z0 - 2 ** -14, t0, x0, y0, z0 + 2 ** -14, t0, 1.0)])
        d = o.quench_drift(seg)
        assert d["anode"][0] == tpc
        k = (t0 + d["t_drift"][0] - cfg["t_window0_us"]) / 0.125
        assert k == int(k)
        ids, mg = o.map_segment(seg, d, 0)
        pix = int(ids[np.argmax(mg)])
        pt = o.hit_points([pix], [int(k)], t_event=t0)[0]
        assert pt[2] == pytest.approx(z0, abs=1e-9)
        assert abs(pt[0] - x0) <= 0.5 * 0.46875 + 1e-12 and abs(pt[1] - y0) <= 0.5 * 0.46875 + 1e-12


def test_track_dqdx_closed_form():
    """Points every delta along a track (charge c each, off-axis by less than
    r_max): every piece of length dx holds dx / delta points; points beyond
    r_max or before the start are left out."""
    rng = np.random.default_rng(2)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    o = np.array([10.0, 20.0, 5.0])
    v = np.cross(u, [0.0, 0.0, 1.0])
    v /= np.linalg.norm(v)
    delta, dx, nb, c = 0.25, 2.0, 7, 1234.5
    s = (np.arange(int(nb * dx / delta)) + 0.5) * delta
    pts = o + s[:, None] * u + 0.3 * v
    far = o + s[:5, None] * u + 2.0 * v                  # beyond r_max
    w = np.cross(u, v)                                    # across the track, with a z component
    assert abs(w[2]) > 0.5 and 1.2 * np.hypot(w[0], w[1]) < 1.0
    far_z = o + s[:5, None] * u + 1.2 * w                 # beyond r_max, though within it in x-y alone
    before = o - 0.6 * u                                  # s < 0
    P = np.vstack([pts, far, far_z, before[None]])
    q = np.full(len(P), c)
    dq, cnt, mg = oracle.Oracle.track_dqdx(P, q, o, u, dx, nb, 1.0)
    assert np.all(cnt == int(dx / delta))
    assert np.allclose(dq / dx, c / delta, rtol=1e-12)
    # margins: the distance of each point's decisions from their edges, from the construction
    # (arc length s and distance from the axis r): min(|r - r_max|, distance of s to a piece boundary)
    arc = np.concatenate([s, s[:5], s[:5], [-0.6]])
    r = np.concatenate([np.full(len(s), 0.3), np.full(5, 2.0), np.full(5, 1.2), [0.0]])
    edge = np.abs(arc - dx * np.round(arc / dx))
    assert np.allclose(mg, np.minimum(np.abs(r - 1.0), edge), rtol=0, atol=1e-9)
