"""Pins of the oracle's pixel map (Sec. 3.3.2) and induced current (Eq. (current)).

Exact cases use a geometry whose pitch, bin width, drift velocity and tick
are binary fractions, so that sample positions and arrival ticks are exact
and the result must reduce to a table lookup.
"""
import numpy as np
import pytest

import oracle
from synth import params, response

KEYS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")


def _seg(rows):
    a = np.asarray(rows, dtype=np.float32)
    return {k: np.ascontiguousarray(a[:, i]) for i, k in enumerate(KEYS)}


# ---------------------------------------------------------------- pixel map --

def test_cheb_distance_against_dense_sampling():
    L = oracle.lib()
    rng = np.random.default_rng(3)
    t = np.linspace(0.0, 1.0, 200001)
    for _ in range(60):
        a = rng.normal(0, 1, 2)
        b = a + rng.normal(0, 1, 2) * rng.choice([0.0, 1e-3, 1.0])
        p = rng.normal(0, 1, 2)
        d = L.ora_cheb_distance(a[0], a[1], b[0], b[1], p[0], p[1])
        xs = a[0] + t * (b[0] - a[0]) - p[0]
        ys = a[1] + t * (b[1] - a[1]) - p[1]
        brute = np.maximum(np.abs(xs), np.abs(ys)).min()
        assert d <= brute + 1e-12
        assert brute - d < 2e-5 * (1 + np.hypot(*(b - a)))


def _exact_cfg(**over):
    c = params.tile_config(pitch_cm=0.46875, vdrift_cm_us=0.125, tick_us=0.125,
                           diff_long_cm2_s=0.0, diff_tran_cm2_s=0.0, n_ticks=128,
                           lifetime_us=1e9)
    c.update(over)
    return c


LUT_SMALL = dict(nb=45, nt=64, bins_per_pitch=30, z0_cm=0.1)


def test_point_maps_to_3x3():
    # sigma_T = 0: map radius (45 + 1/2) bins = 1.5167 pitch; pixel centres at
    # 0 and 1 pitch are inside, 2 pitch outside.
    o = oracle.Oracle(_exact_cfg(), LUT_SMALL)
    p = 0.46875
    xc, yc = 10.5 * p, 20.5 * p
    seg = _seg([(xc, yc, 1.0 - 2 ** -12, 0, xc, yc, 1.0 + 2 ** -12, 0, 1.0)])
    d = o.quench_drift(seg)
    ids, _ = o.map_segment(seg, d, 0, box=False)
    nx = 70
    exp = sorted((20 + dy) * nx + 10 + dx for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    assert sorted(ids.tolist()) == exp


@pytest.mark.parametrize("mx,my,tpc,ix,iy", [(5, 3, 1, 250, 20), (1, 4, 0, 10, 340), (0, 0, 0, 279, 349)])
def test_point_maps_to_3x3_on_non_square_anodes(mx, my, tpc, ix, iy):
    """The 35-module array of 280 x 350-pixel anodes: a point charge on the
    centre of pixel (ix, iy) of module (mx, my) maps to the 3x3 block of ids
    around it, with ids laid out as anode * 280 * 350 + iy * 280 + ix and
    anode = (my * 7 + mx) * 2 + tpc (clipped at the anode's edges)."""
    cfg = params.spill_config(diff_tran_cm2_s=0.0, diff_long_cm2_s=0.0)
    o = oracle.Oracle(cfg, params.LUT)
    p = float(np.float32(0.4434))
    nx, ny = 280, 350
    x = mx * nx * p + (ix + 0.5) * p
    y = my * ny * p + (iy + 0.5) * p
    z = 10.0 if tpc == 0 else 50.0
    seg = _seg([(x, y, z - 2 ** -12, 0, x, y, z + 2 ** -12, 0, 1.0)])
    d = o.quench_drift(seg)
    anode = (my * 7 + mx) * 2 + tpc
    assert d["anode"][0] == anode
    ids, _ = o.map_segment(seg, d, 0, box=False)
    exp = sorted(anode * nx * ny + (iy + dy) * nx + ix + dx for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if 0 <= ix + dx < nx and 0 <= iy + dy < ny)
    assert sorted(ids.tolist()) == exp


def test_a_segment_induces_only_on_its_own_anode():
    """Charge drifts to the anode of its own drift volume: a segment of the
    second volume listed for the pixel of the first anode directly below it
    induces nothing there, and a current on its own anode's pixel."""
    cfg = params.small_config(n_ticks=4000, t_window0_us=-200.0)
    o = oracle.Oracle(cfg, params.LUT, response.lut_for(cfg, params.LUT))
    p = float(np.float32(0.4434))
    x, y = 20.5 * p, 30.5 * p
    seg = _seg([(x, y, 40.0, 0, x + 0.2, y, 40.5, 0, 1.0)])            # TPC 1 (anode at z = 60)
    d = o.quench_drift(seg)
    assert d["anode"][0] == 1
    below = 0 * o.npx_x * o.npx_y + 30 * o.npx_x + 20                     # the same pixel of anode 0
    own = 1 * o.npx_x * o.npx_y + 30 * o.npx_x + 20
    assert not np.any(o.pixel_current(seg, d, below, [0]))
    assert np.any(o.pixel_current(seg, d, own, [0]))


def test_axis_parallel_segment_maps_4x3():
    o = oracle.Oracle(_exact_cfg(), LUT_SMALL)
    p = 0.46875
    xc, yc = 10.5 * p, 20.5 * p
    seg = _seg([(xc, yc, 1.0, 0, xc + p, yc, 1.0, 0, 1.0)])
    d = o.quench_drift(seg)
    ids, _ = o.map_segment(seg, d, 0)
    exp = sorted((20 + dy) * 70 + 10 + dx for dy in (-1, 0, 1) for dx in (-1, 0, 1, 2))
    assert sorted(ids.tolist()) == exp


@pytest.mark.parametrize("box", [True, False])
def test_boundary_distance_counts_as_mapped(box):
    """A pixel whose centre lies exactly R_map from the segment is mapped, in
    the box-restricted map and in the brute force over the whole anode."""
    o = oracle.Oracle(_exact_cfg(), LUT_SMALL)
    p = 0.46875
    R = o.map_radius(0.0)
    assert R == 45.5 * p / 30
    xc, yc = 10.5 * p, 20.5 * p
    # a point exactly R to the right of pixel (10, 20): (10,20) mapped, (9,20) not
    seg = _seg([(xc + R, yc, 1.0 - 2 ** -12, 0, xc + R, yc, 1.0 + 2 ** -12, 0, 1.0)])
    d = o.quench_drift(seg)
    ids, mg = o.map_segment(seg, d, 0, box=box)
    pid = 20 * 70 + 10
    assert pid in ids.tolist()
    assert mg[ids.tolist().index(pid)] == 0.0
    assert 20 * 70 + 9 not in ids.tolist()


def test_pixel_side_map_agrees_with_the_segment_side():
    """The map read per pixel (segments_for_pixel, pair_margin: brute force
    over the segments) equals the map read per segment; a pixel exactly R_map
    away is mapped (margin 0), and a pixel of the other anode is never mapped
    (margin -inf), whatever its x-y distance."""
    from synth import events
    cfg = params.small_config()
    o = oracle.Oracle(cfg, params.LUT)
    seg = events.scatter_event(cfg, 9, 25, max_len=0.8)
    d = o.quench_drift(seg)
    pix, _, _, _ = o.pixel_map(seg, d)
    for p in sorted(pix)[::7]:
        segs, mg = o.segments_for_pixel(seg, d, p)
        assert segs.tolist() == pix[p] and np.all(mg >= 0)
    # the boundary case of test_boundary_distance_counts_as_mapped, read per pixel
    o2 = oracle.Oracle(_exact_cfg(n_tpc=2), LUT_SMALL)            # two drift volumes: anodes 0 and 1
    p_, R = 0.46875, o2.map_radius(0.0)
    xc, yc = 10.5 * p_, 20.5 * p_
    seg2 = _seg([(xc + R, yc, 1.0 - 2 ** -12, 0, xc + R, yc, 1.0 + 2 ** -12, 0, 1.0)])
    d2 = o2.quench_drift(seg2)
    segs, mg = o2.segments_for_pixel(seg2, d2, 20 * 70 + 10)
    assert segs.tolist() == [0] and mg.tolist() == [0.0]
    assert o2.segments_for_pixel(seg2, d2, 20 * 70 + 9)[0].tolist() == []
    other = 1 * 70 * 70 + 20 * 70 + 10                          # the same pixel of anode 1
    assert d2["anode"][0] == 0 and o2.pair_margin(seg2, d2, 0, other) == -np.inf


def test_box_restricted_map_equals_full_brute_force():
    cfg = params.small_config()
    o = oracle.Oracle(cfg, params.LUT)
    from synth import events
    seg = events.scatter_event(cfg, 5, 120, max_len=1.0)
    d = o.quench_drift(seg)
    for s in range(len(seg["x0"])):
        a, ma = o.map_segment(seg, d, s, box=False)
        b, mb = o.map_segment(seg, d, s, box=True)
        assert np.array_equal(a, b) and np.array_equal(ma, mb)


def test_map_contains_every_pixel_with_current():
    cfg = params.small_config(n_ticks=2000)
    o = oracle.Oracle(cfg, params.LUT, response.lut_for(cfg, params.LUT))
    rng = np.random.default_rng(11)
    rows = []
    for _ in range(3):
        x, y, z = 10 + 40 * rng.random(), 10 + 40 * rng.random(), 5 + 50 * rng.random()
        v = rng.normal(size=3)
        v *= 0.05 / np.linalg.norm(v)
        rows.append((x, y, z, 0, x + v[0], y + v[1], z + v[2], 0, 0.1))
    seg = _seg(rows)
    d = o.quench_drift(seg)
    nx = o.npx_x
    for s in range(len(rows)):
        ids, _ = o.map_segment(seg, d, s)
        mapped = set(ids.tolist())
        g = int(d["anode"][s])
        base = g * nx * o.npx_y
        cx = int((seg["x0"][s]) / 0.4434)
        cy = int((seg["y0"][s]) / 0.4434)
        for iy in range(cy - 4, cy + 5):
            for ix in range(cx - 4, cx + 5):
                pid = base + iy * nx + ix
                I = o.pixel_current(seg, d, pid, [s])
                if np.any(I != 0):
                    assert pid in mapped, (s, ix, iy)


# ----------------------------------------------------------- induced current --

def _point(xc, yc, dx, dy, z, t=0.0):
    x = xc + dx
    y = yc + dy
    return (x, y, z - 2 ** -12, t, x, y, z + 2 ** -12, t, 1.0)


@pytest.mark.parametrize("bx,by,sx,sy", [(7, 12, 1, 1), (0, 44, -1, 1), (30, 3, 1, -1), (44, 0, -1, -1)])
def test_point_charge_reads_table_row(bx, by, sx, sy):
    """sigma = 0, one point at a node offset, integer arrival: I[k] = q R[bx, by, k - A + L - 1]."""
    cfg = _exact_cfg()
    rng = np.random.default_rng(bx * 100 + by)
    lut = rng.random((45, 45, 64))          # any table: checks indexing and orientation
    o = oracle.Oracle(cfg, LUT_SMALL, lut)
    p, h = 0.46875, 0.46875 / 30
    xc, yc = 10.5 * p, 20.5 * p
    seg = _seg([_point(xc, yc, sx * (bx + 0.5) * h, sy * (by + 0.5) * h, 1.0)])
    d = o.quench_drift(seg)
    assert d["n_samples"][0] == 1
    I = o.pixel_current(seg, d, 20 * 70 + 10, [0])
    A = 64                                   # 1 cm / 0.125 cm/us / 0.125 us
    exp = np.zeros(128)
    for k in range(128):
        j = k - A + 64 - 1
        if 0 <= j < 64:
            exp[k] = d["Qa"][0] * lut[bx, by, j]
    assert np.array_equal(I, exp)


def test_interpolation_is_superposition_of_nodes():
    """Between nodes and between ticks the current is the weighted sum of node currents."""
    cfg = _exact_cfg()
    lut = np.random.default_rng(5).random((45, 45, 64))
    o = oracle.Oracle(cfg, LUT_SMALL, lut)
    p, h = 0.46875, 0.46875 / 30
    xc, yc = 10.5 * p, 20.5 * p
    pid = 20 * 70 + 10

    def cur(dx, dy, z):
        seg = _seg([_point(xc, yc, dx, dy, z)])
        d = o.quench_drift(seg)
        return o.pixel_current(seg, d, pid, [0]) / d["Qa"][0]   # per unit charge

    # x halfway (1/4 of a bin) between nodes 5 and 6, y on node 9, arrival 64 + 1/4
    z_int, z_q = 1.0, 1.0 + 0.25 * 0.125 * 0.125
    got = cur(5.75 * h, 9.5 * h, z_q)
    base = {}
    for b in (5, 6):
        for z, tag in ((z_int, 0), (1.0 + 0.125 * 0.125, 1)):
            base[(b, tag)] = cur((b + 0.5) * h, 9.5 * h, z)
    exp = (0.75 * (0.75 * base[(5, 0)] + 0.25 * base[(5, 1)])
           + 0.25 * (0.75 * base[(6, 0)] + 0.25 * base[(6, 1)]))
    assert np.allclose(got, exp, rtol=1e-13, atol=1e-15)
    # inside half a bin of the centre the folded table reads node 0
    assert np.array_equal(cur(0.25 * h, 9.5 * h, z_int), cur(0.5 * h, 9.5 * h, z_int))
    assert np.array_equal(cur(-0.25 * h, 9.5 * h, z_int), cur(0.5 * h, 9.5 * h, z_int))
    # beyond the last node the response vanishes
    assert not np.any(cur(45.5 * h, 9.5 * h, z_int))


def test_time_and_space_shifts():
    cfg = _exact_cfg(diff_tran_cm2_s=8.8, diff_long_cm2_s=4.0)
    lut = np.random.default_rng(9).random((45, 45, 64))
    o = oracle.Oracle(cfg, LUT_SMALL, lut)
    p = 0.46875
    row = (5.1, 9.3, 2.0, 0.0, 5.3, 9.2, 2.1, 0.0, 0.4)
    seg = _seg([row])
    d = o.quench_drift(seg)
    pid = int(9.3 / p) * 70 + int(5.1 / p)
    I0 = o.pixel_current(seg, d, pid, [0])
    # t0 shifted by 5 ticks: the current moves by exactly 5 ticks
    r2 = list(row)
    r2[3] += 5 * 0.125
    r2[7] += 5 * 0.125
    seg2 = _seg([r2])
    I1 = o.pixel_current(seg2, o.quench_drift(seg2), pid, [0])
    assert np.allclose(I1[5:], I0[:-5], rtol=1e-12, atol=1e-14)
    # translated by one pitch in x: same current one pixel to the right
    r3 = list(row)
    r3[0] += p
    r3[4] += p
    seg3 = _seg([r3])
    I2 = o.pixel_current(seg3, o.quench_drift(seg3), pid + 1, [0])
    assert np.allclose(I2, I0, rtol=1e-5, atol=1e-12 * np.abs(I0).max())


def test_charge_conservation():
    """Sec. 3.3.1: each response series integrates to one electron, so the
    current summed over pixels and ticks equals the collected charge."""
    cfg = params.small_config(n_ticks=4000, t_window0_us=-200.0)
    lut = response.lut_for(cfg, params.LUT)            # FP64 table
    o = oracle.Oracle(cfg, params.LUT, lut)
    rng = np.random.default_rng(21)
    rows = []
    for z in (2.0, 14.0, 29.0, 44.0):
        x, y = 10 + 30 * rng.random(), 10 + 30 * rng.random()
        v = rng.normal(size=3)
        v *= 0.2 / np.linalg.norm(v)
        rows.append((x, y, z, 0, x + v[0], y + v[1], z + v[2], 0, 0.4))
    seg = _seg(rows)
    d = o.quench_drift(seg)
    pix, _, _, _ = o.pixel_map(seg, d)
    total = sum(o.pixel_current(seg, d, p, s).sum() for p, s in pix.items())
    assert abs(total / d["Qa"].sum() - 1.0) < 1e-12


def _interp_table(tab, h, nb):
    """Independent bilinear reader of a folded table: node values at +-(b+1/2)h, zero node at nb."""
    nodes = (np.arange(nb + 1) + 0.5) * h
    full = np.concatenate([-nodes[::-1], nodes])
    ext = np.zeros((nb + 1, nb + 1))
    ext[:nb, :nb] = tab
    unf = np.block([[ext[::-1, ::-1], ext[::-1, :]], [ext[:, ::-1], ext]])
    from scipy.interpolate import RegularGridInterpolator
    return RegularGridInterpolator((full, full), unf, bounds_error=False, fill_value=0.0)


def test_monte_carlo_converges_to_convolution():
    """Eq. (current) approximates the convolution of the response with the
    diffused charge density at the percent level (Sec. 3.3.2): compare the
    per-pixel collected charge and mean arrival tick with a quadrature of
    the continuous integral."""
    cfg = params.small_config(n_ticks=4000, t_window0_us=-200.0, mc_per_sample=48)
    lut = response.lut_for(cfg, params.LUT)
    o = oracle.Oracle(cfg, params.LUT, lut)
    p = 0.4434
    h = p / 30
    row = (20.1, 21.3, 20.0, 0.0, 20.25, 21.45, 20.05, 0.0, 0.5)
    seg = _seg([row])
    d = o.quench_drift(seg)
    sT = d["sigma_T"][0]
    W = _interp_table(lut.sum(axis=2), h, 45)
    M1 = _interp_table((lut * np.arange(1950)).sum(axis=2), h, 45)
    # quadrature: midpoint along the segment x Gauss-Hermite transverse
    gh, gw = np.polynomial.hermite_e.hermegauss(24)
    gw = gw / gw.sum()
    u = (np.arange(400) + 0.5) / 400
    s = {k: np.float64(seg[k][0]) for k in KEYS}
    xs = s["x0"] + u * (s["x1"] - s["x0"])
    ys = s["y0"] + u * (s["y1"] - s["y0"])
    zs = s["z0"] + u * (s["z1"] - s["z0"])
    a = ((s["t0"] + zs / cfg["vdrift_cm_us"]) - cfg["t_window0_us"]) / np.float32(0.1)
    pix, _, _, _ = o.pixel_map(seg, d)
    Qa = d["Qa"][0]
    checked = 0
    for pid, sl in pix.items():
        iy, ix = divmod(pid % (o.npx_x * o.npx_y), o.npx_x)
        xc, yc = (ix + 0.5) * np.float32(p), (iy + 0.5) * np.float32(p)
        X = xs[:, None, None] + sT * gh[None, :, None] - xc
        Y = ys[:, None, None] + sT * gh[None, None, :] - yc
        pts = np.stack([np.broadcast_to(X, (400, 24, 24)), np.broadcast_to(Y, (400, 24, 24))], -1)
        wts = gw[None, :, None] * gw[None, None, :] / 400
        Wv = W(pts)
        q_exp = Qa * (wts * Wv).sum()
        m_exp = Qa * (wts * (Wv * (a[:, None, None] - 1950 + 1) + M1(pts))).sum()
        I = o.pixel_current(seg, d, pid, sl)
        if q_exp < 0.02 * Qa:
            continue
        checked += 1
        assert abs(I.sum() / q_exp - 1) < 0.02
        mean_tick = (np.arange(len(I)) * I).sum() / I.sum()
        # MC standard error of the mean tick at M = 48 is ~0.05-0.1 tick here
        assert abs(mean_tick - m_exp / q_exp) < 0.3
    assert checked >= 3


def test_longitudinal_spread_matches_sigma_L():
    """A point charge drifting 25 cm: the arrival spread of the current adds
    (sigma_L / (v_d tick))^2 to its variance in ticks (Sec. 3.2)."""
    cfg = params.tile_config(diff_tran_cm2_s=0.0, n_ticks=4000, t_window0_us=-200.0,
                             mc_per_sample=4000)
    lut = response.lut_for(cfg, params.LUT)
    o = oracle.Oracle(cfg, params.LUT, lut)
    p = np.float32(0.4434)
    xc, yc = 20.5 * p, 30.5 * p
    z = 25.0
    seg = _seg([(xc + 0.01, yc + 0.02, z - 2 ** -12, 0, xc + 0.01, yc + 0.02, z + 2 ** -12, 0, 1.0)])
    d = o.quench_drift(seg)
    pid = 30 * 70 + 20
    I = o.pixel_current(seg, d, pid, [0])
    k = np.arange(len(I))

    def var(w):
        m = (k * w).sum() / w.sum()
        return ((k - m) ** 2 * w).sum() / w.sum()

    # same point without longitudinal diffusion, arrival smeared uniformly over one tick
    cfg0 = dict(cfg, diff_long_cm2_s=0.0, mc_per_sample=1)
    o0 = oracle.Oracle(cfg0, params.LUT, lut)
    I0 = np.zeros_like(I)
    for f in (np.arange(64) + 0.5) / 64 - 0.5:
        zz = z + f * 0.16 * 0.1
        s0 = _seg([(xc + 0.01, yc + 0.02, zz - 2 ** -12, 0, xc + 0.01, yc + 0.02, zz + 2 ** -12, 0, 1.0)])
        I0 += o0.pixel_current(s0, o0.quench_drift(s0), pid, [0])
    sa2 = (d["sigma_L"][0] / (np.float32(0.16) * np.float32(0.1))) ** 2
    assert abs((var(I) - var(I0)) / (sa2 - 1.0 / 12) - 1) < 0.08


def test_transverse_perturbations_are_clipped():
    """Diffusion offsets are normals clipped at +-clip (reading 15): a point
    charge with sigma_T = one pitch and clip 0.5 reaches no pixel beyond the
    table's reach plus 0.5 sigma_T, in any direction, while the clipped
    offsets do reach pixels beyond the table's reach alone."""
    p, h = 0.46875, 0.46875 / 30
    z = 1.0                                          # 8 us of drift at 0.125 cm/us
    cfg = _exact_cfg(diff_tran_cm2_s=p * p / (2e-6 * z / 0.125), diff_clip_sigma=0.5, mc_per_sample=200)
    o = oracle.Oracle(cfg, LUT_SMALL, np.random.default_rng(4).random((45, 45, 64)) + 0.1)
    xc, yc = 10.5 * p, 20.5 * p
    seg = _seg([_point(xc, yc, 0.0, 0.0, z)])
    d = o.quench_drift(seg)
    sT = float(d["sigma_T"][0])
    assert abs(sT / p - 1.0) < 1e-3
    reach_table = 45.5 * h
    reach = reach_table + 0.5 * sT
    x, y = float(seg["x0"][0]), float(seg["y0"][0])
    beyond_table = 0
    for iy in range(16, 25):
        for ix in range(6, 15):
            dist = max(abs((ix + 0.5) * p - x), abs((iy + 0.5) * p - y))
            I = o.pixel_current(seg, d, iy * 70 + ix, [0])
            if dist > reach + 1e-6:
                assert not np.any(I), (ix, iy)
            elif dist > reach_table + 1e-6 and np.any(I):
                beyond_table += 1
    assert beyond_table >= 8                         # the ring at two pitches, reached only by clipped offsets


def test_isochronous_segment_arrives_as_one_point():
    """Points are spaced evenly along the segment in space and in time
    (Sec. 3.3.2): a segment drifting straight to the anode whose time runs back
    by exactly its extra drift time (t1 - t0 = -(z1 - z0) / v) delivers all of
    its points at one instant, so without diffusion its current per unit charge
    is that of a point charge at its midpoint."""
    cfg = _exact_cfg()
    lut = np.random.default_rng(6).random((45, 45, 64))
    o = oracle.Oracle(cfg, LUT_SMALL, lut)
    p, h = 0.46875, 0.46875 / 30
    xc, yc = 10.5 * p, 20.5 * p
    x, y = xc + 7.3 * h, yc - 11.6 * h
    seg = _seg([(x, y, 1.0, 4.0, x, y, 1.5, 0.0, 1.0)])       # arrival 4 + 8 = 0 + 12 us for every point
    d = o.quench_drift(seg)
    assert d["n_samples"][0] > 100
    pid = 20 * 70 + 10
    I = o.pixel_current(seg, d, pid, [0]) / d["Qa"][0]
    pt = _seg([(x, y, 1.25 - 2 ** -12, 2.0, x, y, 1.25 + 2 ** -12, 2.0, 1.0)])
    dp = o.quench_drift(pt)
    assert dp["n_samples"][0] == 1
    Ip = o.pixel_current(pt, dp, pid, [0]) / dp["Qa"][0]
    assert np.any(Ip)
    np.testing.assert_allclose(I, Ip, rtol=1e-9, atol=1e-12 * np.abs(Ip).max())


def _onset(I):
    nz = np.nonzero(I)[0]
    return int(nz[0]) if len(nz) else len(I)


def test_per_point_transverse_width_bounds_the_reach_along_the_drift():
    """Per-point drift: each point diffuses with sigma_T of its own drift time
    (Eq. (lifetime) and sigma = sqrt(2 D t) at the point), so on a segment
    running away from the anode only the points beyond the depth z* where
    clip sigma_T(z*) covers the gap can reach a pixel two pitches off the
    track: that pixel's current starts no earlier than the response window of
    a charge arriving from z*, while the pixel under the track sees the near
    points from the first ticks."""
    p, h, v, tick = 0.46875, 0.46875 / 30, 0.125, 0.125
    clip, z0, z1 = 1.5, 0.25, 8.0
    DT = (p / clip) ** 2 / (2e-6 * z1 / v)                     # clip sigma_T(z1) = one pitch
    cfg = _exact_cfg(per_point_drift=1, diff_tran_cm2_s=DT, diff_clip_sigma=clip, mc_per_sample=16, n_ticks=1024)
    o = oracle.Oracle(cfg, LUT_SMALL, np.random.default_rng(8).random((45, 45, 64)) + 0.1)
    xc, yc = 10.5 * p, 20.5 * p
    seg = _seg([(xc, yc, z0, 0.0, xc, yc, z1, 0.0, 2.0)])
    d = o.quench_drift(seg)
    gap = 2 * p - 45.5 * h                                      # offset needed to reach the pixel at +2 pitches
    k_sig = 2e-6 * DT / v                                       # sigma_T(z)^2 = k_sig z
    z_star = (gap / clip) ** 2 / k_sig
    assert z0 + 0.5 < z_star < z1 - 0.5
    k_bound = int(np.floor(z_star / v / tick)) - 64 + 1 - 2    # two ticks of margin for the FP32 inputs
    far = o.pixel_current(seg, d, 20 * 70 + 12, [0])
    near = o.pixel_current(seg, d, 20 * 70 + 10, [0])
    assert _onset(far) >= k_bound
    assert np.any(far)
    assert _onset(near) < k_bound - 20


def test_per_point_longitudinal_width_bounds_the_onset():
    """Per-point drift with longitudinal diffusion only: a point at depth z
    arrives no earlier than from z - clip sigma_L(z) (offsets clipped at
    +-clip, sigma_L of the point's own drift time), so the current starts no
    earlier than the response window of the earliest such arrival over the
    segment; a width taken at the midpoint, or unclipped offsets, would bring
    charge from the near end earlier."""
    p, v, tick = 0.46875, 0.125, 0.125
    clip, z0, z1 = 1.5, 4.0, 12.0
    DL = (3.0 / clip) ** 2 / (2e-6 * z1 / v)                     # clip sigma_L(z1) = 3 cm
    cfg = _exact_cfg(per_point_drift=1, diff_long_cm2_s=DL, diff_clip_sigma=clip, mc_per_sample=16, n_ticks=1280)
    o = oracle.Oracle(cfg, LUT_SMALL, np.random.default_rng(9).random((45, 45, 64)) + 0.1)
    xc, yc = 10.5 * p, 20.5 * p
    seg = _seg([(xc, yc, z0, 0.0, xc, yc, z1, 0.0, 2.0)])
    d = o.quench_drift(seg)
    zs = np.linspace(z0, z1, 8001)
    g = zs - clip * np.sqrt(2e-6 * DL / v * zs)                 # earliest depth each point can arrive from
    assert np.all(np.diff(g) > 0) and g[0] > 0                  # earliest at the near end, on the near side of the anode
    k_bound = int(np.floor(g[0] / v / tick)) - 64 + 1 - 2
    I = o.pixel_current(seg, d, 20 * 70 + 10, [0])
    assert _onset(I) >= k_bound
    # the near end's offsets do reach close to the bound (the clip is met)
    assert _onset(I) <= k_bound + 12


def test_per_point_drift_charge_is_the_pointwise_lifetime_sum():
    """Per-point drift: each point carries Q_a/N exp(-(t_mu - t_mid)/tau) with
    t_mu its own drift time (Eq. (lifetime) at the point), so the charge
    collected over all pixels and ticks is that closed-form geometric sum;
    per-segment drift collects Q_a.  Short lifetime (40 us) and no diffusion
    make the difference large."""
    cfg = params.small_config(n_ticks=4000, t_window0_us=-200.0, lifetime_us=40.0, diff_long_cm2_s=0.0,
                              diff_tran_cm2_s=0.0, per_point_drift=1)
    lut = response.lut_for(cfg, params.LUT)
    o = oracle.Oracle(cfg, params.LUT, lut)
    rows = [(15.3, 20.1, 5.0, 0, 15.4, 20.05, 9.0, 0, 8.0),       # 4 cm along the drift, TPC 0
            (30.2, 12.7, 41.0, 0, 30.1, 12.75, 47.5, 0, 9.0)]      # 6.5 cm, TPC 1
    seg = _seg(rows)
    d = o.quench_drift(seg)
    pix, _, _, _ = o.pixel_map(seg, d)
    for s in range(2):
        total = sum(o.pixel_current(seg, d, p, [s]).sum() for p, sl in pix.items() if s in sl)
        z0, z1 = float(seg["z0"][s]), float(seg["z1"][s])
        za = 0.0 if z0 < 30 else 60.0
        N = int(d["n_samples"][s])
        v = float(np.float32(cfg["vdrift_cm_us"]))
        tau = float(np.float32(cfg["lifetime_us"]))
        t_first = abs(z0 + (z1 - z0) * 0.5 / N - za) / v
        dt = (abs(z0 + (z1 - z0) * 1.5 / N - za) - abs(z0 + (z1 - z0) * 0.5 / N - za)) / v
        r = np.exp(-dt / tau)
        expect = d["Qa"][s] / N * np.exp(-(t_first - d["t_drift"][s]) / tau) * (1 - r ** N) / (1 - r)
        assert abs(total / expect - 1.0) < 1e-9, (s, total, expect)
        assert abs(total / d["Qa"][s] - 1.0) > 1e-3          # differs from the per-segment charge
    # the map radius of per-point drift uses the farther end's width: here zero (no diffusion)
    assert np.all(d["sigma_T"] == 0.0)


def test_per_point_drift_reduces_to_per_segment_without_lifetime_and_diffusion():
    base = dict(lifetime_us=1e12, diff_long_cm2_s=0.0, diff_tran_cm2_s=0.0)
    seg = _seg([(12.0, 9.0, 11.0, 0, 12.6, 9.3, 13.2, 0, 1.5)])
    out = []
    for pp in (0, 1):
        cfg = params.small_config(per_point_drift=pp, **base)
        o = oracle.Oracle(cfg, params.LUT, response.lut_for(cfg, params.LUT))
        d = o.quench_drift(seg)
        pix, _, _, _ = o.pixel_map(seg, d)
        out.append({p: o.pixel_current(seg, d, p, s) for p, s in pix.items()})
    assert out[0].keys() == out[1].keys()
    for p in out[0]:
        np.testing.assert_allclose(out[1][p], out[0][p], rtol=1e-9, atol=1e-12)


def test_per_point_drift_map_width_is_the_farther_end():
    cfg = params.small_config(per_point_drift=1)
    o = oracle.Oracle(cfg, params.LUT)
    seg = _seg([(12.0, 9.0, 3.0, 0, 12.6, 9.3, 13.0, 0, 1.5), (12.0, 9.0, 55.0, 0, 12.6, 9.3, 45.0, 0, 1.5)])
    d = o.quench_drift(seg)
    for s, far in ((0, 13.0), (1, 60.0 - 45.0)):
        t = far / float(np.float32(cfg["vdrift_cm_us"]))
        np.testing.assert_allclose(d["sigma_T"][s], np.sqrt(2 * float(np.float32(cfg["diff_tran_cm2_s"])) * 1e-6 * t),
                                   rtol=1e-12)


@pytest.mark.parametrize("bx,by,frac", [(3, 7, 0.3), (10, 0, 0.7), (44, 20, 0.2)])
def test_nearest_lookup_reads_the_nearest_node_and_tick(bx, by, frac):
    """Nearest-bin variant: a point charge 0.3 bin off node (bx, by), arriving
    `frac` of a tick after tick 64, reads that node's table row shifted to the
    nearest tick, exactly."""
    cfg = _exact_cfg(nearest_lut=1)
    lut = np.random.default_rng(bx * 7 + by).random((45, 45, 64))
    o = oracle.Oracle(cfg, LUT_SMALL, lut)
    p, h = 0.46875, 0.46875 / 30
    xc, yc = 10.5 * p, 20.5 * p
    z = 1.0 + frac * 0.125 * 0.125                # arrival tick 64 + frac
    seg = _seg([_point(xc, yc, (bx + 0.5 + 0.3) * h, (by + 0.5 - 0.3) * h, z)])
    d = o.quench_drift(seg)
    assert d["n_samples"][0] == 1
    I = o.pixel_current(seg, d, 20 * 70 + 10, [0])
    A = 64 + (1 if frac >= 0.5 else 0)
    exp = np.zeros(128)
    for k in range(128):
        j = k - A + 64 - 1
        if 0 <= j < 64:
            exp[k] = d["Qa"][0] * lut[bx, by, j]
    assert np.array_equal(I, exp)
    # the point's roundings lie 0.2 bin / 0.2-0.3 tick from their half-way points: a tie
    # within a band of 0.25, none within 0.1
    for band, ties in ((0.1, 0), (0.25, 1)):
        I2, n_ties = o.pixel_current(seg, d, 20 * 70 + 10, [0], tie_band=band)
        assert n_ties == ties and np.array_equal(I2, I)


def test_nearest_lookup_conserves_charge():
    """Nearest-bin variant: the pitch is a whole number of bins, so every
    pixel's nearest node sits at the same sub-bin position and the table's
    partition of unity still holds: charge is conserved."""
    cfg = params.small_config(nearest_lut=1, n_ticks=4000, t_window0_us=-200.0)
    lut = response.lut_for(cfg, params.LUT)
    o = oracle.Oracle(cfg, params.LUT, lut)
    rng = np.random.default_rng(22)
    rows = []
    for z in (3.0, 17.0, 41.0):
        x, y = 10 + 30 * rng.random(), 10 + 30 * rng.random()
        w = rng.normal(size=3)
        w *= 0.25 / np.linalg.norm(w)
        rows.append((x, y, z, 0, x + w[0], y + w[1], z + w[2], 0, 0.5))
    seg = _seg(rows)
    d = o.quench_drift(seg)
    pix, _, _, _ = o.pixel_map(seg, d)
    total = sum(o.pixel_current(seg, d, p, s).sum() for p, s in pix.items())
    assert abs(total / d["Qa"].sum() - 1.0) < 1e-12


# ------------------------------------------------------------- whole events --

def test_whole_event_map_grows_its_buffer_and_fills_its_capacity_exactly():
    """ora_map_event on a segment mapped to more pixels than its initial
    per-segment buffer (4096: here a 50 cm segment widened by sigma_T ~ 2 cm)
    and with an output capacity of exactly the pair count: the same pairs as
    the per-segment brute-force maps, in segment order."""
    import ctypes as C
    cfg = params.small_config(diff_tran_cm2_s=12000.0)
    o = oracle.Oracle(cfg, params.LUT)
    seg = _seg([(5.0, 31.0, 25.0, 0, 55.0, 31.5, 25.0, 0, 50.0), (20.0, 10.0, 40.0, 0, 20.4, 10.2, 40.1, 0, 0.5)])
    d = o.quench_drift(seg)
    per = [o.map_segment(seg, d, s, box=False)[0] for s in range(2)]
    assert len(per[0]) > 4096
    cols = d["_seg"]
    sT = np.ascontiguousarray(d["sigma_T"], dtype=np.float64)
    an = np.ascontiguousarray(d["anode"], dtype=np.int32)
    P = C.POINTER

    def call(cap):
        ps, pp, pm = np.zeros(max(cap, 1), np.int64), np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1))
        m = o.L.ora_map_event(C.byref(o.c), 2, cols[0].ctypes.data_as(P(C.c_float)),
                              cols[1].ctypes.data_as(P(C.c_float)), cols[4].ctypes.data_as(P(C.c_float)),
                              cols[5].ctypes.data_as(P(C.c_float)), sT.ctypes.data_as(P(C.c_double)),
                              an.ctypes.data_as(P(C.c_int32)), cap, ps.ctypes.data_as(P(C.c_int64)),
                              pp.ctypes.data_as(P(C.c_int32)), pm.ctypes.data_as(P(C.c_double)))
        return m, ps[:min(m, cap)], pp[:min(m, cap)]

    n_pairs = len(per[0]) + len(per[1])
    m, ps, pp = call(n_pairs)
    assert m == n_pairs
    assert np.array_equal(pp, np.concatenate(per)) and np.array_equal(ps, np.repeat([0, 1], [len(x) for x in per]))
    m2, _, pp2 = call(n_pairs - 1)                      # one short: the count is still reported in full
    assert m2 == n_pairs and np.array_equal(pp2, pp[:-1])


def test_whole_event_functions_equal_the_single_pixel_ones():
    """ora_map_event is ora_map_segment_box of every segment; the many-pixel
    current and front end are pixel_current and electronics of each pixel
    alone, bit for bit, whatever the number of threads."""
    from synth import events
    cfg = params.small_config()
    lut64 = response.lut_for(cfg, params.LUT)
    o = oracle.Oracle(cfg, params.LUT, lut64)
    seg = events.scatter_event(cfg, 21, 40, max_len=0.6)
    d = o.quench_drift(seg)
    m = o.map_event(seg, d)
    pix, _, _, _ = o.pixel_map(seg, d)
    assert m["pixels"].tolist() == sorted(pix)
    for i, p in enumerate(m["pixels"].tolist()):
        assert m["segs"][m["off"][i]:m["off"][i + 1]].tolist() == pix[p]
    assert np.all(m["margin"] >= 0)
    pick = np.arange(0, len(m["pixels"]), 7)
    sub_off = np.concatenate([[0], np.cumsum(m["off"][pick + 1] - m["off"][pick])])
    sub_segs = np.concatenate([m["segs"][m["off"][i]:m["off"][i + 1]] for i in pick])
    for threads in (1, 0):
        I = o.pixel_currents(seg, d, m["pixels"][pick], sub_off, sub_segs, event_id=3, n_threads=threads)
        hits = o.electronics_many(m["pixels"][pick], I, event_id=3, band=0.5, n_threads=threads)
        for j, i in enumerate(pick):
            p = int(m["pixels"][i])
            ref = o.pixel_current(seg, d, p, pix[p], event_id=3)
            assert np.array_equal(I[j], ref)
            e = o.electronics(p, ref, event_id=3, band=0.5)
            for k in ("t_cross", "t_adc", "adc", "q"):
                assert np.array_equal(hits[j][k], e[k]), k
            assert hits[j]["tie_tick"] == e["tie_tick"]
    assert sum(len(h["t_cross"]) for h in hits) > 0
