"""Pins of the light-path oracle (Sec. 4) and of its synthetic tables.

Each pin ties an oracle step to an independent statement: a closed-form
solid angle, the quanta sum rule of Sec. 4.1, single-segment table rows,
the closed form of the scintillation kernel and of its truncated sum, the
Poisson quantile function of scipy, numpy's inverse real FFT for the
random-phase noise, and exact linear ramps for the digitiser.
"""
import math

import numpy as np
import pytest

import oracle
from synth import light, params

KEYS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")


def _seg(rows):
    a = np.asarray(rows, dtype=np.float32)
    return {k: np.ascontiguousarray(a[:, i]) for i, k in enumerate(KEYS)}


def _setup(cfg=None, t_start=-0.05, n_ticks=4096, **over):
    cfg = cfg or params.small_config()
    L = dict(light.LIGHT, **over)
    tab = light.tables(cfg, L)
    return cfg, L, tab, oracle.LightOracle(cfg, L, tab, t_start, n_ticks)


def test_visibility_on_axis_closed_form():
    """The rectangle decomposition behind the table: a point on the normal
    through a rectangle's centre sees it under
    4 atan(a b / (2 d sqrt(4 d^2 + a^2 + b^2)))."""
    for d, a, b in ((0.5, 3.9, 30.0), (10.0, 3.9, 30.0), (37.0, 15.5, 30.0), (2.0, 1.0, 1.0)):
        om = 4 * math.atan(a * b / (2 * d * math.sqrt(4 * d * d + a * a + b * b)))
        got = light._rect_solid_angle(d, -a / 2, a / 2, -b / 2, b / 2)
        assert got == pytest.approx(om, rel=1e-12)
    # a point far off the rectangle's corner: four signed terms still add up (against quadrature)
    d, a1, a2, b1, b2 = 3.0, 2.0, 5.0, -1.0, 4.0
    ys = np.linspace(a1, a2, 2001)
    zs = np.linspace(b1, b2, 2001)
    Y, Z = np.meshgrid(0.5 * (ys[1:] + ys[:-1]), 0.5 * (zs[1:] + zs[:-1]), indexing="ij")
    q = (d / (d * d + Y * Y + Z * Z) ** 1.5).sum() * (ys[1] - ys[0]) * (zs[1] - zs[0])
    assert light._rect_solid_angle(d, a1, a2, b1, b2) == pytest.approx(q, rel=1e-5)


def test_visibility_against_quadrature():
    cfg = params.small_config()
    L = dict(light.LIGHT)
    dets = light.detectors(cfg, L)
    V = light.visibility(cfg, L)
    rng = np.random.default_rng(0)
    for _ in range(4):
        ix, iy, iz = (int(rng.integers(0, n)) for n in V.shape[:3])
        k = int(rng.integers(0, len(dets)))
        xw, y1, y2, z1, z2 = dets[k]
        P = (np.array([ix, iy, iz]) + 0.5) * L["vox_cm"]
        ys = np.linspace(y1, y2, 801)
        zs = np.linspace(z1, z2, 801)
        Y, Z = np.meshgrid(0.5 * (ys[1:] + ys[:-1]), 0.5 * (zs[1:] + zs[:-1]), indexing="ij")
        d = abs(P[0] - xw)
        r2 = d * d + (Y - P[1]) ** 2 + (Z - P[2]) ** 2
        om = (d / r2 ** 1.5).sum() * (ys[1] - ys[0]) * (zs[1] - zs[0])
        assert V[ix, iy, iz, k] == pytest.approx(om / (4 * math.pi), rel=2e-3)


def test_yield_sum_rule_voxel_and_tick():
    """N_pe,i / (eps_i V_i) + Q_R = dE / W_ph (Sec. 4.1); a segment centred on
    a voxel centre lands in that voxel; its midpoint time sets the tick."""
    cfg, L, tab, lo = _setup()
    o = oracle.Oracle(cfg, params.LUT)
    v = L["vox_cm"]
    rows = []
    cells = [(2, 3, 1), (5, 1, 6), (0, 7, 3), (12, 14, 6)]     # the last one far from the corner: a
    for (ix, iy, iz), tm in zip(cells, (0.25, 1.0, 2.5, 3.0)):  # voxel size a few % off moves it
        x, y, z = (ix + 0.5) * v, (iy + 0.5) * v, (iz + 0.5) * v
        rows.append((x - 0.2, y, z - 0.1, tm - 0.01, x + 0.2, y, z + 0.1, tm + 0.01, 0.9))
    seg = _seg(rows)
    d = o.quench_drift(seg)
    npe, tick, vox = lo.segments(seg, d)
    nvx, nvy, nvz = tab["vis"].shape[:3]
    for j, (ix, iy, iz) in enumerate(cells):
        assert vox[j] == (ix * nvy + iy) * nvz + iz
        tm = np.float32(0.5) * (seg["t0"][j] + seg["t1"][j])
        assert tick[j] == math.floor((tm - np.float32(-0.05)) / np.float32(L["tick_us"]))   # FP32 operations
        assert abs(tick[j] - (float(tm) + 0.05) / 0.001) <= 1.0
        ng = npe[j] / (tab["eff"].astype(np.float64) * tab["vis"].reshape(-1, L["n_det"])[vox[j]])
        assert np.allclose(ng + d["QR"][j], float(np.float32(0.9)) / float(np.float32(L["w_ph_MeV"])), rtol=1e-12)
    # the voxel's depth is the distance from the segment's own anode: mirrored segments of
    # the second drift volume (anode at z = 2D) land in the same voxels
    D = float(np.float32(cfg["drift_len_cm"]))
    mirror = {k: v.copy() for k, v in seg.items()}
    mirror["z0"] = np.float32(2 * D) - seg["z1"]
    mirror["z1"] = np.float32(2 * D) - seg["z0"]
    dm = o.quench_drift(mirror)
    assert np.all(dm["anode"] == d["anode"] + 1)           # the other TPC of the same module
    _, tick_m, vox_m = lo.segments(mirror, dm)
    assert np.array_equal(vox_m, vox) and np.array_equal(tick_m, tick)


def test_photocurrent_single_segment_is_a_table_row():
    cfg, L, tab, lo = _setup()
    rng = np.random.default_rng(1)
    n, nd = 3, L["n_det"]
    npe = rng.random((n, nd)) * 50
    tick = np.array([100, 100, 37], np.int32)
    vox = np.array([5, 17, 5], np.int32)
    anode = np.array([0, 0, 1], np.int32)
    f = tab["tdist"].reshape(-1, nd, L["nt"]).astype(np.float64)
    for k in (0, 9):
        I = lo.photocurrent(npe, tick, vox, anode, k)                 # anode 0 only
        exp = np.zeros(lo.l.n_ticks)
        exp[100:100 + L["nt"]] = npe[0, k] * f[5, k] + npe[1, k] * f[17, k]
        assert np.allclose(I, exp, rtol=1e-14, atol=0)
        I1 = lo.photocurrent(npe, tick, vox, anode, nd + k)            # anode 1
        e1 = np.zeros(lo.l.n_ticks)
        e1[37:37 + L["nt"]] = npe[2, k] * f[5, k]
        assert np.allclose(I1, e1, rtol=1e-14, atol=0)


def test_scintillation_impulse_and_truncated_sum():
    """A unit impulse at tick 10 gives f_scint(u tick) for u <= n_trunc and 0
    beyond; the truncated sum is the two geometric series."""
    cfg, L, tab, lo = _setup(n_ticks=9000, tau_slow_us=0.5)        # n_trunc = 2500 fits the window
    I = np.zeros(9000)
    I[10] = 1.0
    S = lo.scintillation(I)
    fp, tp, ts, dt = (float(np.float32(L[k])) for k in ("fast_frac", "tau_fast_us", "tau_slow_us", "tick_us"))
    N = lo.n_trunc
    assert N == 2500
    u = np.arange(N + 1)
    exp = fp / tp * np.exp(-u * dt / tp) + (1 - fp) / ts * np.exp(-u * dt / ts)
    assert np.allclose(S[10:11 + N], exp, rtol=1e-12)
    assert np.all(S[:10] == 0) and np.all(S[11 + N:] == 0)
    rp, rs = math.exp(-dt / tp), math.exp(-dt / ts)
    geo = fp / tp * (1 - rp ** (N + 1)) / (1 - rp) + (1 - fp) / ts * (1 - rs ** (N + 1)) / (1 - rs)
    assert S.sum() == pytest.approx(geo, rel=1e-12)
    # an impulse on the window's first tick: the sum's last term (u = t) carries it
    I0 = np.zeros(9000)
    I0[0] = 1.0
    S0 = lo.scintillation(I0)
    assert np.allclose(S0[:N + 1], exp, rtol=1e-12) and np.all(S0[N + 1:] == 0)


def test_poisson_inverse_transform_is_the_quantile():
    """Below the switch the count is the Poisson quantile of the block's
    uniform (scipy.stats.poisson.ppf); above it, lambda + sqrt(lambda) z."""
    stats = pytest.importorskip("scipy.stats")
    cfg, L, tab, lo = _setup(n_ticks=3000)
    rng = np.random.default_rng(5)
    lam = np.concatenate([rng.random(1000) * 0.2, rng.random(1000) * 30.0, 30.0 + rng.random(1000) * 200])
    S = lam / float(np.float32(L["tick_us"]))
    det, ev = 7, 3
    n, mg = lo.fluctuate(S, det, ev)
    seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF
    key = seed ^ ev
    for t in range(3000):
        l = S[t] * float(np.float32(L["tick_us"]))
        if l <= 30.0:
            x = oracle.philox4x32_10([det, t, 5, 0], [key & 0xFFFFFFFF, key >> 32])
            u = (float(x[0]) + 0.5) / 2.0 ** 32
            if mg[t] > 1e-9:
                assert n[t] == stats.poisson.ppf(u, l), (t, l, u)
            # margin: the distance of u from the two CDF values the count was decided between
            # (one for a count of 0), and of the mean from the switch
            k = int(n[t])
            gaps = [abs(u - stats.poisson.cdf(k, l))] + ([abs(u - stats.poisson.cdf(k - 1, l))] if k else [])
            assert abs(mg[t] - min(gaps + [abs(l - 30.0)])) < 1e-12, (t, l, u)
        else:
            assert abs(mg[t] - (l - 30.0)) < 1e-12
            z = oracle.normals(seed, ev, det, t, 6, 0)[0]
            assert n[t] == pytest.approx(max(0.0, l + math.sqrt(l) * z), rel=1e-12)
    # the switch itself: a mean of exactly 30 counts by the Poisson branch (integers), the next
    # double above it by the normal one (reading: the normal law for means above 30)
    tick = float(np.float32(L["tick_us"]))
    s30 = 30.0 / tick
    while s30 * tick > 30.0:
        s30 = math.nextafter(s30, 0.0)
    while s30 * tick < 30.0:
        s30 = math.nextafter(s30, math.inf)
    assert s30 * tick == 30.0
    s_up = s30
    while s_up * tick <= 30.0:
        s_up = math.nextafter(s_up, math.inf)
    n30, _ = lo.fluctuate(np.full(3000, s30), 9, 1)
    nup, _ = lo.fluctuate(np.full(3000, s_up), 9, 1)
    assert np.all(n30 == np.round(n30))
    assert np.mean(nup != np.round(nup)) > 0.99
    # statistics of the small-mean branch: mean and variance ~ lambda
    S2 = np.full(3000, 4.0 / float(np.float32(L["tick_us"])))
    n2, _ = lo.fluctuate(S2, 11, 0)
    assert abs(n2.mean() - 4.0) < 5 * math.sqrt(4.0 / 3000)
    assert abs(n2.var() - 4.0) < 0.5


def test_noise_is_the_inverse_real_fft_and_response_is_linear():
    cfg, L, tab, lo = _setup(n_ticks=2048)
    det, ev = 5, 2
    zero = np.zeros(2048)
    V, vs, code, mg = lo.electronics(zero, det, ev)
    N = L["noise_block"]
    seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF
    key = seed ^ ev
    A = tab["noise"].astype(np.float64)
    assert A[0] == 0 and A[-1] == 0
    for b in range(2):
        phi = np.array([2 * math.pi * (float(oracle.philox4x32_10([det, b, 7, k], [key & 0xFFFFFFFF, key >> 32])[0])
                                       + 0.5) / 2.0 ** 32 for k in range(N // 2 + 1)])
        ref = (N / 2) * np.fft.irfft(A * np.exp(1j * phi), N)
        assert np.allclose(V[b * N:(b + 1) * N], ref, atol=1e-9)
    # response: V(n + impulse) - V(n) = gain * resp shifted
    imp = np.zeros(2048)
    imp[300] = 7.0
    V2, _, _, _ = lo.electronics(imp, det, ev)
    g = float(tab["gain"][det % L["n_det"]])
    r = tab["resp"].astype(np.float64)
    d = V2 - V
    assert np.allclose(d[300:300 + len(r)], 7.0 * g * r, rtol=1e-12, atol=1e-12)
    assert np.allclose(d[:300], 0) and np.allclose(d[300 + len(r):], 0)


def test_digitiser_samples_a_ramp():
    """With no noise and a ramp n, V is a ramp; samples read it at m * ratio
    exactly, and codes round V + pedestal half up."""
    cfg, L, tab, lo = _setup(n_ticks=2048)
    tab2 = dict(tab, noise=np.zeros_like(tab["noise"]), resp=np.array([1.0], np.float32))
    lo2 = oracle.LightOracle(cfg, L, tab2, -0.05, 2048)
    n = np.arange(2048) * 0.37
    V, vs, code, mg = lo2.electronics(n, 3, 0)
    g = float(tab["gain"][3])
    assert np.allclose(V, g * n, rtol=1e-14)
    # a 62.5 MHz digitiser (16 ns) on 1 ns ticks samples every 16 ticks: 128 samples of 2048 ticks
    assert (L["sample_us"], L["tick_us"]) == (0.016, 0.001)
    assert lo2.n_samples == 128
    p = np.arange(lo2.n_samples) * 16.0
    assert np.allclose(vs, g * 0.37 * p, rtol=1e-6)              # FP32 config values: ratio 16 to ~1e-7
    assert np.allclose(vs, g * 0.37 * np.arange(lo2.n_samples) * lo2.ratio, rtol=1e-12)
    ped = float(np.float32(L["pedestal"]))
    exp = np.clip(np.floor(vs + ped + 0.5), 0, 2 ** L["adc_bits"] - 1)
    assert np.array_equal(code, exp.astype(np.int32))
    # each sample's margin: how far v + pedestal + 1/2 lies from the nearest integer (a code boundary)
    w = g * 0.37 * p + ped + 0.5
    assert np.allclose(mg, np.abs(w - np.round(w)), rtol=0, atol=1e-6)
    # a window of 16 k + 1 ticks: its last sample falls on its last tick, read without a neighbour
    lo3 = oracle.LightOracle(cfg, L, tab2, -0.05, 2049)
    assert lo3.n_samples == 129
    _, vs3, _, _ = lo3.electronics(np.arange(2049) * 0.37, 3, 0)
    assert np.allclose(vs3, g * 0.37 * 16.0 * np.arange(129), rtol=1e-12)


def test_light_truth_arrival_time_of_a_one_bin_row():
    """A table row concentrated in bin b gives the mean arrival time
    t_start + (tick + b + 1/2) tick; a general row gives its mean."""
    cfg, L, tab, lo = _setup()
    tab2 = dict(tab)
    td = np.zeros_like(tab["tdist"])
    td[..., 0, 5] = 1.0
    td[..., 1, :] = tab["tdist"][..., 1, :]
    tab2["tdist"] = td
    lo2 = oracle.LightOracle(cfg, L, tab2, -0.05, 4096)
    tick = np.array([100, -3, 7], np.int32)
    vox = np.array([4, 9, -1], np.int32)
    t = lo2.truth(tick, vox)
    dt, t0 = float(np.float32(L["tick_us"])), float(np.float32(-0.05))
    assert t[0, 0] == pytest.approx(t0 + (100 + 5.5) * dt, rel=1e-14)
    assert t[1, 0] == pytest.approx(t0 + (-3 + 5.5) * dt, rel=1e-14)
    f = tab["tdist"].reshape(-1, L["n_det"], L["nt"]).astype(np.float64)[4, 1]
    assert t[0, 1] == pytest.approx(t0 + (100 + ((np.arange(L["nt"]) + 0.5) * f).sum()) * dt, rel=1e-14)
    assert np.all(t[2] == 0.0)
