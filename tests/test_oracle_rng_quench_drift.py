"""Pins of the oracle's generator and of steps 1-2 (Sec. 3.1, Sec. 3.2).

Each check uses something other than the oracle's own formula: published
known-answer vectors, numbers printed in the paper, inverted relations and
invariants that a dropped term, a wrong sign or a swapped constant breaks.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synth import params

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold_values():
    out = {}
    for line in open(os.path.join(GOLD, "paper_values.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val, tol = line.split()[:3]
        out[name] = (float(val), float(tol))
    return out


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]
        n += 1
    assert n == 3


def test_normals_statistics():
    seed, ev = 12345, 7
    v = np.array([oracle.normals(seed, ev, i, 3, 2) for i in range(40000)])
    x = v.reshape(-1)
    assert abs(x.mean()) < 0.02
    assert abs(x.std() - 1.0) < 0.02
    # Box-Muller partners are uncorrelated; 4th moment of a normal is 3
    assert abs(np.corrcoef(v[:, 0], v[:, 1])[0, 1]) < 0.03
    assert abs((x ** 4).mean() - 3.0) < 0.15
    # P(|n| > 2) of a standard normal
    assert abs((np.abs(x) > 2).mean() - 0.0455) < 0.004
    # counters and keys select different streams
    a = oracle.normals(seed, ev, 1, 2, 1)
    assert not np.allclose(a, oracle.normals(seed, ev + 1, 1, 2, 1))
    assert not np.allclose(a, oracle.normals(seed, ev, 1, 2, 2))


def test_paper_values_consistent_with_config():
    g = _gold_values()
    c = params.BASE
    assert c["pitch_cm"] == g["pixel_pitch_cm"][0]
    assert abs(c["px_per_tile"] * c["pitch_cm"] - g["tile_size_cm"][0]) < 1e-9
    assert c["px_per_tile"] ** 2 == g["pixels_per_tile"][0]
    assert c["gain_e_per_mV"] == g["gain_e_per_mV"][0]
    assert g["threshold_mV"][0] * c["gain_e_per_mV"] == g["threshold_e"][0]
    assert abs(c["min_adc_interval_ticks"] * c["tick_us"] - g["min_adc_interval_us"][0]) < 1e-9
    assert abs(c["hold_ticks"] * c["tick_us"] - g["hold_us"][0]) < 1e-9
    assert abs(c["sample_step_cm"] * 1e4 - g["sample_step_um"][0]) < 1e-9


@pytest.mark.parametrize("model", [0, 1])
def test_mip_recombination_around_0p7(model):
    val, tol = _gold_values()["mip_recomb_factor"]
    o = oracle.Oracle(params.tile_config(recomb_model=model), params.LUT)
    assert abs(o.recomb(2.1) - val) < tol


def _recomb_gold():
    rows = []
    for ln in open(os.path.join(GOLD, "recombination_closed_form.txt")):
        ln = ln.split("#")[0].split()
        if ln:
            rows.append((ln[0], float(ln[1]), float(ln[2])))
    return rows


@pytest.mark.parametrize("model", [0, 1])
def test_recombination_closed_form_values(model):
    """R at 2.1, 5, 10 and 20 MeV/cm against the hand-evaluated closed forms of
    Eq. (birks) / Eq. (box) with the paper's parameters (Sec. 3.1), to 1e-5:
    a 1 % error in rho, k_b, beta or the field moves R by more than 1e-3."""
    cfg = params.tile_config(recomb_model=model)
    assert (cfg["efield_kV_cm"], cfg["lar_density_g_cm3"]) == (0.5, 1.38)    # the values the table assumes
    o = oracle.Oracle(cfg, params.LUT)
    name = ("birks", "box")[model]
    rows = [(d, r) for m, d, r in _recomb_gold() if m == name]
    assert len(rows) == 4
    for dedx, R in rows:
        assert abs(o.recomb(dedx) / R - 1.0) < 1e-5, (name, dedx, o.recomb(dedx), R)
    # a MIP on 0.5 cm at the anode: 1.05 MeV / 23.6 eV = 44 491.5 electrons before recombination
    # (W_ion = 23.6 eV, a reading: the paper does not give it), R(2.1 MeV/cm) of them survive it
    mip = _seg([(5.0, 5.0, 0.1, 0.0, 5.5, 5.0, 0.1, 0.0, 1.05)])
    R21 = dict((d, r) for d, r in rows)[2.1]
    q0 = float(np.float32(1.05)) / float(np.float32(23.6e-6))
    assert abs(q0 - 44491.5) < 0.1
    assert abs(o.quench_drift(mip)["QR"][0] / (R21 * q0) - 1.0) < 1e-5
    # through the whole quench step: 0.5 cm segments at the anode carry Q_R = R dE / W_ion
    seg = _seg([(5.0, 5.0, 0.1, 0.0, 5.5, 5.0, 0.1, 0.0, 0.5 * d) for d, _ in rows])
    d = o.quench_drift(seg)
    R_step = d["QR"] * o.c.w_ion / seg["dE"].astype(np.float64)
    assert np.allclose(R_step, [R for _, R in rows], rtol=1e-5, atol=0)


def test_birks_inverted_relation():
    # Eq. (birks) solved for k_b: (A_b / R - 1) / (dE/dx) = k_b / epsilon at every dE/dx
    cfg = params.tile_config(recomb_model=0)
    o = oracle.Oracle(cfg, params.LUT)
    c = o.c
    eps = c.efield * c.density
    for dedx in (0.3, 1.0, 2.1, 5.0, 20.0, 48.0):
        R = o.recomb(dedx)
        assert 0 < R < c.Ab
        assert abs((c.Ab / R - 1.0) / dedx - c.kb / eps) < 1e-12
    assert abs(o.recomb(1e-9) - c.Ab) < 1e-9          # no quenching at vanishing dE/dx
    assert o.recomb(10.0) < o.recomb(5.0) < o.recomb(2.0)


def test_box_inverted_relation():
    # Eq. (box) solved for alpha: exp(R xi) - xi = alpha, xi = (beta/epsilon) dE/dx
    cfg = params.tile_config(recomb_model=1)
    o = oracle.Oracle(cfg, params.LUT)
    c = o.c
    eps = c.efield * c.density
    for dedx in (1.0, 2.1, 5.0, 20.0, 48.0):
        R = o.recomb(dedx)
        xi = c.beta / eps * dedx
        assert abs(math.exp(R * xi) - xi - c.alpha) < 1e-12
    assert o.recomb(20.0) < o.recomb(5.0) < o.recomb(2.1)


def _seg(rows):
    """Segments from rows (x0,y0,z0,t0,x1,y1,z1,t1,dE)."""
    a = np.asarray(rows, dtype=np.float32)
    keys = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1", "dE")
    return {k: np.ascontiguousarray(a[:, i]) for i, k in enumerate(keys)}


def test_quench_drift_invariants():
    cfg = params.module_config()
    o = oracle.Oracle(cfg, params.LUT)
    c = o.c
    # segments 0.5 cm along x at several heights in both drift volumes
    zs = [0.0, 3.0, 15.0, 29.5, 30.5, 45.0, 60.0]
    rows = [(10.0, 20.0, z, 0.0, 10.5, 20.0, z, 0.0, 1.05) for z in zs]
    d = o.quench_drift(_seg(rows))
    assert np.all(d["anode"] >= 0)
    # Q_R = R E / W_ion, R at dE/dx = E / dx
    dx = d["dx"]
    assert np.allclose(d["dedx"] * dx, np.float32(1.05), rtol=1e-12)
    assert np.allclose(d["QR"] * c.w_ion / np.float64(np.float32(1.05)), d["R"], rtol=1e-12)
    # drift distance: to anode z = 0 in TPC 0 and z = 2D in TPC 1
    dist = np.array([z if z < 30 else 60.0 - z for z in zs])
    assert np.allclose(d["t_drift"] * c.vdrift, dist, rtol=1e-12, atol=1e-12)
    # lifetime: ln(Q_a / Q_R) linear in drift time with slope -1/tau
    lr = np.log(d["Qa"] / d["QR"])
    assert np.allclose(lr, -d["t_drift"] / c.lifetime, rtol=1e-12, atol=1e-15)
    # a charge created on the anode is not attenuated and not diffused
    assert d["Qa"][0] == d["QR"][0] and d["sigma_T"][0] == 0 and d["sigma_L"][0] == 0
    # diffusion: sigma^2 / (2 t) = D (cm^2/us) for both directions
    m = d["t_drift"] > 0
    assert np.allclose(d["sigma_T"][m] ** 2 / (2 * d["t_drift"][m]), c.DT * 1e-6, rtol=1e-12)
    assert np.allclose(d["sigma_L"][m] ** 2 / (2 * d["t_drift"][m]), c.DL * 1e-6, rtol=1e-12)
    # mirror symmetry of the two drift volumes about the cathode
    assert d["anode"][1] == 0 and d["anode"][5] == 1
    # full 30 cm drift: attenuation and widths at the cathode
    full = o.quench_drift(_seg([(10, 20, 30.0 - 1e-4, 0, 10.5, 20, 30.0 - 1e-4, 0, 1.0)]))
    assert abs(full["t_drift"][0] - 187.5) < 1e-3
    assert abs(full["Qa"][0] / full["QR"][0] - 0.918304) < 1e-6
    assert abs(full["sigma_T"][0] - 0.0574456) < 1e-6
    assert abs(full["sigma_L"][0] - 0.0387298) < 1e-6


def test_sample_count_and_activity():
    cfg = params.module_config()
    o = oracle.Oracle(cfg, params.LUT)
    rows = [
        (10, 20, 5, 0, 10.5, 20, 5, 0, 1.0),          # 0.5 cm
        (10, 20, 5, 0, 10.0, 20, 5, 0, 1.0),          # zero length: inactive
        (-1, 20, 5, 0, -0.5, 20, 5, 0, 1.0),          # midpoint outside x
        (10, 20, 61, 0, 10.5, 20, 61, 0, 1.0),        # beyond the second anode
        (10, 20, 5, 0, 10.0000, 20.0, 5.0005, 0, 1.0),  # 5 um along z: one point
        (10, 20, 5, 0, 10.3, 20.4, 5, 0, 1.0),        # 0.5 cm diagonal
    ]
    d = o.quench_drift(_seg(rows))
    assert list(d["anode"][[1, 2, 3]]) == [-1, -1, -1]
    assert d["Qa"][1] == 0 and d["n_samples"][1] == 0
    N = d["n_samples"]
    act = d["anode"] >= 0
    # N = smallest integer with N * step >= dx (10 um points)
    assert np.all(N[act] * o.c.step >= d["dx"][act])
    assert np.all((N[act] - 1) * o.c.step < d["dx"][act])
    assert N[4] == 1
    assert abs(N[0] - 500) <= 1 and abs(N[5] - 500) <= 1


def test_anode_numbering_across_modules():
    cfg = params.spill_config()
    o = oracle.Oracle(cfg, params.LUT)
    W = 280 * np.float32(0.4434)
    H = 350 * np.float32(0.4434)
    rows = []
    expect = []
    # near a module's first corner, and near its far corner (modules are 124 x 155 cm: there
    # y / W and y / H floor to different rows)
    for (mx, my, tpc, fx, fy) in [(0, 0, 0, 5.0, 7.0), (6, 0, 1, 5.0, 7.0), (0, 4, 0, 5.0, 7.0), (3, 2, 1, 5.0, 7.0),
                                  (6, 4, 1, 5.0, 7.0), (2, 1, 0, 120.0, 150.0), (5, 3, 1, 120.0, 150.0)]:
        x = mx * W + fx
        y = my * H + fy
        z = 10.0 if tpc == 0 else 50.0
        rows.append((x, y, z, 0, x + 0.4, y, z, 0, 1.0))
        expect.append((my * 7 + mx) * 2 + tpc)
    d = o.quench_drift(_seg(rows))
    assert list(d["anode"]) == expect
