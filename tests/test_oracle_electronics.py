"""Pins of the oracle's front-end model (Sec. 3.4) by closed forms.

With the three noises off and a constant current i per tick the CSA charge
after tick k is (k+1) i, so the first crossing, the digitised charge and the
hit period follow from integer arithmetic alone.
"""
import math

import numpy as np
import pytest

import oracle
from synth import params


def _quiet(**over):
    c = params.tile_config(sigma_reset_e=0.0, sigma_disc_e=0.0, sigma_unc_e=0.0, n_ticks=2000)
    c.update(over)
    return c


def test_constant_current_closed_form():
    cfg = _quiet()
    o = oracle.Oracle(cfg, params.LUT)
    thr = np.float32(cfg["thr_e"])
    lsb_e = np.float64(np.float32(cfg["gain_e_per_mV"])) * np.float64(np.float32(cfg["adc_lsb_mV"]))
    hold = cfg["hold_ticks"]
    for i in (37.0, 333.0, 1250.5, 4999.0, 7000.0):
        r = o.electronics(1234, np.full(2000, i))
        n_up = math.ceil(thr / i)                  # ticks to integrate the threshold
        t1 = n_up - 1
        assert r["t_cross"][0] == t1
        assert r["t_adc"][0] == t1 + hold
        assert r["adc"][0] == min(255, math.floor((t1 + hold + 1) * i / lsb_e))
        # after the reset the charge starts from zero: period = hold + n_up ticks
        period = hold + n_up
        exp_n = 0
        t = t1
        while t + hold < 2000:
            exp_n += 1
            t += period
        assert len(r["t_cross"]) == exp_n
        assert np.all(np.diff(r["t_cross"]) == period)
        assert np.all(r["t_adc"] - r["t_cross"] == hold)


def test_below_threshold_no_hits():
    o = oracle.Oracle(_quiet(), params.LUT)
    I = np.zeros(2000)
    I[100:110] = 499.0          # 4990 e- in total, threshold 5000 e-
    assert len(o.electronics(7, I)["t_cross"]) == 0
    I[500] = 11.0               # now 5001 e-
    r = o.electronics(7, I)
    assert list(r["t_cross"]) == [500]


def test_minimum_adc_interval():
    cfg = _quiet(hold_ticks=2, min_adc_interval_ticks=11)
    o = oracle.Oracle(cfg, params.LUT)
    r = o.electronics(3, np.full(2000, 6000.0))   # crosses on every idle tick
    assert r["t_cross"][0] == 0 and r["t_adc"][0] == 2
    assert np.all(np.diff(r["t_adc"]) == 11)
    assert np.all(r["t_cross"][1:] == r["t_adc"][:-1] + 1)


def test_hits_monotone_in_threshold():
    rng = np.random.default_rng(2)
    I = rng.exponential(150.0, 2000) * (rng.random(2000) < 0.3)
    counts = []
    for thr in (2000.0, 4000.0, 8000.0, 16000.0, 64000.0, 1.0e6):
        o = oracle.Oracle(_quiet(thr_e=thr), params.LUT)
        counts.append(len(o.electronics(5, I)["t_cross"]))
    assert counts == sorted(counts, reverse=True) and counts[-1] == 0 and counts[0] > 0


def test_periodic_reset_discards_subthreshold_charge():
    I = np.full(2000, 10.0)     # 5000 e- after 500 ticks
    o = oracle.Oracle(_quiet(), params.LUT)
    assert o.electronics(9, I)["t_cross"][0] == 499
    o2 = oracle.Oracle(_quiet(periodic_reset_ticks=400), params.LUT)
    assert len(o2.electronics(9, I)["t_cross"]) == 0


def test_adc_code_is_clamped_to_its_range():
    """ADC = clamp(floor(v / lsb), 0, 2^bits - 1) (Sec. 3.4): a current far
    above the range saturates at 2^bits - 1 for 8 and 10 bits, and a charge
    that crossed the threshold and then fell below zero during the hold (a
    bipolar induced current) digitises as 0."""
    for bits in (8, 10):
        cfg = _quiet(adc_bits=bits)
        o = oracle.Oracle(cfg, params.LUT)
        r = o.electronics(11, np.full(2000, 1.0e7))
        lsb_e = float(np.float32(cfg["gain_e_per_mV"])) * float(np.float32(cfg["adc_lsb_mV"]))
        assert len(r["adc"]) > 10 and np.all(r["adc"] == (1 << bits) - 1)
        assert np.all(r["q"] / lsb_e > 2 * (1 << bits))         # far beyond the range
    cfg = _quiet()
    o = oracle.Oracle(cfg, params.LUT)
    thr = float(np.float32(cfg["thr_e"]))
    I = np.zeros(2000)
    I[10] = thr + 10.0                      # crosses at tick 10
    I[11] = -4.0 * thr                      # the charge is negative when the ADC samples it
    r = o.electronics(12, I)
    assert list(r["t_cross"]) == [10] and list(r["t_adc"]) == [10 + cfg["hold_ticks"]]
    assert r["q"][0] < 0 and list(r["adc"]) == [0]


def test_window_starts_discharged_and_periodic_resets_fall_on_multiples():
    """The CSA starts the window discharged, and periodic resets (while idle)
    set it to a pedestal at ticks j * period, j >= 1.  With zero current and
    no other noise the charge changes only at resets, so a pixel's first
    crossing is at one of those ticks, never before the first period."""
    P = 97
    cfg = _quiet(sigma_reset_e=900.0, thr_e=450.0, periodic_reset_ticks=P)
    o = oracle.Oracle(cfg, params.LUT)
    firsts = []
    for pix in range(600):
        t = o.electronics(pix, np.zeros(2000))["t_cross"]
        if len(t):
            firsts.append(int(t[0]))
    f = np.array(firsts)
    assert len(f) > 500                     # P(n0 >= 1/2) = 0.31 per reset, 20 resets per window
    assert np.all(f >= P) and np.all(f % P == 0)
    assert np.sum(f == P) > 120             # the first reset already fires ~31 % of the pixels


def test_noise_statistics_of_idle_comparisons():
    """With zero current and zero threshold the first comparison fires when
    s_unc n_unc >= s_disc n_disc, i.e. with probability 1/2."""
    # a hit needs the ADC tick inside the window: hold = 0 makes it immediate
    cfg0 = params.tile_config(thr_e=0.0, n_ticks=1, hold_ticks=0)
    o0 = oracle.Oracle(cfg0, params.LUT)
    fired = np.array([len(o0.electronics(p, np.zeros(1))["t_cross"]) for p in range(4000)])
    assert abs(fired.mean() - 0.5) < 0.03
    # the digitised charge is the noise itself: mean 0, sigma_unc ~ 500 e-, conditioned on firing
    qs = np.array([o0.electronics(p, np.zeros(1))["q"][0] for p in np.nonzero(fired)[0][:1500]])
    # E[n_unc | s_unc n_unc >= s_disc n_disc] = s_unc / sqrt(s_unc^2 + s_disc^2) * sqrt(2/pi)
    su, sd = 500.0, 650.0
    exp_mean = su * su / math.hypot(su, sd) * math.sqrt(2 / math.pi)
    assert abs(qs.mean() - exp_mean) < 25.0


def test_reset_noise_pedestal():
    """After a digitisation the CSA restarts from a pedestal s_reset n0."""
    cfg = _quiet(sigma_reset_e=900.0)
    o = oracle.Oracle(cfg, params.LUT)
    gaps = []
    for p in range(300):
        r = o.electronics(p, np.full(2000, 100.0))     # 50 ticks to threshold from zero
        t = r["t_cross"]
        if len(t) >= 2:
            gaps.append(t[1] - r["t_adc"][0])
    g = np.array(gaps, dtype=float)
    # pedestal s n0 shortens the next integration by ~ s n0 / 100 ticks
    assert abs(g.mean() - 50.0) < 1.5
    assert 7.0 < g.std() < 11.0


@pytest.mark.parametrize("current, band", [(300.0, 2.0), (60.0, 1.0)])
def test_tie_probability_matches_tie_frequency(current, band):
    """p_tie (the chance, under the noise model, that a trace has a decision
    within the band) predicts how many pixels a band excludes: over 3000
    constant-current pixels (different Philox streams) the tied fraction
    agrees with the mean p_tie within 4 binomial standard errors."""
    cfg = params.small_config(n_ticks=600)
    o = oracle.Oracle(cfg, params.LUT)
    n = 3000
    pix = np.arange(n, dtype=np.int32) * 3
    h = o.electronics_many(pix, np.full((n, 600), current), event_id=9, band=band)
    tied = np.mean([x["tie_tick"] >= 0 for x in h])
    pt = np.mean([x["p_tie"] for x in h])
    assert 0.02 < pt < 0.5
    assert abs(tied - pt) < 4 * np.sqrt(pt * (1 - pt) / n), (tied, pt)
