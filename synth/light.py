"""Synthetic inputs of the light path (arXiv:2212.09807 Sec. 4).

The paper's light tables come from a dedicated Geant4 simulation (visibility
V_i[ix, iy, iz] and arrival-time distribution f_i[ix, iy, iz, it] per voxel
and photosensor, Sec. 4.1-4.2); they are not available here.  These closed
forms stand in for them, with the same shapes and roles:

  * geometry: each TPC has n_det photosensors, n_det / 2 on each of its two
    walls x_local = 0 and x_local = W_x, tiling the wall in y and spanning the
    whole drift length; coordinates are local to the TPC (x, y from the
    module corner, z = distance from the anode);
  * visibility: the solid angle of the detector rectangle seen from the voxel
    centre, over 4 pi (rectangle decomposed at the foot of the perpendicular);
  * arrival time: a direct path at c / n (n = 1.38) plus an exponential
    scattering delay of scale 2 ns + r / (30 cm/ns), integrated over each
    1 ns bin and normalised over the nt bins;
  * impulse response: a bi-exponential pulse (rise 2 ns, fall 30 ns),
    integrated over each bin and normalised to unit sum;
  * noise: amplitudes of a one-sided spectrum on blocks of noise_block ticks,
    flat plus a low-frequency rise, scaled to a chosen RMS.

Each table is computed in FP64 and rounded to FP32; the GPU path and the
oracle receive the same FP32 values.  This module holds no step of the
simulation itself.
"""
from __future__ import annotations

import numpy as np

LIGHT = dict(
    n_det=16,             # photosensors per TPC (8 per wall)
    vox_cm=4.0,           # voxel edge of the visibility / time tables
    nt=64,                # arrival-time bins of the table (one light tick each)
    tick_us=0.001,        # light simulation tick (1 ns)
    eff=0.01,             # detection efficiency epsilon_i of every photosensor
    w_ph_MeV=19.5e-6,     # mean energy per scintillation photon at zero field
    fast_frac=0.3,        # prompt fraction f_p
    tau_fast_us=0.007,    # prompt decay time
    tau_slow_us=1.6,      # slow decay time
    trunc_taus=5.0,       # convolution truncated at trunc_taus * tau_slow
    poisson_max_mean=30.0,
    n_resp=256,           # impulse-response bins (one tick each)
    tau_rise_us=0.002,
    tau_fall_us=0.030,
    gain=5.0,             # ADC per photoelectron (response normalised to unit sum)
    noise_block=1024,     # ticks per block of random-phase noise
    noise_rms=2.0,        # ADC
    sample_us=0.016,      # digitiser sampling period (62.5 MHz)
    adc_bits=14,
    pedestal=1000.0,      # ADC
    n_index=1.38,         # refractive index for the direct path
)


def detectors(cfg: dict, L: dict = LIGHT) -> np.ndarray:
    """[n_det, 5] rectangles (x_wall, y_lo, y_hi, z_lo, z_hi) in TPC-local cm."""
    p = float(np.float32(cfg["pitch_cm"]))
    Wx = cfg["tiles_x"] * cfg["px_per_tile"] * p
    Wy = cfg["tiles_y"] * cfg["px_per_tile"] * p
    D = float(np.float32(cfg["drift_len_cm"]))
    half = L["n_det"] // 2
    out = []
    for wall in (0.0, Wx):
        for k in range(half):
            out.append((wall, k * Wy / half, (k + 1) * Wy / half, 0.0, D))
    return np.array(out)


def voxel_grid(cfg: dict, L: dict = LIGHT):
    p = float(np.float32(cfg["pitch_cm"]))
    Wx = cfg["tiles_x"] * cfg["px_per_tile"] * p
    Wy = cfg["tiles_y"] * cfg["px_per_tile"] * p
    D = float(np.float32(cfg["drift_len_cm"]))
    v = L["vox_cm"]
    n = (int(np.ceil(Wx / v)), int(np.ceil(Wy / v)), int(np.ceil(D / v)))
    return n


def _rect_solid_angle(d, a1, a2, b1, b2):
    """Solid angle of the rectangle [a1, a2] x [b1, b2] in a plane at distance
    d > 0 from the point, whose foot is the origin of (a, b)."""
    def F(a, b):
        return np.arctan(a * b / (d * np.sqrt(d * d + a * a + b * b)))
    return F(a2, b2) - F(a1, b2) - F(a2, b1) + F(a1, b1)


def visibility(cfg: dict, L: dict = LIGHT) -> np.ndarray:
    """V [nvx, nvy, nvz, n_det] at the voxel centres (FP64)."""
    nvx, nvy, nvz = voxel_grid(cfg, L)
    v = L["vox_cm"]
    xc = (np.arange(nvx) + 0.5) * v
    yc = (np.arange(nvy) + 0.5) * v
    zc = (np.arange(nvz) + 0.5) * v
    X, Y, Z = np.meshgrid(xc, yc, zc, indexing="ij")
    dets = detectors(cfg, L)
    out = np.zeros((nvx, nvy, nvz, len(dets)))
    for k, (xw, y1, y2, z1, z2) in enumerate(dets):
        d = np.maximum(np.abs(X - xw), 1e-3)
        out[..., k] = _rect_solid_angle(d, y1 - Y, y2 - Y, z1 - Z, z2 - Z) / (4.0 * np.pi)
    return out


def time_distribution(cfg: dict, L: dict = LIGHT) -> np.ndarray:
    """f [nvx, nvy, nvz, n_det, nt]: fraction of a voxel's detected photons
    arriving in each 1-tick bin after emission (FP64, rows sum to 1)."""
    nvx, nvy, nvz = voxel_grid(cfg, L)
    v = L["vox_cm"]
    xc = (np.arange(nvx) + 0.5) * v
    yc = (np.arange(nvy) + 0.5) * v
    zc = (np.arange(nvz) + 0.5) * v
    X, Y, Z = np.meshgrid(xc, yc, zc, indexing="ij")
    dets = detectors(cfg, L)
    tick_ns = L["tick_us"] * 1e3
    c_ns = 29.9792458 / L["n_index"]                       # cm / ns
    edges = np.arange(L["nt"] + 1) * tick_ns
    out = np.zeros((nvx, nvy, nvz, len(dets), L["nt"]))
    for k, (xw, y1, y2, z1, z2) in enumerate(dets):
        r = np.sqrt((X - xw) ** 2 + (Y - 0.5 * (y1 + y2)) ** 2 + (Z - 0.5 * (z1 + z2)) ** 2)
        td = r / c_ns
        tau = 2.0 + r / 30.0
        cdf = 1.0 - np.exp(-np.maximum(edges[None, None, None, :] - td[..., None], 0.0) / tau[..., None])
        f = np.diff(cdf, axis=-1)
        out[..., k, :] = f / f.sum(axis=-1, keepdims=True)
    return out


def impulse_response(L: dict = LIGHT) -> np.ndarray:
    """Unit-sum bi-exponential pulse over n_resp ticks (FP64)."""
    tr, tf = L["tau_rise_us"], L["tau_fall_us"]
    dt = L["tick_us"]
    e = np.arange(L["n_resp"] + 1) * dt
    P = lambda t: -tf * np.exp(-t / tf) + tr * np.exp(-t / tr)   # noqa: E731  antiderivative
    r = np.diff(P(e))
    return r / r.sum()


def noise_amplitudes(L: dict = LIGHT) -> np.ndarray:
    """Amplitudes A_k, k = 0 .. noise_block / 2, of the noise n(t) =
    sum_k A_k cos(2 pi k t / N + phi_k): no DC term, flat plus a 1/sqrt(k)
    rise, scaled so that the RMS over random phases is noise_rms."""
    N = L["noise_block"]
    k = np.arange(N // 2 + 1, dtype=np.float64)
    A = np.where(k > 0, 1.0 + 4.0 / np.sqrt(np.maximum(k, 1.0)), 0.0)
    A[-1] = 0.0                                               # no Nyquist term
    rms = np.sqrt(0.5 * (A ** 2).sum())
    return A * (L["noise_rms"] / rms)


def tables(cfg: dict, L: dict = LIGHT) -> dict:
    """All FP32 tables of the light path for a configuration."""
    return dict(vis=visibility(cfg, L).astype(np.float32),
                tdist=time_distribution(cfg, L).astype(np.float32),
                eff=np.full(L["n_det"], L["eff"], np.float32),
                gain=np.full(L["n_det"], L["gain"], np.float32),
                resp=impulse_response(L).astype(np.float32),
                noise=noise_amplitudes(L).astype(np.float32))


def window(t_first_us: float, t_last_us: float, L: dict = LIGHT, pre_us: float = 0.05, post_us: float = None):
    """(t_start_us, n_ticks) covering the deposits' times with a pre-buffer and
    a post-buffer of the truncated slow component plus the table's spread."""
    if post_us is None:
        post_us = L["trunc_taus"] * L["tau_slow_us"] + (L["nt"] + L["n_resp"]) * L["tick_us"]
    t0 = t_first_us - pre_us
    n = int(np.ceil((t_last_us + post_us - t0) / L["tick_us"]))
    return float(np.float32(t0)), n
