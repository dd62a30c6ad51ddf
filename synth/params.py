"""Detector, physics, sampling, readout and front-end parameters.

Plain numbers only: no arithmetic of the simulated method lives here.  Both
the CUDA path and the FP64 oracle receive these values; floating-point
entries are carried as FP32 by the C ABI, so every consumer first rounds them
with :func:`as_f32` and the oracle then widens the FP32 value to FP64.

Sources (arXiv:2212.09807):
  * recombination constants A_b, k_b (Birks) and alpha, beta (modified Box):
    Sec. 3.1, Eqs. (birks) and (box);
  * diffusion coefficients D_L = 4 cm^2/s, D_T = 8.8 cm^2/s: Sec. 3.2;
  * 0.1 us tick / 10 MHz clock, 1.6 us hold, 11-cycle minimum ADC interval,
    900/650/500 e- noises, 8-bit ADC: Sec. 3.3.1 and Sec. 3.4;
  * pixel pitch 0.4434 cm, 70x70 pixels per tile, 0.5 kV/cm: Sec. 6;
  * gain 250 e-/mV: Sec. 6.
Values the paper does not give (LAr density, W_ion, ADC LSB, LUT shape,
threshold of the synthetic workloads) are stated readings of this project.
"""
from __future__ import annotations

import copy
import numpy as np

BASE = dict(
    # geometry: modules tile the x-y plane; each module holds n_tpc drift
    # volumes along z (anode of TPC 0 at z=0, cathode at z=drift_len, anode of
    # TPC 1 at z=2*drift_len); every anode is tiles_x x tiles_y LArPix tiles.
    n_mod_x=1, n_mod_y=1, n_tpc=2, tiles_x=1, tiles_y=1, px_per_tile=70,
    pitch_cm=0.4434, drift_len_cm=30.0,
    # recombination (0 = Birks, 1 = modified Box)
    recomb_model=0, birks_Ab=0.800, birks_kb=0.0486, box_alpha=0.93,
    box_beta=0.207, efield_kV_cm=0.5, lar_density_g_cm3=1.38,
    w_ion_MeV=23.6e-6,
    # drift
    vdrift_cm_us=0.16, lifetime_us=2200.0, diff_long_cm2_s=4.0,
    diff_tran_cm2_s=8.8,
    # sampling of eq. (current): 10 um points, M perturbations each
    sample_step_cm=1.0e-3, mc_per_sample=1, diff_clip_sigma=4.0,
    # readout window
    tick_us=0.1, n_ticks=2000, t_window0_us=0.0,
    # LArPix-like front end
    thr_e=5000.0, sigma_reset_e=900.0, sigma_disc_e=650.0, sigma_unc_e=500.0,
    gain_e_per_mV=250.0, adc_lsb_mV=1000.0 / 256.0, hold_ticks=16,
    min_adc_interval_ticks=11, periodic_reset_ticks=0, adc_bits=8,
    # counter-based RNG seed and arithmetic form of the current step
    seed=0x221209807, precision=0, fp64_charge=0, per_point_drift=0, nearest_lut=0,
)

# Field-response look-up table (synthetic closed form, see synth.response)
LUT = dict(nb=45, nt=1950, bins_per_pitch=30, z0_cm=0.1)

FLOAT_KEYS = {k for k, v in BASE.items() if isinstance(v, float)}


def as_f32(cfg: dict) -> dict:
    """Round every floating-point parameter to its FP32 value (as the ABI carries it)."""
    out = dict(cfg)
    for k in FLOAT_KEYS:
        out[k] = float(np.float32(out[k]))
    return out


def tile_config(**over) -> dict:
    """One TPC behind a single 70x70 anode tile (the 200-segment muon workload)."""
    c = copy.deepcopy(BASE)
    c.update(n_mod_x=1, n_mod_y=1, n_tpc=1, tiles_x=1, tiles_y=1)
    c.update(over)
    return c


def module_config(**over) -> dict:
    """One detector module: 2 TPCs sharing a cathode, anodes of 4x5 tiles."""
    c = copy.deepcopy(BASE)
    c.update(n_mod_x=1, n_mod_y=1, n_tpc=2, tiles_x=4, tiles_y=5)
    c.update(over)
    return c


def spill_config(**over) -> dict:
    """A 7x5 array of modules (35 modules, 70 anodes)."""
    c = module_config()
    c.update(n_mod_x=7, n_mod_y=5)
    c.update(over)
    return c


def small_config(**over) -> dict:
    """Small multi-tile case for parity tests: 1 module, 2 TPCs, 2x2 tiles."""
    c = copy.deepcopy(BASE)
    c.update(n_mod_x=1, n_mod_y=1, n_tpc=2, tiles_x=2, tiles_y=2)
    c.update(over)
    return c


def geometry(cfg: dict) -> dict:
    """Derived extents in cm (plain products of the configuration numbers)."""
    p = float(np.float32(cfg["pitch_cm"]))
    nx = cfg["tiles_x"] * cfg["px_per_tile"]
    ny = cfg["tiles_y"] * cfg["px_per_tile"]
    D = float(np.float32(cfg["drift_len_cm"]))
    return dict(pitch=p, npx_x=nx, npx_y=ny, mod_w=nx * p, mod_h=ny * p,
                x_max=cfg["n_mod_x"] * nx * p, y_max=cfg["n_mod_y"] * ny * p,
                z_max=cfg["n_tpc"] * D, drift=D,
                n_anodes=cfg["n_mod_x"] * cfg["n_mod_y"] * cfg["n_tpc"],
                n_pixels=cfg["n_mod_x"] * cfg["n_mod_y"] * cfg["n_tpc"] * nx * ny)
