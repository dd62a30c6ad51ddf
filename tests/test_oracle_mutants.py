"""The oracle's pins against planted mistakes (CPU only).

Each mutant below is one plausible slip in the FP64 oracle -- a dropped term,
a wrong sign, index or constant, a transposed operand -- planted in a copy of
the oracle package (``larsim_oracle.c`` or ``__init__.py``) in a scratch
folder of the repository (``_build/``, git-ignored, removed afterwards).  The copy is compiled there and imported as ``oracle``, and the
oracle's pin tests (tests/test_oracle_*.py) run against it: every mutant must
fail at least one pin.  An unchanged copy run the same way must pass them all
(the control), so that a failure means the pins saw the mistake and not the
harness.

The committed oracle is never modified: the mistakes live only in the copies.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "larsim_oracle.c")
PY = os.path.join(ROOT, "oracle", "__init__.py")
PIN_FILES = ["test_oracle_rng_quench_drift.py", "test_oracle_map_current.py", "test_oracle_electronics.py",
             "test_oracle_hits_post.py", "test_oracle_light.py"]

# (name, the passage the mistake breaks, pin file tried first, original text, planted text)
MUTANTS = [
    # counter-based generator (Salmon et al., SC'11) and its normals
    ("philox_key_word", "Philox4x32-10 round", "rng", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c1 ^ k1;"),
    ("philox_weyl_constant", "Philox4x32-10 key schedule", "rng", "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    ("box_muller_partner", "Box-Muller pair", "rng", "n[1] = r0 * sin(a0);", "n[1] = r0 * cos(a0);"),
    # Sec. 3.1: recombination and quenching
    ("birks_field_inverted", "Sec. 3.1 Eq. (birks)", "rng",
     "return c->Ab / (1.0 + c->kb / eps * dEdx);", "return c->Ab / (1.0 + c->kb * eps * dEdx);"),
    ("box_denominator_no_field", "Sec. 3.1 Eq. (box)", "rng",
     "return log(c->alpha + xi) / xi;", "return log(c->alpha + xi) / (c->beta * dEdx);"),
    ("epsilon_without_density", "Sec. 3.1 (epsilon = E rho)", "rng",
     "double eps = c->efield * c->density;", "double eps = c->efield;"),
    ("q0_times_w_ion", "Sec. 3.1 (Q_0 = E / W_ion)", "rng",
     "double Q0 = (double)dE[i] / c->w_ion;", "double Q0 = (double)dE[i] * c->w_ion;"),
    # Sec. 3.2: drift, lifetime, diffusion
    ("drift_from_z0_not_anode", "Sec. 3.2 Eq. (drift)", "rng",
     "double td = fabs(zm - L.za) / c->vdrift;", "double td = fabs(zm) / c->vdrift;"),
    ("lifetime_sign", "Sec. 3.2 Eq. (lifetime)", "rng",
     "double qa = QR * exp(-td / c->lifetime);", "double qa = QR * exp(td / c->lifetime);"),
    ("sigma_T_from_D_L", "Sec. 3.2 (sigma_T = sqrt(2 D_T t))", "rng",
     "double sT = sqrt(2.0 * (c->DT * 1e-6) * tsig);", "double sT = sqrt(2.0 * (c->DL * 1e-6) * tsig);"),
    ("sigma_L_factor_two", "Sec. 3.2 (sigma_L = sqrt(2 D_L t))", "map",
     "double sL = sqrt(2.0 * (c->DL * 1e-6) * tsig);", "double sL = sqrt((c->DL * 1e-6) * tsig);"),
    ("points_floor", "Sec. 3.3.2 (points every 10 um)", "rng",
     "double N = ceil(dx / c->step);", "double N = floor(dx / c->step);"),
    ("anode_numbering_transposed", "Sec. 6 geometry (module order)", "rng",
     "L.anode = (my * c->n_mod_x + mx) * c->n_tpc + tpc;", "L.anode = (mx * c->n_mod_y + my) * c->n_tpc + tpc;"),
    # Sec. 3.3.2: pixel map
    ("pixel_centre_at_corner", "Sec. 3.3.2 (pixel centres)", "map",
     "*xc = (double)mx * Wx + ((double)ix + 0.5) * c->pitch;", "*xc = (double)mx * Wx + (double)ix * c->pitch;"),
    ("map_radius_half_bin_short", "Sec. 3.3.2 (table reach)", "map",
     "return ((double)c->nb + 0.5) * h + c->clip * sigma_T;", "return ((double)c->nb - 0.5) * h + c->clip * sigma_T;"),
    ("map_radius_no_diffusion", "Sec. 3.3.2 (diffusion reach)", "map",
     "return ((double)c->nb + 0.5) * h + c->clip * sigma_T;", "return ((double)c->nb + 0.5) * h;"),
    ("chebyshev_candidate_dropped", "Sec. 3.3.2 (segment-pixel distance)", "map",
     "    if (du + dv != 0.0) cand[nc++] = -(u0 + v0) / (du + dv);\n", ""),
    ("full_map_boundary_excluded", "Sec. 3.3.2 (distance exactly R_map is mapped)", "map",
     "            if (d <= R) {\n                if (cnt < cap) {\n                    ids[cnt] = pid;\n"
     "                    if (margin) margin[cnt] = R - d;\n                }\n                ++cnt;\n            }\n"
     "        }\n    }\n    return cnt;\n}\n\n/* Same map",
     "            if (d < R) {\n                if (cnt < cap) {\n                    ids[cnt] = pid;\n"
     "                    if (margin) margin[cnt] = R - d;\n                }\n                ++cnt;\n            }\n"
     "        }\n    }\n    return cnt;\n}\n\n/* Same map"),
    ("event_map_buffer_growth_short", "Sec. 3.3.2 (the whole event's map)", "map",
     "            bcap = m;\n", "            bcap = m - 1;\n"),
    ("event_map_not_recomputed_after_growth", "Sec. 3.3.2 (the whole event's map)", "map",
     "            m = ora_map_segment_box(c, x0[s], y0[s], x1[s], y1[s], sigma_T[s], anode[s], ids, mg, bcap);\n"
     "        }", "        }"),
    ("event_map_capacity_off_by_one", "Sec. 3.3.2 (the whole event's map)", "map",
     "            if (total < cap) {\n                pair_seg[total] = s;",
     "            if (total < cap - 1) {\n                pair_seg[total] = s;"),
    ("pair_margin_ignores_the_anode", "Sec. 3.2 (charge drifts to its own anode)", "map",
     "    if (g != anode || anode < 0) return -INFINITY;", "    if (anode < 0) return -INFINITY;"),
    ("pixel_row_and_column_transposed", "pixel ids (row-major over the anode)", "map",
     "int32_t iy = rem / nx, ix = rem % nx;", "int32_t iy = rem / ny, ix = rem % ny;"),
    ("pixel_module_order_transposed", "pixel ids (modules row-major)", "map",
     "int32_t mx = m % c->n_mod_x, my = m / c->n_mod_x;\n    double Wx",
     "int32_t mx = m / c->n_mod_y, my = m % c->n_mod_y;\n    double Wx"),
    ("module_row_from_width", "Sec. 6 geometry (module size)", "rng",
     "int my = (int)floor(y / Wy);", "int my = (int)floor(y / Wx);"),
    ("current_from_another_anode", "Sec. 3.2 (charge drifts to its own anode)", "map",
     "if (anode[s] != g) continue;", "if (0) continue;"),
    # Sec. 3.3.2: charge density rho and Eq. (current)
    ("points_at_interval_starts", "Sec. 3.3.2 (charge density rho)", "map",
     "double u = ((double)mu + 0.5) / (double)N;", "double u = (double)mu / (double)N;"),
    ("point_charge_without_M", "Sec. 3.3.2 (q = Q_a / (N M))", "map",
     "double q = Qa[s] / ((double)N * (double)c->M);", "double q = Qa[s] / (double)N;"),
    ("bilinear_corner_transposed", "Sec. 3.3.1 (table interpolation)", "map",
     "+ wx * (1.0 - wy) * ora_lut(c, lut, bx + 1, by, j)", "+ wx * (1.0 - wy) * ora_lut(c, lut, bx, by + 1, j)"),
    ("tick_weights_swapped", "Eq. (current), time interpolation", "map",
     "I[k] += qp * ((1.0 - f) * r1 + f * r2);", "I[k] += qp * (f * r1 + (1.0 - f) * r2);"),
    ("tick_index_off_by_one", "Eq. (current), table tick", "map",
     "int64_t j1 = (int64_t)k - A + L - 1;", "int64_t j1 = (int64_t)k - A + L;"),
    ("longitudinal_diffusion_dropped", "Sec. 3.3.2 (arrival time of a perturbed point)", "map",
     "double ta = t + fabs(zz - za) / c->vdrift;", "double ta = t + fabs(z - za) / c->vdrift;"),
    ("offset_not_bin_centred", "Sec. 3.3.1 (bin-centred nodes)", "map",
     "double xi = fabs(dxp) / h - 0.5;", "double xi = fabs(dxp) / h;"),
    ("transverse_normals_shared", "Sec. 3.3.2 (independent transverse perturbations)", "map",
     "double dyp = y + sTp * n[1] - yc;", "double dyp = y + sTp * n[0] - yc;"),
    ("per_point_lifetime_absolute", "Eq. (lifetime) per point", "map",
     "qp = q * exp(-(tp - t_drift[s]) / c->lifetime);", "qp = q * exp(-tp / c->lifetime);"),
    ("per_point_sigma_T_at_midpoint", "sigma_T = sqrt(2 D_T t) per point", "map",
     "sTp = sqrt(2.0 * (c->DT * 1e-6) * tp);", "sTp = sqrt(2.0 * (c->DT * 1e-6) * t_drift[s]);"),
    ("per_point_sigma_L_at_midpoint", "sigma_L = sqrt(2 D_L t) per point", "map",
     "sLp = sqrt(2.0 * (c->DL * 1e-6) * tp);", "sLp = sqrt(2.0 * (c->DL * 1e-6) * t_drift[s]);"),
    ("offsets_unclipped_above", "diffusion offsets clipped at +-clip", "map",
     "if (n[d] > c->clip) n[d] = c->clip;", "if (0) n[d] = c->clip;"),
    ("offsets_unclipped_below", "diffusion offsets clipped at +-clip", "map",
     "if (n[d] < -c->clip) n[d] = -c->clip;", "if (0) n[d] = -c->clip;"),
    ("point_time_not_interpolated", "Sec. 3.3.2 (points along the segment in time)", "map",
     "double t = (double)t0[s] + u * ((double)t1[s] - (double)t0[s]);", "double t = (double)t0[s];"),
    # Sec. 3.4: front end
    ("csa_not_integrating", "Sec. 3.4 (CSA integrates the current)", "elec", "q += I[k];", "q = I[k];"),
    ("periodic_reset_keeps_charge", "Sec. 3.4 (periodic reset)", "elec",
     "            q = c->s_reset * n[0];\n        }", "            q += c->s_reset * n[0];\n        }"),
    ("hold_one_tick_short", "Sec. 3.4 (hold time)", "elec", "ta = k + c->hold;", "ta = k + c->hold - 1;"),
    ("min_adc_interval_dropped", "Sec. 3.4 (minimum ADC interval)", "elec",
     "if (last_adc + c->min_int > ta) ta = last_adc + c->min_int;", "if (0) ta = last_adc + c->min_int;"),
    ("adc_rounds_to_nearest", "Sec. 3.4 (ADC)", "elec",
     "double code = floor(v / lsb_e);", "double code = floor(v / lsb_e + 0.5);"),
    ("threshold_without_noise", "Sec. 3.4 (discriminator with noise)", "elec", "if (v >= thr) {", "if (q >= thr) {"),
    ("reset_without_pedestal", "Sec. 3.4 (reset noise)", "elec", "q = c->s_reset * m[0];", "q = 0.0;"),
    ("discriminator_noise_shared", "Sec. 3.4 (independent noise sources)", "elec",
     "double thr = c->thr + c->s_disc * n[1];", "double thr = c->thr + c->s_disc * n[0];"),
    ("lsb_without_gain", "Sec. 3.4 (ADC LSB in electrons)", "elec",
     "double lsb_e = c->gain * c->lsb_mV;", "double lsb_e = c->lsb_mV;"),
    ("adc_not_saturating", "Sec. 3.4 (ADC range)", "elec",
     "if (code > adc_max) code = adc_max;", "if (0) code = adc_max;"),
    ("adc_range_off_by_one", "Sec. 3.4 (ADC range)", "elec",
     "int adc_max = (1 << c->adc_bits) - 1;", "int adc_max = (1 << c->adc_bits);"),
    ("adc_negative_codes", "Sec. 3.4 (ADC range)", "elec", "if (code < 0) code = 0;", "if (0) code = 0;"),
    ("periodic_reset_at_window_start", "Sec. 3.4 (periodic reset)", "elec",
     "if (c->periodic > 0 && idle && k > 0 && k % c->periodic == 0) {",
     "if (c->periodic > 0 && idle && k % c->periodic == 0) {"),
    ("periodic_reset_while_busy", "Sec. 3.4 (periodic reset while idle)", "elec",
     "if (c->periodic > 0 && idle && k > 0 && k % c->periodic == 0) {",
     "if (c->periodic > 0 && k > 0 && k % c->periodic == 0) {"),
    # after the front end (per-hit truth, hit points, dQ/dx)
    ("hit_interval_overlaps_previous", "Sec. 3.4 (integration since the last reset)", "hits",
     "int64_t start = prev_end + 1;", "int64_t start = prev_end;"),
    ("hit_point_direction", "Sec. 6 (inverse of Eq. (drift))", "hits",
     "out[2] = za == 0.0 ? za + dz : za - dz;", "out[2] = za + dz;"),
    ("dqdx_piece_rounded", "Sec. 6 (dQ/dx pieces)", "hits",
     "double fb = floor(s / dx);", "double fb = floor(s / dx + 0.5);"),
    ("dqdx_distance_without_z", "Sec. 6 (distance from the track)", "hits",
     "double d = sqrt(ex * ex + ey * ey + ez * ez);", "double d = sqrt(ex * ex + ey * ey);"),
    # the margins and tie counts the GPU parity tests excuse near-boundary decisions by
    ("dqdx_margin_without_piece_edges", "Sec. 6 (dQ/dx pieces)", "hits",
     "        if (ms < m) m = ms;", "        (void)ms;"),
    ("digitiser_margin_one_sided", "Sec. 4.3 (ADC)", "light",
     "margin[m] = fmin(w - cd, cd + 1.0 - w);", "margin[m] = w - cd;"),
    ("poisson_margin_dropped", "Sec. 4.2 (Poisson fluctuations)", "light",
     "            if (m2 < mg) mg = m2;", "            (void)m2;"),
    ("nearest_ties_not_counted", "nearest-lookup variant", "map",
     "if (mx < tie_band || my < tie_band || ma < tie_band) ++ties;", "if (0) ++ties;"),
    # Sec. 4: light
    ("photons_without_quenched_charge", "Sec. 4.1 (N_gamma)", "light",
     "double ngam = (double)p[8] / L->w_ph - QR;", "double ngam = (double)p[8] / L->w_ph;"),
    ("scintillation_fast_unnormalised", "Sec. 4.2 (scintillation time profile)", "light",
     "double f = L->fast_frac / L->tau_fast * exp(-tu / L->tau_fast) +",
     "double f = L->fast_frac * exp(-tu / L->tau_fast) +"),
    ("photocurrent_shift_reversed", "Sec. 4.2 Eq. (photocurrent)", "light",
     "int64_t t = (int64_t)tick[j] + u;", "int64_t t = (int64_t)tick[j] - u;"),
    ("poisson_switch_excludes_its_bound", "Sec. 4.2 (Poisson up to a mean of 30)", "light",
     "if (lam <= L->poisson_max) {", "if (lam < L->poisson_max) {"),
    ("poisson_term_index", "Sec. 4.2 (Poisson fluctuations)", "light",
     "pk *= lam / (double)k;", "pk *= lam / (double)(k + 1);"),
    ("digitiser_weights_swapped", "Sec. 4.3 (sampling)", "light",
     "(1.0 - fr) * V[i] + fr * V[i + 1]", "fr * V[i] + (1.0 - fr) * V[i + 1]"),
    ("scintillation_sum_without_its_last_term", "Sec. 4.2 (truncated convolution)", "light",
     "int umax = t < L->n_trunc ? t : L->n_trunc;", "int umax = L->n_trunc < t ? L->n_trunc : (t > 0 ? t - 1 : 0);"),
    ("digitiser_last_tick_dropped", "Sec. 4.3 (sampling)", "light",
     "double v = i + 1 < L->n_ticks ? (1.0 - fr) * V[i] + fr * V[i + 1] : V[i];",
     "double v = i + 1 < L->n_ticks ? (1.0 - fr) * V[i] + fr * V[i + 1] : 0.0;"),
    ("light_truth_bin_start", "Sec. 4.4 (mean arrival time)", "light",
     "m += ((double)u + 0.5) * f[u];", "m += (double)u * f[u];"),
    ("light_depth_from_z0", "Sec. 4.1 (voxel of the segment's own drift volume)", "light",
     "float zl = fabsf(zm - za);", "float zl = fabsf(zm);"),
    ("light_voxel_transposed", "Sec. 4.1 (visibility voxel)", "light",
     "int v = (ix * L->nvy + iy) * L->nvz + iz;", "int v = (iy * L->nvx + ix) * L->nvz + iz;"),
    ("photocurrent_all_anodes", "Sec. 4.2 Eq. (photocurrent) per anode", "light",
     "if (anode[j] != a || vox[j] < 0) continue;", "if (vox[j] < 0) continue;"),
    ("scintillation_truncation_short", "Sec. 4.2 (truncated convolution)", "light",
     "int umax = t < L->n_trunc ? t : L->n_trunc;", "int umax = t < L->n_trunc ? t : L->n_trunc - 1;"),
]

# the same, planted in the Python half of the oracle (configuration marshalling, interval sums, light setup)
PY_MUTANTS = [
    ("cfg_diffusion_swapped", "Sec. 3.2 (D_L and D_T)", "rng",
     'c.DL, c.DT = _f32(cfg["diff_long_cm2_s"]), _f32(cfg["diff_tran_cm2_s"])',
     'c.DT, c.DL = _f32(cfg["diff_long_cm2_s"]), _f32(cfg["diff_tran_cm2_s"])'),
    ("cfg_noise_swapped", "Sec. 3.4 (discriminator and uncorrelated noise)", "elec",
     'c.s_disc, c.s_unc = _f32(cfg["sigma_disc_e"]), _f32(cfg["sigma_unc_e"])',
     'c.s_unc, c.s_disc = _f32(cfg["sigma_disc_e"]), _f32(cfg["sigma_unc_e"])'),
    ("hit_truth_drops_adc_tick", "Sec. 3.4 (integration up to the ADC tick)", "hits",
     "Q = cs[:, k1 + 1].T - cs[:, k0].T", "Q = cs[:, k1].T - cs[:, k0].T"),
    ("scintillation_truncation_floored", "Sec. 4.2 (truncation length)", "light",
     "/ tick + 0.5))", "/ tick))"),
    ("light_samples_short", "Sec. 4.3 (samples of the window)", "light",
     "n_samples = int(np.floor((n_ticks - 1) / ratio)) + 1", "n_samples = int(np.floor((n_ticks - 1) / ratio))"),
    ("light_sampling_ratio_inverted", "Sec. 4.3 (sampling period in ticks)", "light",
     'ratio = _f32(L["sample_us"]) / tick', 'ratio = tick / _f32(L["sample_us"])'),
    ("cfg_hold_and_interval_swapped", "Sec. 3.4 (hold, minimum ADC interval)", "elec",
     'c.hold, c.min_int = int(cfg["hold_ticks"]), int(cfg["min_adc_interval_ticks"])',
     'c.min_int, c.hold = int(cfg["hold_ticks"]), int(cfg["min_adc_interval_ticks"])'),
    ("cfg_window_start_ignored", "Eq. (current), arrival tick", "map",
     'c.tick, c.n_ticks, c.t_w0 = _f32(cfg["tick_us"]), int(cfg["n_ticks"]), _f32(cfg["t_window0_us"])',
     'c.tick, c.n_ticks, c.t_w0 = _f32(cfg["tick_us"]), int(cfg["n_ticks"]), 0.0'),
    ("cfg_box_parameters_swapped", "Sec. 3.1 Eq. (box)", "rng",
     'c.alpha, c.beta = _f32(cfg["box_alpha"]), _f32(cfg["box_beta"])',
     'c.beta, c.alpha = _f32(cfg["box_alpha"]), _f32(cfg["box_beta"])'),
    ("cfg_density_typo", "Sec. 3.1 (epsilon = E rho)", "rng",
     'c.efield, c.density = _f32(cfg["efield_kV_cm"]), _f32(cfg["lar_density_g_cm3"])',
     'c.efield, c.density = _f32(cfg["efield_kV_cm"]), 1.396'),
    ("cfg_per_point_ignored", "per-point drift variant", "map",
     'c.per_point = int(cfg.get("per_point_drift", 0))', "c.per_point = 0"),
    ("cfg_nearest_ignored", "nearest-lookup variant", "map",
     'c.nearest = int(cfg.get("nearest_lut", 0))', "c.nearest = 0"),
    ("cfg_seed_truncated", "Philox key = seed ^ event id", "rng",
     'c.seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF', 'c.seed = int(cfg["seed"]) & 0xFFFFFFFF'),
    ("light_time_constants_swapped", "Sec. 4.2 (scintillation time profile)", "light",
     'l.fast_frac, l.tau_fast, l.tau_slow = _f32(L["fast_frac"]), _f32(L["tau_fast_us"]), _f32(L["tau_slow_us"])',
     'l.fast_frac, l.tau_slow, l.tau_fast = _f32(L["fast_frac"]), _f32(L["tau_fast_us"]), _f32(L["tau_slow_us"])'),
    ("light_pedestal_dropped", "Sec. 4.3 (ADC pedestal)", "light",
     'l.poisson_max, l.sample, l.pedestal = _f32(L["poisson_max_mean"]), _f32(L["sample_us"]), _f32(L["pedestal"])',
     'l.poisson_max, l.sample, l.pedestal = _f32(L["poisson_max_mean"]), _f32(L["sample_us"]), 0.0'),
    ("hit_signal_drops_adc_tick", "Sec. 3.4 (integration up to the ADC tick)", "hits",
     "return Q, full[k1 + 1] - full[k0], k0, k1", "return Q, full[k1] - full[k0], k0, k1"),
    ("pixel_side_map_boundary_excluded", "Sec. 3.3.2 (distance exactly R_map is mapped)", "map",
     "            if m >= 0:\n                out.append(s)", "            if m > 0:\n                out.append(s)"),
    ("cfg_w_ion_doubled", "Sec. 3.1 (Q_0 = E / W_ion)", "rng",
     'c.w_ion = _f32(cfg["w_ion_MeV"])', 'c.w_ion = 2 * _f32(cfg["w_ion_MeV"])'),
    ("light_voxel_size_off", "Sec. 4.1 (visibility voxel)", "light",
     'l.vox, l.w_ph, l.tick = _f32(L["vox_cm"]), _f32(L["w_ph_MeV"]), _f32(L["tick_us"])',
     'l.vox, l.w_ph, l.tick = 1.05 * _f32(L["vox_cm"]), _f32(L["w_ph_MeV"]), _f32(L["tick_us"])'),
]

FIRST = {"rng": "test_oracle_rng_quench_drift.py", "map": "test_oracle_map_current.py",
         "elec": "test_oracle_electronics.py", "hits": "test_oracle_hits_post.py", "light": "test_oracle_light.py"}

PLUGIN = '''
import importlib.util
import sys
spec = importlib.util.spec_from_file_location("oracle", {init!r}, submodule_search_locations=[{pkg!r}])
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle"] = mod
spec.loader.exec_module(mod)
mod.build(force=True)
'''


def _run_pins(workdir, c_source, py_source, first):
    """Copy the oracle package into `workdir` with the given sources, compile
    it, import it as `oracle` and run the pin tests on it (the file `first`
    before the others, stopping at the first failure).  Returns (pytest exit
    code, the first failing test or '', output tail)."""
    pkg = os.path.join(workdir, "oracle")
    os.makedirs(pkg, exist_ok=True)
    with open(os.path.join(pkg, "larsim_oracle.c"), "w") as f:
        f.write(c_source)
    with open(os.path.join(pkg, "__init__.py"), "w") as f:
        f.write(py_source)
    with open(os.path.join(workdir, "mutant_oracle_plugin.py"), "w") as f:
        f.write(PLUGIN.format(init=os.path.join(pkg, "__init__.py"), pkg=pkg))
    files = [first] + [p for p in PIN_FILES if p != first]
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([workdir, ROOT]), OMP_NUM_THREADS="1",
               PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-p", "mutant_oracle_plugin",
           "-m", "not gpu"] + [os.path.join(ROOT, "tests", p) for p in files]
    r = subprocess.run(cmd, cwd=workdir, env=env, capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    m = re.search(r"FAILED (\S+)", out)
    if not os.path.exists(os.path.join(pkg, "liblarsim_oracle.so")):
        return -1, "", out[-2000:]                   # the copy did not build or load: not a pin's catch
    return r.returncode, m.group(1).split("/")[-1] if m else "", out[-2000:]


SCRATCH = os.path.join(ROOT, "_build", "oracle_mutants")     # git-ignored; removed after the run


@pytest.fixture(scope="module")
def results():
    base_c, base_py = open(SRC).read(), open(PY).read()
    jobs = {"control": (base_c, base_py, FIRST["rng"])}
    for name, _, first, old, new in MUTANTS:
        assert base_c.count(old) == 1, (name, "the planted text must match exactly one place")
        jobs[name] = (base_c.replace(old, new), base_py, FIRST[first])
    for name, _, first, old, new in PY_MUTANTS:
        assert base_py.count(old) == 1, (name, "the planted text must match exactly one place")
        jobs[name] = (base_c, base_py.replace(old, new), FIRST[first])
    shutil.rmtree(SCRATCH, ignore_errors=True)
    workers = max(1, min(8, os.cpu_count() or 1))
    try:
        with cf.ThreadPoolExecutor(workers) as ex:
            fut = {k: ex.submit(_run_pins, os.path.join(SCRATCH, k), c, py, f) for k, (c, py, f) in jobs.items()}
            out = {k: f.result() for k, f in fut.items()}
    finally:
        shutil.rmtree(SCRATCH, ignore_errors=True)
        try:
            os.rmdir(os.path.dirname(SCRATCH))            # _build/ too, when nothing else is in it
        except OSError:
            pass
    return out


def test_unchanged_copy_passes_every_pin(results):
    rc, failed, tail = results["control"]
    assert rc == 0, (failed, tail)


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS + PY_MUTANTS])
def test_planted_mistake_fails_a_pin(results, name):
    rc, failed, tail = results[name]
    assert rc == 1 and failed, f"{name} was not caught by any pin (rc {rc}):\n{tail}"
