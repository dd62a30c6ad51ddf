"""Synthetic field-response look-up table I_pixel[x, y, t].

The paper's table (Sec. 3.3.1) comes from an FEM model and drift-path
integration that are not available here.  This module writes a closed-form
stand-in with the same layout and properties the method relies on:

* one quadrant of the 3x3-pixel neighbourhood, indexed by the folded offset
  (|dx|, |dy|) of the charge from the pixel centre, in bins of pitch/30
  (45 bins = 1.5 pitch; the paper uses 20 bins of 0.33 mm);
* one series per (x, y) bin in units of electrons per tick, with the charge
  arriving at the end of the last tick (row L-1);
* each series is a point-pixel dipole (image-charge) shape, normalised so that
  it integrates to one electron, as the paper's series are (Sec. 3.3.1);
* the transverse share is a quadratic B-spline of the offset, so that the
  shares of all pixels sum to one for any charge position.

Layout: float[nb][nb][ld] with ld >= nt (rows zero-padded to ld).
"""
from __future__ import annotations

import numpy as np


def bspline2(u: np.ndarray) -> np.ndarray:
    """Quadratic cardinal B-spline, support |u| < 3/2, partition of unity."""
    a = np.abs(u)
    out = np.zeros_like(a, dtype=np.float64)
    m1 = a <= 0.5
    m2 = (a > 0.5) & (a < 1.5)
    out[m1] = 0.75 - a[m1] ** 2
    out[m2] = 0.5 * (1.5 - a[m2]) ** 2
    return out


def make_lut(pitch_cm: float, vdrift_cm_us: float, tick_us: float,
             nb: int = 45, nt: int = 1950, bins_per_pitch: int = 30,
             z0_cm: float = 0.1, bipolar: float = 0.0) -> np.ndarray:
    """Return the FP64 table R[bx, by, j], shape (nb, nb, nt).

    R = w(u_x/p) w(u_y/p) g(j; r) with u_b = (b + 1/2) h, h = p/bins_per_pitch,
    r = sqrt(u_x^2 + u_y^2), g(j; r) proportional to
    (z_j + z0) / ((z_j + z0)^2 + r^2)^{3/2}, z_j = v_d (nt - 1 - j + 1/2) dt,
    normalised to sum 1 over j.  ``bipolar`` adds c w w (g(r) - g(r + p)),
    a zero-integral term that makes neighbour currents bipolar.
    """
    p = float(pitch_cm)
    h = p / bins_per_pitch
    u = (np.arange(nb, dtype=np.float64) + 0.5) * h
    w = bspline2(u / p)
    j = np.arange(nt, dtype=np.float64)
    zj = vdrift_cm_us * (nt - 1 - j + 0.5) * tick_us

    def g(r):
        zz = zj[None, None, :] + z0_cm
        k = zz / (zz ** 2 + r[..., None] ** 2) ** 1.5
        return k / k.sum(axis=-1, keepdims=True)

    r = np.sqrt(u[:, None] ** 2 + u[None, :] ** 2)
    ww = (w[:, None] * w[None, :])[..., None]
    lut = ww * g(r)
    if bipolar:
        lut = lut + bipolar * ww * (g(r) - g(r + p))
    return lut


def pad_rows(lut: np.ndarray, ld: int | None = None, dtype=np.float32) -> np.ndarray:
    """Copy ``lut`` into rows of length ``ld`` (default: nt rounded up to 4)."""
    nb0, nb1, nt = lut.shape
    if ld is None:
        ld = (nt + 3) // 4 * 4
    out = np.zeros((nb0, nb1, ld), dtype=dtype)
    out[..., :nt] = lut
    return out


def lut_for(cfg: dict, lut_par: dict, **kw) -> np.ndarray:
    """FP64 table for a configuration dict (pitch, drift velocity, tick from ``cfg``)."""
    p = float(np.float32(cfg["pitch_cm"]))
    v = float(np.float32(cfg["vdrift_cm_us"]))
    dt = float(np.float32(cfg["tick_us"]))
    return make_lut(p, v, dt, nb=lut_par["nb"], nt=lut_par["nt"],
                    bins_per_pitch=lut_par["bins_per_pitch"], z0_cm=lut_par["z0_cm"], **kw)
