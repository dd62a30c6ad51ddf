// current_records.cuh -- the per-(point, pixel) record of Eq. (current)
// (arXiv:2212.09807 Sec. 3.3.2) shared by both arithmetic forms of the
// induced-current step, so that both sum exactly the same terms.
#pragma once

#include "sim_internal.cuh"

namespace larsim {

// One perturbed point seen from one pixel: arrival tick A + f (integer part
// and fraction), the table bin b0 = bx * nb + by of the folded offset
// (bx, by), and the q-scaled bilinear weights of the four table rows
// (bx, by), (bx+1, by), (bx, by+1), (bx+1, by+1) (zero for rows beyond the table).
struct __align__(16) Rec {
    int A, b0;
    float f, pad;
    float4 w;
};

// Pixel-independent part of the record of point `idx` (= mu M + nu) of a
// segment: position in pitch units relative to the anchor's reference pixel
// corner, the arrival tick relative to the anchor's A0, and the charge.
struct PointPos {
    float fx, fy, lin, q;
};

// Drift constants for per-point lifetime and widths (Sec. 3.2 evaluated at
// each point): off when per_point == 0.
struct DriftPar {
    int per_point;
    float inv_vd, inv_tau, two_dt, two_dl, inv_pitch;   // us/cm, 1/us, cm^2/us, cm^2/us, 1/cm
};

inline DriftPar drift_par_of(const sim_config &c)
{
    DriftPar d;
    d.per_point = c.per_point_drift;
    d.inv_vd = 1.0f / c.vdrift_cm_us;
    d.inv_tau = 1.0f / c.lifetime_us;
    d.two_dt = 2.0f * (c.diff_tran_cm2_s * 1e-6f);
    d.two_dl = 2.0f * (c.diff_long_cm2_s * 1e-6f);
    d.inv_pitch = 1.0f / c.pitch_cm;
    return d;
}

__device__ __forceinline__ PointPos point_position(const Anchor &A, int idx, int M, uint64_t key,
                                                   uint32_t seg_local, float clip, const DriftPar &dp)
{
    const int mu = (M == 1) ? idx : idx / M;
    float3 n = normals3(key, seg_local, (uint32_t)idx, 1u);
    n.x = fminf(fmaxf(n.x, -clip), clip);
    n.y = fminf(fmaxf(n.y, -clip), clip);
    n.z = fminf(fmaxf(n.z, -clip), clip);
    const float u = ((float)mu + 0.5f) / (float)A.N;
    float sTp = A.sTp, sLc = A.sLc, q = A.q;
    if (dp.per_point) {
        // the point's own drift time; the anchor's charge carries the midpoint's attenuation
        const float t = fabsf(A.d0 + u * A.dd) * dp.inv_vd;
        const float tm = fabsf(A.d0 + 0.5f * A.dd) * dp.inv_vd;
        q = A.q * expf(-(t - tm) * dp.inv_tau);
        sTp = sqrtf(dp.two_dt * t) * dp.inv_pitch;
        sLc = A.sLc * sqrtf(dp.two_dl * t);          // A.sLc holds the drift direction (+-1)
    }
    PointPos p;
    p.fx = A.fx0 + u * A.dX + sTp * n.x;
    p.fy = A.fy0 + u * A.dY + sTp * n.y;
    float lin = A.fa0 + u * A.da + sLc * n.z * A.kz;
    const float dmu = A.d0 + u * A.dd + sLc * n.z;
    if (dmu < 0.f) lin -= 2.0f * dmu * A.kz;     // charge beyond the anode plane drifts back
    p.lin = lin;
    p.q = q;
    return p;
}

// Points of a segment that can reach the pixel whose centre is (cx, cy): a
// record needs the point's transverse offsets below (nb + 1/2) / bpp pitch,
// and a point lies within clip * sTp of its undiffused position
// (fx0 + u dX, fy0 + u dY) at u = (mu + 1/2) / N (sTp bounds every point's
// width, also under per-point drift).  Returns the range [i_lo, i_hi) of
// point indices idx = mu M + nu whose undiffused position lies within that
// reach in x and y (slab intersection), widened by one point each side and by
// 1e-3 pitch against rounding: every point outside it is rejected by
// point_record, so generating only this range changes no record.  (Used by
// the per-hit truth, where it saves 16 %; in both current kernels measured
// 1-2 % slower, so they generate every point.)
__device__ __forceinline__ void point_range(const Anchor &A, int M, float cx, float cy, float fbpp, int nb,
                                            float clip, int &i_lo, int &i_hi)
{
    const float R = ((float)nb + 0.5f) / fbpp + clip * A.sTp + 1e-3f;
    float u0 = 0.f, u1 = 1.f;
    const float d[2] = {A.dX, A.dY}, o[2] = {A.fx0 - cx, A.fy0 - cy};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (fabsf(d[k]) < 1e-12f) {
            if (fabsf(o[k]) >= R) u1 = -1.f;              // never within reach
        } else {
            const float ta = (-R - o[k]) / d[k], tb = (R - o[k]) / d[k];
            u0 = fmaxf(u0, fminf(ta, tb));
            u1 = fminf(u1, fmaxf(ta, tb));
        }
    }
    if (!(u0 <= u1)) {
        i_lo = i_hi = 0;
        return;
    }
    const float N = (float)A.N;
    const int mu0 = max(0, (int)floorf(u0 * N - 0.5f) - 1);
    const int mu1 = min(A.N - 1, (int)ceilf(u1 * N - 0.5f) + 1);
    i_lo = mu0 * M;
    i_hi = mu1 >= mu0 ? (mu1 + 1) * M : i_lo;
}

// Record of a point for the pixel whose centre is (cx, cy) in the same pitch
// units; false when the folded offset is beyond the table (nb bins of 1/bpp
// pitch in x or y).  nearest: the nearest node and the nearest tick (halves
// round up) instead of the bilinear/linear reads; node nb reads zero.
__device__ __forceinline__ bool point_record(const Anchor &A, const PointPos &p, float cx, float cy, float fbpp,
                                             int nb, int nearest, Rec &r)
{
    const float fnb = (float)nb;
    const float xi = fmaxf(fabsf((p.fx - cx) * fbpp) - 0.5f, 0.f);
    const float yi = fmaxf(fabsf((p.fy - cy) * fbpp) - 0.5f, 0.f);
    if (!(xi < fnb && yi < fnb)) return false;
    if (nearest) {
        const int nx = (int)floorf(xi + 0.5f), ny = (int)floorf(yi + 0.5f);
        if (nx >= nb || ny >= nb) return false;
        r.A = A.A0 + (int)floorf(p.lin + 0.5f);
        r.b0 = nx * nb + ny;
        r.f = 0.f;
        r.pad = 0.f;
        r.w = make_float4(p.q, 0.f, 0.f, 0.f);
        return true;
    }
    const float fl = floorf(p.lin);
    const int bx = (int)xi, by = (int)yi;
    const float wx = xi - (float)bx, wy = yi - (float)by;
    // node nb (beyond the table) reads zero: far corners get no weight
    const float ex = (bx + 1 < nb) ? 1.f : 0.f, ey = (by + 1 < nb) ? 1.f : 0.f;
    const float q1 = p.q * (1.f - wx), q2 = p.q * wx * ex;
    r.A = A.A0 + (int)fl;
    r.b0 = bx * nb + by;
    r.f = p.lin - fl;
    r.pad = 0.f;
    r.w = make_float4(q1 * (1.f - wy), q2 * (1.f - wy), q1 * wy * ey, q2 * wy * ey);
    return true;
}

}  // namespace larsim
