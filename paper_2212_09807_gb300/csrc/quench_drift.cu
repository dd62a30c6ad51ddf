// quench_drift.cu -- steps 1-2 of the charge path (arXiv:2212.09807 Sec. 3.1
// and Sec. 3.2): recombination (Eq. birks / Eq. box), drift time
// (Eq. drift), lifetime attenuation (Eq. lifetime) and diffusion widths
// sigma = sqrt(2 D t), one thread per segment, plus the per-segment sampling
// anchor consumed by the pixel map and the induced-current kernel.
//
// HBM-bound elementwise pass: 36 B of SoA input and 88 B of output per
// segment, coalesced 4-byte column loads and 16-byte anchor stores.
#include "sim_internal.cuh"

namespace larsim {

// Drift volume of the midpoint, decided in FP64 with explicitly rounded
// operations (no contraction) so that the decision is reproducible.
struct Loc {
    int ok, anode, mx, my, tpc;
    double ox, oy, za;
};

__device__ __forceinline__ Loc locate(const sim_config &c, double x, double y, double z)
{
    Loc L;
    const double pitch = (double)c.pitch_cm;
    const double D = (double)c.drift_len_cm;
    const double Wx = __dmul_rn((double)(c.tiles_x * c.px_per_tile), pitch);
    const double Wy = __dmul_rn((double)(c.tiles_y * c.px_per_tile), pitch);
    const double xmax = __dmul_rn((double)c.n_mod_x, Wx);
    const double ymax = __dmul_rn((double)c.n_mod_y, Wy);
    const double zmax = __dmul_rn((double)c.n_tpc, D);
    L.ok = (x >= 0.0 && x < xmax && y >= 0.0 && y < ymax && z >= 0.0 && z <= zmax);
    int mx = (int)floor(__ddiv_rn(x, Wx));
    int my = (int)floor(__ddiv_rn(y, Wy));
    mx = min(max(mx, 0), c.n_mod_x - 1);
    my = min(max(my, 0), c.n_mod_y - 1);
    L.tpc = (c.n_tpc == 2 && z >= D) ? 1 : 0;
    L.mx = mx;
    L.my = my;
    L.anode = (my * c.n_mod_x + mx) * c.n_tpc + L.tpc;
    L.ox = __dmul_rn((double)mx, Wx);
    L.oy = __dmul_rn((double)my, Wy);
    L.za = L.tpc == 0 ? 0.0 : __dmul_rn(2.0, D);
    return L;
}

__global__ void __launch_bounds__(256) k_quench_drift(sim_config c, sim_segments s, sim_drifted o, EventInfo ev)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const float x0 = __ldg(s.x0 + i), y0 = __ldg(s.y0 + i), z0 = __ldg(s.z0 + i);
    const float t0 = __ldg(s.t0 + i), x1 = __ldg(s.x1 + i), y1 = __ldg(s.y1 + i);
    const float z1 = __ldg(s.z1 + i), t1 = __ldg(s.t1 + i), dE = __ldg(s.dE + i);

    // ---- decisions (FP64, fixed operation order) ----
    const double ddx = __dsub_rn((double)x1, (double)x0);
    const double ddy = __dsub_rn((double)y1, (double)y0);
    const double ddz = __dsub_rn((double)z1, (double)z0);
    const double dx = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)),
                                           __dmul_rn(ddz, ddz)));
    const double xm = __dmul_rn(0.5, __dadd_rn((double)x0, (double)x1));
    const double ym = __dmul_rn(0.5, __dadd_rn((double)y0, (double)y1));
    const double zm = __dmul_rn(0.5, __dadd_rn((double)z0, (double)z1));
    const Loc L = locate(c, xm, ym, zm);
    Anchor a;
    if (!L.ok || dx < 1e-6) {
        o.Qa[i] = 0.f;
        o.t_drift[i] = 0.f;
        o.sigma_T[i] = 0.f;
        o.sigma_L[i] = 0.f;
        o.anode[i] = -1;
        o.n_samples[i] = 0;
        a = Anchor{0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        reinterpret_cast<Anchor *>(o.anchors)[i] = a;
        return;
    }
    double Nd = ceil(__ddiv_rn(dx, (double)c.sample_step_cm));
    if (Nd < 1.0) Nd = 1.0;
    const int N = (int)Nd;

    // ---- step 1: recombination, Q_R = R * dE / W_ion (FP32) ----
    const float dedx = dE / (float)dx;
    const float eps = c.efield_kV_cm * c.lar_density_g_cm3;
    float R;
    if (c.recomb_model == 1) {
        const float xi = c.box_beta / eps * dedx;
        R = logf(c.box_alpha + xi) / xi;
    } else {
        R = c.birks_Ab / (1.0f + c.birks_kb / eps * dedx);
    }
    const float QR = R * (dE / c.w_ion_MeV);

    // ---- step 2: drift time, lifetime, diffusion at the midpoint ----
    const float td = (float)fabs(zm - L.za) / c.vdrift_cm_us;
    const float Qa = QR * expf(-td / c.lifetime_us);
    // widths: at the midpoint, or (per-point drift) at the farther end, which bounds every point's
    float tsig = td;
    if (c.per_point_drift) {
        const float t0d = (float)fabs((double)z0 - L.za) / c.vdrift_cm_us;
        const float t1d = (float)fabs((double)z1 - L.za) / c.vdrift_cm_us;
        tsig = fmaxf(t0d, t1d);
    }
    const float sT = sqrtf(2.0f * (c.diff_tran_cm2_s * 1e-6f) * tsig);
    const float sL = sqrtf(2.0f * (c.diff_long_cm2_s * 1e-6f) * tsig);
    o.Qa[i] = Qa;
    o.t_drift[i] = td;
    o.sigma_T[i] = sT;
    o.sigma_L[i] = sL;
    // in a batch, event slot e owns virtual anodes e * n_anodes ..
    const int slot = slot_of_segment(ev, i);
    o.anode[i] = slot * (c.n_mod_x * c.n_mod_y * c.n_tpc) + L.anode;
    o.n_samples[i] = N;

    // ---- anchor: FP64 start point, FP32 small offsets ----
    const double pitch = (double)c.pitch_cm;
    const double X0 = ((double)x0 - L.ox) / pitch;
    const double Y0 = ((double)y0 - L.oy) / pitch;
    const int ixr = (int)floor((xm - L.ox) / pitch);
    const int iyr = (int)floor((ym - L.oy) / pitch);
    const double sgn = L.tpc == 0 ? 1.0 : -1.0;
    const double d0 = sgn * ((double)z0 - L.za);
    const double dd = sgn * ddz;
    const double tick = (double)c.tick_us;
    const double vt = (double)c.vdrift_cm_us * tick;
    const double a0 = ((double)t0 - (double)c.t_window0_us) / tick + d0 / vt;
    const double A0 = floor(a0);
    a.ix_ref = ixr;
    a.iy_ref = iyr;
    a.A0 = (int32_t)A0;
    a.N = N;
    a.fx0 = (float)(X0 - ixr);
    a.fy0 = (float)(Y0 - iyr);
    a.dX = (float)(ddx / pitch);
    a.dY = (float)(ddy / pitch);
    a.fa0 = (float)(a0 - A0);
    a.da = (float)(((double)t1 - (double)t0) / tick + dd / vt);
    a.q = Qa / ((float)N * (float)c.mc_per_sample);
    // sTp sizes the pixel map (the farther end's width under per-point drift, whose points
    // compute their own widths); under per-point drift sLc keeps only the drift direction
    a.sTp = sT / c.pitch_cm;
    a.sLc = c.per_point_drift ? (float)sgn : (float)sgn * sL;
    a.d0 = (float)d0;
    a.dd = (float)dd;
    a.kz = (float)(1.0 / vt);
    reinterpret_cast<Anchor *>(o.anchors)[i] = a;
}

cudaError_t launch_quench_drift(const sim_config &c, const sim_segments &s, const sim_drifted &o,
                                cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (s.n + threads - 1) / threads;
    k_quench_drift<<<(unsigned)blocks, threads, 0, st>>>(c, s, o, events_of(s));
    return cudaGetLastError();
}

}  // namespace larsim
