// hit_points.cu -- hits -> 3-D points and dQ/dx along a known straight track
// (arXiv:2212.09807 Sec. 6: the reconstruction takes one 3-D point per hit,
// x-y at the pixel centre and z from the hit's tick by the inverse of
// Eq. (drift); dQ/dx is the hits' charge per unit length of a track, in
// pieces of fixed length).
//
// Both kernels are elementwise over the hits (HBM-bound, a few bytes per
// hit).  Their arithmetic is FP64 with explicitly rounded operations (no
// contraction into FMA), in the order of the formula as written, so that
// the point coordinates are the correctly rounded FP32 values of the exact
// FP64 expressions and the piece a point falls in is decided exactly as an
// IEEE FP64 evaluation of the same expressions decides it.  Piece charges
// are summed in fixed point (2^-16 e-, 64-bit integer atomics): exact and
// independent of the order of the additions.
#include "sim_internal.cuh"

namespace larsim {

namespace {

constexpr double kFix = 65536.0;

struct PointArgs {
    const int32_t *pixel, *t_cross;
    const int64_t *n_hits;
    int64_t cap;
    const float *t_event;
    int64_t det_px;
    int32_t npx_x, npx_y, n_tpc, n_mod_x;
    double pitch, drift, t_w0, tick, vdrift;
    float *x, *y, *z;
};

__global__ void k_hit_points(PointArgs a)
{
    const int64_t n = min(*a.n_hits, a.cap);
    const int npx = a.npx_x * a.npx_y;
    const double Wx = __dmul_rn((double)a.npx_x, a.pitch), Wy = __dmul_rn((double)a.npx_y, a.pitch);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t vp = a.pixel[i];
        const int slot = (int)(vp / a.det_px);
        const int32_t p = (int32_t)(vp - (int64_t)slot * a.det_px);
        const int32_t g = p / npx, rem = p - g * npx;
        const int32_t iy = rem / a.npx_x, ix = rem - iy * a.npx_x;
        const int32_t m = g / a.n_tpc, tpc = g - m * a.n_tpc;
        const int32_t mx = m % a.n_mod_x, my = m / a.n_mod_x;
        const double xc = __dadd_rn(__dmul_rn((double)mx, Wx), __dmul_rn((double)ix + 0.5, a.pitch));
        const double yc = __dadd_rn(__dmul_rn((double)my, Wy), __dmul_rn((double)iy + 0.5, a.pitch));
        const double za = tpc == 0 ? 0.0 : 2.0 * a.drift;
        const double t = __dadd_rn(a.t_w0, __dmul_rn((double)a.t_cross[i], a.tick));
        const double te = a.t_event ? (double)a.t_event[slot] : 0.0;
        const double dz = __dmul_rn(a.vdrift, __dsub_rn(t, te));
        a.x[i] = (float)xc;
        a.y[i] = (float)yc;
        a.z[i] = (float)(tpc == 0 ? __dadd_rn(za, dz) : __dsub_rn(za, dz));
    }
}

struct DqdxArgs {
    const float *x, *y, *z, *q;
    const int64_t *n;
    int64_t cap;
    double o[3], u[3];
    double dx, r_max;
    int32_t n_bins;
    unsigned long long *acc;                   // fixed-point sums, in place of dq
    int32_t *count;
};

__global__ void k_track_dqdx(DqdxArgs a)
{
    const int64_t n = min(*a.n, a.cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double px = __dsub_rn((double)a.x[i], a.o[0]);
        const double py = __dsub_rn((double)a.y[i], a.o[1]);
        const double pz = __dsub_rn((double)a.z[i], a.o[2]);
        const double s = __dadd_rn(__dadd_rn(__dmul_rn(px, a.u[0]), __dmul_rn(py, a.u[1])), __dmul_rn(pz, a.u[2]));
        const double ex = __dsub_rn(px, __dmul_rn(s, a.u[0]));
        const double ey = __dsub_rn(py, __dmul_rn(s, a.u[1]));
        const double ez = __dsub_rn(pz, __dmul_rn(s, a.u[2]));
        const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
        const double fb = floor(__ddiv_rn(s, a.dx));
        if (d > a.r_max || s < 0.0 || fb >= (double)a.n_bins) continue;
        const int b = (int)fb;
        const long long qf = __double2ll_rn(__dmul_rn((double)a.q[i], kFix));
        atomicAdd(a.acc + b, (unsigned long long)qf);
        atomicAdd(a.count + b, 1);
    }
}

__global__ void k_dqdx_finish(unsigned long long *acc, int32_t n_bins)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins) return;
    const long long v = (long long)acc[b];
    reinterpret_cast<double *>(acc)[b] = (double)v / kFix;
}

int grid_for(int64_t n, int threads)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_hit_points(const sim_config &c, const sim_hits &h, const float *t_event, float *x, float *y,
                              float *z, cudaStream_t st)
{
    if (h.capacity == 0) return cudaSuccess;
    PointArgs a;
    a.pixel = h.pixel;
    a.t_cross = h.t_cross;
    a.n_hits = h.n_out;
    a.cap = h.capacity;
    a.t_event = t_event;
    const Geo g = geo_of(c);
    a.det_px = detector_pixels(g);
    a.npx_x = g.npx_x;
    a.npx_y = g.npx_y;
    a.n_tpc = c.n_tpc;
    a.n_mod_x = c.n_mod_x;
    a.pitch = (double)c.pitch_cm;
    a.drift = (double)c.drift_len_cm;
    a.t_w0 = (double)c.t_window0_us;
    a.tick = (double)c.tick_us;
    a.vdrift = (double)c.vdrift_cm_us;
    a.x = x;
    a.y = y;
    a.z = z;
    k_hit_points<<<grid_for(h.capacity, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_track_dqdx(const float *x, const float *y, const float *z, const float *q, const int64_t *n,
                              int64_t cap, const double origin[3], const double dir[3], double piece, int32_t n_bins,
                              double r_max, double *dq, int32_t *count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(dq, 0, sizeof(double) * (size_t)n_bins, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)n_bins, st);
    if (e != cudaSuccess) return e;
    DqdxArgs a;
    a.x = x;
    a.y = y;
    a.z = z;
    a.q = q;
    a.n = n;
    a.cap = cap;
    for (int i = 0; i < 3; ++i) {
        a.o[i] = origin[i];
        a.u[i] = dir[i];
    }
    a.dx = piece;
    a.r_max = r_max;
    a.n_bins = n_bins;
    a.acc = reinterpret_cast<unsigned long long *>(dq);
    a.count = count;
    if (cap > 0) k_track_dqdx<<<grid_for(cap, 256), 256, 0, st>>>(a);
    k_dqdx_finish<<<(n_bins + 255) / 256, 256, 0, st>>>(a.acc, n_bins);
    return cudaGetLastError();
}

}  // namespace larsim
