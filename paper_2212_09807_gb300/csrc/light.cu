// light.cu -- the light path (arXiv:2212.09807 Sec. 4) on the segments of
// the charge path: photon yield and photoelectrons per photosensor (4.1),
// photocurrent from the arrival-time table (4.2), truncated scintillation
// convolution and counting fluctuations (4.2), electronics response with
// noise, sampling and ADC (4.3).
//
//  * k_light_yield: one thread per segment; the voxel and tick decisions use
//    explicitly rounded FP32 operations (no contraction) in a fixed order.
//  * k_light_photocurrent: one CTA per block of 256 consecutive segments.
//    The block's segments of one anode whose table rows fall in a window of
//    W ticks add their terms npe * tdist into a shared window of 64-bit
//    fixed-point accumulators (2^-16 p.e., one rounding per term, integer
//    additions: exact and order-free), which is then added to the detector
//    rows with 64-bit integer atomics.  Segments of one interaction are
//    contiguous and share their time, so a block usually needs one window.
//  * k_light_scint: one CTA per photosensor.  The truncated convolution with
//    the two-exponential kernel equals, per component c (amplitude a_c,
//    decay r_c = e^(-tick / tau_c) per tick), y[t] = r_c y[t-1] + a_c x[t] -
//    a_c r_c^(N+1) x[t-N-1]; each thread runs the recurrence over 16
//    consecutive ticks from zero, a CTA scan (FP64) of the threads' end
//    values gives every thread its carry, and the thread reruns its ticks.
//    O(T) work instead of the direct form's O(T N).
//  * k_light_fluct: one thread per tick; the Poisson inverse transform is
//    evaluated in FP64 with explicitly rounded operations.
//  * k_light_noise: one CTA per (photosensor, noise block): random phases,
//    radix-2 inverse FFT of the one-sided spectrum in shared memory.
//  * k_light_response: one CTA per (photosensor, 1024 ticks): the input span
//    and the response in shared memory, four outputs per thread.
//  * k_light_digitize: one thread per sample.
//  * k_light_truth: one thread per (segment, photosensor): the mean arrival
//    time of the segment's photoelectrons (Sec. 4.4 default truth, with the
//    photoelectrons of k_light_yield).
#include "sim_internal.cuh"

namespace larsim {

namespace {

constexpr double kPeFix = 65536.0;               // fixed point of the photocurrent (p.e.)
constexpr int kSegBlock = 256;
constexpr int kScintChunk = 4096;                // ticks per CTA pass (256 threads x 16)
constexpr int kTileT = 1024;                     // ticks per response CTA
constexpr int kMaxResp = 2048;

struct LightGeo {
    int n_mod_x, n_tpc, n_anodes;
    float pitch, Wx, Wy, D;
};

LightGeo light_geo(const sim_config &c)
{
    LightGeo g;
    g.n_mod_x = c.n_mod_x;
    g.n_tpc = c.n_tpc;
    g.n_anodes = c.n_mod_x * c.n_mod_y * c.n_tpc;
    g.pitch = c.pitch_cm;
    g.Wx = (float)(c.tiles_x * c.px_per_tile) * c.pitch_cm;      // one FP32 rounding of the product
    g.Wy = (float)(c.tiles_y * c.px_per_tile) * c.pitch_cm;
    g.D = c.drift_len_cm;
    return g;
}

__global__ void __launch_bounds__(256) k_light_yield(sim_light_config lc, LightGeo g, float lifetime,
                                                     sim_segments s, sim_drifted d, float *npe, int32_t *tick,
                                                     int32_t *vox)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int nd = lc.n_det;
    const int anode = d.anode[i];
    if (anode < 0) {
        for (int k = 0; k < nd; ++k) npe[i * nd + k] = 0.f;
        tick[i] = 0;
        vox[i] = -1;
        return;
    }
    const int a = anode % g.n_anodes;
    const int tpc = a % g.n_tpc, m = a / g.n_tpc;
    const int mx = m % g.n_mod_x, my = m / g.n_mod_x;
    const float x0 = __ldg(s.x0 + i), y0 = __ldg(s.y0 + i), z0 = __ldg(s.z0 + i), t0 = __ldg(s.t0 + i);
    const float x1 = __ldg(s.x1 + i), y1 = __ldg(s.y1 + i), z1 = __ldg(s.z1 + i), t1 = __ldg(s.t1 + i);
    const float dE = __ldg(s.dE + i);
    const float xm = __fmul_rn(0.5f, __fadd_rn(x0, x1)), ym = __fmul_rn(0.5f, __fadd_rn(y0, y1));
    const float zm = __fmul_rn(0.5f, __fadd_rn(z0, z1)), tm = __fmul_rn(0.5f, __fadd_rn(t0, t1));
    const float xl = __fsub_rn(xm, __fmul_rn((float)mx, g.Wx));
    const float yl = __fsub_rn(ym, __fmul_rn((float)my, g.Wy));
    const float za = tpc == 0 ? 0.0f : __fmul_rn(2.0f, g.D);
    const float zl = fabsf(__fsub_rn(zm, za));
    int ix = (int)floorf(__fdiv_rn(xl, lc.vox_cm));
    int iy = (int)floorf(__fdiv_rn(yl, lc.vox_cm));
    int iz = (int)floorf(__fdiv_rn(zl, lc.vox_cm));
    ix = min(max(ix, 0), lc.nvx - 1);
    iy = min(max(iy, 0), lc.nvy - 1);
    iz = min(max(iz, 0), lc.nvz - 1);
    const int v = (ix * lc.nvy + iy) * lc.nvz + iz;
    vox[i] = v;
    tick[i] = (int32_t)floorf(__fdiv_rn(__fsub_rn(tm, lc.t_start_us), lc.tick_us));
    const float QR = d.Qa[i] * expf(d.t_drift[i] / lifetime);
    const float ngam = fmaxf(dE / lc.w_ph_MeV - QR, 0.f);
    for (int k = 0; k < nd; ++k) npe[i * nd + k] = __ldg(lc.eff + k) * __ldg(lc.vis + (size_t)v * nd + k) * ngam;
}

struct PcSmem {
    int tick[kSegBlock], vox[kSegBlock], anode[kSegBlock];
    unsigned char done[kSegBlock];
    int red_a, red_t;
};

__global__ void __launch_bounds__(256) k_light_photocurrent(sim_light_config lc, int64_t n, const int32_t *anode_of,
                                                            const float *npe, const int32_t *tick_of,
                                                            const int32_t *vox_of, unsigned long long *pe, int W)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PcSmem &sm = *reinterpret_cast<PcSmem *>(smem_raw);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(smem_raw + ((sizeof(PcSmem) + 15) & ~15ull));
    const int tid = threadIdx.x;
    const int nd = lc.n_det, nt = lc.nt, T = lc.n_ticks;
    for (int64_t b0 = (int64_t)blockIdx.x * kSegBlock; b0 < n; b0 += (int64_t)gridDim.x * kSegBlock) {
        const int nb = (int)min((int64_t)kSegBlock, n - b0);
        if (tid < kSegBlock) {
            const int64_t j = b0 + tid;
            const bool ok = tid < nb && vox_of[j] >= 0;
            sm.tick[tid] = ok ? tick_of[j] : 0;
            sm.vox[tid] = ok ? vox_of[j] : -1;
            sm.anode[tid] = ok ? anode_of[j] : -1;
            // a segment whose rows miss the window entirely is done
            sm.done[tid] = !ok || tick_of[j] + nt <= 0 || tick_of[j] >= T;
        }
        __syncthreads();
        for (;;) {
            // next window: smallest anode left, then its smallest tick
            if (tid == 0) {
                sm.red_a = INT_MAX;
                sm.red_t = INT_MAX;
            }
            __syncthreads();
            if (!sm.done[tid]) atomicMin(&sm.red_a, sm.anode[tid]);
            __syncthreads();
            const int an = sm.red_a;
            if (an == INT_MAX) break;
            if (!sm.done[tid] && sm.anode[tid] == an) atomicMin(&sm.red_t, sm.tick[tid]);
            for (int i = tid; i < nd * W; i += blockDim.x) acc[i] = 0ull;
            __syncthreads();
            const int s_lo = sm.red_t;
            // thread -> (k, u) pairs: the block's segments of this window, in index order
            for (int j = 0; j < nb; ++j) {
                if (sm.done[j] || sm.anode[j] != an || sm.tick[j] > s_lo + W - nt) continue;   // CTA-uniform
                const int v = sm.vox[j], off = sm.tick[j] - s_lo;
                const float *f = lc.tdist + (size_t)v * nd * nt;
                const float *q = npe + (b0 + j) * nd;
                for (int p = tid; p < nd * nt; p += blockDim.x) {
                    const int k = p / nt, u = p - k * nt;
                    const float term = __fmul_rn(__fmul_rn(__ldg(q + k), __ldg(f + p)), 65536.0f);
                    if (term != 0.f) {
                        long long fx;
                        if (fabsf(term) < 4194304.0f) {
                            // round to nearest even by adding 1.5 * 2^23 (FP32 add, no conversion unit)
                            fx = (long long)(__float_as_int(__fadd_rn(term, 12582912.0f)) - 0x4B400000);
                        } else {
                            fx = __float2ll_rn(term);                  // terms of 64 p.e. and more: rare
                        }
                        atomicAdd(&acc[k * W + off + u], (unsigned long long)fx);
                    }
                }
            }
            __syncthreads();
            if (tid < nb && !sm.done[tid] && sm.anode[tid] == an && sm.tick[tid] <= s_lo + W - nt) sm.done[tid] = 1;
            // window -> detector rows
            for (int i = tid; i < nd * W; i += blockDim.x) {
                const unsigned long long v = acc[i];
                if (v == 0ull) continue;
                const int k = i / W, t = s_lo + (i - k * W);
                if (t < 0 || t >= T) continue;
                atomicAdd(pe + ((size_t)an * nd + k) * T + t, v);
            }
            __syncthreads();
        }
    }
}

struct ScintPar {
    float a[2], r[2], b[2];      // amplitude, per-tick decay, tail coefficient a r^(N+1)
    double r16[2];               // r^16
    int n_trunc;
};

__global__ void __launch_bounds__(256) k_light_scint(sim_light_config lc, ScintPar P, int n_det_total,
                                                     const long long *pe, float *S)
{
    __shared__ double part[2][8];
    __shared__ double nxt[2];
    __shared__ double pw[2][257];                           // r16^i, i = 0 .. 256
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = lc.n_ticks, N = P.n_trunc;
    for (int i = tid; i <= 256; i += blockDim.x) {
        pw[0][i] = pow(P.r16[0], (double)i);
        pw[1][i] = pow(P.r16[1], (double)i);
    }
    __syncthreads();
    for (int det = blockIdx.x; det < n_det_total; det += gridDim.x) {
        const long long *x = pe + (size_t)det * T;
        float *y = S + (size_t)det * T;
        double carry[2] = {0.0, 0.0};
        for (int c0 = 0; c0 < T; c0 += kScintChunk) {
            const int t0 = c0 + tid * 16;
            float z[2][16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int t = t0 + i, to = t - N - 1;
                const float xv = t < T ? (float)((double)x[t] * (1.0 / kPeFix)) : 0.f;
                const float xo = (t < T && to >= 0) ? (float)((double)x[to] * (1.0 / kPeFix)) : 0.f;
#pragma unroll
                for (int c = 0; c < 2; ++c) z[c][i] = P.a[c] * xv - P.b[c] * xo;
            }
            // end value of each thread's 16 ticks from a zero start, then its carry by a scan
            double v[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float e = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) e = P.r[c] * e + z[c][i];
                double w = (double)e, m = P.r16[c];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {          // in-warp inclusive: sum_j r16^(i-j) e_j
                    const double u = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w = m * u + w;
                    m = m * m;
                }
                v[c] = w;
                if (lane == 31) part[c][warp] = w;
            }
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {                // across the 8 warps: multiplier r16^32
                    double w = lane < 8 ? part[c][lane] : 0.0;
                    double m = pw[c][32];
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        const double u = __shfl_up_sync(0xffffffffu, w, o);
                        if (lane >= o) w = m * u + w;
                        m = m * m;
                    }
                    if (lane < 8) part[c][lane] = w;
                }
            }
            __syncthreads();
            float yc[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                double prev = __shfl_up_sync(0xffffffffu, v[c], 1);
                if (lane == 0) prev = 0.0;
                const double before = warp > 0 ? part[c][warp - 1] : 0.0;
                // state before this thread's first tick
                const double cin = prev + pw[c][lane] * before + pw[c][tid] * carry[c];
                yc[c] = (float)cin;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float out = 0.f;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    yc[c] = P.r[c] * yc[c] + z[c][i];
                    out += yc[c];
                }
                if (t0 + i < T) y[t0 + i] = out;
            }
            if (tid == 255) {
                nxt[0] = (double)yc[0];
                nxt[1] = (double)yc[1];
            }
            __syncthreads();
            carry[0] = nxt[0];
            carry[1] = nxt[1];
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_light_fluct(sim_light_config lc, uint64_t key, int n_det_total,
                                                     const float *S, float *out)
{
    const int64_t total = (int64_t)n_det_total * lc.n_ticks;
    const double tick = (double)lc.tick_us, lmax = (double)lc.poisson_max_mean;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int det = (int)(i / lc.n_ticks);
        const int t = (int)(i - (int64_t)det * lc.n_ticks);
        const double lam = __dmul_rn((double)S[i], tick);
        float n;
        if (lam <= lmax) {
            const u32x4 x = philox4x32_10(u32x4{(uint32_t)det, (uint32_t)t, 5u, 0u}, (uint32_t)key,
                                          (uint32_t)(key >> 32));
            // k = 0 iff u <= e^-lambda, i.e. lambda <= -ln u: decided in FP32 when lambda is clear of
            // -ln u by 1e-6 relative plus 3e-7 absolute (the FP32 uniform is within 2^-23 relative of
            // the FP64 one, and the FP32 logarithm within a few ulp), else in FP64 below
            const float nlu = -logf(u01f(x.x));
            if ((float)lam < nlu * 0.999999f - 3e-7f) {
                n = 0.f;
            } else {
                const double u = __dadd_rn(__dmul_rn((double)x.x, 0x1p-32), 0x1p-33);
                double pk = exp(-lam), F = pk;
                int k = 0;
                while (u > F && k < 1000) {
                    ++k;
                    pk = __dmul_rn(pk, __ddiv_rn(lam, (double)k));
                    F = __dadd_rn(F, pk);
                }
                n = (float)k;
            }
        } else {
            const float2 z = normals2(key, (uint32_t)det, (uint32_t)t, 6u);
            const float l = (float)lam;
            n = fmaxf(l + sqrtf(l) * z.x, 0.f);
        }
        out[i] = n;
    }
}

// Noise of one (photosensor, block): inverse FFT of X_k = A_k e^(i phi_k),
// k <= N/2 (zero above), real part.
__global__ void __launch_bounds__(256) k_light_noise(sim_light_config lc, uint64_t key, int n_det_total, int log2n,
                                                     float *V)
{
    extern __shared__ __align__(16) float2 buf[];
    const int N = lc.noise_block, T = lc.n_ticks;
    const int nblk = (T + N - 1) / N;
    const int tid = threadIdx.x;
    for (int64_t w = blockIdx.x; w < (int64_t)n_det_total * nblk; w += gridDim.x) {
        const int det = (int)(w / nblk), b = (int)(w - (int64_t)det * nblk);
        // spectrum in bit-reversed order
        for (int k = tid; k < N; k += blockDim.x) {
            float2 X = make_float2(0.f, 0.f);
            if (k <= N / 2) {
                const float A = __ldg(lc.noise_amp + k);
                if (A != 0.f) {
                    const u32x4 x = philox4x32_10(u32x4{(uint32_t)det, (uint32_t)b, 7u, (uint32_t)k}, (uint32_t)key,
                                                  (uint32_t)(key >> 32));
                    float sn, cs;
                    sincospif(2.0f * u01f(x.x), &sn, &cs);
                    X = make_float2(A * cs, A * sn);
                }
            }
            const int r = (int)(__brev((unsigned)k) >> (32 - log2n));
            buf[r] = X;
        }
        __syncthreads();
        // radix-2 butterflies, exponent +2 pi i (inverse transform, no scaling)
        for (int len = 2; len <= N; len <<= 1) {
            const int half = len >> 1;
            for (int p = tid; p < N / 2; p += blockDim.x) {
                const int grp = p / half, j = p - grp * half;
                const int i0 = grp * len + j, i1 = i0 + half;
                float sn, cs;
                sincospif(2.0f * (float)j / (float)len, &sn, &cs);
                const float2 a = buf[i0], bb = buf[i1];
                const float2 tw = make_float2(bb.x * cs - bb.y * sn, bb.x * sn + bb.y * cs);
                buf[i0] = make_float2(a.x + tw.x, a.y + tw.y);
                buf[i1] = make_float2(a.x - tw.x, a.y - tw.y);
            }
            __syncthreads();
        }
        for (int tau = tid; tau < N; tau += blockDim.x) {
            const int t = b * N + tau;
            if (t < T) V[(size_t)det * T + t] = buf[tau].x;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_light_response(sim_light_config lc, int n_det_total, const float *x,
                                                        float *V)
{
    __shared__ float xs[kTileT + kMaxResp];
    __shared__ float rs[kMaxResp];
    const int T = lc.n_ticks, R = lc.n_resp, tid = threadIdx.x;
    const int ntile = (T + kTileT - 1) / kTileT;
    for (int i = tid; i < R; i += blockDim.x) rs[i] = __ldg(lc.resp + i);
    for (int64_t w = blockIdx.x; w < (int64_t)n_det_total * ntile; w += gridDim.x) {
        const int det = (int)(w / ntile), tl = (int)(w - (int64_t)det * ntile);
        const int t0 = tl * kTileT;
        const float *xr = x + (size_t)det * T;
        __syncthreads();
        // xs[i] = x[t0 - R + 1 + i], zero outside [0, T)
        for (int i = tid; i < kTileT + R - 1; i += blockDim.x) {
            const int t = t0 - R + 1 + i;
            xs[i] = (t >= 0 && t < T) ? xr[t] : 0.f;
        }
        __syncthreads();
        const float g = __ldg(lc.gain + det % lc.n_det);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int u = 0; u < R; ++u) {
            const float r = rs[u];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += xs[tid + 256 * q + R - 1 - u] * r;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + tid + 256 * q;
            if (t < T) V[(size_t)det * T + t] += g * acc[q];
        }
    }
}

__global__ void __launch_bounds__(256) k_light_digitize(sim_light_config lc, int n_det_total, int64_t n_samples,
                                                        double ratio, const float *V, uint16_t *wave)
{
    const int64_t total = (int64_t)n_det_total * n_samples;
    const int T = lc.n_ticks;
    const double top = (double)((1 << lc.adc_bits) - 1), ped = (double)lc.pedestal_adc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int det = (int)(i / n_samples);
        const int64_t m = i - (int64_t)det * n_samples;
        const double p = __dmul_rn((double)m, ratio);
        const double fl = floor(p);
        const int ti = (int)fl;
        const double fr = __dsub_rn(p, fl);
        const float *vr = V + (size_t)det * T;
        const double v = ti + 1 < T ? __dadd_rn(__dmul_rn(__dsub_rn(1.0, fr), (double)vr[ti]), __dmul_rn(fr, (double)vr[ti + 1]))
                                    : (double)vr[ti];
        double cd = floor(__dadd_rn(__dadd_rn(v, ped), 0.5));
        cd = fmin(fmax(cd, 0.0), top);
        wave[i] = (uint16_t)cd;
    }
}

// Sec. 4.4 default truth: mean arrival time of each segment's photoelectrons
// at each photosensor, t_start + (tick + sum_u (u + 1/2) f[u]) tick.
__global__ void __launch_bounds__(256) k_light_truth(sim_light_config lc, int64_t n, const int32_t *tick,
                                                     const int32_t *vox, float *t_arr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nd = lc.n_det;
    if (i >= n * nd) return;
    const int64_t j = i / nd;
    const int k = (int)(i - j * nd);
    const int v = vox[j];
    if (v < 0) {
        t_arr[i] = 0.f;
        return;
    }
    const float *f = lc.tdist + ((size_t)v * nd + k) * lc.nt;
    double m = 0.0;
    for (int u = 0; u < lc.nt; ++u) m += ((double)u + 0.5) * (double)__ldg(f + u);
    t_arr[i] = (float)((double)lc.t_start_us + ((double)tick[j] + m) * (double)lc.tick_us);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

int light_n_det_total(const sim_config &c, const sim_light_config &lc)
{
    return c.n_mod_x * c.n_mod_y * c.n_tpc * lc.n_det;
}

int64_t light_n_samples(const sim_light_config &lc, double *ratio)
{
    const double r = (double)lc.sample_us / (double)lc.tick_us;
    if (ratio) *ratio = r;
    return (int64_t)floor((double)(lc.n_ticks - 1) / r) + 1;
}

int light_n_trunc(const sim_light_config &lc)
{
    return (int)floor((double)lc.trunc_taus * (double)lc.tau_slow_us / (double)lc.tick_us + 0.5);
}

cudaError_t launch_light_yield(const sim_config &c, const sim_light_config &lc, const sim_segments &s,
                               const sim_drifted &d, float *npe, int32_t *tick, int32_t *vox, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    k_light_yield<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(lc, light_geo(c), c.lifetime_us, s, d, npe, tick,
                                                                   vox);
    return cudaGetLastError();
}

cudaError_t launch_light_truth(const sim_light_config &lc, int64_t n, const int32_t *tick, const int32_t *vox,
                               float *t_arr, cudaStream_t st)
{
    const int64_t tot = n * lc.n_det;
    if (tot == 0) return cudaSuccess;
    k_light_truth<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(lc, n, tick, vox, t_arr);
    return cudaGetLastError();
}

size_t light_photocurrent_smem(const sim_light_config &lc, int *W)
{
    // window: 36 KB of accumulators (several CTAs per SM), at least 2 nt
    int w = (36 * 1024) / (8 * lc.n_det);
    w = (w / 64) * 64;
    if (w < 2 * lc.nt) w = ((2 * lc.nt + 63) / 64) * 64;
    if (W) *W = w;
    return ((sizeof(PcSmem) + 15) & ~(size_t)15) + (size_t)8 * lc.n_det * w;
}

cudaError_t launch_light_photocurrent(const sim_config &c, const sim_light_config &lc, const sim_segments &s,
                                      const sim_drifted &d, const float *npe, const int32_t *tick,
                                      const int32_t *vox, int64_t *pe, cudaStream_t st)
{
    const size_t rows = (size_t)light_n_det_total(c, lc) * lc.n_ticks;
    cudaError_t e = cudaMemsetAsync(pe, 0, 8 * rows, st);
    if (e != cudaSuccess || s.n == 0) return e;
    int W = 0;
    const size_t smem = light_photocurrent_smem(lc, &W);
    e = cudaFuncSetAttribute(k_light_photocurrent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (s.n + kSegBlock - 1) / kSegBlock;
    const int grid = (int)(blocks < (int64_t)sm_count() * 4 ? blocks : (int64_t)sm_count() * 4);
    k_light_photocurrent<<<grid, 256, smem, st>>>(lc, s.n, d.anode, npe, tick, vox,
                                                 reinterpret_cast<unsigned long long *>(pe), W);
    return cudaGetLastError();
}

cudaError_t launch_light_scint(const sim_config &c, const sim_light_config &lc, const int64_t *pe, float *S,
                               cudaStream_t st)
{
    ScintPar P;
    const double tick = (double)lc.tick_us;
    const int N = light_n_trunc(lc);
    const double tau[2] = {(double)lc.tau_fast_us, (double)lc.tau_slow_us};
    const double amp[2] = {(double)lc.fast_frac / tau[0], (1.0 - (double)lc.fast_frac) / tau[1]};
    for (int k = 0; k < 2; ++k) {
        const double r = exp(-tick / tau[k]);
        P.a[k] = (float)amp[k];
        P.r[k] = (float)r;
        P.b[k] = (float)(amp[k] * pow(r, (double)(N + 1)));
        P.r16[k] = pow((double)P.r[k], 16.0);
    }
    P.n_trunc = N;
    const int ndt = light_n_det_total(c, lc);
    const int grid = ndt < sm_count() * 8 ? ndt : sm_count() * 8;
    k_light_scint<<<grid, 256, 0, st>>>(lc, P, ndt, reinterpret_cast<const long long *>(pe), S);
    return cudaGetLastError();
}

cudaError_t launch_light_fluct(const sim_config &c, const sim_light_config &lc, uint64_t event_id, const float *S,
                               float *out, cudaStream_t st)
{
    const int ndt = light_n_det_total(c, lc);
    const int64_t total = (int64_t)ndt * lc.n_ticks;
    const int64_t want = (total + 255) / 256;
    const int grid = (int)(want < (int64_t)sm_count() * 16 ? want : (int64_t)sm_count() * 16);
    k_light_fluct<<<grid, 256, 0, st>>>(lc, c.seed ^ event_id, ndt, S, out);
    return cudaGetLastError();
}

cudaError_t launch_light_electronics(const sim_config &c, const sim_light_config &lc, uint64_t event_id,
                                     const float *pe_obs, float *V, uint16_t *wave, cudaStream_t st)
{
    const int ndt = light_n_det_total(c, lc);
    const int N = lc.noise_block;
    int log2n = 0;
    while ((1 << log2n) < N) ++log2n;
    const int sms = sm_count();
    const int64_t nblk = (int64_t)ndt * ((lc.n_ticks + N - 1) / N);
    const size_t smem = sizeof(float2) * (size_t)N;
    cudaError_t e = cudaFuncSetAttribute(k_light_noise, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_light_noise<<<(int)(nblk < (int64_t)sms * 8 ? nblk : (int64_t)sms * 8), 256, smem, st>>>(lc, c.seed ^ event_id,
                                                                                             ndt, log2n, V);
    const int64_t ntile = (int64_t)ndt * ((lc.n_ticks + kTileT - 1) / kTileT);
    k_light_response<<<(int)(ntile < (int64_t)sms * 8 ? ntile : (int64_t)sms * 8), 256, 0, st>>>(lc, ndt, pe_obs, V);
    double ratio = 0.0;
    const int64_t ns = light_n_samples(lc, &ratio);
    const int64_t tot = (int64_t)ndt * ns;
    const int64_t want = (tot + 255) / 256;
    k_light_digitize<<<(int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16), 256, 0, st>>>(lc, ndt, ns, ratio,
                                                                                               V, wave);
    return cudaGetLastError();
}

}  // namespace larsim
