// electronics.cu -- step 5 of the charge path (arXiv:2212.09807 Sec. 3.4):
// the LArPix-like front end of every active pixel: the charge-sensitive
// amplifier integrates the pixel's current; while idle the discriminator
// compares the CSA output plus uncorrelated noise with the threshold plus
// discriminator noise; a crossing schedules the ADC hold_ticks later (and at
// least min_adc_interval_ticks after the previous conversion); the ADC
// digitises the CSA output plus uncorrelated noise to adc_bits and the CSA
// resets to a random pedestal; an optional periodic reset clears idle charge.
//
// One warp per pixel walks the ticks 32 at a time: a warp inclusive scan of
// the 32 currents gives the CSA charge of every lane's tick, and a ballot over
// the lanes still idle finds the first crossing, so the sequential state
// machine costs one scan per 32 ticks plus one Philox block per idle tick.
// Hits are staged per pixel, counted, scanned and compacted in pixel order.
#include "sim_internal.cuh"

namespace larsim {

namespace {

constexpr int kWarps = 8;

struct HitRec {
    int32_t t_cross, t_adc, adc;
    float q;
};

__host__ __device__ inline int max_hits_per_pixel(const sim_config &c)
{
    int per = c.hold_ticks + 1;
    if (c.min_adc_interval_ticks > per) per = c.min_adc_interval_ticks;
    if (per < 1) per = 1;
    return c.n_ticks / per + 1;
}

struct ElArgs {
    sim_config c;
    EventInfo ev;
    int64_t det_px;                             // pixels of one detector copy
    const int32_t *active;
    const float *current;
    const int64_t *counts;
    int64_t pix_cap;
    HitRec *stage;
    int32_t *nhit;
    int hmax;
};

template <typename Acc>
__device__ __forceinline__ Acc warp_incl_scan(Acc v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Acc u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Acc: type of the running CSA charge (float, or double for long windows);
// threshold and ADC decisions compare FP32 roundings of the Acc operands.
template <typename Acc>
__global__ void __launch_bounds__(kWarps * 32) k_electronics(ElArgs a)
{
    if ((a.counts[3] & (SIM_STATUS_PAIR_OVERFLOW | SIM_STATUS_PIXEL_OVERFLOW)) != 0) return;
    const int64_t npix = a.counts[1];
    if (npix > a.pix_cap) return;
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    const sim_config &c = a.c;
    const int T = c.n_ticks;
    const float lsb_e = c.gain_e_per_mV * c.adc_lsb_mV;
    const float adc_max = (float)((1 << c.adc_bits) - 1);
    const int per = c.periodic_reset_ticks;

    for (int64_t pi = wg; pi < npix; pi += nw) {
        // virtual pixel -> event slot (Philox key) and detector pixel id (counter)
        const int32_t vpid = a.active[pi];
        const int slot = (int)(vpid / a.det_px);
        const uint32_t pid = (uint32_t)(vpid - slot * a.det_px);
        if (c.disabled_pixels && ((__ldg(c.disabled_pixels + (pid >> 5)) >> (pid & 31)) & 1u)) {
            if (lane == 0) a.nhit[pi] = 0;      // channel disabled: no hits
            continue;
        }
        const uint64_t key = slot_key(a.c.seed, a.ev, slot);
        const float *I = a.current + (size_t)pi * T;
        HitRec *st = a.stage + (size_t)pi * a.hmax;
        Acc qoff = 0;             // CSA charge before this chunk's first tick
        bool idle = true;
        int t_cross = -1, t_adc = -1;
        int last_adc = -(1 << 30);
        int per_done = 0;         // periodic resets at ticks <= per_done are applied
        int nh = 0;
        for (int k0 = 0; k0 < T; k0 += 32) {
            const int k = k0 + lane;
            const float x = (k < T) ? I[k] : 0.f;
            const Acc sc = warp_incl_scan<Acc>((Acc)x, lane);
            const int nl = min(32, T - k0);
            int pos = 0;
            while (pos < nl) {
                if (idle) {
                    int lim = nl;
                    if (per > 0) {
                        int p0 = max(max(k0 + pos, 1), per_done + 1);
                        const int P = ((p0 + per - 1) / per) * per;
                        if (P < k0 + nl) lim = P - k0;
                    }
                    bool cross = false;
                    if (lane >= pos && lane < lim) {
                        const float2 n = normals2(key, pid, (uint32_t)k, 2u);
                        const Acc v = qoff + sc + (Acc)c.sigma_unc_e * (Acc)n.x;
                        const Acc thr = (Acc)c.thr_e + (Acc)c.sigma_disc_e * (Acc)n.y;
                        cross = (float)v >= (float)thr;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, cross);
                    if (m) {
                        const int cl = __ffs(m) - 1;
                        t_cross = k0 + cl;
                        t_adc = max(t_cross + c.hold_ticks, last_adc + c.min_adc_interval_ticks);
                        idle = false;
                        pos = cl;
                    } else if (lim < nl) {
                        const Acc r = (Acc)c.sigma_reset_e * (Acc)normals2(key, pid, (uint32_t)(k0 + lim), 4u).x;
                        const Acc sprev = __shfl_sync(0xffffffffu, sc, max(lim - 1, 0));
                        qoff = r - (lim > 0 ? sprev : (Acc)0);
                        per_done = k0 + lim;
                        pos = lim;
                    } else {
                        pos = nl;
                    }
                } else {
                    if (t_adc < k0 + nl) {
                        const int l = t_adc - k0;
                        const Acc sl = __shfl_sync(0xffffffffu, sc, l);
                        const float nu = normals2(key, pid, (uint32_t)t_adc, 2u).x;
                        const Acc v = qoff + sl + (Acc)c.sigma_unc_e * (Acc)nu;
                        const float code = fminf(fmaxf(floorf((float)v / lsb_e), 0.f), adc_max);
                        if (lane == 0 && nh < a.hmax) st[nh] = HitRec{t_cross, t_adc, (int32_t)code, (float)v};
                        ++nh;
                        const Acc r = (Acc)c.sigma_reset_e * (Acc)normals2(key, pid, (uint32_t)t_adc, 3u).x;
                        qoff = r - sl;
                        last_adc = t_adc;
                        idle = true;
                        pos = l + 1;
                    } else {
                        pos = nl;
                    }
                }
            }
            qoff += __shfl_sync(0xffffffffu, sc, nl - 1);
        }
        if (lane == 0) a.nhit[pi] = min(nh, a.hmax);
    }
}

// Sets (or clears) the hit-overflow bit and publishes the hit count.
__global__ void k_hits_status(int64_t *counts, int64_t cap, int64_t *n_out)
{
    const int64_t n = counts[2];
    int64_t st = counts[3] & ~(int64_t)SIM_STATUS_HIT_OVERFLOW;
    if (n > cap) st |= SIM_STATUS_HIT_OVERFLOW;
    counts[3] = st;
    if (n_out) *n_out = n;
}

__global__ void __launch_bounds__(kWarps * 32) k_hits_compact(const int32_t *active, const HitRec *stage,
                                                              const int32_t *hoff, int hmax,
                                                              const int64_t *counts, int64_t pix_cap,
                                                              sim_hits out)
{
    if ((counts[3] & (SIM_STATUS_PAIR_OVERFLOW | SIM_STATUS_PIXEL_OVERFLOW)) != 0) return;
    const int64_t npix = counts[1];
    if (npix > pix_cap || counts[2] > out.capacity) return;
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    for (int64_t pi = wg; pi < npix; pi += nw) {
        const int b = hoff[pi], n = hoff[pi + 1] - b;
        const int32_t pid = active[pi];
        for (int h = lane; h < n; h += 32) {
            const HitRec r = stage[(size_t)pi * hmax + h];
            out.pixel[b + h] = pid;
            out.t_cross[b + h] = r.t_cross;
            out.t_adc[b + h] = r.t_adc;
            out.adc[b + h] = (uint8_t)r.adc;
            out.q[b + h] = r.q;
        }
    }
}

}  // namespace

size_t elec_scratch_bytes(const sim_config &c, int64_t pix_cap)
{
    const int hmax = max_hits_per_pixel(c);
    return align256(sizeof(HitRec) * (size_t)pix_cap * hmax) +
           align256(sizeof(int32_t) * (size_t)(pix_cap + 1)) + scan_scratch_bytes(pix_cap + 1);
}

cudaError_t launch_electronics(const sim_config &c, const EventInfo &ev, const int32_t *active,
                               const float *current, int64_t *counts, int64_t pix_cap,
                               const sim_hits &out, void *scratch, cudaStream_t st)
{
    if (pix_cap <= 0) {
        cudaError_t e = cudaMemsetAsync(counts + 2, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return e;
        if (out.n_out) e = cudaMemsetAsync(out.n_out, 0, sizeof(int64_t), st);
        return e;
    }
    const int hmax = max_hits_per_pixel(c);
    char *p = reinterpret_cast<char *>(scratch);
    HitRec *stage = reinterpret_cast<HitRec *>(p);
    p += align256(sizeof(HitRec) * (size_t)pix_cap * hmax);
    int32_t *nhit = reinterpret_cast<int32_t *>(p);
    p += align256(sizeof(int32_t) * (size_t)(pix_cap + 1));
    void *scan_ws = p;

    // pixels beyond the active count contribute zero hits to the scan
    cudaError_t e = cudaMemsetAsync(nhit, 0, sizeof(int32_t) * (size_t)(pix_cap + 1), st);
    if (e != cudaSuccess) return e;
    ElArgs a;
    a.c = c;
    a.ev = ev;
    a.det_px = detector_pixels(geo_of(c));
    a.active = active;
    a.current = current;
    a.counts = counts;
    a.pix_cap = pix_cap;
    a.stage = stage;
    a.nhit = nhit;
    a.hmax = hmax;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (pix_cap + kWarps - 1) / kWarps;
    if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
    if (c.fp64_charge) k_electronics<double><<<(unsigned)grid, kWarps * 32, 0, st>>>(a);
    else k_electronics<float><<<(unsigned)grid, kWarps * 32, 0, st>>>(a);
    e = launch_exclusive_scan(nhit, nhit, pix_cap, counts + 2, scan_ws, st);
    if (e != cudaSuccess) return e;
    k_hits_status<<<1, 1, 0, st>>>(counts, out.capacity, out.n_out);
    k_hits_compact<<<(unsigned)grid, kWarps * 32, 0, st>>>(active, stage, nhit, hmax, counts, pix_cap, out);
    return cudaGetLastError();
}

}  // namespace larsim
