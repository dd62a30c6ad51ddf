// induced_current.cu -- step 4 of the charge path (arXiv:2212.09807
// Sec. 3.3.2): the current induced on each active pixel in each tick,
//   I[p, k] = sum_s sum_mu sum_nu q_s Rt(x_mu + dx - x_p, y_mu + dy - y_p, k - a),
// Eq. (current) with the charge density rho of N points x M perturbations
// per segment, summed over the segments mapped to the pixel (the per-pixel
// sum of Sec. 3.4).
//
// One CTA per active pixel (grid-stride), output-stationary: the pixel's
// current lives in registers, 256 threads x 8 ticks = 2048 ticks per pass,
// thread t owning ticks k0 + t + 256 i so that every table load of a warp is
// one contiguous 128-byte run.  For each of the pixel's segments (increasing
// index) the CTA regenerates the segment's perturbed points 256 at a time
// (Philox keyed by segment and point), keeps those inside the table's reach
// of this pixel in a shared queue, and adds each queued point's
// bilinear-in-space, linear-in-time table row:
//   v(j)  = sum_c w_c R[b_c][j]            (4 table rows, folded offsets)
//   I[k] += q ((1 - f) v(k - A + L - 1) + f v(k - A + L - 2))
// The second tap is the neighbouring lane's first tap (warp shuffle).
#include "sim_internal.cuh"

namespace larsim {

namespace {
constexpr int kThreads = 256;
constexpr int kPT = 8;
constexpr int kChunk = kThreads * kPT;

struct CurArgs {
    sim_config c;
    const float *lut;
    int nb, nt, ld, bpp;
    const Anchor *anch;
    const int32_t *anode;
    const int32_t *active, *off, *segs;
    const int64_t *counts;
    int64_t pix_cap;
    float *current;
    uint64_t key;
    Geo g;
};

__global__ void __launch_bounds__(kThreads) k_induced_current(CurArgs a)
{
    if (a.counts[3] != 0) return;
    const int64_t npix = a.counts[1];
    if (npix > a.pix_cap) return;

    __shared__ int q_row[kThreads];     // b0 = bx * nb + by
    __shared__ int q_A[kThreads];       // integer arrival tick
    __shared__ float4 q_w[kThreads];    // q-scaled bilinear weights (00, 10, 01, 11)
    __shared__ float q_f[kThreads];     // fractional arrival
    __shared__ int warp_n[kThreads / 32];

    const int tid = threadIdx.x, lane = tid & 31;
    const int T = a.c.n_ticks, L = a.nt, M = a.c.mc_per_sample;
    const float clip = a.c.diff_clip_sigma;
    const float fbpp = (float)a.bpp, fnb = (float)a.nb;
    const int npx = a.g.npx_x * a.g.npx_y;

    for (int64_t pi = blockIdx.x; pi < npix; pi += gridDim.x) {
        const int32_t pid = a.active[pi];
        const int an = pid / npx;
        const int rem = pid - an * npx;
        const int iy = rem / a.g.npx_x, ix = rem - iy * a.g.npx_x;
        const int e0 = a.off[pi], e1 = a.off[pi + 1];
        for (int k0 = 0; k0 < T; k0 += kChunk) {
            float acc[kPT];
#pragma unroll
            for (int i = 0; i < kPT; ++i) acc[i] = 0.f;
            for (int e = e0; e < e1; ++e) {
                const int s = a.segs[e];
                const Anchor A = a.anch[s];
                const float cx = (float)(ix - A.ix_ref) + 0.5f;
                const float cy = (float)(iy - A.iy_ref) + 0.5f;
                const int total = A.N * M;
                const float invN = 1.0f / (float)A.N;
                for (int base = 0; base < total; base += kThreads) {
                    const int idx = base + tid;
                    bool ok = false;
                    int row = 0, Ai = 0;
                    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
                    float f = 0.f;
                    if (idx < total) {
                        const int mu = idx / M;
                        float3 n = normals3(a.key, (uint32_t)s, (uint32_t)idx, 1u);
                        n.x = fminf(fmaxf(n.x, -clip), clip);
                        n.y = fminf(fmaxf(n.y, -clip), clip);
                        n.z = fminf(fmaxf(n.z, -clip), clip);
                        const float u = ((float)mu + 0.5f) * invN;
                        const float fx = A.fx0 + u * A.dX + A.sTp * n.x;
                        const float fy = A.fy0 + u * A.dY + A.sTp * n.y;
                        float xi = fabsf((fx - cx) * fbpp) - 0.5f;
                        float yi = fabsf((fy - cy) * fbpp) - 0.5f;
                        xi = fmaxf(xi, 0.f);
                        yi = fmaxf(yi, 0.f);
                        if (xi < fnb && yi < fnb) {
                            ok = true;
                            float lin = A.fa0 + u * A.da + A.sLc * n.z * A.kz;
                            const float dmu = A.d0 + u * A.dd + A.sLc * n.z;
                            if (dmu < 0.f) lin -= 2.0f * dmu * A.kz;
                            const float fl = floorf(lin);
                            f = lin - fl;
                            Ai = A.A0 + (int)fl;
                            const int bx = (int)xi, by = (int)yi;
                            const float wx = xi - (float)bx, wy = yi - (float)by;
                            const float wx1 = (bx + 1 < a.nb) ? wx : 0.f;
                            const float wy1 = (by + 1 < a.nb) ? wy : 0.f;
                            row = bx * a.nb + by;
                            const float q = A.q;
                            w = make_float4(q * (1.f - wx) * (1.f - wy), q * wx1 * (1.f - wy),
                                            q * (1.f - wx) * wy1, q * wx1 * wy1);
                        }
                    }
                    // queue order = point order (warp prefix of ballot counts), so the
                    // FP32 sum is formed in the same order on every run
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    const int warp = tid >> 5;
                    if (lane == 0) warp_n[warp] = __popc(m);
                    __syncthreads();
                    int wbase = 0, nq = 0;
#pragma unroll
                    for (int w2 = 0; w2 < kThreads / 32; ++w2) {
                        const int c2 = warp_n[w2];
                        wbase += (w2 < warp) ? c2 : 0;
                        nq += c2;
                    }
                    if (ok) {
                        const int slot = wbase + __popc(m & ((1u << lane) - 1u));
                        q_row[slot] = row;
                        q_A[slot] = Ai;
                        q_w[slot] = w;
                        q_f[slot] = f;
                    }
                    __syncthreads();
                    for (int r = 0; r < nq; ++r) {
                        const int b0 = q_row[r];
                        const float4 wr = q_w[r];
                        const float fr = q_f[r];
                        const int jb = k0 + tid - q_A[r] + L - 1;   // j of tick k0 + tid
                        const int bx1 = (b0 / a.nb + 1 < a.nb) ? a.nb : 0;
                        const int by1 = (b0 % a.nb + 1 < a.nb) ? 1 : 0;
                        const float *r00 = a.lut + (size_t)b0 * a.ld;
                        const float *r10 = r00 + (size_t)bx1 * a.ld;
                        const float *r01 = r00 + (size_t)by1 * a.ld;
                        const float *r11 = r10 + (size_t)by1 * a.ld;
#pragma unroll
                        for (int i = 0; i < kPT; ++i) {
                            const int j = jb + i * kThreads;
                            float v = 0.f;
                            if ((unsigned)j < (unsigned)L) {
                                v = wr.x * __ldg(r00 + j) + wr.y * __ldg(r10 + j) +
                                    wr.z * __ldg(r01 + j) + wr.w * __ldg(r11 + j);
                            }
                            float vm = __shfl_up_sync(0xffffffffu, v, 1);
                            if (lane == 0) {
                                const int jm = j - 1;
                                vm = 0.f;
                                if ((unsigned)jm < (unsigned)L) {
                                    vm = wr.x * __ldg(r00 + jm) + wr.y * __ldg(r10 + jm) +
                                         wr.z * __ldg(r01 + jm) + wr.w * __ldg(r11 + jm);
                                }
                            }
                            acc[i] += (1.f - fr) * v + fr * vm;
                        }
                    }
                    __syncthreads();
                }
            }
            float *out = a.current + (size_t)pi * T;
#pragma unroll
            for (int i = 0; i < kPT; ++i) {
                const int k = k0 + tid + i * kThreads;
                if (k < T) out[k] = acc[i];
            }
        }
    }
}
}  // namespace

cudaError_t launch_induced_current(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                   const sim_response &r, const int32_t *active,
                                   const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                                   const int64_t *counts, int64_t pix_cap, float *current,
                                   cudaStream_t st)
{
    if (pix_cap <= 0) return cudaSuccess;
    CurArgs a;
    a.c = c;
    a.lut = r.lut;
    a.nb = r.nb;
    a.nt = r.nt;
    a.ld = r.ld;
    a.bpp = r.bins_per_pitch;
    a.anch = reinterpret_cast<const Anchor *>(d.anchors);
    a.anode = d.anode;
    a.active = active;
    a.off = pix_seg_off;
    a.segs = pix_seg_ids;
    a.counts = counts;
    a.pix_cap = pix_cap;
    a.current = current;
    a.key = c.seed ^ s.event_id;
    a.g = geo_of(c);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (int64_t)sms * 8;
    if (grid > pix_cap) grid = pix_cap;
    k_induced_current<<<(unsigned)grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace larsim
