// induced_current.cu -- step 4 of the charge path (arXiv:2212.09807
// Sec. 3.3.2): the current induced on each active pixel in each tick,
//   I[p, k] = sum_s sum_mu sum_nu q_s Rt(x_mu + dx - x_p, y_mu + dy - y_p, k - a),
// Eq. (current) with the charge density rho of N points x M perturbations
// per segment, summed over the segments mapped to the pixel (the per-pixel
// sum of Sec. 3.4).  Each term reads the table bilinearly at the folded
// offset (four rows b0 = (bx, by), (bx+1, by), (bx, by+1), (bx+1, by+1)) and
// linearly at the fractional arrival tick:
//   v(j) = sum_c w_c R[b_c][j],   I[k] += (1 - f) v(k - A + L - 1) + f v(k - A + L - 2)
// (w_c include the point charge q = Q_a / (N M)).
//
// Design: one CTA of 512 threads per active pixel (grid-stride, two CTAs per
// SM), output stationary: 2048 ticks per pass, lane l of warp w owning ticks
// 128 w + 4 l .. + 3 in registers.
//  1. records: the CTA regenerates every perturbed point of the pixel's
//     segments (Philox keyed by segment and point), keeps those within the
//     table's reach of this pixel as records {A, b0, f, w[4]} in its scratch
//     slice (point order), with their bins and a bin histogram in shared memory;
//  2. stable counting sort by bin (one warp computes destinations with
//     match_any ranks from the bins in shared memory; the CTA moves the records);
//  3. per distinct bin: the four table rows are staged once in shared memory
//     (16-byte global reads issued one bin ahead into registers) in a padded
//     layout, address p + p/4, under which the lanes' stride-4 reads hit 32
//     distinct banks for any start; every record of the bin is then applied
//     with 5 shared reads per row per lane (both time taps of 4 ticks), the
//     read offsets being immediates selected by the record's (p mod 4).
// A pixel's records fall on ~1000 of the 2025 bins, ~7 records per bin, so the
// table is read from L2 once per (pixel, bin) instead of once per record.
// Summation order is fixed (chunks in point order, bins increasing, records
// in point order within a bin): results are bitwise reproducible.
#include "sim_internal.cuh"

namespace larsim {

namespace {
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kTPL = 4;                         // consecutive ticks per lane
constexpr int kPass = kThreads * kTPL;          // ticks per pass
constexpr int kRecCap = 8192;                   // records per chunk (per-CTA scratch)
constexpr int kMaxBins = 2048;                  // nb * nb <= kMaxBins
constexpr int kMaxRow = 2048;                   // staged row length (>= nt rounded to 4)
constexpr int kRowPad = kMaxRow + kMaxRow / 4;  // padded row: position p at p + p / 4
constexpr int kF4PerRowThread = 4;              // 128 threads x 4 float4 = 512 float4 = kMaxRow / 4

struct __align__(16) Rec {
    int A, b0;
    float f, pad;
    float4 w;                                   // q-scaled weights of rows (0,0), (1,0), (0,1), (1,1)
};

struct CurArgs {
    sim_config c;
    const float *lut;
    int nb, nt, ld, bpp, lp;                    // lp = nt rounded up to 4
    float inv_nb;
    const Anchor *anch;
    const int32_t *active, *off, *segs;
    const int64_t *counts;
    int64_t pix_cap;
    float *current;
    uint64_t key;
    Geo g;
    Rec *recs;                                  // [grid][kRecCap], point order
    Rec *sorted;                                // [grid][kRecCap], bin order
};

struct Smem {
    float rows[4][kRowPad];
    int hist[kMaxBins];
    int cur[kMaxBins];
    int glist[kMaxBins];
    unsigned short rbin[kRecCap];
    int warp_n[kWarps];
    int scan_tmp[kWarps + 1];
    int n_groups;
};

// Exclusive scan of one int per thread across the CTA; returns the prefix
// and the total in *tot.
__device__ __forceinline__ int block_scan(int v, Smem *s, int *tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s->scan_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kWarps ? s->scan_tmp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < kWarps) s->scan_tmp[lane] = wi - w;
        if (lane == kWarps - 1) s->scan_tmp[kWarps] = wi;
    }
    __syncthreads();
    const int r = s->scan_tmp[warp] + x - v;
    *tot = s->scan_tmp[kWarps];
    __syncthreads();
    return r;
}

// Rows are staged by 128 threads each: thread t handles row t >> 7 and the
// float4 indices (t & 127) + 128 i.  Corners outside the table read row b0
// (their weight is zero).  b0 / nb is formed in FP32: exact, since
// (b0 + 1/2) / nb stays >= 1/(2 nb) away from an integer.
__device__ __forceinline__ void load_rows(const CurArgs &a, int b0, float4 (&r)[kF4PerRowThread])
{
    const int c = threadIdx.x >> 7, q = threadIdx.x & 127;
    const int bx = (int)(((float)b0 + 0.5f) * a.inv_nb), by = b0 - bx * a.nb;
    const int dx = c & 1, dy = c >> 1;
    const int row = (bx + dx < a.nb && by + dy < a.nb) ? b0 + dx * a.nb + dy : b0;
    const float4 *src = reinterpret_cast<const float4 *>(a.lut + (size_t)row * a.ld);
    const int n4 = a.lp >> 2;
#pragma unroll
    for (int i = 0; i < kF4PerRowThread; ++i) {
        const int qi = q + 128 * i;
        if (qi < n4) r[i] = __ldg(src + qi);
    }
}

__device__ __forceinline__ void store_rows(const CurArgs &a, Smem *s, const float4 (&r)[kF4PerRowThread])
{
    const int c = threadIdx.x >> 7, q = threadIdx.x & 127;
    const int n4 = a.lp >> 2;
    float *dst = s->rows[c];
#pragma unroll
    for (int i = 0; i < kF4PerRowThread; ++i) {
        const int qi = q + 128 * i;
        if (qi < n4) {
            const int j = 4 * qi;               // positions j..j+3 live at 5 qi .. 5 qi + 3
            float *d = dst + 5 * qi;
            d[0] = (j + 0 < a.nt) ? r[i].x : 0.f;
            d[1] = (j + 1 < a.nt) ? r[i].y : 0.f;
            d[2] = (j + 2 < a.nt) ? r[i].z : 0.f;
            d[3] = (j + 3 < a.nt) ? r[i].w : 0.f;
        }
    }
}

// v at padded address `ad` of the four staged rows.
__device__ __forceinline__ float vrow(const Smem *s, int ad, const float4 &w)
{
    return w.x * s->rows[0][ad] + w.y * s->rows[1][ad] + w.z * s->rows[2][ad] + w.w * s->rows[3][ad];
}

// One record, all positions of the warp inside the row: positions p0 + m,
// m = 0..4, with p0 = 4 q + R live at 5 q + R + m + ((R + m) >> 2); R is the
// same for every lane of the CTA, so each case uses immediate offsets only.
template <int R>
__device__ __forceinline__ void apply_fast(const Smem *s, int ad5q, const float4 &w, float f, float (&acc)[kTPL])
{
    float v[kTPL + 1];
#pragma unroll
    for (int m = 0; m <= kTPL; ++m) v[m] = vrow(s, ad5q + R + m + ((R + m) >> 2), w);
#pragma unroll
    for (int i = 0; i < kTPL; ++i) acc[i] += (1.f - f) * v[i + 1] + f * v[i];
}

__global__ void __launch_bounds__(kThreads, 2) k_induced_current(CurArgs a)
{
    if (a.counts[3] != 0) return;
    const int64_t npix = a.counts[1];
    if (npix > a.pix_cap) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem *s = reinterpret_cast<Smem *>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = a.c.n_ticks, L = a.nt, M = a.c.mc_per_sample, nb2 = a.nb * a.nb;
    const float clip = a.c.diff_clip_sigma;
    const float fbpp = (float)a.bpp, fnb = (float)a.nb;
    const int npx = a.g.npx_x * a.g.npx_y;
    Rec *recs = a.recs + (size_t)blockIdx.x * kRecCap;
    Rec *sorted = a.sorted + (size_t)blockIdx.x * kRecCap;
    const int lane_tick = warp * (32 * kTPL) + lane * kTPL;       // first tick of this lane in a pass

    for (int64_t pi = blockIdx.x; pi < npix; pi += gridDim.x) {
        const int32_t pid = a.active[pi];
        const int an = pid / npx;
        const int rem = pid - an * npx;
        const int iy = rem / a.g.npx_x, ix = rem - iy * a.g.npx_x;
        const int e0 = a.off[pi], e1 = a.off[pi + 1];
        for (int k0 = 0; k0 < T; k0 += kPass) {
            float acc[kTPL];
#pragma unroll
            for (int i = 0; i < kTPL; ++i) acc[i] = 0.f;
            int e = e0, base = 0;                                     // generation cursor
            while (e < e1) {
                // ---- 1. records of this chunk -------------------------------------
                for (int b = tid; b < nb2; b += kThreads) s->hist[b] = 0;
                __syncthreads();
                int nrec = 0;
                while (e < e1) {
                    const int sg = a.segs[e];
                    const Anchor A = a.anch[sg];
                    const int total = A.N * M;
                    if (base >= total) {
                        ++e;
                        base = 0;
                        continue;
                    }
                    const float cx = (float)(ix - A.ix_ref) + 0.5f;
                    const float cy = (float)(iy - A.iy_ref) + 0.5f;
                    const int idx = base + tid;
                    bool ok = false;
                    Rec r;
                    if (idx < total) {
                        const int mu = (M == 1) ? idx : idx / M;
                        float3 n = normals3(a.key, (uint32_t)sg, (uint32_t)idx, 1u);
                        n.x = fminf(fmaxf(n.x, -clip), clip);
                        n.y = fminf(fmaxf(n.y, -clip), clip);
                        n.z = fminf(fmaxf(n.z, -clip), clip);
                        const float u = ((float)mu + 0.5f) / (float)A.N;
                        const float fx = A.fx0 + u * A.dX + A.sTp * n.x;
                        const float fy = A.fy0 + u * A.dY + A.sTp * n.y;
                        const float xi = fmaxf(fabsf((fx - cx) * fbpp) - 0.5f, 0.f);
                        const float yi = fmaxf(fabsf((fy - cy) * fbpp) - 0.5f, 0.f);
                        if (xi < fnb && yi < fnb) {
                            ok = true;
                            float lin = A.fa0 + u * A.da + A.sLc * n.z * A.kz;
                            const float dmu = A.d0 + u * A.dd + A.sLc * n.z;
                            if (dmu < 0.f) lin -= 2.0f * dmu * A.kz;
                            const float fl = floorf(lin);
                            const int bx = (int)xi, by = (int)yi;
                            const float wx = xi - (float)bx, wy = yi - (float)by;
                            // node nb (beyond the table) reads zero: far corners get no weight
                            const float ex = (bx + 1 < a.nb) ? 1.f : 0.f, ey = (by + 1 < a.nb) ? 1.f : 0.f;
                            const float q1 = A.q * (1.f - wx), q2 = A.q * wx * ex;
                            r.A = A.A0 + (int)fl;
                            r.b0 = bx * a.nb + by;
                            r.f = lin - fl;
                            r.pad = 0.f;
                            r.w = make_float4(q1 * (1.f - wy), q2 * (1.f - wy), q1 * wy * ey, q2 * wy * ey);
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (lane == 0) s->warp_n[warp] = __popc(m);
                    __syncthreads();
                    int wb = 0, nq = 0;
#pragma unroll
                    for (int w2 = 0; w2 < kWarps; ++w2) {
                        const int c2 = s->warp_n[w2];
                        wb += (w2 < warp) ? c2 : 0;
                        nq += c2;
                    }
                    __syncthreads();
                    if (nrec + nq > kRecCap) break;      // chunk full: process it, then redo this batch
                    if (ok) {
                        const int slot = nrec + wb + __popc(m & ((1u << lane) - 1u));
                        recs[slot] = r;
                        s->rbin[slot] = (unsigned short)r.b0;
                        atomicAdd(&s->hist[r.b0], 1);
                    }
                    nrec += nq;
                    base += kThreads;
                }
                __syncthreads();
                if (nrec == 0) continue;
                // ---- 2. bin offsets, bin list, stable move to bin order -----------
                {
                    int v[4], fl[4], sv = 0, sf = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int b = tid * 4 + i;
                        v[i] = (b < nb2) ? s->hist[b] : 0;
                        fl[i] = v[i] > 0 ? 1 : 0;
                        sv += v[i];
                        sf += fl[i];
                    }
                    int tv, tf;
                    int pv = block_scan(sv, s, &tv);
                    int pf = block_scan(sf, s, &tf);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int b = tid * 4 + i;
                        if (b < nb2) {
                            s->cur[b] = pv;
                            if (fl[i]) s->glist[pf] = b;
                        }
                        pv += v[i];
                        pf += fl[i];
                    }
                    if (tid == 0) s->n_groups = tf;
                }
                __syncthreads();
                if (warp == 0) {
                    // destination of record i (stable within a bin) replaces its bin in rbin[i]
                    for (int i0 = 0; i0 < nrec; i0 += 32) {
                        const int i = i0 + lane;
                        const bool v = i < nrec;
                        const int bin = v ? (int)s->rbin[i] : -1 - lane;
                        const unsigned peers = __match_any_sync(0xffffffffu, bin);
                        const int rank = __popc(peers & ((1u << lane) - 1u));
                        const int pos = v ? s->cur[bin] : 0;
                        __syncwarp();
                        if (v) {
                            if (lane == __ffs(peers) - 1) s->cur[bin] = pos + __popc(peers);
                            s->rbin[i] = (unsigned short)(pos + rank);
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();
                for (int i = tid; i < nrec; i += kThreads) sorted[s->rbin[i]] = recs[i];
                __syncthreads();
                // cur[b] is now the end offset of bin b; its start is end - hist[b]
                // ---- 3. per bin: stage rows, apply records ------------------------
                const int ng = s->n_groups;
                const int Pbase = k0 + L - 2;            // position of v(j-1) at tick k0 is Pbase - A
                float4 nxt[kF4PerRowThread];
                load_rows(a, s->glist[0], nxt);
                for (int g = 0; g < ng; ++g) {
                    const int b0 = s->glist[g];
                    const int gend = s->cur[b0], gbeg = gend - s->hist[b0];
                    __syncthreads();                     // previous bin's rows no longer read
                    store_rows(a, s, nxt);
                    if (g + 1 < ng) load_rows(a, s->glist[g + 1], nxt);
                    __syncthreads();
                    Rec rn = sorted[gbeg];
                    for (int ri = gbeg; ri < gend; ++ri) {
                        const Rec rc = rn;
                        if (ri + 1 < gend) rn = sorted[ri + 1];         // prefetch the next record
                        const int wlo = Pbase - rc.A + warp * (32 * kTPL);   // warp's positions [wlo, wlo + 128]
                        if (wlo + 32 * kTPL < 0 || wlo >= L) continue;
                        const float f = rc.f;
                        const int p0 = wlo + lane * kTPL;
                        if (wlo >= 0 && wlo + 32 * kTPL < L) {
                            const int ad5q = 5 * (p0 >> 2);
                            switch (p0 & 3) {
                            case 0: apply_fast<0>(s, ad5q, rc.w, f, acc); break;
                            case 1: apply_fast<1>(s, ad5q, rc.w, f, acc); break;
                            case 2: apply_fast<2>(s, ad5q, rc.w, f, acc); break;
                            default: apply_fast<3>(s, ad5q, rc.w, f, acc); break;
                            }
                        } else {
                            float v[kTPL + 1];
#pragma unroll
                            for (int m2 = 0; m2 <= kTPL; ++m2) {
                                const int p = p0 + m2;
                                const bool in = (unsigned)p < (unsigned)L;
                                const int pc = in ? p : 0;
                                const float t = vrow(s, pc + (pc >> 2), rc.w);
                                v[m2] = in ? t : 0.f;
                            }
#pragma unroll
                            for (int i = 0; i < kTPL; ++i) acc[i] += (1.f - f) * v[i + 1] + f * v[i];
                        }
                    }
                }
                __syncthreads();
            }
            const int kw = k0 + lane_tick;
            float *out = a.current + (size_t)pi * T;
            if (kw + kTPL <= T && (((size_t)pi * T + kw) & 3) == 0) {
                *reinterpret_cast<float4 *>(out + kw) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            } else {
#pragma unroll
                for (int i = 0; i < kTPL; ++i)
                    if (kw + i < T) out[kw + i] = acc[i];
            }
        }
    }
}

int grid_for(int64_t pix_cap)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (int64_t)sms * 2;
    if (g > pix_cap) g = pix_cap;
    return (int)(g < 1 ? 1 : g);
}
}  // namespace

size_t current_scratch_bytes(int64_t pix_cap)
{
    const int g = grid_for(pix_cap > 0 ? pix_cap : 1);
    return 2 * align256((size_t)g * kRecCap * sizeof(Rec));
}

bool current_table_ok(int nb, int nt) { return nb * nb <= kMaxBins && ((nt + 3) / 4) * 4 <= kMaxRow; }

cudaError_t launch_induced_current(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                   const sim_response &r, const int32_t *active,
                                   const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                                   const int64_t *counts, int64_t pix_cap, float *current, void *scratch,
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
    a.lp = ((r.nt + 3) / 4) * 4;
    a.inv_nb = 1.0f / (float)r.nb;
    a.anch = reinterpret_cast<const Anchor *>(d.anchors);
    a.active = active;
    a.off = pix_seg_off;
    a.segs = pix_seg_ids;
    a.counts = counts;
    a.pix_cap = pix_cap;
    a.current = current;
    a.key = c.seed ^ s.event_id;
    a.g = geo_of(c);
    const int grid = grid_for(pix_cap);
    char *p = reinterpret_cast<char *>(scratch);
    a.recs = reinterpret_cast<Rec *>(p);
    a.sorted = reinterpret_cast<Rec *>(p + align256((size_t)grid * kRecCap * sizeof(Rec)));
    const size_t smem = sizeof(Smem);
    const cudaError_t e = cudaFuncSetAttribute(k_induced_current, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
    k_induced_current<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace larsim
