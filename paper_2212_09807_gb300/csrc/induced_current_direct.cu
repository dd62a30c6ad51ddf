// induced_current_direct.cu -- step 4 of the charge path (arXiv:2212.09807
// Sec. 3.3.2), FP32 term-by-term form (precision 3: the direct gather of the
// sum, kept beside the faster node-binned FP32 form of induced_current.cu as
// an independent FP32 evaluation of the same terms): the current induced on
// each active pixel in each tick,
//   I[p, k] = sum_s sum_mu sum_nu q_s Rt(x_mu + dx - x_p, y_mu + dy - y_p, k - a),
// Eq. (current) with the charge density rho of N points x M perturbations
// per segment, summed over the segments mapped to the pixel (the per-pixel
// sum of Sec. 3.4).  Each term reads the table bilinearly at the folded
// offset (four rows b0 = (bx, by), (bx+1, by), (bx, by+1), (bx+1, by+1)) and
// linearly at the fractional arrival tick:
//   v(j) = sum_c w_c R[b_c][j],   I[k] += (1 - f) v(k - A + L - 1) + f v(k - A + L - 2)
// (w_c include the point charge q = Q_a / (N M)).
//
// Design: one CTA of 256 threads per active pixel (grid-stride, three CTAs per
// SM), output stationary: 2048 ticks per pass.  Warp w owns a low block of
// 128 ticks (128 w ..) and its mirror (2048 - 128 (w + 1) ..); in each block
// lane l owns ticks l, 32 + l, 64 + l, 96 + l, in registers.  A record's ticks
// form one interval, which for drifting charge usually starts at the window
// start, so pairing each low block with a high one keeps the warps evenly
// loaded while warps skip the blocks a record does not reach.
//  1. records: the CTA regenerates every perturbed point of the pixel's
//     segments (Philox keyed by segment and point), keeps those within the
//     table's reach of this pixel as records {A, b0, f, w[4]} in its scratch
//     slice (point order), with their bins and a bin histogram in shared memory;
//  2. stable counting sort by bin (one warp computes destinations with
//     match_any ranks from the bins in shared memory; the CTA moves the records);
//  3. per distinct bin: the four table rows are staged once in shared memory
//     (read one bin ahead into registers), interleaved so that each position
//     holds the four corner values as one 16-byte quad, with zero quads beyond
//     both ends of the row.  A record then costs a lane one 16-byte shared
//     read and a 4-term dot product per tick for v(j); v(j - 1) is the
//     neighbouring lane's v(j) (warp shuffle).  Consecutive lanes read
//     consecutive quads: no bank conflicts.
// A pixel's records fall on ~1000 of the 2025 bins, ~7 records per bin, so the
// table is read from L2 once per (pixel, bin) instead of once per record.
// Summation order is fixed (chunks in point order, bins increasing, records
// in point order within a bin): results are bitwise reproducible.  A chunk's
// records (at most kRecCap) are summed in FP32 registers and each chunk's sum
// is added into a compensated (Kahan) running total per tick, kept in a small
// per-CTA scratch row: a dense pixel sums ~1e6 records, whose plain FP32 sum
// drifts by a few 1e-5 of its value; within a chunk the drift is ~5e-6.
#include <algorithm>

#include "current_records.cuh"

namespace larsim {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTPL = 4;                         // consecutive ticks per lane and block
constexpr int kHalf = 32 * kTPL;                // ticks per block
constexpr int kPass = 2 * kThreads * kTPL;      // ticks per pass (two blocks per warp)
constexpr int kRecCap = 8192;                   // records per chunk (per-CTA scratch)
constexpr int kMaxBins = 2048;                  // nb * nb <= kMaxBins
constexpr int kMaxRow = 2048;                   // staged row length (>= nt rounded to 4)
constexpr int kEdge = kHalf + 8;                // zero quads before position 0 and after L - 1
constexpr int kQuads = kMaxRow + 2 * kEdge;     // staged quads (position p at p + kEdge)
constexpr int kPosPerThread = kMaxRow / kThreads;   // positions staged per thread

struct CurArgs {
    sim_config c;
    const float *lut;
    int nb, nt, ld, bpp, lp;                    // lp = nt rounded up to 4
    float inv_nb;
    const Anchor *anch;
    const int32_t *active, *off, *segs;
    const int64_t *counts;
    int64_t pix_cap, pix_begin, pix_end;        // active pixels [pix_begin, min(counts[1], pix_end))
    float *current;
    uint64_t seed;
    EventInfo ev;
    Geo g;
    DriftPar dp;
    Rec *recs;                                  // [grid][kRecCap], point order
    Rec *sorted;                                // [grid][kRecCap], bin order
    float *tot;                                 // [grid][2][kPass]: compensated sums of a pass (total, compensation)
};

struct Smem {
    float4 quad[kQuads];                        // (R00, R10, R01, R11) at each table position
    int hist[kMaxBins];                         // bin counts, then scatter cursors
    unsigned short glist[kMaxBins];             // bins present, increasing
    unsigned short gstart[kMaxBins + 1];        // start of each present bin in bin order
    unsigned short rbin[kRecCap];               // bin of record i, then its destination
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

// Table row of corner c of bin b0; corners outside the table read row b0
// (their weight is zero).  b0 / nb is formed in FP32: exact, since
// (b0 + 1/2) / nb stays >= 1/(2 nb) away from an integer.
__device__ __forceinline__ const float *corner_row(const CurArgs &a, int b0, int c)
{
    const int bx = (int)(((float)b0 + 0.5f) * a.inv_nb), by = b0 - bx * a.nb;
    const int dx = c & 1, dy = c >> 1;
    const int row = (bx + dx < a.nb && by + dy < a.nb) ? b0 + dx * a.nb + dy : b0;
    return a.lut + (size_t)row * a.ld;
}

// Thread t stages positions t + 256 i (i < 8) of the four rows: coalesced
// 4-byte global reads into registers, one bin ahead.
struct RowRegs {
    float v[4][kPosPerThread];
};

__device__ __forceinline__ void load_rows(const CurArgs &a, int b0, RowRegs &r)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float *row = corner_row(a, b0, c);
#pragma unroll
        for (int i = 0; i < kPosPerThread; ++i) {
            const int j = threadIdx.x + kThreads * i;
            r.v[c][i] = (j < a.nt) ? __ldg(row + j) : 0.f;
        }
    }
}

__device__ __forceinline__ void store_rows(Smem *s, const RowRegs &r)
{
#pragma unroll
    for (int i = 0; i < kPosPerThread; ++i)
        s->quad[threadIdx.x + kThreads * i + kEdge] = make_float4(r.v[0][i], r.v[1][i], r.v[2][i], r.v[3][i]);
}

__device__ __forceinline__ float dot4(const float4 &w, const float4 &q)
{
    return w.x * q.x + w.y * q.y + w.z * q.z + w.w * q.w;
}

// One record on one block of a warp.  p1 is the position of v(j) at the
// block's first tick; lane l at iteration i handles tick 32 i + l, reading
// v(j) at p1 + 32 i + l and taking v(j - 1) from lane l - 1 (lane 0: from
// lane 31 of the previous iteration, or read directly at i = 0).
__device__ __forceinline__ void apply_block(const Smem *s, int p1, int L, int lane, const float4 &w, float f,
                                            float (&acc)[kTPL])
{
    if (p1 + kHalf - 1 < 0 || p1 - 1 > L - 1) return;     // block outside the row
    const float4 *q = s->quad + kEdge + p1 + lane;
    float carry = 0.f;
    if (lane == 0) carry = dot4(w, q[-1]);
    const float g = 1.f - f;
#pragma unroll
    for (int i = 0; i < kTPL; ++i) {
        const float v = dot4(w, q[32 * i]);
        float vm = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) vm = carry;
        carry = __shfl_sync(0xffffffffu, v, 31);
        acc[i] = fmaf(g, v, acc[i]);
        acc[i] = fmaf(f, vm, acc[i]);
    }
}

// tot += x with compensation c (Kahan): tot - c is the running sum to a few
// FP32 roundings of the final value, however many partial sums are added.
__device__ __forceinline__ void kahan_add(float &tot, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(tot, y);
    c = __fsub_rn(__fsub_rn(t, tot), y);
    tot = t;
}

// Adds a lane's chunk sums (ticks t0 + 32 i of the pass) into the compensated
// totals tot[t] / tot[kPass + t] (starting them on the first chunk) and clears
// the sums.
__device__ __forceinline__ void add_chunk(float *tot, int t0, float (&acc)[kTPL], bool first)
{
#pragma unroll
    for (int i = 0; i < kTPL; ++i) {
        const int t = t0 + 32 * i;
        float sum = first ? 0.f : tot[t], c = first ? 0.f : tot[kPass + t];
        kahan_add(sum, c, acc[i]);
        tot[t] = sum;
        tot[kPass + t] = c;
        acc[i] = 0.f;
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_induced_current_terms(CurArgs a)
{
    if (a.counts[3] != 0) return;
    const int64_t npix = min(a.counts[1], a.pix_end);
    if (a.counts[1] > a.pix_cap) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem *s = reinterpret_cast<Smem *>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = a.c.n_ticks, L = a.nt, M = a.c.mc_per_sample, nb2 = a.nb * a.nb;
    const float clip = a.c.diff_clip_sigma;
    const float fbpp = (float)a.bpp;
    const int npx = a.g.npx_x * a.g.npx_y;
    Rec *recs = a.recs + (size_t)blockIdx.x * kRecCap;
    Rec *sorted = a.sorted + (size_t)blockIdx.x * kRecCap;
    float *tot = a.tot + (size_t)blockIdx.x * 2 * kPass;
    for (int i = tid; i < kQuads; i += kThreads) s->quad[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int blo_tick = kHalf * warp;                            // first tick of my low block
    const int bhi_tick = kPass - kHalf * (warp + 1);              // first tick of my high block

    for (int64_t pi = a.pix_begin + blockIdx.x; pi < npix; pi += gridDim.x) {
        const int32_t pid = a.active[pi];
        const int an = pid / npx;
        const int rem = pid - an * npx;
        const int iy = rem / a.g.npx_x, ix = rem - iy * a.g.npx_x;
        // event of this (virtual) pixel: key and first segment of its slot
        const int slot = an / a.g.n_anodes;
        const uint64_t key = slot_key(a.seed, a.ev, slot);
        const int64_t seg0 = slot_first(a.ev, slot);
        const int e0 = a.off[pi], e1 = a.off[pi + 1];
        for (int k0 = 0; k0 < T; k0 += kPass) {
            float acc_lo[kTPL], acc_hi[kTPL];               // the current chunk's records
#pragma unroll
            for (int i = 0; i < kTPL; ++i) acc_lo[i] = acc_hi[i] = 0.f;
            bool first_chunk = true;
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
                        const PointPos pp = point_position(A, idx, M, key, (uint32_t)(sg - seg0), clip, a.dp);
                        ok = point_record(A, pp, cx, cy, fbpp, a.nb, a.c.nearest_lut, r);
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
                    constexpr int kB = kMaxBins / kThreads;
                    int v[kB], fl[kB], sv = 0, sf = 0;
#pragma unroll
                    for (int i = 0; i < kB; ++i) {
                        const int b = tid * kB + i;
                        v[i] = (b < nb2) ? s->hist[b] : 0;
                        fl[i] = v[i] > 0 ? 1 : 0;
                        sv += v[i];
                        sf += fl[i];
                    }
                    int tv, tf;
                    int pv = block_scan(sv, s, &tv);
                    int pf = block_scan(sf, s, &tf);
#pragma unroll
                    for (int i = 0; i < kB; ++i) {
                        const int b = tid * kB + i;
                        if (b < nb2) {
                            s->hist[b] = pv;             // scatter cursor
                            if (fl[i]) {
                                s->glist[pf] = (unsigned short)b;
                                s->gstart[pf] = (unsigned short)pv;
                            }
                        }
                        pv += v[i];
                        pf += fl[i];
                    }
                    if (tid == 0) {
                        s->n_groups = tf;
                        s->gstart[tf] = (unsigned short)tv;
                    }
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
                        const int pos = v ? s->hist[bin] : 0;
                        __syncwarp();
                        if (v) {
                            if (lane == __ffs(peers) - 1) s->hist[bin] = pos + __popc(peers);
                            s->rbin[i] = (unsigned short)(pos + rank);
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();
                for (int i = tid; i < nrec; i += kThreads) sorted[s->rbin[i]] = recs[i];
                __syncthreads();
                // ---- 3. per bin: stage rows, apply records ------------------------
                const int ng = s->n_groups;
                const int Pbase = k0 + L - 1;            // position of v(j) at tick k0 is Pbase - A
                RowRegs nxt;
                load_rows(a, s->glist[0], nxt);
                for (int g = 0; g < ng; ++g) {
                    const int gbeg = s->gstart[g], gend = s->gstart[g + 1];
                    __syncthreads();                     // previous bin's rows no longer read
                    store_rows(s, nxt);
                    if (g + 1 < ng) load_rows(a, s->glist[g + 1], nxt);
                    __syncthreads();
                    Rec rn = sorted[gbeg];
                    for (int ri = gbeg; ri < gend; ++ri) {
                        const Rec rc = rn;
                        if (ri + 1 < gend) rn = sorted[ri + 1];         // prefetch the next record
                        const int P = Pbase - rc.A;
                        apply_block(s, P + blo_tick, L, lane, rc.w, rc.f, acc_lo);
                        apply_block(s, P + bhi_tick, L, lane, rc.w, rc.f, acc_hi);
                    }
                }
                // the chunk's sums into the compensated totals (each lane its own ticks)
                add_chunk(tot, blo_tick + lane, acc_lo, first_chunk);
                add_chunk(tot, bhi_tick + lane, acc_hi, first_chunk);
                first_chunk = false;
                __syncthreads();
            }
            float *out = a.current + (size_t)pi * T;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t0 = (h ? bhi_tick : blo_tick) + lane;
#pragma unroll
                for (int i = 0; i < kTPL; ++i) {
                    const int k = k0 + t0 + 32 * i;
                    const float v = first_chunk ? 0.f : __fsub_rn(tot[t0 + 32 * i], tot[kPass + t0 + 32 * i]);
                    if (k < T) out[k] = v;
                }
            }
        }
    }
}

int grid_for(int64_t pix_cap, int ctas_per_sm = 3)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (int64_t)sms * ctas_per_sm;
    if (g > pix_cap) g = pix_cap;
    return (int)(g < 1 ? 1 : g);
}
}  // namespace

size_t current_direct_scratch_bytes(int64_t pix_cap)
{
    const int g = grid_for(pix_cap > 0 ? pix_cap : 1);
    return 2 * align256((size_t)g * kRecCap * sizeof(Rec)) + align256((size_t)g * 2 * kPass * sizeof(float));
}


cudaError_t launch_induced_current_direct(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                   const sim_response &r, const int32_t *active,
                                   const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                                   const int64_t *counts, int64_t pix_cap, int64_t pix_begin, int64_t pix_end,
                                   float *current, void *scratch, cudaStream_t st)
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
    a.pix_begin = pix_begin;
    a.pix_end = pix_end;
    a.current = current;
    a.seed = c.seed;
    a.ev = events_of(s);
    a.g = geo_of(c);
    a.dp = drift_par_of(c);
    const int grid = grid_for(pix_cap, c.direct_ctas_per_sm > 0 ? std::min(c.direct_ctas_per_sm, 3) : 3);
    char *p = reinterpret_cast<char *>(scratch);
    a.recs = reinterpret_cast<Rec *>(p);
    a.sorted = reinterpret_cast<Rec *>(p + align256((size_t)grid * kRecCap * sizeof(Rec)));
    a.tot = reinterpret_cast<float *>(p + 2 * align256((size_t)grid * kRecCap * sizeof(Rec)));
    const size_t smem = sizeof(Smem);
    const cudaError_t e = cudaFuncSetAttribute(k_induced_current_terms, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
    k_induced_current_terms<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace larsim
