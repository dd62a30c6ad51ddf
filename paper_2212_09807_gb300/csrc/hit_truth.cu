// hit_truth.cu -- per-hit charge truth (arXiv:2212.09807: the front end of
// Sec. 3.4 with the truth-propagation scheme of Sec. 4.4 carried over to the
// charge readout): for every hit, the charge that each segment mapped to the
// hit's pixel induced during the ticks the hit digitises, and the hit's whole
// signal charge (noise excluded).
//
// A hit digitises the current of ticks [k0, k1]: k1 is its ADC tick, k0 the
// tick after the previous hit's ADC tick (window start for the first hit), or
// the latest periodic reset at or before its crossing.  One record of
// Eq. (current) (point charge q w_c on the four table rows c, arrival A + f)
// has induced, up to and including tick k,
//   F(k) = (1 - f) C(k - A + L - 1) + f C(k - A + L - 2),
//   C(m) = sum_c w_c cum_c[min(m, L - 1)]   (C = 0 for m < 0),
// with cum the running sum of each table row (sim_response_cumulative,
// accumulated in FP64), so that it puts F(k1) - F(k0 - 1) into the interval:
// two table reads per interval boundary, and the boundary between two
// consecutive hits is shared.
//
// Work plan: the hit list is cut into runs of hits of one pixel; each run is
// cut into units of up to kHC hits x kSegU of the pixel's segments.  A unit's
// CTA cuts the flattened (segment, point) space of its segments into one
// contiguous range per thread; a thread regenerates each perturbed point of
// its range (the same records as the current kernels, current_records.cuh),
// sums each hit's charge in FP32 registers, in point order, while the segment
// stays the same, and adds the sums, rounded to fixed point (2^-16 e-), into
// shared 64-bit integer accumulators per (hit, segment) when it changes
// (integer additions: exact, so the totals do not depend on their order; the
// ranges depend only on the unit's point count); the unit's accumulators are
// written to the run's cell block [hits][segments] in the workspace.  Then one warp per hit adds its row (the signal, exact) and
// picks the K largest |charge| (ties: lower segment index first).  A pixel
// with many hits and segments (a shower core: 1e6 points, 100 hits) is
// spread over many SMs.  Results are bitwise reproducible.
#include "current_records.cuh"

namespace larsim {

namespace {

constexpr int kThreads = 256;
constexpr int kHC = 16;                        // hits of a unit
constexpr int kSegU = 64;                      // segments of a unit
constexpr double kFix = 65536.0;               // fixed point of the cells (e-)

// Workspace counts block (int64): cells needed (exact), runs, units, status,
// and the 32-bit scan's cell total (trusted only when cells <= max_cells < 2^31).
enum { kCntCells = 0, kCntRuns = 1, kCntUnits = 2, kCntStatus = 3, kCntScan = 4 };

struct TruthArgs {
    sim_config c;
    const Anchor *anch;
    const float4 *cum;
    int nb, nt, ld, bpp;
    const int32_t *active, *off, *segs;
    const int64_t *counts;
    int64_t pix_cap;
    const int32_t *hpix, *hta, *htc;
    const int64_t *n_hits;
    int64_t hcap;
    int K;
    int32_t *oseg;
    float *oq, *osig;
    int32_t *ok0;
    uint64_t seed;
    EventInfo ev;
    Geo g;
    DriftPar dp;
    // plan (workspace)
    int64_t *wcnt;
    int64_t max_cells;
    int32_t *rflag;                            // [hcap + 1]: run starts, then their exclusive scan
    int32_t *r_h0, *r_nh, *r_e0, *r_ns;        // per run
    int32_t *ucnt, *ccnt;                      // per run [hcap + 1]: units, cells; then exclusive scans
    unsigned long long *cells;
};

__device__ __forceinline__ bool plan_ok(const TruthArgs &a)
{
    return (a.counts[3] & (SIM_STATUS_PAIR_OVERFLOW | SIM_STATUS_PIXEL_OVERFLOW)) == 0;
}

__device__ __forceinline__ int64_t hit_count(const TruthArgs &a) { return min(*a.n_hits, a.hcap); }

// First tick of the interval of hit h, the first hit of its pixel being h0.
__device__ __forceinline__ int interval_start(const TruthArgs &a, int64_t h, int64_t h0)
{
    int start = h == h0 ? 0 : a.hta[h - 1] + 1;
    const int per = a.c.periodic_reset_ticks;
    if (per > 0) {
        const int r = (a.htc[h] / per) * per;
        if (r > 0 && r > start) start = r;
    }
    return start;
}

__global__ void k_run_flags(TruthArgs a)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h > a.hcap) return;
    const int64_t nh = hit_count(a);
    a.rflag[h] = (h < nh && (h == 0 || a.hpix[h] != a.hpix[h - 1])) ? 1 : 0;
}

// Per run (after the flag scan): first hit, hits, the pixel's segment range,
// and its numbers of units and cells.
__global__ void k_run_fill(TruthArgs a)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nh = hit_count(a);
    if (h >= nh || !(h == 0 || a.hpix[h] != a.hpix[h - 1])) return;
    const int r = a.rflag[h];
    const int32_t pid = a.hpix[h];
    int64_t h1 = h + 1;
    while (h1 < nh && a.hpix[h1] == pid) ++h1;
    const int64_t npix = min(a.counts[1], a.pix_cap);
    int64_t lo = 0, hi = npix - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a.active[mid] < pid) lo = mid + 1; else hi = mid;
    }
    const bool found = plan_ok(a) && npix > 0 && a.active[lo] == pid;
    const int e0 = found ? a.off[lo] : 0, ns = found ? a.off[lo + 1] - e0 : 0;
    const int n = (int)(h1 - h);
    a.r_h0[r] = (int32_t)h;
    a.r_nh[r] = n;
    a.r_e0[r] = e0;
    a.r_ns[r] = ns;
    a.ucnt[r] = ns > 0 ? ((n + kHC - 1) / kHC) * ((ns + kSegU - 1) / kSegU) : 0;
    a.ccnt[r] = n * ns;
    atomicAdd(reinterpret_cast<unsigned long long *>(a.wcnt + kCntCells), (unsigned long long)n * (unsigned long long)ns);
}

// Cells and units of the call (after the scans); too many cells: status, nothing more is done.
__global__ void k_plan_check(TruthArgs a)
{
    if (a.wcnt[kCntCells] > a.max_cells) a.wcnt[kCntStatus] |= 1;
}

struct UnitSmem {
    unsigned long long acc[kHC][kSegU];
    int pre[kSegU + 1];
    int ilo[kSegU];                            // first point of each segment that can reach the pixel
    int klo[kHC], khi[kHC];                    // hit j covers ticks (klo[j], khi[j]]
};

// F(k) of one record: charge it induced up to and including tick k.  Both
// reads are always issued (positions clamped into the row) and masked after,
// so that the reads of all of a record's boundaries are independent.
__device__ __forceinline__ float rec_cum(const Rec &r, const float4 *row, int L, int k)
{
    const int m = k - r.A + L - 1;
    const float4 c1 = __ldg(row + min(max(m, 0), L - 1));
    const float4 c0 = __ldg(row + min(max(m - 1, 0), L - 1));
    const float v1 = m >= 0 ? r.w.x * c1.x + r.w.y * c1.y + r.w.z * c1.z + r.w.w * c1.w : 0.f;
    const float v0 = m >= 1 ? r.w.x * c0.x + r.w.y * c0.y + r.w.z * c0.z + r.w.w * c0.w : 0.f;
    return (1.f - r.f) * v1 + r.f * v0;
}

// Charges of one record in the intervals of NH hits (NH >= nc; hits j >= nc
// read valid positions and are discarded).
template <int NH>
__device__ __forceinline__ void record_hits(const Rec &rc, const float4 *row, int L, const int *klo, const int *khi,
                                            int nc, float (&part)[kHC])
{
    float Fb[NH + 1];
    Fb[0] = rec_cum(rc, row, L, klo[0]);
#pragma unroll
    for (int j = 0; j < NH; ++j) Fb[j + 1] = rec_cum(rc, row, L, khi[j]);
#pragma unroll
    for (int j = 0; j < NH; ++j) {
        if (j < nc) {
            // lower boundary: the previous upper one, unless a periodic reset moved it
            const float lo = klo[j] == (j ? khi[j - 1] : klo[0]) ? Fb[j] : rec_cum(rc, row, L, klo[j]);
            part[j] += Fb[j + 1] - lo;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_truth_units(TruthArgs a)
{
    __shared__ UnitSmem sm;
    if (!plan_ok(a) || a.wcnt[kCntStatus] != 0) return;
    const int64_t R = a.wcnt[kCntRuns];
    const int64_t U = R > 0 ? a.ucnt[R] : 0;
    const int tid = threadIdx.x, lane = tid & 31;
    const int M = a.c.mc_per_sample, nb = a.nb, L = a.nt;
    const float clip = a.c.diff_clip_sigma, fbpp = (float)a.bpp;
    const int npx = a.g.npx_x * a.g.npx_y;
    for (int64_t u = blockIdx.x; u < U; u += gridDim.x) {
        int lo = 0, hi = (int)R - 1;                      // run of unit u: last r with ucnt[r] <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.ucnt[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const int r = lo;
        const int local = (int)(u - a.ucnt[r]);
        const int ns_all = a.r_ns[r], nh_all = a.r_nh[r];
        const int nsc = (ns_all + kSegU - 1) / kSegU;
        const int hc = local / nsc, sc = local - hc * nsc;
        const int64_t h0 = a.r_h0[r];
        const int64_t hb = h0 + (int64_t)hc * kHC;
        const int nc = min(kHC, nh_all - hc * kHC);
        const int sb = sc * kSegU, ns = min(kSegU, ns_all - sb);
        const int eb = a.r_e0[r] + sb;
        const int32_t pid = a.hpix[h0];
        const int an = pid / npx;
        const int rem = pid - an * npx;
        const int iy = rem / a.g.npx_x, ix = rem - iy * a.g.npx_x;
        const int slot = an / a.g.n_anodes;
        const uint64_t key = slot_key(a.seed, a.ev, slot);
        const int64_t seg0 = slot_first(a.ev, slot);
        if (tid < kHC) {
            sm.klo[tid] = tid < nc ? interval_start(a, hb + tid, h0) - 1 : 0;
            sm.khi[tid] = tid < nc ? a.hta[hb + tid] : 0;
        }
        if (tid < 32) {
            int carry = 0;
            for (int i0 = 0; i0 < ns; i0 += 32) {
                const int i = i0 + lane;
                int v = 0;
                if (i < ns) {                                   // the points that can reach this pixel
                    const Anchor A = a.anch[a.segs[eb + i]];
                    int i_lo, i_hi;
                    point_range(A, M, (float)(ix - A.ix_ref) + 0.5f, (float)(iy - A.iy_ref) + 0.5f, fbpp, nb, clip,
                                i_lo, i_hi);
                    v = i_hi - i_lo;
                    sm.ilo[i] = i_lo;
                }
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (i < ns) sm.pre[i] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) sm.pre[ns] = carry;
        }
        for (int i = tid; i < kHC * kSegU; i += kThreads) sm.acc[i / kSegU][i % kSegU] = 0ull;
        __syncthreads();
        const int total = sm.pre[ns];
        // thread tid takes the contiguous points [fb, fe): few segment changes, partial sums in registers
        const int cs = (total + kThreads - 1) / kThreads;
        const int fb = min(total, tid * cs), fe = min(total, fb + cs);
        if (fb < fe) {
            int l2 = 0, h2 = ns - 1;                       // segment of point fb
            while (l2 < h2) {
                const int mid = (l2 + h2 + 1) >> 1;
                if (sm.pre[mid] <= fb) l2 = mid; else h2 = mid - 1;
            }
            int cur = l2;
            int next = sm.pre[cur + 1];
            int sg = a.segs[eb + cur];
            Anchor A = a.anch[sg];
            float cx = (float)(ix - A.ix_ref) + 0.5f, cy = (float)(iy - A.iy_ref) + 0.5f;
            float part[kHC];                               // FP32 partial sums of the current segment
#pragma unroll
            for (int j = 0; j < kHC; ++j) part[j] = 0.f;
            for (int f = fb; f < fe; ++f) {
                while (f >= next) {                        // next segment: flush the partial sums
#pragma unroll
                    for (int j = 0; j < kHC; ++j)
                        if (j < nc && part[j] != 0.f) {
                            atomicAdd(&sm.acc[j][cur], (unsigned long long)__double2ll_rn((double)part[j] * kFix));
                            part[j] = 0.f;
                        }
                    ++cur;
                    next = sm.pre[cur + 1];
                    sg = a.segs[eb + cur];
                    A = a.anch[sg];
                    cx = (float)(ix - A.ix_ref) + 0.5f;
                    cy = (float)(iy - A.iy_ref) + 0.5f;
                }
                const PointPos pp = point_position(A, sm.ilo[cur] + f - sm.pre[cur], M, key, (uint32_t)(sg - seg0),
                                                   clip, a.dp);
                Rec rc;
                if (!point_record(A, pp, cx, cy, fbpp, nb, a.c.nearest_lut, rc)) continue;
                const float4 *row = a.cum + (size_t)rc.b0 * a.ld;
                // F at the boundaries klo[0], khi[0], ..., khi[nc-1]: independent reads, issued together
                if (nc <= 4) record_hits<4>(rc, row, L, sm.klo, sm.khi, nc, part);
                else if (nc <= 8) record_hits<8>(rc, row, L, sm.klo, sm.khi, nc, part);
                else record_hits<16>(rc, row, L, sm.klo, sm.khi, nc, part);
            }
#pragma unroll
            for (int j = 0; j < kHC; ++j)
                if (j < nc && part[j] != 0.f)
                    atomicAdd(&sm.acc[j][cur], (unsigned long long)__double2ll_rn((double)part[j] * kFix));
        }
        __syncthreads();
        unsigned long long *dst = a.cells + a.ccnt[r];
        for (int i = tid; i < nc * ns; i += kThreads) {
            const int j = i / ns, t = i - j * ns;
            dst[(int64_t)(hc * kHC + j) * ns_all + sb + t] = sm.acc[j][t];
        }
        __syncthreads();
    }
}

// (|a|, segment a) ranks before (|b|, segment b): larger |charge| first, then lower index.
__device__ __forceinline__ bool ranks_before(long long qa, int sa, long long qb, int sb)
{
    const unsigned long long aa = (unsigned long long)(qa < 0 ? -qa : qa);
    const unsigned long long ab = (unsigned long long)(qb < 0 ? -qb : qb);
    return aa > ab || (aa == ab && sa < sb);
}

// One warp per hit: signal = sum of its row of cells, and the K best entries.
__global__ void __launch_bounds__(kThreads) k_truth_select(TruthArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t nh = hit_count(a);
    const bool ok = plan_ok(a) && a.wcnt[kCntStatus] == 0;
    const int K = a.K;
    for (int64_t h = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nh;
         h += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int r = a.rflag[h + 1] - 1;                 // run of hit h
        const int64_t h0 = a.r_h0[r];
        const int ns = ok ? a.r_ns[r] : 0;
        const unsigned long long *row = a.cells + (ok ? (int64_t)a.ccnt[r] + (h - h0) * ns : 0);
        long long ssum = 0;
        for (int i = lane; i < ns; i += 32) ssum += (long long)row[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        long long pq = 0;
        int ps = -1;
        for (int t = 0; t < K; ++t) {
            long long bq = 0;
            int bs = -1;
            for (int i = lane; i < ns; i += 32) {
                const long long q = (long long)row[i];
                const int sgi = a.segs[a.r_e0[r] + i];
                if (q == 0 || (ps >= 0 && !ranks_before(pq, ps, q, sgi))) continue;
                if (bs < 0 || ranks_before(q, sgi, bq, bs)) {
                    bq = q;
                    bs = sgi;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long q2 = __shfl_xor_sync(0xffffffffu, bq, o);
                const int s2 = __shfl_xor_sync(0xffffffffu, bs, o);
                if (s2 >= 0 && (bs < 0 || ranks_before(q2, s2, bq, bs))) {
                    bq = q2;
                    bs = s2;
                }
            }
            if (lane == 0) {
                a.oseg[h * K + t] = bs;
                a.oq[h * K + t] = bs >= 0 ? (float)((double)bq / kFix) : 0.f;
            }
            if (bs >= 0) {
                pq = bq;
                ps = bs;
            } else {
                ps = INT_MAX;                              // nothing left: remaining entries empty
                pq = 0;
            }
        }
        if (lane == 0) {
            a.osig[h] = ok ? (float)((double)ssum / kFix) : 0.f;
            if (a.ok0) a.ok0[h] = interval_start(a, h, h0);
        }
    }
}

// Running sums of the table rows, as quads: cum[b][j] = running sums at j of
// rows b, b + nb, b + 1, b + nb + 1 (the four corners of bin b; zero for rows
// beyond the table).  One warp per row: FP64 warp scan, FP32 out.
__global__ void k_cumulate(const float *lut, float4 *cum, int nb, int nt, int ld)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)nb * nb) return;
    const int bx = (int)(w / nb), by = (int)(w - (int64_t)bx * nb);
    const float *src[4];
    bool ok[4];
    for (int c = 0; c < 4; ++c) {
        const int dx = c & 1, dy = c >> 1;
        ok[c] = bx + dx < nb && by + dy < nb;
        src[c] = lut + (size_t)(ok[c] ? w + dx * nb + dy : w) * ld;
    }
    float4 *dst = cum + (size_t)w * ld;
    double carry[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j0 = 0; j0 < nt; j0 += 32) {
        const int j = j0 + lane;
        float out[4];
        for (int c = 0; c < 4; ++c) {
            double v = (j < nt && ok[c]) ? (double)__ldg(src[c] + j) : 0.0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = __dadd_rn(v, y);
            }
            v = __dadd_rn(v, carry[c]);
            out[c] = (float)v;
            carry[c] = __shfl_sync(0xffffffffu, v, 31);
        }
        if (j < nt) dst[j] = make_float4(out[0], out[1], out[2], out[3]);
    }
}

struct TruthLayout {
    size_t rflag, r_h0, r_nh, r_e0, r_ns, ucnt, ccnt, scan, cells, total;
};

TruthLayout truth_layout(int64_t hcap, int64_t max_cells)
{
    TruthLayout L;
    size_t o = 256;                                    // counts block
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    const size_t n1 = (size_t)hcap + 1;
    L.rflag = take(4 * n1);
    L.r_h0 = take(4 * n1);
    L.r_nh = take(4 * n1);
    L.r_e0 = take(4 * n1);
    L.r_ns = take(4 * n1);
    L.ucnt = take(4 * n1);
    L.ccnt = take(4 * n1);
    L.scan = take(scan_scratch_bytes((int64_t)n1));
    L.cells = take(8 * (size_t)max_cells);
    L.total = o;
    return L;
}

}  // namespace

size_t hit_truth_workspace_bytes(int64_t hit_cap, int64_t max_cells) { return truth_layout(hit_cap, max_cells).total; }

cudaError_t launch_response_cumulative(const sim_response &r, float *cum, cudaStream_t st)
{
    const int rows = r.nb * r.nb;
    const int threads = 256;
    const int blocks = (int)(((int64_t)rows * 32 + threads - 1) / threads);
    k_cumulate<<<blocks, threads, 0, st>>>(r.lut, reinterpret_cast<float4 *>(cum), r.nb, r.nt, r.ld);
    return cudaGetLastError();
}

cudaError_t launch_hit_truth(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                             const sim_response &r, const float *cum, const int32_t *active,
                             const int32_t *pix_seg_off, const int32_t *pix_seg_ids, const int64_t *counts,
                             int64_t pix_cap, const sim_hits &hits, const sim_truth &out, int64_t max_cells,
                             void *ws, cudaStream_t st)
{
    const int64_t hcap = hits.capacity < out.capacity ? hits.capacity : out.capacity;
    char *w = reinterpret_cast<char *>(ws);
    cudaError_t e = cudaMemsetAsync(w, 0, 256, st);
    if (e != cudaSuccess || hcap == 0) return e;
    const TruthLayout Lw = truth_layout(hcap, max_cells);
    TruthArgs a;
    a.c = c;
    a.anch = reinterpret_cast<const Anchor *>(d.anchors);
    a.cum = reinterpret_cast<const float4 *>(cum);
    a.nb = r.nb;
    a.nt = r.nt;
    a.ld = r.ld;
    a.bpp = r.bins_per_pitch;
    a.active = active;
    a.off = pix_seg_off;
    a.segs = pix_seg_ids;
    a.counts = counts;
    a.pix_cap = pix_cap;
    a.hpix = hits.pixel;
    a.hta = hits.t_adc;
    a.htc = hits.t_cross;
    a.n_hits = hits.n_out;
    a.hcap = hcap;
    a.K = out.k;
    a.oseg = out.segment;
    a.oq = out.q;
    a.osig = out.q_signal;
    a.ok0 = out.tick_first;
    a.seed = c.seed;
    a.ev = events_of(s);
    a.g = geo_of(c);
    a.dp = drift_par_of(c);
    a.wcnt = reinterpret_cast<int64_t *>(w);
    a.max_cells = max_cells;
    a.rflag = reinterpret_cast<int32_t *>(w + Lw.rflag);
    a.r_h0 = reinterpret_cast<int32_t *>(w + Lw.r_h0);
    a.r_nh = reinterpret_cast<int32_t *>(w + Lw.r_nh);
    a.r_e0 = reinterpret_cast<int32_t *>(w + Lw.r_e0);
    a.r_ns = reinterpret_cast<int32_t *>(w + Lw.r_ns);
    a.ucnt = reinterpret_cast<int32_t *>(w + Lw.ucnt);
    a.ccnt = reinterpret_cast<int32_t *>(w + Lw.ccnt);
    a.cells = reinterpret_cast<unsigned long long *>(w + Lw.cells);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n1 = hcap + 1;
    const int tb = 256;
    const int gb = (int)((n1 + tb - 1) / tb);
    // per-run arrays are read up to the run count only; zero the count arrays' tails for the scans
    e = cudaMemsetAsync(a.ucnt, 0, 4 * (size_t)n1, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.ccnt, 0, 4 * (size_t)n1, st);
    if (e != cudaSuccess) return e;
    k_run_flags<<<gb, tb, 0, st>>>(a);
    e = launch_exclusive_scan(a.rflag, a.rflag, n1 - 1, a.wcnt + kCntRuns, w + Lw.scan, st);
    if (e != cudaSuccess) return e;
    k_run_fill<<<gb, tb, 0, st>>>(a);
    e = launch_exclusive_scan(a.ucnt, a.ucnt, n1 - 1, a.wcnt + kCntUnits, w + Lw.scan, st);
    if (e == cudaSuccess) e = launch_exclusive_scan(a.ccnt, a.ccnt, n1 - 1, a.wcnt + kCntScan, w + Lw.scan, st);
    if (e != cudaSuccess) return e;
    k_plan_check<<<1, 1, 0, st>>>(a);
    k_truth_units<<<sms * 4, kThreads, 0, st>>>(a);
    const int64_t sel_blocks = (hcap * 32 + kThreads - 1) / kThreads;
    k_truth_select<<<(int)(sel_blocks < sms * 16 ? sel_blocks : sms * 16), kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace larsim
