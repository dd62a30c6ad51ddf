// induced_current.cu -- step 4 of the charge path (arXiv:2212.09807
// Sec. 3.3.2), FP32 form on the CUDA cores: the current induced on each
// active pixel in each tick,
//   I[p, k] = sum_s sum_mu sum_nu q_s Rt(x_mu + dx - x_p, y_mu + dy - y_p, k - a),
// Eq. (current) with the charge density rho of N points x M perturbations
// per segment, summed over the segments mapped to the pixel (the per-pixel
// sum of Sec. 3.4).  Each term reads the table bilinearly at the folded
// offset (four table nodes around the point's bin) and linearly at the
// fractional arrival tick: a point record (arrival A + f, bin b0, q-scaled
// corner weights w_c; current_records.cuh) deposits the charge (1 - f) w_c at
// tick A and f w_c at tick A + 1 of node b0 + c.  With Q[p, n, a] the charge
// so binned per (pixel, node, arrival tick),
//   I[p, k] = sum_n sum_a Q[p, n, a] R[n, k - a + L - 1]
// -- the same terms regrouped per node: a pixel's records fall on ~1200 of
// the 2025 nodes, ~4.5 nonzero cells per 16-tick block of a node, so
// collecting the charge first costs one FMA per nonzero cell and table tick
// instead of eight per record and tick.
//
// Design: one CTA of 128 threads per active pixel (dynamic queue, pixels of
// the most candidate points first; four CTAs per SM), output stationary:
// thread t holds 16 consecutive ticks of a 2032-tick pass in registers.
//  1. records: the pixel's segments are taken 128 at a time (one thread
//     loads each anchor) and their candidate points walked 128 per step
//     (Philox keyed by segment and point); those within the table's reach of
//     the pixel become records in a per-CTA scratch buffer, with a bin
//     histogram in shared memory; a chunk holds at most kRecCap records;
//  2. the chunk is scattered into bin order and the table nodes its bins
//     reach are listed;
//  3. node loop, pipelined over two barriers per node: the charge of node
//     n + 1 is deposited into fixed-point cells (integer shared-memory
//     atomics: order-independent, so the result is bitwise reproducible; the
//     scale, a power of two, follows the chunk's largest node entry count and
//     largest weight, so that taps round to ~1e-9 of a node's charge) and its
//     table row copied in (cp.async), while node n is applied: for each
//     present 16-tick arrival block every thread loads the 31 table values its
//     16 ticks need (eight 16-byte shared reads from the row's XOR-swizzled
//     chunks, conflict-free across consecutive threads' windows) and adds
//     q_d R[.] for each nonzero cell d (a CTA-uniform branch), two ticks per
//     paired FMA instruction (fma.rn.f32x2).
// Per tick the terms are summed in a fixed order (chunks in point order,
// nodes increasing, blocks increasing, cells increasing) in FP32, and every
// kKahanNodes nodes the partial sums are added into compensated (Kahan)
// totals in registers: a dense pixel sums ~3e5 cells per tick, whose plain
// FP32 sum would drift by ~1e-5 of its value.  A pixel's current depends on
// its own segments only: the same bits alone, in a batch or in any range of
// a call.
#include <algorithm>

#include "current_records.cuh"

namespace larsim {

namespace {
constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kTPT = 16;                        // consecutive ticks per thread
constexpr int kSpan = kThreads * kTPT;          // ticks the threads hold
constexpr int kPass = kSpan - kTPT;             // ticks per pass (see tick_shift)
constexpr int kBlk = 16;                        // arrival ticks per block
constexpr int kBlocks = 256;                    // blocks of a pass: relative arrival ticks [0, 4096)
constexpr int kRecCap = 65520;                  // records per chunk at most (per-CTA scratch; ~1 chunk per pixel;
                                                // bin ends fit 16 bits)
constexpr int kMaxBins = 2048;                  // nb * nb <= kMaxBins
constexpr int kMaxRow = 2048;                   // table length nt <= kMaxRow
constexpr int kSegBatch = 128;                  // segments loaded together by the generation
constexpr int kKahanNodes = 8;                  // nodes per plain FP32 partial sum
constexpr int kMaxNb = 45;                      // nb <= 45 (nb * nb <= kMaxBins)
constexpr int kNodeWords = (kMaxNb << 6) / 32;  // bit (nx << 6) | ny per node
// Staged table row: value j at position p = j + kEdge, in 16-byte chunk
// c = p / 4 stored at chunk c ^ ((c / 8) mod 4) (an XOR swizzle within each
// group of 8 chunks: the 16-byte window reads of 8 consecutive threads, whose
// windows are 4 chunks apart, span 4 or 5 groups and fall on 8 different bank
// groups for every start and offset; XOR by (c / 8) mod 8 would pair groups 4
// apart and cost 1.5 wavefronts per read).  Thread t holds the
// pass ticks 16 t - sigma + i (i < 16), sigma = L mod 16, so that its
// 32-value window of block bl starts at j0 = 16 (t - bl) + L - 16 - sigma, a
// multiple of 16; windows that touch the row have j0 in [-30, L - 1], so
// positions [2, L + kEdge + 31) are read; those outside [kEdge, kEdge + L)
// hold zero.  The threads hold ticks [-sigma, kSpan - sigma) of the pass:
// a pass writes its first kPass ticks.
constexpr int kEdge = 32;
constexpr int kRowPos = kMaxRow + kEdge + 48;
constexpr int kRowWords = ((kRowPos / 4 + 7) / 8) * 32;

__device__ __forceinline__ int row_chunk(int c) { return c ^ ((c >> 3) & 3); }
__host__ __device__ constexpr int tick_shift(int L) { return L & 15; }

struct CurArgs {
    sim_config c;
    const float *lut;
    int nb, nt, ld, bpp;
    const Anchor *anch;
    const int32_t *active, *off, *segs;
    const int64_t *counts;
    int64_t pix_cap, pix_begin, pix_end;        // active pixels [pix_begin, min(counts[1], pix_end))
    float *current;
    uint64_t seed;
    EventInfo ev;
    Geo g;
    DriftPar dp;
    int *queue;                                 // next entry of `order`
    const int32_t *order;                       // pixel (relative to pix_begin) of each queue entry
    Rec *recs;                                  // [grid][kRecCap], point order
    Rec *sorted;                                // [grid][kRecCap], bin order
    unsigned long long *n_cells;                // counts[5]: nonzero charge cells (statistics)
    int rec_cap;                                // records per chunk (<= kRecCap)
};

struct __align__(16) Smem {
    float row[2][kRowWords];                    // staged table rows of two nodes
    union {
        int cell[2][kBlocks * kBlk];            // fixed-point charge cells of two nodes [block][tick]
        struct {
            Anchor anc[kSegBatch];              // a batch of the pixel's segments
            int sg[kSegBatch];
            int coff[kSegBatch + 1];            // candidate offsets of the batch
            int hist[kMaxBins + 1];             // bin counts, then scatter cursors
        } g;
    } u;
    unsigned short bend[kMaxBins];              // end of each bin in bin order (the node loop's lists)
    uint32_t nfl[kNodeWords];                   // nodes reached: bit (nx << 6) | ny
    uint32_t mask[3][kBlocks / 32];             // arrival blocks present, per node (three in flight)
    int scan_tmp[kWarps + 1];
    int warp_n[kWarps];
    int n_nodes;
    int item;
    int wmax;                                   // largest record weight of the chunk (FP32 bits)
    int emax;
};

static_assert(sizeof(Smem) + 1024 <= 233472 / 4, "four CTAs per SM");

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

// tot += x with compensation c (Kahan): tot - c is the running sum to a few
// FP32 roundings of the final value, however many partial sums are added.
__device__ __forceinline__ void kahan_add(float &tot, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(tot, y);
    c = __fsub_rn(__fsub_rn(t, tot), y);
    tot = t;
}

// Generation cursor of a pixel's records: next segment batch and the
// candidate offset within it where the previous chunk stopped.
struct GenState {
    int e;
    int c0;
};

// Records of the pixel (centre (ix, iy)) from its segments [st.e, e1), in
// point order, into recs, with the bin histogram in s->u.g.hist.  Stops when
// the next step of 128 candidates would overflow the chunk (st keeps the
// place) or after the last segment (st.e = e1).  Returns the records.
__device__ int gen_chunk(const CurArgs &a, Smem *s, GenState &st, int e1, int ix, int iy, uint64_t key,
                         int64_t seg0, Rec *recs)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = a.c.mc_per_sample;
    const float clip = a.c.diff_clip_sigma, fbpp = (float)a.bpp;
    int nrec = 0;
    while (st.e < e1) {
        const int nbat = min(kSegBatch, e1 - st.e);
        int cnt = 0;
        if (tid < nbat) {
            const int sg = a.segs[st.e + tid];
            const Anchor A = a.anch[sg];
            s->u.g.anc[tid] = A;
            s->u.g.sg[tid] = sg;
            cnt = A.N * M;
        }
        int C;
        const int pre = block_scan(cnt, s, &C);
        if (tid < nbat) s->u.g.coff[tid] = pre;
        if (tid == 0) s->u.g.coff[nbat] = C;
        __syncthreads();
        for (int c = st.c0; c < C; c += kThreads) {
            const int cc = c + tid;
            bool ok = false;
            Rec r;
            if (cc < C) {
                int lo = 0;                                  // last j with coff[j] <= cc
#pragma unroll
                for (int step = kSegBatch / 2; step > 0; step >>= 1)
                    if (lo + step < nbat && s->u.g.coff[lo + step] <= cc) lo += step;
                const Anchor &A = s->u.g.anc[lo];
                const float cx = (float)(ix - A.ix_ref) + 0.5f, cy = (float)(iy - A.iy_ref) + 0.5f;
                const PointPos pp = point_position(A, cc - s->u.g.coff[lo], M, key,
                                                   (uint32_t)(s->u.g.sg[lo] - seg0), clip, a.dp);
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
            if (nrec + nq > a.rec_cap) {         // chunk full: process it, then redo this step
                st.c0 = c;
                __syncthreads();
                return nrec;
            }
            if (ok) {
                recs[nrec + wb + __popc(m & ((1u << lane) - 1u))] = r;
                atomicAdd(&s->u.g.hist[r.b0], 1);
            }
            // weights are >= 0: their FP32 bits order as integers
            const int wb_max = __reduce_max_sync(
                0xffffffffu, ok ? __float_as_int(fmaxf(fmaxf(r.w.x, r.w.y), fmaxf(r.w.z, r.w.w))) : 0);
            if (lane == 0 && wb_max > 0) atomicMax(&s->wmax, wb_max);
            nrec += nq;
            __syncthreads();                     // warp_n reused by the next step
        }
        st.e += nbat;
        st.c0 = 0;
        __syncthreads();                         // the batch area is reloaded
    }
    return nrec;
}

// Thread t's share of a table row, copied asynchronously (cp.async, 16 bytes
// each: elements 4 t + 512 i, i < 4) into the staged layout; elements at or
// beyond L are zero-filled.  Rows are 16-byte aligned, and four values at
// p = 0 (mod 4) form one chunk.
__device__ __forceinline__ void stage_row(float *dst, const CurArgs &a, int nxy)
{
    const float *row = a.lut + (size_t)((nxy >> 6) * a.nb + (nxy & 63)) * a.ld;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int j = 4 * threadIdx.x + 512 * i;
        const int bytes = j < a.nt ? 4 * min(4, a.nt - j) : 0;
        const float *src = row + (j < a.nt ? j : 0);
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + 4 * row_chunk((j + kEdge) >> 2));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The four record lists of node n = (nx << 6) | ny (corner c of the bins
// (nx - (c & 1), ny - (c >> 1))) in bin order: begin of each and prefix counts.
struct NodeLists {
    int beg[4];
    int pre[5];
};

__device__ __forceinline__ NodeLists node_lists(const Smem *s, int n, int nb)
{
    NodeLists L;
    const int nx = n >> 6, ny = n & 63;
    L.pre[0] = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int bx = nx - (c & 1), by = ny - (c >> 1);
        int b = 0, e = 0;
        if (bx >= 0 && by >= 0) {
            const int bin = bx * nb + by;
            b = bin > 0 ? s->bend[bin - 1] : 0;
            e = s->bend[bin];
        }
        L.beg[c] = b;
        L.pre[c + 1] = L.pre[c] + (e - b);
    }
    return L;
}

// Record and corner of entry e of a node's concatenated lists.
__device__ __forceinline__ void node_entry(const NodeLists &L, const Rec *sorted, int e, Rec &r, int &c)
{
    c = (e >= L.pre[1]) + (e >= L.pre[2]) + (e >= L.pre[3]);
    // selects, not a runtime index (which would place the lists in local memory)
    const int b = c == 0 ? L.beg[0] : c == 1 ? L.beg[1] : c == 2 ? L.beg[2] : L.beg[3];
    const int p = c == 0 ? L.pre[0] : c == 1 ? L.pre[1] : c == 2 ? L.pre[2] : L.pre[3];
    r = sorted[b + (e - p)];
}

// Fixed-point scale of a node's charge cells: 2^k with k the largest keeping
// n_entries x wmax (a bound of every cell: each entry adds at most one tap of
// at most wmax to a cell) below 2^30, so no cell overflows and a tap is
// rounded to ~n_entries wmax 2^-30.  A power of two: converting back is exact.
// Deterministic: a count and a maximum.
__device__ __forceinline__ float node_scale(int n_entries, float wmax)
{
    const float x = (float)n_entries * wmax;
    if (!(x > 0.f)) return 1.f;
    const int ex = ((__float_as_int(x) >> 23) & 0xff) - 127;      // floor(log2 x) (x normal)
    const int k = min(100, max(-100, 29 - ex));
    return __int_as_float((k + 127) << 23);
}

// The first node after `after` in the bit set (-1: none); uniform across the CTA.
__device__ __forceinline__ int next_node(const uint32_t *nfl, int after)
{
    const int x = after + 1;
    int w = x >> 5;
    if (w >= kNodeWords) return -1;
    uint32_t m = nfl[w] & (0xffffffffu << (x & 31));
    while (m == 0u) {
        if (++w >= kNodeWords) return -1;
        m = nfl[w];
    }
    return (w << 5) + __ffs(m) - 1;
}

// Deposits the two ticks of a record's corner c into the fixed-point cells;
// n_cells counts the cells it makes nonzero (all deposits are >= 0).
__device__ __forceinline__ void deposit(int *cell, uint32_t *mask, const Rec &r, int c, int k0, float scale,
                                        unsigned &n_cells)
{
    const float w = c == 0 ? r.w.x : c == 1 ? r.w.y : c == 2 ? r.w.z : r.w.w;
    uint32_t bits[2] = {0u, 0u};
    int word[2] = {0, 0};
#pragma unroll
    for (int tap = 0; tap < 2; ++tap) {
        const float val = tap ? r.f * w : (1.f - r.f) * w;
        const int rel = r.A - k0 + tap;
        if (val == 0.f || rel < 0 || rel >= kBlocks * kBlk) continue;
        const int add = __float2int_rn(val * scale);
        if (add == 0) continue;
        n_cells += atomicAdd(cell + rel, add) == 0;
        word[tap] = rel >> 9;
        bits[tap] = 1u << ((rel >> 4) & 31);
    }
    if (bits[0] && bits[1] && word[0] == word[1]) {
        atomicOr(mask + word[0], bits[0] | bits[1]);
    } else {
        if (bits[0]) atomicOr(mask + word[0], bits[0]);
        if (bits[1]) atomicOr(mask + word[1], bits[1]);
    }
}

// Node applied to a thread's 16 ticks: for each present block bl, the table
// window W[m] = R[j0 + m] (m < 32, j0 = 16 (t - bl) + L - 16 - sigma) and the
// block's cells q_d: the thread's tick i gains q_d R[j0 + i - d + 15] =
// q_d W[i - d + 15] (zero cells skipped: a CTA-uniform branch).  The cells
// are in fixed point (x the chunk's scale).
// The thread's 16 accumulators as packed pairs for the paired FP32 FMA
// (fma.rn.f32x2, two lanes of independent round-to-nearest FMAs): cells with
// odd d meet even-aligned pairs of the window, (W[m], W[m+1]) with m even, on
// the tick pairs (2k, 2k+1) (ev); cells with even d meet them on the tick
// pairs (2k+1, 2k+2) (od, k < 7; ticks 0 and 15 by single FMAs into ev).
// Tick i is ev[i] + od[i] (od holding ticks 1..14).
struct Acc {
    float2 ev[8];
    float2 od[7];
};

template <int D>
__device__ __forceinline__ void fma_cell(float qf, const float2 (&Wp)[16], Acc &acc)
{
    const float2 q2 = make_float2(qf, qf);
    if (D & 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc.ev[k] = __ffma2_rn(q2, Wp[(2 * k - D + 15) >> 1], acc.ev[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 7; ++k) acc.od[k] = __ffma2_rn(q2, Wp[(2 * k + 16 - D) >> 1], acc.od[k]);
        acc.ev[0].x = fmaf(qf, Wp[(15 - D) >> 1].y, acc.ev[0].x);        // tick 0: W[15 - D] (odd)
        acc.ev[7].y = fmaf(qf, Wp[(30 - D) >> 1].x, acc.ev[7].y);        // tick 15: W[30 - D] (even)
    }
}

__device__ __forceinline__ void apply_node(const float *row, const int *cf, const uint32_t *mask, int L, int sig,
                                           int t, bool live, Acc &acc)
{
#pragma unroll 1
    for (int w = 0; w < kBlocks / 32; ++w) {
        uint32_t m = mask[w];
        while (m) {
            const int bl = 32 * w + __ffs(m) - 1;
            m &= m - 1;
            const int j0 = kTPT * (t - bl) + L - kTPT - sig;
            if (!live || j0 < -30 || j0 > L - 1) continue;      // the window misses the row
            const int c0 = (j0 + kEdge) >> 2;                   // j0 + kEdge = 0 (mod 16)
            float2 Wp[16];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 v = *reinterpret_cast<const float4 *>(row + 4 * row_chunk(c0 + k));
                Wp[2 * k] = make_float2(v.x, v.y);
                Wp[2 * k + 1] = make_float2(v.z, v.w);
            }
            int q[kBlk];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int4 v = reinterpret_cast<const int4 *>(cf + bl * kBlk)[k];
                q[4 * k] = v.x;
                q[4 * k + 1] = v.y;
                q[4 * k + 2] = v.z;
                q[4 * k + 3] = v.w;
            }
#define LARSIM_CELL(D) \
    if (q[D] != 0) fma_cell<D>((float)q[D], Wp, acc);
            LARSIM_CELL(0) LARSIM_CELL(1) LARSIM_CELL(2) LARSIM_CELL(3) LARSIM_CELL(4) LARSIM_CELL(5)
            LARSIM_CELL(6) LARSIM_CELL(7) LARSIM_CELL(8) LARSIM_CELL(9) LARSIM_CELL(10) LARSIM_CELL(11)
            LARSIM_CELL(12) LARSIM_CELL(13) LARSIM_CELL(14) LARSIM_CELL(15)
#undef LARSIM_CELL
        }
    }
}

__global__ void __launch_bounds__(kThreads, 4) k_induced_current(CurArgs a, int64_t n_items_cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem *s = reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const bool go = a.counts[3] == 0 && a.counts[1] <= a.pix_cap;
    const int64_t npix = go ? min(a.counts[1], a.pix_end) : 0;
    const int64_t n_items = min(n_items_cap, max((int64_t)0, npix - a.pix_begin));
    const int T = a.c.n_ticks, L = a.nt, nb = a.nb, nb2 = nb * nb;
    const int sig = tick_shift(L);
    const int npx = a.g.npx_x * a.g.npx_y;
    Rec *recs = a.recs + (size_t)blockIdx.x * kRecCap;
    Rec *sorted = a.sorted + (size_t)blockIdx.x * kRecCap;
    for (int i = tid; i < 2 * kRowWords; i += kThreads) (&s->row[0][0])[i] = 0.f;
    unsigned n_cells = 0;                       // nonzero charge cells made by this thread

    for (;;) {
        __syncthreads();
        if (tid == 0) s->item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int64_t it = s->item;
        if (it >= n_items) break;      // (uniform)
        const int64_t pi = a.pix_begin + a.order[it];
        const int32_t pid = a.active[pi];
        const int an = pid / npx, rem = pid - an * npx;
        const int iy = rem / a.g.npx_x, ix = rem - iy * a.g.npx_x;
        const int slot = an / a.g.n_anodes;            // event of this (virtual) pixel
        const uint64_t key = slot_key(a.seed, a.ev, slot);
        const int64_t seg0 = slot_first(a.ev, slot);
        const int e0 = a.off[pi], e1 = a.off[pi + 1];
        float *out = a.current + (size_t)pi * T;
        for (int k0 = 0; k0 < T; k0 += kPass) {
            // tick chunk of this thread: the warps take the four quarters of the pass in an order
            // rotated per pixel.  The early quarters do the most work (a block reaches the ticks
            // before its arrival), and warp w of every CTA runs on scheduler w: rotating spreads
            // the heavy quarters of the CTAs sharing an SM over its schedulers.
            const int tq = ((((tid >> 5) + (int)(it & 3)) & 3) << 5) | (tid & 31);
            const int t_lo = kTPT * tq - sig;                       // my first tick of the pass
            const bool live = t_lo + kTPT > 0 && t_lo < kPass && k0 + t_lo < T;
            Acc acc;
            float tot[kTPT], cmp[kTPT];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc.ev[k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 7; ++k) acc.od[k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < kTPT; ++i) tot[i] = cmp[i] = 0.f;
            GenState st{e0, 0};
            while (st.e < e1) {
                // ---- 1. records of this chunk ------------------------------------------
                for (int b = tid; b <= nb2; b += kThreads) s->u.g.hist[b] = 0;
                if (tid < kNodeWords) s->nfl[tid] = 0u;
                if (tid == 0) s->wmax = 0, s->emax = 0;
                __syncthreads();
                const int nrec = gen_chunk(a, s, st, e1, ix, iy, key, seg0, recs);
                if (nrec == 0) continue;
                // ---- 2. bin order, nodes reached -----------------------------------------
                {
                    constexpr int kB = kMaxBins / kThreads;
                    int v[kB], sv = 0;
#pragma unroll
                    for (int i = 0; i < kB; ++i) {
                        const int b = tid * kB + i;
                        v[i] = b < nb2 ? s->u.g.hist[b] : 0;
                        sv += v[i];
                    }
                    int tv;
                    int pv = block_scan(sv, s, &tv);
#pragma unroll
                    for (int i = 0; i < kB; ++i) {
                        const int b = tid * kB + i;
                        if (b < nb2) {
                            s->u.g.hist[b] = pv;              // scatter cursor, then the end of bin b
                            if (v[i] > 0) {                   // the bin's corner nodes inside the table
                                const int bx = b / nb, by = b - bx * nb, id = (bx << 6) | by;
                                atomicOr(&s->nfl[id >> 5], 1u << (id & 31));
                                if (bx + 1 < nb) atomicOr(&s->nfl[(id + 64) >> 5], 1u << ((id + 64) & 31));
                                if (by + 1 < nb) atomicOr(&s->nfl[(id + 1) >> 5], 1u << ((id + 1) & 31));
                                if (bx + 1 < nb && by + 1 < nb)
                                    atomicOr(&s->nfl[(id + 65) >> 5], 1u << ((id + 65) & 31));
                            }
                        }
                        pv += v[i];
                    }
                }
                __syncthreads();
                for (int i = tid; i < nrec; i += kThreads) {
                    const Rec r = recs[i];
                    sorted[atomicAdd(&s->u.g.hist[r.b0], 1)] = r;
                }
                __syncthreads();
                for (int b = tid; b < nb2; b += kThreads) s->bend[b] = (unsigned short)s->u.g.hist[b];
                {
                    const int cnt = tid < kNodeWords ? __popc(s->nfl[tid]) : 0;
                    int tf;
                    block_scan(cnt, s, &tf);                    // (its barriers also publish bend)
                    if (tid == 0) s->n_nodes = tf;
                }
                {   // largest node entry count (a deterministic bound of the cells with the chunk's weights)
                    int em = 0;
                    for (int i = tid; i < kNodeWords * 32; i += kThreads)
                        if ((s->nfl[i >> 5] >> (i & 31)) & 1u) em = max(em, node_lists(s, i, nb).pre[4]);
                    em = __reduce_max_sync(0xffffffffu, em);
                    if ((tid & 31) == 0) atomicMax(&s->emax, em);
                }
                __syncthreads();                                // the union becomes the cell buffers
                for (int i = tid; i < 2 * kBlocks * kBlk / 4; i += kThreads)
                    reinterpret_cast<int4 *>(&s->u.cell[0][0])[i] = make_int4(0, 0, 0, 0);
                if (tid < 3 * (kBlocks / 32)) (&s->mask[0][0])[tid] = 0u;
                __syncthreads();
                // ---- 3. node loop ----------------------------------------------------------
                const int nn = s->n_nodes;
                int n_cur = next_node(s->nfl, -1);
                stage_row(s->row[0], a, n_cur);
                const float sc_next = node_scale(s->emax, __int_as_float(s->wmax));   // of the whole chunk
                const float inv_sc = 1.f / sc_next;
                {
                    const NodeLists nl = node_lists(s, n_cur, nb);
                    for (int e = tid; e < nl.pre[4]; e += kThreads) {
                        Rec r;
                        int c;
                        node_entry(nl, sorted, e, r, c);
                        deposit(s->u.cell[0], s->mask[0], r, c, k0, sc_next, n_cells);
                    }
                }
                stage_wait();
                __syncthreads();
                for (int u = 0; u < nn; ++u) {
                    const int x = u & 1;
                    const bool nxt = u + 1 < nn;
                    const int n_nxt = nxt ? next_node(s->nfl, n_cur) : -1;
                    if (nxt) stage_row(s->row[x ^ 1], a, n_nxt);   // lands before the next apply
                    NodeLists nl;
                    Rec r0;
                    int c0 = 0;
                    bool h0 = false;
                    if (nxt) {                                  // first entry of node u + 1 in flight
                        nl = node_lists(s, n_nxt, nb);
                        h0 = tid < nl.pre[4];
                        if (h0) node_entry(nl, sorted, tid, r0, c0);
                    }
                    apply_node(s->row[x], s->u.cell[x], s->mask[u % 3], L, sig, tq, live, acc);
                    if (u % kKahanNodes == kKahanNodes - 1 || u == nn - 1) {
#pragma unroll
                        for (int i = 0; i < kTPT; ++i) {
                            float v = (i & 1) ? acc.ev[i >> 1].y : acc.ev[i >> 1].x;
                            if (i >= 1 && i <= 14) v = __fadd_rn(v, (i & 1) ? acc.od[i >> 1].x : acc.od[(i >> 1) - 1].y);
                            kahan_add(tot[i], cmp[i], v * inv_sc);
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k) acc.ev[k] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < 7; ++k) acc.od[k] = make_float2(0.f, 0.f);
                    }
                    if (nxt) {
                        int *cell = s->u.cell[x ^ 1];
                        uint32_t *mk = s->mask[(u + 1) % 3];
                        if (h0) deposit(cell, mk, r0, c0, k0, sc_next, n_cells);
                        for (int e = tid + kThreads; e < nl.pre[4]; e += kThreads) {
                            Rec r;
                            int c;
                            node_entry(nl, sorted, e, r, c);
                            deposit(cell, mk, r, c, k0, sc_next, n_cells);
                        }
                    }
                    if (tid < kBlocks / 32) s->mask[(u + 2) % 3][tid] = 0u;   // node u - 1's, free since
                    stage_wait();
                    __syncthreads();
                    // node u's cells cleared for node u + 2 (the whole buffer: fewer steps than walking its blocks)
                    for (int i = tid; i < kBlocks * kBlk / 4; i += kThreads)
                        reinterpret_cast<int4 *>(s->u.cell[x])[i] = make_int4(0, 0, 0, 0);
                    __syncthreads();
                    n_cur = n_nxt;
                }
            }
            // compensated totals (zero for a pixel without records)
#pragma unroll
            for (int i = 0; i < kTPT; ++i) {
                const int k = t_lo + i;
                if (k >= 0 && k < kPass && k0 + k < T) out[k0 + k] = __fsub_rn(tot[i], cmp[i]);
            }
        }
    }
    // nonzero charge cells of the call (counts[5], as the tensor-core form reports them)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_cells += __shfl_down_sync(0xffffffffu, n_cells, o);
    if ((tid & 31) == 0 && n_cells) atomicAdd(a.n_cells, (unsigned long long)n_cells);
}

// ---------------------------------------------------------- queue order ----
// Pixels ordered by decreasing work (their candidate points sum_{s -> p} N_s
// M, in 32 classes of floor(log2)), so that the heavy ones start first and the
// tail of the queue is short work.  The order within a class is immaterial:
// each pixel is computed alone.
__global__ void k_fp_classify(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end,
                              const int32_t *off, const int32_t *segs, const int32_t *n_samples, int M,
                              int32_t *cls, int32_t *ccount)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (counts[3] != 0 || counts[1] > pix_cap) return;
    const int64_t n = min(counts[1], end) - begin;
    if (j >= n) return;
    const int64_t pi = begin + j;
    long long w = 1;
    for (int e = off[pi]; e < off[pi + 1]; ++e) w += (long long)n_samples[segs[e]] * M;
    const int c = min(31, 63 - __clzll(w));
    cls[j] = c;
    atomicAdd(&ccount[c], 1);
}

__global__ void k_fp_order(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end, const int32_t *cls,
                           const int32_t *ccount, int32_t *cursor, int32_t *order)
{
    __shared__ int start[32];
    if (threadIdx.x < 32) {
        int s0 = 0;
        for (int c = 31; c > threadIdx.x; --c) s0 += ccount[c];     // heavier classes first
        start[threadIdx.x] = s0;
    }
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (counts[3] != 0 || counts[1] > pix_cap) return;
    const int64_t n = min(counts[1], end) - begin;
    if (j >= n) return;
    const int c = cls[j];
    order[start[c] + atomicAdd(&cursor[c], 1)] = (int32_t)j;
}

int grid_for(int64_t pix_cap, int ctas_per_sm = 4)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (int64_t)sms * ctas_per_sm;
    if (g > pix_cap) g = pix_cap;
    return (int)(g < 1 ? 1 : g);
}

struct FpLayout {
    size_t queue, cls, order, recs, sorted, total;
};

FpLayout fp_layout(int grid, int64_t pix_cap)
{
    FpLayout t;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += align256(b);
        return at;
    };
    t.queue = take(512);                        // [0] queue, [64] class counts, [256] class cursors
    t.cls = take(sizeof(int32_t) * (size_t)pix_cap);
    t.order = take(sizeof(int32_t) * (size_t)pix_cap);
    t.recs = take((size_t)grid * kRecCap * sizeof(Rec));
    t.sorted = take((size_t)grid * kRecCap * sizeof(Rec));
    t.total = o;
    return t;
}
}  // namespace

size_t current_scratch_bytes(int64_t pix_cap)
{
    const int64_t p = pix_cap > 0 ? pix_cap : 1;
    return fp_layout(grid_for(p), p).total;
}

bool current_table_ok(int nb, int nt) { return nb * nb <= kMaxBins && nt <= kMaxRow; }

cudaError_t launch_induced_current(const sim_config &c, const sim_segments &s, const sim_drifted &d,
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
    // the scratch is sized for the default grid: a smaller configured one fits it
    const int grid = grid_for(pix_cap, c.direct_ctas_per_sm > 0 ? c.direct_ctas_per_sm : 4);
    const FpLayout lay = fp_layout(grid_for(pix_cap), pix_cap);
    char *p = reinterpret_cast<char *>(scratch);
    a.queue = reinterpret_cast<int *>(p + lay.queue);
    int32_t *ccount = reinterpret_cast<int32_t *>(p + lay.queue + 64);
    int32_t *cursor = reinterpret_cast<int32_t *>(p + lay.queue + 256);
    int32_t *cls = reinterpret_cast<int32_t *>(p + lay.cls);
    int32_t *order = reinterpret_cast<int32_t *>(p + lay.order);
    a.order = order;
    a.recs = reinterpret_cast<Rec *>(p + lay.recs);
    a.sorted = reinterpret_cast<Rec *>(p + lay.sorted);
    a.n_cells = reinterpret_cast<unsigned long long *>(const_cast<int64_t *>(counts) + 5);
    a.rec_cap = c.tc_record_chunk > 0 ? std::min(c.tc_record_chunk, kRecCap) : kRecCap;
    cudaError_t e = cudaMemsetAsync(p + lay.queue, 0, 512, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(const_cast<int64_t *>(counts) + 4, 0, 2 * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    const int64_t n_cap = pix_cap - (pix_begin < pix_cap ? pix_begin : pix_cap);    // pixels the range can hold
    if (n_cap <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_cap + 255) / 256);
    k_fp_classify<<<blocks, 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, pix_seg_off, pix_seg_ids,
                                          d.n_samples, c.mc_per_sample, cls, ccount);
    k_fp_order<<<blocks, 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, cls, ccount, cursor, order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(Smem);
    e = cudaFuncSetAttribute(k_induced_current, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_induced_current<<<grid, kThreads, smem, st>>>(a, n_cap);
    return cudaGetLastError();
}

}  // namespace larsim
