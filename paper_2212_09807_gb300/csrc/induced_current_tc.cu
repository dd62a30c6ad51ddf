// induced_current_tc.cu -- step 4 of the charge path (arXiv:2212.09807
// Sec. 3.3.2, Eq. (current)) as a tensor-core contraction on sm_103a:
// tcgen05 MMAs with FP16 or BF16 operands and FP32 accumulators in tensor
// memory.  Same terms and the same charge cells as the FP32 form (the records of
// current_records.cuh), different arithmetic.
//
// With the table read bilinearly in the folded offset and linearly in the
// arrival tick, the per-pixel sum of Eq. (current) is a sum of shifted table
// rows of the table nodes:
//   I[p, k] = sum_node sum_a Q[p, node, a] R[node, k - a + L - 1],
// where a record (arrival A + f, bin b0, weights w_c of the four corner nodes
// b0 + c) deposits (1 - f) w_c at tick A and f w_c at tick A + 1 of node
// b0 + c.  Cut the arrival ticks into blocks of 16 (ab) and the output ticks
// into tiles of 128 (t): for one node and one block the contribution to one
// tile is a matrix product
//   D_t[m', p] += sum_{a' < 16} A[m', a'] Q[p, 16 ab + a'],
//   A[m', a'] = R[node, 128 t + 127 - m' - 16 ab - a' + L - 1]
// (zero outside the row; m' = 127 - (tick - 128 t): the accumulator rows run
// backwards in a tile), a Toeplitz block of the row: M = 128 ticks, N = 32
// pixels, K = 16 arrival ticks.  A depends on 16 ab - 128 t + m' + a' only,
// so all the A tiles of a node are views of one buffer (k_phase_table).
//
// Design: one CTA of 256 threads per SM (persistent, dynamic unit queue).
//  - A unit is a group of 32 active pixels, or for a heavy group a range of
//    its table-node rows (the units of a group write partial currents that a
//    second kernel adds in unit order); a CTA takes a unit and a pass of 2048
//    ticks; the accumulators D (16 tiles of 128 ticks x 32 pixels, FP32) live
//    in tensor memory (all 512 columns) and are added into the FP32 currents
//    every 64 nodes.
//  - Each table row is rounded to FP16/BF16 once per call by error diffusion
//    (k_round_rows: its suffix sums, hence the charge a point induces, keep
//    their FP32 values) and laid out as its phase table (k_phase_table: 8
//    shifted copies of the row interleaved in 16-byte rows, 35 KB per node,
//    every A tile a no-swizzle K-major view with overlapping core matrices);
//    the 72 MB of phase tables stay in L2.  For each node the CTA copies its
//    phase table into shared memory with one bulk asynchronous copy,
//    double-buffered.
//  - Records of the unit's pixels are generated into a per-CTA buffer (a
//    pixel's segments 128 at a time, their candidate points walked together)
//    and sorted per pixel by table bin (counting sort).  A node receives the
//    records of four bins (its corners) of each pixel.
//  - Builder warps 4-7 share a node's records evenly and turn them into
//    charge tiles Q[32 blocks][16 ticks][32 pixels], accumulated with integer
//    atomics in fixed point (order-independent, so the result is bitwise
//    reproducible), then converted to FP16/BF16 operand tiles.
//  - Issuer warps 0-3 (one thread each) own tick tiles t = w, w + 4, ... and
//    issue the MMAs of each batch slot by slot; tcgen05.commit on mbarriers
//    returns the operand buffers.  Warps 0-3 read D back (tcgen05.ld,
//    lane = 127 - tick within the tile) at each flush.
// Every mbarrier wait is bounded; a wait that gives up sets
// SIM_STATUS_TIMEOUT in the status word and the CTA drains and returns.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "current_records.cuh"

namespace larsim {

namespace {

#ifndef LARSIM_TC_BUILDERS
#define LARSIM_TC_BUILDERS 128
#endif
constexpr int kBuilders = LARSIM_TC_BUILDERS;   // builder threads (warps 4 ..): 128 or 256
static_assert(kBuilders == 128 || kBuilders == 256, "four or eight builder warps");
constexpr int kThreads = 128 + kBuilders;   // warps 0-3 issue and flush, the rest build
constexpr int kGroup = 32;                  // pixels per group (MMA N)
constexpr int kTileM = 128;                 // ticks per accumulator tile (MMA M)
constexpr int kTiles = 16;                  // tiles in tensor memory
constexpr int kPassTicks = kTileM * kTiles; // ticks per pass
constexpr int kBlk = 16;                    // arrival ticks per block (MMA K)
#ifndef LARSIM_TC_SLOTS
#define LARSIM_TC_SLOTS 32
#endif
constexpr int kSlots = LARSIM_TC_SLOTS;     // blocks per operand batch (a power of two, 16 or 32)
constexpr int kSlotShift = kSlots == 32 ? 5 : 4;
static_assert(kSlots == 16 || kSlots == 32, "operand batches of 16 or 32 blocks");
constexpr int kMaxBins = 2048;              // nb * nb <= kMaxBins
// Phase table of a node's row (see k_phase_table): 128-byte blocks of 8 rows
// of 8 operand values; (nt + 126) / 8 + 18 blocks, at most 289 for nt <= 2048.
constexpr int kMaxPhaseBlocks = 290;
constexpr int kMaxIm = kMaxPhaseBlocks * 128;
__host__ __device__ constexpr int phase_blocks(int L) { return (L + 126) / 8 + 18; }
// records per chunk per CTA unless configured (at most 2^20): 2^20 for calls
// sized for at least 2^17 active pixels (a large event touches each node with
// several chunks' worth of records: shorter chunks issue the same (node,
// block) MMAs once per chunk, 1.7x the MMAs of the 35-module spill at 2^18),
// else 2^18 (a smaller workspace: two buffers of 32-byte records per CTA)
constexpr int kRecDefault = 1 << 18, kRecDefaultLarge = 1 << 20;
constexpr int64_t kLargeCall = 1 << 17;
inline int default_chunk(int64_t pix_cap) { return pix_cap >= kLargeCall ? kRecDefaultLarge : kRecDefault; }
constexpr int kSubsPerSm = 2;               // work-balanced units per SM (target), unless tuned
constexpr int kMaxSplit = 16;               // table-node ranges a pixel group may be cut into
#ifndef LARSIM_TC_FLUSH_NODES
#define LARSIM_TC_FLUSH_NODES 64
#endif
constexpr int kFlushNodes = LARSIM_TC_FLUSH_NODES;   // nodes per accumulation window (see flush_acc)
constexpr float kFix = 4096.f;              // fixed-point scale of the charge accumulators (2^-12 e-)
constexpr int kIssuers = 4;
#ifndef LARSIM_TC_PAIRS
#define LARSIM_TC_PAIRS 128
#endif
constexpr int kPairs = LARSIM_TC_PAIRS;     // (pixel, segment) pairs loaded together by the generation (<= 256)
static_assert(kPairs <= 256 && (kPairs & (kPairs - 1)) == 0, "one pair per generation thread, a power of two");
#ifndef LARSIM_TC_PATCH_ROWS
#define LARSIM_TC_PATCH_ROWS 8
#define LARSIM_TC_PATCH_COLS 4
#endif
// pixel groups are cut from patches of kPatchRows rows x kPatchCols columns (see k_plan_perm)
constexpr int kPatchRows = LARSIM_TC_PATCH_ROWS, kPatchCols = LARSIM_TC_PATCH_COLS;
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxSpin = 1 << 22;           // bounded mbarrier waits (x ~ 0.5 us each), unless configured

struct __align__(16) BatchMeta {
    int node, count, last, pad;
    unsigned char blk[kSlots];              // block index relative to the pass start
};

struct __align__(1024) TcSmem {
    unsigned char im[2][kMaxIm];
    unsigned char bst[2][kSlots * 1024];
    union {
        struct {
            int hist[kMaxBins];
            unsigned char nflag[kMaxBins];
            int scan_tmp[kThreads / 32 + 1];
            int warp_n[kThreads / 32];
            Anchor anc[kPairs];             // a batch of a pixel's segments: anchors,
            int psg[kPairs];                // segment indexes,
            int pr0[kPairs], pn1[kPairs], pr2[kPairs];   // candidate ranges
            int poff[kPairs];               // and candidate offsets
        } g;
        int acc[kSlots * kBlk * kGroup];
    } u;
    unsigned short nodes[kMaxBins];
    BatchMeta meta[2];
    uint64_t full_im[2], empty_im[2], full_b[2], empty_b[2], done;
    uint32_t taddr;
    uint32_t blkmask[8];
    unsigned char rank_of[256], blk_of[256];    // a node's present arrival blocks: block -> rank -> block
    int lst_beg[128], lst_off[128], lst_wsum[8];
    int pin[kGroup];
    long long rowoff[kGroup];               // output row of each pixel slot (elements from the unit's base)
    int n_nodes, group, abort, spin;
};

static_assert(sizeof(TcSmem) + 1024 <= 232448, "shared memory of the tensor-core kernel above 227 KB");
static_assert(sizeof(((TcSmem *)nullptr)->u.g) <= sizeof(((TcSmem *)nullptr)->u.acc), "generation area above the tiles");

// A unit of work: the pixel group at positions [first, first + count) of the
// patch-ordered permutation of the call's active pixels (perm), restricted to
// the table nodes with bx in [nb r / k, nb (r + 1) / k).  Units of a group
// split in k > 1 write partial currents to `slice` (else -1).
struct __align__(16) Unit {
    int first, count, r, k;
    int slice, pad;
    long long work;
};

struct TcArgs {
    sim_config c;
    int nb, nt, bpp, rho0, im_bytes;
    uint32_t idesc;
    float qscale;                           // fixed point -> operand units
    float out_scale;                        // accumulator -> current (1 / table scale)
    const unsigned char *table;             // phase tables of the rows, [nb*nb][im_bytes]
    const Anchor *anch;
    const int32_t *active, *off, *segs;
    const int32_t *perm;                    // active-pixel index of each position in patch order
    const int64_t *counts;
    unsigned long long *status;             // counts[3]; counts[4], [5] receive the MMA and nonzero-cell counts
    int64_t pix_cap;
    float *current;
    uint64_t seed;
    EventInfo ev;
    Geo g;
    DriftPar dp;
    int *queue;                             // next entry of `order`
    const Unit *units;
    const int32_t *order;                   // units by decreasing work
    const int64_t *n_units;
    float *slices;                          // partial currents [slice][kGroup][n_ticks]
    Rec *recs, *sorted;                     // [grid][rec_cap]
    int rec_cap;                            // records per chunk per CTA
    int *offt;                              // [grid][kGroup][kMaxBins + 1]
    uint32_t *bmask;                        // [grid][kGroup][kMaxBins][8]: arrival blocks of each (pixel, bin)
};

// ----------------------------------------------------- PTX wrappers ----
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start, K-direction core-matrix
// stride (LBO), M/N-direction 8-row-group stride (SBO), version bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t a, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A/B format (0 FP16,
// 1 BF16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int fmt, int M, int N)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major tile with 16 K elements:
// 8-row x 16-byte core matrices, K-adjacent ones 128 B apart, row groups 256 B apart.
__host__ __device__ __forceinline__ int core_off(int row, int k)
{
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id)
{
    asm volatile("{\n .reg .pred p;\n setp.eq.u32 p, 1, 1;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d), "l"(a), "l"(b), "r"(id)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t *bar, int n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// Bounded wait for the completion of the phase with the given parity: at
// most s->spin polls (the configured limit).  After an abort it returns false
// at once.  Waits for the CTA's own MMAs and copies (which always complete:
// the accumulator flushes and the teardown) pass own = true: they ignore the
// abort and take the default bound, so that nothing this CTA issued is still
// in flight when it reads tensor memory, frees it or exits, and the phases of
// those barriers never fall behind their waiters.
__device__ __forceinline__ bool bar_wait(TcSmem *s, uint64_t *bar, uint32_t parity, bool own = false)
{
    const bool honor_abort = !own;
    const int lim = own ? kMaxSpin : s->spin;
    for (int it = 0; it < lim; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(saddr(bar)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (honor_abort && *(volatile int *)&s->abort) return false;
    }
    atomicExch(&s->abort, 1);
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kBuilders) : "memory"); }

// Barrier of the builder threads that also returns whether any of them saw
// the abort flag (a uniform decision: no builder is left waiting at a barrier).
__device__ __forceinline__ bool builders_any_abort(TcSmem *s)
{
    const int mine = *(volatile int *)&s->abort;
    int any;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
                 " selp.s32 %0, 1, 0, q;\n}\n"
                 : "=r"(any)
                 : "r"(mine), "n"(kBuilders)
                 : "memory");
    return any != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t ta, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_zero32(uint32_t ta)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
                 "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(ta),
                 "r"(0u)
                 : "memory");
}

// --------------------------------------------------------- helpers ----
// Exclusive scan of one int per thread across the CTA; *tot = total.
__device__ __forceinline__ int block_scan(int v, TcSmem *s, int *tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int W = kThreads / 32;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s->u.g.scan_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < W ? s->u.g.scan_tmp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < W) s->u.g.scan_tmp[lane] = wi - w;
        if (lane == W - 1) s->u.g.scan_tmp[W] = wi;
    }
    __syncthreads();
    const int r = s->u.g.scan_tmp[warp] + x - v;
    *tot = s->u.g.scan_tmp[W];
    __syncthreads();
    return r;
}

// Two operand values; FP16 saturates at its largest finite value.
template <int FMT>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if (FMT == 0) {
        const __half2 h = __floats2half2_rn(fminf(fmaxf(a, -65504.f), 65504.f), fminf(fmaxf(b, -65504.f), 65504.f));
        return *reinterpret_cast<const uint32_t *>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
}

// ------------------------------------------------- record generation ----
// Point ranges of a segment, seen from the pixel whose centre is (cx, cy),
// that can give a record inside a unit's table rows bx in [bx_lo, bx_hi):
// a record's corners span rows bx and bx + 1 of the folded x offset
// xi = |dx| bpp - 1/2 (nearest reads: bx = round(xi)), so its undiffused x
// offset lies in |dx| in [D_lo, D_hi] = [(bx_lo - 1) / bpp, (bx_hi + 1/2) / bpp]
// (D_lo = 0 below row 2), and its y offset within the table,
// |dy| < (nb + 1/2) / bpp, each widened by the diffusion clip * sTp and by
// 1e-3 pitch against rounding.  The x band is two slabs (dx > 0, dx < 0) or one
// (D_lo = 0); each slab, intersected with the y slab, gives a range of u and
// so of points mu (u = (mu + 1/2) / N), widened by one point each side.  Point
// indices idx = mu M + nu in [r0, r1) and [r2, r3) (r1 <= r2, or the second
// empty); every point outside them is rejected by point_record or by the
// unit's row test, so generating only these changes no record.
__device__ __forceinline__ void band_ranges(const Anchor &A, int M, float cx, float cy, float fbpp, int nb, float clip,
                                            int bx_lo, int bx_hi, int &r0, int &r1, int &r2, int &r3)
{
    const float w = clip * A.sTp + 1e-3f;
    const float Ry = ((float)nb + 0.5f) / fbpp + w;
    const float Dhi = ((float)bx_hi + 0.5f) / fbpp + w;
    const float Dlo = bx_lo >= 2 ? (float)(bx_lo - 1) / fbpp - w : 0.f;
    // u-interval of o + u d in [lo, hi] within [0, 1]
    auto slab = [](float o, float d, float lo, float hi, float &u0, float &u1) {
        if (fabsf(d) < 1e-12f) {
            if (o < lo || o > hi) u1 = -1.f;
        } else {
            const float ta = (lo - o) / d, tb = (hi - o) / d;
            u0 = fmaxf(u0, fminf(ta, tb));
            u1 = fminf(u1, fmaxf(ta, tb));
        }
    };
    float y0 = 0.f, y1 = 1.f;
    slab(A.fy0 - cy, A.dY, -Ry, Ry, y0, y1);
    const float ox = A.fx0 - cx;
    float a0 = y0, a1 = y1, b0 = y0, b1 = -1.f;
    if (Dlo > 0.f) {
        slab(ox, A.dX, Dlo, Dhi, a0, a1);
        b1 = y1;
        slab(ox, A.dX, -Dhi, -Dlo, b0, b1);
    } else {
        slab(ox, A.dX, -Dhi, Dhi, a0, a1);
    }
    const float N = (float)A.N;
    auto to_idx = [&](float u0, float u1, int &i0, int &i1) {
        i0 = i1 = 0;
        if (!(u0 <= u1)) return;
        const int mu0 = max(0, (int)floorf(u0 * N - 0.5f) - 1);
        const int mu1 = min(A.N - 1, (int)ceilf(u1 * N - 0.5f) + 1);
        if (mu1 >= mu0) {
            i0 = mu0 * M;
            i1 = (mu1 + 1) * M;
        }
    };
    int p0, p1, q0, q1;
    to_idx(a0, a1, p0, p1);
    to_idx(b0, b1, q0, q1);
    if (p1 <= p0) {                     // only the second (or none)
        p0 = q0;
        p1 = q1;
        q0 = q1 = 0;
    } else if (q1 > q0) {
        if (q0 < p0) {                  // order the two
            int t0 = p0, t1 = p1;
            p0 = q0, p1 = q1, q0 = t0, q1 = t1;
        }
        if (q0 <= p1) {                 // overlapping or adjacent: merge
            p1 = max(p1, q1);
            q0 = q1 = 0;
        }
    }
    r0 = p0, r1 = p1, r2 = q0, r3 = q1;
}

// Generation cursor of a group: pixel slot gp, CSR position e of the first
// segment of the current batch of the pixel's segments (-1: pixel not begun),
// and the offset base of the next step in the batch's concatenated candidates.
struct GenState {
    int gp, e, base;
};

// Generates the records of the group's pixels from the cursor on, until the
// chunk buffer is full or the group is done; sorts each pixel's part by bin
// into `sorted`, writes its bin offsets to offt and, for each (pixel, bin)
// holding records, the 256-bit mask of the arrival blocks its records' two
// ticks fall in (relative to the pass start k0) to bmask; marks the nodes it
// touches.  Returns the number of records of the chunk; st.gp == npg when done.
__device__ int gen_chunk(const TcArgs &a, TcSmem *s, GenState &st, int64_t pi0, int npg, int bx_lo, int bx_hi,
                         Rec *recs, Rec *sorted, int *offt, uint32_t *bmask, int k0)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = a.nb, nb2 = nb * nb, M = a.c.mc_per_sample;
    const float clip = a.c.diff_clip_sigma, fbpp = (float)a.bpp;
    const int npx = a.g.npx_x * a.g.npx_y;
    const bool split = bx_lo > 0 || bx_hi < nb;
    int nrec = 0;
    while (st.gp < npg) {
        const int64_t pi = a.perm[pi0 + st.gp];
        const int32_t pid = a.active[pi];
        const int an = pid / npx;
        const int rem = pid - an * npx;
        const int iy = rem / a.g.npx_x, ix = rem - iy * a.g.npx_x;
        const int slot = an / a.g.n_anodes;
        const uint64_t key = slot_key(a.seed, a.ev, slot);
        const int64_t seg0 = slot_first(a.ev, slot);
        if (st.e < 0) {
            st.e = a.off[pi];
            st.base = 0;
        }
        const int e1 = a.off[pi + 1];
        const int start = nrec;
        bool full = false;
        while (st.e < e1) {
            // a batch of the pixel's segments, one thread each: anchor and candidate points
            // (all of them, or for a unit of a split group the ranges that can reach its rows)
            const int np = min(kPairs, e1 - st.e);
            int cnt = 0;
            if (tid < np) {
                const int sg = a.segs[st.e + tid];
                const Anchor A = a.anch[sg];
                int r0 = 0, r1 = A.N * M, r2 = 0, r3 = 0;
                if (split)
                    band_ranges(A, M, (float)(ix - A.ix_ref) + 0.5f, (float)(iy - A.iy_ref) + 0.5f, fbpp, nb, clip,
                                bx_lo, bx_hi, r0, r1, r2, r3);
                s->u.g.anc[tid] = A;
                s->u.g.psg[tid] = sg;
                s->u.g.pr0[tid] = r0;
                s->u.g.pn1[tid] = r1 - r0;
                s->u.g.pr2[tid] = r2;
                cnt = (r1 - r0) + (r3 - r2);
            }
            int ncand;
            const int off = block_scan(cnt, s, &ncand);
            if (tid < np) s->u.g.poff[tid] = off;
            __syncthreads();
            // the batch's candidates, kThreads at a time
            while (st.base < ncand) {
                const int c = st.base + tid;
                bool ok = false;
                Rec r;
                if (c < ncand) {
                    int q = 0;                  // the pair holding candidate c: last q with poff[q] <= c
#pragma unroll
                    for (int step = kPairs / 2; step > 0; step >>= 1)
                        if (q + step < np && s->u.g.poff[q + step] <= c) q += step;
                    const int loc = c - s->u.g.poff[q], n1 = s->u.g.pn1[q];
                    const int idx = loc < n1 ? s->u.g.pr0[q] + loc : s->u.g.pr2[q] + (loc - n1);
                    const Anchor A = s->u.g.anc[q];
                    const PointPos pp =
                        point_position(A, idx, M, key, (uint32_t)(s->u.g.psg[q] - seg0), clip, a.dp);
                    ok = point_record(A, pp, (float)(ix - A.ix_ref) + 0.5f, (float)(iy - A.iy_ref) + 0.5f, fbpp,
                                      nb, a.c.nearest_lut, r);
                    if (ok) {                   // corner nodes (bx, bx + 1) must reach the unit's range
                        const int bx = r.b0 / nb;
                        ok = bx < bx_hi && bx + 1 >= bx_lo;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                if (lane == 0) s->u.g.warp_n[warp] = __popc(m);
                __syncthreads();
                int wb = 0, nq = 0;
#pragma unroll
                for (int w2 = 0; w2 < kThreads / 32; ++w2) {
                    const int c2 = s->u.g.warp_n[w2];
                    wb += (w2 < warp) ? c2 : 0;
                    nq += c2;
                }
                __syncthreads();
                if (nrec + nq > a.rec_cap) {    // chunk full: this step is redone in the next chunk
                    full = true;
                    break;
                }
                if (ok) {
                    const int d = nrec + wb + __popc(m & ((1u << lane) - 1u));
                    recs[d] = r;
                    atomicAdd(&s->u.g.hist[r.b0], 1);
                }
                nrec += nq;
                st.base += kThreads;
            }
            if (full) break;
            st.e += np;
            st.base = 0;
            __syncthreads();                    // the batch's arrays are read: the next may overwrite them
        }
        __syncthreads();
        if (nrec > start) {
            // bin offsets of this pixel's part, node flags, scatter cursors
            constexpr int kB = (kMaxBins + kThreads - 1) / kThreads;
            int v[kB], sv = 0;
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                const int b = tid * kB + i;
                v[i] = (b < nb2) ? s->u.g.hist[b] : 0;
                sv += v[i];
            }
            int tot;
            int pv = start + block_scan(sv, s, &tot);
            int *orow = offt + (size_t)st.gp * (kMaxBins + 1);
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                const int b = tid * kB + i;
                if (b < nb2) {
                    orow[b] = pv;
                    s->u.g.hist[b] = pv;
                    if (v[i] > 0) {
                        uint4 *mk = reinterpret_cast<uint4 *>(bmask + ((size_t)st.gp * kMaxBins + b) * 8);
                        mk[0] = make_uint4(0u, 0u, 0u, 0u);
                        mk[1] = make_uint4(0u, 0u, 0u, 0u);
                    }
                    if (v[i] > 0) {                 // the bin's corner nodes within the unit's range
                        const int bx = b / nb, by = b - bx * nb;
                        const bool in0 = bx >= bx_lo && bx < bx_hi;
                        const bool in1 = bx + 1 < nb && bx + 1 >= bx_lo && bx + 1 < bx_hi;
                        if (in0) s->u.g.nflag[b] = 1;
                        if (in1) s->u.g.nflag[b + nb] = 1;
                        if (in0 && by + 1 < nb) s->u.g.nflag[b + 1] = 1;
                        if (in1 && by + 1 < nb) s->u.g.nflag[b + nb + 1] = 1;
                    }
                }
                pv += v[i];
            }
            if (tid == 0) {
                orow[nb2] = nrec;
                s->pin[st.gp] = 1;
            }
            __syncthreads();
            uint32_t *bmp = bmask + (size_t)st.gp * kMaxBins * 8;
            for (int i = start + tid; i < nrec; i += kThreads) {
                const Rec r = recs[i];
                sorted[atomicAdd(&s->u.g.hist[r.b0], 1)] = r;
                // blocks of the record's two ticks (a zero-weight tap may mark a block: it only adds zeros)
                const int rel = r.A - k0;
                const int b0k = rel >> 4, b1k = (rel + 1) >> 4;
                if (b0k >= 0 && b0k < 256) atomicOr(bmp + r.b0 * 8 + (b0k >> 5), 1u << (b0k & 31));
                if (b1k != b0k && b1k >= 0 && b1k < 256) atomicOr(bmp + r.b0 * 8 + (b1k >> 5), 1u << (b1k & 31));
            }
            __syncthreads();
            for (int b = tid; b < nb2; b += kThreads) s->u.g.hist[b] = 0;
            __syncthreads();
        }
        if (full) break;
        ++st.gp;
        st.e = -1;
    }
    return nrec;
}

// ------------------------------------------------------------ roles ----
// List L of a node (L = corner c * 32 + pixel) holding flat record index k:
// the last L with lst_off[L] <= k (empty lists share their successor's offset).
__device__ __forceinline__ int find_list(const int *off, int k)
{
    int lo = 0;
#pragma unroll
    for (int step = 64; step > 0; step >>= 1)
        if (off[lo + step] <= k) lo += step;
    return lo;
}

// Loads the records k0 .. min(k0 + U, k_hi) - 1 of a builder's slice of the
// node's concatenated lists (list cursor L2 advances); absent ones get weight 0.
template <int U>
__device__ __forceinline__ void load_recs(const TcSmem *s, const Rec *sorted, int k0, int k_hi, int &L2, int4 (&h)[U],
                                          float (&w)[U], int (&px)[U])
{
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const int k = k0 + j;
        h[j] = make_int4(0, 0, 0, 0);
        w[j] = 0.f;
        px[j] = 0;
        if (k < k_hi) {
            while (L2 < 127 && s->lst_off[L2 + 1] <= k) ++L2;
            const int L = L2;
            const Rec *r = sorted + s->lst_beg[L] + (k - s->lst_off[L]);
            h[j] = *reinterpret_cast<const int4 *>(r);
            w[j] = reinterpret_cast<const float *>(&r->w)[L >> 5];
            px[j] = L & 31;
        }
    }
}

// Adds the two ticks of each record whose arrival block falls in operand batch
// kb into the fixed-point charge tiles (block rank from the node's rank table).
template <int U>
__device__ __forceinline__ void accum_recs(TcSmem *s, const int4 (&h)[U], const float (&w)[U], const int (&px)[U],
                                           int kb)
{
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const float f = __int_as_float(h[j].z);
#pragma unroll
        for (int tap = 0; tap < 2; ++tap) {
            const float val = tap ? f * w[j] : (1.f - f) * w[j];
            const int rel = h[j].x + tap;
            const int rb = rel >> 4;
            if (val == 0.f || rb < 0 || rb >= 256) continue;
            const int rank = s->rank_of[rb];    // the tap's block is present: its records set it
            if ((rank >> kSlotShift) != kb) continue;
            atomicAdd(&s->u.acc[((rank & (kSlots - 1)) * kBlk + (rel & (kBlk - 1))) * kGroup + px[j]],
                      __float2int_rn(val * kFix));
        }
    }
}

// Builder threads (warps 4 .., bt = 0 .. kBuilders - 1).  For each node the 128
// record lists (corner c = bt / 32 of pixel bt % 32, held by builders bt <
// 128: the pixel's records in bin node - c) are concatenated and all the
// builders share the records evenly; the
// charge of each (block, tick, pixel) cell is summed with integer atomics, so
// the order does not matter.  Publishes each node's operand batches in order.
// Control flow is uniform across the builders (their named barriers); after
// an abort they stop at the next node.
template <int FMT>
__device__ void build_batches(const TcArgs &a, TcSmem *s, const Rec *sorted, const int *offt, const uint32_t *bmask,
                              const unsigned short *nodes, int nn, uint32_t &q, unsigned long long &n_cells)
{
#ifndef LARSIM_TC_RECS_IN_FLIGHT
#define LARSIM_TC_RECS_IN_FLIGHT 4
#endif
    constexpr int U = LARSIM_TC_RECS_IN_FLIGHT;         // records in flight per thread
    const int bt = threadIdx.x - 128, lane = bt & 31, cw = bt >> 5;
    const bool owner = bt < 128;                        // holds one of the node's 128 lists
    const int nb = a.nb;
    // the charge tiles share shared memory with the generation's histogram: zero them once
    // here; afterwards the conversion clears every cell it reads
    for (int i = bt; i < kSlots * kBlk * kGroup / 4; i += kBuilders)
        reinterpret_cast<int4 *>(s->u.acc)[i] = make_int4(0, 0, 0, 0);
    // a node's list bounds and block masks are loaded one node ahead (unconditionally: the
    // indexes stay inside this CTA's offset and mask buffers; unused values are discarded)
    auto fetch = [&](int n, int &b, int &beg, int &end, uint4 &mk0, uint4 &mk1) {
        const int nx = n / nb, ny = n - nx * nb;
        const int c = cw & 3;                           // non-owners fetch a copy of an owner's list
        const int bx = nx - (c & 1), by = ny - (c >> 1);
        b = (bx >= 0 && by >= 0) ? bx * nb + by : 0;
        const int *orow = offt + (size_t)lane * (kMaxBins + 1);
        beg = orow[b];
        end = (bx >= 0 && by >= 0) ? orow[b + 1] : beg;
        const uint4 *mk = reinterpret_cast<const uint4 *>(bmask + ((size_t)lane * kMaxBins + b) * 8);
        mk0 = mk[0];
        mk1 = mk[1];
    };
    int fb = 0, fbeg = 0, fend = 0;
    uint4 fm0 = make_uint4(0u, 0u, 0u, 0u), fm1 = fm0;
    if (nn > 0) fetch(nodes[0], fb, fbeg, fend, fm0, fm1);
    const bool pin = owner && s->pin[lane] != 0;
    for (int u = 0; u < nn; ++u) {
        if (builders_any_abort(s)) return;
        const int n = nodes[u];
        const int beg = pin ? fbeg : 0, len = pin ? fend - fbeg : 0;
        // arrival blocks present: OR of the 128 lists' masks (written when the records were sorted)
        uint4 mk0 = make_uint4(0u, 0u, 0u, 0u), mk1 = mk0;
        if (len > 0) {
            mk0 = fm0;
            mk1 = fm1;
        }
        if (u + 1 < nn) fetch(nodes[u + 1], fb, fbeg, fend, fm0, fm1);
        int x = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31 && owner) s->lst_wsum[cw] = x;
        if (bt < 8) s->blkmask[bt] = 0;
        builders_sync();
        {
            const uint32_t w8[8] = {mk0.x, mk0.y, mk0.z, mk0.w, mk1.x, mk1.y, mk1.z, mk1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t o = __reduce_or_sync(0xffffffffu, w8[j]);
                if (lane == 0 && o) atomicOr(&s->blkmask[j], o);
            }
        }
        int R = 0, pre = 0;
#pragma unroll
        for (int w2 = 0; w2 < 4; ++w2) {
            pre += (w2 < cw) ? s->lst_wsum[w2] : 0;
            R += s->lst_wsum[w2];
        }
        if (owner) {
            s->lst_beg[bt] = beg;
            s->lst_off[bt] = pre + x - len;
        }
        builders_sync();
        // each builder takes a contiguous slice of the concatenated lists
        const int k_lo = (int)(((long long)R * bt) / kBuilders), k_hi = (int)(((long long)R * (bt + 1)) / kBuilders);
        const int L_lo = k_lo < k_hi ? find_list(s->lst_off, k_lo) : 0;
        // the first U records of the slice stay in registers for all of the node's batches
        // (most slices are that short); longer slices reload the rest in each batch
        int4 hc[U];
        float wc[U];
        int pc[U];
        int L2c = L_lo;
        load_recs<U>(s, sorted, k_lo, k_hi, L2c, hc, wc, pc);
        // rank of each present arrival block (its order, hence its batch and slot) and the
        // inverse, in shared memory: 256 / kBuilders blocks per builder
#pragma unroll
        for (int i = 0; i < 256 / kBuilders; ++i) {
            const int b = bt + kBuilders * i, wd = b >> 5;
            const uint32_t wm = s->blkmask[wd];
            if ((wm >> (b & 31)) & 1u) {
                int r = __popc(wm & ((1u << (b & 31)) - 1u));
                for (int j = 0; j < wd; ++j) r += __popc(s->blkmask[j]);
                s->rank_of[b] = (unsigned char)r;
                s->blk_of[r] = (unsigned char)b;
            }
        }
        builders_sync();
        int nblk = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) nblk += __popc(s->blkmask[j]);
        const int nbatch = nblk > 0 ? (nblk + kSlots - 1) / kSlots : 1;
        for (int kb = 0; kb < nbatch; ++kb) {
            // pass 2: fixed-point charge of the blocks of this batch
            accum_recs<U>(s, hc, wc, pc, kb);
            int L2 = L2c;
            for (int k0 = k_lo + U; k0 < k_hi; k0 += U) {
                int4 h[U];
                float w[U];
                int px[U];
                load_recs<U>(s, sorted, k0, k_hi, L2, h, w, px);
                accum_recs<U>(s, h, w, px, kb);
            }
            builders_sync();
            const int st = q & 1;
            if (q >= 2) bar_wait(s, &s->empty_b[st], ((q - 2) >> 1) & 1);   // on failure: abort set, go on
            const int count = min(kSlots, nblk - kb * kSlots);
            unsigned char *dst = s->bst[st];
            // one 16-byte core-matrix row (8 ticks of one pixel) per step
            for (int j = bt; j < count * kGroup * 2; j += kBuilders) {
                const int sl = j >> 6, p = j & (kGroup - 1), h = (j >> 5) & 1;
                int *ac = s->u.acc + (sl * kBlk + 8 * h) * kGroup + p;
                int c8[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    c8[e] = ac[e * kGroup];
                    ac[e * kGroup] = 0;                       // read and clear
                    n_cells += c8[e] != 0;                    // nonzero charge cells
                }
                uint4 v;
                v.x = pack2<FMT>((float)c8[0] * a.qscale, (float)c8[1] * a.qscale);
                v.y = pack2<FMT>((float)c8[2] * a.qscale, (float)c8[3] * a.qscale);
                v.z = pack2<FMT>((float)c8[4] * a.qscale, (float)c8[5] * a.qscale);
                v.w = pack2<FMT>((float)c8[6] * a.qscale, (float)c8[7] * a.qscale);
                *reinterpret_cast<uint4 *>(dst + sl * 1024 + core_off(p, 8 * h)) = v;
            }
            if (bt < count) s->meta[st].blk[bt] = s->blk_of[kb * kSlots + bt];   // block of slot bt
            if (bt == 0) {
                s->meta[st].node = n;
                s->meta[st].count = count > 0 ? count : 0;
                s->meta[st].last = (kb == nbatch - 1);
            }
            fence_async_smem();
            builders_sync();
            if (bt == 0) bar_arrive(&s->full_b[st]);
            ++q;
        }
    }
}

// Issuer thread of warp w (0-3): MMAs of tiles t = w, w + 4, ... for every batch.
__device__ void issue_mmas(const TcArgs &a, TcSmem *s, int w, const unsigned short *nodes, int nn, uint32_t S,
                           uint32_t &q, int k0, unsigned long long &n_mma, int64_t (&im_last)[2])
{
    const int T = a.c.n_ticks;
    const uint32_t tm = s->taddr;
    tc_fence_after();
    auto load_im = [&](uint32_t sn, int node) {
        const int b = sn & 1;
        if (sn >= 2 && !bar_wait(s, &s->empty_im[b], ((sn - 2) >> 1) & 1)) return;
        bulk_load(s->im[b], a.table + (size_t)node * a.im_bytes, (uint32_t)a.im_bytes, &s->full_im[b]);
        im_last[b] = sn;                                    // the buffer's latest copy (teardown waits for it)
    };
    if (w == 0 && nn > 0) load_im(S, nodes[0]);
    for (int u = 0; u < nn; ++u) {
        const uint32_t sn = S + u;
        const int ib = sn & 1;
        if (!bar_wait(s, &s->full_im[ib], (sn >> 1) & 1)) return;
        const uint32_t im0 = saddr(s->im[ib]);
        int last = 0;
        do {
            const int st = q & 1;
            if (!bar_wait(s, &s->full_b[st], (q >> 1) & 1)) return;
            const int count = s->meta[st].count;
            last = s->meta[st].last;
            uint32_t b4[kSlots / 4];                          // the slots' blocks, four per word
#pragma unroll
            for (int i = 0; i < kSlots / 16; ++i) {
                const uint4 bw = reinterpret_cast<const uint4 *>(s->meta[st].blk)[i];
                b4[4 * i] = bw.x, b4[4 * i + 1] = bw.y, b4[4 * i + 2] = bw.z, b4[4 * i + 3] = bw.w;
            }
            // descriptors advance by address >> 4: A (the node's phase table) by 16 bytes per unit
            // of `base`, B by 1024 bytes per slot.  A's core matrices: 128 bytes apart in both K
            // and M (they overlap: the Toeplitz structure), rows 16 bytes apart.
            const uint64_t ad0 = smem_desc(im0, 128, 128), bd0 = smem_desc(saddr(s->bst[st]), 128, 256);
            tc_fence_after();
            uint32_t issued = 0;
            // slot-major: consecutive MMAs go to different accumulator tiles (a short N = 32 MMA
            // into the tile the previous one wrote waits for it); each tile still takes its
            // slots in order
#pragma unroll
            for (int i = 0; i < kSlots; ++i) {
                if (i >= count) break;
                const int boff = kBlk * (int)((b4[i >> 2] >> (8 * (i & 3))) & 0xffu);
#pragma unroll
                for (int t = w; t < kTiles; t += kIssuers) {
                    const int base = boff - kTileM * t;            // A tile of this block in tile t
                    if (k0 + kTileM * t < T && base >= 0 && base <= a.rho0) {   // else the A tile is all zero
                        mma_f16(tm + (uint32_t)(kGroup * t), ad0 + (uint64_t)base, bd0 + (uint64_t)(64 * i),
                                a.idesc);
                        ++issued;
                    }
                }
            }
            n_mma += issued;
            mma_commit(&s->empty_b[st]);
            ++q;
        } while (!last);
        mma_commit(&s->empty_im[ib]);
        if (w == 0 && u + 1 < nn) load_im(sn + 1, nodes[u + 1]);
    }
}


// ------------------------------------------------------ work planning ----
// Units of balanced work: the work of a pixel is estimated by its candidate
// points sum_{s -> p} N_s M; a 32-pixel group whose work exceeds
// wcap = total / (kSubsPerSm * SMs) is cut into k (a power of two <= 16)
// units by ranges of table-node rows bx, so that each unit holds at most about
// wcap.  The units of a group issue disjoint MMAs (each node belongs to one
// range); they write partial currents that k_plan_reduce adds in unit order.
// Units are taken from the queue in order of decreasing work.

// Active pixels of the call's range [begin, min(counts[1], end)), counted from begin.
__device__ __forceinline__ int64_t active_count(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end)
{
    if (counts[3] != 0 || counts[1] > pix_cap) return 0;
    return max((int64_t)0, min(counts[1], end) - begin);
}

// First index i in [lo, hi) with act[i] >= v (act increasing).
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *act, int64_t lo, int64_t hi, int32_t v)
{
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (act[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Patch order of the call's active pixels: pixel groups of consecutive
// active ids (a stretch of one row) share few (table node, arrival block)
// pairs, the tiles the MMAs are issued for; 32 pixels of a compact patch, which
// see the same tracks at nearby offsets and times, share more (20 % fewer
// MMAs on the module event).  Order: anode, band of kPatchRows rows, patch of
// kPatchCols columns in the band, row, column.  The position of each pixel is
// counted with binary searches in the increasing active list (the pixels
// before it in that order), so the permutation is deterministic; perm[pos] =
// its active index.
__global__ void k_plan_perm(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end,
                            const int32_t *active, int nx, int ny, int32_t *perm)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = active_count(counts, pix_cap, begin, end);
    if (j >= npix) return;
    const int64_t lo = begin, hi = begin + npix;
    const int32_t pid = active[begin + j];
    const int npx = nx * ny;
    const int an = pid / npx, rem = pid - an * npx;
    const int iy = rem / nx, ix = rem - iy * nx;
    const int r0 = (iy / kPatchRows) * kPatchRows, r1 = min(r0 + kPatchRows, ny);
    const int c0 = (ix / kPatchCols) * kPatchCols, c1 = min(c0 + kPatchCols, nx);
    const int32_t abase = an * npx;
    int64_t pos = lower_bound_i32(active, lo, hi, abase + r0 * nx) - lo;        // earlier anodes and bands
    for (int r = r0; r < r1; ++r) {
        const int32_t rb = abase + r * nx;
        const int64_t a0 = lower_bound_i32(active, lo, hi, rb);
        const int64_t ac0 = lower_bound_i32(active, lo, hi, rb + c0);
        pos += ac0 - a0;                                                        // left of the patch in the band
        if (r < iy) pos += lower_bound_i32(active, lo, hi, rb + c1) - ac0;      // the patch's rows above
    }
    pos += lower_bound_i32(active, lo, hi, pid) - lower_bound_i32(active, lo, hi, abase + iy * nx + c0);
    perm[pos] = (int32_t)(begin + j);
}

// Work of each position of the patch order: the candidate points of its pixel.
__global__ void k_plan_work(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end, const int32_t *off,
                            const int32_t *segs, const int32_t *perm,
                            const int32_t *n_samples, int M, long long *pwork, unsigned long long *total)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = active_count(counts, pix_cap, begin, end);
    long long w = 0;
    if (p < npix) {
        const int64_t pi = perm[p];
        for (int e = off[pi]; e < off[pi + 1]; ++e) w += n_samples[segs[e]];
        w *= M;
        pwork[p] = w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(total, (unsigned long long)w);
}

// Number of units of each group (nunit) and of partial slices (nslice: k when k > 1).
__global__ void k_plan_split(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end, const long long *pwork,
                             const unsigned long long *total, int target, int32_t *nunit, int32_t *nslice,
                             int64_t ngroups_cap)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups_cap) return;
    const int64_t npix = active_count(counts, pix_cap, begin, end);
    int k = 0;
    if (g * kGroup < npix) {
        long long gw = 0;
        for (int64_t p = g * kGroup; p < min(npix, (g + 1) * kGroup); ++p) gw += pwork[p];
        // wcap rounded up: the split units then number fewer than 2 * target in all
        const long long wcap = max(1ll, (long long)((*total + (unsigned long long)target - 1) / (unsigned long long)target));
        k = 1;
        while (k < kMaxSplit && gw > wcap * k) k <<= 1;
    }
    nunit[g] = k;
    nslice[g] = k > 1 ? k : 0;
}

__global__ void k_plan_emit(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end, const long long *pwork,
                            const int32_t *nunit, const int32_t *pos, const int32_t *spos, Unit *units,
                            int64_t ngroups_cap)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups_cap) return;
    const int k = nunit[g];
    if (k == 0) return;
    const int64_t npix = active_count(counts, pix_cap, begin, end);
    const int cnt = (int)min((int64_t)kGroup, npix - g * kGroup);
    long long w = 0;
    for (int i = 0; i < cnt; ++i) w += pwork[g * kGroup + i];
    for (int r = 0; r < k; ++r) {
        Unit u;
        u.first = (int)(g * kGroup);                 // position in the patch order
        u.count = cnt;
        u.r = r;
        u.k = k;
        u.slice = k > 1 ? spos[g] + r : -1;
        u.pad = 0;
        u.work = w / k;
        units[pos[g] + r] = u;
    }
}

// order[rank] = j, rank by decreasing work, ties by index.
__global__ void k_plan_rank(const Unit *units, const int64_t *n_units, int32_t *order)
{
    __shared__ long long tile[1024];
    const int64_t n = *n_units;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const long long wj = j < n ? units[j].work : 0;
    int rank = 0;
    for (int64_t t0 = 0; t0 < n; t0 += 1024) {
        for (int i = threadIdx.x; i < 1024; i += blockDim.x) tile[i] = t0 + i < n ? units[t0 + i].work : 0;
        __syncthreads();
        if (j < n) {
            const int m = (int)min((int64_t)1024, n - t0);
            for (int i = 0; i < m; ++i) {
                const long long wi = tile[i];
                rank += (wi > wj) || (wi == wj && t0 + i < j);
            }
        }
        __syncthreads();
    }
    if (j < n) order[rank] = (int32_t)j;
}

// Current of the pixels of split groups: the partial slices of the group's
// units added in unit order (one CTA per group), into each pixel's row.
__global__ void k_plan_reduce(const int64_t *counts, int64_t pix_cap, int64_t begin, int64_t end,
                              const int32_t *nunit, const int32_t *spos, const int32_t *perm, const float *slices,
                              int T, float *current, int64_t ngroups_cap)
{
    const int64_t g = blockIdx.x;
    if (g >= ngroups_cap) return;
    const int k = nunit[g];
    if (k <= 1) return;
    const int64_t npix = active_count(counts, pix_cap, begin, end);
    const int cnt = (int)min((int64_t)kGroup, npix - g * kGroup);
    const float *src = slices + (size_t)spos[g] * kGroup * T;
    for (int p = 0; p < cnt; ++p) {
        float *dst = current + (size_t)perm[g * kGroup + p] * T;
        const float *sp = src + (size_t)p * T;
        for (int i = threadIdx.x; i < T; i += blockDim.x) {
            float v = sp[i];
            for (int r = 1; r < k; ++r) v += sp[(size_t)r * kGroup * T + i];
            dst[i] = v;
        }
    }
}

// Warps 0-3 (all lanes): waits for every MMA issued so far, adds the
// accumulators to the output rows of the unit (`rows`: the group's current
// rows, or its partial slice; stores them when `first`), and zeroes them.  The tensor cores' FP32 accumulation truncates: summing a
// whole pixel's contributions in one accumulator biased the result low by up
// to ~2e-3 in the densest pixels; a window of kFlushNodes nodes keeps each
// accumulator a small fraction of the final value, and the windows are added
// in FP32 with round-to-nearest (one FMA per window).
__device__ void flush_acc(const TcArgs &a, TcSmem *s, uint32_t tm, uint32_t &flushes, int k0, float *rows, int npg,
                          bool first)
// rows: base of the unit's output rows; pixel slot p writes rows + s->rowoff[p]
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int T = a.c.n_ticks;
    if (lane == 0) mma_commit(&s->done);
    __syncwarp();
    const bool ok = bar_wait(s, &s->done, flushes & 1, true) && !*(volatile int *)&s->abort;
    tc_fence_after();
    // the rows' previous values of tile t + 1 are loaded while tile t is read and stored
    const int lrow = (kTileM - 1) - (32 * warp + lane);     // accumulator rows run backwards in a tile
    float old[kGroup], nxt[kGroup];
    auto load_old = [&](int t, float (&dst)[kGroup]) {
        const int tick = k0 + kTileM * t + lrow;
        const bool use = ok && !first && k0 + kTileM * t < T && tick < T;
#pragma unroll
        for (int p = 0; p < kGroup; ++p) dst[p] = (use && p < npg) ? rows[tick + s->rowoff[p]] : 0.f;
    };
    load_old(0, old);
    for (int t = 0; t < kTiles; ++t) {
        const int tick0 = k0 + kTileM * t;
        if (tick0 >= T) break;
        if (t + 1 < kTiles) load_old(t + 1, nxt);
        const uint32_t ta = tm + ((uint32_t)(32 * warp) << 16) + kGroup * t;
        float v[32];
        tmem_ld32(ta, v);
        const int tick = tick0 + lrow;
        if (ok && tick < T) {
            float *base = rows + tick;
            if (!first) {
#pragma unroll
                for (int p = 0; p < kGroup; ++p) v[p] = fmaf(v[p], a.out_scale, old[p]);
            } else {
#pragma unroll
                for (int p = 0; p < kGroup; ++p) v[p] *= a.out_scale;
            }
#pragma unroll
            for (int p = 0; p < kGroup; ++p)
                if (p < npg) base[s->rowoff[p]] = v[p];
        }
        tmem_zero32(ta);
#pragma unroll
        for (int p = 0; p < kGroup; ++p) old[p] = nxt[p];
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    ++flushes;
}

template <int FMT>
__global__ void __launch_bounds__(kThreads, 1) k_induced_current_tc(TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    TcSmem *s = reinterpret_cast<TcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool go = a.counts[3] == 0 && a.counts[1] <= a.pix_cap;
    const int64_t nsub = go ? *a.n_units : 0;
    const int T = a.c.n_ticks, nb2 = a.nb * a.nb;
    Rec *recs = a.recs + (size_t)blockIdx.x * a.rec_cap;
    Rec *sorted = a.sorted + (size_t)blockIdx.x * a.rec_cap;
    int *offt = a.offt + (size_t)blockIdx.x * kGroup * (kMaxBins + 1);

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            bar_init(&s->full_im[i], 1);
            bar_init(&s->empty_im[i], kIssuers);
            bar_init(&s->full_b[i], 1);
            bar_init(&s->empty_b[i], kIssuers);
        }
        bar_init(&s->done, kIssuers);
        s->abort = 0;
        s->spin = a.c.wait_spin_limit > 0 ? a.c.wait_spin_limit : kMaxSpin;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s->taddr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = s->taddr;
    if (warp < 4) {
        for (int t = 0; t < kTiles; ++t) tmem_zero32(tm + ((uint32_t)(32 * warp) << 16) + kGroup * t);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }

    uint32_t S = 0, q = 0, flushes = 0;     // node, batch and flush sequence numbers (barrier phases)
    unsigned long long n_mma = 0;           // MMAs issued by this thread
    int64_t im_last[2] = {-1, -1};          // sequence number of the latest table copy into each buffer
    unsigned long long n_cells = 0;         // nonzero charge cells converted by this thread
    for (;;) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) s->group = atomicAdd(a.queue, 1);
        __syncthreads();
        const int64_t g = s->group;
        if (g >= nsub || *(volatile int *)&s->abort) break;
        const Unit un = a.units[a.order[g]];
        const int64_t pi0 = un.first;
        const int npg = un.count;
        if (npg <= 0) continue;
        const int bx_lo = a.nb * un.r / un.k, bx_hi = a.nb * (un.r + 1) / un.k;
        float *rows = un.slice < 0 ? a.current : a.slices + (size_t)un.slice * kGroup * T;
        if (tid < kGroup)                       // each slot's row: its pixel's, or its row of the unit's slice
            s->rowoff[tid] = tid < npg ? (un.slice < 0 ? (long long)a.perm[pi0 + tid] * T : (long long)tid * T) : 0;
        for (int k0 = 0; k0 < T; k0 += kPassTicks) {
            GenState st{0, -1, 0};
            bool first = true;                  // no accumulator window stored yet in this pass
            while (st.gp < npg) {
                // ---- chunk: generate and sort records, list the nodes touched ----
                for (int b = tid; b < nb2; b += kThreads) {
                    s->u.g.hist[b] = 0;
                    s->u.g.nflag[b] = 0;
                }
                if (tid < kGroup) s->pin[tid] = 0;
                __syncthreads();
                // records keep arrival ticks relative to the pass start
                uint32_t *bmask = a.bmask + (size_t)blockIdx.x * kGroup * kMaxBins * 8;
                const int nrec = gen_chunk(a, s, st, pi0, npg, bx_lo, bx_hi, recs, sorted, offt, bmask, k0);
                {
                    constexpr int kB = (kMaxBins + kThreads - 1) / kThreads;
                    int fl[kB], sf = 0;
#pragma unroll
                    for (int i = 0; i < kB; ++i) {
                        const int b = tid * kB + i;
                        fl[i] = (b < nb2 && nrec > 0) ? s->u.g.nflag[b] : 0;
                        sf += fl[i];
                    }
                    int tot;
                    int pf = block_scan(sf, s, &tot);
#pragma unroll
                    for (int i = 0; i < kB; ++i) {
                        if (fl[i]) s->nodes[pf++] = (unsigned short)(tid * kB + i);
                    }
                    if (tid == 0) s->n_nodes = tot;
                }
                // shift arrival ticks to the pass start
                if (k0 != 0)
                    for (int i = tid; i < nrec; i += kThreads) sorted[i].A -= k0;
                __syncthreads();
                const int nn = s->n_nodes;
                // ---- node windows: warps 0-3 issue, warps 4-7 build; then flush ----
                for (int u0 = 0; u0 < nn; u0 += kFlushNodes) {
                    const int cnt = min(kFlushNodes, nn - u0);
                    if (warp >= 4) {
                        build_batches<FMT>(a, s, sorted, offt, bmask, s->nodes + u0, cnt, q, n_cells);
                    } else if (lane == 0) {
                        issue_mmas(a, s, warp, s->nodes + u0, cnt, S, q, k0, n_mma, im_last);
                    }
                    S += cnt;
                    // warps 0-3 flush the accumulators while the builders go on with the next
                    // window's first operand batches (the flush touches none of their state;
                    // the operand buffers hand over through their mbarriers as always)
                    if (warp < 4) {
                        __syncwarp();
                        q = __shfl_sync(0xffffffffu, q, 0);   // the two roles agree unless a wait gave up
                        flush_acc(a, s, tm, flushes, k0, rows, npg, first);
                        // every accumulator lane is read and zeroed before an issuer starts the next window
                        asm volatile("bar.sync 2, 128;" ::: "memory");
                    }
                    first = false;
                }
                __syncthreads();                // the chunk's windows are done (the next chunk regenerates)
            }
            // a pass without records still writes its (zero) currents
            if (first) {
                if (warp < 4) flush_acc(a, s, tm, flushes, k0, rows, npg, true);
                __syncthreads();
            }
        }
    }
    // teardown: every MMA and bulk copy this CTA issued has landed before its tensor memory
    // and shared memory go (after an abort some may still be in flight)
    if (warp < 4) {
        if (lane == 0) mma_commit(&s->done);
        __syncwarp();
        bar_wait(s, &s->done, flushes & 1, true);
        if (lane == 0 && warp == 0)
            for (int b = 0; b < 2; ++b)
                if (im_last[b] >= 0) bar_wait(s, &s->full_im[b], (uint32_t)(im_last[b] >> 1) & 1, true);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s->abort) atomicOr(a.status, (unsigned long long)SIM_STATUS_TIMEOUT);
    if (warp < 4 && lane == 0 && n_mma) atomicAdd(a.status + 1, n_mma);
    if (warp >= 4) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_cells += __shfl_down_sync(0xffffffffu, n_cells, o);
        if (lane == 0 && n_cells) atomicAdd(a.status + 2, n_cells);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols) : "memory");
    }
}

// The table rows rounded to the operand type (x scale) by error diffusion, one
// thread per row, from the last tick (the arrival, where the row peaks)
// towards its start: each value is rounded together with the rounding error
// carried from the ticks after it.  Every suffix sum of the rounded row then
// equals the scaled FP32 one within half an operand ulp of a single value, so
// the charge a point induces from any tick on to its arrival, and in
// particular in all (the row's total), survives the rounding; independent
// rounding of each value would let those sums drift by ~1e-5..1e-4 of their
// value.  out: [nb2][L] operand bit patterns.
template <int FMT>
__global__ void k_round_rows(const float *lut, int ld, int L, int nb2, float scale, unsigned short *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nb2) return;
    const float *row = lut + (size_t)n * ld;
    unsigned short *o = out + (size_t)n * L;
    float carry = 0.f;
    for (int j = L - 1; j >= 0; --j) {
        const float v = __fadd_rn(__fmul_rn(row[j], scale), carry);
        float r;
        unsigned short bits;
        if (FMT == 0) {
            const __half h = __float2half_rn(fminf(fmaxf(v, -65504.f), 65504.f));
            r = __half2float(h);
            bits = __half_as_ushort(h);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            r = __bfloat162float(h);
            bits = __bfloat16_as_ushort(h);
        }
        carry = __fsub_rn(v, r);
        o[j] = bits;
    }
}

// Phase table of each rounded row, the A operands of all its MMAs in one
// buffer.  An MMA of block ab in tile t multiplies
//   A[m', a'] = R[128 t + 127 - m' - 16 ab - a' + L - 1]
// (m' = 127 - (tick - 128 t): accumulator rows run backwards in a tile) with
// the charge Q[p][16 ab + a'].  Writing S[x] = R[L + 126 - x] (zero outside
// the row), A[m', a'] = S[base + m' + a'], base = 16 ab - 128 t: constant
// along anti-diagonals, so 8 rows of 8 values B[q][phi][e] = S[8 q + phi + e]
// (phi, e < 8) per 128-byte block q hold every operand: the core matrix
// (m' / 8, a' / 8) starts at block base / 8 + m' / 8 + a' / 8, its row phi
// 16 bytes further.  One thread per 16-byte row; rtab: [nb2][L] operand bits.
__global__ void k_phase_table(const unsigned short *rtab, int L, int nb2, int nq, unsigned char *table)
{
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)nb2 * nq * 8) return;
    const int n = (int)(id / (nq * 8));
    const int rem = (int)(id - (int64_t)n * nq * 8);
    const int q = rem >> 3, phi = rem & 7;
    uint32_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int j = L + 126 - (8 * q + phi + e);
        v[e] = (j >= 0 && j < L) ? (uint32_t)rtab[(size_t)n * L + j] : 0u;     // +0 in both formats
    }
    uint4 o;
    o.x = v[0] | (v[1] << 16);
    o.y = v[2] | (v[3] << 16);
    o.z = v[4] | (v[5] << 16);
    o.w = v[6] | (v[7] << 16);
    *reinterpret_cast<uint4 *>(table + (size_t)n * nq * 128 + (size_t)rem * 16) = o;
}

int tc_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int rho0_of(int L) { return 16 * ((L + 126) / 16); }

struct TcLayout {
    size_t queue, table, rtab, recs, sorted, offt, bmask, perm, pwork, nsub, pos, nslice, spos, units, order, slices,
        scan, total;
};

TcLayout tc_layout(int grid, int64_t pix_cap, int T, int units_per_sm, int rec_chunk)
{
    TcLayout t;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += align256(b);
        return at;
    };
    const int64_t ng = (pix_cap + kGroup - 1) / kGroup;
    t.queue = take(256);                    // [0] queue, [8] work total, [16] units, [24] slices
    t.perm = take(sizeof(int32_t) * (size_t)pix_cap);
    t.pwork = take(sizeof(long long) * (size_t)pix_cap);
    t.nsub = take(sizeof(int32_t) * (size_t)ng);
    t.pos = take(sizeof(int32_t) * (size_t)(ng + 1));
    t.nslice = take(sizeof(int32_t) * (size_t)ng);
    t.spos = take(sizeof(int32_t) * (size_t)(ng + 1));
    t.units = take(sizeof(Unit) * (size_t)ng * kMaxSplit);
    t.order = take(sizeof(int32_t) * (size_t)ng * kMaxSplit);
    // split units number fewer than 2 * target (wcap rounded up), at most 16 per group
    const int64_t max_slices = std::min<int64_t>(2 * (int64_t)units_per_sm * grid, ng * kMaxSplit);
    t.slices = take(sizeof(float) * (size_t)max_slices * kGroup * (size_t)T);
    t.scan = take(scan_scratch_bytes(ng));
    t.table = take((size_t)kMaxBins * kMaxIm);
    t.rtab = take((size_t)kMaxBins * 2048 * sizeof(unsigned short));     // rounded rows, nt <= 2048
    t.recs = take((size_t)grid * rec_chunk * sizeof(Rec));
    t.sorted = take((size_t)grid * rec_chunk * sizeof(Rec));
    t.offt = take((size_t)grid * kGroup * (kMaxBins + 1) * sizeof(int));
    t.bmask = take((size_t)grid * kGroup * kMaxBins * 8 * sizeof(uint32_t));
    t.total = o;
    return t;
}

}  // namespace

size_t current_tc_scratch_bytes(int64_t pix_cap, int T, int units_per_sm, int rec_chunk)
{
    return tc_layout(tc_grid(), pix_cap > 0 ? pix_cap : 1, T, units_per_sm > 0 ? units_per_sm : kSubsPerSm,
                     rec_chunk > 0 ? rec_chunk : default_chunk(pix_cap > 0 ? pix_cap : 1))
        .total;
}

// Operand scales.  FP16: charge tiles in units of 4 e- (the fixed-point
// quantum 2^-12 e- becomes 2^-14, the smallest normal FP16 number: the tensor
// cores flush FP16 subnormals; cells above 262016 e- saturate) and table
// values x 2^15 (rows are normalised to 1; values down to ~2e-9 stay normal),
// products rescaled by 2^-13 when the accumulators are read.  BF16 has the
// FP32 exponent range: no scaling.
cudaError_t launch_induced_current_tc(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                      const sim_response &r, const int32_t *active, const int32_t *pix_seg_off,
                                      const int32_t *pix_seg_ids, const int64_t *counts, int64_t pix_cap,
                                      int64_t pix_begin, int64_t pix_end, float *current, void *scratch,
                                      cudaStream_t st)
{
    if (pix_cap <= 0) return cudaSuccess;
    const int fmt = c.precision == 1 ? 1 : 0;      // 1: BF16, 2: FP16
    const int grid = tc_grid();
    const int units_per_sm = c.tc_units_per_sm > 0 ? c.tc_units_per_sm : kSubsPerSm;
    const int rec_chunk = c.tc_record_chunk > 0 ? c.tc_record_chunk : default_chunk(pix_cap);
    const TcLayout lay = tc_layout(grid, pix_cap, c.n_ticks, units_per_sm, rec_chunk);
    char *p = reinterpret_cast<char *>(scratch);
    TcArgs a;
    a.c = c;
    a.nb = r.nb;
    a.nt = r.nt;
    a.bpp = r.bins_per_pitch;
    a.rho0 = rho0_of(r.nt);                         // the largest base of an MMA with a nonzero A tile
    const int nq = phase_blocks(r.nt);
    a.im_bytes = nq * 128;
    a.idesc = instr_desc(fmt, kTileM, kGroup);
    const float rscale = fmt == 0 ? 32768.f : 1.f, qunit = fmt == 0 ? 4.f : 1.f;
    a.qscale = 1.f / (kFix * qunit);
    a.out_scale = qunit / rscale;
    a.table = reinterpret_cast<const unsigned char *>(p + lay.table);
    a.anch = reinterpret_cast<const Anchor *>(d.anchors);
    a.active = active;
    a.off = pix_seg_off;
    a.segs = pix_seg_ids;
    int32_t *perm = reinterpret_cast<int32_t *>(p + lay.perm);
    a.perm = perm;
    a.counts = counts;
    a.status = reinterpret_cast<unsigned long long *>(const_cast<int64_t *>(counts) + 3);
    a.pix_cap = pix_cap;
    a.current = current;
    a.seed = c.seed;
    a.ev = events_of(s);
    a.g = geo_of(c);
    a.dp = drift_par_of(c);
    a.queue = reinterpret_cast<int *>(p + lay.queue);
    unsigned long long *wtotal = reinterpret_cast<unsigned long long *>(p + lay.queue + 8);
    int64_t *n_units = reinterpret_cast<int64_t *>(p + lay.queue + 16);
    int64_t *n_slices = reinterpret_cast<int64_t *>(p + lay.queue + 24);
    a.n_units = n_units;
    a.units = reinterpret_cast<const Unit *>(p + lay.units);
    a.order = reinterpret_cast<const int32_t *>(p + lay.order);
    a.slices = reinterpret_cast<float *>(p + lay.slices);
    a.recs = reinterpret_cast<Rec *>(p + lay.recs);
    a.sorted = reinterpret_cast<Rec *>(p + lay.sorted);
    a.offt = reinterpret_cast<int *>(p + lay.offt);
    a.bmask = reinterpret_cast<uint32_t *>(p + lay.bmask);
    a.rec_cap = rec_chunk;

    cudaError_t e = cudaMemsetAsync(a.queue, 0, 32, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.status + 1, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    // work plan
    const int64_t ng = (pix_cap + kGroup - 1) / kGroup;
    long long *pwork = reinterpret_cast<long long *>(p + lay.pwork);
    int32_t *nsub = reinterpret_cast<int32_t *>(p + lay.nsub);
    int32_t *pos = reinterpret_cast<int32_t *>(p + lay.pos);
    int32_t *nslice = reinterpret_cast<int32_t *>(p + lay.nslice);
    int32_t *spos = reinterpret_cast<int32_t *>(p + lay.spos);
    k_plan_perm<<<(unsigned)((pix_cap + 255) / 256), 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, active,
                                                                    a.g.npx_x, a.g.npx_y, perm);
    k_plan_work<<<(unsigned)((pix_cap + 255) / 256), 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, pix_seg_off,
                                                                    pix_seg_ids, perm, d.n_samples, c.mc_per_sample,
                                                                    pwork, wtotal);
    k_plan_split<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, pwork, wtotal,
                                                               units_per_sm * grid, nsub, nslice, ng);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_exclusive_scan(nsub, pos, ng, n_units, p + lay.scan, st);
    if (e == cudaSuccess) e = launch_exclusive_scan(nslice, spos, ng, n_slices, p + lay.scan, st);
    if (e != cudaSuccess) return e;
    k_plan_emit<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, pwork, nsub, pos,
                                                              spos, reinterpret_cast<Unit *>(p + lay.units), ng);
    k_plan_rank<<<(unsigned)((ng * kMaxSplit + 255) / 256), 256, 0, st>>>(a.units, n_units,
                                                                         reinterpret_cast<int32_t *>(p + lay.order));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb2 = r.nb * r.nb;
    const int64_t chunks = (int64_t)nb2 * nq * 8;
    const unsigned blocks = (unsigned)((chunks + 255) / 256);
    unsigned char *table = reinterpret_cast<unsigned char *>(p + lay.table);
    unsigned short *rtab = reinterpret_cast<unsigned short *>(p + lay.rtab);
    if (fmt == 1) k_round_rows<1><<<(nb2 + 63) / 64, 64, 0, st>>>(r.lut, r.ld, r.nt, nb2, rscale, rtab);
    else k_round_rows<0><<<(nb2 + 63) / 64, 64, 0, st>>>(r.lut, r.ld, r.nt, nb2, rscale, rtab);
    k_phase_table<<<blocks, 256, 0, st>>>(rtab, r.nt, nb2, nq, table);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(TcSmem) + 1024;
    auto kern = fmt == 1 ? k_induced_current_tc<1> : k_induced_current_tc<0>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_plan_reduce<<<(unsigned)ng, 256, 0, st>>>(counts, pix_cap, pix_begin, pix_end, nsub, spos, perm, a.slices,
                                                c.n_ticks, current, ng);
    return cudaGetLastError();
}

}  // namespace larsim
