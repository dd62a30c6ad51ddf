// pixel_map.cu -- step 3 of the charge path (arXiv:2212.09807 Sec. 3.3.2:
// the pixels each segment can induce on), and its transpose to a
// pixel -> segment CSR used by the pixel-centric induced-current kernel.
//
// Pixel p of the segment's anode is mapped iff the segment's x-y projection
// comes within Chebyshev distance R = (nb + 1/2) h + clip sigma_T of the pixel
// centre (table reach plus diffusion clip).  Enumeration walks the pixel rows
// the segment's band can touch; for each row the t-interval where the row
// condition holds bounds the x-range, so only mapped pixels are visited.
//
// Passes: count (+ pixel histogram) -> scan(seg counts) -> scan(flags) ->
// scan(histogram) -> compact active pixels -> fill both CSRs -> sort each
// pixel's segment list (so the current is summed in a fixed order).
#include "sim_internal.cuh"

namespace larsim {

namespace {

template <class F>
__device__ __forceinline__ int for_each_mapped(const Anchor &a, int anode, const Geo &g, float Rp, F &&f)
{
    const float y_lo = fminf(a.fy0, a.fy0 + a.dY) - Rp;
    const float y_hi = fmaxf(a.fy0, a.fy0 + a.dY) + Rp;
    const int j_lo = max((int)ceilf(y_lo - 0.5f), -a.iy_ref);
    const int j_hi = min((int)floorf(y_hi - 0.5f), g.npx_y - 1 - a.iy_ref);
    const int64_t base = (int64_t)anode * g.npx_x * g.npx_y;
    int cnt = 0;
    for (int j = j_lo; j <= j_hi; ++j) {
        const float cy = (float)j + 0.5f;
        float t0 = 0.f, t1 = 1.f;
        if (a.dY != 0.f) {
            const float ta = (cy - Rp - a.fy0) / a.dY;
            const float tb = (cy + Rp - a.fy0) / a.dY;
            t0 = fmaxf(0.f, fminf(ta, tb));
            t1 = fminf(1.f, fmaxf(ta, tb));
            if (t0 > t1) continue;
        } else if (fabsf(a.fy0 - cy) > Rp) {
            continue;
        }
        const float xa = a.fx0 + t0 * a.dX;
        const float xb = a.fx0 + t1 * a.dX;
        const float x_lo = fminf(xa, xb) - Rp;
        const float x_hi = fmaxf(xa, xb) + Rp;
        const int i_lo = max((int)ceilf(x_lo - 0.5f), -a.ix_ref);
        const int i_hi = min((int)floorf(x_hi - 0.5f), g.npx_x - 1 - a.ix_ref);
        const int64_t row = base + (int64_t)(a.iy_ref + j) * g.npx_x + a.ix_ref;
        for (int i = i_lo; i <= i_hi; ++i) {
            f((int32_t)(row + i), cnt);
            ++cnt;
        }
    }
    return cnt;
}

struct MapArgs {
    const Anchor *anch;
    const int32_t *anode;
    int64_t n;
    Geo g;
    int nb, bpp;
    float clip;
};

__global__ void __launch_bounds__(256) k_map_count(MapArgs m, int32_t *seg_count, int32_t *hist)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m.n) return;
    const int an = m.anode[s];
    int cnt = 0;
    if (an >= 0) {
        const Anchor a = m.anch[s];
        const float Rp = map_radius_pitch(m.nb, m.bpp, m.clip, a.sTp);
        cnt = for_each_mapped(a, an, m.g, Rp, [&](int32_t pid, int) { atomicAdd(hist + pid, 1); });
    }
    seg_count[s] = cnt;
}

__global__ void k_map_status(int64_t *counts, int64_t pair_cap, int64_t pix_cap)
{
    int64_t st = 0;
    if (counts[0] > pair_cap) st |= SIM_STATUS_PAIR_OVERFLOW;
    if (counts[1] > pix_cap) st |= SIM_STATUS_PIXEL_OVERFLOW;
    counts[3] = st;
}

__global__ void __launch_bounds__(256) k_map_compact(const int32_t *hist_flag_scan, const int32_t *cursor,
                                                     const int32_t *flags_src, int64_t n_total,
                                                     const int64_t *counts, int32_t *active,
                                                     int32_t *pix_seg_off)
{
    if (counts[3] != 0) return;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) pix_seg_off[counts[1]] = (int32_t)counts[0];
    if (p >= n_total) return;
    // flags_src[p] > 0 iff pixel p has at least one segment
    const int32_t a = hist_flag_scan[p];
    if (hist_flag_scan[p + 1] != a) {
        (void)flags_src;
        active[a] = (int32_t)p;
        pix_seg_off[a] = cursor[p];
    }
}

__global__ void __launch_bounds__(256) k_map_fill(MapArgs m, const int64_t *counts, const int32_t *seg_off,
                                                  int32_t *seg_pix_ids, int32_t *cursor,
                                                  int32_t *pix_seg_ids)
{
    if (counts[3] != 0) return;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m.n) return;
    const int an = m.anode[s];
    if (an < 0) return;
    const Anchor a = m.anch[s];
    const float Rp = map_radius_pitch(m.nb, m.bpp, m.clip, a.sTp);
    int32_t *dst = seg_pix_ids + seg_off[s];
    for_each_mapped(a, an, m.g, Rp, [&](int32_t pid, int k) {
        dst[k] = pid;
        const int32_t pos = atomicAdd(cursor + pid, 1);
        pix_seg_ids[pos] = (int32_t)s;
    });
}

// Insertion sort of each pixel's segment list (lists are short: O(10-100)).
constexpr int kSortMax = 8192;                  // longest list sorted in shared memory

// Each pixel's segment list in increasing order (the current is summed in this
// order).  A CTA takes 256 pixels: lists of up to 32 entries are sorted by
// their own thread (insertion sort), longer ones by the whole CTA, one after
// the other, with a bitonic sort in shared memory (lists beyond kSortMax,
// which the configurations here never reach, fall back to the thread's
// insertion sort).  The sorted order is unique: the result is deterministic.
__global__ void __launch_bounds__(256) k_map_sort(const int64_t *counts, const int32_t *pix_seg_off,
                                                  int32_t *pix_seg_ids)
{
    __shared__ int32_t buf[kSortMax];
    __shared__ int long_list[256];
    __shared__ int n_long;
    if (counts[3] != 0) return;
    const int64_t np = counts[1];
    const int tid = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < np; base += (int64_t)gridDim.x * blockDim.x) {
        if (tid == 0) n_long = 0;
        __syncthreads();
        const int64_t i = base + tid;
        if (i < np) {
            int32_t *v = pix_seg_ids + pix_seg_off[i];
            const int n = pix_seg_off[i + 1] - pix_seg_off[i];
            if (n > 32 && n <= kSortMax) {
                long_list[atomicAdd(&n_long, 1)] = tid;
            } else {
                for (int a = 1; a < n; ++a) {
                    const int32_t x = v[a];
                    int b = a - 1;
                    while (b >= 0 && v[b] > x) {
                        v[b + 1] = v[b];
                        --b;
                    }
                    v[b + 1] = x;
                }
            }
        }
        __syncthreads();
        for (int q = 0; q < n_long; ++q) {
            const int64_t pi = base + long_list[q];
            int32_t *v = pix_seg_ids + pix_seg_off[pi];
            const int n = pix_seg_off[pi + 1] - pix_seg_off[pi];
            int P = 64;
            while (P < n) P <<= 1;
            for (int j = tid; j < P; j += blockDim.x) buf[j] = j < n ? v[j] : INT_MAX;
            __syncthreads();
            for (int k = 2; k <= P; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int t = tid; t < P; t += blockDim.x) {
                        const int u = t ^ j;
                        if (u > t) {
                            const int32_t x = buf[t], y = buf[u];
                            if (((t & k) == 0) == (x > y)) {
                                buf[t] = y;
                                buf[u] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int j = tid; j < n; j += blockDim.x) v[j] = buf[j];
            __syncthreads();
        }
    }
}

}  // namespace

// Pixel ids of the (virtual) detector: one copy of the geometry per event slot.
static int64_t n_total_pixels(const sim_config &c, int64_t slots)
{
    return detector_pixels(geo_of(c)) * slots;
}

size_t map_scratch_bytes(const sim_config &c, int64_t n_seg, int64_t slots)
{
    const int64_t nt = n_total_pixels(c, slots);
    const int64_t big = nt > n_seg ? nt : n_seg;
    return 2 * align256(sizeof(int32_t) * (size_t)(nt + 1)) + scan_scratch_bytes(big + 1);
}

cudaError_t launch_pixel_map(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                             int nb, int bins_per_pitch, int32_t *seg_pix_off, int32_t *seg_pix_ids,
                             int64_t pair_cap, int32_t *active, int32_t *pix_seg_off,
                             int32_t *pix_seg_ids, int64_t pix_cap, int64_t *counts, void *scratch,
                             cudaStream_t st)
{
    const int64_t nt = n_total_pixels(c, n_slots(events_of(s)));
    char *p = reinterpret_cast<char *>(scratch);
    int32_t *hist = reinterpret_cast<int32_t *>(p);
    p += align256(sizeof(int32_t) * (size_t)(nt + 1));
    int32_t *flags = reinterpret_cast<int32_t *>(p);
    p += align256(sizeof(int32_t) * (size_t)(nt + 1));
    void *scan_ws = p;

    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)(nt + 1), st);
    if (e != cudaSuccess) return e;
    MapArgs m;
    m.anch = reinterpret_cast<const Anchor *>(d.anchors);
    m.anode = d.anode;
    m.n = s.n;
    m.g = geo_of(c);
    m.nb = nb;
    m.bpp = bins_per_pitch;
    m.clip = c.diff_clip_sigma;
    const int T = 256;
    const unsigned gs = (unsigned)((s.n + T - 1) / T);
    const unsigned gp = (unsigned)((nt + T - 1) / T);
    if (s.n > 0) k_map_count<<<gs, T, 0, st>>>(m, seg_pix_off, hist);
    // pairs: segment counts -> offsets (total to counts[0])
    e = launch_exclusive_scan(seg_pix_off, seg_pix_off, s.n, counts + 0, scan_ws, st);
    if (e != cudaSuccess) return e;
    // active pixels: flags of the histogram -> index (total to counts[1])
    e = launch_flag_scan(hist, flags, nt, counts + 1, scan_ws, st);
    if (e != cudaSuccess) return e;
    k_map_status<<<1, 1, 0, st>>>(counts, pair_cap, pix_cap);
    // histogram -> per-pixel start offsets (cursor), in place
    e = launch_exclusive_scan(hist, hist, nt, nullptr, scan_ws, st);
    if (e != cudaSuccess) return e;
    k_map_compact<<<gp, T, 0, st>>>(flags, hist, nullptr, nt, counts, active, pix_seg_off);
    if (s.n > 0) k_map_fill<<<gs, T, 0, st>>>(m, counts, seg_pix_off, seg_pix_ids, hist, pix_seg_ids);
    const unsigned gpc = (unsigned)((pix_cap + T - 1) / T);
    if (pix_cap > 0) k_map_sort<<<gpc, T, 0, st>>>(counts, pix_seg_off, pix_seg_ids);
    return cudaGetLastError();
}

}  // namespace larsim
