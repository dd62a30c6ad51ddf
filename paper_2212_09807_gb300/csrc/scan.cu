// scan.cu -- device-wide exclusive prefix sums used to build the CSR maps and
// to compact hits: tile reduce -> single-CTA scan of tile sums -> tile scan.
// Each tile is 2048 int32 (256 threads x 8 consecutive items, 32-byte
// vector loads); the whole pass moves ~3 x 4 bytes per element.
#include "sim_internal.cuh"

namespace larsim {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <bool kFlag>
__device__ __forceinline__ int32_t val(const int32_t *in, int64_t i, int64_t n)
{
    if (i >= n) return 0;
    const int32_t v = in[i];
    return kFlag ? (v > 0 ? 1 : 0) : v;
}

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread across the CTA; returns the prefix
// and writes the CTA total to *total.
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *smem, int32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t inc = warp_incl_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < (kThreads / 32) ? smem[lane] : 0;
        const int32_t wi = warp_incl_scan(w);
        if (lane < (kThreads / 32)) smem[lane] = wi - w;
        if (lane == (kThreads / 32) - 1) smem[kThreads / 32] = wi;
    }
    __syncthreads();
    const int32_t r = smem[warp] + inc - v;
    *total = smem[kThreads / 32];
    __syncthreads();
    return r;
}

template <bool kFlag>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const int32_t *in, int64_t n, int32_t *sums)
{
    __shared__ int32_t smem[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) s += val<kFlag>(in, base + k, n);
    int32_t tot;
    block_excl_scan(s, smem, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the tile sums in place (exclusive) and stores the grand total.
__global__ void __launch_bounds__(kThreads) k_scan_sums(int32_t *sums, int64_t nt, int64_t *total64,
                                                        int32_t *out_total)
{
    __shared__ int32_t smem[kThreads / 32 + 1];
    int32_t carry = 0;
    for (int64_t b = 0; b < nt; b += kThreads) {
        const int64_t i = b + threadIdx.x;
        const int32_t v = i < nt ? sums[i] : 0;
        int32_t tot;
        const int32_t e = block_excl_scan(v, smem, &tot);
        if (i < nt) sums[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (total64) *total64 = carry;
        *out_total = carry;
    }
}

template <bool kFlag>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const int32_t *in, int32_t *out, int64_t n,
                                                        const int32_t *sums)
{
    __shared__ int32_t smem[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int32_t v[kItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = val<kFlag>(in, base + k, n);
        s += v[k];
    }
    int32_t tot;
    int32_t run = block_excl_scan(s, smem, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

template <bool kFlag>
cudaError_t scan_impl(const int32_t *in, int32_t *out, int64_t n, int64_t *total64, void *scratch,
                      cudaStream_t st)
{
    const int64_t nt = (n + kTile - 1) / kTile;
    int32_t *sums = reinterpret_cast<int32_t *>(scratch);
    if (n > 0) {
        k_tile_reduce<kFlag><<<(unsigned)nt, kThreads, 0, st>>>(in, n, sums);
    }
    // out[n] receives the total; when n == 0 the sums loop is empty and the total is 0
    k_scan_sums<<<1, kThreads, 0, st>>>(sums, nt, total64, out + n);
    if (n > 0) {
        k_tile_scan<kFlag><<<(unsigned)nt, kThreads, 0, st>>>(in, out, n, sums);
    }
    return cudaGetLastError();
}
}  // namespace

size_t scan_scratch_bytes(int64_t n) { return align256(sizeof(int32_t) * (size_t)((n + kTile - 1) / kTile + 1)); }

cudaError_t launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int64_t *total64,
                                  void *scratch, cudaStream_t st)
{
    return scan_impl<false>(in, out, n, total64, scratch, st);
}

cudaError_t launch_flag_scan(const int32_t *in, int32_t *out, int64_t n, int64_t *total64,
                             void *scratch, cudaStream_t st)
{
    return scan_impl<true>(in, out, n, total64, scratch, st);
}

}  // namespace larsim
