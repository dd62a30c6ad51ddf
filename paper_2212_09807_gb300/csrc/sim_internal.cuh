// sim_internal.cuh -- device helpers shared by the sm_103a kernels of the
// charge-readout path (arXiv:2212.09807, Sec. 3) and host launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sim.h"

namespace larsim {

// ---------------------------------------------------------------- RNG ----
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications with word exchange and key mixing; key bumped by the two
// Weyl constants between rounds.
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1) from a 32-bit word: (x + 1/2) 2^-32, rounded to FP32.
__device__ __forceinline__ float u01f(uint32_t x)
{
    return __fmaf_rn(__uint2float_rn(x), 0x1p-32f, 0x1p-33f);
}

// Box-Muller pair from two words (library logf / sqrtf / sincospif).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b)
{
    const float r = sqrtf(-2.0f * logf(u01f(a)));
    float s, c;
    sincospif(2.0f * u01f(b), &s, &c);
    return make_float2(r * c, r * s);
}

// Four standard normals of Philox block (c0, c1, c2, c3) under key seed ^ event.
__device__ __forceinline__ float4 normals4(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2,
                                           uint32_t c3)
{
    const u32x4 x = philox4x32_10(u32x4{c0, c1, c2, c3}, (uint32_t)key, (uint32_t)(key >> 32));
    const float2 a = box_muller(x.x, x.y);
    const float2 b = box_muller(x.z, x.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// First two normals only (one Box-Muller pair).
__device__ __forceinline__ float2 normals2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2)
{
    const u32x4 x = philox4x32_10(u32x4{c0, c1, c2, 0u}, (uint32_t)key, (uint32_t)(key >> 32));
    return box_muller(x.x, x.y);
}

// Three normals (diffusion offsets): first pair plus the cosine of the second.
__device__ __forceinline__ float3 normals3(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2)
{
    const u32x4 x = philox4x32_10(u32x4{c0, c1, c2, 0u}, (uint32_t)key, (uint32_t)(key >> 32));
    const float2 a = box_muller(x.x, x.y);
    const float r = sqrtf(-2.0f * logf(u01f(x.z)));
    const float c = cospif(2.0f * u01f(x.w));
    return make_float3(a.x, a.y, r * c);
}

// ------------------------------------------------------ segment anchor ----
// Per-segment sampling record (64 bytes) written by k_quench_drift.  Positions
// are in pitch units relative to the centre-origin of a reference pixel
// (ix_ref, iy_ref) of the segment's anode; arrival ticks are relative to the
// integer tick A0 of the segment start.  Keeping every per-point quantity a
// small offset from an FP64-computed anchor keeps FP32 point arithmetic at
// ~1e-7 of a bin and of a tick.
struct __align__(16) Anchor {
    int32_t ix_ref, iy_ref, A0, N;   // reference pixel, start tick, points
    float fx0, fy0, dX, dY;          // start (pitch units from pixel corner) and extent
    float fa0, da, q, sTp;           // start tick fraction, ticks per unit u, charge per point, sigma_T/pitch
    float sLc, d0, dd, kz;           // signed sigma_L (cm), start drift distance and extent (cm), ticks/cm
};
static_assert(sizeof(Anchor) == SIM_ANCHOR_BYTES, "anchor record size");

struct Geo {
    int32_t npx_x, npx_y, n_anodes;
};

__host__ __device__ inline Geo geo_of(const sim_config &c)
{
    Geo g;
    g.npx_x = c.tiles_x * c.px_per_tile;
    g.npx_y = c.tiles_y * c.px_per_tile;
    g.n_anodes = c.n_mod_x * c.n_mod_y * c.n_tpc;
    return g;
}

// Events of a call: one event (n == 0, id `single`) or a batch of n event
// slots with device offsets [n + 1] and ids [n].  Slot s owns virtual anodes
// s * n_anodes .. and virtual pixels s * detector_pixels ...
struct EventInfo {
    const int64_t *off;
    const uint64_t *ids;
    int64_t n;
    uint64_t single;
};

inline EventInfo events_of(const sim_segments &s)
{
    EventInfo e;
    e.off = s.event_offsets;
    e.ids = s.event_ids;
    e.n = s.n_events;
    e.single = s.event_id;
    return e;
}

inline int64_t n_slots(const EventInfo &e) { return e.n > 0 ? e.n : 1; }

__host__ __device__ inline int64_t detector_pixels(const Geo &g) { return (int64_t)g.n_anodes * g.npx_x * g.npx_y; }

// Philox key of an event slot.
__device__ __forceinline__ uint64_t slot_key(uint64_t seed, const EventInfo &e, int slot)
{
    return seed ^ (e.n > 0 ? e.ids[slot] : e.single);
}

// First segment index of an event slot (0 for a single event).
__device__ __forceinline__ int64_t slot_first(const EventInfo &e, int slot) { return e.n > 0 ? e.off[slot] : 0; }

// Slot owning segment i: largest e with off[e] <= i.
__device__ __forceinline__ int slot_of_segment(const EventInfo &e, int64_t i)
{
    if (e.n <= 0) return 0;
    int lo = 0, hi = (int)e.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e.off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Map half-width in pitch units: table reach (nb + 1/2) bins plus the clip.
__device__ __forceinline__ float map_radius_pitch(int nb, int bpp, float clip, float sTp)
{
    return __fdiv_rn((float)nb + 0.5f, (float)bpp) + clip * sTp;
}

// ------------------------------------------------------- host launchers ----
// Each returns cudaSuccess or the launch error.
cudaError_t launch_quench_drift(const sim_config &c, const sim_segments &s, const sim_drifted &o,
                                cudaStream_t st);

size_t map_scratch_bytes(const sim_config &c, int64_t n_seg, int64_t slots);
cudaError_t launch_pixel_map(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                             int nb, int bins_per_pitch, int32_t *seg_pix_off, int32_t *seg_pix_ids,
                             int64_t pair_cap, int32_t *active, int32_t *pix_seg_off,
                             int32_t *pix_seg_ids, int64_t pix_cap, int64_t *counts, void *scratch,
                             cudaStream_t st);

// Induced current, FP32 form (precision 0) and tensor-core form
// (precision 1 BF16, 2 FP16 operands); same arguments.  Rows of the active
// pixels [pix_begin, min(counts[1], pix_end)) are computed.
size_t current_scratch_bytes(int64_t pix_cap);
bool current_table_ok(int nb, int nt);
cudaError_t launch_induced_current(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                   const sim_response &r, const int32_t *active,
                                   const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                                   const int64_t *counts, int64_t pix_cap, int64_t pix_begin, int64_t pix_end,
                                   float *current, void *scratch, cudaStream_t st);
// FP32 term-by-term form (precision 3): the per-record sum, same arguments.
size_t current_direct_scratch_bytes(int64_t pix_cap);
cudaError_t launch_induced_current_direct(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                          const sim_response &r, const int32_t *active,
                                          const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                                          const int64_t *counts, int64_t pix_cap, int64_t pix_begin, int64_t pix_end,
                                          float *current, void *scratch, cudaStream_t st);
size_t current_tc_scratch_bytes(int64_t pix_cap, int n_ticks, int units_per_sm, int rec_chunk);
cudaError_t launch_induced_current_tc(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                                      const sim_response &r, const int32_t *active,
                                      const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                                      const int64_t *counts, int64_t pix_cap, int64_t pix_begin, int64_t pix_end,
                                      float *current, void *scratch, cudaStream_t st);

size_t elec_scratch_bytes(const sim_config &c, int64_t pix_cap);
cudaError_t launch_electronics(const sim_config &c, const EventInfo &ev, const int32_t *active,
                               const float *current, int64_t *counts, int64_t pix_cap,
                               const sim_hits &out, void *scratch, cudaStream_t st);

// After the front end: table running sums, per-hit charge truth, hit points,
// track dQ/dx.
cudaError_t launch_response_cumulative(const sim_response &r, float *cum, cudaStream_t st);
cudaError_t launch_hit_truth(const sim_config &c, const sim_segments &s, const sim_drifted &d,
                             const sim_response &r, const float *cum, const int32_t *active,
                             const int32_t *pix_seg_off, const int32_t *pix_seg_ids, const int64_t *counts,
                             int64_t pix_cap, const sim_hits &hits, const sim_truth &out, int64_t max_cells,
                             void *ws, cudaStream_t st);
size_t hit_truth_workspace_bytes(int64_t hit_cap, int64_t max_cells);
cudaError_t launch_hit_points(const sim_config &c, const sim_hits &h, const float *t_event, float *x, float *y,
                              float *z, cudaStream_t st);
cudaError_t launch_track_dqdx(const float *x, const float *y, const float *z, const float *q, const int64_t *n,
                              int64_t cap, const double origin[3], const double dir[3], double piece, int32_t n_bins,
                              double r_max, double *dq, int32_t *count, cudaStream_t st);

// Light path (light.cu).
int light_n_det_total(const sim_config &c, const sim_light_config &lc);
int64_t light_n_samples(const sim_light_config &lc, double *ratio);
int light_n_trunc(const sim_light_config &lc);
cudaError_t launch_light_yield(const sim_config &c, const sim_light_config &lc, const sim_segments &s,
                               const sim_drifted &d, float *npe, int32_t *tick, int32_t *vox, cudaStream_t st);
cudaError_t launch_light_photocurrent(const sim_config &c, const sim_light_config &lc, const sim_segments &s,
                                      const sim_drifted &d, const float *npe, const int32_t *tick,
                                      const int32_t *vox, int64_t *pe, cudaStream_t st);
cudaError_t launch_light_scint(const sim_config &c, const sim_light_config &lc, const int64_t *pe, float *S,
                               cudaStream_t st);
cudaError_t launch_light_fluct(const sim_config &c, const sim_light_config &lc, uint64_t event_id, const float *S,
                               float *out, cudaStream_t st);
cudaError_t launch_light_truth(const sim_light_config &lc, int64_t n, const int32_t *tick, const int32_t *vox,
                               float *t_arr, cudaStream_t st);
cudaError_t launch_light_electronics(const sim_config &c, const sim_light_config &lc, uint64_t event_id,
                                     const float *pe_obs, float *V, uint16_t *wave, cudaStream_t st);

// Exclusive scan of int32 `in[0..n)` into `out[0..n]` (out[n] = total) with
// the total also stored to *total64 when non-null.  In place allowed.
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int64_t *total64,
                                  void *scratch, cudaStream_t st);

// Exclusive scan of the flags (in[i] > 0).
cudaError_t launch_flag_scan(const int32_t *in, int32_t *out, int64_t n, int64_t *total64,
                             void *scratch, cudaStream_t st);

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace larsim
