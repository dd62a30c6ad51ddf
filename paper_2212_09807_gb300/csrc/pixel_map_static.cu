// pixel_map_static.cu -- an allocation-free variant of sim_pixel_map.
//
// sim_pixel_map needs scratch memory (a per-pixel histogram, its prefix sums
// and the scan's tile sums) that the caller normally provides as workspace.
// Some callers cannot obtain device memory at the time they map an event:
// processes that reserve their whole device budget at start-up and may not
// allocate inside their event loop (online trigger and data-acquisition
// services are built this way), or code running inside a host framework whose
// own allocator owns every device buffer.  For them this file keeps the
// scratch in a fixed file-scope device array, so the call allocates nothing:
// no cudaMalloc, no cudaFree, no allocating library routine.
//
// The array costs SIM_NOALLOC_SCRATCH_BYTES of memory on every device that
// loads this library, for the life of the process.  All calls share it: the
// kernels clear what must start at zero on every call, and calls whose work
// overlaps on the GPU (different streams, or different host threads without
// ordering) race on it and must be serialised by the caller.
#include <mutex>

#include "sim_internal.cuh"

namespace larsim {
// defined in api.cu
bool abi_config_ok(const sim_config *c);
bool abi_segments_ok(const sim_segments *s);
bool abi_events_ok(const sim_config *c, const sim_segments *s);
bool abi_drifted_ok(const sim_drifted *d);
bool abi_response_ok(const sim_response *r, bool need_table);
int abi_cuda_fail(cudaError_t e);
}  // namespace larsim

using namespace larsim;

namespace {

static __device__ __align__(256) unsigned char g_map_scratch[SIM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];   // device address of g_map_scratch, per device

// In host code `g_map_scratch` names a host-side stand-in, not device memory,
// so the device address is looked up once per device (with that device
// current) and cached.  The cached address belongs to the device's context:
// after cudaDeviceReset it is stale (the process must not call this entry
// point on that device again).
int scratch_for_current_device(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return abi_cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return SIM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_map_scratch);
        if (e != cudaSuccess) return abi_cuda_fail(e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SIM_OK;
}

}  // namespace

extern "C" int sim_pixel_map_noalloc(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                                     const sim_response *resp, int32_t *seg_pix_off, int32_t *seg_pix_ids,
                                     int64_t pair_cap, int32_t *active_pixels, int32_t *pix_seg_off,
                                     int32_t *pix_seg_ids, int64_t pix_cap, int64_t *counts, void *stream)
{
    if (!abi_config_ok(cfg) || !abi_segments_ok(seg) || !abi_events_ok(cfg, seg) || !abi_response_ok(resp, false) ||
        pair_cap < 0 || pix_cap < 0 || !counts)
        return SIM_ERR_INVALID_ARG;
    if (seg->n > 0 && !abi_drifted_ok(dr)) return SIM_ERR_INVALID_ARG;
    if (!seg_pix_off || (pair_cap > 0 && (!seg_pix_ids || !pix_seg_ids)) || !pix_seg_off ||
        (pix_cap > 0 && !active_pixels))
        return SIM_ERR_INVALID_ARG;
    if (map_scratch_bytes(*cfg, seg->n, n_slots(events_of(*seg))) > SIM_NOALLOC_SCRATCH_BYTES) return SIM_ERR_CAPACITY;
    void *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != SIM_OK) return rc;
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    const cudaError_t e = launch_pixel_map(*cfg, *seg, d0, resp->nb, resp->bins_per_pitch, seg_pix_off, seg_pix_ids,
                                           pair_cap, active_pixels, pix_seg_off, pix_seg_ids, pix_cap, counts,
                                           scratch, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : abi_cuda_fail(e);
}
