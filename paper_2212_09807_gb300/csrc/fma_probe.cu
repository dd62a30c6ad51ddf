// fma_probe.cu -- measurement support, not a step of the method: a kernel
// that issues only independent FP32 fused multiply-adds, so that its rate is
// the device's FP32 FMA throughput.  The benchmark divides the FP32 form's
// algorithmic flops by this measured rate (its "alu" roofline).
#include "sim_internal.cuh"

namespace larsim {
namespace {

constexpr int kChains = 8;           // independent dependency chains per thread (hides the FMA latency)

__global__ void __launch_bounds__(256) k_fma_probe(int iters, float seed, float *out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + (float)(threadIdx.x * kChains + c) * 1e-7f;
    const float a = 0.999999f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace
int abi_cuda_fail(cudaError_t e);   // api.cu
}  // namespace larsim

using namespace larsim;

extern "C" int sim_probe_fma(int64_t blocks, int32_t iters, float *sink, double *flops, void *stream)
{
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || !sink || !flops) return SIM_ERR_INVALID_ARG;
    k_fma_probe<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(iters, 1.0f, sink);
    *flops = 2.0 * (double)blocks * 256.0 * (double)iters * 16.0 * kChains;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIM_OK : abi_cuda_fail(e);
}
