// The device random-number generator as a C-ABI call: Philox4x32-10 (Salmon
// et al., SC'11) evaluated by the same inline function the trace kernels draw
// their Monte Carlo samples with (Sect. 3.2: launch positions, interaction
// points and directions are sampled), so that it can be checked against the
// generator's published known answers.
#include <cuda_runtime.h>

#include <vector>

#include "skirt_internal.cuh"

namespace skirt {
namespace {

__global__ void philox_kernel(const uint4* __restrict__ ctr, const uint2* __restrict__ key, uint4* __restrict__ out,
                              int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox10(ctr[i], key[i].x, key[i].y);
}

}  // namespace
}  // namespace skirt

using namespace skirt;

extern "C" int skirt_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    if (n < 0 || n > (1 << 24)) return set_error(SKIRT_ERR_INVALID_ARG, "n must be in [0, 2^24]");
    if (n == 0) return SKIRT_OK;
    if (!ctr || !key || !out) return set_error(SKIRT_ERR_INVALID_ARG, "ctr / key / out is NULL");
    if (int r = check_device()) return r;
    const size_t bc = sizeof(uint4) * (size_t)n, bk = sizeof(uint2) * (size_t)n;
    unsigned char* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, 2 * bc + bk);
    if (e != cudaSuccess) return set_error(SKIRT_ERR_OOM, "philox buffers: %s", cudaGetErrorString(e));
    uint4* d_ctr = (uint4*)d;
    uint4* d_out = (uint4*)(d + bc);
    uint2* d_key = (uint2*)(d + 2 * bc);
    if ((e = cudaMemcpy(d_ctr, ctr, bc, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemcpy(d_key, key, bk, cudaMemcpyHostToDevice)) == cudaSuccess) {
        philox_kernel<<<(n + 255) / 256, 256>>>(d_ctr, d_key, d_out, n);
        if ((e = cudaGetLastError()) == cudaSuccess) e = cudaMemcpy(out, d_out, bc, cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    if (e != cudaSuccess) return set_error(SKIRT_ERR_CUDA, "philox: %s", cudaGetErrorString(e));
    return SKIRT_OK;
}
