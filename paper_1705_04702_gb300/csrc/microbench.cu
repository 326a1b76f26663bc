// Microbenchmarks that give the rooflines of the trace kernel the rates the
// measured-peaks file does not hold: FP64 and FP32 FMA issue rate, FP32->FP64
// conversion rate, random-address red.global.add.f64 throughput, and
// random-address FP32 gathers (the dust-density reads of a traversal).
#include <cuda_runtime.h>

#include "skirt_internal.cuh"

namespace skirt {
namespace {

template <typename T>
__global__ void fma_kernel(T* out, int iters, T seed)
{
    T a0 = seed + (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    const T b = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == (T)-12345) out[0] = s;  // keeps the chain alive
}

__global__ void cvt_kernel(double* out, int iters, float seed)
{
    float f0 = seed + threadIdx.x, f1 = f0 + 1.f, f2 = f0 + 2.f, f3 = f0 + 3.f;
    double acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    for (int i = 0; i < iters; ++i) {
        // each iteration: 4 FP32->FP64 and 4 FP64->FP32 conversions
        f0 = (float)((double)f0 * 1.0000001);
        f1 = (float)((double)f1 * 1.0000001);
        f2 = (float)((double)f2 * 1.0000001);
        f3 = (float)((double)f3 * 1.0000001);
    }
    acc0 = f0 + f1 + f2 + f3;
    if (acc0 + acc1 + acc2 + acc3 == -12345.0) out[0] = acc0;
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

__global__ void red_kernel(double* table, unsigned long long n, int per_thread)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < per_thread; ++i) {
        const unsigned long long idx = ((unsigned long long)hash32(t * 2654435761u + i * 97u) *
                                        (unsigned long long)hash32(i + 17u * t)) % n;
        atomicAdd(table + idx, 1.0);
    }
}

__global__ void gather_kernel(const float* __restrict__ table, unsigned long long n, int per_thread, float* out)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.f;
    uint32_t h = hash32(t);
    for (int i = 0; i < per_thread; ++i) {
        const unsigned long long idx = ((unsigned long long)h * 2654435761ull + (unsigned long long)(s > 1e30f)) % n;
        s += __ldg(table + idx);
        h = hash32(h + i);
    }
    if (s == -12345.f) out[0] = s;
}

}  // namespace
}  // namespace skirt

using namespace skirt;

extern "C" int skirt_microbench(int kind, long long size, double* rate, float* ms)
{
    if (!rate || !ms) return set_error(SKIRT_ERR_INVALID_ARG, "rate / ms is NULL");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(SKIRT_ERR_NO_DEVICE, "no device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    void* buf = nullptr;
    double ops = 0;
    const int block = 256, grid = sms * 8;
    const long long threads = (long long)block * grid;
    cudaError_t err = cudaSuccess;
    switch (kind) {
    case 0:
    case 1:
    case 2: {
        err = cudaMalloc(&buf, 64);
        if (err) break;
        const int iters = 4096;
        for (int rep = 0; rep < 2; ++rep) {  // first pass warms up
            cudaEventRecord(e0);
            if (kind == 0) fma_kernel<double><<<grid, block>>>((double*)buf, iters, 1.0);
            else if (kind == 1) fma_kernel<float><<<grid, block>>>((float*)buf, iters * 8, 1.0f);
            else cvt_kernel<<<grid, block>>>((double*)buf, iters, 1.0f);
            cudaEventRecord(e1);
        }
        ops = (double)threads * iters * 8 * (kind == 1 ? 8 : 1);  // FMAs, or conversions
        break;
    }
    case 3: {  // random FP64 reductions into a table of `size` doubles
        if (size < 1024) return set_error(SKIRT_ERR_INVALID_ARG, "size must be >= 1024");
        err = cudaMalloc(&buf, sizeof(double) * size);
        if (err) break;
        cudaMemset(buf, 0, sizeof(double) * size);
        const int per = 256;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0);
            red_kernel<<<grid, block>>>((double*)buf, (unsigned long long)size, per);
            cudaEventRecord(e1);
        }
        ops = (double)threads * per;
        break;
    }
    case 4: {  // random FP32 gathers from a table of `size` floats
        if (size < 1024) return set_error(SKIRT_ERR_INVALID_ARG, "size must be >= 1024");
        err = cudaMalloc(&buf, sizeof(float) * (size + 16));
        if (err) break;
        cudaMemset(buf, 0, sizeof(float) * (size + 16));
        const int per = 256;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0);
            gather_kernel<<<grid, block>>>((const float*)buf, (unsigned long long)size, per, (float*)buf + size);
            cudaEventRecord(e1);
        }
        ops = (double)threads * per;
        break;
    }
    default:
        return set_error(SKIRT_ERR_INVALID_ARG, "unknown microbenchmark %d", kind);
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    if (buf) cudaFree(buf);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return set_error(SKIRT_ERR_CUDA, "microbenchmark: %s", cudaGetErrorString(err));
    *ms = t;
    *rate = ops / (t * 1e-3);
    return SKIRT_OK;
}
