// Dust-cell source (dust emission phase, Sect. 3.2): a packet at wavelength
// j starts in cell m with probability emission[m][j] / sum_m emission[m][j].
// This file builds, per wavelength, the normalised cumulative distribution
// over the cells: the [cell][wavelength] emission table is transposed into
// [wavelength][cell] rows (the single-device counterpart of switching the
// table from row to column representation, Sect. 5.2) and every row is
// prefix-summed in FP64 with a three-pass tiled scan.
#include <cuda_runtime.h>

#include <vector>

#include "skirt_internal.cuh"

namespace skirt {
namespace {

constexpr int TILE = 2048;   // cells per scan tile
constexpr int SCAN_T = 256;  // threads per scan block (8 cells each)

__global__ void transpose_kernel(const double* __restrict__ em, double* __restrict__ out, long long ncell,
                                 int nl, unsigned int* bad)
{
    __shared__ double t[32][33];
    const long long m0 = (long long)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long m = m0 + r;
        const int j = j0 + threadIdx.x;
        double v = 0.0;
        if (m < ncell && j < nl) {
            v = em[m * nl + j];
            if (!(v >= 0.0) || !isfinite(v)) {
                atomicOr(bad, 1u);
                v = 0.0;
            }
        }
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const long long m = m0 + threadIdx.x;
        if (m < ncell && j < nl) out[(size_t)j * ncell + m] = t[threadIdx.x][r];
    }
}

// inclusive scan of the 8*SCAN_T values held 8 per thread; returns the block total
__device__ double block_scan8(double v[8], double* sh)
{
#pragma unroll
    for (int i = 1; i < 8; ++i) v[i] += v[i - 1];
    double x = v[7];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        double s = lane < SCAN_T / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_T / 32) sh[lane] = s;
    }
    __syncthreads();
    const double before = (w > 0 ? sh[w - 1] : 0.0) + (x - v[7]);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] += before;
    const double total = sh[SCAN_T / 32 - 1];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_T) tile_sum_kernel(const double* __restrict__ rows, double* __restrict__ tsum,
                                                          long long ncell, int ntiles)
{
    __shared__ double sh[SCAN_T / 32];
    const int j = blockIdx.y, t = blockIdx.x;
    const double* row = rows + (size_t)j * ncell;
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long m = (long long)t * TILE + threadIdx.x * 8 + i;
        v[i] = m < ncell ? row[m] : 0.0;
    }
    const double total = block_scan8(v, sh);
    if (threadIdx.x == 0) tsum[(size_t)j * ntiles + t] = total;
}

// exclusive scan of the tile sums of one wavelength (one block per wavelength)
__global__ void __launch_bounds__(SCAN_T) tile_offset_kernel(double* __restrict__ tsum, double* __restrict__ totals,
                                                             int ntiles)
{
    __shared__ double sh[SCAN_T / 32];
    const int j = blockIdx.x;
    double* ts = tsum + (size_t)j * ntiles;
    double carry = 0.0;
    for (int base = 0; base < ntiles; base += TILE) {
        double v[8], orig[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = base + threadIdx.x * 8 + i;
            orig[i] = v[i] = k < ntiles ? ts[k] : 0.0;
        }
        const double total = block_scan8(v, sh);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = base + threadIdx.x * 8 + i;
            if (k < ntiles) ts[k] = carry + v[i] - orig[i];
        }
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[j] = carry;
}

__global__ void __launch_bounds__(SCAN_T) tile_scan_kernel(double* __restrict__ rows, const double* __restrict__ toff,
                                                           const double* __restrict__ totals, long long ncell,
                                                           int ntiles)
{
    __shared__ double sh[SCAN_T / 32];
    const int j = blockIdx.y, t = blockIdx.x;
    double* row = rows + (size_t)j * ncell;
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long m = (long long)t * TILE + threadIdx.x * 8 + i;
        v[i] = m < ncell ? row[m] : 0.0;
    }
    block_scan8(v, sh);
    const double off = toff[(size_t)j * ntiles + t];
    const double tot = totals[j];
    const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long m = (long long)t * TILE + threadIdx.x * 8 + i;
        if (m < ncell) row[m] = (m == ncell - 1) ? 1.0 : fmin((off + v[i]) * inv, 1.0);
    }
}

}  // namespace

int build_dust_cdf(skirt_grid_s* g, const double* emission, int nl, const uint64_t* npk, cudaStream_t s,
                   std::vector<double>* totals_out)
{
    const long long ncell = g->ncell;
    const int ntiles = (int)((ncell + TILE - 1) / TILE);
    cudaError_t e;
    if ((e = g->cdf.ensure(sizeof(double) * (size_t)nl * ncell)) != cudaSuccess)
        return set_error(SKIRT_ERR_OOM, "dust cdf: %s", cudaGetErrorString(e));
    const size_t aux = sizeof(double) * ((size_t)nl * ntiles + nl) + 256;
    if ((e = g->cdf_aux.ensure(aux)) != cudaSuccess) return set_error(SKIRT_ERR_OOM, "dust cdf aux: %s", cudaGetErrorString(e));
    double* rows = (double*)g->cdf.p;
    double* tsum = (double*)g->cdf_aux.p;
    double* totals = tsum + (size_t)nl * ntiles;
    unsigned int* bad = (unsigned int*)(totals + nl);
    if ((e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s)) != cudaSuccess)
        return set_error(SKIRT_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    dim3 tb(32, 8), tg((unsigned)((ncell + 31) / 32), (unsigned)((nl + 31) / 32));
    transpose_kernel<<<tg, tb, 0, s>>>(emission, rows, ncell, nl, bad);
    tile_sum_kernel<<<dim3(ntiles, nl), SCAN_T, 0, s>>>(rows, tsum, ncell, ntiles);
    tile_offset_kernel<<<nl, SCAN_T, 0, s>>>(tsum, totals, ntiles);
    tile_scan_kernel<<<dim3(ntiles, nl), SCAN_T, 0, s>>>(rows, tsum, totals, ncell, ntiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(SKIRT_ERR_CUDA, "dust cdf kernels: %s", cudaGetErrorString(e));
    std::vector<double> h(nl + 1);
    if ((e = cudaMemcpyAsync(h.data(), totals, sizeof(double) * nl + sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return set_error(SKIRT_ERR_CUDA, "dust cdf totals: %s", cudaGetErrorString(e));
    unsigned int badv = 0;
    memcpy(&badv, h.data() + nl, sizeof badv);
    if (badv) return set_error(SKIRT_ERR_INVALID_ARG, "dust emission holds negative or non-finite values");
    for (int j = 0; j < nl; ++j)
        if (npk[j] > 0 && !(h[j] > 0.0 && isfinite(h[j])))
            return set_error(SKIRT_ERR_INVALID_ARG, "dust emission at wavelength %d is zero but has packets", j);
    if (totals_out) totals_out->assign(h.begin(), h.begin() + nl);
    return SKIRT_OK;
}

}  // namespace skirt
