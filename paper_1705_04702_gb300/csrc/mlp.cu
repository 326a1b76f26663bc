// MLP surrogate of the dust-emission step: 32 band features -> 128 -> 128 ->
// 100 emission-shape logits (SiLU, SiLU, softmax).
//
// Inference (mlp_infer_kernel): one warp per 16 rows, the three layers as
// BF16 tensor-core products with FP32 accumulation (mma.sync m16n8k16 in
// inline PTX); weights staged once per block in shared memory; the FP32
// accumulator fragment of one layer, passed through SiLU and packed to BF16,
// is exactly the A-operand fragment of the next layer, so activations never
// leave registers.  Softmax over the 100 outputs is reduced across the four
// lanes that hold a row; the result times the cell's absorbed power is
// written as FP64 emission.  The same pass flags rows whose raw features
// leave the training hull.
//
// Training (skirt_mlp_train): FP32 master weights; every step is one fused
// tensor-core kernel per 32 rows (forward, softmax cross-entropy, backward,
// weight-gradient products; mlp_train.cu) and one kernel that sums the
// partial gradients in order, takes the Adam step (cosine step decay) and
// refreshes the BF16 weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "skirt_internal.cuh"

namespace skirt {
namespace {

constexpr int NIN = SKIRT_NBANDS;      // 32
constexpr int NH = SKIRT_MLP_HIDDEN;   // 128
constexpr int NO = SKIRT_NEMIT;        // 100
constexpr int NO_PAD = 104;            // 13 n-tiles of 8
constexpr int NPARAM = SKIRT_MLP_NPARAM;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH;
static_assert(OFF_B3 + NO == NPARAM, "packed parameter layout");

#define MCK(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return set_error(e_ == cudaErrorMemoryAllocation ? SKIRT_ERR_OOM : SKIRT_ERR_CUDA,          \
                             "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// --------------------------------------------------------------------------
// inference
// --------------------------------------------------------------------------
constexpr int INF_WARPS = 8;
constexpr int INF_ROWS = 16 * INF_WARPS;
// shared memory: W1 [128][32], W2 [128][128], W3 [104][128] (bf16) with
// every row padded by 8 elements, so that the eight rows one fragment load
// touches start 4 banks apart (conflict-free); biases [128 + 128 + 104]
// (fp32); mean / inv_std / lo / hi [32] each; per-warp feature staging
constexpr int KP1 = NIN + 8, KP2 = NH + 8;
constexpr size_t SM_W1 = 0;
constexpr size_t SM_W2 = SM_W1 + sizeof(uint16_t) * NH * KP1;
constexpr size_t SM_W3 = SM_W2 + sizeof(uint16_t) * NH * KP2;
constexpr size_t SM_B = SM_W3 + sizeof(uint16_t) * NO_PAD * KP2;
constexpr size_t SM_ST = SM_B + sizeof(float) * (NH + NH + NO_PAD);
// per warp: two 16-row feature tiles [16][32] fp32 that the bulk copy engine
// fills asynchronously (128-byte aligned), and their two mbarriers
constexpr size_t SM_X = (SM_ST + sizeof(float) * 4 * NIN + 127) & ~(size_t)127;
constexpr size_t SM_BAR = SM_X + sizeof(float) * INF_WARPS * 2 * 16 * NIN;
constexpr size_t SM_TOTAL = SM_BAR + sizeof(unsigned long long) * INF_WARPS * 2;
static_assert((KP1 * 2) % 16 == 0 && (KP2 * 2) % 16 == 0, "padded rows keep 16-byte alignment");

// Bulk asynchronous copies (global -> shared) completing on an mbarrier, in
// inline PTX.  Waits are bounded: a wait that runs out sets g_mlp_timeout and
// the kernel stops instead of spinning on.
__device__ unsigned g_mlp_timeout;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// orders this thread's earlier generic accesses to shared memory before later
// asynchronous-proxy writes (the next bulk copy into a buffer just read)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    for (int i = 0; i < (1 << 20); ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// FP32 -> FP64 for a non-negative float by IEEE-754 field manipulation on the
// integer pipe (exact for normal floats; zero and subnormals map to zero), so
// that the epilogue issues no FP64-pipe instruction; infinities, NaN and
// negative values take the ordinary conversion
__device__ __forceinline__ double widen_pos(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = u >> 23;
    if (e >= 255u) return (double)f;
    return e ? __hiloint2double((int)((u >> 3) + 0x38000000u), (int)(u << 29)) : 0.0;
}

// acc[j][0..3] for n-tiles j: rows (g, g+8), cols 8j + 2t + {0,1}; produces
// the next layer's A fragments: k-tile kk from n-tiles 2kk, 2kk+1
template <int NT>
__device__ __forceinline__ void to_afrag(const float (&acc)[NT][4], uint32_t (&a)[NT / 2][4])
{
#pragma unroll
    for (int kk = 0; kk < NT / 2; ++kk) {
        a[kk][0] = pack_bf16(silu_f(acc[2 * kk][0]), silu_f(acc[2 * kk][1]));
        a[kk][1] = pack_bf16(silu_f(acc[2 * kk][2]), silu_f(acc[2 * kk][3]));
        a[kk][2] = pack_bf16(silu_f(acc[2 * kk + 1][0]), silu_f(acc[2 * kk + 1][1]));
        a[kk][3] = pack_bf16(silu_f(acc[2 * kk + 1][2]), silu_f(acc[2 * kk + 1][3]));
    }
}

// one layer: out[NT] n-tiles = A (KT k-tiles) x W^T, W [rows = 8*NT][cols = 16*KT] bf16 in smem
// with row stride KP elements
template <int NT, int KT, int KP>
__device__ __forceinline__ void layer(const uint32_t (&a)[KT][4], const uint16_t* __restrict__ W,
                                      const float* __restrict__ bias, float (&out)[NT][4], int g, int t)
{
    constexpr int K = KP;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
        out[j][0] = b0; out[j][1] = b1; out[j][2] = b0; out[j][3] = b1;
        const uint16_t* wr = W + (size_t)(8 * j + g) * K + 2 * t;
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const uint32_t b0w = *reinterpret_cast<const uint32_t*>(wr + 16 * kk);
            const uint32_t b1w = *reinterpret_cast<const uint32_t*>(wr + 16 * kk + 8);
            mma_bf16(out[j], a[kk][0], a[kk][1], a[kk][2], a[kk][3], b0w, b1w);
        }
    }
}

__global__ void __launch_bounds__(32 * INF_WARPS, 2) mlp_infer_kernel(
    const uint16_t* __restrict__ Wg, const float* __restrict__ Bg, const float* __restrict__ stats,
    const float* __restrict__ features, const double* __restrict__ total, long long n,
    double* __restrict__ emission, unsigned char* __restrict__ flags, float inv_share_max)
{
    extern __shared__ __align__(16) unsigned char sm[];
    // stage the weights (bf16, contiguous W1 W2 W3) and biases / statistics
    {
        // 16-byte chunks of the contiguous global rows into the padded rows
        const uint4* src = reinterpret_cast<const uint4*>(Wg);
        constexpr int c1 = NIN / 8, c2 = NH / 8;  // chunks per row
        for (int i = threadIdx.x; i < NH * c1; i += blockDim.x)
            *reinterpret_cast<uint4*>(sm + SM_W1 + sizeof(uint16_t) * ((i / c1) * KP1 + 8 * (i % c1))) = src[i];
        src += NH * c1;
        for (int i = threadIdx.x; i < NH * c2; i += blockDim.x)
            *reinterpret_cast<uint4*>(sm + SM_W2 + sizeof(uint16_t) * ((i / c2) * KP2 + 8 * (i % c2))) = src[i];
        src += NH * c2;
        for (int i = threadIdx.x; i < NO_PAD * c2; i += blockDim.x)
            *reinterpret_cast<uint4*>(sm + SM_W3 + sizeof(uint16_t) * ((i / c2) * KP2 + 8 * (i % c2))) = src[i];
        float* sb = reinterpret_cast<float*>(sm + SM_B);
        for (int i = threadIdx.x; i < NH + NH + NO_PAD; i += blockDim.x) sb[i] = Bg[i];
        float* ss = reinterpret_cast<float*>(sm + SM_ST);
        for (int i = threadIdx.x; i < 4 * NIN; i += blockDim.x) ss[i] = stats[i];
    }
    __syncthreads();
    const uint16_t* W1 = reinterpret_cast<const uint16_t*>(sm + SM_W1);
    const uint16_t* W2 = reinterpret_cast<const uint16_t*>(sm + SM_W2);
    const uint16_t* W3 = reinterpret_cast<const uint16_t*>(sm + SM_W3);
    const float* B1 = reinterpret_cast<const float*>(sm + SM_B);
    const float* B2 = B1 + NH;
    const float* B3 = B2 + NH;
    const float* mean = reinterpret_cast<const float*>(sm + SM_ST);
    const float* istd = mean + NIN;
    const float* hlo = istd + NIN;
    const float* hhi = hlo + NIN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float* xbuf = reinterpret_cast<float*>(sm + SM_X) + warp * 2 * 16 * NIN;  // [2][16][32]
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + SM_BAR) + warp * 2;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    const long long stride = (long long)gridDim.x * INF_ROWS;
    // the 16 feature rows of the tile at row b (fewer at the end), 128 bytes each
    auto fetch = [&](long long b, int buf) {
        const long long rows = n - b < 16 ? n - b : 16;
        fence_proxy_async();
        bulk_load(xbuf + buf * 16 * NIN, features + b * NIN, (unsigned)(rows * NIN * sizeof(float)), &bar[buf]);
    };
    long long base = (long long)blockIdx.x * INF_ROWS + warp * 16;
    if (lane == 0 && base < n) fetch(base, 0);
    for (long long k = 0; base < n; base += stride, ++k) {
        const int buf = (int)(k & 1);
        // the next tile streams in while this one is computed
        if (lane == 0 && base + stride < n) fetch(base + stride, buf ^ 1);
        if (!mbar_wait(&bar[buf], (unsigned)((k >> 1) & 1))) {
            atomicOr(&g_mlp_timeout, 1u);
            if (lane == 0 && base + stride < n) mbar_wait(&bar[buf ^ 1], (unsigned)(((k + 1) >> 1) & 1));
            break;
        }
        // the rows' absorbed powers for the epilogue, requested before the layers so that
        // their latency overlaps with the products
        const long long r0 = base + g, r1 = base + g + 8;
        const double tot0 = r0 < n ? __ldcs(total + r0) : 0.0;
        const double tot1 = r1 < n ? __ldcs(total + r1) : 0.0;
        const float* xs = xbuf + buf * 16 * NIN;  // [16][32]; rows past n hold stale values
        // ---- guard: row i, lane = feature.  A row leaves the training hull when a
        // feature leaves its range, or when its dominant band holds a larger share of
        // the cell's absorbed power than the guard allows: sum_b 10^(f_b - f_max) is
        // the inverse of that share.  One ballot per row.
        if (flags) {
            bool mine = false;
            const float lo_f = hlo[lane], hi_f = hhi[lane];
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const float v = xs[i * NIN + lane];
                float m = v;
#pragma unroll
                for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                float e = exp2f((v - m) * 3.32192809f);
#pragma unroll
                for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
                const unsigned out = __ballot_sync(0xffffffffu, !(v >= lo_f && v <= hi_f) || e < inv_share_max);
                if (lane == i) mine = out != 0;
            }
            const long long r = base + lane;
            // a cell without absorbed power emits nothing: no fallback needed
            if (lane < 16 && r < n) flags[r] = (mine && total[r] > 0.0) ? 1 : 0;
        }
        // a tile none of whose rows absorbs power (empty space): its emission rows
        // are zeros (the epilogue scales every row by its FP32 total), so the
        // layers are skipped
        if (!__any_sync(0xffffffffu, (float)tot0 != 0.f || (float)tot1 != 0.f)) {
#pragma unroll
            for (int j = 0; j < NO_PAD / 8; ++j) {
                const int c = 8 * j + 2 * t;
                if (c < NO) {
                    if (r0 < n) __stcs(reinterpret_cast<double2*>(emission + r0 * NO + c), make_double2(0.0, 0.0));
                    if (r1 < n) __stcs(reinterpret_cast<double2*>(emission + r1 * NO + c), make_double2(0.0, 0.0));
                }
            }
            __syncwarp();  // every lane is done with this buffer before it is refilled
            continue;
        }
        uint32_t a1[2][4];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int c = 16 * kk + 2 * t;
            auto sx = [&](int row, int col) { return (xs[row * NIN + col] - mean[col]) * istd[col]; };
            a1[kk][0] = pack_bf16(sx(g, c), sx(g, c + 1));
            a1[kk][1] = pack_bf16(sx(g + 8, c), sx(g + 8, c + 1));
            a1[kk][2] = pack_bf16(sx(g, c + 8), sx(g, c + 9));
            a1[kk][3] = pack_bf16(sx(g + 8, c + 8), sx(g + 8, c + 9));
        }
        __syncwarp();
        // ---- layers
        float h[NH / 8][4];
        layer<NH / 8, 2, KP1>(a1, W1, B1, h, g, t);
        uint32_t a2[NH / 16][4];
        to_afrag<NH / 8>(h, a2);
        layer<NH / 8, NH / 16, KP2>(a2, W2, B2, h, g, t);
        to_afrag<NH / 8>(h, a2);
        float z[NO_PAD / 8][4];
        layer<NO_PAD / 8, NH / 16, KP2>(a2, W3, B3, z, g, t);
        // ---- softmax over the 100 outputs of rows g and g+8 (4 lanes per row)
        float m0 = -3.0e38f, m1 = -3.0e38f;
#pragma unroll
        for (int j = 0; j < NO_PAD / 8; ++j) {
            if (8 * j + 2 * t < NO) { m0 = fmaxf(m0, fmaxf(z[j][0], z[j][1])); m1 = fmaxf(m1, fmaxf(z[j][2], z[j][3])); }
        }
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int j = 0; j < NO_PAD / 8; ++j) {
            const bool ok = 8 * j + 2 * t < NO;
            z[j][0] = ok ? __expf(z[j][0] - m0) : 0.f;
            z[j][1] = ok ? __expf(z[j][1] - m0) : 0.f;
            z[j][2] = ok ? __expf(z[j][2] - m1) : 0.f;
            z[j][3] = ok ? __expf(z[j][3] - m1) : 0.f;
            s0 += z[j][0] + z[j][1];
            s1 += z[j][2] + z[j][3];
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        // emission = shape x absorbed power, formed in FP32 (the shape is an FP32
        // softmax) and widened exactly to FP64
        const float f0 = r0 < n ? (float)tot0 / s0 : 0.f;
        const float f1 = r1 < n ? (float)tot1 / s1 : 0.f;
#pragma unroll
        for (int j = 0; j < NO_PAD / 8; ++j) {
            const int c = 8 * j + 2 * t;
            if (c < NO) {
                if (r0 < n)
                    __stcs(reinterpret_cast<double2*>(emission + r0 * NO + c),
                           make_double2(widen_pos(f0 * z[j][0]), widen_pos(f0 * z[j][1])));
                if (r1 < n)
                    __stcs(reinterpret_cast<double2*>(emission + r1 * NO + c),
                           make_double2(widen_pos(f1 * z[j][2]), widen_pos(f1 * z[j][3])));
            }
        }
        __syncwarp();  // every lane is done with this buffer before it is refilled
    }
}

// --------------------------------------------------------------------------
// training helpers (the step itself is in mlp_train.cu)
// --------------------------------------------------------------------------
// out[r][c] = in[r][c] / sum_c in[r][c] in FP32 (one warp per row; zero rows stay zero)
__global__ void normalize_rows_kernel(const double* __restrict__ in, float* __restrict__ out, long long rows)
{
    const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    double s = 0.0;
    for (int c = lane; c < NO; c += 32) s += in[r * NO + c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int c = lane; c < NO; c += 32) out[r * NO + c] = (float)(in[r * NO + c] * inv);
}

// share of a row's absorbed power in its dominant band, from its 32 band
// features (log10 of the band powers per unit mass): 1 / sum_b 10^(f_b - f_max)
__global__ void dominant_share_kernel(const float* __restrict__ feat, long long n, float* __restrict__ share)
{
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const float* f = feat + r * NIN;
        float m = f[0];
        for (int b = 1; b < NIN; ++b) m = fmaxf(m, f[b]);
        float e = 0.f;
        for (int b = 0; b < NIN; ++b) e += exp2f((f[b] - m) * 3.32192809f);
        share[r] = 1.f / e;
    }
}

// per-feature sums over n samples: sum, sum of squares, min, max (one block per feature)
__global__ void feature_stats_kernel(const float* feat, long long n, double* out)
{
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    float lo = 3.0e38f, hi = -3.0e38f;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) {
        const float v = feat[r * NIN + c];
        s += v;
        s2 += (double)v * v;
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    __shared__ double rs[256], rs2[256];
    __shared__ float rl[256], rh[256];
    rs[threadIdx.x] = s; rs2[threadIdx.x] = s2; rl[threadIdx.x] = lo; rh[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            rs[threadIdx.x] += rs[threadIdx.x + o];
            rs2[threadIdx.x] += rs2[threadIdx.x + o];
            rl[threadIdx.x] = fminf(rl[threadIdx.x], rl[threadIdx.x + o]);
            rh[threadIdx.x] = fmaxf(rh[threadIdx.x], rh[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[4 * c + 0] = rs[0];
        out[4 * c + 1] = rs2[0];
        out[4 * c + 2] = rl[0];
        out[4 * c + 3] = rh[0];
    }
}

// bf16 copies of the weights (W3 padded to 104 rows with zeros) and the fp32
// biases (b3 padded with -inf-like values so that padded logits vanish)
__global__ void pack_inference_kernel(const float* __restrict__ P, uint16_t* __restrict__ W, float* __restrict__ B)
{
    const int nW = NH * NIN + NH * NH + NO_PAD * NH;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nW; i += gridDim.x * blockDim.x) {
        float v;
        if (i < NH * NIN) v = P[OFF_W1 + i];
        else if (i < NH * NIN + NH * NH) v = P[OFF_W2 + (i - NH * NIN)];
        else {
            const int k = i - NH * NIN - NH * NH;
            v = k < NO * NH ? P[OFF_W3 + k] : 0.f;
        }
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        W[i] = *reinterpret_cast<uint16_t*>(&b);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH + NH + NO_PAD; i += gridDim.x * blockDim.x) {
        if (i < NH) B[i] = P[OFF_B1 + i];
        else if (i < 2 * NH) B[i] = P[OFF_B2 + i - NH];
        else B[i] = (i - 2 * NH) < NO ? P[OFF_B3 + i - 2 * NH] : -1.0e30f;
    }
}

int blocks_for(long long n, int block)
{
    long long b = (n + block - 1) / block;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

// splitmix64: the library's host-side generator for the initial weights
uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace skirt

using namespace skirt;

struct skirt_mlp_s {
    float* P = nullptr;        // FP32 master parameters [NPARAM]
    float* G = nullptr;        // gradient [NPARAM]
    float* Mo = nullptr;       // Adam first moment
    float* Vo = nullptr;       // Adam second moment
    uint16_t* Wb = nullptr;    // bf16 weights for inference
    float* Bb = nullptr;       // fp32 biases for inference (b3 padded)
    float* stats = nullptr;    // device: mean[32], 1/std[32], lo[32], hi[32]
    float host_stats[4 * NIN]; // mean, std, lo, hi
    float share_max = 1.f;     // guard: rows whose dominant band holds more of the power go to the exact solver
    bool packed = false;
    // working tables of skirt_dust_emission's surrogate mode (features, totals,
    // flags, fallback rows), grown on demand and kept until the network is
    // destroyed; ws_mu serialises the calls that use them
    std::mutex ws_mu;
    void* ws = nullptr;
    size_t ws_bytes = 0;
};

namespace skirt {

static int upload_stats(skirt_mlp_s* net)
{
    float d[4 * NIN];
    for (int k = 0; k < NIN; ++k) {
        d[k] = net->host_stats[k];
        d[NIN + k] = 1.f / net->host_stats[NIN + k];
        d[2 * NIN + k] = net->host_stats[2 * NIN + k];
        d[3 * NIN + k] = net->host_stats[3 * NIN + k];
    }
    MCK(cudaMemcpy(net->stats, d, sizeof d, cudaMemcpyHostToDevice));
    return SKIRT_OK;
}

static int repack(skirt_mlp_s* net, cudaStream_t s)
{
    pack_inference_kernel<<<64, 256, 0, s>>>(net->P, net->Wb, net->Bb);
    MCK(cudaGetLastError());
    net->packed = true;
    return SKIRT_OK;
}

std::mutex& mlp_workspace_mutex(skirt_mlp_s* net) { return net->ws_mu; }

int mlp_workspace(skirt_mlp_s* net, size_t bytes, void** p)
{
    if (bytes > net->ws_bytes) {
        // the previous calls have synchronised their streams: the old tables are idle
        cudaFree(net->ws);
        net->ws = nullptr;
        net->ws_bytes = 0;
        MCK(cudaMalloc(&net->ws, bytes));
        net->ws_bytes = bytes;
    }
    *p = net->ws;
    return SKIRT_OK;
}

int mlp_forward_internal(skirt_mlp_s* net, const float* features, const double* total, long long n, double* emission,
                         unsigned char* flags, cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(features) & 15) != 0)
        return set_error(SKIRT_ERR_INVALID_ARG, "features must be 16-byte aligned");
    if (!net->packed) {
        int r = repack(net, s);
        if (r) return r;
    }
    const unsigned zero = 0;
    MCK(cudaMemcpyToSymbolAsync(g_mlp_timeout, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s));
    MCK(cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_TOTAL));
    int sms = 0, dev = 0, per_sm = 0;
    MCK(cudaGetDevice(&dev));
    MCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_infer_kernel, 32 * INF_WARPS, SM_TOTAL));
    long long tiles = (n + INF_ROWS - 1) / INF_ROWS;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    const float inv_share_max = net->share_max > 0.f ? 1.f / net->share_max : 3.0e38f;
    mlp_infer_kernel<<<(int)grid, 32 * INF_WARPS, SM_TOTAL, s>>>(net->Wb, net->Bb, net->stats, features, total, n,
                                                                  emission, flags, inv_share_max);
    MCK(cudaGetLastError());
    return SKIRT_OK;
}

int mlp_check_timeout()
{
    unsigned v = 0;
    MCK(cudaMemcpyFromSymbol(&v, g_mlp_timeout, sizeof v));
    if (v) return set_error(SKIRT_ERR_CUDA, "surrogate inference: a feature copy did not complete in time");
    return SKIRT_OK;
}

}  // namespace skirt

// ---------------------------------------------------------------- C ABI
extern "C" int skirt_mlp_create(skirt_mlp_t* out, uint64_t seed)
{
    if (!out) return set_error(SKIRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    skirt_mlp_s* net = new skirt_mlp_s;
    auto bail = [&](int code) {
        skirt_mlp_destroy(net);
        return code;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&net->P, sizeof(float) * NPARAM)) || (e = cudaMalloc(&net->G, sizeof(float) * NPARAM)) ||
        (e = cudaMalloc(&net->Mo, sizeof(float) * NPARAM)) || (e = cudaMalloc(&net->Vo, sizeof(float) * NPARAM)) ||
        (e = cudaMalloc(&net->Wb, sizeof(uint16_t) * (NH * NIN + NH * NH + NO_PAD * NH))) ||
        (e = cudaMalloc(&net->Bb, sizeof(float) * (NH + NH + NO_PAD))) ||
        (e = cudaMalloc(&net->stats, sizeof(float) * 4 * NIN)))
        return bail(set_error(SKIRT_ERR_OOM, "mlp buffers: %s", cudaGetErrorString(e)));
    // Kaiming-uniform weights U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)), zero biases
    std::vector<float> h(NPARAM, 0.f);
    uint64_t st = seed;
    auto fill = [&](int off, int rows, int cols) {
        const double b = std::sqrt(6.0 / cols);
        for (int i = 0; i < rows * cols; ++i) {
            const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            h[off + i] = (float)((2.0 * u - 1.0) * b);
        }
    };
    fill(OFF_W1, NH, NIN);
    fill(OFF_W2, NH, NH);
    fill(OFF_W3, NO, NH);
    if ((e = cudaMemcpy(net->P, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice)))
        return bail(set_error(SKIRT_ERR_CUDA, "mlp init: %s", cudaGetErrorString(e)));
    for (int k = 0; k < NIN; ++k) {
        net->host_stats[k] = 0.f;
        net->host_stats[NIN + k] = 1.f;
        net->host_stats[2 * NIN + k] = -3.0e38f;
        net->host_stats[3 * NIN + k] = 3.0e38f;
    }
    if (int r = upload_stats(net)) return bail(r);
    *out = net;
    return SKIRT_OK;
}

extern "C" int skirt_mlp_destroy(skirt_mlp_t net)
{
    if (!net) return SKIRT_OK;
    cudaFree(net->P);
    cudaFree(net->G);
    cudaFree(net->Mo);
    cudaFree(net->Vo);
    cudaFree(net->Wb);
    cudaFree(net->Bb);
    cudaFree(net->stats);
    cudaFree(net->ws);
    delete net;
    return SKIRT_OK;
}

extern "C" int skirt_mlp_set_params(skirt_mlp_t net, const float* params, const float* x_mean, const float* x_std,
                                    const float* hull_lo, const float* hull_hi)
{
    if (!net) return set_error(SKIRT_ERR_INVALID_ARG, "net is NULL");
    if (params) {
        for (int i = 0; i < NPARAM; ++i)
            if (!std::isfinite(params[i])) return set_error(SKIRT_ERR_INVALID_ARG, "params[%d] is not finite", i);
        MCK(cudaMemcpy(net->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
        net->packed = false;
    }
    if (x_std)
        for (int k = 0; k < NIN; ++k)
            if (!(x_std[k] > 0)) return set_error(SKIRT_ERR_INVALID_ARG, "x_std[%d] must be > 0", k);
    if (x_mean) std::memcpy(net->host_stats, x_mean, sizeof(float) * NIN);
    if (x_std) std::memcpy(net->host_stats + NIN, x_std, sizeof(float) * NIN);
    if (hull_lo) std::memcpy(net->host_stats + 2 * NIN, hull_lo, sizeof(float) * NIN);
    if (hull_hi) std::memcpy(net->host_stats + 3 * NIN, hull_hi, sizeof(float) * NIN);
    return upload_stats(net);
}

extern "C" int skirt_mlp_set_guard(skirt_mlp_t net, float share_max)
{
    if (!net) return set_error(SKIRT_ERR_INVALID_ARG, "net is NULL");
    if (!(share_max > 0.f)) return set_error(SKIRT_ERR_INVALID_ARG, "share_max must be > 0");
    net->share_max = share_max;
    return SKIRT_OK;
}

extern "C" int skirt_mlp_get_guard(skirt_mlp_t net, float* share_max)
{
    if (!net || !share_max) return set_error(SKIRT_ERR_INVALID_ARG, "net / share_max is NULL");
    *share_max = net->share_max;
    return SKIRT_OK;
}

extern "C" int skirt_mlp_get_params(skirt_mlp_t net, float* params, float* x_mean, float* x_std, float* hull_lo,
                                    float* hull_hi)
{
    if (!net) return set_error(SKIRT_ERR_INVALID_ARG, "net is NULL");
    if (params) MCK(cudaMemcpy(params, net->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    if (x_mean) std::memcpy(x_mean, net->host_stats, sizeof(float) * NIN);
    if (x_std) std::memcpy(x_std, net->host_stats + NIN, sizeof(float) * NIN);
    if (hull_lo) std::memcpy(hull_lo, net->host_stats + 2 * NIN, sizeof(float) * NIN);
    if (hull_hi) std::memcpy(hull_hi, net->host_stats + 3 * NIN, sizeof(float) * NIN);
    return SKIRT_OK;
}

extern "C" int skirt_mlp_train_opts_default(skirt_mlp_train_opts* o)
{
    if (!o) return set_error(SKIRT_ERR_INVALID_ARG, "opts is NULL");
    o->epochs = 200;
    o->batch = 2048;
    o->lr = 2e-3f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->eps = 1e-8f;
    o->seed = 1;
    o->guard_quantile = 0.99f;
    return SKIRT_OK;
}

namespace {

// Per-call scratch of a training step: the per-CTA partial gradients and
// losses, the loss accumulator and the reduction's block counter.
struct Work {
    float* part = nullptr;
    float* part_loss = nullptr;
    float* loss = nullptr;
    unsigned* done = nullptr;
    cudaError_t alloc(int rows, cudaStream_t s)
    {
        const int ncta = (rows + train_rows_per_cta() - 1) / train_rows_per_cta();
        cudaError_t e;
        if ((e = cudaMallocAsync((void**)&part, sizeof(float) * (size_t)ncta * NPARAM, s))) return e;
        if ((e = cudaMallocAsync((void**)&part_loss, sizeof(float) * (size_t)ncta, s))) return e;
        if ((e = cudaMallocAsync((void**)&loss, sizeof(float), s))) return e;
        if ((e = cudaMallocAsync((void**)&done, sizeof(unsigned), s))) return e;
        if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s))) return e;
        return cudaMemsetAsync(done, 0, sizeof(unsigned), s);
    }
    void release(cudaStream_t s)
    {
        for (float** p : {&part, &part_loss, &loss}) {
            if (*p) cudaFreeAsync(*p, s);
            *p = nullptr;
        }
        if (done) cudaFreeAsync(done, s);
        done = nullptr;
    }
};

// Everything a training call acquires, released on every return path (the
// stream-ordered frees go on the caller's stream, after the private stream's
// work has been joined to it).
struct TrainScope {
    cudaStream_t s = nullptr;
    Work w;
    float* target = nullptr;
    float* x_in = nullptr;    // the gradient call's copies of its rows
    float* t_in = nullptr;
    double* d_st = nullptr;
    unsigned long long* d_ab = nullptr;
    float* d_sched = nullptr;
    long long* d_t = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ready = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    explicit TrainScope(cudaStream_t st) : s(st) {}
    ~TrainScope()
    {
        if (cs) {
            if (ready && cudaEventRecord(ready, cs) == cudaSuccess) cudaStreamWaitEvent(s, ready, 0);
            cudaStreamSynchronize(cs);
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (ready) cudaEventDestroy(ready);
        w.release(s);
        if (target) cudaFreeAsync(target, s);
        if (x_in) cudaFreeAsync(x_in, s);
        if (t_in) cudaFreeAsync(t_in, s);
        if (d_st) cudaFreeAsync(d_st, s);
        if (d_ab) cudaFreeAsync(d_ab, s);
        if (d_sched) cudaFreeAsync(d_sched, s);
        if (d_t) cudaFreeAsync(d_t, s);
        cudaGetLastError();
    }
};

}  // namespace

extern "C" int skirt_mlp_grad(skirt_mlp_t net, const float* x_std, const float* target, int n, float* grad,
                              float* loss, void* stream)
{
    if (!net || !x_std || !target || n < 1) return set_error(SKIRT_ERR_INVALID_ARG, "net / x_std / target / n");
    cudaStream_t s = (cudaStream_t)stream;
    TrainScope sc(s);
    Work& w = sc.w;
    MCK(w.alloc(n, s));
    float*& d_x = sc.x_in;
    float*& d_t = sc.t_in;
    MCK(cudaMallocAsync((void**)&d_x, sizeof(float) * (size_t)n * NIN, s));
    MCK(cudaMallocAsync((void**)&d_t, sizeof(float) * (size_t)n * NO, s));
    MCK(cudaMemcpyAsync(d_x, x_std, sizeof(float) * (size_t)n * NIN, cudaMemcpyDefault, s));
    MCK(cudaMemcpyAsync(d_t, target, sizeof(float) * (size_t)n * NO, cudaMemcpyDefault, s));
    if (int r = repack(net, s)) return r;
    MCK(launch_train_step(net->Wb, net->P, nullptr, d_t, nullptr, nullptr, nullptr, 0, n, d_x, n, w.part, w.part_loss,
                          net->G, 0, nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, nullptr, w.loss, w.done, s));
    if (grad) MCK(cudaMemcpyAsync(grad, net->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
    float l = 0.f;
    MCK(cudaMemcpyAsync(&l, w.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    if (loss) *loss = l;
    return SKIRT_OK;
}

extern "C" int skirt_mlp_train(skirt_mlp_t net, const float* features, const double* emission, long long n,
                               const skirt_mlp_train_opts* opts, float* loss_history, void* stream)
{
    if (!net || !features || !emission || !opts) return set_error(SKIRT_ERR_INVALID_ARG, "net / data / opts is NULL");
    const int B = opts->batch;
    if (B < 32 || B > (1 << 16) || n < B) return set_error(SKIRT_ERR_INVALID_ARG, "batch must be in [32, 65536] and <= n");
    if (opts->epochs < 1 || !(opts->lr > 0)) return set_error(SKIRT_ERR_INVALID_ARG, "epochs / lr invalid");
    if (!(opts->guard_quantile > 0.f)) return set_error(SKIRT_ERR_INVALID_ARG, "guard_quantile must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    TrainScope sc(s);
    // target shapes: every emission row normalised to sum 1
    float*& target = sc.target;
    MCK(cudaMallocAsync((void**)&target, sizeof(float) * NO * (size_t)n, s));
    normalize_rows_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(emission, target, n);
    MCK(cudaGetLastError());
    // standardisation and hull from the training features
    double*& d_st = sc.d_st;
    MCK(cudaMallocAsync((void**)&d_st, sizeof(double) * 4 * NIN, s));
    feature_stats_kernel<<<NIN, 256, 0, s>>>(features, n, d_st);
    MCK(cudaGetLastError());
    double st[4 * NIN];
    MCK(cudaMemcpyAsync(st, d_st, sizeof st, cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    for (int k = 0; k < NIN; ++k) {
        const double mean = st[4 * k] / (double)n;
        const double var = st[4 * k + 1] / (double)n - mean * mean;
        net->host_stats[k] = (float)mean;
        net->host_stats[NIN + k] = (float)std::sqrt(var > 1e-12 ? var : 1e-12);
        net->host_stats[2 * NIN + k] = (float)st[4 * k + 2];
        net->host_stats[3 * NIN + k] = (float)st[4 * k + 3];
    }
    if (int r = upload_stats(net)) return r;
    // the guard: the guard_quantile quantile of the training rows' dominant-band share
    if (opts->guard_quantile >= 1.f) {
        net->share_max = 1.f;
    } else {
        float*& d_share = sc.x_in;
        MCK(cudaMallocAsync((void**)&d_share, sizeof(float) * (size_t)n, s));
        dominant_share_kernel<<<blocks_for(n, 256), 256, 0, s>>>(features, n, d_share);
        MCK(cudaGetLastError());
        std::vector<float> sh((size_t)n);
        MCK(cudaMemcpyAsync(sh.data(), d_share, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        const size_t k = (size_t)((double)opts->guard_quantile * (double)(n - 1));
        std::nth_element(sh.begin(), sh.begin() + k, sh.end());
        net->share_max = sh[k];
    }
    MCK(cudaMemsetAsync(net->Mo, 0, sizeof(float) * NPARAM, s));
    MCK(cudaMemsetAsync(net->Vo, 0, sizeof(float) * NPARAM, s));
    Work& w = sc.w;
    MCK(w.alloc(B, s));
    const long long steps = n / B;
    const long long total_steps = steps * opts->epochs;
    // per-epoch permutations (affine i -> (a i + b) mod n with a coprime to n)
    // and the per-step schedule (cosine learning rate, Adam bias corrections),
    // computed on the host and read on the device at the step counter
    std::vector<unsigned long long> ab(2 * (size_t)opts->epochs);
    std::vector<float> sched(3 * (size_t)total_steps);
    uint64_t rs = opts->seed ^ 0x5DEECE66Dull;
    auto gcd = [](unsigned long long x, unsigned long long y) {
        while (y) { unsigned long long r = x % y; x = y; y = r; }
        return x;
    };
    for (int ep = 0; ep < opts->epochs; ++ep) {
        unsigned long long a = (splitmix64(rs) % (unsigned long long)n) | 1ull;
        while (gcd(a, (unsigned long long)n) != 1) a += 2;
        ab[2 * ep] = a;
        ab[2 * ep + 1] = splitmix64(rs) % (unsigned long long)n;
    }
    for (long long t = 0; t < total_steps; ++t) {
        const double frac = (double)t / (double)(total_steps > 1 ? total_steps - 1 : 1);
        sched[3 * t] = (float)(opts->lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(M_PI * frac))));
        sched[3 * t + 1] = 1.f - std::pow(opts->beta1, (float)(t + 1));
        sched[3 * t + 2] = 1.f - std::pow(opts->beta2, (float)(t + 1));
    }
    unsigned long long*& d_ab = sc.d_ab;
    float*& d_sched = sc.d_sched;
    long long*& d_t = sc.d_t;
    MCK(cudaMallocAsync((void**)&d_ab, sizeof(unsigned long long) * ab.size(), s));
    MCK(cudaMallocAsync((void**)&d_sched, sizeof(float) * sched.size(), s));
    MCK(cudaMallocAsync((void**)&d_t, sizeof(long long), s));
    MCK(cudaMemcpyAsync(d_ab, ab.data(), sizeof(unsigned long long) * ab.size(), cudaMemcpyHostToDevice, s));
    MCK(cudaMemcpyAsync(d_sched, sched.data(), sizeof(float) * sched.size(), cudaMemcpyHostToDevice, s));
    MCK(cudaMemsetAsync(d_t, 0, sizeof(long long), s));

    // the BF16 weights the first step reads
    if (int r = repack(net, s)) return r;
    // one training step (the fused tensor-core tile kernel, then the ordered
    // gradient sum with the Adam step and the step counter) as a CUDA graph,
    // captured on a private stream and replayed for every step
    cudaStream_t& cs = sc.cs;
    MCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t& ready = sc.ready;
    MCK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    MCK(cudaEventRecord(ready, s));
    MCK(cudaStreamWaitEvent(cs, ready, 0));
    cudaGraph_t& graph = sc.graph;
    cudaGraphExec_t& gexec = sc.gexec;
    int rc = SKIRT_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = launch_train_step(net->Wb, net->P, features, target, net->stats, d_ab, d_t, steps, n, nullptr, B, w.part,
                              w.part_loss, net->G, 1, net->P, net->Mo, net->Vo, d_sched, opts->beta1, opts->beta2,
                              opts->eps, net->Wb, w.loss, w.done, cs);
        if (e != cudaSuccess) {
            cudaGraph_t broken = nullptr;
            cudaStreamEndCapture(cs, &broken);
            if (broken) cudaGraphDestroy(broken);
            return set_error(SKIRT_ERR_CUDA, "training step launch: %s", cudaGetErrorString(e));
        }
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
    if (e != cudaSuccess) rc = set_error(SKIRT_ERR_CUDA, "training graph: %s", cudaGetErrorString(e));
    for (int ep = 0; ep < opts->epochs && rc == SKIRT_OK; ++ep) {
        e = cudaMemsetAsync(w.loss, 0, sizeof(float), cs);
        for (long long k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(gexec, cs);
        if (e == cudaSuccess && loss_history) {
            float l = 0.f;
            e = cudaMemcpyAsync(&l, w.loss, sizeof(float), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            loss_history[ep] = l / (float)steps;
        }
        if (e != cudaSuccess) rc = set_error(SKIRT_ERR_CUDA, "training step: %s", cudaGetErrorString(e));
    }
    if (rc) return rc;  // the scope joins the private stream and frees everything
    // join the private stream before the repack on the caller's stream
    MCK(cudaEventRecord(ready, cs));
    MCK(cudaStreamWaitEvent(s, ready, 0));
    if (int r = repack(net, s)) return r;
    MCK(cudaStreamSynchronize(s));
    return SKIRT_OK;
}

extern "C" int skirt_mlp_forward(skirt_mlp_t net, const float* features, const double* total, long long n,
                                 double* emission, unsigned char* flags, void* stream)
{
    if (!net || !features || !total || !emission || n < 0) return set_error(SKIRT_ERR_INVALID_ARG, "mlp forward args");
    if (n == 0) return SKIRT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int r = mlp_forward_internal(net, features, total, n, emission, flags, s);
    if (r) return r;
    MCK(cudaStreamSynchronize(s));
    return mlp_check_timeout();
}
