// Training step of the MLP surrogate on the tensor cores (BF16 products,
// FP32 accumulation, FP32 master weights).
//
// train_tile_kernel: one CTA per 32 rows of the batch, 8 warps.  The CTA
// stages the BF16 weights in shared memory, gathers and standardises its rows,
// and runs the whole step for them with mma.sync m16n8k16 in inline PTX:
//   forward   Z1 = X W1^T + b1, A1 = SiLU(Z1), Z2, A2, Z3 (logits);
//   softmax and cross-entropy, dZ3 = (p - t) / n;
//   backward  dZ2 = (dZ3 W3) * SiLU'(Z2), dZ1 = (dZ2 W2) * SiLU'(Z1)
//             (the products with W^T read W, stored [out][in], through
//             ldmatrix.trans);
//   weights   dW3 = dZ3^T A2, dW2 = dZ2^T A1, dW1 = dZ1^T X, biases = column
//             sums (the row dimension is the contraction; both operands come
//             from the row-major activation tiles through ldmatrix.trans).
// Every operand of a product is rounded to BF16 once: the standardised
// inputs, the weights, the activations and the dZ tiles; the SiLU
// derivatives, the softmax, the bias sums and the accumulators stay FP32.
// Each CTA writes its partial gradient (packed parameter layout) and its
// partial loss.
//
// train_reduce_kernel: the partial gradients summed over the CTAs in CTA
// order (deterministic), then (training) the Adam step at the learning rate
// and bias corrections of the device step counter, the refreshed BF16
// weights for the next step, and the loss; the last block to finish
// advances the step counter.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "skirt_internal.cuh"

namespace skirt {
namespace {

constexpr int NIN = SKIRT_NBANDS;      // 32
constexpr int NH = SKIRT_MLP_HIDDEN;   // 128
constexpr int NO = SKIRT_NEMIT;        // 100
constexpr int NOP = 104;               // 13 n-tiles of 8 (forward output of layer 3)
constexpr int NOK = 112;               // 7 k-tiles of 16 (dZ3 as a contraction operand)
constexpr int NPARAM = SKIRT_MLP_NPARAM;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH;

constexpr int TR = 32;      // rows per CTA
constexpr int TWARPS = 8;   // warps per CTA
// shared-memory row strides (elements), each row padded by 8 BF16 (16 bytes)
// so that the eight rows an ldmatrix touches start in different bank groups
constexpr int P1 = NIN + 8;   // 40
constexpr int P2 = NH + 8;    // 136
constexpr int P3 = NOK + 8;   // 120
constexpr size_t S_W1 = 0;                                            // [128][P1]
constexpr size_t S_W2 = S_W1 + 2 * NH * P1;                           // [128][P2]
constexpr size_t S_W3 = S_W2 + 2 * NH * P2;                           // [112][P2], rows >= 100 zero
constexpr size_t S_X = S_W3 + 2 * NOK * P2;                           // [32][P1]
constexpr size_t S_A1 = S_X + 2 * TR * P1;                            // [32][P2]
constexpr size_t S_A2 = S_A1 + 2 * TR * P2;
constexpr size_t S_D3 = S_A2 + 2 * TR * P2;                           // [32][P3], cols >= 100 zero
constexpr size_t S_D2 = S_D3 + 2 * TR * P3;                           // [32][P2]
constexpr size_t S_D1 = S_D2 + 2 * TR * P2;
constexpr size_t S_G1 = S_D1 + 2 * TR * P2;                           // fp32 [32][128]: SiLU'(Z1), then dZ1
constexpr size_t S_G2 = S_G1 + 4 * TR * NH;                           // fp32 [32][128]: SiLU'(Z2), then dZ2
constexpr size_t S_Z3 = S_G2 + 4 * TR * NH;                           // fp32 [32][104]: logits, then dZ3
constexpr size_t S_LOSS = S_Z3 + 4 * TR * NOP;                        // fp32 [32]
constexpr size_t S_TOTAL = S_LOSS + 4 * TR;
static_assert(S_TOTAL <= 227 * 1024, "shared memory of one CTA");
static_assert(S_X % 16 == 0 && S_A1 % 16 == 0 && S_D3 % 16 == 0 && S_G1 % 16 == 0, "16-byte aligned tiles");

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(su32(p)));
}

__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(su32(p)));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&b);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}

__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + expf(-z)); }

// A fragment (16 x 16) of the row-major tile S [rows][stride] at (r0, c0)
template <int STRIDE>
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const uint16_t* S, int r0, int c0, int lane)
{
    const int m = lane >> 3, j = lane & 7;
    ldsm4(a, S + (size_t)(r0 + (m & 1) * 8 + j) * STRIDE + c0 + (m >> 1) * 8);
}

// A fragment (16 x 16) of S^T at (m0, k0), S row-major [k][m]
template <int STRIDE>
__device__ __forceinline__ void frag_at(uint32_t (&a)[4], const uint16_t* S, int m0, int k0, int lane)
{
    const int m = lane >> 3, j = lane & 7;
    ldsm4t(a, S + (size_t)(k0 + (m >> 1) * 8 + j) * STRIDE + m0 + (m & 1) * 8);
}

// B fragments of two n-tiles (n0, n0 + 8) for the k-tile at k0, where
// B[k][n] = S[k][n] with S row-major: b[0], b[1] for n-tile n0; b[2], b[3] for n0 + 8
template <int STRIDE>
__device__ __forceinline__ void frag_b2t(uint32_t (&b)[4], const uint16_t* S, int k0, int n0, int lane)
{
    const int m = lane >> 3, j = lane & 7;
    ldsm4t(b, S + (size_t)(k0 + (m & 1) * 8 + j) * STRIDE + n0 + (m >> 1) * 8);
}

// forward layer tile: C (16 x 8 per n-tile) = A (16 x 16*KT) x W^T for the
// n-tiles nts[] (W row-major [out][in] in shared memory)
template <int KT, int STRIDE_A, int STRIDE_W>
__device__ __forceinline__ void fwd_tile(float (&c)[4], const uint32_t (&a)[KT][4], const uint16_t* W, int nt, int g,
                                         int t)
{
    const uint16_t* wr = W + (size_t)(8 * nt + g) * STRIDE_W + 2 * t;
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 16 * kk);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 16 * kk + 8);
        mma16816(c, a[kk], b0, b1);
    }
}

// dst[o][i] (o < mrows, row stride outK) = sum over the 32 rows r of D[r][o] Act[r][i]
// for the output rows of m-tile mt and all ntiles n-tiles of i: A = D^T, B = Act,
// both through ldmatrix.trans of the row-major tiles
template <int SD, int SA>
__device__ __forceinline__ void wgrad(const uint16_t* D, const uint16_t* Act, int ntiles, int mt, int outK, int mrows,
                                      float* dst, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    uint32_t a0[4], a1[4];
    frag_at<SD>(a0, D, 16 * mt, 0, lane);
    frag_at<SD>(a1, D, 16 * mt, 16, lane);
    for (int np = 0; np < ntiles; np += 2) {
        float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t b[4];
        frag_b2t<SA>(b, Act, 0, 8 * np, lane);
        mma16816(acc0, a0, b[0], b[1]);
        mma16816(acc1, a0, b[2], b[3]);
        frag_b2t<SA>(b, Act, 16, 8 * np, lane);
        mma16816(acc0, a1, b[0], b[1]);
        mma16816(acc1, a1, b[2], b[3]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float* acc = u ? acc1 : acc0;
            const int c = 8 * (np + u) + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = 16 * mt + g + 8 * h;
                if (o < mrows)
                    *reinterpret_cast<float2*>(dst + (size_t)o * outK + c) = make_float2(acc[2 * h], acc[2 * h + 1]);
            }
        }
    }
}

struct TileArgs {
    const uint16_t* Wb;       // bf16 W1 [128][32], W2 [128][128], W3 [104][128] (rows >= 100 zero)
    const float* P;           // fp32 parameters (biases read from here)
    // rows: either gathered (feat != nullptr: row r of step t is (a (k B + r) + b) mod n_data of the
    // epoch's permutation, features standardised with stats) or direct (x_std, target)
    const float* feat;
    const float* target;      // [n_data][100] row shapes
    const float* stats;       // mean[32], 1/std[32]
    const unsigned long long* ab;
    const long long* t_dev;
    long long steps, n_data;
    const float* x_std;       // direct rows [nrows][32]
    int nrows;                // rows in this batch
    float inv_n;              // 1 / nrows
    float* part;              // [ncta][NPARAM] partial gradients
    float* part_loss;         // [ncta]
};

__global__ void __launch_bounds__(32 * TWARPS, 1) train_tile_kernel(const TileArgs A)
{
    extern __shared__ __align__(16) unsigned char sm[];
    uint16_t* W1 = reinterpret_cast<uint16_t*>(sm + S_W1);
    uint16_t* W2 = reinterpret_cast<uint16_t*>(sm + S_W2);
    uint16_t* W3 = reinterpret_cast<uint16_t*>(sm + S_W3);
    uint16_t* X = reinterpret_cast<uint16_t*>(sm + S_X);
    uint16_t* A1 = reinterpret_cast<uint16_t*>(sm + S_A1);
    uint16_t* A2 = reinterpret_cast<uint16_t*>(sm + S_A2);
    uint16_t* D3 = reinterpret_cast<uint16_t*>(sm + S_D3);
    uint16_t* D2 = reinterpret_cast<uint16_t*>(sm + S_D2);
    uint16_t* D1 = reinterpret_cast<uint16_t*>(sm + S_D1);
    float* G1 = reinterpret_cast<float*>(sm + S_G1);
    float* G2 = reinterpret_cast<float*>(sm + S_G2);
    float* Z3 = reinterpret_cast<float*>(sm + S_Z3);
    float* LS = reinterpret_cast<float*>(sm + S_LOSS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int row0 = blockIdx.x * TR;
    const int nvalid = min(TR, A.nrows - row0);

    // ---- stage the weights (16-byte chunks into padded rows), zero the pads
    {
        const uint4* src = reinterpret_cast<const uint4*>(A.Wb);
        for (int i = tid; i < NH * (NIN / 8); i += blockDim.x)
            *reinterpret_cast<uint4*>(W1 + (i / (NIN / 8)) * P1 + 8 * (i % (NIN / 8))) = src[i];
        src += NH * (NIN / 8);
        for (int i = tid; i < NH * (NH / 8); i += blockDim.x)
            *reinterpret_cast<uint4*>(W2 + (i / (NH / 8)) * P2 + 8 * (i % (NH / 8))) = src[i];
        src += NH * (NH / 8);
        for (int i = tid; i < NOK * (NH / 8); i += blockDim.x) {
            const int r = i / (NH / 8);
            *reinterpret_cast<uint4*>(W3 + r * P2 + 8 * (i % (NH / 8))) =
                r < NOP ? src[i] : make_uint4(0u, 0u, 0u, 0u);
        }
        // dZ3 columns 100..111 take part in the W3 products as zeros
        for (int i = tid; i < TR * (NOK - NO); i += blockDim.x) D3[(i / (NOK - NO)) * P3 + NO + i % (NOK - NO)] = 0;
    }
    // ---- the rows: standardised features (bf16) in X
    unsigned long long pa = 0, pb = 0;
    long long first = 0;
    if (A.feat) {
        const long long st = *A.t_dev;
        pa = A.ab[2 * (st / A.steps)];
        pb = A.ab[2 * (st / A.steps) + 1];
        first = (st % A.steps) * (long long)A.nrows;
    }
    auto data_row = [&](int r) -> long long {
        const long long q = first + row0 + r;
        return A.feat ? (long long)((pa * (unsigned long long)q + pb) % (unsigned long long)A.n_data) : (long long)(row0 + r);
    };
    for (int i = tid; i < TR * NIN; i += blockDim.x) {
        const int r = i / NIN, c = i % NIN;
        float v = 0.f;
        if (r < nvalid) {
            const long long s = data_row(r);
            v = A.feat ? (A.feat[s * NIN + c] - A.stats[c]) * A.stats[NIN + c] : A.x_std[s * NIN + c];
        }
        X[r * P1 + c] = bf16_bits(v);
    }
    __syncthreads();

    const int rt = warp & 1;          // row tile of this warp in the forward and backward products
    const int q4 = warp >> 1;         // its group of four n-tiles
    const float* b1v = A.P + OFF_B1;
    const float* b2v = A.P + OFF_B2;
    const float* b3v = A.P + OFF_B3;

    // ---- layer 1: Z1 = X W1^T + b1; A1 = SiLU(Z1) (bf16), G1 = SiLU'(Z1)
    {
        uint32_t a[2][4];
        frag_a<P1>(a[0], X, 16 * rt, 0, lane);
        frag_a<P1>(a[1], X, 16 * rt, 16, lane);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nt = 4 * q4 + j;
            const int c = 8 * nt + 2 * t;
            float acc[4] = {b1v[c], b1v[c + 1], b1v[c], b1v[c + 1]};
            fwd_tile<2, P1, P1>(acc, a, W1, nt, g, t);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 16 * rt + g + 8 * h;
                const float z0 = acc[2 * h], z1 = acc[2 * h + 1];
                const float s0 = sigmoid_f(z0), s1 = sigmoid_f(z1);
                *reinterpret_cast<uint32_t*>(A1 + r * P2 + c) = pack2(z0 * s0, z1 * s1);
                *reinterpret_cast<float2*>(G1 + r * NH + c) =
                    make_float2(s0 * (1.f + z0 * (1.f - s0)), s1 * (1.f + z1 * (1.f - s1)));
            }
        }
    }
    __syncthreads();
    // ---- layer 2
    {
        uint32_t a[8][4];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) frag_a<P2>(a[kk], A1, 16 * rt, 16 * kk, lane);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nt = 4 * q4 + j;
            const int c = 8 * nt + 2 * t;
            float acc[4] = {b2v[c], b2v[c + 1], b2v[c], b2v[c + 1]};
            fwd_tile<8, P2, P2>(acc, a, W2, nt, g, t);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 16 * rt + g + 8 * h;
                const float z0 = acc[2 * h], z1 = acc[2 * h + 1];
                const float s0 = sigmoid_f(z0), s1 = sigmoid_f(z1);
                *reinterpret_cast<uint32_t*>(A2 + r * P2 + c) = pack2(z0 * s0, z1 * s1);
                *reinterpret_cast<float2*>(G2 + r * NH + c) =
                    make_float2(s0 * (1.f + z0 * (1.f - s0)), s1 * (1.f + z1 * (1.f - s1)));
            }
        }
    }
    __syncthreads();
    // ---- layer 3: logits Z3 (n-tiles q4, q4 + 4, q4 + 8, q4 + 12 < 13)
    {
        uint32_t a[8][4];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) frag_a<P2>(a[kk], A2, 16 * rt, 16 * kk, lane);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nt = q4 + 4 * j;
            if (nt < NOP / 8) {
                const int c = 8 * nt + 2 * t;
                const float bb0 = c < NO ? b3v[c] : 0.f, bb1 = c + 1 < NO ? b3v[c + 1] : 0.f;
                float acc[4] = {bb0, bb1, bb0, bb1};
                fwd_tile<8, P2, P2>(acc, a, W3, nt, g, t);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = 16 * rt + g + 8 * h;
                    *reinterpret_cast<float2*>(Z3 + r * NOP + c) = make_float2(acc[2 * h], acc[2 * h + 1]);
                }
            }
        }
    }
    __syncthreads();
    // ---- softmax and cross-entropy, one warp per row: dZ3 = (p - t) / n
    for (int r = warp; r < TR; r += TWARPS) {
        float v[4], m = -3.0e38f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            v[k] = c < NO ? Z3[r * NOP + c] : -3.0e38f;
            m = fmaxf(m, v[k]);
        }
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) s += (lane + 32 * k < NO) ? expf(v[k] - m) : 0.f;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float ls = logf(s);
        const bool live = r < nvalid;
        const long long srow = live ? data_row(r) : 0;
        const float* tr = A.target + srow * NO;
        float l = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            if (c < NO) {
                float d = 0.f;
                if (live) {
                    const float tv = tr[c];
                    const float logp = v[k] - m - ls;
                    l -= tv * logp;
                    d = (expf(logp) - tv) * A.inv_n;
                }
                Z3[r * NOP + c] = d;  // the FP32 dZ3, for the bias sums
                D3[r * P3 + c] = bf16_bits(d);
            }
        }
        for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) LS[r] = l * A.inv_n;
    }
    __syncthreads();
    // ---- dZ2 = (dZ3 W3) * SiLU'(Z2): K = 112 (7 k-tiles), W3^T through ldmatrix.trans
    {
        uint32_t a[7][4];
#pragma unroll
        for (int kk = 0; kk < 7; ++kk) frag_a<P3>(a[kk], D3, 16 * rt, 16 * kk, lane);
#pragma unroll
        for (int jp = 0; jp < 2; ++jp) {
            const int nt = 4 * q4 + 2 * jp;  // n-tiles nt, nt + 1
            float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) {
                uint32_t b[4];
                frag_b2t<P2>(b, W3, 16 * kk, 8 * nt, lane);
                mma16816(acc0, a[kk], b[0], b[1]);
                mma16816(acc1, a[kk], b[2], b[3]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float* acc = u ? acc1 : acc0;
                const int c = 8 * (nt + u) + 2 * t;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = 16 * rt + g + 8 * h;
                    float2 gs = *reinterpret_cast<const float2*>(G2 + r * NH + c);
                    const float d0 = acc[2 * h] * gs.x, d1 = acc[2 * h + 1] * gs.y;
                    *reinterpret_cast<float2*>(G2 + r * NH + c) = make_float2(d0, d1);
                    *reinterpret_cast<uint32_t*>(D2 + r * P2 + c) = pack2(d0, d1);
                }
            }
        }
    }
    __syncthreads();
    // ---- dZ1 = (dZ2 W2) * SiLU'(Z1)
    {
        uint32_t a[8][4];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) frag_a<P2>(a[kk], D2, 16 * rt, 16 * kk, lane);
#pragma unroll
        for (int jp = 0; jp < 2; ++jp) {
            const int nt = 4 * q4 + 2 * jp;
            float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                uint32_t b[4];
                frag_b2t<P2>(b, W2, 16 * kk, 8 * nt, lane);
                mma16816(acc0, a[kk], b[0], b[1]);
                mma16816(acc1, a[kk], b[2], b[3]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float* acc = u ? acc1 : acc0;
                const int c = 8 * (nt + u) + 2 * t;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = 16 * rt + g + 8 * h;
                    float2 gs = *reinterpret_cast<const float2*>(G1 + r * NH + c);
                    const float d0 = acc[2 * h] * gs.x, d1 = acc[2 * h + 1] * gs.y;
                    *reinterpret_cast<float2*>(G1 + r * NH + c) = make_float2(d0, d1);
                    *reinterpret_cast<uint32_t*>(D1 + r * P2 + c) = pack2(d0, d1);
                }
            }
        }
    }
    __syncthreads();
    float* part = A.part + (size_t)blockIdx.x * NPARAM;
    // ---- bias gradients: column sums of the FP32 dZ tiles over the 32 rows, in row order
    for (int c = tid; c < NH + NH + NO; c += blockDim.x) {
        float s = 0.f;
        if (c < NH) {
            for (int r = 0; r < TR; ++r) s += G1[r * NH + c];
            part[OFF_B1 + c] = s;
        } else if (c < 2 * NH) {
            for (int r = 0; r < TR; ++r) s += G2[r * NH + c - NH];
            part[OFF_B2 + c - NH] = s;
        } else {
            for (int r = 0; r < TR; ++r) s += Z3[r * NOP + c - 2 * NH];
            part[OFF_B3 + c - 2 * NH] = s;
        }
    }
    if (tid == 0) {
        float l = 0.f;
        for (int r = 0; r < TR; ++r) l += r < nvalid ? LS[r] : 0.f;
        A.part_loss[blockIdx.x] = l;
    }
    // ---- weight gradients dW = dZ^T Act over the 32 rows (2 k-tiles):
    // warp w takes m-tile w of dW2 and dW1 and, for w < 7, of dW3
    wgrad<P2, P2>(D2, A1, NH / 8, warp, NH, NH, part + OFF_W2, lane);
    if (warp < 7) wgrad<P3, P2>(D3, A2, NH / 8, warp, NH, NO, part + OFF_W3, lane);
    wgrad<P2, P1>(D1, X, NIN / 8, warp, NIN, NH, part + OFF_W1, lane);
}

// g = sum over the CTAs of their partial gradients (in CTA order); with
// adam: the Adam step of the FP32 parameters and their BF16 copies for the
// next step, the loss, and (last block) the step counter
__global__ void train_reduce_kernel(const float* __restrict__ part, const float* __restrict__ part_loss, int ncta,
                                    float* __restrict__ G, int adam, float* __restrict__ P, float* __restrict__ Mo,
                                    float* __restrict__ Vo, const float* __restrict__ sched, long long* t_dev, float b1,
                                    float b2, float eps, uint16_t* __restrict__ Wb, float* loss_acc,
                                    unsigned* done)
{
    long long st = 0;
    float lr = 0.f, c1 = 1.f, c2 = 1.f;
    if (adam) {
        st = *t_dev;
        lr = sched[3 * st];
        c1 = sched[3 * st + 1];
        c2 = sched[3 * st + 2];
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        float gi = 0.f;
        for (int c = 0; c < ncta; ++c) gi += part[(size_t)c * NPARAM + i];
        G[i] = gi;
        if (adam) {
            const float mi = b1 * Mo[i] + (1.f - b1) * gi;
            const float vi = b2 * Vo[i] + (1.f - b2) * gi * gi;
            Mo[i] = mi;
            Vo[i] = vi;
            const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
            P[i] = p;
            // the bf16 copy of a weight (biases stay fp32): W1, W2, W3 contiguous
            int w = -1;
            if (i < OFF_B1) w = i;
            else if (i >= OFF_W2 && i < OFF_B2) w = NH * NIN + (i - OFF_W2);
            else if (i >= OFF_W3 && i < OFF_B3) w = NH * NIN + NH * NH + (i - OFF_W3);
            if (w >= 0) Wb[w] = bf16_bits(p);
        }
    }
    // the last block: loss of the step (partials in CTA order) and the step counter
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        float l = 0.f;
        for (int c = 0; c < ncta; ++c) l += part_loss[c];
        *loss_acc += l;
        if (adam) *t_dev = st + 1;
        *done = 0;
    }
}

}  // namespace

size_t train_tile_smem_bytes() { return S_TOTAL; }
int train_rows_per_cta() { return TR; }

// One step (or one gradient): nrows rows, either gathered from feat/target
// with the permutation schedule (feat != nullptr) or taken from x_std/target.
cudaError_t launch_train_step(const uint16_t* Wb, const float* P, const float* feat, const float* target,
                              const float* stats, const unsigned long long* ab, long long* t_dev,
                              long long steps, long long n_data, const float* x_std, int nrows, float* part,
                              float* part_loss, float* G, int adam, float* Pw, float* Mo, float* Vo,
                              const float* sched, float b1, float b2, float eps, uint16_t* Wb_out, float* loss_acc,
                              unsigned* done, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(train_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)S_TOTAL);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    TileArgs A;
    A.Wb = Wb;
    A.P = P;
    A.feat = feat;
    A.target = target;
    A.stats = stats;
    A.ab = ab;
    A.t_dev = t_dev;
    A.steps = steps;
    A.n_data = n_data;
    A.x_std = x_std;
    A.nrows = nrows;
    A.inv_n = 1.f / (float)nrows;
    A.part = part;
    A.part_loss = part_loss;
    const int ncta = (nrows + TR - 1) / TR;
    train_tile_kernel<<<ncta, 32 * TWARPS, S_TOTAL, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    train_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(part, part_loss, ncta, G, adam, Pw, Mo, Vo, sched, t_dev, b1,
                                                             b2, eps, Wb_out, loss_acc, done);
    return cudaGetLastError();
}

}  // namespace skirt
