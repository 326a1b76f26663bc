// Dust emission step (Sect. 3.2, dust emission phases; Sect. 1, instantaneous
// dust emission): per-cell emission spectra from the absorbed spectra.
//
//  * dust_mass_kernel      M = kappa*rho * cell volume
//  * band_features_kernel  32 log-spaced band sums per unit mass (log10) and
//                          the total absorbed power, one cell per lane
//  * exact_kernel          equilibrium temperatures of three grain
//                          populations by bracketed Newton on ln T (FP64
//                          per population, Planck terms in double-float),
//                          then the energy-conserving emission spectrum
// and skirt_dust_emission, which runs either the exact solver on every cell
// or the MLP surrogate (mlp.cu) with the exact solver as the fallback for
// cells outside the network's training hull.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "dfloat.cuh"
#include "skirt_internal.cuh"

namespace skirt {
namespace {

constexpr int NOUT = SKIRT_NEMIT;
constexpr int NB = SKIRT_NBANDS;
constexpr int NPOP = 3;
constexpr double T_REF = 30.0, T_LO = 3.0, T_HI = 2000.0;
const double DELTA[NPOP] = {-0.5, 0.0, 0.5};
const double BETA[NPOP] = {1.5, 2.0, 2.0};
// h c / k_B in micron kelvin from the exact SI constants
const double HCK_UM = 6.62607015e-34 * 299792458.0 / 1.380649e-23 * 1e6;

__constant__ double c_a[NOUT];          // hc/(k lambda_l)
__constant__ double c_K[NPOP][NOUT];    // W_l kappa_i(lambda_l) lambda_l^-5
__constant__ double c_lnc[NPOP];        // ln c_i = -ln G_i(30 K)
__constant__ double c_lnG_lo[NPOP];     // ln G_i(3 K)
__constant__ double c_lnG_hi[NPOP];     // ln G_i(2000 K)
__constant__ double c_beta[NPOP];
// ln G_i and d ln G_i / d ln T at NTAB log-spaced temperatures over [T_LO,
// T_HI]: the starting point of the Newton solve (read through the L1 path);
// 4096 intervals, so that every 2^k-th point also spans [T_LO, T_HI]
constexpr int NTAB = 4097;
__device__ double g_lnG_tab[NPOP][NTAB];
__device__ double g_dlnG_tab[NPOP][NTAB];
// (a_l, K_il) of slot s = i * NOUT + l as double-float pairs (the exact solve's terms)
__device__ float4 g_slot[NPOP * NOUT];

struct HostModel {
    double lam[NOUT], W[NOUT], a[NOUT], K[NPOP][NOUT];
    double lnc[NPOP], lnG_lo[NPOP], lnG_hi[NPOP];
    double tab[NPOP][NTAB], dtab[NPOP][NTAB];
    float slot[NPOP * NOUT][4];  // (a_l, K_il) of slot i * NOUT + l as double-float pairs
};

// v = hi + lo with hi = v rounded to binary32, lo = the rest rounded
void split_float(double v, float& hi, float& lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

double host_G(const HostModel& h, int i, double T)
{
    double g = 0.0;
    for (int l = 0; l < NOUT; ++l) g += h.K[i][l] / std::expm1(h.a[l] / T);
    return g;
}

const HostModel& host_model()
{
    static HostModel h;
    static bool ready = false;
    if (!ready) {
        for (int l = 0; l < NOUT; ++l)  // log-spaced 1 .. 1000 micron
            h.lam[l] = std::pow(10.0, 3.0 * (double)l / (double)(NOUT - 1));
        for (int l = 0; l < NOUT; ++l) {
            const double left = l > 0 ? h.lam[l] - h.lam[l - 1] : 0.0;
            const double right = l < NOUT - 1 ? h.lam[l + 1] - h.lam[l] : 0.0;
            h.W[l] = 0.5 * (left + right);
            h.a[l] = HCK_UM / h.lam[l];
            for (int i = 0; i < NPOP; ++i)
                h.K[i][l] = h.W[l] * std::pow(h.lam[l] / 100.0, -BETA[i]) * std::pow(h.lam[l], -5.0);
        }
        for (int i = 0; i < NPOP; ++i) {
            h.lnc[i] = -std::log(host_G(h, i, T_REF));
            h.lnG_lo[i] = std::log(host_G(h, i, T_LO));
            h.lnG_hi[i] = std::log(host_G(h, i, T_HI));
            for (int k = 0; k < NTAB; ++k) {
                const double T = std::exp(std::log(T_LO) + (std::log(T_HI) - std::log(T_LO)) * k / (NTAB - 1));
                double g = 0.0, d = 0.0;
                for (int l = 0; l < NOUT; ++l) {
                    const double x = h.a[l] / T;
                    if (x > 700.0) continue;
                    const double q = 1.0 / std::expm1(x);
                    g += h.K[i][l] * q;
                    d += h.K[i][l] * q * x * (1.0 + q);
                }
                h.tab[i][k] = std::log(g);
                h.dtab[i][k] = d / g;
            }
        }
        for (int i = 0; i < NPOP; ++i)
            for (int l = 0; l < NOUT; ++l) {
                float* q = h.slot[i * NOUT + l];
                split_float(h.a[l], q[0], q[1]);
                split_float(h.K[i][l], q[2], q[3]);
            }
        ready = true;
    }
    return h;
}

cudaError_t upload_model(cudaStream_t s)
{
    const HostModel& h = host_model();
    cudaError_t e;
    if ((e = cudaMemcpyToSymbolAsync(c_a, h.a, sizeof h.a, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_K, h.K, sizeof h.K, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_lnc, h.lnc, sizeof h.lnc, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_lnG_lo, h.lnG_lo, sizeof h.lnG_lo, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_lnG_hi, h.lnG_hi, sizeof h.lnG_hi, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(g_lnG_tab, h.tab, sizeof h.tab, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(g_dlnG_tab, h.dtab, sizeof h.dtab, 0, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyToSymbolAsync(g_slot, h.slot, sizeof h.slot, 0, cudaMemcpyHostToDevice, s))) return e;
    return cudaMemcpyToSymbolAsync(c_beta, BETA, sizeof BETA, 0, cudaMemcpyHostToDevice, s);
}

// vol: the cell volume; on an octree (leaf != NULL) the finest-lattice cell
// volume, times 8^(levels - level) for each leaf
__global__ void dust_mass_kernel(const float* __restrict__ kr, long long n, float vol, float* __restrict__ mass,
                                 const int4* __restrict__ leaf, int levels)
{
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x)
        mass[m] = kr[m] * (leaf ? ldexpf(vol, 3 * (levels - leaf[m].w)) : vol);
}

// FP64 -> FP32 by truncation of the significand, on the integer pipe (GB300
// retires FP64 and conversion instructions slowly); values below the FP32
// normal range map to zero, values above it take the ordinary conversion.
__device__ __forceinline__ float narrow_trunc(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7FF) - 1023 + 127;
    if (e >= 255) return (float)x;
    if (e <= 0) return 0.f;
    return __uint_as_float((unsigned)(u >> 32 & 0x80000000u) | ((unsigned)e << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
}

// band b covers the input wavelengths [start[b], start[b+1]) (sorted input
// grid).  One cell per lane, 32 cells per warp pass.  The warp walks the
// input wavelengths in order in blocks of 32 columns; each block of its 32
// rows is copied to shared memory by asynchronous copies (one 256-byte row
// segment per instruction, coalesced), which keep the kernel at 64 registers
// and 16 warps per SM (a register-staged block took 148 registers, 12 warps
// per SM, and 18% longer).  Each lane sums its row's bands in wavelength
// order (FP64) and, as the walk passes each band's end, adds the band sum to
// the cell's total (FP64, band order): per cell about n_in/32 + 1 FP64 warp
// instructions, a floor near the HBM time on GB300; each lane's serial walk
// and the staging latency set the rest.  The walk adds each band's columns of
// a block in one inner loop (the next band end held in a register); 32 empty
// cells in a row skip their FP64 adds.  The features are formed in FP32 and
// leave through a shared-memory transpose as coalesced rows.
constexpr int BF_WARPS = 2;  // warps per block
static_assert(NB == 32, "32 bands");

__global__ void __launch_bounds__(32 * BF_WARPS) band_features_kernel(
    const double* __restrict__ A, long long ncell, int n_in, const int* __restrict__ start,
    const float* __restrict__ mass, float* __restrict__ features, double* __restrict__ total)
{
    __shared__ int s_start[NB + 1];
    __shared__ double s_tile[BF_WARPS][32][33];  // staged column block [row][column], one padding column
    __shared__ float s_band[BF_WARPS][32][33];   // band sums, then features [row][band]
    for (int b = threadIdx.x; b <= NB; b += blockDim.x) s_start[b] = start[b];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double (*tile)[33] = s_tile[warp];
    float (*band)[33] = s_band[warp];
    for (long long base = ((long long)blockIdx.x * BF_WARPS + warp) * 32; base < ncell;
         base += (long long)gridDim.x * BF_WARPS * 32) {
        const int nrow = ncell - base < 32 ? (int)(ncell - base) : 32;
        int b = 0;
        double sb = 0.0, tot = 0.0;
        int nxt = s_start[1];  // the first column after band b
        bool live = false;     // warp-uniform: some staged block of these rows held a nonzero value
        for (int c0 = 0; c0 < n_in; c0 += 32) {
            const bool col_ok = c0 + lane < n_in;
            // the block's 32 row segments straight into shared memory (8-byte
            // asynchronous copies, one per lane and row: no register staging)
            __syncwarp();
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) {
                if (rr < nrow && col_ok) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(&tile[rr][lane]);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                                 "l"(A + (size_t)(base + rr) * n_in + c0 + lane) : "memory");
                } else {
                    tile[rr][lane] = 0.0;
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            const int cend = n_in - c0 < 32 ? n_in - c0 : 32;
            // a block that is zero on all 32 rows (a run of empty cells) adds nothing to
            // any band sum: the warp then skips its FP64 adds as a whole.  The test reads
            // the bits on the integer pipes and decides a real branch (a predicated-off
            // FP64 instruction would still hold the FP64 pipe for its full slot).  Once a
            // block of the 32 rows has held a nonzero value the rows are taken as live and
            // the later blocks are summed untested (cells are empty at every wavelength or
            // at few), which keeps the test's cost off the dense case.
            if (!live) {
                unsigned long long bits = 0ull;
                for (int jj = 0; jj < cend; ++jj)
                    bits |= (unsigned long long)__double_as_longlong(tile[lane][jj]);
                live = __any_sync(0xffffffffu, bits != 0ull);
            }
            if (live) {
                int jj = 0;
                while (jj < cend) {
                    // close the bands that end before this column (empty ones included)
                    while (b < NB && nxt <= c0 + jj) {
                        band[lane][b] = narrow_trunc(sb);
                        tot += sb;
                        sb = 0.0;
                        ++b;
                        nxt = b < NB ? s_start[b + 1] : 0x7fffffff;
                    }
                    // the columns of band b in this block, in order
                    const int seg = nxt - c0 < cend ? nxt - c0 : cend;
                    for (; jj < seg; ++jj) sb += tile[lane][jj];
                }
            } else {
                // the same closures, with no column to add
                while (b < NB && nxt <= c0 + cend - 1) {
                    band[lane][b] = narrow_trunc(sb);
                    tot += sb;
                    sb = 0.0;
                    ++b;
                    nxt = b < NB ? s_start[b + 1] : 0x7fffffff;
                }
            }
        }
        for (; b < NB; ++b) {
            band[lane][b] = narrow_trunc(sb);
            tot += sb;
            sb = 0.0;
        }
        const long long r = base + lane;
        const float M = lane < nrow ? mass[r] : 0.f;
        const float fl = 1e-6f * narrow_trunc(tot) / NB;
        const bool ok = M > 0.f && tot > 0.0;
        // an empty band sits 6 dex (per band) below the cell's total power
        for (int k = 0; k < NB; ++k)
            band[lane][k] = log10f(fmaxf(ok ? fmaxf(band[lane][k], fl) / M : 0.f, 1e-30f));
        if (lane < nrow) total[r] = tot;
        __syncwarp();
        for (int rr = 0; rr < nrow; ++rr) features[(size_t)(base + rr) * NB + lane] = band[rr][lane];
        __syncwarp();
    }
}

int band_blocks(long long ncell)
{
    long long b = (ncell + 32 * BF_WARPS - 1) / (32 * BF_WARPS);
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}

// The exact solve, one warp per batch of EX_BATCH rows.
//
// Per row and population i the solve needs P_i = sum_j w_ij A_j, the target
// ln G_i(T_i) = ln(P_i / M) - ln c_i, a start and bracket for T_i, one
// evaluation of G_i(T_i) = sum_l K_il / expm1(a_l / T_i) with T dG_i/dT, and
// a Newton test; the emission row is e_l = sum_i (P_i / G_i) K_il / expm1(a_l / T_i).
//
//  * Per population (FP64, lane 3r + i holds row r's population i, so the
//    EX_BATCH rows share each FP64 instruction): the target, the clamp to
//    3 or 2000 K, the table start, T_i, and after the evaluation the Newton
//    test on ln T.
//  * Per term (double-float, FP32 pipe; dfloat.cuh): the 300 terms of a row,
//    slots s = i * NOUT + l, lane j holding slots j + 32 k.  x = a_l / T_i,
//    expm1(x), its reciprocal, the term t = K_il q and its T dG/dT part
//    t x (1 + q) (binary32: it only sets the Newton step).  Terms with x > 70
//    are left out: over 3..2000 K they carry less than 4e-23 of G_i.
//  * The output row: with E the binary exponent of max_i P_i, the scaled
//    P_i 2^-E over G_i times each term, summed over the populations in
//    double-float, widened to FP64 and scaled by 2^E: every row sums to
//    sum_i P_i to the double-float rounding (~1e-14).
// The table start is within a few 1e-14 of the root, so the first evaluation
// passes the 1e-13 convergence test; a population that does not (the coarse-
// start diagnostic, or a rare target) continues Newton over the whole warp,
// and its row is evaluated and written again.
constexpr int NS = NPOP * NOUT;
constexpr int EX_SLOTS = (NS + 31) / 32;
constexpr int EX_WARPS = 4;   // warps per block
constexpr int EX_BATCH = 10;  // rows per warp batch: lanes 3r + i, r < 10
constexpr float X_CUT = 70.f;

// binary32 -> FP64 on the integer pipe: exact for normal numbers, zero for
// zero and subnormals (which the double-float terms only reach below 1e-23
// of a row)
__device__ __forceinline__ double widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    return e ? __hiloint2double((int)((u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u)), (int)(u << 29))
             : 0.0;
}

__device__ __forceinline__ double df_to_double(dfl::df2 v) { return widen(v.hi) + widen(v.lo); }

// v * 2^e for a normal v: the exponent field moved on the integer pipe; a
// result that would leave the normal range takes the multiplication
__device__ __forceinline__ double scale_pow2(double v, int e)
{
    const long long u = __double_as_longlong(v);
    const int ev = (int)((u >> 52) & 0x7FF);
    if (ev == 0 || ev + e <= 0 || ev + e >= 0x7FF) return v * __longlong_as_double((long long)(e + 1023) << 52);
    return __longlong_as_double(u + ((long long)e << 52));
}

// the warp sums of three values on every lane: one butterfly that halves the
// set of partial sums a lane carries at the first two levels (6 FP64 adds
// instead of 15); lanes 8k .. 8k+7 end with the sum of value k, broadcast
__device__ __forceinline__ void warp_sum3(double& a, double& b, double& c)
{
    const int lane = threadIdx.x & 31;
    const bool up = lane & 16;
    // level 16: the lower half keeps (a, b), the upper half (c, 0)
    double k0 = up ? c : a, k1 = up ? 0.0 : b;
    const double s0 = up ? a : c, s1 = up ? b : 0.0;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    // level 8: lanes with bit 3 keep the second value
    const bool hi8 = lane & 8;
    double k = hi8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    a = __shfl_sync(0xffffffffu, k, 0);
    b = __shfl_sync(0xffffffffu, k, 8);
    c = __shfl_sync(0xffffffffu, k, 16);
}

__device__ __forceinline__ dfl::df2 df_from_double(double v)
{
    const float h = __double2float_rn(v);
    return dfl::make(h, __double2float_rn(v - (double)h));
}

// a / b for b > 0 (double-float): the binary32 quotient and one correction
__device__ __forceinline__ dfl::df2 df_div(dfl::df2 a, dfl::df2 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    float p, e;
    dfl::two_prod(b.hi, q1, p, e);
    float r = __fsub_rn(a.hi, p);  // exact: q1 b.hi is within an ulp of a.hi
    r = __fsub_rn(r, e);
    r = __fadd_rn(r, a.lo);
    r = fmaf(-b.lo, q1, r);
    return dfl::renorm(q1, __fdiv_rn(r, b.hi));
}

struct TermOut {
    float th, tl, d;
};

// term of slot (a, K) at 1/T (double-float): t = K / expm1(a / T), and d =
// t x (1 + q) in binary32 (one copy of the code for every caller)
__device__ __noinline__ TermOut slot_term(float4 aK, float ih, float il)
{
    const dfl::df2 x = dfl::mul(dfl::make(aK.x, aK.y), dfl::make(ih, il));
    TermOut o = {0.f, 0.f, 0.f};
    if (x.hi <= X_CUT) {
        const dfl::df2 q = dfl::recip(dfl::expm1(x));
        const dfl::df2 t = dfl::mul(dfl::make(aK.z, aK.w), q);
        o.th = t.hi;
        o.tl = t.lo;
        o.d = t.hi * x.hi * (1.f + q.hi);
    }
    return o;
}

__device__ __forceinline__ void warp_sum_df(dfl::df2& v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const dfl::df2 w = dfl::make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
        v = dfl::add(v, w);  // add(a, b) == add(b, a) bit for bit: every lane ends with the same sum
    }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One row: every slot at its population's 1/T (populations with on bit i),
// G_i (double-float) and T dG_i/dT (binary32) over the warp, and the output
// row written from the same terms (staged in buf) with the scaled powers
// Pp_i (P_i 2^-E).  The slot loop is not unrolled and the term is one
// non-inlined routine: unrolled, the solve's code outgrew the instruction
// cache and the warps stalled on instruction fetch.
__device__ __forceinline__ void eval_row(const float4* __restrict__ slot, const dfl::df2 (&iT)[NPOP], unsigned on,
                                         const dfl::df2 (&Pp)[NPOP], int scale_e, double* __restrict__ out,
                                         float2* __restrict__ buf, int lane, dfl::df2 (&G)[NPOP], float (&D)[NPOP])
{
    if (on == 0u) {  // no population absorbs (a dust-free or unheated cell): a zero row
#pragma unroll
        for (int i = 0; i < NPOP; ++i) {
            G[i] = dfl::make(0.f, 0.f);
            D[i] = 0.f;
        }
        for (int l = lane; l < NOUT; l += 32) __stcs(out + l, 0.0);
        return;
    }
    dfl::df2 g0 = dfl::make(0.f, 0.f), g1 = g0, g2 = g0;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll 1
    for (int j = 0; j < EX_SLOTS; ++j) {
        const int s = lane + 32 * j;
        const int i = s < NOUT ? 0 : (s < 2 * NOUT ? 1 : 2);
        TermOut o = {0.f, 0.f, 0.f};
        if (s < NS && ((on >> i) & 1u)) {
            const dfl::df2 it = i == 0 ? iT[0] : (i == 1 ? iT[1] : iT[2]);
            o = slot_term(slot[s], it.hi, it.lo);
        }
        if (s < NS) buf[s] = make_float2(o.th, o.tl);
        const dfl::df2 tt = dfl::make(o.th, o.tl);
        if (i == 0) { g0 = dfl::add(g0, tt); d0 += o.d; }
        else if (i == 1) { g1 = dfl::add(g1, tt); d1 += o.d; }
        else { g2 = dfl::add(g2, tt); d2 += o.d; }
    }
    warp_sum_df(g0); warp_sum_df(g1); warp_sum_df(g2);
    G[0] = g0; G[1] = g1; G[2] = g2;
    D[0] = warp_sum_f(d0); D[1] = warp_sum_f(d1); D[2] = warp_sum_f(d2);
    dfl::df2 PS[NPOP];
#pragma unroll
    for (int i = 0; i < NPOP; ++i)
        PS[i] = (((on >> i) & 1u) && G[i].hi > 0.f) ? df_div(Pp[i], G[i]) : dfl::make(0.f, 0.f);
    __syncwarp();
    for (int l = lane; l < NOUT; l += 32) {
        const float2 b0 = buf[l], b1 = buf[NOUT + l], b2 = buf[2 * NOUT + l];
        const dfl::df2 e = dfl::add(dfl::add(dfl::mul(PS[0], dfl::make(b0.x, b0.y)), dfl::mul(PS[1], dfl::make(b1.x, b1.y))),
                                    dfl::mul(PS[2], dfl::make(b2.x, b2.y)));
        __stcs(out + l, scale_pow2(df_to_double(e), scale_e));
    }
    __syncwarp();
}

// G_i and T dG_i/dT at 1/T for one population, the lanes splitting the
// wavelengths (the rare Newton solve that needs more than one evaluation)
__device__ void pop_G_warp(const float4* __restrict__ slot, int i, dfl::df2 iT, int lane, double& G, double& D)
{
    dfl::df2 g = dfl::make(0.f, 0.f);
    float d = 0.f;
    for (int l = lane; l < NOUT; l += 32) {
        const TermOut o = slot_term(slot[i * NOUT + l], iT.hi, iT.lo);
        g = dfl::add(g, dfl::make(o.th, o.tl));
        d += o.d;
    }
    warp_sum_df(g);
    G = df_to_double(g);
    D = (double)warp_sum_f(d);
}

// Starting point and bracket of the Newton solve for ln G_i(e^y) = target:
// the table interval holding the target (binary search), and the cubic
// Hermite inverse of ln G on it (slopes dy/d lnG = 1 / (d lnG / dy)).  With
// 4096 intervals over [ln 3, ln 2000] the start is within a few 1e-14 of the
// root (the Hermite error falls as the fourth power of the spacing).  stride
// > 1 uses every stride-th point only (a coarser start that needs further
// Newton steps; a diagnostic setting).
__device__ __forceinline__ void start_T(int i, double target, int stride, double& y, double& lo, double& hi)
{
    const double* tab = &g_lnG_tab[i][0];
    const double* dtab = &g_dlnG_tab[i][0];
    int a = 0, b = (NTAB - 1) / stride;  // tab[a stride] <= target < tab[b stride]
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (__ldg(tab + mid * stride) <= target) a = mid; else b = mid;
    }
    const double dy = (log(T_HI) - log(T_LO)) / (NTAB - 1) * stride;
    lo = log(T_LO) + a * dy;
    hi = lo + dy;
    a *= stride;
    b *= stride;
    const double ga = __ldg(tab + a), gb = __ldg(tab + b);
    const double h = gb - ga, u = (target - ga) / h;
    const double sa = 1.0 / __ldg(dtab + a), sb = 1.0 / __ldg(dtab + b);
    const double u2 = u * u, u3 = u2 * u;
    y = (2.0 * u3 - 3.0 * u2 + 1.0) * lo + (u3 - 2.0 * u2 + u) * h * sa + (3.0 * u2 - 2.0 * u3) * hi +
        (u3 - u2) * h * sb;
    if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
}

// Exact emission for rows m = rows ? rows[k] : k, k < nrows.  A second
// absorbed table A2 [ncell][n2] with its shares w2 (may be NULL) adds its
// power to each population's.
__global__ void __launch_bounds__(32 * EX_WARPS) exact_kernel(
    const double* __restrict__ A, int n_in, const double* __restrict__ w, const double* __restrict__ A2, int n2,
    const double* __restrict__ w2, const float* __restrict__ mass, const unsigned* __restrict__ rows, long long nrows,
    double* __restrict__ emission, float* __restrict__ temperature, int stride)
{
    __shared__ float4 s_slot[NS];
    __shared__ float2 s_buf[EX_WARPS][NS];
    for (int s = threadIdx.x; s < NS; s += blockDim.x) s_slot[s] = g_slot[s];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* buf = s_buf[warp];
    const int my_r = lane / NPOP, my_i = lane - NPOP * (lane / NPOP);  // this lane's (row, population)
    for (long long base = ((long long)blockIdx.x * EX_WARPS + warp) * EX_BATCH; base < nrows;
         base += (long long)gridDim.x * EX_WARPS * EX_BATCH) {
        const int nb = nrows - base < EX_BATCH ? (int)(nrows - base) : EX_BATCH;
        const bool mine = my_r < nb;
        const long long my_m = mine ? (rows ? (long long)rows[base + my_r] : base + my_r) : 0;
        // ---- population powers, one row at a time over the lanes (FP64)
        double P = 0.0;
        int E = 0;
        for (int r = 0; r < nb; ++r) {
            const long long m = rows ? (long long)rows[base + r] : base + r;
            const double* row = A + (size_t)m * n_in;
            double p0 = 0.0, p1 = 0.0, p2 = 0.0;
            for (int j = lane; j < n_in; j += 32) {
                const double v = __ldcs(row + j);
                p0 += __ldg(w + j) * v;
                p1 += __ldg(w + n_in + j) * v;
                p2 += __ldg(w + 2 * n_in + j) * v;
            }
            if (A2) {
                const double* row2 = A2 + (size_t)m * n2;
                for (int j = lane; j < n2; j += 32) {
                    const double v = __ldcs(row2 + j);
                    p0 += __ldg(w2 + j) * v;
                    p1 += __ldg(w2 + n2 + j) * v;
                    p2 += __ldg(w2 + 2 * n2 + j) * v;
                }
            }
            warp_sum3(p0, p1, p2);
            if (my_r == r) {
                P = my_i == 0 ? p0 : (my_i == 1 ? p1 : p2);
                // binary exponent of the row's largest population power (0 if none is positive)
                const double pm = fmax(fmax(p0, p1), p2);
                E = pm > 0.0 ? ((__double2hiint(pm) >> 20) & 0x7FF) - 1023 : 0;
                E = E < -1000 ? -1000 : (E > 1000 ? 1000 : E);
            }
        }
        // ---- per population (FP64): target, clamp or table start, 1/T, scaled power
        const float M = mine ? mass[my_m] : 0.f;
        int kind = 0;  // 0 no power, 1 clamped, 2 Newton
        double tg = 0.0, y = 0.0, lo = 0.0, hi = 0.0, T = 0.0;
        dfl::df2 iT = dfl::make(0.f, 0.f), Pp = dfl::make(0.f, 0.f);
        if (mine && P > 0.0 && M > 0.f) {
            tg = log(P / (double)M) - c_lnc[my_i];
            if (c_lnG_lo[my_i] - tg >= 0.0) {
                kind = 1;
                T = T_LO;
            } else if (c_lnG_hi[my_i] - tg <= 0.0) {
                kind = 1;
                T = T_HI;
            } else {
                kind = 2;
                start_T(my_i, tg, stride, y, lo, hi);
                T = exp(y);
            }
            iT = df_from_double(1.0 / T);
            Pp = df_from_double(P * __longlong_as_double((long long)(1023 - E) << 52));
        }
        const unsigned on_all = __ballot_sync(0xffffffffu, kind != 0);
        // ---- one evaluation per row (double-float); lane 3r + i keeps its G_i, D_i
        dfl::df2 Gm = dfl::make(0.f, 0.f);
        float Dm = 0.f;
        for (int r = 0; r < nb; ++r) {
            const int l0 = NPOP * r;
            dfl::df2 iTr[NPOP], Ppr[NPOP], G[NPOP];
            float D[NPOP];
#pragma unroll
            for (int i = 0; i < NPOP; ++i) {
                iTr[i] = dfl::make(__shfl_sync(0xffffffffu, iT.hi, l0 + i), __shfl_sync(0xffffffffu, iT.lo, l0 + i));
                Ppr[i] = dfl::make(__shfl_sync(0xffffffffu, Pp.hi, l0 + i), __shfl_sync(0xffffffffu, Pp.lo, l0 + i));
            }
            const int Er = __shfl_sync(0xffffffffu, E, l0);
            const long long m = rows ? (long long)rows[base + r] : base + r;
            eval_row(s_slot, iTr, (on_all >> l0) & 7u, Ppr, Er, emission + (size_t)m * NOUT, buf, lane, G, D);
            if (my_r == r) {
                Gm = my_i == 0 ? G[0] : (my_i == 1 ? G[1] : G[2]);
                Dm = my_i == 0 ? D[0] : (my_i == 1 ? D[1] : D[2]);
            }
        }
        // ---- Newton test of every population (FP64)
        bool redo = false;
        if (kind == 2) {
            // converged when the Newton step is below 1e-13 of ln T (tested before the
            // bracket: a start exact to the last bit gives a zero step, and y itself
            // then sits on the updated bracket's end)
            const double G = df_to_double(Gm);
            const double f = log(G) - tg;
            const double step = f * G / (double)Dm;
            if (!(fabs(step) <= 1e-13 * fabs(y))) {
                if (f < 0.0) lo = y; else hi = y;
                double y_new = y - step;
                if (!(y_new > lo && y_new < hi)) y_new = 0.5 * (lo + hi);
                redo = true;
                y = y_new;
            }
        }
        unsigned redo_mask = __ballot_sync(0xffffffffu, redo);
        while (redo_mask) {  // rare: Newton continues for one population over the whole warp
            const int L = __ffs(redo_mask) - 1;
            redo_mask &= redo_mask - 1;
            const int ri = L / NPOP, ii = L - NPOP * ri;
            double yi = __shfl_sync(0xffffffffu, y, L), loi = __shfl_sync(0xffffffffu, lo, L),
                   hii = __shfl_sync(0xffffffffu, hi, L);
            const double tgi = __shfl_sync(0xffffffffu, tg, L);
            double Ti = exp(yi), Gi = 0.0, Di = 0.0;
            for (int it = 1; it < 100; ++it) {
                Ti = exp(yi);
                pop_G_warp(s_slot, ii, df_from_double(1.0 / Ti), lane, Gi, Di);
                const double f = log(Gi) - tgi;
                const double step = f * Gi / Di;
                if (fabs(step) <= 1e-13 * fabs(yi)) break;
                if (f < 0.0) loi = yi; else hii = yi;
                double y_new = yi - step;
                if (!(y_new > loi && y_new < hii)) y_new = 0.5 * (loi + hii);
                yi = y_new;
                if (it == 99) Ti = exp(yi);  // iteration limit: the last point
            }
            if (lane == L) {
                T = Ti;
                iT = df_from_double(1.0 / Ti);
            }
            // the row again, with the population's final temperature
            const int l0 = NPOP * ri;
            dfl::df2 iTr[NPOP], Ppr[NPOP], G[NPOP];
            float D[NPOP];
#pragma unroll
            for (int i = 0; i < NPOP; ++i) {
                iTr[i] = dfl::make(__shfl_sync(0xffffffffu, iT.hi, l0 + i), __shfl_sync(0xffffffffu, iT.lo, l0 + i));
                Ppr[i] = dfl::make(__shfl_sync(0xffffffffu, Pp.hi, l0 + i), __shfl_sync(0xffffffffu, Pp.lo, l0 + i));
            }
            const int Er = __shfl_sync(0xffffffffu, E, l0);
            const long long m = rows ? (long long)rows[base + ri] : base + ri;
            eval_row(s_slot, iTr, (on_all >> l0) & 7u, Ppr, Er, emission + (size_t)m * NOUT, buf, lane, G, D);
        }
        if (temperature && mine) temperature[(size_t)my_m * NPOP + my_i] = (float)T;
    }
}

__global__ void compact_flags_kernel(const unsigned char* __restrict__ flags, long long n,
                                     unsigned* __restrict__ rows, unsigned long long* __restrict__ count)
{
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
        const bool f = flags[m] != 0;
        const unsigned mask = __ballot_sync(__activemask(), f);
        if (!f) continue;
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(mask) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
        base = __shfl_sync(mask, base, leader);
        rows[base + __popc(mask & ((1u << lane) - 1u))] = (unsigned)m;
    }
}

__global__ void zero_temperature_kernel(float* t, long long n)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        t[k] = 0.f;
}

int grid_blocks(long long n, int block)
{
    long long b = (n + block - 1) / block;
    if (b > 152LL * 64) b = 152LL * 64;
    return (int)(b < 1 ? 1 : b);
}

bool is_device(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_lambda(const double* lambda_in, int n_in)
{
    if (!lambda_in || n_in < 1 || n_in > 65536) return set_error(SKIRT_ERR_INVALID_ARG, "lambda_in / n_in invalid");
    for (int j = 0; j < n_in; ++j) {
        if (!(lambda_in[j] > 0) || !std::isfinite(lambda_in[j]))
            return set_error(SKIRT_ERR_INVALID_ARG, "lambda_in[%d] must be finite and > 0", j);
        if (j > 0 && !(lambda_in[j] > lambda_in[j - 1]))
            return set_error(SKIRT_ERR_INVALID_ARG, "lambda_in must be strictly increasing");
    }
    return SKIRT_OK;
}

// band start indices over a sorted grid: band b = floor(32 ln(l/lmin) / ln(lmax/lmin)) clamped
std::vector<int> band_starts(const double* lam, int n)
{
    std::vector<int> idx(n, 0);
    const double lo = lam[0], hi = lam[n - 1];
    for (int j = 0; j < n; ++j) {
        int b = 0;
        if (hi > lo) b = (int)std::floor(NB * std::log(lam[j] / lo) / std::log(hi / lo));
        idx[j] = b < 0 ? 0 : (b > NB - 1 ? NB - 1 : b);
    }
    std::vector<int> start(NB + 1, n);
    for (int b = NB; b >= 0; --b) {
        int s = n;
        for (int j = 0; j < n; ++j)
            if (idx[j] >= b) { s = j; break; }
        start[b] = b == NB ? n : s;
    }
    return start;
}

std::vector<double> share_table(const double* lam, int n)
{
    std::vector<double> w((size_t)NPOP * n);
    for (int j = 0; j < n; ++j) {
        double r[NPOP], sum = 0.0;
        for (int i = 0; i < NPOP; ++i) {
            r[i] = std::pow(lam[j] / 0.55, DELTA[i]);
            sum += r[i];
        }
        for (int i = 0; i < NPOP; ++i) w[(size_t)i * n + j] = r[i] / sum;
    }
    return w;
}

#define ECK(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return set_error(e_ == cudaErrorMemoryAllocation ? SKIRT_ERR_OOM : SKIRT_ERR_CUDA,          \
                             "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

}  // namespace

int launch_exact_emission(const double* absorbed, int n_in, const double* w_dev, const float* mass,
                          const unsigned* rows, long long nrows, double* emission, float* temperature,
                          cudaStream_t s, const double* absorbed2, int n2, const double* w2_dev)
{
    ECK(upload_model(s));
    // one warp per batch of rows, every row list alike (all cells, or the
    // surrogate's fallback rows).  SKIRT_EXACT_TABLE_STRIDE (a power of two up to 64)
    // starts the Newton solves from a coarser table: the same results through
    // more Newton steps, a diagnostic of that path.
    int stride = 1;
    if (const char* e = std::getenv("SKIRT_EXACT_TABLE_STRIDE")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 64 && (v & (v - 1)) == 0) stride = v;
    }
    if (nrows > 0) {
        long long blocks = (nrows + EX_WARPS * EX_BATCH - 1) / (EX_WARPS * EX_BATCH);
        if (blocks > 152LL * 32) blocks = 152LL * 32;
        exact_kernel<<<(int)blocks, 32 * EX_WARPS, 0, s>>>(absorbed, n_in, w_dev, absorbed2, n2, w2_dev, mass, rows,
                                                           nrows, emission, temperature, stride);
    }
    ECK(cudaGetLastError());
    return SKIRT_OK;
}

}  // namespace skirt

using namespace skirt;

extern "C" int skirt_emission_grid(double* lambda_um, double* weights)
{
    const HostModel& h = host_model();
    if (lambda_um) std::memcpy(lambda_um, h.lam, sizeof h.lam);
    if (weights) std::memcpy(weights, h.W, sizeof h.W);
    return SKIRT_OK;
}

extern "C" int skirt_dust_mass(skirt_grid_t g, float* mass, void* stream)
{
    if (!g || !mass) return set_error(SKIRT_ERR_INVALID_ARG, "grid / mass is NULL");
    if (!is_device(mass)) return set_error(SKIRT_ERR_INVALID_ARG, "mass must be device memory");
    const double vol = (g->bbox[1] - g->bbox[0]) / g->nx * (g->bbox[3] - g->bbox[2]) / g->ny *
                       (g->bbox[5] - g->bbox[4]) / g->nz;
    dust_mass_kernel<<<grid_blocks(g->ncell, 256), 256, 0, (cudaStream_t)stream>>>(g->kr32, g->ncell, (float)vol, mass,
                                                                                  g->oct_leaf, g->oct_levels);
    ECK(cudaGetLastError());
    ECK(cudaStreamSynchronize((cudaStream_t)stream));
    return SKIRT_OK;
}

extern "C" int skirt_band_features(const double* absorbed, long long ncell, int n_in, const double* lambda_in,
                                   const float* mass, float* features, double* total, void* stream)
{
    if (ncell < 0) return set_error(SKIRT_ERR_INVALID_ARG, "ncell < 0");
    if (int r = check_lambda(lambda_in, n_in)) return r;
    if (ncell == 0) return SKIRT_OK;
    if (!is_device(absorbed) || !is_device(mass) || !is_device(features) || !is_device(total))
        return set_error(SKIRT_ERR_INVALID_ARG, "absorbed / mass / features / total must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> start = band_starts(lambda_in, n_in);
    int* d_start = nullptr;
    ECK(cudaMallocAsync((void**)&d_start, sizeof(int) * (NB + 1), s));
    ECK(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * (NB + 1), cudaMemcpyHostToDevice, s));
    band_features_kernel<<<band_blocks(ncell), 32 * BF_WARPS, 0, s>>>(absorbed, ncell, n_in, d_start, mass, features, total);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d_start, s);
    if (e != cudaSuccess) return set_error(SKIRT_ERR_CUDA, "band features: %s", cudaGetErrorString(e));
    ECK(cudaStreamSynchronize(s));
    return SKIRT_OK;
}

extern "C" int skirt_dust_emission(const double* absorbed, long long ncell, int n_in, const double* lambda_in,
                                   const float* mass, int mode, skirt_mlp_t net, double* emission, float* temperature,
                                   skirt_emission_stats* stats, void* stream)
{
    if (ncell < 0) return set_error(SKIRT_ERR_INVALID_ARG, "ncell < 0");
    if (int r = check_lambda(lambda_in, n_in)) return r;
    if (mode != SKIRT_EMIT_EXACT && mode != SKIRT_EMIT_SURROGATE)
        return set_error(SKIRT_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (mode == SKIRT_EMIT_SURROGATE && !net) return set_error(SKIRT_ERR_INVALID_ARG, "surrogate mode needs a network");
    if (stats) std::memset(stats, 0, sizeof *stats);
    if (ncell == 0) return SKIRT_OK;
    if (ncell >= (1ll << 32)) return set_error(SKIRT_ERR_INVALID_ARG, "ncell must be < 2^32");
    if (!is_device(absorbed) || !is_device(mass) || !is_device(emission) || (temperature && !is_device(temperature)))
        return set_error(SKIRT_ERR_INVALID_ARG, "absorbed / mass / emission / temperature must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> w = share_table(lambda_in, n_in);
    double* d_w = nullptr;
    ECK(cudaMallocAsync((void**)&d_w, sizeof(double) * w.size(), s));
    ECK(cudaMemcpyAsync(d_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s));
    cudaEvent_t ev[4];
    for (auto& e : ev) ECK(cudaEventCreate(&e));
    int rc = SKIRT_OK;
    unsigned long long nfb = 0;
    if (mode == SKIRT_EMIT_EXACT) {
        ECK(cudaEventRecord(ev[0], s));
        rc = launch_exact_emission(absorbed, n_in, d_w, mass, nullptr, ncell, emission, temperature, s);
        ECK(cudaEventRecord(ev[1], s));
    } else {
        // the working tables live in the network's workspace (grown on demand, kept
        // between calls): a stream-ordered allocation of ~2.5 GB per call cost ~5 ms
        std::unique_lock<std::mutex> ws_lock(mlp_workspace_mutex(net));
        // on every way out of this block (errors included) the stream drains
        // before the lock is released, so no other call reuses tables in use
        struct DrainOnExit {
            cudaStream_t s;
            ~DrainOnExit() { cudaStreamSynchronize(s); }
        } drain{s};
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t o_tot = 0, o_cnt = o_tot + al(sizeof(double) * (size_t)ncell), o_start = o_cnt + al(8),
                     o_feat = o_start + al(sizeof(int) * (NB + 1)),
                     o_rows = o_feat + al(sizeof(float) * NB * (size_t)ncell),
                     o_flag = o_rows + al(sizeof(unsigned) * (size_t)ncell), ws_total = o_flag + al((size_t)ncell);
        unsigned char* ws = nullptr;
        if (int r = mlp_workspace(net, ws_total, (void**)&ws)) {
            cudaFreeAsync(d_w, s);
            for (auto& e : ev) cudaEventDestroy(e);
            return r;
        }
        double* d_tot = (double*)(ws + o_tot);
        unsigned long long* d_cnt = (unsigned long long*)(ws + o_cnt);
        int* d_start = (int*)(ws + o_start);
        float* d_feat = (float*)(ws + o_feat);
        unsigned* d_rows = (unsigned*)(ws + o_rows);
        unsigned char* d_flag = ws + o_flag;
        ECK(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s));
        std::vector<int> start = band_starts(lambda_in, n_in);
        ECK(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * (NB + 1), cudaMemcpyHostToDevice, s));
        if (temperature) zero_temperature_kernel<<<grid_blocks(3 * ncell, 256), 256, 0, s>>>(temperature, 3 * ncell);
        ECK(cudaEventRecord(ev[0], s));
        band_features_kernel<<<band_blocks(ncell), 32 * BF_WARPS, 0, s>>>(absorbed, ncell, n_in, d_start, mass, d_feat, d_tot);
        ECK(cudaGetLastError());
        ECK(cudaEventRecord(ev[1], s));
        rc = mlp_forward_internal(net, d_feat, d_tot, ncell, emission, d_flag, s);
        if (rc == SKIRT_OK) {
            compact_flags_kernel<<<grid_blocks(ncell, 256), 256, 0, s>>>(d_flag, ncell, d_rows, d_cnt);
            ECK(cudaGetLastError());
            ECK(cudaEventRecord(ev[2], s));
            ECK(cudaMemcpyAsync(&nfb, d_cnt, sizeof nfb, cudaMemcpyDeviceToHost, s));
            ECK(cudaStreamSynchronize(s));
            rc = launch_exact_emission(absorbed, n_in, d_w, mass, d_rows, (long long)nfb, emission, temperature, s);
            ECK(cudaEventRecord(ev[3], s));
        }
    }
    cudaFreeAsync(d_w, s);
    ECK(cudaStreamSynchronize(s));
    if (rc == SKIRT_OK && mode == SKIRT_EMIT_SURROGATE) rc = mlp_check_timeout();
    if (stats && rc == SKIRT_OK) {
        stats->n_cells = (unsigned long long)ncell;
        stats->n_fallback = nfb;
        float a = 0.f, b = 0.f, c = 0.f;
        if (mode == SKIRT_EMIT_EXACT) {
            cudaEventElapsedTime(&c, ev[0], ev[1]);
        } else {
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b, ev[1], ev[2]);
            cudaEventElapsedTime(&c, ev[2], ev[3]);
        }
        stats->ms_features = a;
        stats->ms_surrogate = b;
        stats->ms_exact = c;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
}

extern "C" int skirt_dust_emission_pair(const double* absorbed_a, long long ncell, int n_a, const double* lambda_a,
                                        const double* absorbed_b, int n_b, const double* lambda_b, const float* mass,
                                        double* emission, float* temperature, void* stream)
{
    if (ncell < 0) return set_error(SKIRT_ERR_INVALID_ARG, "ncell < 0");
    if (int r = check_lambda(lambda_a, n_a)) return r;
    if (absorbed_b || n_b) {
        if (!absorbed_b) return set_error(SKIRT_ERR_INVALID_ARG, "absorbed_b is NULL with n_b > 0");
        if (int r = check_lambda(lambda_b, n_b)) return r;
    }
    if (ncell == 0) return SKIRT_OK;
    if (ncell >= (1ll << 32)) return set_error(SKIRT_ERR_INVALID_ARG, "ncell must be < 2^32");
    if (!is_device(absorbed_a) || (absorbed_b && !is_device(absorbed_b)) || !is_device(mass) ||
        !is_device(emission) || (temperature && !is_device(temperature)))
        return set_error(SKIRT_ERR_INVALID_ARG, "absorbed / mass / emission / temperature must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> w = share_table(lambda_a, n_a);
    if (absorbed_b) {
        const std::vector<double> wb = share_table(lambda_b, n_b);
        w.insert(w.end(), wb.begin(), wb.end());
    }
    double* d_w = nullptr;
    ECK(cudaMallocAsync((void**)&d_w, sizeof(double) * w.size(), s));
    ECK(cudaMemcpyAsync(d_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s));
    int rc = launch_exact_emission(absorbed_a, n_a, d_w, mass, nullptr, ncell, emission, temperature, s, absorbed_b,
                                   absorbed_b ? n_b : 0, absorbed_b ? d_w + (size_t)NPOP * n_a : nullptr);
    cudaFreeAsync(d_w, s);
    ECK(cudaStreamSynchronize(s));
    return rc;
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Allocation-free exact emission.
//
// skirt_dust_emission allocates its per-call working table (the absorption
// share of every input wavelength for the three grain populations) with the
// stream-ordered allocator.  Some callers cannot allocate device memory at
// call time: a process whose framework allocator has already reserved the
// device memory it may use, or a loop with a fixed memory budget decided up
// front.  skirt_dust_emission_exact_static does the same exact solve with that
// table in the fixed array below instead (3 x 4096 doubles = 96 KiB, held by
// every device that loads the library until the process exits).
// ---------------------------------------------------------------------------
namespace {

constexpr int STATIC_MAX_NIN = 4096;
static __device__ __align__(256) double g_static_shares[NPOP * STATIC_MAX_NIN];

std::mutex g_static_mutex;
double* g_static_ptr[64] = {};  // device address of g_static_shares, per device ordinal
double g_static_host[NPOP * STATIC_MAX_NIN];  // host copy of the table (guarded by g_static_mutex)

// shares w_i(lambda_j) = (lambda_j/0.55)^delta_i / sum_k (lambda_j/0.55)^delta_k into out[i*n + j]
void fill_shares(const double* lam, int n, double* out)
{
    for (int j = 0; j < n; ++j) {
        double r[NPOP], sum = 0.0;
        for (int i = 0; i < NPOP; ++i) {
            r[i] = std::pow(lam[j] / 0.55, DELTA[i]);
            sum += r[i];
        }
        for (int i = 0; i < NPOP; ++i) out[(size_t)i * n + j] = r[i] / sum;
    }
}

}  // namespace

extern "C" int skirt_dust_emission_exact_static(const double* absorbed, long long ncell, int n_in,
                                                const double* lambda_in, const float* mass, double* emission,
                                                float* temperature, void* stream)
{
    if (ncell < 0) return set_error(SKIRT_ERR_INVALID_ARG, "ncell < 0");
    if (n_in > STATIC_MAX_NIN)
        return set_error(SKIRT_ERR_INVALID_ARG, "n_in = %d exceeds the static table's maximum of %d wavelengths",
                         n_in, STATIC_MAX_NIN);
    if (int r = check_lambda(lambda_in, n_in)) return r;
    if (ncell == 0) return SKIRT_OK;
    if (ncell >= (1ll << 32)) return set_error(SKIRT_ERR_INVALID_ARG, "ncell must be < 2^32");
    if (!is_device(absorbed) || !is_device(mass) || !is_device(emission) || (temperature && !is_device(temperature)))
        return set_error(SKIRT_ERR_INVALID_ARG, "absorbed / mass / emission / temperature must be device memory");
    int dev = 0;
    ECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(SKIRT_ERR_NO_DEVICE, "device ordinal %d out of range", dev);
    cudaStream_t s = (cudaStream_t)stream;
    double* shares = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        // once per device, with that device current: the device address of the array
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_shares);
            if (e != cudaSuccess || !p)
                return set_error(SKIRT_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_static_ptr[dev] = (double*)p;
        }
        shares = g_static_ptr[dev];
        // the table is rewritten in full by every call (no part needs zeroing).  The copy
        // reads the shared host buffer, so it has to finish before another thread may
        // refill that buffer: the stream is synchronised before the lock is released
        // (CUDA does not promise that an asynchronous copy from pageable memory has
        // read its source when the call returns).
        fill_shares(lambda_in, n_in, g_static_host);
        ECK(cudaMemcpyAsync(shares, g_static_host, sizeof(double) * NPOP * n_in, cudaMemcpyHostToDevice, s));
        ECK(cudaStreamSynchronize(s));
    }
    int rc = launch_exact_emission(absorbed, n_in, shares, mass, nullptr, ncell, emission, temperature, s);
    ECK(cudaStreamSynchronize(s));
    return rc;
}
