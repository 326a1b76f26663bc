// Photon-packet life cycle on the GPU, mixed form: FP32 cell traversal,
// directions, phase-function sampling and packet luminosity; FP64 cumulative
// optical depth, tallies and energy ledger.
//
// Same method as the FP64 form (Sect. 3.2 stellar emission phase: launch,
// peel-off towards every instrument, continuous absorption into the
// [cell, wavelength] table, forced scattering, life until a negligible
// luminosity is left; Sect. 1 for the techniques; Sect. 5.2 for the table
// layout and lock-free additions), organised for a GPU whose FP64 unit
// retires a warp instruction only every few dozen cycles per sub-partition:
// every FP64 or FP32<->FP64 conversion instruction a warp issues, even with
// one lane active, costs that much.  So:
//
//  * Warp-coherent stepping.  All lanes of a warp step one cell per round
//    whatever traversal they are in (deposit, forced-interaction search,
//    peel-off line of sight).  A lane whose traversal ended idles until fewer
//    than step_min lanes are still stepping; then the idle lanes handle
//    their events (launch, scattering, peel-off tally) together.
//  * Per cell crossing only FP32 arithmetic.  The optical depth of every
//    crossing is FP32 and the running optical depth is their error-free
//    double-float sum (Knuth two-sum: hi + lo, ~46-bit significand, exact
//    up to its final rounding); at every event it is formed as an FP64
//    value.  The sum depends only on the packet, never on the schedule.
//    Deposits are formed in FP32 and widened to FP64 by integer bit
//    operations for the reduction.
//  * Positions are double-float pairs (hi + lo, ~48 bits).  Face planes come
//    from exact per-grid tables; the distance from a start point to its first
//    faces and the snapping of an interaction point onto the plane through
//    which its cell was entered keep full relative precision for points deep
//    inside optically thick cells (~1/(kappa rho) from a face).  The
//    interaction cell found by the search is carried into the next
//    traversals.
//  * Per event, escaped / absorbed / scattered come from one
//    om = 1 - e^{-tau_path}, so they add up to the packet luminosity.
//  * Per-thread state used only at events lives in shared memory.
#include <cuda_runtime.h>
#include <math.h>

#include "skirt_internal.cuh"
#include "trace_device.cuh"

namespace skirt {
namespace {

constexpr int MAXB = 256;       // threads per block of the mixed kernel (upper bound)
constexpr int ROUND = 8;        // cell crossings per stepping round between warp votes

// FP32 -> FP64 by IEEE-754 field manipulation on the integer pipe: exact for
// normal floats; zero and FP32 subnormals map to zero.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xFFu;
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                    ((unsigned long long)(ex + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return ex ? __longlong_as_double((long long)bits) : 0.0;
}

// FP32 -> FP64 for a positive normal float: the double's high word is the
// float's bits shifted right by 3 with the exponent re-biased by 1023 - 127,
// its low word the three mantissa bits shifted out.
__device__ __forceinline__ double f2d_pos(float f)
{
    const unsigned u = __float_as_uint(f);
    return __hiloint2double((int)((u >> 3) + 0x38000000u), (int)(u << 29));
}

// e^{-x} for x >= 0 as 2^{-x log2 e} with the PTX base-2 exponential
// (ex2.approx, relative error ~2^-22); the FP32 product x log2 e contributes
// an error of the same order as the FP32 rounding of x itself.  Results below
// the FP32 normal range flush to zero.
__device__ __forceinline__ float exp_neg(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-1.4426950408889634f * x));
    return y;
}

// 1 - e^{-x} for x >= 0, accurate in relative terms: below 1/4 the Taylor
// series x (1 - x g(x)) with g(x) = 1/2! - x/3! + x^2/4! - ... - x^5/7!
// (Horner form with constant coefficients: six multiply-adds), whose first
// omitted term is below 4e-10 of the result; 1 - e^{-x} above, where no
// cancellation occurs.  Both branches are evaluated and selected.
__device__ __forceinline__ float one_minus_exp_neg(float x)
{
    const float g = fmaf(fmaf(fmaf(fmaf(fmaf(-1.f / 5040.f, x, 1.f / 720.f), x, -1.f / 120.f), x, 1.f / 24.f), x,
                         -1.f / 6.f), x, 0.5f);
    const float p = x * fmaf(g, -x, 1.f);
    const float q = 1.f - exp_neg(x);
    return x < 0.25f ? p : q;
}

// (hi, lo) += v, error-free: hi takes the rounded sum, lo collects the exact
// rounding errors (two-sum).
__device__ __forceinline__ void df_accumulate(float& hi, float& lo, float v)
{
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// Double-float arithmetic (Knuth / Dekker error-free transformations), with
// round-to-nearest intrinsics so that nothing is contracted into an FMA.
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb)), __fadd_rn(lo, pe));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

__device__ __forceinline__ float df_diff(float2 f, float xh, float xl)
{
    return __fadd_rn(__fsub_rn(f.x, xh), __fsub_rn(f.y, xl));
}

// Per-thread state used only at events, struct of arrays in shared memory.
struct Cold {
    double l_emit[MAXB], l_abs[MAXB], l_esc[MAXB], l_res[MAXB];
    unsigned long long q[MAXB], q_end[MAXB];
    unsigned long long c_dep[MAXB], c_loc[MAXB], c_peel[MAXB], c_scat[MAXB];
    float L0[MAXB], p_esc[MAXB], p_abs[MAXB], p_res[MAXB], p_peel[MAXB], om[MAXB], peel_w[MAXB], alb[MAXB];
    float xl0[MAXB], xl1[MAXB], xl2[MAXB];  // low words of the double-float position
    int lam[MAXB], led_lam[MAXB], nscat[MAXB], peel_i[MAXB], after_peel[MAXB], peel_kind[MAXB];
    unsigned pk[MAXB], ev[MAXB], started[MAXB];
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// OCT: octree grid (Sect. 7.9).  The traversal state then names a leaf
// (node, level, lattice corner) instead of a cell; a crossing reads the face
// neighbour and descends from it by the lattice cell of the entry point.
template <bool OCT>
__global__ void __launch_bounds__(MAXB, 3) trace_mixed_kernel(const TraceArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    InstrDev* sins = reinterpret_cast<InstrDev*>(smem);
    Cold& C = *reinterpret_cast<Cold*>(smem + align16(sizeof(InstrDev) * A.ninstr));
    for (int i = threadIdx.x; i < A.ninstr; i += blockDim.x) sins[i] = A.ins[i];
    const int t = threadIdx.x;
    C.l_emit[t] = C.l_abs[t] = C.l_esc[t] = C.l_res[t] = 0.0;
    C.q[t] = C.q_end[t] = 0;
    C.c_dep[t] = C.c_loc[t] = C.c_peel[t] = C.c_scat[t] = 0;
    C.lam[t] = -1;
    C.led_lam[t] = -1;
    C.started[t] = 0;
    __syncthreads();

    const int NL = A.nlambda;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const float lo0 = (float)A.lo[0], lo1 = (float)A.lo[1], lo2 = (float)A.lo[2];
    const float d0 = (float)A.d[0], d1 = (float)A.d[1], d2 = (float)A.d[2];
    const float INF = __int_as_float(0x7f800000);
    const float* __restrict__ kr = A.kr32;
    const float2* __restrict__ fx = A.faces;
    const float2* __restrict__ fy = A.faces + (nx + 1);
    const float2* __restrict__ fz = A.faces + (nx + 1) + (ny + 1);
    double* __restrict__ absorbed = A.absorbed;
    const int step_min = A.step_min > 0 ? A.step_min : 20;
    const float tau_cut = A.tau_cut;  // optical depth after which a deposit / peel-off traversal stops

    // ---- stepping state (registers)
    int mode = M_NONE;
    int c0 = 0, c1 = 0, c2 = 0, s0 = 0, s1 = 0, s2 = 0;
    float iv0 = 0.f, iv1 = 0.f, iv2 = 0.f, tn0 = 0.f, tn1 = 0.f, tn2 = 0.f, tcur = 0.f;
    float tau_h = 0.f, tau_l = 0.f;  // running optical depth of the traversal (double-float)
    float rem_f = 0.f;               // interaction optical depth (search)
    unsigned nsteps = 0;
    float labs_f = 0.f;
    float s_found = 0.f, last_dusty_end = 0.f;
    bool found = false;
    int last_axis = -1;  // axis of the face through which the current cell was entered
    int cur_m = 0;       // index of the current cell
    float kr_cur = 0.f;  // its extinction coefficient (loaded one crossing ahead)
    const int nxy = nx * ny;
    // octree: the current leaf's node and level (c0..c2: its lattice corner),
    // the traversal direction, the node of the interaction leaf
    const int OL = A.oct_levels;
    const OctNode* __restrict__ nodes = A.oct_nodes;
    const float id0 = 1.f / d0, id1 = 1.f / d1, id2 = 1.f / d2;
    int onode = 0, olev = 0, pc_node = 0;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    // ---- packet state (registers)
    int stage = ST_NEW;
    bool alive = true;
    int lam = 0;
    float krs = 0.f, gg = 0.f, L = 0.f;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;  // position, high words
    float k0 = 0.f, k1 = 0.f, k2 = 0.f;
    bool have_pc = false;
    int pc0 = 0, pc1 = 0, pc2 = 0;

    auto axis_cell = [&](float xh, float xl, float lo, float d, int n, const float2* f) {
        int c = (int)fminf(fmaxf(floorf((xh - lo) / d), 0.f), (float)(n - 1));
        if (c > 0 && df_diff(__ldg(f + c), xh, xl) > 0.f) --c;
        else if (c < n - 1 && df_diff(__ldg(f + c + 1), xh, xl) <= 0.f) ++c;
        return c;
    };

    // octree: enter the leaf holding lattice cell (j0, j1, j2), descending
    // from `node` (a leaf, or a node of level `lev`)
    auto oct_enter = [&](int node, int lev, int j0, int j1, int j2) {
        int2 h = __ldg(reinterpret_cast<const int2*>(nodes + node));
        while (h.x >= 0 && lev < OL) {
            ++lev;
            const int b = OL - lev;
            node = h.x + (((j0 >> b) & 1) | (((j1 >> b) & 1) << 1) | (((j2 >> b) & 1) << 2));
            h = __ldg(reinterpret_cast<const int2*>(nodes + node));
        }
        onode = node;
        olev = oct_leaf_level(h.x);
        cur_m = oct_leaf_index(h.x);
        kr_cur = __int_as_float(h.y);
        const int mask = ~((1 << (OL - olev)) - 1);
        c0 = j0 & mask;
        c1 = j1 & mask;
        c2 = j2 & mask;
    };

    auto begin = [&](int m, float vx, float vy, float vz) {
        mode = m;
        const float l0 = C.xl0[t], l1 = C.xl1[t], l2 = C.xl2[t];
        if (have_pc) {
            c0 = pc0; c1 = pc1; c2 = pc2;
        } else {
            c0 = axis_cell(x0, l0, lo0, d0, nx, fx);
            c1 = axis_cell(x1, l1, lo1, d1, ny, fy);
            c2 = axis_cell(x2, l2, lo2, d2, nz, fz);
        }
        if constexpr (OCT) {
            if (have_pc) oct_enter(pc_node, 0, c0, c1, c2);
            else oct_enter(0, 0, c0, c1, c2);
            v0 = vx; v1 = vy; v2 = vz;
        }
        s0 = vx > 0.f ? 1 : (vx < 0.f ? -1 : 0);
        s1 = vy > 0.f ? 1 : (vy < 0.f ? -1 : 0);
        s2 = vz > 0.f ? 1 : (vz < 0.f ? -1 : 0);
        iv0 = s0 ? 1.f / vx : 0.f;
        iv1 = s1 ? 1.f / vy : 0.f;
        iv2 = s2 ? 1.f / vz : 0.f;
        // first faces from the exact face planes and the double-float position
        const int e = OCT ? 1 << (OL - olev) : 1;  // the cell's extent in lattice cells
        tn0 = s0 ? df_diff(__ldg(fx + c0 + (s0 > 0 ? e : 0)), x0, l0) * iv0 : INF;
        tn1 = s1 ? df_diff(__ldg(fy + c1 + (s1 > 0 ? e : 0)), x1, l1) * iv1 : INF;
        tn2 = s2 ? df_diff(__ldg(fz + c2 + (s2 > 0 ? e : 0)), x2, l2) * iv2 : INF;
        tcur = 0.f;
        tau_h = tau_l = 0.f;
        nsteps = 0;
        last_axis = -1;
        if constexpr (!OCT) {
            cur_m = (c2 * ny + c1) * nx + c0;
            kr_cur = __ldg(kr + cur_m);
        }
    };

    // one leaf crossing of an octree traversal: the face neighbour and its
    // node are loaded before the crossing's work
    auto step_oct = [&]() {
        const float tmin = fminf(fminf(tn0, tn1), tn2);
        const int axis = (tn0 == tmin) ? 0 : ((tn1 == tmin) ? 1 : 2);
        const int ss = axis == 0 ? s0 : (axis == 1 ? s1 : s2);
        // a face inside the parent leads to the sibling, whose index follows
        // from the leaf's own (children blocks start at multiples of 8);
        // only a face on the parent's boundary needs the stored neighbour
        const bool inner = olev > 0 && ((onode >> axis) & 1) == (ss < 0 ? 1 : 0);
        const int nb = inner ? onode ^ (1 << axis) : __ldg(&nodes[onode].nb[2 * axis + (ss > 0)]);
        const bool out = nb < 0;
        const int2 nbh = out ? make_int2(0, 0) : __ldg(reinterpret_cast<const int2*>(nodes + nb));
        const float ds = fmaxf(tmin - tcur, 0.f);
        const int m = cur_m;
        const float krl = kr_cur * krs;
        const float dtau = krl * ds;
        ++nsteps;
        bool done = false;
        const float tau_prev = tau_h + tau_l;
        if (mode == M_LOCATE) {
            if (krl > 0.f) {
                if (tau_h + (tau_l + dtau) >= rem_f) {
                    s_found = (rem_f - tau_prev) / krl;
                    found = true;
                    done = true;
                } else {
                    last_dusty_end = tmin;
                }
            }
        } else if (mode == M_DEPOSIT && dtau > 0.f) {
            const float dep = labs_f * exp_neg(tau_prev) * one_minus_exp_neg(dtau);
            if (dep >= 1.17549435e-38f)
                atomicAdd(absorbed + ((size_t)m * A.abs_cs + (size_t)lam * A.abs_ls), f2d_pos(dep));
        }
        df_accumulate(tau_h, tau_l, dtau);
        if (!done) {
            tcur = tmin;
            if (out) {
                done = true;
            } else if (nsteps > (unsigned)A.oct_step_cap) {
                atomicOr(A.err, (unsigned)ERRBIT_PATH);
                done = true;
            } else {
                // lattice cell of the entry point: across the exit face along
                // `axis`, elsewhere the crossing point's cell kept within the
                // current leaf's cross-section
                const int e = 1 << (OL - olev);
                const float p0 = floorf((x0 + tmin * v0 - lo0) * id0);
                const float p1 = floorf((x1 + tmin * v1 - lo1) * id1);
                const float p2 = floorf((x2 + tmin * v2 - lo2) * id2);
                int j0 = (int)fminf(fmaxf(p0, (float)c0), (float)(c0 + e - 1));
                int j1 = (int)fminf(fmaxf(p1, (float)c1), (float)(c1 + e - 1));
                int j2 = (int)fminf(fmaxf(p2, (float)c2), (float)(c2 + e - 1));
                const int ja = ss > 0 ? (axis == 0 ? c0 : (axis == 1 ? c1 : c2)) + e
                                      : (axis == 0 ? c0 : (axis == 1 ? c1 : c2)) - 1;
                j0 = axis == 0 ? ja : j0;
                j1 = axis == 1 ? ja : j1;
                j2 = axis == 2 ? ja : j2;
                // a neighbour that is not a leaf has the current level
                if (nbh.x < 0) {
                    onode = nb;
                    olev = oct_leaf_level(nbh.x);
                    cur_m = oct_leaf_index(nbh.x);
                    kr_cur = __int_as_float(nbh.y);
                    const int mask = ~((1 << (OL - olev)) - 1);
                    c0 = j0 & mask;
                    c1 = j1 & mask;
                    c2 = j2 & mask;
                } else {
                    oct_enter(nb, olev, j0, j1, j2);
                }
                const int en = 1 << (OL - olev);
                tn0 = s0 ? (lo0 + (float)(c0 + (s0 > 0 ? en : 0)) * d0 - x0) * iv0 : INF;
                tn1 = s1 ? (lo1 + (float)(c1 + (s1 > 0 ? en : 0)) * d1 - x1) * iv1 : INF;
                tn2 = s2 ? (lo2 + (float)(c2 + (s2 > 0 ? en : 0)) * d2 - x2) * iv2 : INF;
                last_axis = axis;
            }
        }
        if (tau_h > tau_cut && mode != M_LOCATE) done = true;
        if (done) mode = M_NONE;
    };

    // one cell crossing of the current traversal
    auto step = [&]() {
        const float tmin = fminf(fminf(tn0, tn1), tn2);
        const int axis = (tn0 == tmin) ? 0 : ((tn1 == tmin) ? 1 : 2);
        // the next cell is known before the current one is processed: issue
        // its density load now so that it overlaps with this crossing's work
        const int cs = axis == 0 ? c0 : (axis == 1 ? c1 : c2);
        const int ss = axis == 0 ? s0 : (axis == 1 ? s1 : s2);
        const int na = axis == 0 ? nx : (axis == 1 ? ny : nz);
        const int cn = cs + ss;
        const bool out = (unsigned)cn >= (unsigned)na;
        const int mn = cur_m + ss * (axis == 0 ? 1 : (axis == 1 ? nx : nxy));
        const float kr_next = out ? 0.f : __ldg(kr + mn);
        const float ds = fmaxf(tmin - tcur, 0.f);
        const int m = cur_m;
        const float krl = kr_cur * krs;
        const float dtau = krl * ds;
        ++nsteps;
        bool done = false;
        const float tau_prev = tau_h + tau_l;
        if (mode == M_LOCATE) {
            if (krl > 0.f) {
                if (tau_h + (tau_l + dtau) >= rem_f) {
                    s_found = (rem_f - tau_prev) / krl;  // distance inside the current cell
                    found = true;
                    done = true;
                } else {
                    last_dusty_end = tmin;
                }
            }
        } else if (mode == M_DEPOSIT && dtau > 0.f) {
            const float dep = labs_f * exp_neg(tau_prev) * one_minus_exp_neg(dtau);
            if (dep >= 1.17549435e-38f)
                atomicAdd(absorbed + ((size_t)m * A.abs_cs + (size_t)lam * A.abs_ls), f2d_pos(dep));
        }
        df_accumulate(tau_h, tau_l, dtau);
        if (!done) {
            tcur = tmin;
            if (out) {
                done = true;
            } else {
                cur_m = mn;
                kr_cur = kr_next;
                const float loa = axis == 0 ? lo0 : (axis == 1 ? lo1 : lo2);
                const float da = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
                const float xa = axis == 0 ? x0 : (axis == 1 ? x1 : x2);
                const float iva = axis == 0 ? iv0 : (axis == 1 ? iv1 : iv2);
                const float tnew = (loa + (float)(cn + (ss > 0)) * da - xa) * iva;
                c0 = axis == 0 ? cn : c0;
                c1 = axis == 1 ? cn : c1;
                c2 = axis == 2 ? cn : c2;
                tn0 = axis == 0 ? tnew : tn0;
                tn1 = axis == 1 ? tnew : tn1;
                tn2 = axis == 2 ? tnew : tn2;
                last_axis = axis;
            }
        }
        // Beyond tau = tau_cut (30) a line of sight transmits < e^-30 (1e-13) and a
        // deposit path has handed < e^-30 of the luminosity to its remaining
        // cells; 1 - e^-tau is 1 in FP32 from tau = 17 on, so the forced
        // scattering draw does not change: the traversal ends there (the search
        // never gets that far, since tau_int < 17 in FP32).
        if (tau_h > tau_cut && mode != M_LOCATE) done = true;
        if (done) mode = M_NONE;
    };

    auto draw = [&](uint32_t event, uint32_t block) -> uint4 {
        return philox10(make_uint4(C.pk[t], (uint32_t)lam, event, (A.phase << 24) | block), A.key0, A.key1);
    };

    auto flush_ledger = [&]() {
        const int ll = C.led_lam[t];
        if (ll >= 0) {
            double* lg = A.ledger + 4 * (size_t)ll;
            atomicAdd(lg + 0, C.l_emit[t]);
            atomicAdd(lg + 1, C.l_abs[t]);
            atomicAdd(lg + 2, C.l_esc[t]);
            atomicAdd(lg + 3, C.l_res[t]);
        }
        C.l_emit[t] = C.l_abs[t] = C.l_esc[t] = C.l_res[t] = 0.0;
    };

    auto start_peel = [&](int i) {
        const InstrDev& I = sins[i];
        float w;
        if (C.peel_kind[t] == 0) {
            w = L;  // isotropic emission: phase factor 1
        } else {
            const float mu = k0 * I.kobs_f[0] + k1 * I.kobs_f[1] + k2 * I.kobs_f[2];
            w = L * hg_phase<float>(gg, mu);
        }
        C.peel_w[t] = w;
        if (w > 0.f) begin(M_PEEL, I.kobs_f[0], I.kobs_f[1], I.kobs_f[2]);
        else nsteps = 0;
    };

    // event handling: runs the lane's stages until it enters a traversal or
    // runs out of packets
    auto events = [&]() {
        while (mode == M_NONE && alive) {
            if (stage == ST_NEW) {
                if (C.q[t] >= C.q_end[t]) {
                    if (!A.persistent) {
                        if (C.started[t]) { alive = false; break; }
                        C.started[t] = 1;
                        const unsigned long long q = A.q_base + (unsigned long long)blockIdx.x * blockDim.x + t;
                        C.q[t] = q;
                        C.q_end[t] = (q < A.q_base + A.q_count) ? q + 1 : q;
                        if (C.q[t] >= C.q_end[t]) { alive = false; break; }
                    } else {
                        const unsigned mask = __activemask();
                        const int lane = t & 31;
                        const int leader = __ffs(mask) - 1;
                        const unsigned rank = __popc(mask & ((1u << lane) - 1u));
                        unsigned long long base = 0;
                        if (lane == leader)
                            base = atomicAdd(A.queue, (unsigned long long)__popc(mask) * (unsigned long long)A.chunk);
                        base = __shfl_sync(mask, base, leader);
                        const unsigned long long q = base + (unsigned long long)rank * A.chunk;
                        if (q >= A.total) { alive = false; break; }
                        C.q[t] = q;
                        C.q_end[t] = q + A.chunk < A.total ? q + A.chunk : A.total;
                    }
                }
                const unsigned long long qq = C.q[t]++;
                int ll = C.lam[t];
                if (ll < 0 || qq < __ldg(A.offsets + ll) || qq >= __ldg(A.offsets + ll + 1)) {
                    int a = 0, b = NL - 1;  // last wavelength whose offset <= qq
                    while (a < b) {
                        const int mid = (a + b + 1) >> 1;
                        if (__ldg(A.offsets + mid) <= qq) a = mid; else b = mid - 1;
                    }
                    ll = a;
                    C.lam[t] = ll;
                    C.alb[t] = __ldg(A.albedo_f + ll);
                    C.L0[t] = __ldg(A.L0_f + ll);
                    if (C.led_lam[t] != ll) {
                        flush_ledger();
                        C.led_lam[t] = ll;
                    }
                }
                lam = ll;
                krs = __ldg(A.kscale_f + lam);
                gg = __ldg(A.g_f + lam);
                C.pk[t] = (unsigned)(qq - __ldg(A.offsets + lam) + __ldg(A.pk_first + lam));
                L = C.L0[t];
                C.p_esc[t] = C.p_abs[t] = C.p_res[t] = C.p_peel[t] = 0.f;
                C.ev[t] = 0;
                C.nscat[t] = 0;
                C.l_emit[t] += f2d(L);
                have_pc = false;
                float l0 = 0.f, l1 = 0.f, l2 = 0.f;

                // ---- launch (Sect. 3.2)
                bool isotropic = true;
                if (A.src_kind == SKIRT_SRC_BEAM || A.src_kind == SKIRT_SRC_POINT) {
                    x0 = A.src_df[0].x; x1 = A.src_df[1].x; x2 = A.src_df[2].x;
                    l0 = A.src_df[0].y; l1 = A.src_df[1].y; l2 = A.src_df[2].y;
                    if (A.src_kind == SKIRT_SRC_BEAM) {
                        k0 = A.src_dir_f[0]; k1 = A.src_dir_f[1]; k2 = A.src_dir_f[2];
                        isotropic = false;
                    }
                } else if (A.src_kind == SKIRT_SRC_DISK) {
                    const float hR = (float)A.h_R, hz = (float)A.h_z;
                    for (uint32_t tries = 0;; ++tries) {
                        const uint4 r = draw(0u, tries == 0 ? 0u : tries + 1u);
                        const float u0 = u01f(r.x), u1 = u01f(r.y), u2 = u01f(r.z), u3 = u01f(r.w);
                        const float Rr = -hR * (logf(u0) + logf(u1));
                        const float z = (u2 < 0.5f) ? hz * logf(2.f * u2) : -hz * logf(2.f * (1.f - u2));
                        float sp, cp;
                        sincospif(2.f * u3, &sp, &cp);
                        x0 = A.src_df[0].x + Rr * cp;
                        x1 = A.src_df[1].x + Rr * sp;
                        x2 = A.src_df[2].x + z;
                        if (x0 >= lo0 && x0 <= A.hi_f[0] && x1 >= lo1 && x1 <= A.hi_f[1] && x2 >= lo2 && x2 <= A.hi_f[2])
                            break;
                        if (tries + 1 >= 64) {
                            atomicOr(A.err, (unsigned)ERRBIT_SOURCE);
                            x0 = A.src_df[0].x; x1 = A.src_df[1].x; x2 = A.src_df[2].x;
                            break;
                        }
                    }
                } else {  // SKIRT_SRC_DUST
                    const uint4 r = draw(0u, 0u);
                    const long long ncell = A.ncell;
                    const double* cdf = A.cdf + (size_t)lam * ncell;
                    const double u0 = f2d(u01f(r.x));
                    long long a = 0, b = ncell - 1;  // first cell with cdf > u0
                    while (a < b) {
                        const long long mid = (a + b) >> 1;
                        if (__ldg(cdf + mid) > u0) b = mid; else a = mid + 1;
                    }
                    float side = 1.f;  // the cell's extent in lattice cells
                    if constexpr (OCT) {
                        // uniform point in the leaf's box; its leaf is found again
                        // from the position
                        const int4 lf = __ldg(&A.oct_leaf[a]);
                        pc0 = lf.x; pc1 = lf.y; pc2 = lf.z;
                        side = (float)(1 << (OL - lf.w));
                    } else {
                        pc0 = (int)(a % nx);
                        pc1 = (int)((a / nx) % ny);
                        pc2 = (int)(a / ((long long)nx * ny));
                    }
                    const float2 f0 = __ldg(fx + pc0), f1 = __ldg(fy + pc1), f2 = __ldg(fz + pc2);
                    x0 = f0.x; l0 = f0.y;
                    x1 = f1.x; l1 = f1.y;
                    x2 = f2.x; l2 = f2.y;
                    df_add_prod(x0, l0, u01f(r.y), side * d0);
                    df_add_prod(x1, l1, u01f(r.z), side * d1);
                    df_add_prod(x2, l2, u01f(r.w), side * d2);
                    have_pc = !OCT;
                }
                C.xl0[t] = l0; C.xl1[t] = l1; C.xl2[t] = l2;
                if (isotropic) {
                    const uint4 r = draw(0u, 1u);
                    const float mu = 2.f * u01f(r.x) - 1.f;
                    const float st = sqrtf(fmaxf(1.f - mu * mu, 0.f));
                    float sp, cp;
                    sincospif(2.f * u01f(r.y), &sp, &cp);
                    k0 = st * cp; k1 = st * sp; k2 = mu;
                }
                if (isotropic && A.peel && A.ninstr > 0) {
                    C.peel_kind[t] = 0;
                    C.peel_i[t] = 0;
                    C.after_peel[t] = ST_START_DEP;
                    stage = ST_PEEL_DONE;
                    start_peel(0);
                } else {
                    stage = ST_START_DEP;
                }
                continue;
            }

            if (stage == ST_START_DEP) {
                C.ev[t] += 1;
                labs_f = L * (1.f - C.alb[t]);
                begin(M_DEPOSIT, k0, k1, k2);
                stage = ST_DEPOSIT_DONE;
                continue;
            }

            if (stage == ST_DEPOSIT_DONE) {
                C.c_dep[t] += nsteps;
                const double tau_path = f2d(tau_h) + f2d(tau_l);  // the path's optical depth, FP64
                // om = 1 - e^{-tau_path}: from expm1 for small tau, from 1 - exp for
                // large tau, so that both om and 1 - om keep FP32 relative precision
                const float tf = tau_h + tau_l;
                float om, E;
                if (tf < 0.6931472f) { om = -expm1f(-tf); E = 1.f - om; }
                else { E = expf(-tf); om = 1.f - E; }
                C.p_esc[t] += L * E;
                C.p_abs[t] += L * (1.f - C.alb[t]) * om;
                if (!(tau_path > 0.0)) {
                    if (!(tau_path == 0.0)) atomicOr(A.err, (unsigned)ERRBIT_NONFINITE);
                    L = 0.f;
                    C.nscat[t] = (int)C.ev[t] - 1;
                    stage = ST_END_PACKET;
                    continue;
                }
                C.om[t] = om;
                // forced scattering: tau_int from the exponential truncated at tau_path
                const uint4 r = draw(C.ev[t], 0u);
                const float tau_int = -log1pf(-u01f(r.x) * om);
                begin(M_LOCATE, k0, k1, k2);
                rem_f = tau_int;
                found = false;
                last_dusty_end = 0.f;
                stage = ST_LOCATE_DONE;
                continue;
            }

            if (stage == ST_LOCATE_DONE) {
                C.c_loc[t] += nsteps;
                float l0 = C.xl0[t], l1 = C.xl1[t], l2 = C.xl2[t];
                if (found && last_axis >= 0) {
                    // entry point of the interaction cell, snapped onto the exact face plane
                    df_add_prod(x0, l0, tcur, k0);
                    df_add_prod(x1, l1, tcur, k1);
                    df_add_prod(x2, l2, tcur, k2);
                    const int e = OCT ? 1 << (OL - olev) : 1;
                    if (last_axis == 0) { const float2 f = __ldg(fx + c0 + (s0 < 0 ? e : 0)); x0 = f.x; l0 = f.y; }
                    else if (last_axis == 1) { const float2 f = __ldg(fy + c1 + (s1 < 0 ? e : 0)); x1 = f.x; l1 = f.y; }
                    else { const float2 f = __ldg(fz + c2 + (s2 < 0 ? e : 0)); x2 = f.x; l2 = f.y; }
                    df_add_prod(x0, l0, s_found, k0);
                    df_add_prod(x1, l1, s_found, k1);
                    df_add_prod(x2, l2, s_found, k2);
                } else {
                    const float s = found ? s_found : last_dusty_end;
                    df_add_prod(x0, l0, s, k0);
                    df_add_prod(x1, l1, s, k1);
                    df_add_prod(x2, l2, s, k2);
                }
                C.xl0[t] = l0; C.xl1[t] = l1; C.xl2[t] = l2;
                have_pc = found;
                if (found) { pc0 = c0; pc1 = c1; pc2 = c2; pc_node = onode; }
                L = L * C.alb[t] * C.om[t];
                C.nscat[t] = (int)C.ev[t];
                if (L > 0.f && A.peel && A.ninstr > 0) {
                    C.peel_kind[t] = 1;
                    C.peel_i[t] = 0;
                    C.after_peel[t] = ST_AFTER_SCATTER;
                    stage = ST_PEEL_DONE;
                    start_peel(0);
                } else {
                    stage = ST_AFTER_SCATTER;
                }
                continue;
            }

            if (stage == ST_PEEL_DONE) {
                C.c_peel[t] += nsteps;
                const int pi = C.peel_i[t];
                const InstrDev& I = sins[pi];
                const float w = C.peel_w[t];
                if (w > 0.f) {
                    const float tobs = tau_h + tau_l;
                    const float flux = w * expf(-tobs) * I.flux_norm_f;
                    C.p_peel[t] += flux;
                    const float a = x0 * I.e1_f[0] + x1 * I.e1_f[1] + x2 * I.e1_f[2] +
                                    (C.xl0[t] * I.e1_f[0] + C.xl1[t] * I.e1_f[1] + C.xl2[t] * I.e1_f[2]);
                    const float b = x0 * I.e2_f[0] + x1 * I.e2_f[1] + x2 * I.e2_f[2] +
                                    (C.xl0[t] * I.e2_f[0] + C.xl1[t] * I.e2_f[1] + C.xl2[t] * I.e2_f[2]);
                    const float fa = floorf((a + I.half_fov_f) * I.inv_dpx_f);
                    const float fb = floorf((b + I.half_fov_f) * I.inv_dpx_f);
                    if (flux >= 1.17549435e-38f) {
                        // one FP64 reduction per peel-off (lanes of a warp rarely share a
                        // pixel; aggregating them measured no faster)
                        if (fa >= 0.f && fa < (float)I.npx && fb >= 0.f && fb < (float)I.npx) {
                            const long long pix = (long long)fb * I.npx + (long long)fa;
                            atomicAdd(A.images + I.img_off + pix * NL + lam, f2d(flux));
                        } else {
                            atomicAdd(A.oof + (size_t)pi * NL + lam, f2d(flux));
                        }
                    }
                }
                C.peel_i[t] = pi + 1;
                if (pi + 1 < A.ninstr) start_peel(pi + 1);
                else stage = C.after_peel[t];
                continue;
            }

            if (stage == ST_AFTER_SCATTER) {
                if (L <= A.w_min_f * C.L0[t]) {
                    C.p_res[t] += L;
                    stage = ST_END_PACKET;
                } else if ((int)C.ev[t] >= A.max_events) {
                    atomicOr(A.err, (unsigned)ERRBIT_EVENT_CAP);
                    C.p_res[t] += L;
                    stage = ST_END_PACKET;
                } else {
                    // Henyey-Greenstein scattering: mu by inverse CDF, azimuth uniform
                    const uint4 r = draw(C.ev[t], 0u);
                    const float mu = hg_mu<float>(gg, u01f(r.y));
                    float sp, cp;
                    sincospif(2.f * u01f(r.z), &sp, &cp);
                    hg_rotate<float>(k0, k1, k2, mu, sp, cp);
                    stage = ST_START_DEP;
                }
                continue;
            }

            // ST_END_PACKET
            C.c_scat[t] += (unsigned long long)C.nscat[t];
            const float pe = C.p_esc[t], pa = C.p_abs[t], pr = C.p_res[t], pp = C.p_peel[t];
            C.l_abs[t] += f2d(pa);
            C.l_esc[t] += f2d(pe);
            C.l_res[t] += f2d(pr);
            if (!isfinite(pe + pa + pr + pp)) atomicOr(A.err, (unsigned)ERRBIT_NONFINITE);
            const unsigned pk = C.pk[t] - (unsigned)__ldg(A.pk_first + lam);  // index within this call
            if (pk < (unsigned)A.nrec) {
                double* rec = A.records + ((size_t)lam * A.nrec + pk) * SKIRT_REC_FIELDS;
                rec[0] = (double)C.nscat[t];
                rec[1] = f2d(pe);
                rec[2] = f2d(pa);
                rec[3] = f2d(pr);
                rec[4] = f2d(pp);
                rec[5] = f2d(x0) + f2d(C.xl0[t]);
                rec[6] = f2d(x1) + f2d(C.xl1[t]);
                rec[7] = f2d(x2) + f2d(C.xl2[t]);
            }
            stage = ST_NEW;
        }
    };

    for (;;) {
        const bool stepping = mode != M_NONE;
        const unsigned sm = __ballot_sync(0xffffffffu, stepping);
        const unsigned wm = __ballot_sync(0xffffffffu, !stepping && alive);
        if (!(sm | wm)) break;
        if (sm && (__popc(sm) >= step_min || !wm)) {
#pragma unroll 1
            for (int r = 0; r < ROUND; ++r) {
                if constexpr (OCT) {
                    if (mode != M_NONE) step_oct();
                } else {
                    if (mode != M_NONE) step();
                }
            }
            continue;
        }
        if (!stepping && alive) events();
    }

    flush_ledger();
    atomicAdd(A.counters + 0, C.c_scat[t]);
    atomicAdd(A.counters + 1, C.c_dep[t]);
    atomicAdd(A.counters + 2, C.c_loc[t]);
    atomicAdd(A.counters + 3, C.c_peel[t]);
}

}  // namespace

size_t trace_mixed_smem_bytes(int ninstr, int block)
{
    (void)block;
    return align16(sizeof(InstrDev) * ninstr) + sizeof(Cold);
}

static cudaError_t set_smem_limit()
{
    cudaError_t e = cudaFuncSetAttribute(trace_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)trace_mixed_smem_bytes(16, MAXB));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(trace_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)trace_mixed_smem_bytes(16, MAXB));
}

cudaError_t launch_trace_mixed(const TraceArgs& a, int block, int grid, cudaStream_t s)
{
    if (block > MAXB || block % 32) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_limit();
    if (e != cudaSuccess) return e;
    if (a.oct_levels > 0)
        trace_mixed_kernel<true><<<grid, block, trace_mixed_smem_bytes(a.ninstr, block), s>>>(a);
    else
        trace_mixed_kernel<false><<<grid, block, trace_mixed_smem_bytes(a.ninstr, block), s>>>(a);
    return cudaGetLastError();
}

cudaError_t trace_mixed_occupancy(int block, int* blocks_per_sm, bool octree)
{
    if (block > MAXB || block % 32) {
        *blocks_per_sm = 0;
        return cudaSuccess;
    }
    cudaError_t e = set_smem_limit();
    if (e != cudaSuccess) return e;
    return octree ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_mixed_kernel<true>, block,
                                                                  trace_mixed_smem_bytes(16, block))
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_mixed_kernel<false>, block,
                                                                  trace_mixed_smem_bytes(16, block));
}

}  // namespace skirt
