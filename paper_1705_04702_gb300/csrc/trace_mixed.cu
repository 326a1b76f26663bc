// Photon-packet life cycle on the GPU, mixed form: FP32 positions,
// directions, cell traversal and phase-function sampling; FP64 cumulative
// optical depth, packet luminosity and tallies.
//
// Same method as the FP64 form (Sect. 3.2 stellar emission phase: launch,
// peel-off towards every instrument, continuous absorption into the
// [cell, wavelength] table, forced scattering, life until a negligible
// luminosity is left; Sect. 1 for the techniques; Sect. 5.2 for the table
// layout and lock-free additions), organised for a GPU whose FP64 and
// FP32<->FP64 conversion rates are ~1/64 of its FP32 rate:
//
//  * Warp-coherent stepping.  All lanes of a warp step one cell per round
//    whatever traversal they are in (deposit, forced-interaction search,
//    peel-off line of sight).  A lane whose traversal ended idles until fewer
//    than step_min lanes are still stepping; then the idle lanes handle
//    their events (launch, scattering, peel-off tally) together.  This keeps
//    the long, branchy event code from running with one lane active.
//  * No FP64 per cell crossing.  The optical depth of each crossing is FP32;
//    up to FLUSH of them are summed in FP32 and the partial sum is added to
//    an FP64 running total.  The forced-interaction search compares in FP32
//    against the remainder (tau_int - FP64 total).  The deposit factor
//    e^{-tau_prev}(1 - e^{-dtau}) is evaluated in FP32 and widened once for
//    the FP64 reduction.
//  * The packet position is kept in FP64 (touched only at events).  Each
//    traversal takes the distance to its first faces in FP64 and the later
//    faces in FP32.  An interaction point is placed on the exact plane of the
//    face through which its cell was entered plus the in-cell distance, so
//    that points deep inside optically thick cells (where the interaction
//    sits ~1/(kappa rho) from the face) keep their relative precision.  The
//    interaction cell found by the search (a decision taken on the optical
//    depth) is carried into the next traversals.
//  * Per event, the escaped / absorbed / scattered split uses one
//    om = 1 - e^{-tau_path}, so escaped + absorbed + scattered = L to FP64
//    rounding, and the per-packet absorbed luminosity is L (1 - albedo) om.
//  * Cold per-thread state (bookkeeping touched only at events) lives in
//    shared memory, leaving registers for the stepping state.
#include <cuda_runtime.h>
#include <math.h>

#include "skirt_internal.cuh"
#include "trace_device.cuh"

namespace skirt {
namespace {

constexpr int MAXB = 256;   // threads per block of the mixed kernel (upper bound)
constexpr int FLUSH = 16;   // FP32 partial optical depths per FP64 accumulation
constexpr int ROUND = 4;    // cell crossings per stepping round between warp votes

// Per-thread state used only at events, struct of arrays in shared memory.
struct Cold {
    double L0[MAXB], p_esc[MAXB], p_abs[MAXB], p_res[MAXB], p_peel[MAXB];
    double tau_t[MAXB], om[MAXB], peel_w[MAXB];
    double xd0[MAXB], xd1[MAXB], xd2[MAXB];  // packet position (FP64)
    double l_emit[MAXB], l_abs[MAXB], l_esc[MAXB], l_res[MAXB];
    unsigned long long q[MAXB], q_end[MAXB];
    unsigned long long c_dep[MAXB], c_loc[MAXB], c_peel[MAXB], c_scat[MAXB];
    float alb[MAXB];
    int lam[MAXB], led_lam[MAXB], nscat[MAXB], peel_i[MAXB], after_peel[MAXB], peel_kind[MAXB];
    unsigned pk[MAXB], ev[MAXB], started[MAXB];
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__global__ void __launch_bounds__(MAXB, 3) trace_mixed_kernel(const TraceArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    InstrDev* sins = reinterpret_cast<InstrDev*>(smem);
    Cold& C = *reinterpret_cast<Cold*>(smem + align16(sizeof(InstrDev) * A.ninstr));
    double* wbuf_all = reinterpret_cast<double*>(smem + align16(sizeof(InstrDev) * A.ninstr) + sizeof(Cold));
    for (int i = threadIdx.x; i < A.ninstr; i += blockDim.x) sins[i] = A.ins[i];
    const int t = threadIdx.x;
    double* wbuf = wbuf_all + (t & ~31);
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
    const double Dlo0 = A.lo[0], Dlo1 = A.lo[1], Dlo2 = A.lo[2], Dd0 = A.d[0], Dd1 = A.d[1], Dd2 = A.d[2];
    const float INF = __int_as_float(0x7f800000);
    const float* __restrict__ kr = A.kr32;
    double* __restrict__ absorbed = A.absorbed;
    const int step_min = A.step_min > 0 ? A.step_min : 16;

    // ---- stepping state (registers)
    int mode = M_NONE;
    int c0 = 0, c1 = 0, c2 = 0, s0 = 0, s1 = 0, s2 = 0;
    float iv0 = 0.f, iv1 = 0.f, iv2 = 0.f, tn0 = 0.f, tn1 = 0.f, tn2 = 0.f, tcur = 0.f;
    double tau_hi = 0.0;
    float tau_lo = 0.f, tau_hi_f = 0.f, rem_f = 0.f;
    int nflush = FLUSH;
    unsigned nsteps = 0;
    float labs_f = 0.f;
    float s_found = 0.f, last_dusty_end = 0.f;
    bool found = false;
    // ---- packet state (registers)
    int stage = ST_NEW;
    bool alive = true;
    int lam = 0;
    float krs = 0.f, gg = 0.f;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, k0 = 0.f, k1 = 0.f, k2 = 0.f;  // x: FP32 copy of the position
    int last_axis = -1;  // axis of the face through which the current cell was entered
    double L = 0.0;
    bool have_pc = false;
    int pc0 = 0, pc1 = 0, pc2 = 0;

    auto begin = [&](int m, float vx, float vy, float vz) {
        mode = m;
        const double X0 = C.xd0[t], X1 = C.xd1[t], X2 = C.xd2[t];
        if (have_pc) {
            c0 = pc0; c1 = pc1; c2 = pc2;
        } else {
            c0 = cell_index<double>(X0, Dlo0, Dd0, nx);
            c1 = cell_index<double>(X1, Dlo1, Dd1, ny);
            c2 = cell_index<double>(X2, Dlo2, Dd2, nz);
        }
        x0 = (float)X0; x1 = (float)X1; x2 = (float)X2;
        s0 = vx > 0.f ? 1 : (vx < 0.f ? -1 : 0);
        s1 = vy > 0.f ? 1 : (vy < 0.f ? -1 : 0);
        s2 = vz > 0.f ? 1 : (vz < 0.f ? -1 : 0);
        iv0 = s0 ? 1.f / vx : 0.f;
        iv1 = s1 ? 1.f / vy : 0.f;
        iv2 = s2 ? 1.f / vz : 0.f;
        // first faces in FP64: a start point close to a face keeps its short first segment
        tn0 = s0 ? (float)((Dlo0 + (double)(c0 + (s0 > 0)) * Dd0 - X0) * (double)iv0) : INF;
        tn1 = s1 ? (float)((Dlo1 + (double)(c1 + (s1 > 0)) * Dd1 - X1) * (double)iv1) : INF;
        tn2 = s2 ? (float)((Dlo2 + (double)(c2 + (s2 > 0)) * Dd2 - X2) * (double)iv2) : INF;
        tcur = 0.f;
        tau_hi = 0.0;
        tau_lo = tau_hi_f = 0.f;
        nflush = FLUSH;
        nsteps = 0;
        last_axis = -1;
    };

    // one cell crossing of the current traversal
    auto step = [&]() {
        const float tmin = fminf(fminf(tn0, tn1), tn2);
        const int axis = (tn0 == tmin) ? 0 : ((tn1 == tmin) ? 1 : 2);
        const float ds = fmaxf(tmin - tcur, 0.f);
        const int m = (c2 * ny + c1) * nx + c0;
        const float krl = __ldg(kr + m) * krs;
        const float dtau = krl * ds;
        ++nsteps;
        bool done = false;
        if (mode == M_LOCATE) {
            if (krl > 0.f) {
                if (tau_lo + dtau >= rem_f) {
                    s_found = (rem_f - tau_lo) / krl;  // distance inside the current cell
                    found = true;
                    done = true;
                } else {
                    last_dusty_end = tmin;
                }
            }
        } else if (mode == M_DEPOSIT && dtau > 0.f) {
            const float dep = labs_f * expf(-(tau_hi_f + tau_lo)) * (-expm1f(-dtau));
            if (dep > 0.f) atomicAdd(absorbed + (size_t)m * NL + lam, (double)dep);
        }
        tau_lo += dtau;
        if (!done) {
            tcur = tmin;
            const int cs = axis == 0 ? c0 : (axis == 1 ? c1 : c2);
            const int ss = axis == 0 ? s0 : (axis == 1 ? s1 : s2);
            const int na = axis == 0 ? nx : (axis == 1 ? ny : nz);
            const int cn = cs + ss;
            if ((unsigned)cn >= (unsigned)na) {
                done = true;
            } else {
                const float loa = axis == 0 ? lo0 : (axis == 1 ? lo1 : lo2);
                const float da = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
                const float xa = axis == 0 ? x0 : (axis == 1 ? x1 : x2);
                const float iva = axis == 0 ? iv0 : (axis == 1 ? iv1 : iv2);
                const float tnew = (loa + (float)(cn + (ss > 0)) * da - xa) * iva;
                if (axis == 0) { c0 = cn; tn0 = tnew; }
                else if (axis == 1) { c1 = cn; tn1 = tnew; }
                else { c2 = cn; tn2 = tnew; }
                last_axis = axis;
            }
        }
        if (--nflush == 0 || done) {
            tau_hi += (double)tau_lo;
            tau_lo = 0.f;
            tau_hi_f = (float)tau_hi;
            nflush = FLUSH;
            if (mode == M_LOCATE && !done) rem_f = (float)(C.tau_t[t] - tau_hi);
        }
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
        double w;
        if (C.peel_kind[t] == 0) {
            w = L;  // isotropic emission: phase factor 1
        } else {
            const float mu = k0 * I.kobs_f[0] + k1 * I.kobs_f[1] + k2 * I.kobs_f[2];
            w = L * (double)hg_phase<float>(gg, mu);
        }
        C.peel_w[t] = w;
        if (w > 0.0) begin(M_PEEL, I.kobs_f[0], I.kobs_f[1], I.kobs_f[2]);
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
                    C.alb[t] = (float)__ldg(A.albedo + ll);
                    C.L0[t] = __ldg(A.L0 + ll);
                    if (C.led_lam[t] != ll) {
                        flush_ledger();
                        C.led_lam[t] = ll;
                    }
                }
                lam = ll;
                krs = (float)__ldg(A.kscale + lam);
                gg = (float)__ldg(A.g + lam);
                C.pk[t] = (unsigned)(qq - __ldg(A.offsets + lam));
                L = C.L0[t];
                C.p_esc[t] = C.p_abs[t] = C.p_res[t] = C.p_peel[t] = 0.0;
                C.ev[t] = 0;
                C.nscat[t] = 0;
                C.l_emit[t] += L;
                have_pc = false;

                // ---- launch (Sect. 3.2)
                bool isotropic = true;
                if (A.src_kind == SKIRT_SRC_BEAM) {
                    x0 = (float)A.src_pos[0]; x1 = (float)A.src_pos[1]; x2 = (float)A.src_pos[2];
                    k0 = (float)A.src_dir[0]; k1 = (float)A.src_dir[1]; k2 = (float)A.src_dir[2];
                    isotropic = false;
                } else if (A.src_kind == SKIRT_SRC_DISK) {
                    const float hR = (float)A.h_R, hz = (float)A.h_z;
                    for (uint32_t tries = 0;; ++tries) {
                        const uint4 r = draw(0u, tries == 0 ? 0u : tries + 1u);
                        const float u0 = u01f(r.x), u1 = u01f(r.y), u2 = u01f(r.z), u3 = u01f(r.w);
                        const float Rr = -hR * (logf(u0) + logf(u1));
                        const float z = (u2 < 0.5f) ? hz * logf(2.f * u2) : -hz * logf(2.f * (1.f - u2));
                        float sp, cp;
                        sincospif(2.f * u3, &sp, &cp);
                        x0 = (float)A.src_pos[0] + Rr * cp;
                        x1 = (float)A.src_pos[1] + Rr * sp;
                        x2 = (float)A.src_pos[2] + z;
                        if (x0 >= lo0 && x0 <= (float)A.hi[0] && x1 >= lo1 && x1 <= (float)A.hi[1] && x2 >= lo2 &&
                            x2 <= (float)A.hi[2])
                            break;
                        if (tries + 1 >= 64) {
                            atomicOr(A.err, (unsigned)ERRBIT_SOURCE);
                            x0 = (float)A.src_pos[0]; x1 = (float)A.src_pos[1]; x2 = (float)A.src_pos[2];
                            break;
                        }
                    }
                } else if (A.src_kind == SKIRT_SRC_DUST) {
                    const uint4 r = draw(0u, 0u);
                    const long long ncell = (long long)nx * ny * nz;
                    const double* cdf = A.cdf + (size_t)lam * ncell;
                    const double u0 = (double)u01f(r.x);
                    long long a = 0, b = ncell - 1;  // first cell with cdf > u0
                    while (a < b) {
                        const long long mid = (a + b) >> 1;
                        if (__ldg(cdf + mid) > u0) b = mid; else a = mid + 1;
                    }
                    pc0 = (int)(a % nx);
                    pc1 = (int)((a / nx) % ny);
                    pc2 = (int)(a / ((long long)nx * ny));
                    x0 = lo0 + ((float)pc0 + u01f(r.y)) * d0;
                    x1 = lo1 + ((float)pc1 + u01f(r.z)) * d1;
                    x2 = lo2 + ((float)pc2 + u01f(r.w)) * d2;
                    have_pc = true;
                } else {
                    x0 = (float)A.src_pos[0]; x1 = (float)A.src_pos[1]; x2 = (float)A.src_pos[2];
                }
                if (A.src_kind == SKIRT_SRC_POINT || A.src_kind == SKIRT_SRC_BEAM) {
                    C.xd0[t] = A.src_pos[0]; C.xd1[t] = A.src_pos[1]; C.xd2[t] = A.src_pos[2];
                } else if (A.src_kind == SKIRT_SRC_DUST) {
                    const uint4 r = draw(0u, 0u);
                    C.xd0[t] = Dlo0 + ((double)pc0 + (double)u01f(r.y)) * Dd0;
                    C.xd1[t] = Dlo1 + ((double)pc1 + (double)u01f(r.z)) * Dd1;
                    C.xd2[t] = Dlo2 + ((double)pc2 + (double)u01f(r.w)) * Dd2;
                } else {
                    C.xd0[t] = x0; C.xd1[t] = x1; C.xd2[t] = x2;
                }
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
                labs_f = (float)(L * (1.0 - (double)C.alb[t]));
                begin(M_DEPOSIT, k0, k1, k2);
                stage = ST_DEPOSIT_DONE;
                continue;
            }

            if (stage == ST_DEPOSIT_DONE) {
                C.c_dep[t] += nsteps;
                const double tau_path = tau_hi;
                // om = 1 - e^{-tau_path}: from expm1 for small tau, from 1 - exp for large
                // tau, so that both om and 1 - om keep FP32 relative precision
                const float tf = (float)tau_path;
                const double om = tf < 0.6931472f ? (double)(-expm1f(-tf)) : 1.0 - (double)expf(-tf);
                const float om_f = (float)om;
                C.p_esc[t] += L * (1.0 - om);
                C.p_abs[t] += L * (1.0 - (double)C.alb[t]) * om;
                if (!(tau_path > 0.0)) {
                    if (!(tau_path == 0.0)) atomicOr(A.err, (unsigned)ERRBIT_NONFINITE);
                    L = 0.0;
                    C.nscat[t] = (int)C.ev[t] - 1;
                    stage = ST_END_PACKET;
                    continue;
                }
                C.om[t] = om;
                // forced scattering: tau_int from the exponential truncated at tau_path
                const uint4 r = draw(C.ev[t], 0u);
                const float tau_int = -log1pf(-u01f(r.x) * om_f);
                C.tau_t[t] = (double)tau_int;
                begin(M_LOCATE, k0, k1, k2);
                rem_f = tau_int;
                found = false;
                last_dusty_end = 0.f;
                stage = ST_LOCATE_DONE;
                continue;
            }

            if (stage == ST_LOCATE_DONE) {
                C.c_loc[t] += nsteps;
                double X0 = C.xd0[t], X1 = C.xd1[t], X2 = C.xd2[t];
                const double K0 = k0, K1 = k1, K2 = k2;
                if (found && last_axis >= 0) {
                    // entry point of the interaction cell, snapped onto the exact face plane
                    const double te = (double)tcur;
                    X0 += te * K0; X1 += te * K1; X2 += te * K2;
                    if (last_axis == 0) X0 = Dlo0 + (double)(c0 + (s0 < 0)) * Dd0;
                    else if (last_axis == 1) X1 = Dlo1 + (double)(c1 + (s1 < 0)) * Dd1;
                    else X2 = Dlo2 + (double)(c2 + (s2 < 0)) * Dd2;
                    const double si = (double)s_found;
                    X0 += si * K0; X1 += si * K1; X2 += si * K2;
                } else {
                    const double s = found ? (double)s_found : (double)last_dusty_end;
                    X0 += s * K0; X1 += s * K1; X2 += s * K2;
                }
                C.xd0[t] = X0; C.xd1[t] = X1; C.xd2[t] = X2;
                x0 = (float)X0; x1 = (float)X1; x2 = (float)X2;
                have_pc = found;
                if (found) { pc0 = c0; pc1 = c1; pc2 = c2; }
                L = L * (double)C.alb[t] * C.om[t];
                C.nscat[t] = (int)C.ev[t];
                if (L > 0.0 && A.peel && A.ninstr > 0) {
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
                const double w = C.peel_w[t];
                if (w > 0.0) {
                    const double flux = w * (double)expf(-(float)tau_hi) * I.flux_norm;
                    C.p_peel[t] += flux;
                    const double X0 = C.xd0[t], X1 = C.xd1[t], X2 = C.xd2[t];
                    const double a = X0 * I.e1[0] + X1 * I.e1[1] + X2 * I.e1[2];
                    const double b = X0 * I.e2[0] + X1 * I.e2[1] + X2 * I.e2[2];
                    const double fa = floor((a + I.half_fov) * I.inv_dpx);
                    const double fb = floor((b + I.half_fov) * I.inv_dpx);
                    if (fa >= 0.0 && fa < (double)I.npx && fb >= 0.0 && fb < (double)I.npx) {
                        const long long pix = (long long)fb * I.npx + (long long)fa;
                        red_agg(A.images + I.img_off + pix * NL + lam, flux, wbuf);
                    } else {
                        red_agg(A.oof + (size_t)pi * NL + lam, flux, wbuf);
                    }
                }
                C.peel_i[t] = pi + 1;
                if (pi + 1 < A.ninstr) start_peel(pi + 1);
                else stage = C.after_peel[t];
                continue;
            }

            if (stage == ST_AFTER_SCATTER) {
                if (L <= A.w_min * C.L0[t]) {
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
            const double pe = C.p_esc[t], pa = C.p_abs[t], pr = C.p_res[t], pp = C.p_peel[t];
            C.l_abs[t] += pa;
            C.l_esc[t] += pe;
            C.l_res[t] += pr;
            if (!isfinite(pe + pa + pr + pp)) atomicOr(A.err, (unsigned)ERRBIT_NONFINITE);
            const unsigned pk = C.pk[t];
            if (pk < (unsigned)A.nrec) {
                double* rec = A.records + ((size_t)lam * A.nrec + pk) * SKIRT_REC_FIELDS;
                rec[0] = (double)C.nscat[t];
                rec[1] = pe;
                rec[2] = pa;
                rec[3] = pr;
                rec[4] = pp;
                rec[5] = C.xd0[t];
                rec[6] = C.xd1[t];
                rec[7] = C.xd2[t];
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
            for (int r = 0; r < ROUND; ++r)
                if (mode != M_NONE) step();
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
    return align16(sizeof(InstrDev) * ninstr) + sizeof(Cold) + sizeof(double) * MAXB;
}

static cudaError_t set_smem_limit()
{
    return cudaFuncSetAttribute(trace_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)trace_mixed_smem_bytes(16, MAXB));
}

cudaError_t launch_trace_mixed(const TraceArgs& a, int block, int grid, cudaStream_t s)
{
    if (block > MAXB || block % 32) return cudaErrorInvalidValue;
    cudaError_t e = set_smem_limit();
    if (e != cudaSuccess) return e;
    trace_mixed_kernel<<<grid, block, trace_mixed_smem_bytes(a.ninstr, block), s>>>(a);
    return cudaGetLastError();
}

cudaError_t trace_mixed_occupancy(int block, int* blocks_per_sm)
{
    if (block > MAXB || block % 32) {
        *blocks_per_sm = 0;
        return cudaSuccess;
    }
    cudaError_t e = set_smem_limit();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_mixed_kernel, block,
                                                         trace_mixed_smem_bytes(16, block));
}

}  // namespace skirt
