// Photon-packet life cycle on the GPU, plain FP64 form: one packet per
// thread, written as a per-thread state machine so that every iteration of
// the main loop does one cell crossing for every lane that is inside a
// traversal, whatever kind of traversal it is (absorption deposit,
// forced-interaction search, or peel-off line of sight).  Lanes that just
// finished a traversal handle their event (launch, scattering, peel-off
// tally) and rejoin the stepping loop.  Every quantity is FP64.  The mixed
// form lives in trace_mixed.cu.
//
// Method (arXiv:1705.04702): Sect. 3.2 (stellar emission phase: packets per
// wavelength, Monte Carlo launch / interaction sampling, peel-off to every
// instrument on each scattering, continuous absorption into the absorbed
// table, life until a negligible luminosity is left); Sect. 1 (peel-off,
// continuous absorption, forced scattering); Sect. 5.2 (absorbed table
// element (cell, wavelength) at cell * N_lambda + wavelength, updated with
// lock-free atomic additions -- here native FP64 reductions in L2); Sect. 7.9
// (octree dust grid: a cell crossing steps from a leaf to the leaf across its
// exit face, through the precomputed face neighbour and a descent by the
// lattice cell of the entry point).
#include <cuda_runtime.h>
#include <math.h>

#include "skirt_internal.cuh"
#include "trace_device.cuh"

namespace skirt {
namespace {

// Arithmetic policy of the plain form (R = double throughout).
template <typename R> struct P;

template <> struct P<double> {
    static __device__ __forceinline__ double kr(const TraceArgs& a, int m) { return __ldg(a.kr64 + m); }
    static __device__ __forceinline__ double logr(double x) { return log(x); }
    static __device__ __forceinline__ double sqrtr(double x) { return sqrt(x); }
    static __device__ __forceinline__ double floorr(double x) { return floor(x); }
    static __device__ __forceinline__ void sincospi2(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
    static __device__ __forceinline__ double u(uint32_t x) { return (double)u01f(x); }
    // e^{-tau_prev} (1 - e^{-dtau}) for the deposit
    static __device__ __forceinline__ double dep_factor(double tau_prev, double dtau) {
        return exp(-tau_prev) * (-expm1(-dtau));
    }
    static __device__ __forceinline__ double kobs(const InstrDev& I, int a) { return I.kobs[a]; }
    static __device__ __forceinline__ double e1(const InstrDev& I, int a) { return I.e1[a]; }
    static __device__ __forceinline__ double e2(const InstrDev& I, int a) { return I.e2[a]; }
    static __device__ __forceinline__ double half_fov(const InstrDev& I) { return I.half_fov; }
    static __device__ __forceinline__ double inv_dpx(const InstrDev& I) { return I.inv_dpx; }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

// Distance along the ray from o (inverse direction component iv) to the
// face plane lo + k d.  One fused multiply-add for the plane, so that every
// grid kind evaluates the same plane to the same value.
template <typename R>
__device__ __forceinline__ R face_dist(R lo, int k, R d, R o, R iv)
{
    return (fma((R)k, d, lo) - o) * iv;
}

template <typename R, bool OCT>
__global__ void __launch_bounds__(512) trace_kernel(const TraceArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InstrDev* sins = reinterpret_cast<InstrDev*>(smem_raw);
    for (int i = threadIdx.x; i < A.ninstr; i += blockDim.x) sins[i] = A.ins[i];
    __syncthreads();

    const int NL = A.nlambda;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const R lo0 = (R)A.lo[0], lo1 = (R)A.lo[1], lo2 = (R)A.lo[2];
    const R d0 = (R)A.d[0], d1 = (R)A.d[1], d2 = (R)A.d[2];
    const R INF = P<R>::inf();

    // ---- traversal state
    int mode = M_NONE;
    int c0 = 0, c1 = 0, c2 = 0;
    int s0 = 0, s1 = 0, s2 = 0;
    R o0 = 0, o1 = 0, o2 = 0;   // traversal origin
    R v0 = 0, v1 = 0, v2 = 0;   // traversal direction
    R iv0 = 0, iv1 = 0, iv2 = 0; // its inverse
    R tn0 = 0, tn1 = 0, tn2 = 0; // distance to the next face on each axis
    R tcur = 0;
    double tau = 0.0;           // optical depth accumulated along this traversal
    double tau_t = 0.0;         // interaction optical depth (locate)
    double labs = 0.0;          // L (1 - albedo) (deposit)
    R s_found = 0, last_dusty_end = 0;
    bool found = false;
    // octree: current leaf (node, level, leaf index, kr); c0..c2 hold its
    // lattice corner
    const int OL = A.oct_levels;
    int onode = 0, olev = 0, oleaf = 0, osteps = 0;
    float okr = 0.f;

    // ---- packet state
    int stage = ST_NEW;
    int lam = -1;
    unsigned long long q = 0, q_end = 0;
    bool started = false;
    uint32_t pk = 0;
    double L = 0.0, L0 = 0.0, tau_path = 0.0;
    R x0 = 0, x1 = 0, x2 = 0;   // position
    R k0 = 0, k1 = 0, k2 = 0;   // direction
    uint32_t ev = 0;
    int nscat = 0;
    R krs = 0, gg = 0;
    double alb = 0.0;
    int peel_i = 0, peel_kind = 0, after_peel = 0;
    double peel_w = 0.0;
    double p_esc = 0.0, p_abs = 0.0, p_res = 0.0, p_peel = 0.0;

    // ---- thread-level ledger for the current wavelength, and work counters
    int led_lam = -1;
    double l_emit = 0.0, l_abs = 0.0, l_esc = 0.0, l_res = 0.0;
    unsigned long long c_scat = 0, c_dep = 0, c_loc = 0, c_peel = 0;

    // octree: the leaf holding lattice cell (j0, j1, j2), found by descending
    // from `node` (a node of level `lev`, or a leaf)
    auto oct_enter = [&](int node, int lev, int j0, int j1, int j2) {
        int r = __ldg(&A.oct_nodes[node].ref);
        while (r >= 0 && lev < OL) {
            ++lev;
            const int b = OL - lev;
            node = r + (((j0 >> b) & 1) | (((j1 >> b) & 1) << 1) | (((j2 >> b) & 1) << 2));
            r = __ldg(&A.oct_nodes[node].ref);
        }
        onode = node;
        olev = oct_leaf_level(r);
        oleaf = oct_leaf_index(r);
        okr = __ldg(&A.oct_nodes[node].kr);
        const int mask = ~((1 << (OL - olev)) - 1);
        c0 = j0 & mask;
        c1 = j1 & mask;
        c2 = j2 & mask;
    };

    auto begin = [&](int m, R ox, R oy, R oz, R vx, R vy, R vz) {
        mode = m;
        o0 = ox; o1 = oy; o2 = oz;
        v0 = vx; v1 = vy; v2 = vz;
        c0 = cell_index<R>(ox, lo0, d0, nx);
        c1 = cell_index<R>(oy, lo1, d1, ny);
        c2 = cell_index<R>(oz, lo2, d2, nz);
        if (OCT) {
            oct_enter(0, 0, c0, c1, c2);
            osteps = 0;
        }
        s0 = vx > (R)0 ? 1 : (vx < (R)0 ? -1 : 0);
        s1 = vy > (R)0 ? 1 : (vy < (R)0 ? -1 : 0);
        s2 = vz > (R)0 ? 1 : (vz < (R)0 ? -1 : 0);
        iv0 = s0 ? (R)1 / vx : (R)0;
        iv1 = s1 ? (R)1 / vy : (R)0;
        iv2 = s2 ? (R)1 / vz : (R)0;
        if (!OCT) {
            tn0 = s0 ? face_dist<R>(lo0, c0 + (s0 > 0), d0, ox, iv0) : INF;
            tn1 = s1 ? face_dist<R>(lo1, c1 + (s1 > 0), d1, oy, iv1) : INF;
            tn2 = s2 ? face_dist<R>(lo2, c2 + (s2 > 0), d2, oz, iv2) : INF;
        }
        tcur = (R)0;
        tau = 0.0;
    };

    auto flush_ledger = [&]() {
        if (led_lam >= 0) {
            double* lg = A.ledger + 4 * (size_t)led_lam;
            atomicAdd(lg + 0, l_emit);
            atomicAdd(lg + 1, l_abs);
            atomicAdd(lg + 2, l_esc);
            atomicAdd(lg + 3, l_res);
        }
        l_emit = l_abs = l_esc = l_res = 0.0;
    };

    auto draw = [&](uint32_t event, uint32_t block) -> uint4 {
        return philox10(make_uint4(pk, (uint32_t)lam, event, (A.phase << 24) | block), A.key0, A.key1);
    };

    for (;;) {
        if (mode != M_NONE) {
            // ---------------- one cell crossing ----------------
            int osz = 1;
            if (OCT) {
                // exit distances from the current leaf's box
                osz = 1 << (OL - olev);
                tn0 = s0 ? face_dist<R>(lo0, c0 + (s0 > 0 ? osz : 0), d0, o0, iv0) : INF;
                tn1 = s1 ? face_dist<R>(lo1, c1 + (s1 > 0 ? osz : 0), d1, o1, iv1) : INF;
                tn2 = s2 ? face_dist<R>(lo2, c2 + (s2 > 0 ? osz : 0), d2, o2, iv2) : INF;
            }
            const int axis = (tn0 <= tn1) ? ((tn0 <= tn2) ? 0 : 2) : ((tn1 <= tn2) ? 1 : 2);
            const R tnext = axis == 0 ? tn0 : (axis == 1 ? tn1 : tn2);
            R ds = tnext - tcur;
            if (ds < (R)0) ds = (R)0;
            const int m = OCT ? oleaf : (c2 * ny + c1) * nx + c0;
            const R krl = (OCT ? (R)okr : P<R>::kr(A, m)) * krs;
            const R dtau_r = krl * ds;
            const double dtau = (double)dtau_r;
            bool done = false;
            if (mode == M_DEPOSIT) {
                ++c_dep;
                if (dtau_r > (R)0) {
                    const double dep = labs * P<R>::dep_factor(tau, dtau_r);
                    if (dep > 0.0) {
                        atomicAdd(A.absorbed + ((size_t)m * A.abs_cs + (size_t)lam * A.abs_ls), dep);
                        p_abs += dep;
                    }
                }
                tau += dtau;
            } else if (mode == M_LOCATE) {
                ++c_loc;
                if (krl > (R)0 && tau + dtau >= tau_t) {
                    s_found = tcur + (R)(tau_t - tau) / krl;
                    found = true;
                    done = true;
                } else {
                    tau += dtau;
                    if (krl > (R)0) last_dusty_end = tnext;
                }
            } else {
                ++c_peel;
                tau += dtau;
            }
            if (!done && OCT) {
                tcur = tnext;
                const int sa = axis == 0 ? s0 : (axis == 1 ? s1 : s2);
                const int nb = __ldg(&A.oct_nodes[onode].nb[2 * axis + (sa > 0)]);
                if (nb < 0) {
                    done = true;  // the exit face lies on the root box
                } else if (++osteps > A.oct_step_cap) {
                    atomicOr(A.err, (unsigned)ERRBIT_PATH);
                    done = true;
                } else {
                    // lattice cell of the entry point into the next leaf: across
                    // the exit face along `axis`; along the other axes the
                    // cell of the crossing point, kept within the current
                    // leaf's cross-section
                    int j[3];
                    const int cc[3] = {c0, c1, c2};
                    const R oo[3] = {o0, o1, o2}, vv[3] = {v0, v1, v2}, ll[3] = {lo0, lo1, lo2},
                            dd[3] = {d0, d1, d2};
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        if (b == axis) {
                            j[b] = sa > 0 ? cc[b] + osz : cc[b] - 1;
                        } else {
                            const R f = P<R>::floorr((oo[b] + tnext * vv[b] - ll[b]) / dd[b]);
                            const int jb = f < (R)cc[b] ? cc[b] : (f > (R)(cc[b] + osz - 1) ? cc[b] + osz - 1 : (int)f);
                            j[b] = jb;
                        }
                    }
                    // a neighbour that is not a leaf has the current level
                    oct_enter(nb, olev, j[0], j[1], j[2]);
                }
            } else if (!done) {
                tcur = tnext;
                if (axis == 0) {
                    c0 += s0;
                    if ((unsigned)c0 >= (unsigned)nx) done = true;
                    else tn0 = face_dist<R>(lo0, c0 + (s0 > 0), d0, o0, iv0);
                } else if (axis == 1) {
                    c1 += s1;
                    if ((unsigned)c1 >= (unsigned)ny) done = true;
                    else tn1 = face_dist<R>(lo1, c1 + (s1 > 0), d1, o1, iv1);
                } else {
                    c2 += s2;
                    if ((unsigned)c2 >= (unsigned)nz) done = true;
                    else tn2 = face_dist<R>(lo2, c2 + (s2 > 0), d2, o2, iv2);
                }
            }
            if (done) mode = M_NONE;
            continue;
        }

        // ---------------- event handling ----------------
        if (stage == ST_NEW) {
            if (q >= q_end) {
                if (!A.persistent) {
                    if (started) break;
                    started = true;
                    q = A.q_base + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
                    q_end = (q < A.q_base + A.q_count) ? q + 1 : q;
                    if (q >= q_end) break;
                } else {
                    // warp-aggregated refill from the global work queue
                    const unsigned mask = __activemask();
                    const int lane = threadIdx.x & 31;
                    const int leader = __ffs(mask) - 1;
                    const unsigned rank = __popc(mask & ((1u << lane) - 1u));
                    unsigned long long base = 0;
                    if (lane == leader)
                        base = atomicAdd(A.queue, (unsigned long long)__popc(mask) * (unsigned long long)A.chunk);
                    base = __shfl_sync(mask, base, leader);
                    q = base + (unsigned long long)rank * A.chunk;
                    if (q >= A.total) break;
                    q_end = q + A.chunk;
                    if (q_end > A.total) q_end = A.total;
                }
            }
            const unsigned long long qq = q++;
            if (lam < 0 || qq < __ldg(A.offsets + lam) || qq >= __ldg(A.offsets + lam + 1)) {
                int a = 0, b = NL - 1;  // last wavelength whose offset <= qq
                while (a < b) {
                    const int mid = (a + b + 1) >> 1;
                    if (__ldg(A.offsets + mid) <= qq) a = mid; else b = mid - 1;
                }
                lam = a;
                krs = (R)__ldg(A.kscale + lam);
                alb = __ldg(A.albedo + lam);
                gg = (R)__ldg(A.g + lam);
                L0 = __ldg(A.L0 + lam);
                if (led_lam != lam) {
                    flush_ledger();
                    led_lam = lam;
                }
            }
            pk = (uint32_t)(qq - __ldg(A.offsets + lam) + __ldg(A.pk_first + lam));
            L = L0;
            p_esc = p_abs = p_res = p_peel = 0.0;
            ev = 0;
            nscat = 0;
            l_emit += L0;

            // ---- launch (Sect. 3.2): position from the source, isotropic direction
            bool isotropic = true;
            if (A.src_kind == SKIRT_SRC_BEAM) {
                x0 = (R)A.src_pos[0]; x1 = (R)A.src_pos[1]; x2 = (R)A.src_pos[2];
                k0 = (R)A.src_dir[0]; k1 = (R)A.src_dir[1]; k2 = (R)A.src_dir[2];
                isotropic = false;
            } else if (A.src_kind == SKIRT_SRC_DISK) {
                const R hR = (R)A.h_R, hz = (R)A.h_z;
                for (uint32_t tries = 0;; ++tries) {
                    const uint4 r = draw(0u, tries == 0 ? 0u : tries + 1u);
                    const R u0 = P<R>::u(r.x), u1 = P<R>::u(r.y), u2 = P<R>::u(r.z), u3 = P<R>::u(r.w);
                    const R Rr = -hR * (P<R>::logr(u0) + P<R>::logr(u1));
                    const R z = (u2 < (R)0.5) ? hz * P<R>::logr((R)2 * u2) : -hz * P<R>::logr((R)2 * ((R)1 - u2));
                    R sp, cp;
                    P<R>::sincospi2(u3, &sp, &cp);
                    x0 = (R)A.src_pos[0] + Rr * cp;
                    x1 = (R)A.src_pos[1] + Rr * sp;
                    x2 = (R)A.src_pos[2] + z;
                    const bool inside = x0 >= lo0 && x0 <= (R)A.hi[0] && x1 >= lo1 && x1 <= (R)A.hi[1] &&
                                        x2 >= lo2 && x2 <= (R)A.hi[2];
                    if (inside) break;
                    if (tries + 1 >= 64) {
                        atomicOr(A.err, (unsigned)ERRBIT_SOURCE);
                        x0 = (R)A.src_pos[0]; x1 = (R)A.src_pos[1]; x2 = (R)A.src_pos[2];
                        break;
                    }
                }
            } else if (A.src_kind == SKIRT_SRC_DUST) {
                const uint4 r = draw(0u, 0u);
                const long long ncell = A.ncell;
                const double* cdf = A.cdf + (size_t)lam * ncell;
                const double u0 = (double)u01f(r.x);
                long long a = 0, b = ncell - 1;  // first cell with cdf > u0
                while (a < b) {
                    const long long mid = (a + b) >> 1;
                    if (__ldg(cdf + mid) > u0) b = mid; else a = mid + 1;
                }
                if (OCT) {
                    // uniform point in the leaf's box
                    const int4 lf = __ldg(&A.oct_leaf[a]);
                    const R side = (R)(1 << (OL - lf.w));
                    x0 = lo0 + ((R)lf.x + P<R>::u(r.y) * side) * d0;
                    x1 = lo1 + ((R)lf.y + P<R>::u(r.z) * side) * d1;
                    x2 = lo2 + ((R)lf.z + P<R>::u(r.w) * side) * d2;
                } else {
                    const int ix = (int)(a % nx), iy = (int)((a / nx) % ny), iz = (int)(a / ((long long)nx * ny));
                    x0 = lo0 + ((R)ix + P<R>::u(r.y)) * d0;
                    x1 = lo1 + ((R)iy + P<R>::u(r.z)) * d1;
                    x2 = lo2 + ((R)iz + P<R>::u(r.w)) * d2;
                }
            } else {
                x0 = (R)A.src_pos[0]; x1 = (R)A.src_pos[1]; x2 = (R)A.src_pos[2];
            }
            if (isotropic) {
                const uint4 r = draw(0u, 1u);
                const R mu = (R)2 * P<R>::u(r.x) - (R)1;
                const R st = P<R>::sqrtr(fmax((R)1 - mu * mu, (R)0));
                R sp, cp;
                P<R>::sincospi2(P<R>::u(r.y), &sp, &cp);
                k0 = st * cp; k1 = st * sp; k2 = mu;
            }
            if (isotropic && A.peel && A.ninstr > 0) {
                // emission peel-off: isotropic emission, phase factor 1
                peel_kind = 0;
                peel_i = 0;
                peel_w = L;
                after_peel = ST_START_DEP;
                stage = ST_PEEL_DONE;
                if (peel_w > 0.0) {
                    const InstrDev& I = sins[0];
                    begin(M_PEEL, x0, x1, x2, P<R>::kobs(I, 0), P<R>::kobs(I, 1), P<R>::kobs(I, 2));
                } else {
                    tau = 0.0;
                }
            } else {
                stage = ST_START_DEP;
            }
            continue;
        }

        if (stage == ST_START_DEP) {
            ++ev;
            labs = L * (1.0 - alb);
            begin(M_DEPOSIT, x0, x1, x2, k0, k1, k2);
            stage = ST_DEPOSIT_DONE;
            continue;
        }

        if (stage == ST_DEPOSIT_DONE) {
            tau_path = tau;
            p_esc += L * exp(-tau_path);
            if (!(tau_path > 0.0)) {
                if (!(tau_path == 0.0)) atomicOr(A.err, (unsigned)ERRBIT_NONFINITE);
                L = 0.0;
                nscat = (int)ev - 1;
                stage = ST_END_PACKET;
                continue;
            }
            // forced scattering: tau_int from the exponential truncated at tau_path
            const uint4 r = draw(ev, 0u);
            const double u0 = (double)u01f(r.x);
            tau_t = -log1p(-u0 * (-expm1(-tau_path)));
            begin(M_LOCATE, x0, x1, x2, k0, k1, k2);
            last_dusty_end = (R)0;
            found = false;
            stage = ST_LOCATE_DONE;
            continue;
        }

        if (stage == ST_LOCATE_DONE) {
            const R s = found ? s_found : last_dusty_end;
            x0 += s * k0;
            x1 += s * k1;
            x2 += s * k2;
            L = L * alb * (-expm1(-tau_path));
            nscat = (int)ev;
            if (L > 0.0 && A.peel && A.ninstr > 0) {
                peel_kind = 1;
                peel_i = 0;
                const InstrDev& I = sins[0];
                const R mu = k0 * P<R>::kobs(I, 0) + k1 * P<R>::kobs(I, 1) + k2 * P<R>::kobs(I, 2);
                peel_w = L * (double)hg_phase<R>(gg, mu);
                after_peel = ST_AFTER_SCATTER;
                stage = ST_PEEL_DONE;
                begin(M_PEEL, x0, x1, x2, P<R>::kobs(I, 0), P<R>::kobs(I, 1), P<R>::kobs(I, 2));
            } else {
                stage = ST_AFTER_SCATTER;
            }
            continue;
        }

        if (stage == ST_PEEL_DONE) {
            const InstrDev& I = sins[peel_i];
            if (peel_w > 0.0) {
                const double flux = peel_w * exp(-tau) * I.flux_norm;
                p_peel += flux;
                const R a = x0 * P<R>::e1(I, 0) + x1 * P<R>::e1(I, 1) + x2 * P<R>::e1(I, 2);
                const R b = x0 * P<R>::e2(I, 0) + x1 * P<R>::e2(I, 1) + x2 * P<R>::e2(I, 2);
                const R fa = P<R>::floorr((a + P<R>::half_fov(I)) * P<R>::inv_dpx(I));
                const R fb = P<R>::floorr((b + P<R>::half_fov(I)) * P<R>::inv_dpx(I));
                if (fa >= (R)0 && fa < (R)I.npx && fb >= (R)0 && fb < (R)I.npx) {
                    const long long pix = (long long)fb * I.npx + (long long)fa;
                    atomicAdd(A.images + I.img_off + pix * NL + lam, flux);
                } else {
                    atomicAdd(A.oof + (size_t)peel_i * NL + lam, flux);
                }
            }
            ++peel_i;
            if (peel_i < A.ninstr) {
                const InstrDev& J = sins[peel_i];
                if (peel_kind == 0) {
                    peel_w = L;
                } else {
                    const R mu = k0 * P<R>::kobs(J, 0) + k1 * P<R>::kobs(J, 1) + k2 * P<R>::kobs(J, 2);
                    peel_w = L * (double)hg_phase<R>(gg, mu);
                }
                if (peel_w > 0.0) begin(M_PEEL, x0, x1, x2, P<R>::kobs(J, 0), P<R>::kobs(J, 1), P<R>::kobs(J, 2));
            } else {
                stage = after_peel;
            }
            continue;
        }

        if (stage == ST_AFTER_SCATTER) {
            if (L <= A.w_min * L0) {
                p_res += L;
                stage = ST_END_PACKET;
            } else if ((int)ev >= A.max_events) {
                atomicOr(A.err, (unsigned)ERRBIT_EVENT_CAP);
                p_res += L;
                stage = ST_END_PACKET;
            } else {
                // Henyey-Greenstein scattering: mu by inverse CDF, azimuth uniform
                const uint4 r = draw(ev, 0u);
                const R mu = hg_mu<R>(gg, P<R>::u(r.y));
                R sp, cp;
                P<R>::sincospi2(P<R>::u(r.z), &sp, &cp);
                hg_rotate<R>(k0, k1, k2, mu, sp, cp);
                stage = ST_START_DEP;
            }
            continue;
        }

        // ST_END_PACKET
        c_scat += (unsigned long long)nscat;
        l_abs += p_abs;
        l_esc += p_esc;
        l_res += p_res;
        if (!isfinite(p_esc + p_abs + p_res + p_peel)) atomicOr(A.err, (unsigned)ERRBIT_NONFINITE);
        const uint32_t li = pk - (uint32_t)__ldg(A.pk_first + lam);  // index within this call
        if (li < (uint32_t)A.nrec) {
            double* rec = A.records + ((size_t)lam * A.nrec + li) * SKIRT_REC_FIELDS;
            rec[0] = (double)nscat;
            rec[1] = p_esc;
            rec[2] = p_abs;
            rec[3] = p_res;
            rec[4] = p_peel;
            rec[5] = (double)x0;
            rec[6] = (double)x1;
            rec[7] = (double)x2;
        }
        stage = ST_NEW;
    }

    flush_ledger();
    atomicAdd(A.counters + 0, c_scat);
    atomicAdd(A.counters + 1, c_dep);
    atomicAdd(A.counters + 2, c_loc);
    atomicAdd(A.counters + 3, c_peel);
}

// SED = sum over the pixels of every image plus the out-of-frame peel-offs.
// images of instrument q are [npx*npx][nlambda]; thread (lambda lane, row
// group) sums a strided set of pixel rows for one wavelength column.
__global__ void sed_finalize_kernel(const double* __restrict__ img, const double* __restrict__ oof,
                                    double* __restrict__ sed, long long npix, int nlambda, int q, double sign)
{
    __shared__ double part[8][33];
    const int lam = blockIdx.x * 32 + threadIdx.x;
    const int rg = threadIdx.y;
    double s = 0.0;
    if (lam < nlambda)
        for (long long p = (long long)blockIdx.y * 8 + rg; p < npix; p += (long long)gridDim.y * 8)
            s += img[p * nlambda + lam];
    part[rg][threadIdx.x] = s;
    __syncthreads();
    if (rg == 0 && lam < nlambda) {
        double t = 0.0;
        for (int r = 0; r < 8; ++r) t += part[r][threadIdx.x];
        t *= sign;
        if (blockIdx.y == 0 && oof) t += oof[(size_t)q * nlambda + lam];
        atomicAdd(sed + (size_t)q * nlambda + lam, t);
    }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, long long n,
                                  unsigned int* bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = in[i];
        if (!(v >= 0.0f) || !isfinite(v)) atomicOr(bad, 1u);
        out[i] = (double)v;
    }
}

}  // namespace

// The FP64 form keeps only the instruments in shared memory.  Its lanes run
// independent state machines with no point where the warp is known to be
// converged, so its peel-off tallies are plain reductions.
size_t trace_smem_bytes(int ninstr, int block)
{
    (void)block;
    return sizeof(InstrDev) * (size_t)ninstr;
}

cudaError_t launch_trace(const TraceArgs& a, int precision, int block, int grid, cudaStream_t s)
{
    if (precision == SKIRT_PREC_MIXED) return launch_trace_mixed(a, block, grid, s);
    const size_t smem = trace_smem_bytes(a.ninstr, block);
    if (a.oct_levels > 0)
        trace_kernel<double, true><<<grid, block, smem, s>>>(a);
    else
        trace_kernel<double, false><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t trace_occupancy(int precision, int block, int* blocks_per_sm, bool octree)
{
    if (precision == SKIRT_PREC_MIXED) return trace_mixed_occupancy(block, blocks_per_sm, octree);
    const size_t smem = trace_smem_bytes(16, block);
    return octree ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<double, true>, block, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<double, false>, block, smem);
}

namespace {

// out[c][l] (+)= in[l][c], 32 x 32 tiles through shared memory (one padding
// column): coalesced reads along the cells and writes along the wavelengths.
__global__ void transpose_absorbed_kernel(const double* __restrict__ in, double* __restrict__ out, long long ncell,
                                          int nl, int add)
{
    __shared__ double tile[32][33];
    const long long c0 = (long long)blockIdx.x * 32;
    const int l0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long c = c0 + threadIdx.x;
        const int l = l0 + k;
        tile[k][threadIdx.x] = (c < ncell && l < nl) ? in[(size_t)l * ncell + c] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long c = c0 + k;
        const int l = l0 + threadIdx.x;
        if (c < ncell && l < nl) {
            double* o = out + (size_t)c * nl + l;
            *o = add ? *o + tile[threadIdx.x][k] : tile[threadIdx.x][k];
        }
    }
}

}  // namespace

cudaError_t launch_transpose_absorbed(const double* in, double* out, long long ncell, int nlambda, bool add,
                                      cudaStream_t s)
{
    const long long bx = (ncell + 31) / 32;
    if (bx > 0x7fffffffLL) return cudaErrorInvalidValue;
    transpose_absorbed_kernel<<<dim3((unsigned)bx, (unsigned)((nlambda + 31) / 32)), dim3(32, 8), 0, s>>>(
        in, out, ncell, nlambda, add ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_sed_finalize(const double* images, const double* oof, double* sed, int ninstr,
                                const int* npx_host, int nlambda, double sign, cudaStream_t s)
{
    long long off = 0;
    for (int q = 0; q < ninstr; ++q) {
        const long long npix = (long long)npx_host[q] * npx_host[q];
        dim3 block(32, 8);
        long long rows = (npix + 7) / 8;
        int gy = (int)(rows < 256 ? rows : 256);
        if (gy < 1) gy = 1;
        dim3 grid((nlambda + 31) / 32, gy);
        sed_finalize_kernel<<<grid, block, 0, s>>>(images + off, oof, sed, npix, nlambda, q, sign);
        off += npix * nlambda;
    }
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* in, double* out, long long n, unsigned int* bad, cudaStream_t s)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    if (blocks < 1) blocks = 1;
    f32_to_f64_kernel<<<(int)blocks, 256, 0, s>>>(in, out, n, bad);
    return cudaGetLastError();
}

}  // namespace skirt
