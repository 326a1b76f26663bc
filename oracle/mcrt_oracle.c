/*
 * Plain, slow, single-threaded FP64 oracle of the Monte Carlo photon-packet
 * life cycle (launch, peel-off, continuous absorption, forced scattering,
 * Henyey-Greenstein scattering) -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may call this code.  It shares nothing with the CUDA library: its own
 * Philox, its own ray/grid intersection (all face crossings listed and
 * merged, cells found from segment midpoints) and its own bookkeeping.
 *
 * What the paper fixes and what is a reading:
 *  - Sect. 3.2 (stellar emission phase): for each wavelength a fixed number
 *    of packets is launched; Monte Carlo sampling picks launch position,
 *    interaction positions and directions; on every scattering event a
 *    fraction of the luminosity is peeled off towards each instrument into a
 *    per-pixel, per-wavelength table; between events the packet loses
 *    luminosity continuously by absorption, written to the absorbed
 *    luminosity table [cell, wavelength]; the packet lives until all but a
 *    negligible part of its luminosity is gone.
 *  - Sect. 1 names the techniques (peel-off, continuous absorption, forced
 *    scattering); their equations are the standard ones and are written out
 *    below at the point of use.
 *  - Sect. 5.2 (lock-free additions): absorb(m, ell, DeltaL) adds DeltaL to
 *    element (m, ell) of the absorption table; here a plain += since the
 *    oracle is single-threaded.
 *  - Readings where the paper is silent: Philox4x32-10 keyed by
 *    (seed, packet, wavelength, event); termination at w_min of the launch
 *    luminosity, the last scattering still peeled off, the remainder booked
 *    as "residual"; distant-observer instruments.
 *  - Sect. 7.9 runs on an octree dust grid (up to 13 division levels); its
 *    cells are the leaves of a recursive split of the root box into 8 equal
 *    boxes.  The grid is either regular or such a tree; the tree's paths
 *    come from the planes of its finest lattice (see og_path_tree).
 */
#include "mcrt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OG_PI 3.14159265358979323846

/* ------------------------------------------------------------------------
 * Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 S-box with multipliers
 * 0xD2511F53 / 0xCD9E8D57; the key is bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds.
 * ------------------------------------------------------------------------ */
void og_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): the top 23 bits k of x give (k + 1/2) / 2^23, an odd
 * multiple of 2^-24 and therefore exactly representable in FP32 and FP64. */
double og_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* The four uniforms of draw block `block` of event `event` of packet
 * `packet` at wavelength index `lam`: counter (packet, lam, event,
 * phase<<24 | block), key (seed low word, seed high word). */
static void og_draw(const og_problem* P, int lam, uint64_t packet, uint32_t event,
                    uint32_t block, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)packet, (uint32_t)lam, event, (P->phase << 24) | block};
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    uint32_t r[4];
    og_philox4x32_10(ctr, key, r);
    for (int q = 0; q < 4; ++q) u[q] = og_uniform(r[q]);
}

/* ------------------------------------------------------------------------
 * Grid geometry.
 * ------------------------------------------------------------------------ */
static void og_axes(const og_problem* P, double lo[3], double hi[3], double d[3], int n[3])
{
    n[0] = P->nx; n[1] = P->ny; n[2] = P->nz;
    for (int a = 0; a < 3; ++a) {
        lo[a] = P->bbox[2 * a];
        hi[a] = P->bbox[2 * a + 1];
        d[a] = (hi[a] - lo[a]) / (double)n[a];
    }
}

static int og_index(double x, double lo, double d, int n)
{
    double f = floor((x - lo) / d);
    if (f < 0.0) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int)f;
}

/* ------------------------------------------------------------------------
 * Octree grid (the adaptive grid of the paper's ERIS run, Sect. 7.9): the
 * root box is split into 8 equal boxes, recursively, and the leaves hold the
 * dust.  A leaf of level l at integer position (ix, iy, iz) spans
 * [ix, ix+1) 2^(L-l) cells of the finest lattice (L levels) along x, and so
 * on.  The oracle keeps its own pointer tree: node n has 8 consecutive
 * children from child[n] on (-1: none) or is leaf leaf[n] (-1: not a leaf);
 * child octant = x bit + 2 y bit + 4 z bit.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t* child;
    int64_t* leaf;
    int64_t n, cap;
    int levels;
} og_tree;

static void og_tree_free(og_tree* T)
{
    free(T->child);
    free(T->leaf);
    T->child = NULL;
    T->leaf = NULL;
    T->n = T->cap = 0;
}

static int64_t og_tree_alloc8(og_tree* T)
{
    if (T->n + 8 > T->cap) {
        int64_t cap = T->cap ? 2 * T->cap : 64;
        while (cap < T->n + 8) cap *= 2;
        T->child = (int32_t*)realloc(T->child, sizeof(int32_t) * (size_t)cap);
        T->leaf = (int64_t*)realloc(T->leaf, sizeof(int64_t) * (size_t)cap);
        T->cap = cap;
    }
    int64_t first = T->n;
    for (int q = 0; q < 8; ++q) {
        T->child[first + q] = -1;
        T->leaf[first + q] = -1;
    }
    T->n += 8;
    return first;
}

/* Inserts every leaf from the root down; returns 0, or -1 when a leaf lies
 * outside the lattice, two leaves overlap, or the leaves leave a hole. */
static int og_tree_build(const og_problem* P, og_tree* T)
{
    memset(T, 0, sizeof *T);
    T->levels = P->oct_levels;
    if (P->oct_levels < 1 || P->oct_levels > 20 || P->oct_nleaf < 1) return -1;
    og_tree_alloc8(T); /* node 0 is the root; nodes 1..7 of this block stay unused */
    for (int q = 1; q < 8; ++q) T->leaf[q] = -2;
    for (int64_t m = 0; m < P->oct_nleaf; ++m) {
        const int32_t* lf = P->oct_leaves + 4 * m;
        int l = lf[0];
        if (l < 0 || l > P->oct_levels) return -1;
        for (int a = 1; a < 4; ++a)
            if (lf[a] < 0 || (int64_t)lf[a] >= ((int64_t)1 << l)) return -1;
        int64_t node = 0;
        for (int d = 0; d < l; ++d) {
            if (T->leaf[node] >= 0) return -1;
            if (T->child[node] < 0) {
                int64_t first = og_tree_alloc8(T);
                if (first > 0x7fffffff) return -1;
                T->child[node] = (int32_t)first;
            }
            int bit = l - 1 - d;
            int oct = ((lf[1] >> bit) & 1) | (((lf[2] >> bit) & 1) << 1) | (((lf[3] >> bit) & 1) << 2);
            node = T->child[node] + oct;
        }
        if (T->leaf[node] >= 0 || T->child[node] >= 0) return -1;
        T->leaf[node] = m;
    }
    for (int64_t node = 0; node < T->n; ++node)
        if (T->leaf[node] == -1 && T->child[node] < 0) return -1;
    return 0;
}

/* The leaf holding finest-lattice cell (j0, j1, j2). */
static int64_t og_tree_find(const og_tree* T, int j0, int j1, int j2)
{
    int64_t node = 0;
    for (int d = 0; T->leaf[node] < 0; ++d) {
        int bit = T->levels - 1 - d;
        int oct = ((j0 >> bit) & 1) | (((j1 >> bit) & 1) << 1) | (((j2 >> bit) & 1) << 2);
        node = T->child[node] + oct;
    }
    return T->leaf[node];
}

int og_octree_check(const og_problem* P)
{
    og_tree T;
    int r = og_tree_build(P, &T);
    og_tree_free(&T);
    return r;
}

/* Cells crossed by the ray p + t k (t > 0) up to the grid boundary, with the
 * length inside each.  Every interior face plane the ray crosses before the
 * exit is listed per axis (each list is already sorted in t), the lists are
 * merged, and each non-empty interval between consecutive crossings is
 * attributed to the cell containing its midpoint.  On an octree the planes
 * are those of the finest lattice, every interval lies in one lattice cell
 * and so in one leaf, and consecutive intervals in the same leaf (a box,
 * entered once) form one segment from its first to its last crossing.
 * Returns the number of segments, or -1 if `cap` is too small. */
static int og_path_tree(const og_problem* P, const og_tree* T, const double p[3], const double k[3], int* cells,
                        double* lens, int cap)
{
    double lo[3], hi[3], d[3];
    int n[3];
    og_axes(P, lo, hi, d, n);

    double texit = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (k[a] > 0.0) texit = fmin(texit, (hi[a] - p[a]) / k[a]);
        else if (k[a] < 0.0) texit = fmin(texit, (lo[a] - p[a]) / k[a]);
    }
    if (!(texit > 0.0) || !isfinite(texit)) return 0;

    double* ts[3];
    int cnt[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        ts[a] = (double*)malloc(sizeof(double) * (size_t)(n[a] + 1));
        if (k[a] == 0.0) continue;
        for (int q = 1; q < n[a]; ++q) {
            int qq = (k[a] > 0.0) ? q : n[a] - q; /* ascending t either way */
            double plane = lo[a] + (double)qq * d[a];
            double t = (plane - p[a]) / k[a];
            if (t > 0.0 && t < texit) ts[a][cnt[a]++] = t;
        }
    }

    int head[3] = {0, 0, 0};
    double tprev = 0.0, tseg = 0.0;
    int nseg = 0;
    for (;;) {
        double tnext = texit;
        for (int a = 0; a < 3; ++a)
            if (head[a] < cnt[a] && ts[a][head[a]] < tnext) tnext = ts[a][head[a]];
        for (int a = 0; a < 3; ++a)
            while (head[a] < cnt[a] && ts[a][head[a]] <= tnext) head[a]++;
        if (tnext > tprev) {
            double tm = 0.5 * (tprev + tnext);
            int ix = og_index(p[0] + tm * k[0], lo[0], d[0], n[0]);
            int iy = og_index(p[1] + tm * k[1], lo[1], d[1], n[1]);
            int iz = og_index(p[2] + tm * k[2], lo[2], d[2], n[2]);
            int cell = T ? (int)og_tree_find(T, ix, iy, iz) : (iz * n[1] + iy) * n[0] + ix;
            if (T && nseg > 0 && cells[nseg - 1] == cell) {
                lens[nseg - 1] = tnext - tseg;
            } else {
                if (nseg >= cap) { nseg = -1; break; }
                cells[nseg] = cell;
                lens[nseg] = tnext - tprev;
                tseg = tprev;
                nseg++;
            }
        }
        tprev = tnext;
        if (tnext >= texit) break;
    }
    for (int a = 0; a < 3; ++a) free(ts[a]);
    return nseg;
}

int og_path(const og_problem* P, const double p[3], const double k[3], int* cells, double* lens, int cap)
{
    if (P->oct_levels <= 0) return og_path_tree(P, NULL, p, k, cells, lens, cap);
    og_tree T;
    int r = -1;
    if (og_tree_build(P, &T) == 0) r = og_path_tree(P, &T, p, k, cells, lens, cap);
    og_tree_free(&T);
    return r;
}

/* ------------------------------------------------------------------------
 * Henyey-Greenstein phase function.  Phi(mu) = (1-g^2)/(1+g^2-2 g mu)^{3/2},
 * normalised so that its average over the sphere is 1; mu is sampled by
 * inverting its cumulative distribution.
 * ------------------------------------------------------------------------ */
static double og_hg_phase(double g, double mu)
{
    double den = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (den * sqrt(den));
}

double og_hg_mu(double g, double u)
{
    if (fabs(g) < 1e-6) return 2.0 * u - 1.0;
    double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    double mu = (1.0 + g * g - t * t) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* New direction at polar angle acos(mu) and azimuth phi around k. */
void og_rotate(const double k[3], double mu, double phi, double out[3])
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double cp = cos(phi), sp = sin(phi);
    if (fabs(k[2]) > 0.99999) {
        out[0] = st * cp;
        out[1] = st * sp;
        out[2] = (k[2] > 0.0) ? mu : -mu;
        return;
    }
    double s = sqrt(1.0 - k[2] * k[2]);
    out[0] = st * (k[0] * k[2] * cp - k[1] * sp) / s + k[0] * mu;
    out[1] = st * (k[1] * k[2] * cp + k[0] * sp) / s + k[1] * mu;
    out[2] = -st * cp * s + k[2] * mu;
}

static void og_isotropic(double u0, double u1, double k[3])
{
    double mu = 2.0 * u0 - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double phi = 2.0 * OG_PI * u1;
    k[0] = st * cos(phi);
    k[1] = st * sin(phi);
    k[2] = mu;
}

/* ------------------------------------------------------------------------
 * Per-packet state and bookkeeping.
 * ------------------------------------------------------------------------ */
typedef struct {
    int* cells;
    double* lens;
    int cap;
    const og_tree* tree; /* octree grid, else NULL */
    /* per-packet record */
    double escaped, absorbed, residual, peel;
} og_work;

static double og_tau(const og_problem* P, int lam, const int* cells, const double* lens, int nseg)
{
    double tau = 0.0;
    for (int s = 0; s < nseg; ++s) tau += P->kr[cells[s]] * P->kscale[lam] * lens[s];
    return tau;
}

/* Peel-off (Sect. 1, Sect. 3.2): the fraction of the luminosity that would
 * leave towards each instrument.  weight[q] is the luminosity times the
 * phase-function value for the direction of instrument q; it is attenuated
 * by exp(-tau) along the line of sight to the grid boundary and recorded as
 * flux L/(4 pi d^2) in the pixel hit by the parallel projection of x, and in
 * the instrument's SED (also when the point falls outside the frame). */
static void og_peel(og_problem* P, int lam, const double x[3], const double* weight, og_work* W)
{
    size_t img_off = 0;
    for (int q = 0; q < P->ninstr; ++q) {
        const double* ins = P->instr + 5 * q;
        double dist = ins[0];
        double inc = ins[1] * OG_PI / 180.0, az = ins[2] * OG_PI / 180.0;
        double fov = ins[3];
        int npx = (int)ins[4];
        double kobs[3] = {sin(inc) * cos(az), sin(inc) * sin(az), cos(inc)};
        double e1[3] = {-sin(az), cos(az), 0.0};
        double e2[3] = {kobs[1] * e1[2] - kobs[2] * e1[1],
                        kobs[2] * e1[0] - kobs[0] * e1[2],
                        kobs[0] * e1[1] - kobs[1] * e1[0]};
        if (weight[q] > 0.0) {
            int nseg = og_path_tree(P, W->tree, x, kobs, W->cells, W->lens, W->cap);
            if (nseg < 0) { P->status |= OG_ERR_NONFINITE; nseg = 0; }
            P->counters[3] += (double)nseg;
            double tau = og_tau(P, lam, W->cells, W->lens, nseg);
            double flux = weight[q] * exp(-tau) / (4.0 * OG_PI * dist * dist);
            W->peel += flux;
            P->sed[(size_t)q * P->nlambda + lam] += flux;
            double dpx = fov / (double)npx;
            double a = x[0] * e1[0] + x[1] * e1[1] + x[2] * e1[2];
            double b = x[0] * e2[0] + x[1] * e2[1] + x[2] * e2[2];
            double fa = floor((a + 0.5 * fov) / dpx), fb = floor((b + 0.5 * fov) / dpx);
            if (fa >= 0.0 && fa < (double)npx && fb >= 0.0 && fb < (double)npx) {
                size_t pix = (size_t)fb * (size_t)npx + (size_t)fa;
                P->images[img_off + pix * (size_t)P->nlambda + (size_t)lam] += flux;
            }
        }
        img_off += (size_t)npx * (size_t)npx * (size_t)P->nlambda;
    }
}

static int og_inside(const og_problem* P, const double x[3])
{
    for (int a = 0; a < 3; ++a)
        if (!(x[a] >= P->bbox[2 * a] && x[a] <= P->bbox[2 * a + 1])) return 0;
    return 1;
}

/* Launch (Sect. 3.2): position from the source, direction isotropic except
 * for the collimated test beam.  Draw block 0 (and 2, 3, ... for rejected
 * disk positions) places the packet, block 1 orients it. */
static int og_launch(og_problem* P, int lam, uint64_t i, double x[3], double k[3])
{
    double u[4];
    int isotropic = 1;
    switch (P->src_kind) {
    case OG_SRC_POINT:
        for (int a = 0; a < 3; ++a) x[a] = P->src_pos[a];
        break;
    case OG_SRC_BEAM:
        for (int a = 0; a < 3; ++a) { x[a] = P->src_pos[a]; k[a] = P->src_dir[a]; }
        isotropic = 0;
        break;
    case OG_SRC_DISK: {
        /* surface density ~ exp(-R/h_R): R ~ Gamma(2, h_R) = sum of two
         * exponential deviates; vertical density ~ exp(-|z|/h_z): Laplace
         * deviate by inverse CDF; points outside the grid are redrawn. */
        int tries = 0;
        for (;;) {
            og_draw(P, lam, i, 0u, tries == 0 ? 0u : (uint32_t)(tries + 1), u);
            double R = -P->h_R * (log(u[0]) + log(u[1]));
            double z = (u[2] < 0.5) ? P->h_z * log(2.0 * u[2]) : -P->h_z * log(2.0 * (1.0 - u[2]));
            double phi = 2.0 * OG_PI * u[3];
            x[0] = P->src_pos[0] + R * cos(phi);
            x[1] = P->src_pos[1] + R * sin(phi);
            x[2] = P->src_pos[2] + z;
            if (og_inside(P, x)) break;
            if (++tries >= 64) {
                P->status |= OG_ERR_SOURCE;
                for (int a = 0; a < 3; ++a) x[a] = P->src_pos[a];
                break;
            }
        }
        break;
    }
    case OG_SRC_DUST: {
        /* cell drawn from the per-wavelength cumulative emission, then a
         * uniform point inside it */
        double lo[3], hi[3], d[3];
        int n[3];
        og_axes(P, lo, hi, d, n);
        size_t ncell = P->oct_levels > 0 ? (size_t)P->oct_nleaf : (size_t)n[0] * n[1] * n[2];
        const double* cdf = P->cell_cdf + (size_t)lam * ncell;
        og_draw(P, lam, i, 0u, 0u, u);
        size_t a0 = 0, a1 = ncell - 1; /* first cell with cdf > u */
        while (a0 < a1) {
            size_t mid = (a0 + a1) / 2;
            if (cdf[mid] > u[0]) a1 = mid; else a0 = mid + 1;
        }
        size_t m = a0;
        if (P->oct_levels > 0) {
            /* leaf box: lattice corner c = index << (L - level), side 2^(L - level) */
            const int32_t* lf = P->oct_leaves + 4 * m;
            int shift = P->oct_levels - lf[0];
            double side = (double)(1 << shift);
            for (int a = 0; a < 3; ++a)
                x[a] = lo[a] + ((double)(lf[1 + a] << shift) + u[1 + a] * side) * d[a];
            break;
        }
        int ix = (int)(m % (size_t)n[0]);
        int iy = (int)((m / (size_t)n[0]) % (size_t)n[1]);
        int iz = (int)(m / ((size_t)n[0] * n[1]));
        x[0] = lo[0] + ((double)ix + u[1]) * d[0];
        x[1] = lo[1] + ((double)iy + u[2]) * d[1];
        x[2] = lo[2] + ((double)iz + u[3]) * d[2];
        break;
    }
    default:
        return 0;
    }
    if (isotropic) {
        og_draw(P, lam, i, 0u, 1u, u);
        og_isotropic(u[0], u[1], k);
    }
    return isotropic;
}

static void og_packet(og_problem* P, int lam, uint64_t i, og_work* W)
{
    const size_t NL = (size_t)P->nlambda;
    const double L0 = P->lsrc[lam] / (double)P->npk[lam];
    const double albedo = P->albedo[lam];
    const double g = P->g[lam];
    double L = L0;
    double x[3], k[3];
    double weight[64];
    W->escaped = W->absorbed = W->residual = W->peel = 0.0;

    int isotropic = og_launch(P, lam, i, x, k);
    if (isotropic && P->peel) {
        /* isotropic emission: the phase factor towards every instrument is 1 */
        for (int q = 0; q < P->ninstr; ++q) weight[q] = L;
        og_peel(P, lam, x, weight, W);
    }

    int nscat = 0;
    for (uint32_t e = 1;; ++e) {
        /* Continuous absorption (Sect. 1, 3.2) along the whole path to the
         * grid boundary: segment m with optical depth dtau_m, cumulative
         * tau_{m-1} before it, receives L (1-albedo)(e^{-tau_{m-1}} -
         * e^{-tau_m}) = L (1-albedo) e^{-tau_{m-1}} (1 - e^{-dtau_m}). */
        int nseg = og_path_tree(P, W->tree, x, k, W->cells, W->lens, W->cap);
        if (nseg < 0) { P->status |= OG_ERR_NONFINITE; nseg = 0; }
        P->counters[1] += (double)nseg;
        double tau = 0.0;
        for (int s = 0; s < nseg; ++s) {
            int m = W->cells[s];
            double dtau = P->kr[m] * P->kscale[lam] * W->lens[s];
            double dep = L * (1.0 - albedo) * exp(-tau) * (-expm1(-dtau));
            tau += dtau;
            if (dep > 0.0) {
                P->absorbed[(size_t)m * NL + (size_t)lam] += dep; /* absorb(m, ell, DeltaL) */
                W->absorbed += dep;
            }
        }
        double tau_path = tau;
        W->escaped += L * exp(-tau_path);
        if (!(tau_path > 0.0)) {
            if (!(tau_path == 0.0)) P->status |= OG_ERR_NONFINITE;
            L = 0.0; /* nothing on the path: the whole packet escapes */
            break;
        }

        /* Forced scattering (Sect. 1): the interaction optical depth is drawn
         * from the exponential distribution truncated at tau_path,
         * tau_int = -ln(1 - u (1 - e^{-tau_path})); the packet moves to the
         * point where the cumulative optical depth reaches tau_int and keeps
         * the scattered part L albedo (1 - e^{-tau_path}). */
        double u[4];
        og_draw(P, lam, i, e, 0u, u);
        double tau_int = -log1p(-u[0] * (-expm1(-tau_path)));
        double tcum = 0.0, s_enter = 0.0, s_int = -1.0;
        double last_dusty_end = 0.0;
        int located = 0;
        for (int s = 0; s < nseg; ++s) {
            int m = W->cells[s];
            double krl = P->kr[m] * P->kscale[lam];
            double dtau = krl * W->lens[s];
            P->counters[2] += 1.0;
            if (krl > 0.0 && tcum + dtau >= tau_int) {
                s_int = s_enter + (tau_int - tcum) / krl;
                located = 1;
                break;
            }
            tcum += dtau;
            s_enter += W->lens[s];
            if (krl > 0.0) last_dusty_end = s_enter;
        }
        if (!located) s_int = last_dusty_end; /* rounding left tau just short */
        for (int a = 0; a < 3; ++a) x[a] += s_int * k[a];

        L = L * albedo * (-expm1(-tau_path));
        nscat = (int)e;

        /* scattering peel-off with the Henyey-Greenstein phase function */
        if (L > 0.0 && P->peel) {
            for (int q = 0; q < P->ninstr; ++q) {
                const double* ins = P->instr + 5 * q;
                double inc = ins[1] * OG_PI / 180.0, az = ins[2] * OG_PI / 180.0;
                double kobs[3] = {sin(inc) * cos(az), sin(inc) * sin(az), cos(inc)};
                double mu = k[0] * kobs[0] + k[1] * kobs[1] + k[2] * kobs[2];
                weight[q] = L * og_hg_phase(g, mu);
            }
            og_peel(P, lam, x, weight, W);
        }

        /* termination once all but w_min of the launch luminosity is gone */
        if (L < P->w_min * L0) {
            W->residual += L;
            break;
        }
        if ((int)e >= P->max_events) {
            P->status |= OG_ERR_EVENT_CAP;
            W->residual += L;
            break;
        }
        double mu = og_hg_mu(g, u[1]);
        double phi = 2.0 * OG_PI * u[2];
        double knew[3];
        og_rotate(k, mu, phi, knew);
        for (int a = 0; a < 3; ++a) k[a] = knew[a];
    }
    P->counters[0] += (double)nscat;

    double* led = P->ledger + 4 * (size_t)lam;
    led[0] += L0;
    led[1] += W->absorbed;
    led[2] += W->escaped;
    led[3] += W->residual;
    if (!isfinite(W->escaped + W->absorbed + W->residual + W->peel)) P->status |= OG_ERR_NONFINITE;
    if (i < (uint64_t)P->nrec) {
        double* r = P->records + ((size_t)lam * (size_t)P->nrec + (size_t)i) * OG_REC_FIELDS;
        r[0] = (double)nscat;
        r[1] = W->escaped;
        r[2] = W->absorbed;
        r[3] = W->residual;
        r[4] = W->peel;
        r[5] = x[0];
        r[6] = x[1];
        r[7] = x[2];
    }
}

int og_trace(og_problem* P)
{
    if (P->ninstr > 64) return -1;
    og_work W;
    og_tree T;
    W.tree = NULL;
    if (P->oct_levels > 0) {
        if (og_tree_build(P, &T) != 0) {
            og_tree_free(&T);
            P->status |= OG_ERR_TREE;
            return P->status;
        }
        W.tree = &T;
    }
    W.cap = P->nx + P->ny + P->nz + 8;
    W.cells = (int*)malloc(sizeof(int) * (size_t)W.cap);
    W.lens = (double*)malloc(sizeof(double) * (size_t)W.cap);
    for (int lam = 0; lam < P->nlambda; ++lam) {
        uint64_t end = P->npk[lam] < P->pk_end ? P->npk[lam] : P->pk_end;
        for (uint64_t i = P->pk_begin; i < end; ++i) og_packet(P, lam, i, &W);
    }
    free(W.cells);
    free(W.lens);
    if (W.tree) og_tree_free(&T);
    return P->status;
}
