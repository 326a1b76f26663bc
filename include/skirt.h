/*
 * skirt.h -- C ABI of the GB300 Monte Carlo dust radiative transfer library.
 *
 * The library traces photon packets through a 3-D dust grid (Cartesian, or
 * an adaptive octree as in the paper's Sect. 7.9) on one
 * NVIDIA GB300 (sm_103a) and accumulates the absorbed luminosity per cell and
 * wavelength, per-pixel per-wavelength instrument images and SEDs.  The
 * operations follow the method of Verstocken et al. (arXiv:1705.04702):
 *   Sect. 3.2   simulation phases: setup builds the dust grid; in the stellar
 *               emission phase a fixed number of packets per wavelength is
 *               launched, sampled by Monte Carlo, peeled off towards the
 *               instruments on every scattering event, and continuously
 *               absorbed into the absorbed-luminosity table, until all but a
 *               negligible part of the luminosity is gone;
 *   Sect. 1     the acceleration techniques used: peel-off, continuous
 *               absorption, forced scattering;
 *   Sect. 5.2   the absorbed table is a [cell, wavelength] table of doubles,
 *               element (i, j) at i * N_lambda + j; the instrument table is
 *               indexed on pixel and wavelength; concurrent updates are
 *               lock-free atomic additions.
 *
 * Conventions for every entry point:
 *   - Return value: SKIRT_OK (0) or one of the SKIRT_ERR_* codes below;
 *     skirt_last_error() then gives a message (per calling thread).  Nothing
 *     aborts the process.
 *   - Device: calls run on the CUDA device that is current on the calling
 *     thread; a grid may only be used on the device it was created on.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Every call is synchronous on return (it synchronises `stream`).
 *   - Pointers: "device-or-host" buffers are classified with
 *     cudaPointerGetAttributes; host outputs are staged through device
 *     memory owned by the grid handle and copied back before return.
 *   - Ownership: the caller owns every array it passes; the library owns the
 *     grid handle and the scratch memory attached to it.
 */
#ifndef SKIRT_H
#define SKIRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    SKIRT_OK = 0,
    SKIRT_ERR_INVALID_ARG = 1, /* an argument failed validation; no work done */
    SKIRT_ERR_OOM = 2,         /* device or pinned host allocation failed */
    SKIRT_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SKIRT_ERR_EVENT_CAP = 4,   /* some packet hit max_events; outputs valid, packet ended early */
    SKIRT_ERR_NONFINITE = 5,   /* a NaN/Inf appeared in a packet's bookkeeping */
    SKIRT_ERR_SOURCE = 6,      /* a source position could not be placed inside the grid */
    SKIRT_ERR_NO_DEVICE = 7    /* no CUDA device, or the grid lives on another device */
};

/* Message for the last error returned on this thread ("" if none). */
const char* skirt_last_error(void);

/* Library version string. */
const char* skirt_version(void);

/* Diagnostic environment variables (read at every call; results stay
 * within the parity bars either way, so they serve tests that show what a
 * reading of the method changes):
 *   SKIRT_MIXED_TAU_CUT       mixed form: optical depth at which a deposit or
 *                             peel-off traversal stops, if above the default 30
 *                             (e.g. 1e30: walk every path to the boundary);
 *   SKIRT_EXACT_TABLE_STRIDE  exact dust emission: start the Newton solves from
 *                             every 2^k-th point (k <= 6) of the temperature
 *                             table, so that they take more Newton steps. */

/* ------------------------------------------------------------ dust grid */
/* Setup (Sect. 3.2): the dust grid is the discretisation of the dust
 * distribution into cells.  Cartesian grid of nx*ny*nz cells over the box
 * bbox = {xmin, xmax, ymin, ymax, zmin, zmax} (xmin < xmax, ...); cell
 * (ix, iy, iz) has index m = (iz*ny + iy)*nx + ix.
 *
 * kr: device-or-host float[nx*ny*nz], the extinction coefficient kappa*rho
 * [1/length] of every cell at the reference wavelength (finite, >= 0).
 * The values are copied (FP32, plus an exact FP64 copy for the FP64 form);
 * the caller may free kr on return.  Errors: INVALID_ARG for bad sizes or
 * values (ncell must be < 2^31), OOM, CUDA. */
typedef struct skirt_grid_s* skirt_grid_t;
int skirt_grid_create(skirt_grid_t* out, int nx, int ny, int nz, const double bbox[6],
                      const float* kr);
/* Octree dust grid (the adaptive grid of the ERIS run, Sect. 7.9: up to 13
 * division levels, 8.2 million cells).  The root box bbox is split into 8
 * equal boxes, recursively; the leaves are the cells.  Leaf m (0 <= m <
 * nleaf) is leaves[4m .. 4m+3] = {level, ix, iy, iz}: the box at integer
 * position (ix, iy, iz) among the 2^level boxes per axis of that level
 * (0 <= level <= max_level, 0 <= ix, iy, iz < 2^level).  The leaves must
 * tile the root box exactly: no overlap, no hole.  Every per-cell table of
 * the library (absorbed, dust-source emission, mass, features) is then
 * indexed by leaf in this order.
 *
 * max_level: 1 .. 15.  leaves: host int32[nleaf][4], read during the call.
 * kr: device-or-host float[nleaf] as for skirt_grid_create.  nleaf < 2^27.
 * The library builds a node array with the face neighbours of every leaf
 * (the neighbour of the same or a larger size) on the device and copies kr.
 * Traversal: the FP64 form (precision SKIRT_PREC_FP64) and the mixed form.
 * Errors: INVALID_ARG for sizes, values or leaves that do not tile the box
 * (the message names the first offending leaf), OOM, CUDA. */
int skirt_octree_create(skirt_grid_t* out, int max_level, const double bbox[6], long long nleaf,
                        const int32_t* leaves, const float* kr);

/* Frees the grid and all scratch attached to it.  NULL is accepted. */
int skirt_grid_destroy(skirt_grid_t grid);

/* --------------------------------------------------------------- sources */
enum {
    SKIRT_SRC_POINT = 0, /* isotropic point source at pos */
    SKIRT_SRC_DISK = 1,  /* exponential disk centred on pos, axis +z:
                            surface density ~ exp(-R/h_R), vertical ~ exp(-|z|/h_z);
                            positions outside the grid are redrawn */
    SKIRT_SRC_BEAM = 2,  /* collimated beam from pos along dir (unit); no emission peel-off */
    SKIRT_SRC_DUST = 3   /* dust cells: cell drawn with probability proportional to
                            emission[cell, lambda], uniform point inside it; isotropic */
};

typedef struct {
    int kind;               /* SKIRT_SRC_* */
    double pos[3];          /* point / beam origin / disk centre (inside the grid) */
    double dir[3];          /* beam direction, unit length */
    double h_R, h_z;        /* disk scale length and height (> 0) */
    const double* emission; /* DUST only: device double[ncell][nlambda], >= 0, not all zero
                               for any wavelength with packets */
} skirt_source;

/* ----------------------------------------------------------- wavelengths */
/* One column of the absorbed table per wavelength (Sect. 5.2).  All arrays
 * are host double[n]. */
typedef struct {
    int n;                /* number of wavelengths, 1 <= n <= 65536 */
    const double* kscale; /* kappa_ext(lambda) / kappa_ext(reference), finite, >= 0 */
    const double* albedo; /* scattering albedo in [0, 1] */
    const double* g;      /* Henyey-Greenstein asymmetry, |g| < 1 */
    const double* lsrc;   /* luminosity emitted in this wavelength bin, >= 0; may be NULL for a
                             dust-cell source: then the column sums of its emission table */
} skirt_wavelengths;

/* ----------------------------------------------------------- instruments */
/* Distant observer (peel-off target, Sect. 3.2): direction of observation
 * k = (sin i cos a, sin i sin a, cos i) for inclination i and azimuth a;
 * image axes e1 = (-sin a, cos a, 0), e2 = k x e1; pixel (row, col) =
 * floor((x.e2 + fov/2)/(fov/npx)), floor((x.e1 + fov/2)/(fov/npx)).
 * A peel-off adds L e^{-tau} / (4 pi distance^2) to that pixel (when inside
 * the frame) and to the SED. */
typedef struct {
    double distance;        /* > 0 */
    double inclination_deg;
    double azimuth_deg;
    double fov;             /* > 0, square field centred on the origin */
    int npx;                /* 1 .. 16384 pixels per side */
} skirt_instrument;

/* --------------------------------------------------------------- tracing */
enum { SKIRT_PREC_FP64 = 0, SKIRT_PREC_MIXED = 1 };
enum { SKIRT_SCHED_PER_LAMBDA = 0, SKIRT_SCHED_PERSISTENT = 1 };
enum { SKIRT_REC_FIELDS = 8 };

typedef struct {
    int precision;     /* SKIRT_PREC_FP64: the plain form, FP64 throughout.
                          SKIRT_PREC_MIXED: FP32 directions, cell traversal, phase-function
                          sampling and packet luminosity; positions as FP32 (hi, lo) pairs;
                          the cumulative optical depth of a traversal summed error-free
                          (double-float) and formed in FP64 at every event; all tallies and
                          the energy ledger in FP64.  A deposit or peel-off traversal ends
                          once its optical depth exceeds 30 (what is left is below 1e-13 of
                          the packet's luminosity). */
    int schedule;      /* SKIRT_SCHED_PER_LAMBDA: one launch per wavelength, one packet per
                          thread.  SKIRT_SCHED_PERSISTENT: one persistent launch for all
                          wavelengths; threads refill from a global work queue. */
    double w_min;      /* a packet ends once its luminosity drops below w_min times its
                          launch luminosity (<= 0 selects 1e-4) */
    int max_events;    /* scattering cap per packet (<= 0 selects 10000); reaching it ends the
                          packet, books the rest as residual and returns SKIRT_ERR_EVENT_CAP */
    int peel;          /* 1: peel-off towards the instruments; 0: none (dust self-absorption) */
    int accumulate;    /* 0: outputs are zeroed first; 1: tallies are added to their contents */
    int block;         /* threads per block: a multiple of 32, up to 256 (mixed form) or 512
                          (FP64 form); 0 = default 256 */
    int chunk;         /* packets a thread takes per queue refill (persistent); 0 = default */
    int blocks_per_sm; /* persistent grid = blocks_per_sm x SM count; 0 = from occupancy */
    int use_graph;     /* 1: record the launch sequence in a CUDA graph, cached on the grid
                          and replayed by later calls with identical arguments */
    int step_min;      /* mixed form: a warp keeps stepping cells while at least step_min of
                          its lanes are inside a traversal, then handles the events of the
                          idle lanes together (1..32; 0 = default 20) */
    uint32_t phase;    /* random-stream phase: 0 stellar, 1 dust re-emission (< 256) */
    int nrec;          /* >= 0: per-packet records for packet indices < nrec */
    double* records;   /* device-or-host double[n][nrec][8]: scatterings, escaped, absorbed,
                          residual, peeled flux, x, y, z of the last interaction */
    /* Packet ranges (the task split of Sect. 5.2: each process launches its own
     * share of every wavelength's packets and the tables are summed).  Both
     * host uint64[n] or NULL.  Packet i (0 <= i < npackets[j]) of wavelength j
     * is packet first_packet[j] + i of the run: that index keys its random
     * stream, while records stay indexed by i.  The luminosity per packet is
     * lsrc[j] / total_packets[j].  NULL first_packet means all zeros, NULL
     * total_packets means npackets.  Then first_packet[j] + npackets[j] must
     * not exceed total_packets[j], nor 2^32.  Calls over disjoint ranges of the
     * same run therefore trace exactly the packets of one call over all of
     * them, and their tables add up to its tables. */
    const uint64_t* first_packet;
    const uint64_t* total_packets;
} skirt_trace_opts;

/* Fills *opts with the defaults (mixed precision, persistent, peel on). */
int skirt_trace_opts_default(skirt_trace_opts* opts);

/* Energy ledger and work counters of one trace call (all wavelengths). */
typedef struct {
    double emitted, absorbed, escaped, residual; /* emitted = absorbed+escaped+residual */
    double scatterings;                           /* forced interactions */
    double deposit_steps, locate_steps, peel_steps; /* cell crossings per traversal kind */
    int status_bits;                              /* 1 event cap, 2 source, 4 non-finite,
                                                     8 an octree path over its crossing bound */
    float kernel_ms;                              /* device time of the trace launches */
} skirt_ledger;

/* Stellar (or dust) emission phase (Sect. 3.2): npackets[j] packets at every
 * wavelength j, each carrying lsrc[j]/npackets[j], traced with peel-off,
 * continuous absorption and forced Henyey-Greenstein scattering.  Packet i
 * at wavelength j draws its random numbers from Philox4x32-10 with key
 * (seed low, seed high) and counter (i, j, event, phase<<24 | draw), so
 * every packet history is reproducible and independent of the schedule.
 *
 * Outputs (device-or-host, all double):
 *   absorbed  [ncell][n]                    (Sect. 5.2 table layout)
 *   images    per instrument q: [npx_q*npx_q][n], concatenated in order q
 *   sed       [ninstr][n]
 * images and sed may be NULL when ninstr == 0.  ledger (host) may be NULL;
 * ledger_per_lambda (host double[n][4], emitted/absorbed/escaped/residual)
 * may be NULL.
 * With n > 1 the packets deposit into a wavelength-major copy of the
 * absorbed table ([n][ncell], grid scratch of the same size as the table)
 * that one transpose turns into the [ncell][n] result (or adds to it with
 * accumulate); without room for the copy they deposit in place.
 * Limits: npackets[j] < 2^32; 0 <= ninstr <= 16.
 * Errors: INVALID_ARG, OOM, CUDA; EVENT_CAP / NONFINITE / SOURCE after a
 * completed trace whose ledger flagged the condition (NONFINITE also for an
 * octree traversal abandoned after 3 * 2^levels + 8 crossings). */
int skirt_trace(skirt_grid_t grid, const skirt_source* src, const skirt_wavelengths* wl,
                const uint64_t* npackets, uint64_t seed, const skirt_instrument* ins, int ninstr,
                const skirt_trace_opts* opts, double* absorbed, double* images, double* sed,
                skirt_ledger* ledger, double* ledger_per_lambda, void* stream);

/* Autotuner (the GPU counterpart of choosing the hybrid scheme for the
 * hardware, Sect. 6.2): times the persistent schedule on a sample of
 * the workload (every npackets[j] scaled by sample_fraction, at least one
 * packet where npackets[j] > 0).  Candidates: the schedule *opts asks for
 * (its zero fields at their defaults), then block sizes {64, 128, 256} (and
 * 512 for the FP64 form) x refill chunks {1, 4, 16} x step_min {16, 20, 24}
 * (mixed form) x resident blocks per SM from the occupancy limit down,
 * halving.  After one untimed warm-up launch, every candidate is timed
 * `repeats` times (<= 0 selects 2) and scored by its fastest launch.  A
 * small sample favours schedules that end a short run evenly, so the three
 * fastest candidates and the requested schedule are timed again on a sample
 * five times larger (at most the whole workload); the fastest of those
 * replaces the requested schedule only if it is faster there by more than
 * 2%.  The result is written into opts->block / chunk / blocks_per_sm /
 * step_min.  report (may be NULL) receives the sweep.  The outputs are used
 * as scratch and left zeroed.  Errors as skirt_trace. */
enum { SKIRT_TUNE_MAX_POINTS = 256 };
typedef struct {
    int block, chunk, blocks_per_sm, step_min;
    float ms;                /* fastest of the repeats, device time of the trace launch */
    float ms_confirm;        /* time on the larger sample (0: not re-timed) */
} skirt_tune_point;
typedef struct {
    int n;                   /* candidates timed; point 0 is the requested schedule */
    int chosen;              /* index of the schedule written into opts */
    int repeats;
    unsigned long long sample_packets, confirm_packets;
    skirt_tune_point points[SKIRT_TUNE_MAX_POINTS];
} skirt_tune_report;
int skirt_autotune(skirt_grid_t grid, const skirt_source* src, const skirt_wavelengths* wl,
                   const uint64_t* npackets, uint64_t seed, const skirt_instrument* ins, int ninstr,
                   skirt_trace_opts* opts, double sample_fraction, int repeats, double* absorbed,
                   double* images, double* sed, skirt_tune_report* report, void* stream);

/* ---------------------------------------------------------- dust emission */
/* Dust emission phase (Sect. 3.2: the emission spectrum of every dust cell
 * is computed from the amount of absorbed radiation; Sect. 1: instantaneous
 * dust emission).  Model (the paper gives none; equilibrium emission of three
 * grain populations):
 *   absorption shares w_i(lambda) ~ (lambda/0.55um)^delta_i, delta = (-0.5, 0, 0.5),
 *     normalised to sum 1; P_i(m) = sum_j w_i(lambda_j) absorbed(m, j);
 *   output grid: 100 wavelengths log-spaced over 1-1000 um, trapezoid weights W_l;
 *   opacities kappa_i = (lambda/100um)^-beta_i, beta = (1.5, 2, 2);
 *   B(lambda, T) = lambda^-5 / (exp(hc/(k lambda T)) - 1);
 *   energy balance M c_i G_i(T_i) = P_i, G_i(T) = sum_l W_l kappa_i B(lambda_l, T),
 *     c_i = 1/G_i(30 K), M = dust mass of the cell (extinction coefficient x volume);
 *     T_i by bracketed Newton on ln T in [3, 2000] K (clamped), accepted when the
 *     step is below 1e-13 of ln T; the per-population steps run in FP64, the
 *     Planck terms in double-float (~2e-14 relative; terms with
 *     hc/(k lambda T) > 70, below 4e-23 of G_i, are left out);
 *   emission(m, l) = sum_i P_i W_l kappa_i B(lambda_l, T_i) / G_i(T_i)
 *     (luminosity in output bin l; the row sums to the absorbed power). */
enum { SKIRT_EMIT_EXACT = 0, SKIRT_EMIT_SURROGATE = 1 };
enum { SKIRT_NBANDS = 32, SKIRT_NEMIT = 100, SKIRT_MLP_HIDDEN = 128 };
/* Number of floats in a packed parameter vector: W1[128][32] b1[128]
 * W2[128][128] b2[128] W3[100][128] b3[100] (rows = outputs). */
enum { SKIRT_MLP_NPARAM = 128 * 32 + 128 + 128 * 128 + 128 + 100 * 128 + 100 };

/* The output wavelength grid: lambda[100] in micron and its trapezoid
 * weights W[100] (host arrays, either may be NULL). */
int skirt_emission_grid(double* lambda_um, double* weights);

/* Dust mass of every cell, M = kr * cell volume (the leaf's box on an
 * octree grid), device float[ncell]. */
int skirt_dust_mass(skirt_grid_t grid, float* mass, void* stream);

/* Band compression: B_b(m) = sum of absorbed(m, j) over the input
 * wavelengths j in band b, 32 bands log-spaced over [min, max] of lambda_in;
 * T(m) = sum_b B_b(m), features(m, b) = log10(max(B_b, 1e-6 T / 32) / M)
 * (a band without absorbed power sits 6 dex below the cell's total; cells
 * without dust or absorbed power get -30), total(m) = T(m).  B_b and T are
 * summed in FP64 (T exact to FP64 rounding); the features are formed in FP32
 * from B_b truncated to FP32 (a few FP32 ulp).  absorbed: device double[ncell][n_in];
 * lambda_in: host double[n_in] (micron, > 0); mass: device float[ncell];
 * features: device float[ncell][32]; total: device double[ncell]. */
int skirt_band_features(const double* absorbed, long long ncell, int n_in, const double* lambda_in,
                        const float* mass, float* features, double* total, void* stream);

/* The MLP surrogate 32 -> 128 -> 128 -> 100 (SiLU, SiLU, softmax): input
 * the 32 band features standardised with the training set's mean / std,
 * output the normalised emission shape, times total(m).  Inference and
 * training run on the tensor cores with BF16 operands and FP32 accumulation;
 * training keeps FP32 master weights (and FP32 SiLU derivatives, softmax and
 * bias sums).  The network also stores the
 * per-feature range [lo, hi] of its training inputs (the "hull"). */
typedef struct skirt_mlp_s* skirt_mlp_t;
int skirt_mlp_create(skirt_mlp_t* out, uint64_t seed); /* Kaiming-uniform init from seed */
int skirt_mlp_destroy(skirt_mlp_t net);
/* Host float arrays: params[SKIRT_MLP_NPARAM], x_mean/x_std/hull_lo/hull_hi[32]; any may be NULL. */
int skirt_mlp_set_params(skirt_mlp_t net, const float* params, const float* x_mean, const float* x_std,
                         const float* hull_lo, const float* hull_hi);
int skirt_mlp_get_params(skirt_mlp_t net, float* params, float* x_mean, float* x_std, float* hull_lo,
                         float* hull_hi);

typedef struct {
    int epochs;          /* passes over the training set (default 200) */
    int batch;           /* samples per Adam step (default 2048) */
    float lr;            /* Adam step size (default 2e-3, cosine-decayed to lr/20) */
    float beta1, beta2, eps; /* Adam moments (defaults 0.9, 0.999, 1e-8) */
    uint64_t seed;       /* batch order */
    float guard_quantile; /* the guard's threshold: this quantile of the training rows' dominant-band
                             share (default 0.99; >= 1 disables the guard) */
} skirt_mlp_train_opts;
int skirt_mlp_train_opts_default(skirt_mlp_train_opts* opts);

/* The guard that sends rows to the exact solver besides the range hull: a
 * row whose dominant band holds more than share_max of the cell's absorbed
 * power (share = 1 / sum_b 10^(f_b - max_b f_b), from the raw features) is
 * outside it.  Such cells are rare in training (their emission depends on
 * where within the band the power sits, which the features do not say) and
 * carry most of the surrogate's large errors.  share_max > 0; >= 1 disables
 * it.  skirt_mlp_train sets it from the training rows (guard_quantile). */
int skirt_mlp_set_guard(skirt_mlp_t net, float share_max);
int skirt_mlp_get_guard(skirt_mlp_t net, float* share_max);

/* Trains on n samples: features (device float[n][32], raw band features)
 * and emission (device double[n][100], e.g. the exact solver's output; every
 * row is normalised to sum 1 on the device and used as the target shape t)
 * with the cross-entropy loss -sum_l t_l log p_l.  Sets the standardisation,
 * the hull and the guard from the training features.  loss_history: host
 * float[epochs] (mean loss per epoch) or NULL. */
int skirt_mlp_train(skirt_mlp_t net, const float* features, const double* emission, long long n,
                    const skirt_mlp_train_opts* opts, float* loss_history, void* stream);

/* One batch of the training arithmetic: loss and gradient of the mean
 * cross-entropy with respect to the packed FP32 parameters, for the
 * standardised inputs x_std (device-or-host float[n][32]) and target shapes
 * (device-or-host float[n][100]) -> grad: host float[SKIRT_MLP_NPARAM].
 * Every operand of a product is rounded to BF16 (inputs, weights,
 * activations, back-propagated dz); accumulation, SiLU derivatives, softmax
 * and the bias sums are FP32. */
int skirt_mlp_grad(skirt_mlp_t net, const float* x_std, const float* target, int n, float* grad, float* loss,
                   void* stream);

/* Tensor-core inference: emission (device double[n][100]) = softmax(MLP(
 * (features - mean) / std)) * total (device double[n]).  features: device
 * float[n][32], 16-byte aligned (its 128-byte rows are fetched by bulk
 * asynchronous copies).  If flags is not NULL (device unsigned char[n]) it
 * receives 1 for rows with total > 0 whose features fall outside the hull or
 * the guard (skirt_mlp_set_guard).
 * Errors: INVALID_ARG (also for unaligned features), CUDA. */
int skirt_mlp_forward(skirt_mlp_t net, const float* features, const double* total, long long n,
                      double* emission, unsigned char* flags, void* stream);

typedef struct {
    unsigned long long n_cells;     /* cells processed */
    unsigned long long n_fallback;  /* surrogate mode: cells sent to the exact solver */
    float ms_features, ms_surrogate, ms_exact; /* device time of the three stages */
} skirt_emission_stats;

/* Emission of every cell from its absorbed spectrum.  mode EXACT: the exact
 * solver on every cell.  mode SURROGATE: band features -> MLP on every cell,
 * then the exact solver overwrites the rows whose features fall outside the
 * network's hull or guard (net required).  absorbed: device double[ncell][n_in];
 * lambda_in: host double[n_in]; mass: device float[ncell]; emission: device
 * double[ncell][100]; temperature: device float[ncell][3] or NULL (exact rows
 * only; 0 for surrogate rows); stats: host or NULL.  Surrogate mode keeps its
 * working tables (~150 bytes per cell) in the network handle, allocated on the
 * first call that needs them and freed by skirt_mlp_destroy; calls that share
 * a network run one at a time. */
int skirt_dust_emission(const double* absorbed, long long ncell, int n_in, const double* lambda_in,
                        const float* mass, int mode, skirt_mlp_t net, double* emission, float* temperature,
                        skirt_emission_stats* stats, void* stream);

/* Per-wavelength luminosity of a dust emission table (Sect. 3.2: the dust
 * cells are the sources of the dust emission phases): the column sums over
 * the cells of emission [ncell][nlambda] (device doubles, ncell = the grid's
 * cells), in FP64, into host totals[nlambda].  These are the source
 * luminosities skirt_trace takes for a dust-cell source without lsrc, so a
 * caller can give packets only to wavelengths that carry luminosity.  Uses
 * the grid's scratch memory; synchronises the stream.  Errors: INVALID_ARG
 * (also for negative or non-finite entries), OOM, CUDA. */
int skirt_emission_totals(skirt_grid_t grid, const double* emission, int nlambda, double* totals, void* stream);

/* Exact dust emission of cells heated by two absorbed fields on two
 * wavelength grids (Sect. 3.2, dust self-absorption phase: each cycle's
 * emission follows from the absorbed stellar radiation plus the absorbed
 * emission of the dust itself, kept in a separate table).  The power each
 * grain population absorbs adds:
 * P_i(m) = sum_j w_i(lambda_a,j) A(m, j) + sum_l w_i(lambda_b,l) B(m, l),
 * then the same equilibrium solve and emission rows as skirt_dust_emission
 * in SKIRT_EMIT_EXACT mode (rows sum to P_0 + P_1 + P_2).
 * absorbed_a: device double[ncell][n_a] on the host grid lambda_a;
 * absorbed_b: device double[ncell][n_b] on lambda_b, or NULL with n_b = 0
 * (then the result equals skirt_dust_emission's); mass: device float[ncell];
 * emission: device double[ncell][100]; temperature: device float[ncell][3] or
 * NULL.  Synchronises the stream on return.  Errors: INVALID_ARG, OOM, CUDA. */
int skirt_dust_emission_pair(const double* absorbed_a, long long ncell, int n_a, const double* lambda_a,
                             const double* absorbed_b, int n_b, const double* lambda_b, const float* mass,
                             double* emission, float* temperature, void* stream);

/* Exact emission without allocating (the paper has no counterpart: it is an
 * interface for callers that cannot allocate device memory at call time,
 * e.g. a process whose framework allocator has already reserved the device
 * memory it may use, or a loop run on a memory budget fixed up front).
 * Same result as skirt_dust_emission in SKIRT_EMIT_EXACT mode, same argument
 * meaning (all arrays device memory, lambda_in host, temperature may be NULL),
 * no statistics.  Its only working table, the absorption shares of the input
 * wavelengths, lives in a fixed device array of 3 x 4096 doubles (96 KiB) that
 * every device loading the library holds until the process exits: n_in above
 * 4096 is rejected with SKIRT_ERR_INVALID_ARG.  The first call on a device
 * looks up the array's device address (once per device, with that device
 * current); make that first call before any stream capture.  Every call
 * rewrites the table in full; calls share it, so calls that overlap on the
 * GPU (other threads or streams) race.  Synchronises the stream on return. */
int skirt_dust_emission_exact_static(const double* absorbed, long long ncell, int n_in, const double* lambda_in,
                                     const float* mass, double* emission, float* temperature, void* stream);

/* The device random-number generator: Philox4x32-10 (Salmon, Moraes, Dror &
 * Shaw, SC'11), the function every trace kernel draws its Monte Carlo samples
 * with (Sect. 3.2; counter = (packet, wavelength, event, phase << 24 | block),
 * key = (seed low, seed high)).  ctr: host uint32[n][4]; key: host
 * uint32[n][2]; out: host uint32[n][4] receives the n output blocks.
 * 0 <= n <= 2^24; synchronous (legacy default stream).  Errors: INVALID_ARG,
 * NO_DEVICE, OOM, CUDA. */
int skirt_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n);

/* Microbenchmarks for the rooflines of the trace kernel (no counterpart in
 * the paper, which ran on CPUs): kind 0 FP64 FMA rate, 1 FP32 FMA rate,
 * 2 FP32<->FP64 conversion rate, 3 random-address red.global.add.f64 into a
 * table of `size` doubles, 4 random FP32 gathers from a table of `size`
 * floats.  *rate receives operations per second, *ms the kernel time.
 * Allocates and frees its own device buffers.  Errors: INVALID_ARG, CUDA. */
int skirt_microbench(int kind, long long size, double* rate, float* ms);

#ifdef __cplusplus
}
#endif
#endif /* SKIRT_H */
