/*
 * skirt.h -- C ABI of the GB300 Monte Carlo dust radiative transfer library.
 *
 * The library traces photon packets through a 3-D Cartesian dust grid on one
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
    const double* lsrc;   /* luminosity emitted in this wavelength bin, >= 0 */
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
                          SKIRT_PREC_MIXED: FP32 positions, directions, cell traversal and
                          phase-function sampling; FP64 cumulative optical depth, packet
                          luminosity, and all tallies. */
    int schedule;      /* SKIRT_SCHED_PER_LAMBDA: one launch per wavelength, one packet per
                          thread.  SKIRT_SCHED_PERSISTENT: one persistent launch for all
                          wavelengths; threads refill from a global work queue. */
    double w_min;      /* a packet ends once its luminosity drops below w_min times its
                          launch luminosity (<= 0 selects 1e-4) */
    int max_events;    /* scattering cap per packet (<= 0 selects 10000); reaching it ends the
                          packet, books the rest as residual and returns SKIRT_ERR_EVENT_CAP */
    int peel;          /* 1: peel-off towards the instruments; 0: none (dust self-absorption) */
    int accumulate;    /* 0: outputs are zeroed first; 1: tallies are added to their contents */
    int block;         /* threads per block (multiple of 32, <= 1024); 0 = default 256 */
    int chunk;         /* packets a thread takes per queue refill (persistent); 0 = default */
    int blocks_per_sm; /* persistent grid = blocks_per_sm x SM count; 0 = from occupancy */
    int use_graph;     /* 1: record the launch sequence in a CUDA graph, cached on the grid
                          and replayed by later calls with identical arguments */
    int step_min;      /* mixed form: a warp keeps stepping cells while at least step_min of
                          its lanes are inside a traversal, then handles the events of the
                          idle lanes together (1..32; 0 = default 16) */
    uint32_t phase;    /* random-stream phase: 0 stellar, 1 dust re-emission (< 256) */
    int nrec;          /* >= 0: per-packet records for packet indices < nrec */
    double* records;   /* device-or-host double[n][nrec][8]: scatterings, escaped, absorbed,
                          residual, peeled flux, x, y, z of the last interaction */
} skirt_trace_opts;

/* Fills *opts with the defaults (mixed precision, persistent, peel on). */
int skirt_trace_opts_default(skirt_trace_opts* opts);

/* Energy ledger and work counters of one trace call (all wavelengths). */
typedef struct {
    double emitted, absorbed, escaped, residual; /* emitted = absorbed+escaped+residual */
    double scatterings;                           /* forced interactions */
    double deposit_steps, locate_steps, peel_steps; /* cell crossings per traversal kind */
    int status_bits;                              /* 1 event cap, 2 source, 4 non-finite */
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
 * Limits: npackets[j] < 2^32; 0 <= ninstr <= 16.
 * Errors: INVALID_ARG, OOM, CUDA; EVENT_CAP / NONFINITE / SOURCE after a
 * completed trace whose ledger flagged the condition. */
int skirt_trace(skirt_grid_t grid, const skirt_source* src, const skirt_wavelengths* wl,
                const uint64_t* npackets, uint64_t seed, const skirt_instrument* ins, int ninstr,
                const skirt_trace_opts* opts, double* absorbed, double* images, double* sed,
                skirt_ledger* ledger, double* ledger_per_lambda, void* stream);

/* Autotuner (the GPU counterpart of choosing the hybrid scheme for the
 * hardware, Sect. 6.2): times the persistent schedule on a sample of
 * the workload (every npackets[j] scaled by sample_fraction, at least one
 * packet where npackets[j] > 0) over block sizes {64,128,256,512}, refill
 * chunks {1,2,4,8,16} and 1..max resident blocks per SM, and writes the
 * fastest block / chunk / blocks_per_sm into *opts.  The outputs are used as
 * scratch and left zeroed.  Errors as skirt_trace. */
int skirt_autotune(skirt_grid_t grid, const skirt_source* src, const skirt_wavelengths* wl,
                   const uint64_t* npackets, uint64_t seed, const skirt_instrument* ins, int ninstr,
                   skirt_trace_opts* opts, double sample_fraction, double* absorbed,
                   double* images, double* sed, void* stream);

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
