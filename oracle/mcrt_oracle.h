/*
 * CPU FP64 oracle of the photon-packet life cycle -- TEST INFRASTRUCTURE.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark use this; the product path is the CUDA library and never calls
 * into here.  Nothing in this directory shares code with the CUDA library.
 */
#ifndef MCRT_ORACLE_H
#define MCRT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OG_SRC_POINT = 0, OG_SRC_DISK = 1, OG_SRC_BEAM = 2, OG_SRC_DUST = 3 };
enum { OG_ERR_EVENT_CAP = 1, OG_ERR_SOURCE = 2, OG_ERR_NONFINITE = 4, OG_ERR_TREE = 8 };
enum { OG_REC_FIELDS = 8 };

typedef struct {
    /* dust grid: kr[(iz*ny + iy)*nx + ix] = extinction coefficient at the
       reference wavelength */
    int nx, ny, nz;
    double bbox[6];
    const double* kr;
    /* source */
    int src_kind;
    double src_pos[3];
    double src_dir[3];
    double h_R, h_z;
    const double* cell_cdf; /* dust source: [nlambda][ncell] cumulative, last = 1 */
    /* wavelengths */
    int nlambda;
    const double* kscale;
    const double* albedo;
    const double* g;
    const double* lsrc;
    const uint64_t* npk;
    uint64_t seed;
    uint32_t phase;
    /* instruments: [ninstr][5] = distance, inclination(deg), azimuth(deg), fov, npx */
    int ninstr;
    const double* instr;
    double w_min;
    int max_events;
    int peel;
    /* packet-index range run at every wavelength: [pk_begin, min(pk_end, npk)) */
    uint64_t pk_begin, pk_end;
    /* outputs, accumulated into */
    double* absorbed; /* [ncell][nlambda] */
    double* images;   /* per instrument: [npx*npx][nlambda], concatenated */
    double* sed;      /* [ninstr][nlambda] */
    double* ledger;   /* [nlambda][4] emitted, absorbed, escaped, residual */
    double* counters; /* [4] scatterings, deposit segments, locate segments, peel segments */
    int nrec;         /* per-packet records for packet indices < nrec */
    double* records;  /* [nlambda][nrec][8] */
    int status;       /* OR of OG_ERR_* */
    /* octree grid instead of the regular one when oct_levels > 0: the root
       box is bbox, nx = ny = nz = 2^oct_levels is the finest lattice, and
       oct_leaves[m] = (level, ix, iy, iz) places leaf m at its own level;
       kr, absorbed and cell_cdf are then indexed by leaf */
    int oct_levels;
    int64_t oct_nleaf;
    const int32_t* oct_leaves;
} og_problem;

void og_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double og_uniform(uint32_t x);
int og_path(const og_problem* P, const double p[3], const double k[3], int* cells, double* lens, int cap);
double og_hg_mu(double g, double u);
void og_rotate(const double k[3], double mu, double phi, double out[3]);
int og_trace(og_problem* P);
int og_octree_check(const og_problem* P);

#ifdef __cplusplus
}
#endif
#endif
