// Internal declarations shared by the translation units of libskirt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "skirt.h"

namespace skirt {

// ---------------------------------------------------------------------------
// Counter-based random numbers: Philox4x32 with 10 rounds (Salmon et al.,
// SC'11).  Round: multiply words 0 and 2 by the two Philox multipliers, swap
// the halves across and xor the high halves with the other words and the
// round key; the key advances by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t h0 = __umulhi(m0, c.x), l0 = m0 * c.x;
        uint32_t h1 = __umulhi(m1, c.z), l1 = m1 * c.z;
        c = make_uint4(h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform deviate in (0, 1): (top 23 bits + 1/2) * 2^-23.  Exactly
// representable in FP32, so both precisions see identical values.
__device__ __forceinline__ float u01f(uint32_t x) { return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-7f; }

// Per-instrument constants (host-computed in FP64, FP32 copies for the mixed form).
struct InstrDev {
    double kobs[3], e1[3], e2[3];
    double half_fov, inv_dpx, flux_norm;
    float kobs_f[3], e1_f[3], e2_f[3];
    float half_fov_f, inv_dpx_f, flux_norm_f;
    int npx;
    long long img_off;  // element offset of this instrument in the images array
};

enum { ERRBIT_EVENT_CAP = 1, ERRBIT_SOURCE = 2, ERRBIT_NONFINITE = 4, ERRBIT_PATH = 8 };

// Octree node (32 bytes, one sector).  ref >= 0: internal node whose 8
// children are nodes ref .. ref+7 (octant x + 2y + 4z; ref is a multiple of
// 8, node 0 is the root and nodes 1..7 are unused); ref < 0: a leaf,
// ~ref = level << 27 | leaf index (levels up to 15).  kr: the leaf's extinction coefficient.
// nb[2a + (positive side)]: for a leaf, the node across that face along
// axis a of the same level, or the leaf of a larger size that covers it
// (-1 outside the root box).
struct __align__(16) OctNode {
    int ref;
    float kr;
    int nb[6];
};
constexpr int OCT_LEAF_BITS = 27;
__host__ __device__ __forceinline__ int oct_leaf_index(int ref) { return (~ref) & ((1 << OCT_LEAF_BITS) - 1); }
__host__ __device__ __forceinline__ int oct_leaf_level(int ref) { return (~ref) >> OCT_LEAF_BITS; }

struct TraceArgs {
    const float* kr32;
    const double* kr64;
    int nx, ny, nz;
    long long ncell;                       // nx*ny*nz, or the number of octree leaves
    double lo[3], d[3], hi[3];
    int nlambda;
    const double* kscale;
    const double* albedo;
    const double* g;
    const double* L0;                      // luminosity per packet at each wavelength
    const float* kscale_f;                 // FP32 copies of the four tables (mixed form)
    const float* albedo_f;
    const float* g_f;
    const float* L0_f;
    const float2* faces;                   // face planes as (hi, lo) FP32 pairs: x [nx+1], y [ny+1], z [nz+1]
    float2 src_df[3];                      // source position as (hi, lo) FP32 pairs
    float src_dir_f[3];
    float hi_f[3];
    float w_min_f;
    const unsigned long long* offsets;     // [nlambda + 1] prefix sums of packet counts
    const unsigned long long* pk_first;    // [nlambda] stream index of each wavelength's first packet
    unsigned long long total;
    int src_kind;
    double src_pos[3], src_dir[3], h_R, h_z;
    const double* cdf;                     // dust source: [nlambda][ncell] cumulative, normalised
    int ninstr;
    const InstrDev* ins;
    double* absorbed;                      // element (cell, lambda) at cell * abs_cs + lambda * abs_ls
    long long abs_cs, abs_ls;              // [cell][lambda]: (nlambda, 1); [lambda][cell]: (1, ncell)
    double* images;                        // per instrument [npx*npx][nlambda]
    double* oof;                           // [ninstr][nlambda] peel-offs outside the frame
    double* ledger;                        // [nlambda][4]
    unsigned long long* counters;          // [4]
    unsigned int* err;
    int nrec;
    double* records;                       // [nlambda][nrec][8]
    double w_min;
    int max_events;
    int peel;
    uint32_t key0, key1, phase;
    unsigned long long* queue;
    int chunk;
    int persistent;
    unsigned long long q_base, q_count;    // per-wavelength schedule: this launch's packets
    int step_min;                          // mixed form: lanes still stepping below which a warp
                                           // switches to handling the events of its idle lanes
    // octree grid (oct_levels > 0): nx = ny = nz = 2^oct_levels is the finest
    // lattice, d its cell size; cells are leaves
    int oct_levels;
    const OctNode* oct_nodes;
    const int4* oct_leaf;                  // per leaf: lattice corner x, y, z and level
    int oct_step_cap;                      // crossings after which a traversal is abandoned
    float tau_cut;                         // mixed form: optical depth at which a deposit or peel-off
                                           // traversal stops (30; larger values are a diagnostic)
};

// trace.cu (FP64 form; dispatches the mixed form to trace_mixed.cu)
cudaError_t launch_trace(const TraceArgs& a, int precision, int block, int grid, cudaStream_t s);
cudaError_t trace_occupancy(int precision, int block, int* blocks_per_sm, bool octree);
size_t trace_smem_bytes(int ninstr, int block);
// trace_mixed.cu
cudaError_t launch_trace_mixed(const TraceArgs& a, int block, int grid, cudaStream_t s);
cudaError_t trace_mixed_occupancy(int block, int* blocks_per_sm, bool octree);
size_t trace_mixed_smem_bytes(int ninstr, int block);
// out[cell][lambda] (+)= in[lambda][cell]: the absorbed table from the trace's
// wavelength-major accumulation to the API's cell-major layout
cudaError_t launch_transpose_absorbed(const double* in, double* out, long long ncell, int nlambda, bool add,
                                      cudaStream_t s);
// sed[q][lambda] += sign * (sum over the pixels of images_q) + oof[q][lambda] (oof may be NULL)
cudaError_t launch_sed_finalize(const double* images, const double* oof, double* sed, int ninstr,
                                const int* npx_host, int nlambda, double sign, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float* in, double* out, long long n, unsigned int* bad,
                              cudaStream_t s);

// Device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n)
    {
        if (n <= bytes && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, n ? n : 16);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n ? n : 16;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

// Pinned host buffer that only grows.
struct PinnedBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n)
    {
        if (n <= bytes && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMallocHost(&p, n ? n : 16);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n ? n : 16;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
    }
};

// mlp_train.cu: one training step (adam = 1) or one gradient (adam = 0) of the
// emission surrogate on nrows rows (see the kernels there)
int train_rows_per_cta();
size_t train_tile_smem_bytes();
cudaError_t launch_train_step(const uint16_t* Wb, const float* P, const float* feat, const float* target,
                              const float* stats, const unsigned long long* ab, long long* t_dev,
                              long long steps, long long n_data, const float* x_std, int nrows, float* part,
                              float* part_loss, float* G, int adam, float* Pw, float* Mo, float* Vo,
                              const float* sched, float b1, float b2, float eps, uint16_t* Wb_out, float* loss_acc,
                              unsigned* done, cudaStream_t s);

// error reporting shared by the translation units (api.cu)
int set_error(int code, const char* fmt, ...);

// api.cu: the common part of grid creation (sizes, bbox, kr in FP32 and FP64,
// face planes of the nx x ny x nz lattice, events, capture stream)
int grid_init(skirt_grid_s* g, int nx, int ny, int nz, long long ncell, const double bbox[6], const float* kr);
int check_bbox(const double* bbox);  // finite, non-empty along every axis
int check_device();                  // a CUDA device is present

}  // namespace skirt

// The grid handle: the dust densities on the device and the scratch memory
// that the calls on this grid reuse.  Not thread-safe: one call at a time.
struct skirt_grid_s {
    int device = 0;
    int sm_count = 0;
    int nx = 0, ny = 0, nz = 0;
    long long ncell = 0;
    double bbox[6] = {0, 0, 0, 0, 0, 0};
    float* kr32 = nullptr;
    double* kr64 = nullptr;
    float2* faces = nullptr;  // exact face planes as (hi, lo) FP32 pairs, x then y then z
    skirt::DevBuf scratch;  // per-call tables, accumulators, work queue
    skirt::DevBuf stage;    // device images of host outputs
    skirt::DevBuf cdf;      // dust source: [nlambda][ncell] cumulative distributions
    skirt::DevBuf cdf_aux;  // dust source: tile sums and totals
    skirt::DevBuf abs_lmajor;  // wavelength-major absorbed table of the current call
    int oct_levels = 0;              // octree grid: finest lattice 2^oct_levels per axis
    long long oct_nnode = 0;
    skirt::OctNode* oct_nodes = nullptr;
    int4* oct_leaf = nullptr;        // per leaf: lattice corner and level
    skirt::PinnedBuf pinned;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
};

struct skirt_mlp_s;

namespace skirt {
// mlp.cu: tensor-core inference of the emission surrogate (stream-ordered, no sync)
int mlp_forward_internal(skirt_mlp_s* net, const float* features, const double* total, long long n,
                         double* emission, unsigned char* flags, cudaStream_t s);
// after the stream has synchronised: INVALID (CUDA) when an inference launch
// gave up waiting for a feature copy
int mlp_check_timeout();
// the network's working tables for skirt_dust_emission (at least `bytes`,
// 256-byte aligned); the caller holds mlp_workspace_mutex(net) while it uses them
std::mutex& mlp_workspace_mutex(skirt_mlp_s* net);
int mlp_workspace(skirt_mlp_s* net, size_t bytes, void** p);
// emission.cu: exact FP64 emission of rows (all rows when rows == NULL); a
// second absorbed table [ncell][n2] with its shares (NULL: none) adds its power
int launch_exact_emission(const double* absorbed, int n_in, const double* w_dev, const float* mass,
                          const unsigned* rows, long long nrows, double* emission, float* temperature,
                          cudaStream_t s, const double* absorbed2 = nullptr, int n2 = 0,
                          const double* w2_dev = nullptr);
// dust_source.cu: per-wavelength cumulative distribution of emission[cell][lambda]
// over the cells, normalised to 1, into grid->cdf; the per-wavelength totals
// into *totals_out (may be NULL).  INVALID_ARG when a wavelength with packets
// has no (or non-finite / negative) emission.
int build_dust_cdf(skirt_grid_s* g, const double* emission, int nlambda, const uint64_t* npk, cudaStream_t s,
                   std::vector<double>* totals_out);
}  // namespace skirt
