// C ABI of libskirt: argument validation, the grid handle and its scratch
// memory, parameter upload, launch of the trace kernels (optionally recorded
// once in a CUDA graph and replayed), SED finalisation and the energy ledger.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "skirt_internal.cuh"

using namespace skirt;

namespace skirt {

thread_local std::string g_err;

int set_error(int code, const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace skirt

namespace {

#define fail skirt::set_error

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? SKIRT_ERR_OOM : SKIRT_ERR_CUDA,            \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device pointers (or managed) can be handed to kernels; anything else is a
// host buffer that is staged.
bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

constexpr double kPi = 3.14159265358979323846;

}  // namespace

namespace {

struct Layout {
    size_t kscale, albedo, g, L0, kscale_f, albedo_f, g_f, L0_f, offsets, first, ins, ledger, oof, counters, err, queue, total;
    size_t zero_begin, zero_bytes;  // accumulators zeroed every call
};

Layout make_layout(int NL, int ninstr)
{
    Layout l{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    l.kscale = take(sizeof(double) * NL);
    l.albedo = take(sizeof(double) * NL);
    l.g = take(sizeof(double) * NL);
    l.L0 = take(sizeof(double) * NL);
    l.kscale_f = take(sizeof(float) * NL);
    l.albedo_f = take(sizeof(float) * NL);
    l.g_f = take(sizeof(float) * NL);
    l.L0_f = take(sizeof(float) * NL);
    l.offsets = take(sizeof(unsigned long long) * (NL + 1));
    l.first = take(sizeof(unsigned long long) * NL);
    l.ins = take(sizeof(InstrDev) * (ninstr > 0 ? ninstr : 1));
    l.ledger = take(sizeof(double) * 4 * NL);
    l.oof = take(sizeof(double) * (size_t)(ninstr > 0 ? ninstr : 1) * NL);
    l.counters = take(sizeof(unsigned long long) * 4);
    l.err = take(sizeof(unsigned int));
    l.queue = take(sizeof(unsigned long long));
    l.total = o;
    l.zero_begin = l.ledger;
    l.zero_bytes = o - l.ledger;
    return l;
}

void fill_instrument(const skirt_instrument& s, InstrDev& d, long long img_off)
{
    const double inc = s.inclination_deg * kPi / 180.0, az = s.azimuth_deg * kPi / 180.0;
    const double k[3] = {sin(inc) * cos(az), sin(inc) * sin(az), cos(inc)};
    const double e1[3] = {-sin(az), cos(az), 0.0};
    const double e2[3] = {k[1] * e1[2] - k[2] * e1[1], k[2] * e1[0] - k[0] * e1[2], k[0] * e1[1] - k[1] * e1[0]};
    for (int a = 0; a < 3; ++a) {
        d.kobs[a] = k[a];
        d.e1[a] = e1[a];
        d.e2[a] = e2[a];
        d.kobs_f[a] = (float)k[a];
        d.e1_f[a] = (float)e1[a];
        d.e2_f[a] = (float)e2[a];
    }
    d.half_fov = 0.5 * s.fov;
    d.inv_dpx = (double)s.npx / s.fov;
    d.half_fov_f = (float)d.half_fov;
    d.inv_dpx_f = (float)d.inv_dpx;
    d.flux_norm = 1.0 / (4.0 * kPi * s.distance * s.distance);
    d.flux_norm_f = (float)d.flux_norm;
    d.npx = s.npx;
    d.img_off = img_off;
}

bool finite_all(const double* v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

// ------------------------------------------------------------------------ misc
extern "C" const char* skirt_last_error(void) { return g_err.c_str(); }
extern "C" const char* skirt_version(void) { return "skirt-gb300 0.1 (sm_103a)"; }

extern "C" int skirt_trace_opts_default(skirt_trace_opts* o)
{
    if (!o) return fail(SKIRT_ERR_INVALID_ARG, "opts is NULL");
    std::memset(o, 0, sizeof *o);
    o->precision = SKIRT_PREC_MIXED;
    o->schedule = SKIRT_SCHED_PERSISTENT;
    o->w_min = 1e-4;
    o->max_events = 10000;
    o->peel = 1;
    o->block = 256;
    o->chunk = 4;
    return SKIRT_OK;
}

// ------------------------------------------------------------------------ grid
namespace skirt {

int grid_init(skirt_grid_s* g, int nx, int ny, int nz, long long ncell, const double bbox[6], const float* kr)
{
    cudaError_t e;
    if ((e = cudaGetDevice(&g->device)) != cudaSuccess) return fail(SKIRT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    g->nx = nx; g->ny = ny; g->nz = nz; g->ncell = ncell;
    std::memcpy(g->bbox, bbox, sizeof g->bbox);
    if ((e = cudaMalloc(&g->kr32, sizeof(float) * ncell)) != cudaSuccess) return fail(SKIRT_ERR_OOM, "kr32: %s", cudaGetErrorString(e));
    if ((e = cudaMalloc(&g->kr64, sizeof(double) * ncell)) != cudaSuccess) return fail(SKIRT_ERR_OOM, "kr64: %s", cudaGetErrorString(e));
    {
        // face planes lo + k d (k < n) and the upper bound, split into (hi, lo) FP32 pairs
        std::vector<float2> f;
        const int nn[3] = {nx, ny, nz};
        for (int a = 0; a < 3; ++a) {
            const double lo = bbox[2 * a], hi = bbox[2 * a + 1], d = (hi - lo) / nn[a];
            for (int k = 0; k <= nn[a]; ++k) {
                const double v = k < nn[a] ? lo + (double)k * d : hi;
                const float h = (float)v;
                f.push_back(make_float2(h, (float)(v - (double)h)));
            }
        }
        if ((e = cudaMalloc(&g->faces, sizeof(float2) * f.size())) != cudaSuccess)
            return fail(SKIRT_ERR_OOM, "faces: %s", cudaGetErrorString(e));
        if ((e = cudaMemcpy(g->faces, f.data(), sizeof(float2) * f.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(SKIRT_ERR_CUDA, "faces: %s", cudaGetErrorString(e));
    }
    if ((e = cudaEventCreate(&g->ev0)) != cudaSuccess || (e = cudaEventCreate(&g->ev1)) != cudaSuccess)
        return fail(SKIRT_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    if ((e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(SKIRT_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpy(g->kr32, kr, sizeof(float) * ncell, cudaMemcpyDefault)) != cudaSuccess)
        return fail(SKIRT_ERR_CUDA, "copy kr: %s", cudaGetErrorString(e));
    if ((e = g->scratch.ensure(256)) != cudaSuccess) return fail(SKIRT_ERR_OOM, "scratch: %s", cudaGetErrorString(e));
    unsigned int* bad_d = (unsigned int*)g->scratch.p;
    unsigned int bad = 0;
    if ((e = cudaMemset(bad_d, 0, sizeof(unsigned int))) != cudaSuccess ||
        (e = launch_f32_to_f64(g->kr32, g->kr64, ncell, bad_d, 0)) != cudaSuccess ||
        (e = cudaMemcpy(&bad, bad_d, sizeof bad, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(SKIRT_ERR_CUDA, "convert kr: %s", cudaGetErrorString(e));
    if (bad) return fail(SKIRT_ERR_INVALID_ARG, "kr holds negative or non-finite values");
    return SKIRT_OK;
}

int check_bbox(const double* bbox)
{
    if (!finite_all(bbox, 6)) return fail(SKIRT_ERR_INVALID_ARG, "bbox must be finite");
    for (int a = 0; a < 3; ++a)
        if (!(bbox[2 * a] < bbox[2 * a + 1])) return fail(SKIRT_ERR_INVALID_ARG, "bbox axis %d is empty", a);
    return SKIRT_OK;
}

int check_device()
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SKIRT_ERR_NO_DEVICE, "no CUDA device");
    }
    return SKIRT_OK;
}

}  // namespace skirt

extern "C" int skirt_grid_create(skirt_grid_t* out, int nx, int ny, int nz, const double bbox[6], const float* kr)
{
    if (!out) return fail(SKIRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(SKIRT_ERR_INVALID_ARG, "grid sizes must be >= 1");
    const long long ncell = (long long)nx * ny * nz;
    if (ncell >= (1ll << 31)) return fail(SKIRT_ERR_INVALID_ARG, "ncell must be < 2^31");
    if (!bbox || !kr) return fail(SKIRT_ERR_INVALID_ARG, "bbox / kr is NULL");
    if (int r = check_bbox(bbox)) return r;
    if (int r = check_device()) return r;
    skirt_grid_s* g = new skirt_grid_s;
    if (int r = grid_init(g, nx, ny, nz, ncell, bbox, kr)) {
        skirt_grid_destroy(g);
        return r;
    }
    *out = g;
    return SKIRT_OK;
}

extern "C" int skirt_emission_totals(skirt_grid_t g, const double* emission, int nlambda, double* totals,
                                     void* stream)
{
    if (!g || !emission || !totals) return fail(SKIRT_ERR_INVALID_ARG, "grid / emission / totals is NULL");
    if (nlambda < 1 || nlambda > 65536) return fail(SKIRT_ERR_INVALID_ARG, "nlambda %d out of range", nlambda);
    if (!is_device_ptr(emission)) return fail(SKIRT_ERR_INVALID_ARG, "emission must be device memory");
    const std::vector<uint64_t> none((size_t)nlambda, 0);
    std::vector<double> t;
    if (int r = build_dust_cdf(g, emission, nlambda, none.data(), (cudaStream_t)stream, &t)) return r;
    std::memcpy(totals, t.data(), sizeof(double) * (size_t)nlambda);
    return SKIRT_OK;
}

extern "C" int skirt_grid_destroy(skirt_grid_t g)
{
    if (!g) return SKIRT_OK;
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->kr32) cudaFree(g->kr32);
    if (g->kr64) cudaFree(g->kr64);
    if (g->faces) cudaFree(g->faces);
    if (g->oct_nodes) cudaFree(g->oct_nodes);
    if (g->oct_leaf) cudaFree(g->oct_leaf);
    g->scratch.release();
    g->stage.release();
    g->cdf.release();
    g->cdf_aux.release();
    g->abs_lmajor.release();
    g->pinned.release();
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    delete g;
    return SKIRT_OK;
}

// ------------------------------------------------------------------------ trace
namespace {

struct Prepared {
    int NL = 0, ninstr = 0;
    std::vector<int> npx;
    long long img_elems = 0;
    unsigned long long total = 0;
    std::vector<unsigned long long> offsets;
    Layout lay{};
};

int validate(skirt_grid_t g, const skirt_source* src, const skirt_wavelengths* wl, const uint64_t* npk,
             const skirt_instrument* ins, int ninstr, const skirt_trace_opts* opts, Prepared& P)
{
    if (!g) return fail(SKIRT_ERR_INVALID_ARG, "grid is NULL");
    if (!src || !wl || !npk || !opts) return fail(SKIRT_ERR_INVALID_ARG, "src / wl / npackets / opts is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return fail(SKIRT_ERR_NO_DEVICE, "grid lives on device %d, current device is %d", g->device, dev);
    if (wl->n < 1 || wl->n > 65536) return fail(SKIRT_ERR_INVALID_ARG, "wavelength count %d out of range", wl->n);
    if (!wl->kscale || !wl->albedo || !wl->g) return fail(SKIRT_ERR_INVALID_ARG, "wavelength table is NULL");
    if (!wl->lsrc && src->kind != SKIRT_SRC_DUST)
        return fail(SKIRT_ERR_INVALID_ARG, "lsrc may be NULL only for a dust-cell source");
    if (ninstr < 0 || ninstr > 16) return fail(SKIRT_ERR_INVALID_ARG, "ninstr must be in [0, 16]");
    if (ninstr > 0 && !ins) return fail(SKIRT_ERR_INVALID_ARG, "instruments are NULL");
    P.NL = wl->n;
    P.ninstr = ninstr;
    for (int j = 0; j < P.NL; ++j) {
        if (!std::isfinite(wl->kscale[j]) || wl->kscale[j] < 0) return fail(SKIRT_ERR_INVALID_ARG, "kscale[%d] invalid", j);
        if (!(wl->albedo[j] >= 0 && wl->albedo[j] <= 1)) return fail(SKIRT_ERR_INVALID_ARG, "albedo[%d] not in [0,1]", j);
        if (!(std::fabs(wl->g[j]) < 1)) return fail(SKIRT_ERR_INVALID_ARG, "|g[%d]| must be < 1", j);
        if (wl->lsrc && (!std::isfinite(wl->lsrc[j]) || wl->lsrc[j] < 0))
            return fail(SKIRT_ERR_INVALID_ARG, "lsrc[%d] invalid", j);
        if (npk[j] >= (1ull << 32)) return fail(SKIRT_ERR_INVALID_ARG, "npackets[%d] must be < 2^32", j);
        const uint64_t first = opts && opts->first_packet ? opts->first_packet[j] : 0;
        if (first > (1ull << 32) - npk[j])
            return fail(SKIRT_ERR_INVALID_ARG, "first_packet[%d] + npackets[%d] must not exceed 2^32", j, j);
        if (opts && opts->total_packets) {
            const uint64_t tot = opts->total_packets[j];
            if (tot >= (1ull << 32) || first + npk[j] > tot)
                return fail(SKIRT_ERR_INVALID_ARG,
                            "first_packet[%d] + npackets[%d] must not exceed total_packets[%d] (< 2^32)", j, j, j);
        }
    }
    P.offsets.assign(P.NL + 1, 0);
    for (int j = 0; j < P.NL; ++j) P.offsets[j + 1] = P.offsets[j] + npk[j];
    P.total = P.offsets[P.NL];
    P.npx.resize(ninstr);
    P.img_elems = 0;
    for (int q = 0; q < ninstr; ++q) {
        const skirt_instrument& s = ins[q];
        if (!(s.distance > 0) || !std::isfinite(s.distance)) return fail(SKIRT_ERR_INVALID_ARG, "instrument %d distance", q);
        if (!(s.fov > 0) || !std::isfinite(s.fov)) return fail(SKIRT_ERR_INVALID_ARG, "instrument %d fov", q);
        if (!std::isfinite(s.inclination_deg) || !std::isfinite(s.azimuth_deg))
            return fail(SKIRT_ERR_INVALID_ARG, "instrument %d angles", q);
        if (s.npx < 1 || s.npx > 16384) return fail(SKIRT_ERR_INVALID_ARG, "instrument %d npx", q);
        P.npx[q] = s.npx;
        P.img_elems += (long long)s.npx * s.npx * P.NL;
    }
    switch (src->kind) {
    case SKIRT_SRC_POINT:
    case SKIRT_SRC_BEAM:
    case SKIRT_SRC_DISK:
    case SKIRT_SRC_DUST:
        break;
    default:
        return fail(SKIRT_ERR_INVALID_ARG, "unknown source kind %d", src->kind);
    }
    if (!finite_all(src->pos, 3)) return fail(SKIRT_ERR_INVALID_ARG, "source position");
    if (src->kind != SKIRT_SRC_DUST) {
        for (int a = 0; a < 3; ++a)
            if (!(src->pos[a] >= g->bbox[2 * a] && src->pos[a] <= g->bbox[2 * a + 1]))
                return fail(SKIRT_ERR_INVALID_ARG, "source position outside the grid");
    }
    if (src->kind == SKIRT_SRC_BEAM) {
        if (!finite_all(src->dir, 3)) return fail(SKIRT_ERR_INVALID_ARG, "beam direction");
        const double n2 = src->dir[0] * src->dir[0] + src->dir[1] * src->dir[1] + src->dir[2] * src->dir[2];
        if (std::fabs(n2 - 1.0) > 1e-9) return fail(SKIRT_ERR_INVALID_ARG, "beam direction must be a unit vector");
    }
    if (src->kind == SKIRT_SRC_DISK && !(src->h_R > 0 && src->h_z > 0 && std::isfinite(src->h_R) && std::isfinite(src->h_z)))
        return fail(SKIRT_ERR_INVALID_ARG, "disk scale lengths must be > 0");
    if (src->kind == SKIRT_SRC_DUST && !src->emission) return fail(SKIRT_ERR_INVALID_ARG, "dust source needs emission");
    if (opts->precision != SKIRT_PREC_FP64 && opts->precision != SKIRT_PREC_MIXED)
        return fail(SKIRT_ERR_INVALID_ARG, "unknown precision %d", opts->precision);
    if (opts->schedule != SKIRT_SCHED_PER_LAMBDA && opts->schedule != SKIRT_SCHED_PERSISTENT)
        return fail(SKIRT_ERR_INVALID_ARG, "unknown schedule %d", opts->schedule);
    if (opts->block != 0 && (opts->block < 32 || opts->block % 32 ||
                             opts->block > (opts->precision == SKIRT_PREC_MIXED ? 256 : 512)))
        return fail(SKIRT_ERR_INVALID_ARG, "block must be a multiple of 32 up to 256 (mixed) or 512 (FP64)");
    if (opts->step_min < 0 || opts->step_min > 32) return fail(SKIRT_ERR_INVALID_ARG, "step_min must be in [0, 32]");
    if (opts->chunk < 0 || opts->chunk > (1 << 20)) return fail(SKIRT_ERR_INVALID_ARG, "chunk out of range");
    if (opts->blocks_per_sm < 0 || opts->blocks_per_sm > 64) return fail(SKIRT_ERR_INVALID_ARG, "blocks_per_sm out of range");
    if (opts->phase > 255) return fail(SKIRT_ERR_INVALID_ARG, "phase must be < 256");
    if (opts->nrec < 0) return fail(SKIRT_ERR_INVALID_ARG, "nrec must be >= 0");
    if (opts->nrec > 0 && !opts->records) return fail(SKIRT_ERR_INVALID_ARG, "records is NULL");
    if (!std::isfinite(opts->w_min) || opts->w_min >= 1) return fail(SKIRT_ERR_INVALID_ARG, "w_min must be < 1");
    P.lay = make_layout(P.NL, ninstr);
    return SKIRT_OK;
}

}  // namespace

extern "C" int skirt_trace(skirt_grid_t g, const skirt_source* src, const skirt_wavelengths* wl,
                           const uint64_t* npk, uint64_t seed, const skirt_instrument* ins, int ninstr,
                           const skirt_trace_opts* opts, double* absorbed, double* images, double* sed,
                           skirt_ledger* ledger, double* ledger_per_lambda, void* stream_v)
{
    Prepared P;
    int rc = validate(g, src, wl, npk, ins, ninstr, opts, P);
    if (rc) return rc;
    if (!absorbed) return fail(SKIRT_ERR_INVALID_ARG, "absorbed is NULL");
    if (ninstr > 0 && opts->peel && (!images || !sed)) return fail(SKIRT_ERR_INVALID_ARG, "images / sed is NULL");
    cudaStream_t s = (cudaStream_t)stream_v;
    const int NL = P.NL;
    const Layout& L = P.lay;

    // ---- dust source: per-wavelength cumulative distribution over the cells;
    // its column totals are the source luminosities when lsrc is NULL
    const double* d_cdf = nullptr;
    std::vector<double> dust_totals;
    if (src->kind == SKIRT_SRC_DUST) {
        int r = build_dust_cdf(g, src->emission, NL, npk, s, &dust_totals);
        if (r) return r;
        d_cdf = (const double*)g->cdf.p;
    }
    const double* lsrc = wl->lsrc ? wl->lsrc : dust_totals.data();

    // ---- host staging: parameter tables and read-back area
    const size_t rb_ledger = sizeof(double) * 4 * NL, rb_counters = sizeof(unsigned long long) * 4;
    const size_t pinned_bytes = L.total + rb_ledger + rb_counters + 64;
    CK(g->pinned.ensure(pinned_bytes));
    CK(g->scratch.ensure(L.total));
    unsigned char* hp = (unsigned char*)g->pinned.p;
    unsigned char* dp = (unsigned char*)g->scratch.p;
    double* h_ks = (double*)(hp + L.kscale);
    double* h_al = (double*)(hp + L.albedo);
    double* h_g = (double*)(hp + L.g);
    double* h_L0 = (double*)(hp + L.L0);
    float* h_ksf = (float*)(hp + L.kscale_f);
    float* h_alf = (float*)(hp + L.albedo_f);
    float* h_gf = (float*)(hp + L.g_f);
    float* h_L0f = (float*)(hp + L.L0_f);
    for (int j = 0; j < NL; ++j) {
        h_ks[j] = wl->kscale[j];
        h_al[j] = wl->albedo[j];
        h_g[j] = wl->g[j];
        const uint64_t ntot = opts->total_packets ? opts->total_packets[j] : npk[j];
        h_L0[j] = npk[j] ? lsrc[j] / (double)ntot : 0.0;
        h_ksf[j] = (float)h_ks[j];
        h_alf[j] = (float)h_al[j];
        h_gf[j] = (float)h_g[j];
        h_L0f[j] = (float)h_L0[j];
    }
    std::memcpy(hp + L.offsets, P.offsets.data(), sizeof(unsigned long long) * (NL + 1));
    {
        unsigned long long* h_first = (unsigned long long*)(hp + L.first);
        for (int j = 0; j < NL; ++j) h_first[j] = opts->first_packet ? opts->first_packet[j] : 0;
    }
    InstrDev* h_ins = (InstrDev*)(hp + L.ins);
    {
        long long off = 0;
        for (int q = 0; q < ninstr; ++q) {
            std::memset(&h_ins[q], 0, sizeof(InstrDev));
            fill_instrument(ins[q], h_ins[q], off);
            off += (long long)ins[q].npx * ins[q].npx * NL;
        }
    }
    CK(cudaMemcpyAsync(dp, hp, L.zero_begin, cudaMemcpyHostToDevice, s));

    // ---- outputs: device pointers are used in place, host ones are staged
    const size_t abs_bytes = sizeof(double) * (size_t)g->ncell * NL;
    const size_t img_bytes = sizeof(double) * (size_t)P.img_elems;
    const size_t sed_bytes = sizeof(double) * (size_t)ninstr * NL;
    const size_t rec_bytes = sizeof(double) * (size_t)NL * opts->nrec * SKIRT_REC_FIELDS;
    const bool peel = opts->peel && ninstr > 0;
    const bool abs_dev = is_device_ptr(absorbed);
    const bool img_dev = !peel || is_device_ptr(images);
    const bool sed_dev = !peel || is_device_ptr(sed);
    const bool rec_dev = opts->nrec == 0 || is_device_ptr(opts->records);
    size_t st_abs = 0, st_img = 0, st_sed = 0, st_rec = 0, st_total = 0;
    if (!abs_dev) { st_abs = st_total; st_total = align_up(st_total + abs_bytes, 256); }
    if (!img_dev) { st_img = st_total; st_total = align_up(st_total + img_bytes, 256); }
    if (!sed_dev) { st_sed = st_total; st_total = align_up(st_total + sed_bytes, 256); }
    if (!rec_dev) { st_rec = st_total; st_total = align_up(st_total + rec_bytes, 256); }
    if (st_total) CK(g->stage.ensure(st_total));
    unsigned char* sp = (unsigned char*)g->stage.p;
    double* d_abs = abs_dev ? absorbed : (double*)(sp + st_abs);
    double* d_img = !peel ? nullptr : (img_dev ? images : (double*)(sp + st_img));
    double* d_sed = !peel ? nullptr : (sed_dev ? sed : (double*)(sp + st_sed));
    double* d_rec = opts->nrec == 0 ? nullptr : (rec_dev ? opts->records : (double*)(sp + st_rec));
    if (opts->accumulate) {
        if (!abs_dev) CK(cudaMemcpyAsync(d_abs, absorbed, abs_bytes, cudaMemcpyHostToDevice, s));
        if (peel && !img_dev) CK(cudaMemcpyAsync(d_img, images, img_bytes, cudaMemcpyHostToDevice, s));
        if (peel && !sed_dev) CK(cudaMemcpyAsync(d_sed, sed, sed_bytes, cudaMemcpyHostToDevice, s));
    }


    // ---- kernel arguments
    TraceArgs A;
    std::memset(&A, 0, sizeof A);
    A.kr32 = g->kr32;
    A.kr64 = g->kr64;
    A.nx = g->nx; A.ny = g->ny; A.nz = g->nz;
    A.ncell = g->ncell;
    A.oct_levels = g->oct_levels;
    A.oct_nodes = g->oct_nodes;
    A.oct_leaf = g->oct_leaf;
    A.oct_step_cap = g->nx + g->ny + g->nz + 8;
    // the mixed form's optical-depth cut-off; SKIRT_MIXED_TAU_CUT (a value above
    // 30, e.g. 1e30 for none) moves it: a diagnostic showing that the cut
    // changes no packet history
    A.tau_cut = 30.f;
    if (const char* e = std::getenv("SKIRT_MIXED_TAU_CUT")) {
        const float v = std::strtof(e, nullptr);
        if (v > 30.f) A.tau_cut = v;
    }
    const int nn[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        A.lo[a] = g->bbox[2 * a];
        A.hi[a] = g->bbox[2 * a + 1];
        A.d[a] = (A.hi[a] - A.lo[a]) / (double)nn[a];
    }
    A.nlambda = NL;
    A.kscale = (const double*)(dp + L.kscale);
    A.albedo = (const double*)(dp + L.albedo);
    A.g = (const double*)(dp + L.g);
    A.L0 = (const double*)(dp + L.L0);
    A.kscale_f = (const float*)(dp + L.kscale_f);
    A.albedo_f = (const float*)(dp + L.albedo_f);
    A.g_f = (const float*)(dp + L.g_f);
    A.L0_f = (const float*)(dp + L.L0_f);
    A.faces = g->faces;
    for (int a = 0; a < 3; ++a) {
        const float hi = (float)src->pos[a];
        A.src_df[a] = make_float2(hi, (float)(src->pos[a] - (double)hi));
        A.src_dir_f[a] = (float)src->dir[a];
        A.hi_f[a] = (float)g->bbox[2 * a + 1];
    }
    A.offsets = (const unsigned long long*)(dp + L.offsets);
    A.pk_first = (const unsigned long long*)(dp + L.first);
    A.total = P.total;
    A.src_kind = src->kind;
    for (int a = 0; a < 3; ++a) {
        A.src_pos[a] = src->pos[a];
        A.src_dir[a] = src->dir[a];
    }
    A.h_R = src->h_R;
    A.h_z = src->h_z;
    A.cdf = d_cdf;
    A.ninstr = peel ? ninstr : 0;
    A.ins = (const InstrDev*)(dp + L.ins);
    // With more than one wavelength the packets deposit into a wavelength-major
    // table (consecutive cells of a wavelength adjacent, as the traversals
    // visit them) and one transpose writes the [cell][lambda] result (the
    // counterpart of the paper's column-to-row representation switch,
    // Sect. 5.2); without room for that table they deposit in place.
    bool lmajor = NL > 1;
    double* d_acc = d_abs;
    if (lmajor) {
        if (g->abs_lmajor.ensure(abs_bytes) == cudaSuccess) {
            d_acc = (double*)g->abs_lmajor.p;
        } else {
            cudaGetLastError();
            lmajor = false;
        }
    }
    A.absorbed = d_acc;
    A.abs_cs = lmajor ? 1 : NL;
    A.abs_ls = lmajor ? g->ncell : 1;
    A.images = d_img;
    A.oof = (double*)(dp + L.oof);
    A.ledger = (double*)(dp + L.ledger);
    A.counters = (unsigned long long*)(dp + L.counters);
    A.err = (unsigned int*)(dp + L.err);
    A.nrec = opts->nrec;
    A.records = d_rec;
    A.w_min = opts->w_min > 0 ? opts->w_min : 1e-4;
    A.w_min_f = (float)A.w_min;
    A.max_events = opts->max_events > 0 ? opts->max_events : 10000;
    A.peel = peel ? 1 : 0;
    A.key0 = (uint32_t)(seed & 0xffffffffu);
    A.key1 = (uint32_t)(seed >> 32);
    A.phase = opts->phase;
    A.queue = (unsigned long long*)(dp + L.queue);
    A.chunk = opts->chunk > 0 ? opts->chunk : 4;
    A.step_min = opts->step_min > 0 ? opts->step_min : 20;

    const int block = opts->block > 0 ? opts->block : 256;
    int bps = opts->blocks_per_sm;
    if (bps <= 0) {
        CK(trace_occupancy(opts->precision, block, &bps, g->oct_levels > 0));
        if (bps < 1) bps = 1;
    }
    const int pgrid = g->sm_count * bps;
    if (opts->precision == SKIRT_PREC_FP64 && trace_smem_bytes(A.ninstr, block) > 48 * 1024)
        return fail(SKIRT_ERR_INVALID_ARG, "block too large for the shared-memory budget");

    // ---- the device work of one call (recorded into a graph when asked)
    auto enqueue = [&](cudaStream_t s, bool events) -> int {
        if (lmajor) CK(cudaMemsetAsync(d_acc, 0, abs_bytes, s));
        if (!opts->accumulate) {
            if (!lmajor) CK(cudaMemsetAsync(d_abs, 0, abs_bytes, s));
            if (peel) {
                CK(cudaMemsetAsync(d_img, 0, img_bytes, s));
                CK(cudaMemsetAsync(d_sed, 0, sed_bytes, s));
            }
        } else if (peel) {
            // remove the images' previous content from the SED so that the
            // finalisation below adds only this call's peel-offs
            CK(launch_sed_finalize(d_img, nullptr, d_sed, ninstr, P.npx.data(), NL, -1.0, s));
        }
        if (d_rec && rec_bytes) CK(cudaMemsetAsync(d_rec, 0, rec_bytes, s));
        CK(cudaMemsetAsync(dp + L.zero_begin, 0, L.zero_bytes, s));
        CK(events ? cudaEventRecord(g->ev0, s) : cudaEventRecordWithFlags(g->ev0, s, cudaEventRecordExternal));
        if (P.total > 0) {
            if (opts->schedule == SKIRT_SCHED_PERSISTENT) {
                A.persistent = 1;
                CK(launch_trace(A, opts->precision, block, pgrid, s));
            } else {
                for (int j = 0; j < NL; ++j) {
                    if (!npk[j]) continue;
                    TraceArgs Aj = A;
                    Aj.persistent = 0;
                    Aj.q_base = P.offsets[j];
                    Aj.q_count = npk[j];
                    const unsigned long long nb = (npk[j] + block - 1) / block;
                    CK(launch_trace(Aj, opts->precision, block, (int)nb, s));
                }
            }
        }
        CK(events ? cudaEventRecord(g->ev1, s) : cudaEventRecordWithFlags(g->ev1, s, cudaEventRecordExternal));
        if (lmajor) CK(launch_transpose_absorbed(d_acc, d_abs, g->ncell, NL, opts->accumulate != 0, s));
        if (peel) CK(launch_sed_finalize(d_img, A.oof, d_sed, ninstr, P.npx.data(), NL, 1.0, s));
        return SKIRT_OK;
    };

    if (opts->use_graph) {
        // key: everything the recorded work depends on
        std::vector<unsigned char> key;
        auto put = [&](const void* p, size_t n) {
            const unsigned char* c = (const unsigned char*)p;
            key.insert(key.end(), c, c + n);
        };
        int ints[8] = {opts->precision, opts->schedule, block, pgrid, opts->accumulate, opts->nrec, ninstr, NL};
        put(ints, sizeof ints);
        put(&A, sizeof A);
        put(&s, sizeof s);
        // output pointers the recorded work writes outside A: the transpose's
        // destination (the caller's table, or its staging area) and the SEDs
        put(&d_abs, sizeof d_abs);
        put(&d_img, sizeof d_img);
        put(&d_sed, sizeof d_sed);
        put(npk, sizeof(uint64_t) * NL);
        put(P.npx.data(), sizeof(int) * ninstr);
        if (!g->gexec || key != g->gkey) {
            if (g->gexec) {
                cudaGraphExecDestroy(g->gexec);
                g->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(g->capture_stream, cudaStreamCaptureModeThreadLocal));
            int r = enqueue(g->capture_stream, false);
            cudaError_t e = cudaStreamEndCapture(g->capture_stream, &graph);
            if (r) {
                if (graph) cudaGraphDestroy(graph);
                return r;
            }
            if (e != cudaSuccess) return fail(SKIRT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&g->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                g->gexec = nullptr;
                return fail(SKIRT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
            g->gkey = key;
        }
        CK(cudaGraphLaunch(g->gexec, s));
    } else {
        int r = enqueue(s, true);
        if (r) return r;
    }

    // ---- read back
    unsigned char* rb = hp + align_up(L.total, 64);
    CK(cudaMemcpyAsync(rb, dp + L.ledger, rb_ledger, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rb + rb_ledger, dp + L.counters, rb_counters, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rb + rb_ledger + rb_counters, dp + L.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    if (!abs_dev) CK(cudaMemcpyAsync(absorbed, d_abs, abs_bytes, cudaMemcpyDeviceToHost, s));
    if (peel && !img_dev) CK(cudaMemcpyAsync(images, d_img, img_bytes, cudaMemcpyDeviceToHost, s));
    if (peel && !sed_dev) CK(cudaMemcpyAsync(sed, d_sed, sed_bytes, cudaMemcpyDeviceToHost, s));
    if (d_rec && !rec_dev) CK(cudaMemcpyAsync(opts->records, d_rec, rec_bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    const double* led = (const double*)rb;
    const unsigned long long* cnt = (const unsigned long long*)(rb + rb_ledger);
    const unsigned int errbits = *(const unsigned int*)(rb + rb_ledger + rb_counters);
    if (ledger_per_lambda) std::memcpy(ledger_per_lambda, led, rb_ledger);
    if (ledger) {
        std::memset(ledger, 0, sizeof *ledger);
        for (int j = 0; j < NL; ++j) {
            ledger->emitted += led[4 * j + 0];
            ledger->absorbed += led[4 * j + 1];
            ledger->escaped += led[4 * j + 2];
            ledger->residual += led[4 * j + 3];
        }
        ledger->scatterings = (double)cnt[0];
        ledger->deposit_steps = (double)cnt[1];
        ledger->locate_steps = (double)cnt[2];
        ledger->peel_steps = (double)cnt[3];
        ledger->status_bits = (int)errbits;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev0, g->ev1) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.f;
        }
        ledger->kernel_ms = ms;
    }
    if (errbits & ERRBIT_NONFINITE) return fail(SKIRT_ERR_NONFINITE, "non-finite value in a packet's bookkeeping");
    if (errbits & ERRBIT_PATH)
        return fail(SKIRT_ERR_NONFINITE, "an octree traversal exceeded its crossing bound and was abandoned");
    if (errbits & ERRBIT_SOURCE) return fail(SKIRT_ERR_SOURCE, "a source position could not be placed in the grid");
    if (errbits & ERRBIT_EVENT_CAP) return fail(SKIRT_ERR_EVENT_CAP, "a packet reached max_events");
    g_err.clear();
    return SKIRT_OK;
}

// ------------------------------------------------------------------------ autotune
extern "C" int skirt_autotune(skirt_grid_t g, const skirt_source* src, const skirt_wavelengths* wl,
                              const uint64_t* npk, uint64_t seed, const skirt_instrument* ins, int ninstr,
                              skirt_trace_opts* opts, double frac, int repeats, double* absorbed, double* images,
                              double* sed, skirt_tune_report* report, void* stream)
{
    if (!g || !opts || !wl || !npk) return fail(SKIRT_ERR_INVALID_ARG, "grid / opts / wl / npackets is NULL");
    if (!(frac > 0 && frac <= 1)) return fail(SKIRT_ERR_INVALID_ARG, "sample_fraction must be in (0, 1]");
    if (wl->n < 1 || wl->n > 65536) return fail(SKIRT_ERR_INVALID_ARG, "wavelength count %d out of range", wl->n);
    if (repeats <= 0) repeats = 2;
    if (repeats > 16) return fail(SKIRT_ERR_INVALID_ARG, "repeats must be <= 16");
    auto make_sample = [&](double f, std::vector<uint64_t>& smp) {
        unsigned long long tot = 0;
        smp.assign(wl->n, 0);
        for (int j = 0; j < wl->n; ++j) {
            uint64_t n = (uint64_t)std::llround((double)npk[j] * f);
            smp[j] = (npk[j] > 0 && n == 0) ? 1 : n;
            tot += smp[j];
        }
        return tot;
    };
    std::vector<uint64_t> sample, confirm;
    const unsigned long long nsample = make_sample(frac, sample);
    const unsigned long long nconfirm = make_sample(std::min(1.0, 5.0 * frac), confirm);
    skirt_trace_opts o = *opts;
    o.schedule = SKIRT_SCHED_PERSISTENT;
    o.use_graph = 0;
    o.accumulate = 0;
    o.nrec = 0;
    o.records = nullptr;
    o.first_packet = nullptr;
    o.total_packets = nullptr;
    const bool mixed = o.precision == SKIRT_PREC_MIXED;
    const bool oct = g->oct_levels > 0;

    // the candidates: the requested schedule (defaults resolved), then the sweep
    std::vector<skirt_tune_point> cand;
    {
        skirt_tune_point p{};
        p.block = o.block > 0 ? o.block : 256;
        p.chunk = o.chunk > 0 ? o.chunk : 4;
        p.step_min = o.step_min > 0 ? o.step_min : 20;
        int maxbps = 0;
        CK(trace_occupancy(o.precision, p.block, &maxbps, oct));
        p.blocks_per_sm = o.blocks_per_sm > 0 ? o.blocks_per_sm : (maxbps > 0 ? maxbps : 1);
        cand.push_back(p);
    }
    const int blocks[4] = {64, 128, 256, 512};
    const int chunks[3] = {1, 4, 16};
    const int step_mins[3] = {16, 20, 24};
    for (int bi = 0; bi < (mixed ? 3 : 4); ++bi) {
        int maxbps = 0;
        CK(trace_occupancy(o.precision, blocks[bi], &maxbps, oct));
        if (maxbps < 1) continue;
        for (int ci = 0; ci < 3; ++ci)
            for (int si = 0; si < (mixed ? 3 : 1); ++si)
                for (int bps = maxbps; bps >= 1; bps = (bps > 1 ? (bps + 1) / 2 : 0)) {
                    skirt_tune_point p{blocks[bi], chunks[ci], bps, mixed ? step_mins[si] : 20, 0.f, 0.f};
                    const skirt_tune_point& d = cand[0];
                    const bool same = p.block == d.block && p.chunk == d.chunk && p.blocks_per_sm == d.blocks_per_sm &&
                                      (!mixed || p.step_min == d.step_min);
                    if (!same && (int)cand.size() < SKIRT_TUNE_MAX_POINTS) cand.push_back(p);
                    if (bps == 1) break;
                }
    }
    auto run = [&](const skirt_tune_point& p, float* ms, const std::vector<uint64_t>& smp) -> int {
        o.block = p.block;
        o.chunk = p.chunk;
        o.blocks_per_sm = p.blocks_per_sm;
        o.step_min = p.step_min;
        skirt_ledger led;
        int r = skirt_trace(g, src, wl, smp.data(), seed, ins, ninstr, &o, absorbed, images, sed, &led, nullptr,
                            stream);
        if (r && r != SKIRT_ERR_EVENT_CAP) return r;
        *ms = led.kernel_ms > 0 ? led.kernel_ms : 1e30f;
        return SKIRT_OK;
    };
    float warm = 0.f;
    if (int r = run(cand[0], &warm, sample)) return r;
    for (auto& p : cand) {
        p.ms = 1e30f;
        p.ms_confirm = 0.f;
        for (int k = 0; k < repeats; ++k) {
            float ms = 0.f;
            if (int r = run(p, &ms, sample)) return r;
            if (ms < p.ms) p.ms = ms;
        }
    }
    // the three fastest and the requested schedule, again on the larger sample
    std::vector<int> order(cand.size());
    for (size_t i = 0; i < cand.size(); ++i) order[i] = (int)i;
    std::sort(order.begin() + 1, order.end(), [&](int a, int b) { return cand[a].ms < cand[b].ms; });
    const int nconf = std::min<int>(4, (int)cand.size());
    if (int r = run(cand[0], &warm, confirm)) return r;  // warm-up at the larger size
    for (int q = 0; q < nconf; ++q) {
        float ms = 0.f;
        if (int r = run(cand[order[q]], &ms, confirm)) return r;
        cand[order[q]].ms_confirm = ms;
    }
    int best = 0;
    for (int q = 1; q < nconf; ++q)
        if (cand[order[q]].ms_confirm < cand[best].ms_confirm) best = order[q];
    const int chosen = cand[best].ms_confirm < 0.98f * cand[0].ms_confirm ? best : 0;
    opts->block = cand[chosen].block;
    opts->chunk = cand[chosen].chunk;
    opts->blocks_per_sm = cand[chosen].blocks_per_sm;
    if (mixed) opts->step_min = cand[chosen].step_min;
    if (report) {
        std::memset(report, 0, sizeof *report);
        report->n = (int)cand.size();
        report->chosen = chosen;
        report->repeats = repeats;
        report->sample_packets = nsample;
        report->confirm_packets = nconfirm;
        for (size_t i = 0; i < cand.size(); ++i) report->points[i] = cand[i];
    }
    // leave the outputs zeroed
    skirt_trace_opts z = o;
    std::vector<uint64_t> none(wl->n, 0);
    return skirt_trace(g, src, wl, none.data(), seed, ins, ninstr, &z, absorbed, images, sed, nullptr, nullptr, stream);
}
