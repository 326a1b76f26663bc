// Octree dust grid (arXiv:1705.04702, Sect. 7.9: the ERIS run uses an
// octree grid with up to 13 division levels and 8.2 million cells).
//
// The caller lists the leaves (level and integer position at that level);
// the host inserts them from the root down into a node array (children of a
// node are 8 consecutive nodes) and checks that they tile the root box; a
// kernel then finds, for every leaf and each of its 6 faces, the node across
// that face: the node of the same level if the tree has one, else the leaf
// of a larger size that covers it.  A traversal (trace.cu) crosses a face by
// reading that neighbour and, when the neighbour is split further, descending
// from it by the finest-lattice cell of the entry point.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "skirt_internal.cuh"

namespace skirt {
namespace {

// One thread per leaf: the neighbour across each face, found by descending
// from the root towards the same-level box on the other side, stopping at a
// leaf (a larger one covers that box) or at the same level.
__global__ void oct_neighbours_kernel(OctNode* nodes, const int4* leaf, const int* leaf_node, long long nleaf,
                                      int levels)
{
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nleaf;
         m += (long long)gridDim.x * blockDim.x) {
        const int4 lf = leaf[m];
        const int lev = lf.w, sh = levels - lev;
        const int c[3] = {lf.x >> sh, lf.y >> sh, lf.z >> sh};
        const int n = 1 << lev;
        int nb[6];
        for (int f = 0; f < 6; ++f) {
            int q[3] = {c[0], c[1], c[2]};
            q[f >> 1] += (f & 1) ? 1 : -1;
            int node = -1;
            if (q[f >> 1] >= 0 && q[f >> 1] < n) {
                node = 0;
                for (int d = 0; d < lev; ++d) {
                    const int r = nodes[node].ref;
                    if (r < 0) break;
                    const int b = lev - 1 - d;
                    node = r + (((q[0] >> b) & 1) | (((q[1] >> b) & 1) << 1) | (((q[2] >> b) & 1) << 2));
                }
            }
            nb[f] = node;
        }
        OctNode* me = nodes + leaf_node[m];
        for (int f = 0; f < 6; ++f) me->nb[f] = nb[f];
    }
}

}  // namespace
}  // namespace skirt

using namespace skirt;

extern "C" int skirt_octree_create(skirt_grid_t* out, int max_level, const double bbox[6], long long nleaf,
                                   const int32_t* leaves, const float* kr)
{
    if (!out) return set_error(SKIRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_level < 1 || max_level > 15) return set_error(SKIRT_ERR_INVALID_ARG, "max_level must be in [1, 15]");
    if (nleaf < 1 || nleaf >= (1ll << OCT_LEAF_BITS))
        return set_error(SKIRT_ERR_INVALID_ARG, "nleaf must be in [1, 2^27)");
    if (!bbox || !leaves || !kr) return set_error(SKIRT_ERR_INVALID_ARG, "bbox / leaves / kr is NULL");
    if (int r = check_bbox(bbox)) return r;

    // ---- insert the leaves from the root down (kind: 0 empty, 1 split, 2 leaf,
    // 3 unused).  The root is node 0 and nodes 1..7 stay unused, so that every
    // block of 8 children starts at a multiple of 8: a node's octant is then
    // its index mod 8, and its sibling across an axis is index ^ (1 << axis).
    std::vector<int> ref(8, 0);
    std::vector<unsigned char> kind(8, 3);
    kind[0] = 0;
    std::vector<int> leaf_node((size_t)nleaf);
    std::vector<int4> leaf_tab((size_t)nleaf);
    for (long long m = 0; m < nleaf; ++m) {
        const int32_t* lf = leaves + 4 * m;
        const int lev = lf[0];
        if (lev < 0 || lev > max_level)
            return set_error(SKIRT_ERR_INVALID_ARG, "leaf %lld: level %d not in [0, %d]", m, lev, max_level);
        for (int a = 1; a < 4; ++a)
            if (lf[a] < 0 || (long long)lf[a] >= (1ll << lev))
                return set_error(SKIRT_ERR_INVALID_ARG, "leaf %lld: position outside its level's range", m);
        size_t node = 0;
        for (int d = 0; d < lev; ++d) {
            if (kind[node] == 2) return set_error(SKIRT_ERR_INVALID_ARG, "leaf %lld lies inside another leaf", m);
            if (kind[node] == 0) {
                if (ref.size() + 8 > 0x7fffffffu) return set_error(SKIRT_ERR_INVALID_ARG, "too many nodes");
                kind[node] = 1;
                ref[node] = (int)ref.size();
                ref.resize(ref.size() + 8, 0);
                kind.resize(kind.size() + 8, 0);
            }
            const int b = lev - 1 - d;
            node = (size_t)ref[node] + (((lf[1] >> b) & 1) | (((lf[2] >> b) & 1) << 1) | (((lf[3] >> b) & 1) << 2));
        }
        if (kind[node] != 0) return set_error(SKIRT_ERR_INVALID_ARG, "leaf %lld overlaps another leaf", m);
        kind[node] = 2;
        ref[node] = ~((lev << OCT_LEAF_BITS) | (int)m);
        leaf_node[(size_t)m] = (int)node;
        const int sh = max_level - lev;
        leaf_tab[(size_t)m] = make_int4(lf[1] << sh, lf[2] << sh, lf[3] << sh, lev);
    }
    for (size_t node = 0; node < kind.size(); ++node)
        if (kind[node] == 0) return set_error(SKIRT_ERR_INVALID_ARG, "the leaves leave a hole in the root box");
    if (int r = check_device()) return r;

    // ---- the grid: finest lattice 2^max_level per axis, one cell per leaf
    skirt_grid_s* g = new skirt_grid_s;
    auto bail = [&](int code) {
        skirt_grid_destroy(g);
        return code;
    };
    const int n = 1 << max_level;
    if (int r = grid_init(g, n, n, n, nleaf, bbox, kr)) return bail(r);
    g->oct_levels = max_level;
    g->oct_nnode = (long long)ref.size();

    std::vector<float> krh((size_t)nleaf);
    cudaError_t e;
    if ((e = cudaMemcpy(krh.data(), g->kr32, sizeof(float) * (size_t)nleaf, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bail(set_error(SKIRT_ERR_CUDA, "copy kr: %s", cudaGetErrorString(e)));
    std::vector<OctNode> nodes(ref.size());
    for (size_t i = 0; i < ref.size(); ++i) {
        std::memset(&nodes[i], 0, sizeof(OctNode));
        nodes[i].ref = ref[i];
        for (int f = 0; f < 6; ++f) nodes[i].nb[f] = -1;
    }
    for (long long m = 0; m < nleaf; ++m) nodes[(size_t)leaf_node[(size_t)m]].kr = krh[(size_t)m];

    int* d_leaf_node = nullptr;
    auto upload = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(dst, bytes);
        if (r != cudaSuccess) return r;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    if ((e = upload((void**)&g->oct_nodes, nodes.data(), sizeof(OctNode) * nodes.size())) != cudaSuccess ||
        (e = upload((void**)&g->oct_leaf, leaf_tab.data(), sizeof(int4) * leaf_tab.size())) != cudaSuccess ||
        (e = upload((void**)&d_leaf_node, leaf_node.data(), sizeof(int) * leaf_node.size())) != cudaSuccess) {
        if (d_leaf_node) cudaFree(d_leaf_node);
        return bail(set_error(e == cudaErrorMemoryAllocation ? SKIRT_ERR_OOM : SKIRT_ERR_CUDA, "octree upload: %s",
                              cudaGetErrorString(e)));
    }
    long long blocks = (nleaf + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    oct_neighbours_kernel<<<(int)blocks, 256>>>(g->oct_nodes, g->oct_leaf, d_leaf_node, nleaf, max_level);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_leaf_node);
    if (e != cudaSuccess) return bail(set_error(SKIRT_ERR_CUDA, "octree neighbours: %s", cudaGetErrorString(e)));
    *out = g;
    return SKIRT_OK;
}
