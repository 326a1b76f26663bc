// Device helpers shared by the FP64 and the mixed-precision trace kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "skirt_internal.cuh"

namespace skirt {

enum { M_NONE = 0, M_DEPOSIT = 1, M_LOCATE = 2, M_PEEL = 3 };
enum {
    ST_NEW = 0,
    ST_START_DEP,
    ST_DEPOSIT_DONE,
    ST_LOCATE_DONE,
    ST_PEEL_DONE,
    ST_AFTER_SCATTER,
    ST_END_PACKET,
};

// Henyey-Greenstein phase function, normalised to average 1 over the sphere.
template <typename R>
__device__ __forceinline__ R hg_phase(R g, R mu)
{
    const R den = (R)1 + g * g - (R)2 * g * mu;
    return ((R)1 - g * g) / (den * sqrt(den));
}

// Scattering-angle cosine by inversion of the HG cumulative distribution.
template <typename R>
__device__ __forceinline__ R hg_mu(R g, R u)
{
    if (fabs(g) < (R)1e-6) return (R)2 * u - (R)1;
    const R t = ((R)1 - g * g) / ((R)1 - g + (R)2 * g * u);
    const R mu = ((R)1 + g * g - t * t) / ((R)2 * g);
    return fmin(fmax(mu, (R)-1), (R)1);
}

// Direction at polar cosine mu and azimuth (sin, cos) = (sp, cp) around k.
template <typename R>
__device__ __forceinline__ void hg_rotate(R& k0, R& k1, R& k2, R mu, R sp, R cp)
{
    const R st = sqrt(fmax((R)1 - mu * mu, (R)0));
    R n0, n1, n2;
    if (fabs(k2) > (R)0.99999) {
        n0 = st * cp;
        n1 = st * sp;
        n2 = (k2 > (R)0) ? mu : -mu;
    } else {
        const R s = sqrt((R)1 - k2 * k2);
        n0 = st * (k0 * k2 * cp - k1 * sp) / s + k0 * mu;
        n1 = st * (k1 * k2 * cp + k0 * sp) / s + k1 * mu;
        n2 = -st * cp * s + k2 * mu;
    }
    k0 = n0;
    k1 = n1;
    k2 = n2;
}

// Cell index along one axis: floor((x - lo) / d) clamped to [0, n-1].
template <typename R>
__device__ __forceinline__ int cell_index(R x, R lo, R d, int n)
{
    const R f = floor((x - lo) / d);
    if (f < (R)0) return 0;
    if (f > (R)(n - 1)) return n - 1;
    return (int)f;
}

}  // namespace skirt
