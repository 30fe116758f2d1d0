// iesh_cheb.cuh -- Chebyshev degree and Bessel coefficients of the
// exponential integrator (internal to the library; shared by the
// propagator set-up kernels).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "iesh_common.cuh"

namespace iesh {

// Bessel J_0..J_K(rho) by Miller's backward recurrence normalised with
// J_0 + 2 sum_{k>=1} J_2k = 1.
__device__ inline void bessel_j(double rho, int K, double *J)
{
    if (rho == 0.0) {
        J[0] = 1.0;
        for (int k = 1; k <= K; ++k) J[k] = 0.0;
        return;
    }
    int top = (K > (int)rho ? K : (int)rho) + 24 + (int)(2.0 * sqrt((double)K + rho + 1.0));
    top += top & 1;
    double jp1 = 0.0, j = 1e-280, norm = 0.0;
    const double inv = 2.0 / rho;
    for (int k = top; k >= 1; --k) {
        const double jm1 = k * inv * j - jp1;
        jp1 = j;
        j = jm1;
        const int km = k - 1;
        if (km <= K) J[km] = j;
        if (km >= 2 && (km & 1) == 0) norm += 2.0 * j;
        if (fabs(j) > 1e250) {
            j *= 1e-250;
            jp1 *= 1e-250;
            norm *= 1e-250;
            for (int q = km; q <= K && q <= top; ++q)
                if (q >= km) J[q] *= 1e-250;
        }
    }
    norm += j;  // J_0
    const double sc = 1.0 / norm;
    for (int k = 0; k <= K; ++k) J[k] *= sc;
}

// Number of Chebyshev terms for the half-width rho at tolerance tol: the
// smallest K whose tail bound 2 sum_{k>K} (rho/2)^k / k! is below tol, at
// most kChebMax - 2.
__host__ __device__ inline int cheb_terms(double rho, double tol)
{
    int K = 0;
    double term = rho * 0.5;  // (rho/2)^{K+1} / (K+1)!
    while (K < kChebMax - 2) {
        const double ratio = (rho * 0.5) / (K + 2);
        const double tail = (ratio < 1.0) ? 2.0 * term / (1.0 - ratio) : 1e300;
        if (tail <= tol) break;
        ++K;
        term *= (rho * 0.5) / (K + 1);
    }
    return K;
}

// Chebyshev degree and coefficients for a spectrum inside [lo, hi] (in units
// of dt): K = cheb_terms(rho, tol) and J_0..J_K(rho).  Called by one thread
// per trajectory.
__device__ inline void cheb_setup(const DevState &s, int64_t t, double lo, double hi, double tol)
{
    double *cb = s.cheb + t * kChebStride;
    const double c = 0.5 * (lo + hi), rho = 0.5 * (hi - lo);
    const int K = cheb_terms(rho, tol);
    if (K >= kChebMax - 2) atomicOr(&s.status[t], ST_PROP);
    cb[0] = c;
    cb[1] = rho;
    cb[2] = (double)K;
    bessel_j(rho, K, cb + 3);
}

}  // namespace iesh
