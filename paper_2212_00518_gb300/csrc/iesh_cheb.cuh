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

// 1/k for k < kChebMax + 2, so that the term count needs no division (it
// runs in one thread of a block, where each FP64 instruction costs a whole
// warp's pipe slot).
struct RecipTable {
    double v[kChebMax + 2];
    constexpr RecipTable() : v()
    {
        for (int k = 1; k < kChebMax + 2; ++k) v[k] = 1.0 / k;
    }
};
static __constant__ RecipTable kRecip = RecipTable();

// Number of Chebyshev terms for the half-width rho at tolerance tol: the
// smallest K whose tail bound 2 sum_{k>K} (rho/2)^k / k! is below tol, at
// most kChebMax - 2.  The tail is bounded by the geometric series of ratio
// (rho/2)/(K+2): 2 term / (1 - ratio) <= tol, tested as 2 term <= tol (1 -
// ratio).
__device__ inline int cheb_terms(double rho, double tol)
{
    int K = 0;
    const double h = rho * 0.5;
    double term = h;  // (rho/2)^{K+1} / (K+1)!
    while (K < kChebMax - 2) {
        const double ratio = h * kRecip.v[K + 2];
        if (ratio < 1.0 && 2.0 * term <= tol * (1.0 - ratio)) break;
        ++K;
        term *= h * kRecip.v[K + 1];
    }
    return K;
}

// Bound on the amplification, by the series over [c - rho, c + rho], of a
// component along an eigenvector whose eigenvalue mu lies outside it:
// |J_0| + 2 sum_{k=1..K} |J_k(rho)| |T_k(mu_x)|, mu_x = (mu - c) / rho.
__device__ inline double cheb_amplification(const double *cb, double mu)
{
    const double c = cb[0], rho = cb[1];
    const int K = (int)cb[2];
    const double *J = cb + 3;
    const double x = rho > 0.0 ? (mu - c) / rho : 0.0;
    double tm = 1.0, tk = x, A = fabs(J[0]);
    for (int k = 1; k <= K; ++k) {
        A += 2.0 * fabs(J[k]) * fabs(tk);
        const double tn = 2.0 * x * tk - tm;
        tm = tk;
        tk = tn;
    }
    return A;
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
