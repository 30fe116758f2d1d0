// iesh_overlap.cu -- diabatic-basis (overlap) propagator variant, FP64.
//
// Over a step the electronic evolution in the fixed diabatic basis is split
// symmetrically, exp(-i H(x1) dt/2) exp(-i H(x0) dt/2); in the adiabatic
// frame of the two ends this is
//   C <- exp(-i L1 dt/2) O exp(-i L0 dt/2) C,   O = Q1^T Q0,
// with Q0, Q1 the eigenvector matrices at the start and the end of the step
// (second order in dt, exact for frozen nuclei; an alternative to the
// exponential of the averaged generator of Sec. II C).
//
// O is never formed from eigenvectors.  For the arrowhead H = [[h, z^T],
// [z, diag(eps)]] with z_k = s_k f(x), orbital i has impurity component q_i
// and bath components z_k q_i / (lam_i - eps_k), so
//   O_ij = q1_i q0_j [1 + f0 f1 sum_k s_k^2 / ((lam1_i - eps_k)(lam0_j - eps_k))].
// Partial fractions and the secular equation at each end
// (sum_k s_k^2 / (lam - eps_k) = (lam - h) / f^2 at every root) collapse the
// sum for i != j:
//   O_ij = q1_i q0_j [(h1 - h0) + a (lam1_i - h1) + b (lam0_j - h0)] / (lam1_i - lam0_j),
//   a = (f1 - f0) / f1,  b = (f1 - f0) / f0,
// a Cauchy-like matrix whose entries are O(dt) and carry no cancellation.
// The denominators use the roots' exact offsets from their origin poles
// (lam = eps_o + tau).  The diagonal follows from the orthogonality of O,
// O_ii = sqrt(1 - sum_{j != i} O_ij^2) (> 0 in the gauge q > 0), and falls
// back to the direct sum above when the off-diagonal weight of a row
// exceeds 1/2 (large steps near avoided crossings).
#include <cuda_runtime.h>
#include <stdint.h>

#include "iesh_common.cuh"
#include "iesh_kernels.h"
#include "iesh_secular.cuh"

namespace iesh {

namespace {

constexpr int kOvThreads = 256;

// O^T (OT[j N + i] = O_ij) into the trajectory's scratch.
__global__ void __launch_bounds__(kOvThreads) k_overlap_build(DevState s)
{
    extern __shared__ double ov_sh[];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, M = s.M;
    double *l0 = ov_sh, *l1 = l0 + N, *q0 = l1 + N, *q1 = q0 + N, *d0 = q1 + N, *d1 = d0 + N;
    double *w = d1 + N;                              // [M] s_k^2
    int *o0 = reinterpret_cast<int *>(w + M), *o1 = o0 + N;
    __shared__ int s_bad;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        l0[i] = s.lam_prev[t * N + i];
        l1[i] = s.lam[t * N + i];
        q0[i] = s.q0_prev[t * N + i];
        q1[i] = s.q0[t * N + i];
        d0[i] = s.rt_prev[t * N + i];
        d1[i] = s.rt[t * N + i];
        o0[i] = s.ro_prev[t * N + i];
        o1[i] = s.ro[t * N + i];
    }
    for (int k = threadIdx.x; k < M; k += blockDim.x) w[k] = s.z0[k] * s.z0[k];
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const double h0 = s.geo_prev[t * 4], h1 = s.geo[t * 4];
    const double f0 = s.fx_prev[t], f1 = s.fx[t];
    if (!(f0 != 0.0 && f1 != 0.0)) {  // decoupled end: the closed form needs f != 0
        if (threadIdx.x == 0) atomicOr(&s.status[t], ST_PROP);
        return;
    }
    const double a = (f1 - f0) / f1, b = (f1 - f0) / f0, dh = h1 - h0;
    double *OT = s.scratch + t * s.scratch_stride;
    // off-diagonal entries
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int j = idx / N, i = idx - j * N;  // consecutive threads: consecutive i
        double v = 0.0;
        if (i != j) {
            const double den = s.poled[(size_t)o0[j] * M + o1[i]] + (d1[i] - d0[j]);  // lam1_i - lam0_j
            const double num = dh + a * (l1[i] - h1) + b * (l0[j] - h0);
            v = q1[i] * q0[j] * num * pole_recip<double>(den);
        }
        OT[idx] = v;
    }
    __syncthreads();
    // diagonal: orthogonality, or the direct pole sum for strongly mixed rows
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double off = 0.0;
        for (int j = 0; j < N; ++j) off = fma(OT[(size_t)j * N + i], OT[(size_t)j * N + i], off);
        double oii;
        if (off <= 0.5) {
            oii = sqrt(1.0 - off);
        } else {
            double sum = 0.0;
            for (int k = 0; k < M; ++k) {
                const double r1 = pole_recip<double>(s.poled[(size_t)k * M + o1[i]] + d1[i]);
                const double r0 = pole_recip<double>(s.poled[(size_t)k * M + o0[i]] + d0[i]);
                sum = fma(w[k], r1 * r0, sum);
            }
            oii = q1[i] * q0[i] * (1.0 + f0 * f1 * sum);
        }
        if (!isfinite(oii)) s_bad = 1;
        OT[(size_t)i * N + i] = oii;
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(&s.status[t], ST_PROP);
}

// C <- exp(-i L1 dt/2) O exp(-i L0 dt/2) C.  CTA = (electron block of
// G x EPT electrons, trajectory); thread (g, row i) forms row i of the
// product for EPT electrons; the phased input block sits in shared memory.
template <int EPT>
__global__ void __launch_bounds__(1024) k_overlap_apply(DevState s, double dt, int G, int64_t t_base)
{
    extern __shared__ __align__(16) unsigned char ova_smem[];
    double *tk = reinterpret_cast<double *>(ova_smem);  // [N][2 G EPT]
    const int64_t t = traj_of(s, t_base + blockIdx.y);
    if (t < 0 || (s.status[t] & (ST_DONE | ST_PROP))) return;
    const int N = s.N, Ne = s.Ne;
    const int NB = G * EPT, W2 = 2 * NB;
    const int g = threadIdx.x / N, i = threadIdx.x - g * N;
    const bool act = g < G;
    const int e0 = blockIdx.x * NB + g * EPT;
    double2 *C = reinterpret_cast<double2 *>(s.C) + (int64_t)t * Ne * N;
    const double *__restrict__ OT = s.scratch + t * s.scratch_stride;
    if (act) {
        double sn, cs;
        sincos(0.5 * dt * s.lam_prev[t * N + i], &sn, &cs);  // exp(-i lam0 dt/2) on row i
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            double2 v = make_double2(0.0, 0.0);
            if (e0 + e < Ne) v = C[(int64_t)(e0 + e) * N + i];
            tk[i * W2 + 2 * EPT * g + 2 * e] = fma(cs, v.x, sn * v.y);
            tk[i * W2 + 2 * EPT * g + 2 * e + 1] = fma(cs, v.y, -(sn * v.x));
        }
    }
    __syncthreads();
    if (!act) return;
    double y[2 * EPT];
#pragma unroll
    for (int q = 0; q < 2 * EPT; ++q) y[q] = 0.0;
    const double *col = tk + 2 * EPT * g;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {
        const double o = OT[(size_t)j * N + i];  // O_ij
        const double *row = col + j * W2;
#pragma unroll
        for (int q = 0; q < 2 * EPT; ++q) y[q] = fma(o, row[q], y[q]);
    }
    double sn, cs;
    sincos(0.5 * dt * s.lam[t * N + i], &sn, &cs);  // exp(-i lam1 dt/2)
#pragma unroll
    for (int e = 0; e < EPT; ++e)
        if (e0 + e < Ne)
            C[(int64_t)(e0 + e) * N + i] = make_double2(fma(cs, y[2 * e], sn * y[2 * e + 1]),
                                                        fma(cs, y[2 * e + 1], -(sn * y[2 * e])));
}

}  // namespace

size_t overlap_build_smem(int N, int M)
{
    return (size_t)(6 * N + M) * sizeof(double) + (size_t)2 * N * sizeof(int);
}

cudaError_t launch_overlap(const DevState &s, double dt, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    k_overlap_build<<<(unsigned)s.n, kOvThreads, overlap_build_smem(s.N, s.M), st>>>(s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int ept, G;
    cheb_shape(s.N, s.Ne, ept, G);
    if (s.cheb_ept > 0 && s.cheb_G > 0 && s.cheb_ept <= 2) {
        ept = s.cheb_ept;
        G = s.cheb_G;
    }
    const int nb = G * ept;
    const size_t smem = (size_t)s.N * 2 * nb * sizeof(double);
    const int threads = (G * s.N + 31) & ~31;
    for (int64_t t0 = 0; t0 < s.n; t0 += 65535) {
        const int64_t cnt = (s.n - t0 < 65535) ? s.n - t0 : 65535;
        dim3 grid((unsigned)((s.Ne + nb - 1) / nb), (unsigned)cnt);
        if (ept == 2) k_overlap_apply<2><<<grid, threads, smem, st>>>(s, dt, G, t0);
        else k_overlap_apply<1><<<grid, threads, smem, st>>>(s, dt, G, t0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace iesh
