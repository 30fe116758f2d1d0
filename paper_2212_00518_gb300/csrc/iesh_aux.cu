// iesh_aux.cu -- per-step unitarity check of the coefficient matrix, per-
// trajectory observables and the batch status summary (internal launchers
// of the C-ABI in iesh_capi.cu).
#include <cuda_runtime.h>

#include "../../include/iesh.h"
#include "iesh_common.cuh"
#include "iesh_kernels.h"
#include "iesh_secular.cuh"

namespace iesh {

// The exponential integrator of Sec. II C is unitary, so every electron's
// coefficient column keeps unit norm.  One warp per (work item, electron
// column), eight per CTA, so that many independent column reads are in
// flight; the column's sum of |c_ie|^2 is formed in the storage precision
// (float for the mixed path, whose own rounding is far above FP32's) and the
// trajectory gets ST_NORM when | ||c_e||^2 - 1 | exceeds tol or is not
// finite.
template <class T2, class R>
__global__ void __launch_bounds__(256) k_norm_check(DevState s, double tol)
{
    const int Ne = s.Ne, N = s.N;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t item = w / Ne;
    const int e = (int)(w - item * Ne);
    const int64_t t = traj_of(s, item);
    if (t < 0) return;
    const T2 *col = reinterpret_cast<const T2 *>(s.C) + ((size_t)t * Ne + e) * N;
    R acc = 0;
    for (int i = lane; i < N; i += 32) {
        const T2 c = col[i];
        acc = fma((R)c.x, (R)c.x, acc);
        acc = fma((R)c.y, (R)c.y, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && !(fabs((double)acc - 1.0) <= tol)) atomicOr(&s.status[t], ST_NORM);
}

cudaError_t launch_norm_check(const DevState &s, bool fp32, double tol, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    const int64_t warps = s.n * s.Ne;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    if (fp32) k_norm_check<float2, float><<<blocks, 256, 0, st>>>(s, tol);
    else k_norm_check<double2, double><<<blocks, 256, 0, st>>>(s, tol);
    return cudaGetLastError();
}

// Observables of every trajectory at its current state (one CTA of 128
// threads each): kinetic energy p^2 / 2m; potential energy of the classical
// IESH Hamiltonian (Sec. II B), U0(x) + sum_{i in s} lambda_i; impurity
// population on the occupied surface, sum_{i in s} q0_i^2, and from the
// wavefunction, sum_e | sum_i q0_i c_ie |^2.  out[4][n].
template <class T2>
__global__ void __launch_bounds__(128) k_observables(DevState s, double mass, double *out)
{
    const int64_t t = blockIdx.x;
    if (t >= s.n) return;
    const int N = s.N, Ne = s.Ne;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red[2][4];
    const T2 *C = reinterpret_cast<const T2 *>(s.C) + (size_t)t * Ne * N;
    const double *q0 = s.q0 + (size_t)t * N;
    double wf = 0.0;
    for (int e = warp; e < Ne; e += 4) {
        double re = 0.0, im = 0.0;
        for (int i = lane; i < N; i += 32) {
            const T2 c = C[(size_t)e * N + i];
            re = fma(q0[i], (double)c.x, re);
            im = fma(q0[i], (double)c.y, im);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        wf += re * re + im * im;
    }
    double lsum = 0.0, sh = 0.0;
    for (int a = threadIdx.x; a < Ne; a += blockDim.x) {
        const int i = s.occ[t * Ne + a];
        lsum += s.lam[(size_t)t * N + i];
        sh += q0[i] * q0[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        sh += __shfl_xor_sync(0xffffffffu, sh, o);
    }
    if (lane == 0) {
        red[0][warp] = lsum;
        red[1][warp] = sh;
    }
    __shared__ double wred[4];
    if (lane == 0) wred[warp] = wf;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double p = s.p[t];
        out[t] = 0.5 * p * p / mass;
        out[s.n + t] = s.geo[t * 4 + 3] + ((red[0][0] + red[0][1]) + (red[0][2] + red[0][3]));
        out[2 * s.n + t] = (red[1][0] + red[1][1]) + (red[1][2] + red[1][3]);
        out[3 * s.n + t] = (wred[0] + wred[1]) + (wred[2] + wred[3]);
    }
}

cudaError_t launch_observables(const DevState &s, bool fp32, double mass, double *out,
                               cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    if (fp32) k_observables<float2><<<(unsigned)s.n, 128, 0, st>>>(s, mass, out);
    else k_observables<double2><<<(unsigned)s.n, 128, 0, st>>>(s, mass, out);
    return cudaGetLastError();
}

// OR of the status words of the batch and, per bit b < 8, the number of
// trajectories that carry it: out[0] = OR, out[1 + b] = count (out zeroed by
// the caller).
__global__ void __launch_bounds__(256) k_status_summary(const uint32_t *__restrict__ status,
                                                        int64_t n, uint32_t *__restrict__ out)
{
    uint32_t acc = 0;
    uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = status[i];
        acc |= v;
#pragma unroll
        for (int b = 0; b < 8; ++b) cnt[b] += (v >> b) & 1u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc |= __shfl_xor_sync(0xffffffffu, acc, o);
#pragma unroll
        for (int b = 0; b < 8; ++b) cnt[b] += __shfl_xor_sync(0xffffffffu, cnt[b], o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (acc) atomicOr(&out[0], acc);
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (cnt[b]) atomicAdd(&out[1 + b], cnt[b]);
    }
}

cudaError_t launch_status_summary(const uint32_t *status, int64_t n, uint32_t *out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 9 * sizeof(uint32_t), st);
    if (e != cudaSuccess || n == 0) return e;
    const int64_t blocks = (n + 255) / 256;
    k_status_summary<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(status, n, out);
    return cudaGetLastError();
}

// The refined reciprocal of the secular sums and the couplings, element by
// element (diagnostic for iesh_diag_reciprocal).
__global__ void k_diag_recip(int64_t n, const double *__restrict__ d, double *__restrict__ r)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = pole_recip<double>(d[i]);
}

}  // namespace iesh

extern "C" iesh_status iesh_diag_reciprocal(int64_t n, const double *d, double *r, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!d || !r))) return IESH_EINVAL;
    if (n == 0) return IESH_OK;
    iesh::k_diag_recip<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(n, d, r);
    return cudaGetLastError() == cudaSuccess ? IESH_OK : IESH_ECUDA;
}
