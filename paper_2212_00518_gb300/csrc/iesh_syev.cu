// iesh_syev.cu -- batched dense symmetric eigensolver behind the C-ABI
// (iesh_syev_batched): one matrix per CTA for the Householder reduction and
// the back-transformation set-up; the QL iterations one matrix per thread
// (eigenvalues only) or per CTA (with eigenvectors: the rotations of each
// sweep applied to all rows of P in parallel); one matrix per CTA for the
// ordering and the output.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "../../include/iesh.h"
#include "iesh_syev.cuh"

using namespace iesh;

namespace {

constexpr int kSyevThreads = 256;
constexpr size_t kSyevSmemCap = 200 * 1024;  // matrix in shared memory up to this size

template <class T>
__host__ __device__ inline int syev_lda(int n)
{
    return n | 1;  // odd row stride: the rows of a warp's column reads fall on distinct banks
}

template <class T>
__host__ __device__ inline bool syev_in_smem(int n)
{
    return (size_t)n * syev_lda<T>(n) * sizeof(T) + (size_t)6 * n * sizeof(T) + 64 * sizeof(T) <= kSyevSmemCap;
}

// Per-matrix workspace (elements of T): d[n], e[n], tau[n], the matrix copy
// (n x lda, unless it lives in shared memory) and P^T [n][n] when the
// eigenvectors are wanted.
template <class T>
inline size_t syev_work_elems(int n, bool vectors)
{
    size_t w = 3 * (size_t)n;
    if (!syev_in_smem<T>(n)) w += (size_t)n * syev_lda<T>(n);
    if (vectors) w += (size_t)n * n;
    return (w + 31) & ~(size_t)31;
}

// Reduction to tridiagonal form; with vectors, P^T = (H_0 ... H_{n-3})^T is
// formed by backward accumulation: P <- H_k P for k = n-3 .. 0, i.e. with
// z = P_sub^T v, P_sub -= tau v z^T, written on P^T (rows c of P^T are the
// columns of P).
template <class T>
__global__ void __launch_bounds__(kSyevThreads) k_syev_reduce(int64_t B, int n, const T *__restrict__ Ain,
                                                              T *__restrict__ work, size_t wstride, int vectors)
{
    extern __shared__ __align__(16) unsigned char syev_sh[];
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    const int lda = syev_lda<T>(n);
    T *wk = work + b * wstride;
    T *d = wk, *e = wk + n, *tau = wk + 2 * n;
    const bool sm = syev_in_smem<T>(n);
    T *vec = reinterpret_cast<T *>(syev_sh);  // v[n], w[n], sh[8]
    T *A = sm ? vec + 2 * n + 8 : wk + 3 * n;
    T *Pt = wk + 3 * n + (sm ? 0 : (size_t)n * lda);
    const T *src = Ain + (size_t)b * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        A[(size_t)i * lda + j] = src[idx];
    }
    __syncthreads();
    householder_tridiag<T>(A, lda, n, d, e, tau, vec, vec + n, nullptr, vec + 2 * n);
    if (!vectors) return;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Pt[idx] = (idx / n == idx % n) ? T(1) : T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *v = vec, *z = vec + n;
    for (int k = n - 3; k >= 0; --k) {
        const T t = tau[k];
        if (t == T(0)) continue;  // uniform: tau is in global memory written before the barrier
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) v[i] = A[(size_t)i * lda + k];
        __syncthreads();
        for (int c = k + 1 + warp; c < n; c += nw) {  // z_c = (P_sub^T v)_c = sum_r Pt[c][r] v_r
            const T *row = Pt + (size_t)c * n;
            T acc = 0;
            for (int r = k + 1 + lane; r < n; r += 32) acc = fma(row[r], v[r], acc);
            acc = syev_warp_sum(acc);
            if (lane == 0) z[c] = t * acc;
        }
        __syncthreads();
        for (int c = k + 1 + warp; c < n; c += nw) {
            T *row = Pt + (size_t)c * n;
            const T zc = z[c];
            for (int r = k + 1 + lane; r < n; r += 32) row[r] = fma(-zc, v[r], row[r]);
        }
        __syncthreads();
    }
}

// QL iterations, one matrix per thread; the rotations act on the n rows of
// P (stored as P^T, i.e. entry i of row r at Pt[i n + r]).
template <class T>
__global__ void __launch_bounds__(32) k_syev_ql(int64_t B, int n, T *__restrict__ work, size_t wstride,
                                                 int vectors, uint32_t *__restrict__ info)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    T *wk = work + b * wstride;
    const int lda = syev_lda<T>(n);
    T *Pt = wk + 3 * n + (syev_in_smem<T>(n) ? 0 : (size_t)n * lda);
    const bool ok = ql_implicit<T>(n, wk, wk + n, vectors ? Pt : nullptr, vectors ? n : 0);
    if (info) info[b] = ok ? 0u : 1u;
}

// QL iterations with all n rows of P, one matrix per CTA (see
// ql_implicit_rows): the scalar recurrence by one thread, the rotations of
// each sweep applied to the rows of P by all threads.
template <class T>
__global__ void __launch_bounds__(128) k_syev_qlv(int64_t B, int n, T *__restrict__ work, size_t wstride,
                                                  uint32_t *__restrict__ info)
{
    extern __shared__ __align__(16) unsigned char qlv_sh[];
    __shared__ int flags[4];
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    T *wk = work + b * wstride;
    const int lda = syev_lda<T>(n);
    T *Pt = wk + 3 * n + (syev_in_smem<T>(n) ? 0 : (size_t)n * lda);
    T *d = reinterpret_cast<T *>(qlv_sh), *e = d + n, *rc = e + n, *rs = rc + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = wk[i];
        e[i] = wk[n + i];
    }
    __syncthreads();
    const bool ok = ql_implicit_rows<T>(n, d, e, Pt, n, rc, rs, flags);
    for (int i = threadIdx.x; i < n; i += blockDim.x) wk[i] = d[i];
    if (threadIdx.x == 0 && info) info[b] = ok ? 0u : 1u;
}

// Ascending order (ties by index), eigenvectors as rows, each signed so that
// its largest-magnitude component (the first on a tie) is positive.
template <class T>
__global__ void __launch_bounds__(kSyevThreads) k_syev_out(int64_t B, int n, const T *__restrict__ work,
                                                           size_t wstride, int vectors, T *__restrict__ lam,
                                                           T *__restrict__ V)
{
    __shared__ T ev[256];
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    const T *wk = work + b * wstride;
    const int lda = syev_lda<T>(n);
    const T *Pt = wk + 3 * n + (syev_in_smem<T>(n) ? 0 : (size_t)n * lda);
    for (int i = threadIdx.x; i < n; i += blockDim.x) ev[i] = wk[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T li = ev[i];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += (ev[j] < li) || (ev[j] == li && j < i);
        lam[(size_t)b * n + rank] = li;
        if (vectors) {
            const T *col = Pt + (size_t)i * n;
            int big = 0;
            T bv = fabs(col[0]);
            for (int r = 1; r < n; ++r) {
                const T a = fabs(col[r]);
                if (a > bv) {
                    bv = a;
                    big = r;
                }
            }
            const T sg = col[big] < T(0) ? T(-1) : T(1);
            T *out = V + ((size_t)b * n + rank) * n;
            for (int r = 0; r < n; ++r) out[r] = sg * col[r];
        }
    }
}

template <class T>
iesh_status syev_run(int64_t B, int n, const T *A, T *lam, T *V, uint32_t *info, void *work,
                     size_t work_bytes, cudaStream_t st, char *err, size_t err_len)
{
    const bool vectors = V != nullptr;
    const size_t wstride = syev_work_elems<T>(n, vectors);
    const size_t need = (size_t)B * wstride * sizeof(T);
    auto report = [&](iesh_status s, const char *msg) {
        if (err && err_len) {
            strncpy(err, msg, err_len - 1);
            err[err_len - 1] = '\0';
        }
        return s;
    };
    if (work_bytes < need) return report(IESH_EINVAL, "workspace smaller than iesh_syev_work_bytes");
    T *wk = (T *)work;
    cudaError_t e = cudaSuccess;
    const size_t smem = (size_t)(2 * n + 8) * sizeof(T) + (syev_in_smem<T>(n) ? (size_t)n * syev_lda<T>(n) * sizeof(T) : 0);
    if (smem > 48 * 1024) {
        // a process-wide function attribute: only ever raised, to the cap of
        // every size this kernel takes in shared memory
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_syev_reduce<T>);
        if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < (int)smem)
            e = cudaFuncSetAttribute(k_syev_reduce<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kSyevSmemCap + 2048));
    }
    if (e == cudaSuccess) {
        k_syev_reduce<T><<<(unsigned)B, kSyevThreads, smem, st>>>(B, n, A, wk, wstride, vectors ? 1 : 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        // eigenvalues only: one matrix per thread; with eigenvectors: one per
        // CTA, the rotations applied to all rows of P in parallel
        if (vectors)
            k_syev_qlv<T><<<(unsigned)B, 128, (size_t)4 * n * sizeof(T), st>>>(B, n, wk, wstride, info);
        else
            k_syev_ql<T><<<(unsigned)((B + 31) / 32), 32, 0, st>>>(B, n, wk, wstride, 0, info);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_syev_out<T><<<(unsigned)B, kSyevThreads, 0, st>>>(B, n, wk, wstride, vectors ? 1 : 0, lam, V);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return report(IESH_ECUDA, cudaGetErrorString(e));
    return report(IESH_OK, "");
}

}  // namespace

extern "C" {

size_t iesh_syev_work_bytes(int64_t B, int n, int precision, int vectors)
{
    if (B < 0 || n < 1 || n > 256) return 0;
    const size_t el = precision == IESH_PREC_MIXED ? syev_work_elems<float>(n, vectors != 0) * sizeof(float)
                                                   : syev_work_elems<double>(n, vectors != 0) * sizeof(double);
    return (size_t)B * el;
}

iesh_status iesh_syev_batched(int64_t B, int n, int precision, const void *A, void *lam, void *V,
                              uint32_t *info, void *work, size_t work_bytes, void *cuda_stream,
                              char *err, size_t err_len)
{
    auto report = [&](iesh_status s, const char *msg) {
        if (err && err_len) {
            strncpy(err, msg, err_len - 1);
            err[err_len - 1] = '\0';
        }
        return s;
    };
    if (B < 0) return report(IESH_EINVAL, "B must be >= 0");
    if (n < 1 || n > 256) return report(IESH_EINVAL, "n outside 1..256");
    if (precision != IESH_PREC_FP64 && precision != IESH_PREC_MIXED)
        return report(IESH_EINVAL, "precision must be IESH_PREC_FP64 or IESH_PREC_MIXED (FP32)");
    if (B == 0) return report(IESH_OK, "");
    if (!A || !lam || !work) return report(IESH_EINVAL, "A, lam and work must be device pointers");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (precision == IESH_PREC_MIXED)
        return syev_run<float>(B, n, (const float *)A, (float *)lam, (float *)V, info, work, work_bytes,
                               st, err, err_len);
    return syev_run<double>(B, n, (const double *)A, (double *)lam, (double *)V, info, work, work_bytes,
                            st, err, err_len);
}

}  // extern "C"
