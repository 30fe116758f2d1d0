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
    householder_tridiag<T>(A, lda, n, d, e, tau, vec, vec + n, nullptr, vec + 2 * n, sm);
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
        // z_c = (P_sub^T v)_c = sum_r Pt[c][r] v_r, 8 lanes per row c (three
        // FP64 additions per reduction instead of a warp's five)
        for (int c0 = k + 1 + 4 * warp; c0 < n; c0 += 4 * nw) {
            const int c = c0 + (lane >> 3);
            T acc = 0;
            if (c < n) {
                const T *row = Pt + (size_t)c * n;
                for (int r = k + 1 + (lane & 7); r < n; r += 8) acc = fma(row[r], v[r], acc);
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if ((lane & 7) == 0 && c < n) z[c] = t * acc;
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

// QL iterations for eigenvalues only: L matrices per warp in lockstep
// (ql_lockstep), four warps per CTA; matrix b = (warp index) L + lane.
template <class T>
__global__ void __launch_bounds__(128) k_syev_ql(int64_t B, int n, T *__restrict__ work, size_t wstride,
                                                 int L, uint32_t *__restrict__ info)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw * L >= B) return;  // the whole warp: no matrix
    const int64_t b = gw * L + lane;
    const bool valid = lane < L && b < B;
    T *wk = work + (valid ? b : 0) * wstride;
    const bool ok = ql_lockstep<T, 0>(n, wk, wk + n, 1, nullptr, 0, 0, valid);
    if (valid && info) info[b] = ok ? 0u : 1u;
}

// QL iterations with all n rows of P, L matrices per CTA, as a two-stage
// pipeline: warp 0 runs the lockstep recurrence of the L matrices (lane j:
// matrix blockIdx.x L + j) and stores sweep t+1's rotations in one shared
// buffer, (c, s) of rotation i of lane j at [i L + j], while the other warps
// apply sweep t's rotations from the other buffer to the rows of each
// matrix's P (entry i of row r at Pt[i n + r]), one (matrix, row) per thread
// at a time, entry i+1 carried in a register and entry i-1 loaded ahead.
template <class T>
__global__ void __launch_bounds__(1024) k_syev_qlv(int64_t B, int n, T *__restrict__ work, size_t wstride, int L,
                                                   uint32_t *__restrict__ info)
{
    extern __shared__ __align__(16) unsigned char qlv_sh[];
    __shared__ int s_low[2][32], s_m[2][32], s_more[2];
    T *rot = reinterpret_cast<T *>(qlv_sh);  // [buffer][c | s][i L + j]
    const size_t plane = (size_t)L * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * L;
    const int lda = syev_lda<T>(n);
    const size_t poff = 3 * (size_t)n + (syev_in_smem<T>(n) ? 0 : (size_t)n * lda);
    QlLane<T> q;
    T *d = nullptr, *e = nullptr;
    if (warp == 0) {
        q.live = lane < L && b0 + lane < B;
        T *wk = work + (q.live ? b0 + lane : 0) * wstride;
        d = wk;
        e = wk + n;
    }
    const bool valid = q.live;
    auto produce = [&](int buf) {  // warp 0: the next sweep into buffer buf
        const bool more = ql_lockstep_next<T>(n, d, e, 1, q);
        int low = -1;
        if (more) {
            T *rc = rot + (size_t)buf * 2 * plane;
            low = ql_lockstep_sweep<T, 0>(n, d, e, 1, (T *)nullptr, 0, 0, rc + lane, rc + plane + lane, L, q);
        }
        s_low[buf][lane] = low;
        s_m[buf][lane] = q.m;
        if (lane == 0) s_more[buf] = more ? 1 : 0;
    };
    if (warp == 0) produce(0);
    __syncthreads();
    for (int t = 0;; ++t) {
        const int cb = t & 1;
        if (!s_more[cb]) break;
        if (warp == 0) {
            produce(cb ^ 1);
        } else {
            const T *rc = rot + (size_t)cb * 2 * plane, *rs = rc + plane;
            for (int it = tid - 32; it < L * n; it += blockDim.x - 32) {
                const int j = it / n, r = it - j * n;
                const int low = s_low[cb][j], m = s_m[cb][j];
                if (low < 0) continue;
                T *Pt = work + (b0 + j) * wstride + poff;
                T yj = Pt[(size_t)m * n + r];
                T yi = Pt[(size_t)(m - 1) * n + r];
                for (int i = m - 1; i >= low; --i) {
                    const T ynext = i > low ? Pt[(size_t)(i - 1) * n + r] : T(0);
                    const T c = rc[(size_t)i * L + j], sn = rs[(size_t)i * L + j];
                    Pt[(size_t)(i + 1) * n + r] = sn * yi + c * yj;
                    yj = c * yi - sn * yj;
                    yi = ynext;
                }
                Pt[(size_t)low * n + r] = yj;
            }
        }
        __syncthreads();
    }
    if (warp == 0 && valid && info) info[b0 + lane] = q.ok ? 0u : 1u;
}

// Matrices per CTA of k_syev_qlv.  FP64: twice the lockstep width for B
// matrices, since the FP64 recurrence warp is then amortised over more rows;
// FP32: a quarter of it, since the FP32 recurrence is cheap and fewer
// matrices per CTA keep more CTAs (and their rows) in flight.  Halved until
// the two rotation buffers (4 L n entries) fit in kQlvSmemCap bytes.
// Threads: warp 0 plus about one applying thread per six (matrix, row)
// items.  These choices measured best at n = 102 and 256 in both precisions
// in a sweep over L and the thread count.
constexpr size_t kQlvSmemCap = 96 * 1024;

template <class T>
int qlv_lanes(int64_t B, int n, int sms)
{
    int L = sizeof(T) == 8 ? ql_lockstep_lanes(B, sms) * 2 : ql_lockstep_lanes(B, sms) / 4;
    if (L > 32) L = 32;
    if (L < 1) L = 1;
    while (L > 1 && (size_t)4 * L * n * sizeof(T) > kQlvSmemCap) L >>= 1;
    return L;
}

inline int qlv_threads(int L, int n)
{
    const int t = 32 + (L * n / 6 + 31) / 32 * 32;
    return t < 128 ? 128 : (t > 1024 ? 1024 : t);
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
        // eigenvalues only: L matrices per warp in lockstep; with
        // eigenvectors: one per CTA, the rotations applied to all rows of P
        // in parallel
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess && vectors) {
            const int L = qlv_lanes<T>(B, n, sms);
            const size_t qsm = (size_t)4 * L * n * sizeof(T);
            if (qsm > 48 * 1024) {
                cudaFuncAttributes fa;
                e = cudaFuncGetAttributes(&fa, k_syev_qlv<T>);
                if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < (int)qsm)
                    e = cudaFuncSetAttribute(k_syev_qlv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kQlvSmemCap);
            }
            if (e == cudaSuccess)
                k_syev_qlv<T><<<(unsigned)((B + L - 1) / L), qlv_threads(L, n), qsm, st>>>(B, n, wk, wstride, L,
                                                                                          info);
        } else if (e == cudaSuccess) {
            const int L = ql_lockstep_lanes(B, sms);
            const int64_t warps = (B + L - 1) / L;
            k_syev_ql<T><<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(B, n, wk, wstride, L, info);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
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
