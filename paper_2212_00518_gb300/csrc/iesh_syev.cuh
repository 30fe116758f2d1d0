// iesh_syev.cuh -- device building blocks of the batched dense symmetric
// eigensolver (internal): Householder reduction to tridiagonal form by one
// CTA, and implicit-shift QL iterations on the tridiagonal matrix (one
// matrix per lane of a warp in lockstep, or one per CTA with every row of
// the reflector product rotated), with the rotations applied to selected
// rows of the reflector product.
//
// Method (Householder 1958 reduction; the QL algorithm with implicit
// Wilkinson shifts of Bowdler, Martin, Reinsch and Wilkinson 1968):
//   T = P^T A P, P = H_0 H_1 ... H_{n-3}, H_k = I - tau_k v_k v_k^T, v_k
//   supported on indices k+1..n-1;  T = Z diag(lambda) Z^T by plane
//   rotations;  the eigenvectors are the columns of P Z.  Row r of P Z is
//   row r of P rotated like Z's rows, so a caller that needs only some rows
//   of the eigenvector matrix tracks only those rows (O(n) per rotation
//   each) and never forms P.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace iesh {

template <class T>
struct SyevEps;
template <>
struct SyevEps<double> {
    static constexpr double u = 1.1102230246251565e-16;  // 2^-53
};
template <>
struct SyevEps<float> {
    static constexpr float u = 5.9604645e-08f;  // 2^-24
};

constexpr int kSyevMaxIter = 60;  // QL iterations per eigenvalue before giving up

// Plane rotation taking (g, f) to (r, 0): r = sqrt(f^2 + g^2), s = f / r,
// c = g / r.  Where f^2 + g^2 is far from under- and overflow (binary
// exponent within +-960 for double, +-100 for float) one reciprocal square
// root gives all three (each within a few units in the last place); else
// the scaled hypot and two divisions.  Returns r; s and c are left
// untouched when r == 0.
__device__ __forceinline__ double syev_rot(double f, double g, double &s, double &c)
{
    const double q = fma(f, f, g * g);
    const int ex = (__double2hiint(q) >> 20) & 0x7ff;  // biased exponent of q
    if (ex > 1023 - 960 && ex < 1023 + 960) {
        const double ir = rsqrt(q);
        s = f * ir;
        c = g * ir;
        return q * ir;
    }
    const double r = hypot(f, g);
    if (r != 0.0) {
        s = f / r;
        c = g / r;
    }
    return r;
}
__device__ __forceinline__ float syev_rot(float f, float g, float &s, float &c)
{
    const float q = fmaf(f, f, g * g);
    const int ex = (__float_as_int(q) >> 23) & 0xff;
    if (ex > 127 - 100 && ex < 127 + 100) {
        const float ir = rsqrtf(q);
        s = f * ir;
        c = g * ir;
        return q * ir;
    }
    const float r = hypotf(f, g);
    if (r != 0.0f) {
        s = f / r;
        c = g / r;
    }
    return r;
}

template <class T>
__device__ __forceinline__ T syev_warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Householder reduction of the symmetric n x n matrix A (row-major with
// leading dimension lda, both triangles stored, in shared or global memory)
// by the whole CTA (blockDim.x a multiple of 32; every thread calls).  On
// return d[0..n-1] is the diagonal of T and e[0..n-2] its off-diagonal
// (e[i] = T_{i,i+1}, e[n-1] = 0), tau[k] the reflector factors and column k
// of A below the diagonal the reflector vector v_k (a zero tau_k: H_k = I).
// r1 (optional, n entries) receives row 1 of P (row 0 of P is e_0 because
// every reflector leaves index 0 alone).  v, w: n entries each; sh: 6
// entries; all of these in shared memory.  lower_only (for A in shared
// memory): read and update only the lower triangle (j <= i) of the trailing
// matrix, and form w = A v one thread per row, the upper half of each row
// read down the columns.  A warp per row spends five FP64 additions per row
// on its reduction, more than its three or four FMAs at n near 100, and on
// this GPU an FP64 instruction costs the same whatever its active lanes; a
// thread per row has no reduction, and its column-wise reads of shared
// memory (odd lda) are conflict-free.  The upper triangle is left stale.
template <class T>
__device__ void householder_tridiag(T *A, int lda, int n, T *d, T *e, T *tau, T *v, T *w, T *r1, T *sh,
                                    bool lower_only)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (r1)
        for (int i = tid; i < n; i += blockDim.x) r1[i] = (i == 1) ? T(1) : T(0);
    for (int k = 0; k + 2 < n; ++k) {
        T *shk = sh + 2 * (k & 1);  // double-buffered: the next k writes the other pair
        if (warp == 0) {
            // x = A[k+1.., k]; H_k x = alpha e_{k+1} with alpha = -sign(x_0) |x|
            T s = 0;
            for (int i = k + 2 + lane; i < n; i += 32) {
                const T a = A[(size_t)i * lda + k];
                s = fma(a, a, s);
            }
            s = syev_warp_sum(s);
            if (lane == 0) {
                const T x0 = A[(size_t)(k + 1) * lda + k];
                T alpha = x0, t = 0, v0 = 0;
                if (s > T(0)) {
                    const T mu = sqrt(fma(x0, x0, s));
                    alpha = x0 > T(0) ? -mu : mu;
                    v0 = x0 - alpha;  // no cancellation: opposite signs
                    t = T(2) / fma(v0, v0, s);
                }
                d[k] = A[(size_t)k * lda + k];  // final: later reflectors leave index k alone
                e[k] = alpha;
                tau[k] = t;
                shk[0] = t;
                shk[1] = v0;
            }
        }
        __syncthreads();
        const T t = shk[0];
        if (t == T(0)) continue;  // uniform over the CTA
        const T v0 = shk[1];
        for (int i = k + 1 + tid; i < n; i += blockDim.x) {
            const T vi = (i == k + 1) ? v0 : A[(size_t)i * lda + k];
            v[i] = vi;
            A[(size_t)i * lda + k] = vi;
        }
        __syncthreads();
        // w = t A_sub v
        if (lower_only) {
            for (int i = k + 1 + tid; i < n; i += blockDim.x) {
                T acc = 0;
                for (int j = k + 1; j < n; ++j) {
                    const T a = j <= i ? A[(size_t)i * lda + j] : A[(size_t)j * lda + i];
                    acc = fma(a, v[j], acc);
                }
                w[i] = t * acc;
            }
        } else {  // A in global memory: a warp per row, coalesced
            for (int i = k + 1 + warp; i < n; i += nw) {
                const T *row = A + (size_t)i * lda;
                T acc = 0;
                for (int j = k + 1 + lane; j < n; j += 32) acc = fma(row[j], v[j], acc);
                acc = syev_warp_sum(acc);
                if (lane == 0) w[i] = t * acc;
            }
        }
        __syncthreads();
        // w -= (t/2)(v.w) v (then A_sub - v w^T - w v^T = H_k A_sub H_k);
        // r1 <- r1 H_k = r1 - t (r1.v) v^T
        if (warp == 0) {
            T a = 0, b = 0;
            for (int i = k + 1 + lane; i < n; i += 32) {
                a = fma(v[i], w[i], a);
                if (r1) b = fma(r1[i], v[i], b);
            }
            a = syev_warp_sum(a);
            b = syev_warp_sum(b);
            if (lane == 0) {
                sh[4] = T(0.5) * t * a;
                sh[5] = t * b;
            }
        }
        __syncthreads();
        const T Kc = sh[4], rb = sh[5];
        for (int i = k + 1 + tid; i < n; i += blockDim.x) {
            w[i] = fma(-Kc, v[i], w[i]);
            if (r1) r1[i] = fma(-rb, v[i], r1[i]);
        }
        __syncthreads();
        for (int i = k + 1 + warp; i < n; i += nw) {
            T *row = A + (size_t)i * lda;
            const T vi = v[i], wi = w[i];
            const int jend = lower_only ? i + 1 : n;
            for (int j = k + 1 + lane; j < jend; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], row[j]));
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            d[n - 2] = A[(size_t)(n - 2) * lda + n - 2];
            d[n - 1] = A[(size_t)(n - 1) * lda + n - 1];
            e[n - 2] = A[(size_t)(n - 1) * lda + n - 2];
            if (n >= 3) tau[n - 2] = 0;
        } else {
            d[0] = A[0];
        }
        e[n - 1] = 0;
    }
    __syncthreads();
}

// Implicit-shift QL on symmetric tridiagonal matrices of order n, one per
// lane of a warp, the lanes in lockstep.  A thread-per-matrix loop diverges
// at once (every matrix deflates after its own number of sweeps, and each
// sweep has its own length), and a divergent warp issues one instruction per
// lane; the FP64 pipe then costs a full warp slot per lane-instruction.  So
// the whole warp works on eigenvalue l together: it scans for each lane's
// first negligible off-diagonal entry m, runs one sweep i = max(m) - 1 .. l
// in which lane j takes part while i < m_j, and repeats until every lane has
// deflated d[l]; then l + 1.  A lane computes exactly what it would compute
// alone (the same rotations in the same order).
//
// Lane data: d[i ld], e[i ld] (e[i] = T_{i,i+1}, e[n-1] = 0).  The
// eigenvalues overwrite d, in no particular order; e is destroyed.  Every
// lane of the warp calls (the votes need the full warp); a lane that is not
// live touches no memory.

// Per-lane state of the lockstep iteration between sweeps.
template <class T>
struct QlLane {
    int l = 0, iter = 0, m = 0;
    bool live = false, ok = true, act = false;
};

// Advance to the next sweep: for the warp's current l, each live lane's m
// (first index >= l with |e[m]| <= u (|d[m]| + |d[m+1]|), else n - 1); a
// lane takes part (act) when m != l.  When no lane does, l moves on.
// Returns false once l == n (warp-uniform): every eigenvalue has converged
// or its lane has given up after kSyevMaxIter sweeps (ok = false).
template <class T>
__device__ bool ql_lockstep_next(int n, const T *d, const T *e, int ld, QlLane<T> &q)
{
    constexpr unsigned kFull = 0xffffffffu;
    for (; q.l < n; ++q.l, q.iter = 0) {
        int m = n - 1;
        bool found = !q.live;
        for (int k = q.l;; ++k) {
            if (!found) {
                if (k >= n - 1) {
                    found = true;
                } else {
                    const T dd = fabs(d[(size_t)k * ld]) + fabs(d[(size_t)(k + 1) * ld]);
                    if (fabs(e[(size_t)k * ld]) <= SyevEps<T>::u * dd) {
                        m = k;
                        found = true;
                    }
                }
            }
            if (__all_sync(kFull, found)) break;
        }
        q.m = m;
        q.act = q.live && m != q.l;
        if (q.act && ++q.iter > kSyevMaxIter) {
            q.ok = false;
            q.live = false;
            q.act = false;
        }
        if (__any_sync(kFull, q.act)) return true;
    }
    return false;
}

// One sweep i = max(m) - 1 .. l of the active lanes (Wilkinson shift: the
// eigenvalue of the leading 2 x 2 block nearer d[l]).  Every rotation that
// acts on Z's columns i, i+1 is applied to entries i, i+1 of the R tracked
// rows (entry i of row q at Y[i yld + q yq]; entry i+1 of the previous
// rotation carried in a register) and, when rc is given, stored as
// (rc, rs)[i rld].  Returns the lowest index the sweep's rotations reached
// (l, or i + 1 when the bulge vanished at i and the matrix split there), or
// -1 in a lane that took no part.
template <class T, int R>
__device__ int ql_lockstep_sweep(const int n, T *d, T *e, int ld, T *Y, int yld, int yq, T *rc, T *rs, int rld,
                                 const QlLane<T> &q)
{
    constexpr unsigned kFull = 0xffffffffu;
    const int l = q.l, m = q.m;
    const int mx = __reduce_max_sync(kFull, q.act ? m : 0);
    T g = 0, s = 1, c = 1, p = 0, yj[R > 0 ? R : 1];
    if (q.act) {
        const T dl = d[(size_t)l * ld], el = e[(size_t)l * ld];
        g = (d[(size_t)(l + 1) * ld] - dl) / (T(2) * el);
        const T r = hypot(g, T(1));
        g = d[(size_t)m * ld] - dl + el / (g + copysign(r, g));
#pragma unroll
        for (int k = 0; k < R; ++k) yj[k] = Y[(size_t)m * yld + k * yq];
    }
    bool run = q.act;
    int low = q.act ? l : -1;
    for (int i = mx - 1; i >= l; --i) {
        if (run && i < m) {
            const T ei = e[(size_t)i * ld];
            const T f = s * ei, b = c * ei;
            T r = syev_rot(f, g, s, c);
            e[(size_t)(i + 1) * ld] = r;
            if (r == T(0)) {  // the bulge vanished: split here, rescan
                d[(size_t)(i + 1) * ld] -= p;
                e[(size_t)m * ld] = 0;
#pragma unroll
                for (int k = 0; k < R; ++k) Y[(size_t)(i + 1) * yld + k * yq] = yj[k];
                run = false;
                low = i + 1;
            } else {
                g = d[(size_t)(i + 1) * ld] - p;
                r = (d[(size_t)i * ld] - g) * s + T(2) * c * b;
                p = s * r;
                d[(size_t)(i + 1) * ld] = g + p;
                g = c * r - b;
                if (rc) {
                    rc[(size_t)i * rld] = c;
                    rs[(size_t)i * rld] = s;
                }
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const T yi = Y[(size_t)i * yld + k * yq];
                    Y[(size_t)(i + 1) * yld + k * yq] = s * yi + c * yj[k];
                    yj[k] = c * yi - s * yj[k];
                }
            }
        }
    }
    if (run) {
        d[(size_t)l * ld] -= p;
        e[(size_t)l * ld] = g;
        e[(size_t)m * ld] = 0;
#pragma unroll
        for (int k = 0; k < R; ++k) Y[(size_t)l * yld + k * yq] = yj[k];
    }
    return low;
}

// The whole iteration with R tracked rows.  Returns false in a lane whose
// eigenvalue needed more than kSyevMaxIter iterations.
template <class T, int R>
__device__ bool ql_lockstep(int n, T *d, T *e, int ld, T *Y, int yld, int yq, bool valid)
{
    QlLane<T> q;
    q.live = valid;
    while (ql_lockstep_next<T>(n, d, e, ld, q))
        ql_lockstep_sweep<T, R>(n, d, e, ld, Y, yld, yq, (T *)nullptr, (T *)nullptr, 0, q);
    return q.ok;
}

// Lanes per warp for ql_lockstep over `items` matrices on a GPU with `sms`
// SMs: the FP64 pipe of each SM sub-partition takes one warp instruction at
// a time whatever its active lanes, so the matrices are spread over one warp
// per sub-partition (4 per SM) first and packed into wider warps only when
// there are more of them.  A power of two in [1, 32].
__host__ __device__ inline int ql_lockstep_lanes(int64_t items, int sms)
{
    const int64_t slots = 4LL * (sms > 0 ? sms : 1);
    int L = 1;
    while (L < 32 && (int64_t)L * slots < items) L <<= 1;
    return L;
}

}  // namespace iesh
