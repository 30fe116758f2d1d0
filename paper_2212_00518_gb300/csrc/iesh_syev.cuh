// iesh_syev.cuh -- device building blocks of the batched dense symmetric
// eigensolver (internal): Householder reduction to tridiagonal form by one
// CTA, and implicit-shift QL iterations on the tridiagonal matrix by one
// thread, with the rotations applied to selected rows of the reflector
// product.
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
// entries; all of these in shared memory.
template <class T>
__device__ void householder_tridiag(T *A, int lda, int n, T *d, T *e, T *tau, T *v, T *w, T *r1, T *sh)
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
        // w = t A_sub v, one warp per row
        for (int i = k + 1 + warp; i < n; i += nw) {
            const T *row = A + (size_t)i * lda;
            T acc = 0;
            for (int j = k + 1 + lane; j < n; j += 32) acc = fma(row[j], v[j], acc);
            acc = syev_warp_sum(acc);
            if (lane == 0) w[i] = t * acc;
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
            for (int j = k + 1 + lane; j < n; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], row[j]));
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

// Implicit-shift QL on the symmetric tridiagonal matrix (d, e) of order n
// (e[i] = T_{i,i+1}, e[n-1] = 0), by one thread.  The eigenvalues overwrite
// d, in no particular order; e is destroyed.  Every plane rotation that acts
// on Z's columns i, i+1 is applied to entries i, i+1 of the R tracked rows
// Y (entry i of row q at Y[i * R + q]).  Returns false when an eigenvalue
// needed more than kSyevMaxIter iterations.
template <class T>
__device__ bool ql_implicit(int n, T *d, T *e, T *Y, int R)
{
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            // first negligible off-diagonal entry at or after l
            int m = l;
            for (; m < n - 1; ++m) {
                const T dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= SyevEps<T>::u * dd) break;
            }
            if (m == l) break;  // d[l] is an eigenvalue
            if (++iter > kSyevMaxIter) return false;
            // Wilkinson shift: the eigenvalue of the leading 2 x 2 block nearer
            // d[l], entering as g = d[m] - shift
            T g = (d[l + 1] - d[l]) / (T(2) * e[l]);
            T r = hypot(g, T(1));
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            T s = 1, c = 1, p = 0;
            bool restart = false;
            for (int i = m - 1; i >= l; --i) {
                const T f = s * e[i], b = c * e[i];
                r = syev_rot(f, g, s, c);
                e[i + 1] = r;
                if (r == T(0)) {  // the bulge vanished: split the matrix here
                    d[i + 1] -= p;
                    e[m] = 0;
                    restart = true;
                    break;
                }
                g = d[i + 1] - p;
                r = (d[i] - g) * s + T(2) * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                for (int q = 0; q < R; ++q) {
                    const T yi = Y[(size_t)i * R + q], yj = Y[(size_t)(i + 1) * R + q];
                    Y[(size_t)(i + 1) * R + q] = s * yi + c * yj;
                    Y[(size_t)i * R + q] = c * yi - s * yj;
                }
            }
            if (restart) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0;
        }
    }
    return true;
}

// The same iteration with all n rows of the reflector product tracked, by a
// CTA: thread 0 runs the scalar recurrence of a sweep (the rotations of one
// implicit QL step, i = m-1 down to l) and stores each rotation's (c, s) in
// shared memory; then every thread applies the sweep to its own rows r of
// P, entry i of row r at P[i ld + r] (so a warp's threads touch consecutive
// addresses), carrying entry i+1 of the previous rotation in a register.
// d, e in shared memory (d, e, rc, rs: n entries each; flags: 4 ints).
// Every thread calls; the result (false: an eigenvalue needed more than
// kSyevMaxIter iterations) is the same in every thread.
template <class T>
__device__ bool ql_implicit_rows(int n, T *d, T *e, T *P, int ld, T *rc, T *rs, int *flags)
{
    const int tid = threadIdx.x;
    // flags[0]: next sweep's l, flags[1]: its m (l == m: done), flags[2]: failed
    int l = 0, iter = 0;
    if (tid == 0) flags[2] = 0;
    for (;;) {
        if (tid == 0) {
            int ls = -1, ms = -1;
            while (l < n) {
                int m = l;
                for (; m < n - 1; ++m) {
                    const T dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= SyevEps<T>::u * dd) break;
                }
                if (m == l) {  // d[l] converged
                    ++l;
                    iter = 0;
                    continue;
                }
                if (++iter > kSyevMaxIter) {
                    flags[2] = 1;
                    l = n;
                    break;
                }
                T g = (d[l + 1] - d[l]) / (T(2) * e[l]);
                T r = hypot(g, T(1));
                g = d[m] - d[l] + e[l] / (g + copysign(r, g));
                T sn = 1, cs = 1, p = 0;
                int i = m - 1;
                bool split = false;
                for (; i >= l; --i) {
                    const T f = sn * e[i], b = cs * e[i];
                    r = syev_rot(f, g, sn, cs);
                    e[i + 1] = r;
                    if (r == T(0)) {
                        d[i + 1] -= p;
                        e[m] = 0;
                        split = true;
                        break;
                    }
                    g = d[i + 1] - p;
                    r = (d[i] - g) * sn + T(2) * cs * b;
                    p = sn * r;
                    d[i + 1] = g + p;
                    g = cs * r - b;
                    rc[i] = cs;
                    rs[i] = sn;
                }
                if (split) {
                    // rotations m-1 .. i+1 were taken; apply those, restart at l
                    ls = i + 1;
                    ms = m;
                    break;
                }
                d[l] -= p;
                e[l] = g;
                e[m] = 0;
                ls = l;
                ms = m;
                break;
            }
            flags[0] = ls;
            flags[1] = ms;
        }
        __syncthreads();
        const int ls = flags[0], ms = flags[1];
        if (ls < 0) break;  // every eigenvalue converged (or the cap was hit)
        for (int row = tid; row < n; row += blockDim.x) {
            T yj = P[(size_t)ms * ld + row];
            for (int i = ms - 1; i >= ls; --i) {
                const T yi = P[(size_t)i * ld + row];
                P[(size_t)(i + 1) * ld + row] = rs[i] * yi + rc[i] * yj;
                yj = rc[i] * yi - rs[i] * yj;
            }
            P[(size_t)ls * ld + row] = yj;
        }
        __syncthreads();
    }
    const bool ok = flags[2] == 0;
    __syncthreads();
    return ok;
}

}  // namespace iesh
