// iesh_cheb_tc16.cu -- Chebyshev propagator of the mixed-precision path on the
// tensor cores with FP16 split operands, two CTAs per SM (N <= 128, Ne <= 56).
//
// The exponential integrator of Sec. II C, as k_cheb_tc (iesh_cheb_tc.cu):
//   exp(-i H) C = e^{-ic} sum_k (2 - delta_k0) (-i)^k J_k(rho) T_k(X) C,
//   X = (H - c) / rho,  T_{k+1} = 2 X T_k - T_{k-1},
// with the dense contraction of every order, D = (2 / rho) W T_k, on the
// tensor cores (M = 128 rows >= N, K = N rounded up to 16, N_mma = 2Ne
// rounded up to 16).  The operands are scaled FP16 pairs: W' = 2^13 (2 /
// rho) W and T' = 2^14 T_k split as x = hi + lo with hi = fp16(x) and lo =
// fp16(x - hi), each pair carrying about 22 bits; D = W'_hi T'_hi + W'_hi
// T'_lo + W'_lo T'_hi (kind::f16, FP32 accumulation in tensor memory), then
// scaled by 2^-27.  |2/rho W| <= 2 (rho bounds the Gershgorin radius) and
// |T_k| <= 1 (unit coefficient columns, spectrum of X in [-1, 1]) keep
// every scaled value inside the FP16 range; the dropped W'_lo T'_lo term is
// about 2^-22 of |W||T|, as in the 3xTF32 kernel.
//
// What differs from k_cheb_tc is the footprint: FP16 planes halve the shared
// memory (A 2 x ceil(N/8) x (K/8) x 128 bytes, B 2 x (Nmma/8) x (K/8) x 144
// bytes: about 103 KB at N = 101, Ne = 50) and the Chebyshev sum lives in tensor
// memory next to D (columns 128..255), so two CTAs (512 threads, at most 64
// registers each) share an SM and one CTA's update runs while the other's
// MMAs do.  T_k for the recurrence is read back from its own B entries (hi
// + lo), T_{k-1} is held in registers.
//
// One CTA per trajectory, 512 threads: warp w reads TMEM lanes 32 (w % 4) ..
// +31 (orbital row j = 32 (w % 4) + lane) and owns the electrons e = 4q + w/4
// (so that each thread's B entries step by one 8-column group per electron).  Each order: one thread issues the 3 x K/16 MMAs
// and commits them to an mbarrier; every thread waits (bounded), loads its D
// and Chebyshev-sum entries from tensor memory, forms T_{k+1} for its row
// and columns, stores the sum back and rewrites its B entries in place.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "iesh_common.cuh"
#include "iesh_kernels.h"
#include "iesh_tc.cuh"

namespace iesh {

namespace {

constexpr int kT16M = 128;          // MMA rows (orbitals, padded)
constexpr int kT16Threads = 512;    // 4 lane quarters x 4 column groups
constexpr int kT16MaxPairs = 14;    // electrons per thread (e = 4 q + column group): Ne <= 56
constexpr int kT16LboA = 128, kT16LboB = 144;
constexpr int kT16Cols = 256;       // TMEM columns: D [0, 128), Chebyshev sum [128, 256)
constexpr int kT16AccCol = 128;
constexpr int kT16WaitLimit = 1 << 22;
constexpr float kT16SW = 8192.0f, kT16ST = 16384.0f;  // 2^13, 2^14
constexpr float kT16InvST = 1.0f / 16384.0f;
constexpr float kT16DScaled = 1.0f / 8192.0f;  // D' = 2^27 D, read in the 2^14 unit of T

// Shared layout: A_hi and A_lo hold only their rg = ceil(N/8) used row
// groups, back to back, then B_hi and B_lo.  An MMA still reads 16 row groups
// of A from each base: past row 8 rg it reads the next buffer's bytes, finite
// FP16 values whose products land in D rows >= N, which nobody reads (row j
// of D depends on row j of A alone).  `total` also covers the reads of A_lo
// past the end of B.
struct T16Shape {
    int Kp, NB, rg, sboA, sboB, usedA, bytesB, total;
};

__host__ __device__ inline T16Shape t16_shape(int N, int Ne)
{
    T16Shape t;
    t.Kp = (N + 15) & ~15;
    t.NB = (2 * Ne + 15) & ~15;
    t.rg = (N + 7) / 8;
    t.sboA = (t.Kp / 8) * kT16LboA;
    t.sboB = (t.Kp / 8) * kT16LboB;
    t.usedA = t.rg * t.sboA;
    t.bytesB = (t.NB / 8) * t.sboB;
    const int a = 2 * t.usedA + 2 * t.bytesB, b = t.usedA + (kT16M / 8) * t.sboA;
    t.total = a > b ? a : b;
    return t;
}

// Byte offset of element (row, k) of A and of (column n, k) of B in a plane.
__device__ __forceinline__ int t16_offA(const T16Shape &sh, int row, int k)
{
    return (row >> 3) * sh.sboA + (k >> 3) * kT16LboA + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ int t16_offB(const T16Shape &sh, int n, int k)
{
    return (n >> 3) * sh.sboB + (k >> 3) * kT16LboB + (n & 7) * 16 + (k & 7) * 2;
}

// hi = fp16(x), lo = fp16(x - hi)
__device__ __forceinline__ void split16(float x, __half &hi, __half &lo)
{
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}
// the same for a pair (Re, Im) with paired conversions
__device__ __forceinline__ void split16x2(float xr, float xi, __half2 &hi, __half2 &lo)
{
    hi = __floats2half2_rn(xr, xi);
    const float2 hf = __half22float2(hi);
    lo = __floats2half2_rn(xr - hf.x, xi - hf.y);
}

__global__ void __launch_bounds__(kT16Threads, 2) k_cheb_tc16(DevState s, double dt, int64_t t_base)
{
    extern __shared__ __align__(1024) unsigned char t16_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ float s_cj[kChebMax], s_sc[3];
    const int64_t t = traj_of(s, t_base + blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;  // uniform over the CTA
    const int N = s.N, Ne = s.Ne, Np = (N + 3) & ~3;
    const T16Shape sh = t16_shape(N, Ne);
    unsigned char *Ahi = t16_smem, *Alo = t16_smem + sh.usedA;
    unsigned char *Bhi = t16_smem + 2 * sh.usedA, *Blo = Bhi + sh.bytesB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = 32 * (warp & 3) + lane;  // my orbital row = my TMEM lane
    const int cg = warp >> 2;              // my column group: electrons e = 4 q + cg
    const int npair = (Ne + 3) / 4;        // my electrons (q < npair; e < Ne checked)
    const bool rowok = j < N;
    // B entry (column n, row j) of electron e = 4q + cg: n = 2e in the 8-column
    // group q at 32 cg bytes into it (Re; Im 16 bytes on), so q steps by sboB
    const int jb = (j >> 3) * kT16LboB + (j & 7) * 2 + 32 * cg;
    // TMEM: D of electron e at columns 2e, 2e + 1 (8q + 2cg); my Chebyshev
    // sums at kT16AccCol + 28 cg + 2q (private to my column group)
    const uint32_t accc = (uint32_t)(kT16AccCol + 2 * kT16MaxPairs * cg);

    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc(&tmem_slot, (uint32_t)kT16Cols);

    // A: 2^13 (2 / rho) W (rows j, columns k; stored [N][Np] in FP32), one
    // 16-byte core-matrix row (8 consecutive k) per item, zero past N (the
    // used row groups only)
    const float *__restrict__ W = reinterpret_cast<const float *>(s.scratch + t * s.scratch_stride);
    const double rho0 = s.cheb[t * kChebStride + 1];
    const float ws = rho0 > 0.0 ? (float)(2.0 / rho0) * kT16SW : 0.0f;
    const int kc8 = sh.Kp / 8;
    // consecutive threads take consecutive rows of one K chunk: their 16-byte
    // stores fill whole core matrices (no bank conflicts)
    const int nrow = 8 * sh.rg;
    for (int it = tid; it < nrow * kc8; it += kT16Threads) {
        const int kc = it / nrow, row = it - kc * nrow;
        __align__(16) __half hi[8], lo[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = 8 * kc + q;
            const float v = (row < N && k < N) ? ws * W[(int64_t)row * Np + k] : 0.0f;
            split16(v, hi[q], lo[q]);
        }
        *reinterpret_cast<uint4 *>(Ahi + t16_offA(sh, row, 8 * kc)) = *reinterpret_cast<const uint4 *>(hi);
        *reinterpret_cast<uint4 *>(Alo + t16_offA(sh, row, 8 * kc)) = *reinterpret_cast<const uint4 *>(lo);
    }
    // B (and the tail past it): columns beyond 2Ne and K entries beyond N
    // stay zero
    {
        const int words = (sh.total - 2 * sh.usedA) / 4;
        uint32_t *B = reinterpret_cast<uint32_t *>(Bhi);
        for (int w = tid; w < words; w += kT16Threads) B[w] = 0u;
    }
    const double *cb = s.cheb + t * kChebStride;
    const double c = cb[0];
    const int K = (int)cb[2];
    const double *J = cb + 3;
    for (int q = tid; q <= K; q += kT16Threads) s_cj[q] = (float)(2.0 * J[q]);
    if (tid == 0) {
        double scd, ccd;
        sincos(c, &scd, &ccd);
        s_sc[1] = (float)scd;
        s_sc[2] = (float)ccd;
    }
    __syncthreads();  // B zeroed before the T_0 entries land; TMEM base published
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t my_lane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    float2 *C = reinterpret_cast<float2 *>(s.C) + (int64_t)t * Ne * N;
    const float w2 = rho0 > 0.0 ? (float)(2.0 / rho0) : 0.0f;
    // 2 (L_j - c) / rho, the diagonal's share of 2 X
    const float Lc = rowok ? w2 * (float)(0.5 * dt * (s.lam_prev[t * N + j] + s.lam[t * N + j]) - c) : 0.0f;
    const float J0 = (float)J[0];

    // T_0 = C: my row, my electrons; the Chebyshev sum J_0 C into tensor memory
    float prv[2 * kT16MaxPairs];
#pragma unroll
    for (int q = 0; q < kT16MaxPairs; q += 2) {
        if (q >= npair) break;  // uniform
        float a[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = 4 * (q + h) + cg;
            const bool mine = q + h < npair && rowok && e < Ne;
            float2 v = make_float2(0.f, 0.f);
            if (mine) v = C[(int64_t)e * N + j];
            prv[2 * (q + h)] = 0.f;
            prv[2 * (q + h) + 1] = 0.f;
            a[2 * h] = J0 * v.x;
            a[2 * h + 1] = J0 * v.y;
            if (mine) {
                const int ob = (q + h) * sh.sboB + jb;
                __half hr, lr, hi_, li;
                split16(kT16ST * v.x, hr, lr);
                split16(kT16ST * v.y, hi_, li);
                *reinterpret_cast<__half *>(Bhi + ob) = hr;
                *reinterpret_cast<__half *>(Blo + ob) = lr;
                *reinterpret_cast<__half *>(Bhi + ob + 16) = hi_;
                *reinterpret_cast<__half *>(Blo + ob + 16) = li;
            }
        }
        tc::tmem_st4(my_lane + accc + 2 * q, a[0], a[1], a[2], a[3]);
    }
    tc::tmem_wait_st();
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t idesc = tc::idesc_f16(kT16M, sh.NB);
    const uint32_t aHi = tc::smem_addr(Ahi), aLo = tc::smem_addr(Alo);
    const uint32_t bHi = tc::smem_addr(Bhi), bLo = tc::smem_addr(Blo);

    bool ok = true;
    for (int k = 0; k < K; ++k) {
        if (tid == 0) {
            // D = W'_hi T'_hi + W'_hi T'_lo + W'_lo T'_hi
            uint32_t accum = 0;
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t a = pass == 2 ? aLo : aHi, b = pass == 1 ? bLo : bHi;
                for (int ks = 0; ks < sh.Kp / 16; ++ks) {
                    tc::mma_f16(tmem, tc::smem_desc(a + ks * 2 * kT16LboA, kT16LboA, sh.sboA),
                                tc::smem_desc(b + ks * 2 * kT16LboB, kT16LboB, sh.sboB), idesc, accum);
                    accum = 1;
                }
            }
            tc::commit(&mbar);
        }
        const bool done = tc::mbar_wait(&mbar, (uint32_t)(k & 1), kT16WaitLimit);
        if (__syncthreads_or(!done)) {
            ok = false;
            break;
        }
        tc::fence_after_sync();
        // T_k, T_{k+1} and T_{k-1} (prv) are handled in the scaled unit of
        // the B operand (2^14 T): D enters as 2^-13 D' and the Chebyshev
        // coefficients carry the 2^-14 back
        const float cj = s_cj[k + 1] * kT16InvST;
        const int ph = (k + 1) & 3;  // (-i)^(k+1) = (1, 0), (0, -1), (-1, 0), (0, 1)
        const float ca = ph == 0 ? cj : (ph == 2 ? -cj : 0.f), cbf = ph == 1 ? -cj : (ph == 3 ? cj : 0.f);
        const bool first = k == 0;
#pragma unroll
        for (int q = 0; q < kT16MaxPairs; q += 2) {
            if (q >= npair) break;  // uniform
            float d[4], a[4];
            tc::tmem_ld2(my_lane + (uint32_t)(8 * q + 2 * cg), d[0], d[1]);
            tc::tmem_ld2(my_lane + (uint32_t)(8 * (q + 1) + 2 * cg), d[2], d[3]);
            tc::tmem_ld4(my_lane + accc + 2 * q, a[0], a[1], a[2], a[3]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = 4 * (q + h) + cg;
                if (q + h < npair && rowok && e < Ne) {
                    const int ob = (q + h) * sh.sboB + jb;
                    // 2^14 T_k from its own B entries
                    const float own_r = __half2float(*reinterpret_cast<const __half *>(Bhi + ob)) +
                                        __half2float(*reinterpret_cast<const __half *>(Blo + ob));
                    const float own_i = __half2float(*reinterpret_cast<const __half *>(Bhi + ob + 16)) +
                                        __half2float(*reinterpret_cast<const __half *>(Blo + ob + 16));
                    // 2 (X t)_j = 2 ((L_j - c) t_j - i (W t)_j) / rho, D_j = 2 (W t)_j / rho
                    const float xr = fmaf(d[2 * h + 1], kT16DScaled, Lc * own_r);
                    const float xi = fmaf(-d[2 * h], kT16DScaled, Lc * own_i);
                    float *pp = prv + 2 * (q + h);
                    const float nr = first ? 0.5f * xr : xr - pp[0];
                    const float ni = first ? 0.5f * xi : xi - pp[1];
                    pp[0] = own_r;
                    pp[1] = own_i;
                    // acc += cj (-i)^(k+1) n without a branch: (ca, cbf) = cj (-i)^(k+1)
                    a[2 * h] = fmaf(ca, nr, fmaf(-cbf, ni, a[2 * h]));
                    a[2 * h + 1] = fmaf(ca, ni, fmaf(cbf, nr, a[2 * h + 1]));
                    __half2 hi2, lo2;
                    split16x2(nr, ni, hi2, lo2);
                    *reinterpret_cast<__half *>(Bhi + ob) = __low2half(hi2);
                    *reinterpret_cast<__half *>(Blo + ob) = __low2half(lo2);
                    *reinterpret_cast<__half *>(Bhi + ob + 16) = __high2half(hi2);
                    *reinterpret_cast<__half *>(Blo + ob + 16) = __high2half(lo2);
                }
            }
            tc::tmem_st4(my_lane + accc + 2 * q, a[0], a[1], a[2], a[3]);
        }
        tc::tmem_wait_st();
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok) {
        // a commit did not arrive: record it, wait once more (bounded) for
        // the MMAs in flight, and skip the write-back
        if (tid == 0) atomicOr(&s.status[t], ST_TC_WAIT);
        tc::mbar_wait(&mbar, 0u, kT16WaitLimit);
        tc::mbar_wait(&mbar, 1u, kT16WaitLimit);
    } else {
        const float sc = s_sc[1], cc = s_sc[2];
#pragma unroll
        for (int q = 0; q < kT16MaxPairs; q += 2) {
            if (q >= npair) break;  // uniform
            float a[4];
            tc::tmem_ld4(my_lane + accc + 2 * q, a[0], a[1], a[2], a[3]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = 4 * (q + h) + cg;
                if (q + h < npair && rowok && e < Ne) {
                    const float ar = a[2 * h], ai = a[2 * h + 1];
                    C[(int64_t)e * N + j] = make_float2(fmaf(cc, ar, sc * ai), fmaf(cc, ai, -(sc * ar)));
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)kT16Cols);
}

}  // namespace

size_t cheb_tc16_smem_bytes(int N, int Ne) { return (size_t)t16_shape(N, Ne).total; }

bool cheb_tc16_eligible(int N, int Ne)
{
    return N >= 2 && N <= kT16M && Ne >= 1 && Ne <= 4 * kT16MaxPairs &&
           cheb_tc16_smem_bytes(N, Ne) <= kChebTc16MaxSmem;
}

void configure_cheb_tc16()
{
    cudaFuncSetAttribute(k_cheb_tc16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChebTc16MaxSmem);
    // all of the unified L1 / shared memory as shared, so that two CTAs fit
    cudaFuncSetAttribute(k_cheb_tc16, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaGetLastError();
}

cudaError_t launch_cheb_tc16(const DevState &s, double dt, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    if (!cheb_tc16_eligible(s.N, s.Ne)) return cudaErrorInvalidValue;
    const size_t smem = cheb_tc16_smem_bytes(s.N, s.Ne);
    for (int64_t t0 = 0; t0 < s.n; t0 += 2147483647LL) {
        const int64_t cnt = (s.n - t0 < 2147483647LL) ? s.n - t0 : 2147483647LL;
        k_cheb_tc16<<<(unsigned)cnt, kT16Threads, smem, st>>>(s, dt, t0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace iesh
