// iesh_cheb_tc.cu -- Chebyshev propagator of the mixed-precision path on the
// tensor cores (tcgen05, kind::tf32), for N <= 128 orbitals and Ne <= 56.
//
// The exponential integrator of Sec. II C applied to the N x Ne coefficient
// matrix, as in the SIMT kernels: with H = Abar dt = L - i W (L diagonal,
// W the real antisymmetric step-averaged coupling generator) inside
// [c - rho, c + rho],
//   exp(-i H) C = e^{-ic} sum_k (2 - delta_k0) (-i)^k J_k(rho) T_k(X) C,
//   X = (H - c) / rho,  T_{k+1} = 2 X T_k - T_{k-1}.
// The dense contraction of every order, (W T_k) with T_k viewed as the real
// N x 2Ne matrix [Re t_e, Im t_e]_e, runs on the tensor cores as
// D = W T_k (M = 128 rows >= N, K = N rounded up to 8, N_mma = 2Ne rounded
// up to 16).  FP32 accuracy comes from the 3xTF32 split: W = W_hi + W_lo and
// T = T_hi + T_lo with TF32 high parts, D = W_hi T_hi + W_hi T_lo + W_lo T_hi
// accumulated in FP32 in tensor memory (the dropped W_lo T_lo term is about
// 2^-22 of |W| |T|).  A .tf32 operand uses the top 19 bits of each 32-bit
// element, so the high planes hold the FP32 values themselves (read as
// their truncation) and the low planes x - trunc(x).  W enters scaled by
// 2 / rho, which folds the recurrence's factor into the contraction.
//
// One CTA per trajectory, 512 threads: warp w reads TMEM lanes 32 (w % 4)
// .. +31, i.e. orbital row j = 32 (w % 4) + lane, and owns the column
// quarter w / 4 of the 2Ne real columns.  Each order: one thread issues the
// 3 x K/8 MMAs and commits them to an mbarrier; every thread waits (bounded),
// loads its D entries from tensor memory, forms T_{k+1} for its row and
// columns (T_{k-1} and the Chebyshev sum kept in registers, T_k read back
// from the high plane of the B operand), and
// rewrites its entries of the B operand in place (nobody else reads them
// once the MMAs of the order have completed).
//
// Shared memory (bytes): A = W_hi, W_lo: 2 x 16 x (K/4) x 128; B = T_hi,
// T_lo: 2 x (Nmma/8) x (K/4) x 144.  The 16-byte gap after every core
// matrix of B (LBO = 144) puts the 8 K-chunks touched by a warp (32
// consecutive rows j of one column) on distinct banks.
#include <cuda_runtime.h>
#include <stdint.h>

#include "iesh_common.cuh"
#include "iesh_kernels.h"
#include "iesh_tc.cuh"

namespace iesh {

namespace {

constexpr int kTcM = 128;          // MMA rows (orbitals, padded)
constexpr int kTcThreads = 512;    // 4 lane quarters x 4 column groups
constexpr int kTcMaxChunks = 7;    // 4-column chunks per thread: 2 Ne <= 112
constexpr int kTcLboA = 128, kTcLboB = 144;
constexpr int kTcWaitLimit = 1 << 22;

struct TcShape {
    int Kp, NB, cpt, sboA, sboB, bytesA, bytesB, ncols;
};

__host__ __device__ inline TcShape tc_shape(int N, int Ne)
{
    TcShape t;
    t.Kp = (N + 7) & ~7;
    t.NB = (2 * Ne + 15) & ~15;
    t.cpt = t.NB / 4;
    t.sboA = (t.Kp / 4) * kTcLboA;
    t.sboB = (t.Kp / 4) * kTcLboB;
    t.bytesA = (kTcM / 8) * t.sboA;
    t.bytesB = (t.NB / 8) * t.sboB;
    int c = 32;
    while (c < t.NB) c <<= 1;
    t.ncols = c;
    return t;
}

__device__ __forceinline__ int offA(const TcShape &sh, int row, int k)
{
    return (row >> 3) * sh.sboA + (k >> 2) * kTcLboA + (row & 7) * 16 + (k & 3) * 4;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_cheb_tc(DevState s, double dt, int64_t t_base)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    // per-trajectory scalars in FP32, formed once (FP64 work costs every warp
    // that issues it): 2 J_k, 1 / rho, sin c, cos c
    __shared__ float s_cj[kChebMax], s_sc[3];
    const int64_t t = traj_of(s, t_base + blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;  // uniform over the CTA
    const int N = s.N, Ne = s.Ne, Np = (N + 3) & ~3;
    const TcShape sh = tc_shape(N, Ne);
    unsigned char *Ahi = tc_smem, *Alo = tc_smem + sh.bytesA;
    unsigned char *Bhi = tc_smem + 2 * sh.bytesA, *Blo = Bhi + sh.bytesB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = 32 * (warp & 3) + lane;  // my orbital row = my TMEM lane
    const int cg = warp >> 2;              // my column quarter
    const int c0 = cg * sh.cpt;
    const int nch = sh.cpt / 4;
    const bool rowok = j < N;

    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc(&tmem_slot, (uint32_t)sh.ncols);

    // A operand: (2 / rho) W (rows j, columns i; stored [N][Np]) as TF32
    // high part (the FP32 value itself) and low part.  The scale folds the
    // recurrence's 2 / rho into the contraction.  Every 16-byte piece (row
    // j, 4 consecutive columns: one core-matrix row) is copied by cp.async
    // into the high plane, all of them in flight at once, zero-filled past
    // N rows and Np columns; each thread then scales its own pieces in
    // place and forms their low parts.
    const float *__restrict__ W = reinterpret_cast<const float *>(s.scratch + t * s.scratch_stride);
    const double rho0 = s.cheb[t * kChebStride + 1];
    const float w2 = rho0 > 0.0 ? 2.0f / (float)rho0 : 0.0f;
    // piece pc: 8-row group pc / (8 kch), then column quad, then row, so that
    // 8 consecutive threads fill one 128-byte core matrix
    const int kch = sh.Kp / 4, npc = kTcM * kch;  // 16-byte pieces of a plane
    auto piece = [&](int pc, int &row, int &kc) {
        const int rg = pc / (8 * kch), w = pc - rg * 8 * kch;
        kc = w >> 3;
        row = 8 * rg + (w & 7);
    };
    for (int pc = tid; pc < npc; pc += kTcThreads) {
        int row, kc;
        piece(pc, row, kc);
        const bool in = row < N && 4 * kc < Np;
        cp_async16_zfill(Ahi + offA(sh, row, 4 * kc), in ? W + (int64_t)row * Np + 4 * kc : W, in ? 16u : 0u);
    }
    cp_async_commit();
    cp_async_wait<0>();
    for (int pc = tid; pc < npc; pc += kTcThreads) {
        int row, kc;
        piece(pc, row, kc);
        float4 *h = reinterpret_cast<float4 *>(Ahi + offA(sh, row, 4 * kc));
        const float4 v = *h;
        const float4 a = make_float4(w2 * v.x, w2 * v.y, w2 * v.z, w2 * v.w);
        *h = a;
        *reinterpret_cast<float4 *>(Alo + offA(sh, row, 4 * kc)) =
            make_float4(tc::lo_tf32(a.x), tc::lo_tf32(a.y), tc::lo_tf32(a.z), tc::lo_tf32(a.w));
    }
    // B operand rows (columns of T) beyond 2Ne and K entries beyond N stay zero
    {
        const int words = 2 * sh.bytesB / 4;
        float *B = reinterpret_cast<float *>(Bhi);
        for (int w = tid; w < words; w += kTcThreads) B[w] = 0.0f;
    }
    __syncthreads();

    const double *cb = s.cheb + t * kChebStride;
    const double c = cb[0];
    const int K = (int)cb[2];
    const double *J = cb + 3;
    for (int q = tid; q <= K; q += kTcThreads) s_cj[q] = (float)(2.0 * J[q]);
    if (tid == 0) {
        double scd, ccd;
        sincos(c, &scd, &ccd);
        s_sc[1] = (float)scd;
        s_sc[2] = (float)ccd;
    }
    float2 *C = reinterpret_cast<float2 *>(s.C) + (int64_t)t * Ne * N;
    // 2 (L_j - c) / rho, the diagonal's share of 2 X
    const float Lc = rowok ? w2 * (float)(0.5 * dt * (s.lam_prev[t * N + j] + s.lam[t * N + j]) - c) : 0.0f;
    const float J0 = (float)J[0];

    // T_0 = C: my row, my columns.  B entry (col, j) of this thread sits at
    // colpart(col) + jb; col and col + 1 (one electron) share an 8-column
    // group, 16 bytes apart.
    const int jb = (j >> 2) * kTcLboB + (j & 3) * 4;
    const int loB = sh.bytesB;  // T_lo follows T_hi
    float prv[4 * kTcMaxChunks], acc[4 * kTcMaxChunks];
#pragma unroll
    for (int ch = 0; ch < kTcMaxChunks; ++ch) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = c0 + 4 * ch + 2 * h, e = col >> 1;
            const bool mine = ch < nch && rowok && e < Ne;
            float2 v = make_float2(0.f, 0.f);
            if (mine) v = C[(int64_t)e * N + j];
            prv[4 * ch + 2 * h] = 0.f;
            prv[4 * ch + 2 * h + 1] = 0.f;
            acc[4 * ch + 2 * h] = J0 * v.x;
            acc[4 * ch + 2 * h + 1] = J0 * v.y;  // single products: no contraction possible
            if (mine) {
                unsigned char *b0 = Bhi + (col >> 3) * sh.sboB + (col & 7) * 16 + jb;
                *reinterpret_cast<float *>(b0) = v.x;
                *reinterpret_cast<float *>(b0 + loB) = tc::lo_tf32(v.x);
                *reinterpret_cast<float *>(b0 + 16) = v.y;
                *reinterpret_cast<float *>(b0 + loB + 16) = tc::lo_tf32(v.y);
            }
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc::idesc_tf32(kTcM, sh.NB);
    const uint32_t aHi = tc::smem_addr(Ahi), aLo = tc::smem_addr(Alo);
    const uint32_t bHi = tc::smem_addr(Bhi), bLo = tc::smem_addr(Blo);
    const uint32_t my_lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);

    bool ok = true;
    for (int k = 0; k < K; ++k) {
        if (tid == 0) {
            // D = W_hi T_hi + W_hi T_lo + W_lo T_hi
            uint32_t accum = 0;
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t a = pass == 2 ? aLo : aHi, b = pass == 1 ? bLo : bHi;
                for (int ks = 0; ks < sh.Kp / 8; ++ks) {
                    tc::mma_tf32(tmem, tc::smem_desc(a + ks * 2 * kTcLboA, kTcLboA, sh.sboA),
                                 tc::smem_desc(b + ks * 2 * kTcLboB, kTcLboB, sh.sboB), idesc, accum);
                    accum = 1;
                }
            }
            tc::commit(&mbar);
        }
        const bool done = tc::mbar_wait(&mbar, (uint32_t)(k & 1), kTcWaitLimit);
        if (__syncthreads_or(!done)) {
            ok = false;
            break;
        }
        tc::fence_after_sync();
        const float cj = s_cj[k + 1];
        const int ph = (k + 1) & 3;  // (-i)^(k+1) = (1, 0), (0, -1), (-1, 0), (0, 1)
        const float ca = ph == 0 ? cj : (ph == 2 ? -cj : 0.f), cb = ph == 1 ? -cj : (ph == 3 ? cj : 0.f);
        const bool first = k == 0;
        // D entries in flight four chunks at a time, one wait per group
        float dv[16];
#pragma unroll
        for (int ch = 0; ch < kTcMaxChunks; ++ch) {
            if ((ch & 3) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (ch + q < nch && ch + q < kTcMaxChunks)  // warp-uniform
                        tc::tmem_ld4(my_lane_addr + (uint32_t)(c0 + 4 * (ch + q)), dv[4 * q], dv[4 * q + 1],
                                     dv[4 * q + 2], dv[4 * q + 3]);
                tc::tmem_wait_ld();
            }
            if (ch < nch) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int col = c0 + 4 * ch + 2 * h, e = col >> 1;
                    if (rowok && e < Ne) {
                        const float *d = dv + 4 * (ch & 3) + 2 * h;
                        float *pp = prv + 4 * ch + 2 * h, *aa = acc + 4 * ch + 2 * h;
                        unsigned char *b0 = Bhi + (col >> 3) * sh.sboB + (col & 7) * 16 + jb;
                        // T_k exactly: the high operand is the FP32 value
                        const float own_r = *reinterpret_cast<const float *>(b0);
                        const float own_i = *reinterpret_cast<const float *>(b0 + 16);
                        // 2 (X t)_j = 2 ((L_j - c) t_j - i (W t)_j) / rho, D_j = 2 (W t)_j / rho
                        const float xr = fmaf(Lc, own_r, d[1]);
                        const float xi = fmaf(Lc, own_i, -d[0]);
                        const float nr = first ? 0.5f * xr : xr - pp[0];
                        const float ni = first ? 0.5f * xi : xi - pp[1];
                        pp[0] = own_r;
                        pp[1] = own_i;
                        // acc += cj (-i)^(k+1) n without a branch: (ca, cb) = cj (-i)^(k+1)
                        aa[0] = fmaf(ca, nr, fmaf(-cb, ni, aa[0]));
                        aa[1] = fmaf(ca, ni, fmaf(cb, nr, aa[1]));
                        *reinterpret_cast<float *>(b0) = nr;
                        *reinterpret_cast<float *>(b0 + loB) = tc::lo_tf32(nr);
                        *reinterpret_cast<float *>(b0 + 16) = ni;
                        *reinterpret_cast<float *>(b0 + loB + 16) = tc::lo_tf32(ni);
                    }
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok) {
        // a commit did not arrive: record it, wait once more (bounded) for
        // the MMAs in flight, and skip the write-back
        if (tid == 0) atomicOr(&s.status[t], ST_TC_WAIT);
        tc::mbar_wait(&mbar, 0u, kTcWaitLimit);
        tc::mbar_wait(&mbar, 1u, kTcWaitLimit);
    } else if (rowok) {
        const float sc = s_sc[1], cc = s_sc[2];
#pragma unroll
        for (int ch = 0; ch < kTcMaxChunks; ++ch)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = (c0 + 4 * ch + 2 * h) >> 1;
                if (ch < nch && e < Ne) {
                    const float ar = acc[4 * ch + 2 * h], ai = acc[4 * ch + 2 * h + 1];
                    C[(int64_t)e * N + j] = make_float2(fmaf(cc, ar, sc * ai), fmaf(cc, ai, -(sc * ar)));
                }
            }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)sh.ncols);
}

}  // namespace

size_t cheb_tc_smem_bytes(int N, int Ne)
{
    const TcShape sh = tc_shape(N, Ne);
    return (size_t)2 * sh.bytesA + (size_t)2 * sh.bytesB;
}

bool cheb_tc_eligible(int N, int Ne)
{
    return N >= 2 && N <= kTcM && Ne >= 1 && 2 * Ne <= 4 * 4 * kTcMaxChunks &&
           cheb_tc_smem_bytes(N, Ne) <= kChebTcMaxSmem;
}

void configure_cheb_tc()
{
    cudaFuncSetAttribute(k_cheb_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChebTcMaxSmem);
    cudaGetLastError();
}

cudaError_t launch_cheb_tc(const DevState &s, double dt, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    if (!cheb_tc_eligible(s.N, s.Ne)) return cudaErrorInvalidValue;
    const size_t smem = cheb_tc_smem_bytes(s.N, s.Ne);
    for (int64_t t0 = 0; t0 < s.n; t0 += 2147483647LL) {
        const int64_t cnt = (s.n - t0 < 2147483647LL) ? s.n - t0 : 2147483647LL;
        k_cheb_tc<<<(unsigned)cnt, kTcThreads, smem, st>>>(s, dt, t0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace iesh
