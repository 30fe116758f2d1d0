// iesh_hop_gj.cu -- hop probabilities of the mixed-precision path by
// Gauss-Jordan column elimination in registers (N <= 128, Ne <= 56), and in
// registers plus shared memory for N <= 256, Ne <= 112 (k_hop_gjl).
//
// The candidate that puts orbital m in slot a has amplitude det S *
// R_{m a}, R = C_u S^{-1} (Sec. II B, determinant ratios).  Right-multiplying
// the N x Ne matrix Z = C^T (Z_{o e} = C_e(o): the rows of the occupied
// orbitals form S, the others C_u) by S^{-1} turns the S rows into the
// identity and leaves R in the unoccupied rows.  This is done by column
// operations: step i takes slot i's orbital s_i as the pivot row, chooses
// the pivot column j among the columns not chosen yet by the largest
// |Z_{s_i j}| (partial pivoting), scales column j by 1 / Z_{s_i j} and
// subtracts Z_{s_i c} times the scaled column from every other column c.
// After the Ne steps column j(i) belongs to slot i: R_{m i} = Z_{m j(i)}.
//
// Compared with an LU of S and two triangular solves per unoccupied orbital
// this does about twice the arithmetic, but every step is the same rank-one
// update of a register-resident matrix: 256 threads, thread (tr, tc) =
// (tid / 8, tid % 8) holds Z_{rc} for r = tr + 32 k (k < 4) and c = tc + 8 q
// (q < 7); the zero padding beyond N and Ne stays zero under every update.
// Per step the 8 lanes that hold the pivot row choose the pivot with a
// shuffle reduction and publish the pivot row through shared memory, each
// thread takes the pivot column's entries of its rows by a shuffle within its
// warp, and every thread updates its 28 entries: one barrier per step.  FP32 throughout
// (the coefficients are FP32 in the mixed path), the couplings d_{m, s_a}
// included: their numerators from lam - h rounded once from FP64, their
// eigenvalue gaps from double-float (hi, lo) eigenvalues, so nearly
// degenerate pairs keep FP32 relative accuracy.  The selection and the
// rescale are FP64 as in k_hop.  The skip bound of
// Sec. II C saves no work here (the elimination is the ratio solve) and is
// not applied; hop decisions are the same either way.
#include <cuda_runtime.h>
#include <stdint.h>

#include "iesh_common.cuh"
#include "iesh_hop.cuh"
#include "iesh_kernels.h"

namespace iesh {

namespace {

constexpr int kGjThreads = 256, kGjTR = 32, kGjTC = 8, kGjRPT = 4, kGjCPT = 7;
constexpr int kGjMaxN = kGjTR * kGjRPT;   // 128 orbitals
constexpr int kGjMaxNe = kGjTC * kGjCPT;  // 56 electrons

// z[k][q] for a warp-uniform q: a uniform switch, so the register array is
// never indexed at run time.
__device__ __forceinline__ float2 pick_col(const float2 (&z)[kGjRPT][kGjCPT], int k, int q)
{
    switch (q) {
    case 0: return z[k][0];
    case 1: return z[k][1];
    case 2: return z[k][2];
    case 3: return z[k][3];
    case 4: return z[k][4];
    case 5: return z[k][5];
    default: return z[k][6];
    }
}
static_assert(kGjRPT == 4 && kGjCPT == 7, "pick_col covers 4 x 7 register tiles");

template <bool EXT>
__global__ void __launch_bounds__(kGjThreads, 3) k_hop_gj(DevState s, double dt, double mass, uint64_t seed,
                                                          double *g_out)
{
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Ne = s.Ne;
    const int tid = threadIdx.x, tr = tid >> 3, tc = tid & 7;
    __shared__ float2 rowbuf[2][kGjMaxNe];
    __shared__ double lam_s[kGjMaxN], q0_s[kGjMaxN], red[64];
    __shared__ int occ_s[kGjMaxNe], slot_of[kGjMaxNe], isocc[kGjMaxN], unocc[kGjMaxN];
    __shared__ int s_j[2], s_hop_a, s_hop_m;
    __shared__ float2 s_pv[2];
    // FP32 coupling data: adsorbate components, lam - h_a, lam as (hi, lo)
    __shared__ float qa_s[kGjMaxN], qb_s[EXT ? kGjMaxN : 1], ma_s[kGjMaxN], mb_s[EXT ? kGjMaxN : 1];
    __shared__ float2 ld_s[kGjMaxN];
    const double *gv = EXT ? s.geo2 + t * 8 : s.geo + t * 4;  // h, h', kappa (EXT: h_0, h_1, projections)

    for (int i = tid; i < N; i += kGjThreads) {
        const double l = s.lam[t * N + i], qa = s.q0[t * N + i];
        lam_s[i] = l;
        q0_s[i] = qa;
        qa_s[i] = (float)qa;
        ma_s[i] = (float)(l - gv[0]);
        const float lh = (float)l;
        ld_s[i] = make_float2(lh, (float)(l - (double)lh));
        if constexpr (EXT) {
            qb_s[i] = (float)s.q2[t * N + i];
            mb_s[i] = (float)(l - gv[1]);
        }
        isocc[i] = 0;
    }
    if (tid == 0) {
        s_hop_a = -1;
        s_hop_m = -1;
    }
    __syncthreads();
    for (int a = tid; a < Ne; a += kGjThreads) {
        occ_s[a] = s.occ[t * Ne + a];
        isocc[occ_s[a]] = 1;
    }
    const float2 *Ct = reinterpret_cast<const float2 *>(s.C) + (int64_t)t * Ne * N;
    float2 z[kGjRPT][kGjCPT];
#pragma unroll
    for (int k = 0; k < kGjRPT; ++k)
#pragma unroll
        for (int q = 0; q < kGjCPT; ++q) {
            const int r = tr + kGjTR * k, c = tc + kGjTC * q;
            z[k][q] = (r < N && c < Ne) ? Ct[(int64_t)c * N + r] : make_float2(0.f, 0.f);
        }
    __syncthreads();
    if (tid == 0) {
        int u = 0;
        for (int m = 0; m < N; ++m)
            if (!isocc[m]) unocc[u++] = m;
    }

    // ---- elimination: one barrier per step.  The 8 lanes holding the next
    // pivot row choose its pivot right after their own update and publish
    // the pivot and the row (double-buffered); every thread takes column j
    // of its rows from the lane of its row class that holds it (a shuffle).
    unsigned used = 0;  // bit q: my column tc + 8 q is a pivot column already
    bool singular = false;
    auto search = [&](int i) {
        const int p = occ_s[i], kp = p / kGjTR;
        if (tr != (p & (kGjTR - 1))) return;  // the 8 lanes holding row p (an aligned group)
        float2 row[kGjCPT];  // my entries of row p (kp is uniform: one switch)
        switch (kp) {
        case 0:
#pragma unroll
            for (int q = 0; q < kGjCPT; ++q) row[q] = z[0][q];
            break;
        case 1:
#pragma unroll
            for (int q = 0; q < kGjCPT; ++q) row[q] = z[1][q];
            break;
        case 2:
#pragma unroll
            for (int q = 0; q < kGjCPT; ++q) row[q] = z[2][q];
            break;
        default:
#pragma unroll
            for (int q = 0; q < kGjCPT; ++q) row[q] = z[3][q];
        }
        int bk = -1, bc = kGjMaxNe;
#pragma unroll
        for (int q = 0; q < kGjCPT; ++q) {
            const int key = ((used >> q) & 1u) ? -1 : pivot_key(row[q]);
            if (key > bk) {  // ascending columns: ties keep the lower one
                bk = key;
                bc = tc + kGjTC * q;
            }
        }
        const unsigned grp = 0xFFu << ((tid & 31) & ~7);
#pragma unroll
        for (int o = 1; o < kGjTC; o <<= 1) {
            const int ok = __shfl_xor_sync(grp, bk, o), oc = __shfl_xor_sync(grp, bc, o);
            if (ok > bk || (ok == bk && oc < bc)) {
                bk = ok;
                bc = oc;
            }
        }
        const int buf = i & 1;
        if (tc == 0) s_j[buf] = bk > 0 ? bc : -1;  // key 0: the row of S is zero in every free column
#pragma unroll
        for (int q = 0; q < kGjCPT; ++q) {
            float2 v = row[q];
            if (tc + kGjTC * q == bc) {  // the lane holding the pivot
                s_pv[buf] = v;
                // the pivot column itself: z - (pv - 1) z / pv = z / pv
                v = make_float2(v.x - 1.f, v.y);
            }
            rowbuf[buf][tc + kGjTC * q] = v;
        }
    };
    search(0);
    __syncthreads();
    const int src0 = (tid & 31) & ~7;  // first lane of my row class
    for (int i = 0; i < Ne; ++i) {
        const int buf = i & 1;
        const int j = s_j[buf];
        if (j < 0) {  // uniform: every thread read the same s_j
            singular = true;
            break;
        }
        const float2 pinv = crcp(s_pv[buf]);
        const int qj = j / kGjTC;
        if (tc == (j & (kGjTC - 1))) used |= 1u << qj;
        if (tid == 0) slot_of[j] = i;
        float2 cb[kGjRPT];
#pragma unroll
        for (int k = 0; k < kGjRPT; ++k) {
            const float2 v = pick_col(z, k, qj);
            const float vx = __shfl_sync(0xffffffffu, v.x, src0 | (j & (kGjTC - 1)));
            const float vy = __shfl_sync(0xffffffffu, v.y, src0 | (j & (kGjTC - 1)));
            cb[k] = cmul(make_float2(vx, vy), pinv);
        }
#pragma unroll
        for (int k = 0; k < kGjRPT; ++k)
#pragma unroll
            for (int q = 0; q < kGjCPT; ++q) z[k][q] = cfms(z[k][q], rowbuf[buf][tc + kGjTC * q], cb[k]);
        if (i + 1 < Ne) search(i + 1);
        __syncthreads();
    }
    if (singular && tid == 0) atomicOr(&s.status[t], ST_SINGULAR);

    // ---- probabilities g_{a->m} = max(0, -2 dt v Re(R_ma) d_{m, s_a})
    const double v = EXT ? 1.0 : s.p[t] / mass;  // the six-coordinate coupling carries its velocity
    const double geo_h = gv[0], geo_dh = gv[1], geo_k = gv[2];
    const float fac = (float)(-2.0 * dt * v);
    // numerator factors: h' + kappa (.) (EXT: the two orbitals' projections)
    const float ha = (float)(EXT ? gv[2] : gv[1]), ka = (float)(EXT ? gv[4] : gv[2]);
    const float hb = (float)(EXT ? gv[3] : 0.0), kb = (float)(EXT ? gv[5] : 0.0);
    double *scr = s.scratch + t * s.scratch_stride;
    double *G = g_out ? g_out + (int64_t)t * Ne * N : scr + 2 * (int64_t)Ne * N;  // [Ne][N]
    if (!singular) {
#pragma unroll
        for (int k = 0; k < kGjRPT; ++k) {
            const int m = tr + kGjTR * k;
            if (m < N && !isocc[m]) {
#pragma unroll
                for (int q = 0; q < kGjCPT; ++q) {
                    const int c = tc + kGjTC * q;
                    if (c < Ne) {
                        const int a = slot_of[c], sa = occ_s[a];
                        // T_{m s_a} (times v for EXT) and lam_{s_a} - lam_m in FP32
                        float T = qa_s[m] * qa_s[sa] * fmaf(ka, ma_s[m] + ma_s[sa], ha);
                        if constexpr (EXT) T = fmaf(qb_s[m] * qb_s[sa], fmaf(kb, mb_s[m] + mb_s[sa], hb), T);
                        const float2 lm = ld_s[m], ls = ld_s[sa];
                        const float gap = (ls.x - lm.x) + (ls.y - lm.y);
                        const float gam = fac * z[k][q].x * __fdividef(T, gap);  // at most 2 ulp
                        G[(int64_t)a * N + m] = gam > 0.f ? (double)gam : 0.0;
                    }
                }
            }
        }
        if (g_out)
            for (int idx = tid; idx < Ne * Ne; idx += kGjThreads) G[(int64_t)(idx / Ne) * N + occ_s[idx % Ne]] = 0.0;
    } else if (g_out) {
        for (int idx = tid; idx < Ne * N; idx += kGjThreads) G[idx] = 0.0;
    }
    __syncthreads();
    if (g_out) return;
    const U4 rn = draw_traj(s, seed, t, kStreamHop, (uint64_t)s.nstep[t]);
    const double zeta = u53(rn.v[0], rn.v[1]);
    hop_finish<float2, EXT>(s, t, mass, zeta, !singular, G, red, scr, unocc, occ_s, lam_s, q0_s, geo_h, geo_dh,
                            geo_k, s_hop_a, s_hop_m, Ct);
}

// ------------------------------------------------------------ large shapes
// The same elimination for N <= 256 and Ne <= 112 (k_hop_gjl): 512 threads,
// thread (tr, tc) = (tid / 16, tid % 16) holds Z_{rc} for c = tc + 16 q
// (q < 7) and r = tr + 32 k (k < 4) in registers, and r = 128 + tr + 32 k in
// shared memory (zs, rows 128 .. N - 1, 112 columns each), where its 16-lane
// row class reads and writes whole 128-byte lines.  A step takes the pivot
// column of the shared rows from zs and of the register rows by a shuffle
// within the half warp; a warp barrier separates those reads from the
// updates.  One block barrier per step, as above.
constexpr int kGlThreads = 512, kGlTR = 32, kGlTC = 16, kGlRPT = 4, kGlCPT = 7;
constexpr int kGlRegRows = kGlTR * kGlRPT;  // 128 rows in registers
static_assert(kGlRPT == kGjRPT && kGlCPT == kGjCPT, "pick_col serves both register tiles");
constexpr int kGlMaxN = 2 * kGlRegRows;     // 256 orbitals
constexpr int kGlMaxNe = kGlTC * kGlCPT;    // 112 electrons

template <bool EXT>
__global__ void __launch_bounds__(kGlThreads, 1) k_hop_gjl(DevState s, double dt, double mass, uint64_t seed,
                                                           double *g_out)
{
    extern __shared__ __align__(16) float2 zs[];  // [N - 128][kGlMaxNe]
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Ne = s.Ne;
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    __shared__ float2 rowbuf[2][kGlMaxNe];
    __shared__ double lam_s[kGlMaxN], q0_s[kGlMaxN], red[64];
    __shared__ int occ_s[kGlMaxNe], slot_of[kGlMaxNe], isocc[kGlMaxN], unocc[kGlMaxN];
    __shared__ int s_j[2], s_hop_a, s_hop_m;
    __shared__ float2 s_pv[2];
    __shared__ float qa_s[kGlMaxN], qb_s[EXT ? kGlMaxN : 1], ma_s[kGlMaxN], mb_s[EXT ? kGlMaxN : 1];
    __shared__ float2 ld_s[kGlMaxN];
    const double *gv = EXT ? s.geo2 + t * 8 : s.geo + t * 4;

    for (int i = tid; i < N; i += kGlThreads) {
        const double l = s.lam[t * N + i], qa = s.q0[t * N + i];
        lam_s[i] = l;
        q0_s[i] = qa;
        qa_s[i] = (float)qa;
        ma_s[i] = (float)(l - gv[0]);
        const float lh = (float)l;
        ld_s[i] = make_float2(lh, (float)(l - (double)lh));
        if constexpr (EXT) {
            qb_s[i] = (float)s.q2[t * N + i];
            mb_s[i] = (float)(l - gv[1]);
        }
        isocc[i] = 0;
    }
    if (tid == 0) {
        s_hop_a = -1;
        s_hop_m = -1;
    }
    __syncthreads();
    for (int a = tid; a < Ne; a += kGlThreads) {
        occ_s[a] = s.occ[t * Ne + a];
        isocc[occ_s[a]] = 1;
    }
    const float2 *Ct = reinterpret_cast<const float2 *>(s.C) + (int64_t)t * Ne * N;
    float2 z[kGlRPT][kGlCPT];
#pragma unroll
    for (int k = 0; k < kGlRPT; ++k)
#pragma unroll
        for (int q = 0; q < kGlCPT; ++q) {
            const int r = tr + kGlTR * k, c = tc + kGlTC * q;
            z[k][q] = (r < N && c < Ne) ? Ct[(int64_t)c * N + r] : make_float2(0.f, 0.f);
        }
    for (int k = 0; k < kGlRPT; ++k) {
        const int r = kGlRegRows + tr + kGlTR * k;
        if (r < N)
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) {
                const int c = tc + kGlTC * q;
                zs[(r - kGlRegRows) * kGlMaxNe + c] = c < Ne ? Ct[(int64_t)c * N + r] : make_float2(0.f, 0.f);
            }
    }
    __syncthreads();
    if (tid == 0) {
        int u = 0;
        for (int m = 0; m < N; ++m)
            if (!isocc[m]) unocc[u++] = m;
    }

    unsigned used = 0;  // bit q: my column tc + 16 q is a pivot column already
    bool singular = false;
    auto search = [&](int i) {
        const int p = occ_s[i], kp = p / kGlTR;
        if (tr != (p & (kGlTR - 1))) return;  // the 16 lanes holding row p (a half warp)
        float2 row[kGlCPT];
        switch (kp) {
        case 0:
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) row[q] = z[0][q];
            break;
        case 1:
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) row[q] = z[1][q];
            break;
        case 2:
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) row[q] = z[2][q];
            break;
        case 3:
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) row[q] = z[3][q];
            break;
        default:
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) row[q] = zs[(p - kGlRegRows) * kGlMaxNe + tc + kGlTC * q];
        }
        int bk = -1, bc = kGlMaxNe;
#pragma unroll
        for (int q = 0; q < kGlCPT; ++q) {
            const int key = ((used >> q) & 1u) ? -1 : pivot_key(row[q]);
            if (key > bk) {  // ascending columns: ties keep the lower one
                bk = key;
                bc = tc + kGlTC * q;
            }
        }
        const unsigned grp = 0xFFFFu << ((tid & 31) & ~15);
#pragma unroll
        for (int o = 1; o < kGlTC; o <<= 1) {
            const int ok = __shfl_xor_sync(grp, bk, o), oc = __shfl_xor_sync(grp, bc, o);
            if (ok > bk || (ok == bk && oc < bc)) {
                bk = ok;
                bc = oc;
            }
        }
        const int buf = i & 1;
        if (tc == 0) s_j[buf] = bk > 0 ? bc : -1;  // key 0: the row of S is zero in every free column
#pragma unroll
        for (int q = 0; q < kGlCPT; ++q) {
            float2 v = row[q];
            if (tc + kGlTC * q == bc) {  // the lane holding the pivot
                s_pv[buf] = v;
                v = make_float2(v.x - 1.f, v.y);  // the pivot column: z - (pv - 1) z / pv = z / pv
            }
            rowbuf[buf][tc + kGlTC * q] = v;
        }
    };
    search(0);
    __syncthreads();
    const int src0 = (tid & 31) & ~15;  // first lane of my row class
    for (int i = 0; i < Ne; ++i) {
        const int buf = i & 1;
        const int j = s_j[buf];
        if (j < 0) {  // uniform: every thread read the same s_j
            singular = true;
            break;
        }
        const float2 pinv = crcp(s_pv[buf]);
        const int qj = j / kGlTC;
        if (tc == (j & (kGlTC - 1))) used |= 1u << qj;
        if (tid == 0) slot_of[j] = i;
        float2 cb[2 * kGlRPT];
#pragma unroll
        for (int k = 0; k < kGlRPT; ++k) {
            const float2 v = pick_col(z, k, qj);
            const float vx = __shfl_sync(0xffffffffu, v.x, src0 | (j & (kGlTC - 1)));
            const float vy = __shfl_sync(0xffffffffu, v.y, src0 | (j & (kGlTC - 1)));
            cb[k] = cmul(make_float2(vx, vy), pinv);
        }
#pragma unroll
        for (int k = 0; k < kGlRPT; ++k) {
            const int r = kGlRegRows + tr + kGlTR * k;
            cb[kGlRPT + k] = r < N ? cmul(zs[(r - kGlRegRows) * kGlMaxNe + j], pinv) : make_float2(0.f, 0.f);
        }
        __syncwarp();  // the pivot column is read before its lane rewrites it
#pragma unroll
        for (int k = 0; k < kGlRPT; ++k)
#pragma unroll
            for (int q = 0; q < kGlCPT; ++q) z[k][q] = cfms(z[k][q], rowbuf[buf][tc + kGlTC * q], cb[k]);
#pragma unroll
        for (int k = 0; k < kGlRPT; ++k) {
            const int r = kGlRegRows + tr + kGlTR * k;
            if (r < N) {
                float2 *zr = zs + (r - kGlRegRows) * kGlMaxNe + tc;
#pragma unroll
                for (int q = 0; q < kGlCPT; ++q) zr[kGlTC * q] = cfms(zr[kGlTC * q], rowbuf[buf][tc + kGlTC * q], cb[kGlRPT + k]);
            }
        }
        if (i + 1 < Ne) search(i + 1);
        __syncthreads();
    }
    if (singular && tid == 0) atomicOr(&s.status[t], ST_SINGULAR);

    // ---- probabilities g_{a->m} = max(0, -2 dt v Re(R_ma) d_{m, s_a})
    const double v = EXT ? 1.0 : s.p[t] / mass;
    const double geo_h = gv[0], geo_dh = gv[1], geo_k = gv[2];
    const float fac = (float)(-2.0 * dt * v);
    const float ha = (float)(EXT ? gv[2] : gv[1]), ka = (float)(EXT ? gv[4] : gv[2]);
    const float hb = (float)(EXT ? gv[3] : 0.0), kb = (float)(EXT ? gv[5] : 0.0);
    double *scr = s.scratch + t * s.scratch_stride;
    double *G = g_out ? g_out + (int64_t)t * Ne * N : scr + 2 * (int64_t)Ne * N;  // [Ne][N]
    auto emit = [&](int m, int c, float zr) {
        const int a = slot_of[c], sa = occ_s[a];
        float T = qa_s[m] * qa_s[sa] * fmaf(ka, ma_s[m] + ma_s[sa], ha);
        if constexpr (EXT) T = fmaf(qb_s[m] * qb_s[sa], fmaf(kb, mb_s[m] + mb_s[sa], hb), T);
        const float2 lm = ld_s[m], ls = ld_s[sa];
        const float gap = (ls.x - lm.x) + (ls.y - lm.y);
        const float gam = fac * zr * __fdividef(T, gap);  // at most 2 ulp
        G[(int64_t)a * N + m] = gam > 0.f ? (double)gam : 0.0;
    };
    if (!singular) {
#pragma unroll
        for (int k = 0; k < kGlRPT; ++k) {
            const int m = tr + kGlTR * k;
            if (m < N && !isocc[m])
#pragma unroll
                for (int q = 0; q < kGlCPT; ++q)
                    if (tc + kGlTC * q < Ne) emit(m, tc + kGlTC * q, z[k][q].x);
        }
        for (int k = 0; k < kGlRPT; ++k) {
            const int m = kGlRegRows + tr + kGlTR * k;
            if (m < N && !isocc[m])
#pragma unroll
                for (int q = 0; q < kGlCPT; ++q)
                    if (tc + kGlTC * q < Ne)
                        emit(m, tc + kGlTC * q, zs[(m - kGlRegRows) * kGlMaxNe + tc + kGlTC * q].x);
        }
        if (g_out)
            for (int idx = tid; idx < Ne * Ne; idx += kGlThreads) G[(int64_t)(idx / Ne) * N + occ_s[idx % Ne]] = 0.0;
    } else if (g_out) {
        for (int idx = tid; idx < Ne * N; idx += kGlThreads) G[idx] = 0.0;
    }
    __syncthreads();
    if (g_out) return;
    const U4 rn = draw_traj(s, seed, t, kStreamHop, (uint64_t)s.nstep[t]);
    const double zeta = u53(rn.v[0], rn.v[1]);
    hop_finish<float2, EXT>(s, t, mass, zeta, !singular, G, red, scr, unocc, occ_s, lam_s, q0_s, geo_h, geo_dh,
                            geo_k, s_hop_a, s_hop_m, Ct);
}

size_t gjl_smem_bytes(int N) { return (size_t)(N > kGlRegRows ? N - kGlRegRows : 1) * kGlMaxNe * sizeof(float2); }

}  // namespace

bool hop_gj_eligible(int N, int Ne) { return N <= kGjMaxN && Ne <= kGjMaxNe && Ne < N; }

bool hop_gjl_eligible(int N, int Ne) { return N <= kGlMaxN && Ne <= kGlMaxNe && Ne < N; }

void configure_hop_gjl()
{
    cudaFuncSetAttribute(k_hop_gjl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gjl_smem_bytes(kGlMaxN));
    cudaFuncSetAttribute(k_hop_gjl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gjl_smem_bytes(kGlMaxN));
    cudaGetLastError();
}

cudaError_t launch_hop_gjl(const DevState &s, double dt, double mass, uint64_t seed, double *g_out,
                           cudaStream_t st, bool ext)
{
    if (s.n == 0) return cudaSuccess;
    if (!hop_gjl_eligible(s.N, s.Ne)) return cudaErrorInvalidValue;
    const size_t smem = gjl_smem_bytes(s.N);
    if (ext) k_hop_gjl<true><<<(unsigned)s.n, kGlThreads, smem, st>>>(s, dt, mass, seed, g_out);
    else k_hop_gjl<false><<<(unsigned)s.n, kGlThreads, smem, st>>>(s, dt, mass, seed, g_out);
    return cudaGetLastError();
}

cudaError_t launch_hop_gj(const DevState &s, double dt, double mass, uint64_t seed, double *g_out,
                          cudaStream_t st, bool ext)
{
    if (s.n == 0) return cudaSuccess;
    if (!hop_gj_eligible(s.N, s.Ne)) return cudaErrorInvalidValue;
    if (ext) k_hop_gj<true><<<(unsigned)s.n, kGjThreads, 0, st>>>(s, dt, mass, seed, g_out);
    else k_hop_gj<false><<<(unsigned)s.n, kGjThreads, 0, st>>>(s, dt, mass, seed, g_out);
    return cudaGetLastError();
}

}  // namespace iesh
