// iesh_hop.cuh -- pieces shared by the hop kernels (internal): complex
// arithmetic in FP64 and FP32, pivot keys, the closed-form coupling of the
// one-coordinate model, and the stochastic selection, momentum rescale and
// bookkeeping that follow the hop probabilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "iesh_common.cuh"
#include "iesh_secular.cuh"

namespace iesh {

// d_jk = <j|d_x k> = T_jk / (lam_k - lam_j) with the closed form of
// T = Q^T (dH/dx) Q for the arrowhead: T_jk = q0_j q0_k [h' + kappa
// (lam_j + lam_k - 2h)], kappa = f'/f (all couplings share f(x)).
__device__ __forceinline__ double nac(double lj, double qj, double lk, double qk, double h,
                                      double dh, double kap)
{
    return qj * qk * (dh + kap * (lj + lk - 2.0 * h)) * pole_recip<double>(lk - lj);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfms(double2 acc, double2 a, double2 b)  // acc - a b
{
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 crcp(double2 a)
{
    const double m = fma(a.x, a.x, a.y * a.y);
    const double d = m >= 2.2250738585072014e-308 ? pole_recip<double>(m) : 1.0 / m;
    return make_double2(a.x * d, -a.y * d);
}
// Pivot key of a complex entry: max(|re|, |im|) to 20 mantissa bits, from
// the high words of the doubles (integer ops: the FP64 pipe is the
// bottleneck of the factorisation).  Monotonic in the magnitude; 0 only for
// zero (or below 2^-1042) entries; -1 marks "no candidate".
__device__ __forceinline__ int pivot_key(double2 v)
{
    const int a = __double2hiint(v.x) & 0x7fffffff, b = __double2hiint(v.y) & 0x7fffffff;
    return a > b ? a : b;
}
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfmsf(float2 acc, float2 a, float2 b)  // acc - a b
{
    return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
// FP32 factorisation (mixed path): the same operations in single precision.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return cmulf(a, b); }
__device__ __forceinline__ float2 cfms(float2 acc, float2 a, float2 b) { return cfmsf(acc, a, b); }
__device__ __forceinline__ float2 crcp(float2 a)
{
    const float d = 1.0f / fmaf(a.x, a.x, a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ int pivot_key(float2 v)  // max(|re|, |im|), monotonic
{
    const int a = __float_as_int(v.x) & 0x7fffffff, b = __float_as_int(v.y) & 0x7fffffff;
    return a > b ? a : b;
}


// After the hop probabilities G[a][m] (slot a, orbital m; FP64, written and
// followed by a barrier): the selection with one uniform zeta in the order
// (slot a ascending, m ascending), then either the hand-over of the chosen
// pair to the six-coordinate acceptance kernel (EXT), or the hop with the
// energy-conserving rescale, the force on the new surface, counters, the
// finished test and the population records.  All threads of the CTA call
// it; s_hop_a, s_hop_m are shared and -1 on entry.
template <class CT, bool EXT>
__device__ __forceinline__ void hop_finish(const DevState &s, int64_t t, double mass, double zeta, bool do_ratios,
                                           const double *G, double *red, double *scr, const int *unocc, int *occ_s,
                                           const double *lam_s, const double *q0_s, double geo_h, double geo_dh,
                                           double geo_k, int &s_hop_a, int &s_hop_m, const CT *Ct)
{
    const int N = s.N, Ne = s.Ne, nu = N - Ne;
    // ---- stochastic selection in the order (slot a ascending, m ascending)
    if (do_ratios) {
        double *slot_sum = (Ne <= 64) ? red : scr + 3 * (int64_t)Ne * N;
        for (int a = threadIdx.x; a < Ne; a += blockDim.x) {
            double sa = 0.0;
            for (int u = 0; u < nu; ++u) sa += G[(int64_t)a * N + unocc[u]];
            slot_sum[a] = sa;
        }
        __syncthreads();
        // The running sum in that order, by warp 0: each lane sums a run of
        // consecutive slots (then of candidates), a warp scan gives the sums
        // before each run, and each lane walks its run; the first lane whose
        // run crosses zeta holds the hop.  (One thread walking all Ne + nu
        // terms would issue each FP64 addition alone, and on this GPU an
        // FP64 instruction costs a warp its slot on the pipe whatever its
        // active lanes.)  The sums round differently from a single serial
        // sum only at the last bit.
        if (threadIdx.x < 32) {
            constexpr unsigned kFull = 0xffffffffu;
            const int lane = threadIdx.x;
            auto scan_excl = [&](double v) {  // sum of v over the lanes below
                double inc = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double w = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o) inc += w;
                }
                const double ex = __shfl_up_sync(kFull, inc, 1);
                return lane == 0 ? 0.0 : ex;
            };
            const int pa = (Ne + 31) / 32, a0 = lane * pa, a1 = min(Ne, a0 + pa);
            double loc = 0.0;
            for (int a = a0; a < a1; ++a) loc += slot_sum[a];
            double cum = scan_excl(loc), cum_hit = 0.0;
            int hit = -1;
            for (int a = a0; a < a1; ++a) {
                if (hit < 0 && cum + slot_sum[a] > zeta) {
                    hit = a;
                    cum_hit = cum;
                }
                cum += slot_sum[a];
            }
            const unsigned ba = __ballot_sync(kFull, hit >= 0);
            if (ba) {
                const int src = __ffs(ba) - 1;
                const int a_hit = __shfl_sync(kFull, hit, src);
                const double base = __shfl_sync(kFull, cum_hit, src);
                const double *Ga = G + (int64_t)a_hit * N;
                const int pu = (nu + 31) / 32, u0 = lane * pu, u1 = min(nu, u0 + pu);
                double l2 = 0.0;
                for (int u = u0; u < u1; ++u) l2 += Ga[unocc[u]];
                double c2 = base + scan_excl(l2);
                int m_hit = -1;
                for (int u = u0; u < u1; ++u) {
                    c2 += Ga[unocc[u]];
                    if (m_hit < 0 && c2 > zeta) m_hit = unocc[u];
                }
                const unsigned bm = __ballot_sync(kFull, m_hit >= 0);
                const int m_sel = bm ? __shfl_sync(kFull, m_hit, __ffs(bm) - 1) : -1;
                if (lane == 0 && m_sel >= 0) {
                    s_hop_a = a_hit;
                    s_hop_m = m_sel;
                }
            }
        }
        __syncthreads();
    }

    if constexpr (EXT) {  // rescale and bookkeeping in the six-coordinate acceptance kernel
        if (threadIdx.x == 0) s.hop_pair[t] = s_hop_a >= 0 ? s_hop_a * N + s_hop_m : -1;
        return;
    }
    // ---- hop, rescale, force, counters (thread 0)
    if (threadIdx.x == 0) {
        double p = s.p[t];
        if (s_hop_a >= 0) {
            const int a = s_hop_a, m = s_hop_m;
            const double dE = lam_s[m] - lam_s[occ_s[a]];
            const double p2 = p * p - 2.0 * mass * dE;
            if (p2 >= 0.0) {
                p = (p >= 0.0 ? 1.0 : -1.0) * sqrt(p2);
                // replace s_a by m and keep the list sorted
                int b = a;
                occ_s[b] = m;
                while (b > 0 && occ_s[b - 1] > occ_s[b]) {
                    const int tmp = occ_s[b - 1];
                    occ_s[b - 1] = occ_s[b];
                    occ_s[b] = tmp;
                    --b;
                }
                while (b < Ne - 1 && occ_s[b + 1] < occ_s[b]) {
                    const int tmp = occ_s[b + 1];
                    occ_s[b + 1] = occ_s[b];
                    occ_s[b] = tmp;
                    ++b;
                }
                for (int q = 0; q < Ne; ++q) s.occ[t * Ne + q] = (int16_t)occ_s[q];
                double F = -s.dU0[t];
                for (int q = 0; q < Ne; ++q) {
                    const int i = occ_s[q];
                    F -= q0_s[i] * q0_s[i] * (geo_dh + 2.0 * geo_k * (lam_s[i] - geo_h));
                }
                s.F[t] = F;
                s.p[t] = p;
                s.hops[t] += 1;
            } else {
                s.frus[t] += 1;
            }
        }
        s.vprev[t] = p / mass;
        const int64_t ns = s.nstep[t] + 1;
        s.nstep[t] = ns;
        if (s.z_done > 0.0 && s.x[t] > s.z_done) atomicOr(&s.status[t], ST_DONE);
    }
    // ---- observables
    if (s.record_every > 0) {
        __syncthreads();
        const int64_t ns = s.nstep[t];
        if (ns % s.record_every == 0) {
            const int64_t r = ns / s.record_every - 1;
            if (r < s.max_records) {
                double psh = 0.0, pwf = 0.0;
                for (int a = threadIdx.x; a < Ne; a += blockDim.x) {
                    const double q = q0_s[occ_s[a]];
                    psh += q * q;
                    double ar = 0.0, ai = 0.0;
                    for (int i = 0; i < N; ++i) {
                        const double2 cv = to_d2(Ct[(int64_t)a * N + i]);
                        ar = fma(q0_s[i], cv.x, ar);
                        ai = fma(q0_s[i], cv.y, ai);
                    }
                    pwf += ar * ar + ai * ai;
                }
                psh = block_sum(psh, red);
                pwf = block_sum(pwf, red);
                if (threadIdx.x == 0) {
                    s.rec_sh[r * s.n + t] = psh;
                    s.rec_wf[r * s.n + t] = pwf;
                }
            }
        }
    }
}

}  // namespace iesh
