// iesh_secular.cuh -- roots of the secular equation of an arrowhead matrix
// (internal to the library), templated on the arithmetic type.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "iesh_common.cuh"

namespace iesh {

template <class R>
struct Roundoff;
template <>
struct Roundoff<double> {
    static constexpr double u = 1.1102230246251565e-16;  // 2^-53
    static constexpr double tiny = 1e-300;
};
template <>
struct Roundoff<float> {
    static constexpr float u = 5.9604645e-08f;  // 2^-24
    static constexpr float tiny = 1e-37f;
};


// Reciprocal of a pole distance.  FP64: the PTX approximate reciprocal
// r0 = 1/d (1 + e'), e = 1 - d r0, refined by the first terms of the
// geometric series 1/d = r0 / (1 - e) = r0 (1 + e + e^2 + ...); with the
// estimate's relative error |e| far below 2^-18 the truncated e^3 term is
// below 2^-54, so the result is within about an ulp of 1/d.  Three FMAs
// replace a full division in the secular sums, which are the FP64-bound
// part of the eigen solve, in the couplings d_jk and in the iteration's
// safeguarded proposals.  Inputs are pole distances, eigenvalue gaps and
// proposal denominators; a zero or subnormal input (the estimate flushes
// subnormals to zero) gives a non-finite result, which the callers either
// cannot produce or reject.
template <class R>
__device__ __forceinline__ R pole_recip(R d)
{
    return R(1) / d;
}
template <>
__device__ __forceinline__ double pole_recip<double>(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// Double-float numbers (hi + lo, two FP32 values, about 48 significant bits)
// for the secular sums of the mixed-precision path: the FP32 pipe is 64x
// wider than the FP64 pipe on this part.  Error-free transformations:
// Knuth's TwoSum, Dekker's Fast2Sum (|a| >= |b|) and the FMA product error.
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl dfl_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl dfl_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
// a + b with an error of a few units of 2^-46 (|a| + |b|)
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b)
{
    dfl s = dfl_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return dfl_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dfl_fast_two_sum(p, e);
}
// 1/a: the rounded FP32 reciprocal r0 corrected by r0 (1 - a r0)
__device__ __forceinline__ dfl dfl_rcp(dfl a)
{
    const float r0 = __frcp_rn(a.hi);
    float e = fmaf(-a.hi, r0, 1.0f);
    e = fmaf(-a.lo, r0, e);
    return dfl_fast_two_sum(r0, r0 * e);
}
__device__ __forceinline__ dfl dfl_from(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double dfl_value(dfl a) { return (double)a.hi + (double)a.lo; }

// Pole data of the secular sums.  diff (optional): FP64 table of the pole
// differences diff[k M + o] = eps_o - eps_k; ddf, z2df (double-float mode):
// the same differences and z_k^2 as double-float pairs.
// Two-orbital double-float mode (EV_TWO_DF): the M poles are nb bath poles
// with one extra pole h_- inserted at index hpos (hpos < 0: none); ddf is
// the bath table [nb][nb], hdf[k] = h_- - eps_k as double-float pairs, and
// z2df the weights of all M poles in sorted order.
// Nested double-float mode (EV_NESTED): the M poles are roots mu_k = eps_{ob[k]}
// + tau_k of an inner arrowhead over nb bath poles; ddf is the bath table
// [nb][nb], hdf[k] = tau_k as a double-float pair and ob[k] its bath pole,
// so mu_o - mu_k = (eps_{ob[o]} - eps_{ob[k]}) + (tau_o - tau_k) keeps its
// relative accuracy however close the two roots are.
template <class R>
struct Poles {
    int M;
    const R *__restrict__ eps, *__restrict__ z2, *__restrict__ diff;
    const float2 *__restrict__ ddf, *__restrict__ z2df;
    int nb, hpos;
    R hm;
    const float2 *__restrict__ hdf;
    const int *__restrict__ ob;
};

// Evaluation modes of the secular sums: EV_PLAIN (eps_o - eps_k formed per
// term), EV_TABLE (FP64 table), EV_DFLOAT (double-float sums on the FP32
// pipe; the origin term and everything outside the sums stay FP64), EV_TWO_DF
// and EV_NESTED (double-float, see Poles).
enum { EV_PLAIN = 0, EV_TABLE = 1, EV_DFLOAT = 2, EV_TWO_DF = 3, EV_NESTED = 4 };

// mu_o - mu_k + td for the nested poles (EV_NESTED), in double-float.
template <class R>
__device__ __forceinline__ dfl nested_gap(const Poles<R> &P, int o, int k, dfl td)
{
    const float2 e = P.ddf[(size_t)P.ob[k] * P.nb + P.ob[o]];  // eps_ob[o] - eps_ob[k]
    const float2 to = P.hdf[o], tk = P.hdf[k];
    const dfl dtau = dfl_add({to.x, to.y}, {-tk.x, -tk.y});
    return dfl_add(dfl_add({e.x, e.y}, dtau), td);
}

// ============================================================= eigenpairs
// The one-electron Hamiltonian of Sec. II B is an arrowhead matrix:
// diag(h, eps_1..eps_M) bordered by z_k = V_k(x).  Its eigenvalues are the
// roots of g(lam) = lam - h - sum_k z_k^2 / (lam - eps_k), one in each gap
// of the sorted poles, and the eigenvector of root lam has impurity
// component q0 = 1 / sqrt(g'(lam)) (chosen > 0) and bath components
// z_k q0 / (lam - eps_k).  Each root is found in the shifted variable
// tau = lam - eps_o relative to its nearer pole o, so lam - eps_k =
// (eps_o - eps_k) + tau keeps full relative accuracy.
template <class R>
struct Sec {
    R g, gp, gp_rest, qo, sabs;
};

// With ABS the sum of |z_k^2 / (lam - eps_k)| over k != o (the scale of the
// rounding error of g, for the stopping test) is accumulated into e.sabs;
// without it e.sabs is left at zero for the caller to fill in.  EV selects
// how the sums over k != o are formed (see EV_*); the terms k != o have
// |lam - eps_k| >= half a pole gap, so their double-float range is safe.
template <class R, bool ABS, int EV>
__device__ __forceinline__ Sec<R> sec_eval(const Poles<R> &P, int o, R tau, R eomh)
{
    const int M = P.M;
    R s1 = 0, s2 = 0, sa = 0;
    if constexpr (EV == EV_DFLOAT) {
        // two accumulator sets (even and odd poles), added at the end: the
        // double-float additions are a serial chain, two chains run at once
        const dfl td = dfl_from((double)tau);
        dfl d1[2] = {{0.f, 0.f}, {0.f, 0.f}}, d2[2] = {{0.f, 0.f}, {0.f, 0.f}}, da[2] = {{0.f, 0.f}, {0.f, 0.f}};
        auto term = [&](int k, int h) {
            const float2 dk = P.ddf[(size_t)k * M + o], zk = P.z2df[k];
            const dfl r = dfl_rcp(dfl_add({dk.x, dk.y}, td));  // 1 / (lam - eps_k)
            const dfl q = dfl_mul({zk.x, zk.y}, r);
            if (k != o) {
                d1[h] = dfl_add(d1[h], q);
                d2[h] = dfl_add(d2[h], dfl_mul(q, r));
                if (ABS) da[h] = dfl_add(da[h], q.hi < 0.f ? dfl{-q.hi, -q.lo} : q);
            }
        };
        int k = 0;
        for (; k + 1 < M; k += 2) {
            term(k, 0);
            term(k + 1, 1);
        }
        if (k < M) term(k, 0);
        s1 = (R)dfl_value(dfl_add(d1[0], d1[1]));
        s2 = (R)dfl_value(dfl_add(d2[0], d2[1]));
        sa = (R)dfl_value(dfl_add(da[0], da[1]));
    } else if constexpr (EV == EV_NESTED) {
        // two accumulator sets, as above
        const dfl td = dfl_from((double)tau);
        dfl d1[2] = {{0.f, 0.f}, {0.f, 0.f}}, d2[2] = {{0.f, 0.f}, {0.f, 0.f}}, da[2] = {{0.f, 0.f}, {0.f, 0.f}};
        auto term = [&](int k, int h) {
            if (k == o) return;
            const dfl r = dfl_rcp(nested_gap(P, o, k, td));  // 1 / (lam - mu_k)
            const float2 zk = P.z2df[k];
            const dfl q = dfl_mul({zk.x, zk.y}, r);
            d1[h] = dfl_add(d1[h], q);
            d2[h] = dfl_add(d2[h], dfl_mul(q, r));
            if (ABS) da[h] = dfl_add(da[h], q.hi < 0.f ? dfl{-q.hi, -q.lo} : q);
        };
        int k = 0;
        for (; k + 1 < M; k += 2) {
            term(k, 0);
            term(k + 1, 1);
        }
        if (k < M) term(k, 0);
        s1 = (R)dfl_value(dfl_add(d1[0], d1[1]));
        s2 = (R)dfl_value(dfl_add(d2[0], d2[1]));
        sa = (R)dfl_value(dfl_add(da[0], da[1]));
    } else if constexpr (EV == EV_TWO_DF) {
        // bath poles in double-float from the bath table (origin a bath pole)
        // or from hdf (origin h_-); the h_- term itself in R.  Two
        // accumulator sets, as above
        const dfl td = dfl_from((double)tau);
        const bool oh = o == P.hpos;
        const int ob = oh ? 0 : ((P.hpos >= 0 && o > P.hpos) ? o - 1 : o);
        dfl d1[2] = {{0.f, 0.f}, {0.f, 0.f}}, d2[2] = {{0.f, 0.f}, {0.f, 0.f}}, da[2] = {{0.f, 0.f}, {0.f, 0.f}};
        auto term = [&](int k, int h) {
            const int q = (P.hpos >= 0 && k >= P.hpos) ? k + 1 : k;
            const float2 dk = oh ? P.hdf[k] : P.ddf[(size_t)k * P.nb + ob], zk = P.z2df[q];
            const dfl r = dfl_rcp(dfl_add({dk.x, dk.y}, td));  // 1 / (lam - eps_k)
            const dfl qv = dfl_mul({zk.x, zk.y}, r);
            if (q != o) {
                d1[h] = dfl_add(d1[h], qv);
                d2[h] = dfl_add(d2[h], dfl_mul(qv, r));
                if (ABS) da[h] = dfl_add(da[h], qv.hi < 0.f ? dfl{-qv.hi, -qv.lo} : qv);
            }
        };
        int k = 0;
        for (; k + 1 < P.nb; k += 2) {
            term(k, 0);
            term(k + 1, 1);
        }
        if (k < P.nb) term(k, 0);
        s1 = (R)dfl_value(dfl_add(d1[0], d1[1]));
        s2 = (R)dfl_value(dfl_add(d2[0], d2[1]));
        sa = (R)dfl_value(dfl_add(da[0], da[1]));
        if (P.hpos >= 0 && !oh) {
            const R r = pole_recip<R>((P.eps[o] - P.hm) + tau);
            const R qv = P.z2[P.hpos] * r;
            s1 += qv;
            s2 = fma(qv, r, s2);
            if (ABS) sa += fabs(qv);
        }
    } else {
        const R eo = P.eps[o];
#pragma unroll 4
        for (int k = 0; k < M; ++k) {
            const R dko = EV == EV_TABLE ? P.diff[(size_t)k * M + o] : (eo - P.eps[k]);
            const R r = pole_recip<R>(dko + tau);
            const R q = P.z2[k] * r;
            if (k != o) {
                s1 += q;
                s2 = fma(q, r, s2);
                if (ABS) sa += fabs(q);
            }
        }
    }
    // origin term: one reciprocal of tau (never zero or subnormal: the
    // iteration keeps it strictly inside its bracket) serves both quotients
    const R rt = pole_recip<R>(tau);
    const R qo = P.z2[o] * rt;
    Sec<R> e;
    e.g = (eomh + tau) - s1 - qo;
    e.gp_rest = R(1) + s2;
    e.gp = e.gp_rest + qo * rt;
    e.qo = qo;
    e.sabs = sa;
    return e;
}

// Fixed-weight iteration for one root in the shifted variable tau about the
// origin pole o: the origin pole is kept exactly and the rest of g is
// modelled by one more pole at tau = +D (kind 0) or -D (kind 1), or by a
// linear term for the two outermost roots (kind 2: below all poles, kind 3:
// above), matched in value and slope; each model root is safeguarded by the
// bracket [lo, hi] of sign changes.  On return e is evaluated at tau.
template <class R, int EV>
__device__ bool sec_iterate(const Poles<R> &P, R h, int o, int kind, R D, R &lo, R &hi, R &tau,
                            Sec<R> &e, bool have)
{
    // rounding unit of the sums: 2^-44 covers the double-float sums
    const R u = (EV == EV_DFLOAT || EV == EV_TWO_DF || EV == EV_NESTED) ? R(5.684341886080802e-14)
                                                                       : Roundoff<R>::u;
    const R eomh = P.eps[o] - h;
    const R s = P.z2[o];
    // the non-origin part of the error scale varies slowly with tau (those
    // poles are at least half a gap away): take it from the first evaluation
    R sa_rest;
    if (have) {
        sa_rest = e.sabs;
    } else {
        e = sec_eval<R, true, EV>(P, o, tau, eomh);
        sa_rest = e.sabs;
        have = true;
    }
    for (int it = 0; it < 80; ++it) {
        if (!have) e = sec_eval<R, false, EV>(P, o, tau, eomh);
        have = false;
        e.sabs = sa_rest + fabs(e.qo) + fabs(eomh) + fabs(tau);
        if (fabs(e.g) <= R(8) * u * e.sabs) return true;
        if (e.g < R(0)) lo = tau;
        else hi = tau;
        // The quotients below are model-root proposals, safeguarded by the
        // bracket: reciprocals (pole_recip, within about an ulp) instead of
        // correctly rounded divisions, which cost several FP64 instructions
        // each on the iteration's serial path.  A zero or subnormal
        // denominator gives a non-finite proposal and the bisection step.
        R tn;
        const R rt = pole_recip<R>(tau);
        if (kind <= 1) {
            // model root of c tau^2 + B tau + s D = 0 in the gap, by the form
            // without cancellation for the sign of B (B < 0 happens when the
            // origin pole's weight s is small against the other end's)
            const R sg = kind == 0 ? R(1) : R(-1);
            const R tp = tau - sg * D;
            const R t = e.gp_rest * tp * tp;
            const R c = sg * (e.g + s * rt + t * pole_recip<R>(tp));
            const R B = c * D + s + t;
            const R sq = sqrt(fmax(B * B - R(4) * c * s * D, R(0)));
            if (B >= R(0) || c == R(0)) tn = sg * R(2) * s * D * pole_recip<R>(B + sq);
            else tn = sg * (B - sq) * pole_recip<R>(R(2) * c);
        } else {
            const R ee = e.gp_rest;
            const R c = e.g - ee * tau + s * rt;
            const R sq = sqrt(fmax(c * c + R(4) * ee * s, R(0)));
            if (kind == 2)
                tn = (c >= R(0)) ? (-c - sq) * pole_recip<R>(R(2) * ee) : -R(2) * s * pole_recip<R>(sq - c);
            else
                tn = (c <= R(0)) ? (sq - c) * pole_recip<R>(R(2) * ee) : R(2) * s * pole_recip<R>(c + sq);
        }
        if (!(tn > lo && tn < hi)) tn = R(0.5) * (lo + hi);
        const bool tiny = fabs(tn - tau) <= R(2) * u * fabs(tn);
        tau = tn;
        if (tiny) {
            e = sec_eval<R, false, EV>(P, o, tau, eomh);
            return true;
        }
    }
    e = sec_eval<R, false, EV>(P, o, tau, eomh);
    return false;
}

// Root r (0..M) of the secular equation, lam and q0 = 1/sqrt(g'(lam)), and
// optionally its origin pole o and offset tau = lam - eps_o (unrounded).
// Cold start: the sign of g at the middle of the pole gap picks the nearer
// pole as origin and the half-gap as bracket.  Warm start (previous root
// `guess`, which lies in the same gap): origin = pole nearer the guess,
// bracket = the whole gap, started at the guess; if the root ends in the
// far half of the gap it is refined once more about the other pole.
// EV: how the secular sums are formed (see sec_eval).
template <class R, int EV = EV_PLAIN>
__device__ void secular_root(int r, const Poles<R> &P, R h, R Z2, bool warm, R guess, R &lam, R &q0,
                             uint32_t &st, int *o_out = nullptr, R *tau_out = nullptr)
{
    const int M = P.M;
    const R *__restrict__ eps = P.eps;
    int o, kind;
    R lo, hi, D = 0, tau;
    Sec<R> e;
    bool have = false, conv;
    if (r > 0 && r < M) {
        const int L = r - 1;
        D = eps[r] - eps[L];
        if (warm && guess > eps[L] && guess < eps[r]) {
            if (guess - eps[L] <= eps[r] - guess) {
                o = L; kind = 0; lo = 0; hi = D; tau = guess - eps[L];
            } else {
                o = r; kind = 1; lo = -D; hi = 0; tau = guess - eps[r];
            }
            conv = sec_iterate<R, EV>(P, h, o, kind, D, lo, hi, tau, e, false);
            if (kind == 0 && tau > R(0.5) * D) {
                o = r; kind = 1; lo = fmin(lo - D, -R(0.5) * D); hi = 0; tau = tau - D;
                conv = sec_iterate<R, EV>(P, h, o, kind, D, lo, hi, tau, e, false);
            } else if (kind == 1 && tau < -R(0.5) * D) {
                o = L; kind = 0; lo = 0; hi = fmax(hi + D, R(0.5) * D); tau = tau + D;
                conv = sec_iterate<R, EV>(P, h, o, kind, D, lo, hi, tau, e, false);
            }
        } else {
            const Sec<R> em = sec_eval<R, true, EV>(P, L, R(0.5) * D, eps[L] - h);
            if (em.g >= R(0)) {
                o = L; kind = 0; lo = 0; hi = R(0.5) * D; tau = R(0.5) * D; e = em; have = true;
            } else {
                o = r; kind = 1; lo = -R(0.5) * D; hi = 0; tau = -R(0.5) * D;
            }
            conv = sec_iterate<R, EV>(P, h, o, kind, D, lo, hi, tau, e, have);
        }
    } else {
        if (r == 0) {
            o = 0; kind = 2;
            const R t = h - eps[0];
            const R lb = R(0.5) * ((h + eps[0]) - sqrt(t * t + R(4) * Z2));
            lo = (lb - eps[0]) * (R(1) + R(64) * Roundoff<R>::u) - Roundoff<R>::tiny;
            hi = 0;
            tau = R(0.5) * lo;
        } else {
            o = M - 1; kind = 3;
            const R t = h - eps[M - 1];
            const R ub = R(0.5) * ((h + eps[M - 1]) + sqrt(t * t + R(4) * Z2));
            lo = 0;
            hi = (ub - eps[M - 1]) * (R(1) + R(64) * Roundoff<R>::u) + Roundoff<R>::tiny;
            tau = R(0.5) * hi;
        }
        if (warm) {
            const R tg = guess - eps[o];
            if (tg > lo && tg < hi) tau = tg;
        }
        conv = sec_iterate<R, EV>(P, h, o, kind, D, lo, hi, tau, e, false);
    }
    if (!conv) st |= ST_SECULAR;
    lam = eps[o] + tau;
    q0 = R(1) / sqrt(e.gp);
    if (o_out) *o_out = o;  // lam = eps[o] + tau with tau exact
    if (tau_out) *tau_out = tau;
}


}  // namespace iesh
