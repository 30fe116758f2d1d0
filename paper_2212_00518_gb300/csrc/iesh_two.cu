// iesh_two.cu -- IESH dynamics of a two-orbital adsorbate over six nuclear
// coordinates: kernels and the iesh2_* C-ABI.
//
// Electrons: adsorbate orbitals a = 0, 1 with levels h_a(x), each coupled to
// bath state k by c_a(x) sqrt(w_k), c_a = vbar_a f_a(x) (the occupied-energy
// model).  Both border vectors are proportional to sqrt(w_k), so with
// c^2 = c_0^2 + c_1^2 the combination |+> = (c_0|0> + c_1|1>)/c couples to
// the bath and |-> = (-c_1|0> + c_0|1>)/c couples only to |+> (through
// t = c_0 c_1 (h_1 - h_0) / c^2).  Eliminating |-> and the bath leaves one
// arrowhead secular equation with the M bath poles and one more pole at
// h_- = <-|H|-> of weight t^2 (M + 2 roots, one per orbital):
//   lam - h_+ - sum_k c^2 w_k / (lam - eps_k) - t^2 / (lam - h_-) = 0,
// root j has q_+ = 1/sqrt(g'(lam)) (> 0: the gauge), q_- = t q_+ / (lam - h_-)
// and adsorbate components Q_0j = (c_0 q_+ - c_1 q_-)/c, Q_1j = (c_1 q_+ + c_0 q_-)/c.
// With t = 0, |-> is itself an eigenvector (lam = h_-); with c = 0 the
// Hamiltonian is diagonal.
//
// Derivative couplings: on an eigenvector c_a B_k = (lam_k - h_a) Q_ak
// (B_k = sum_k' sqrt(w_k') X_k'k), so for every direction y the matrix
// T^y = Q^T (dH/dy) Q is the one-orbital closed form summed over the two
// adsorbate orbitals,
//   T^y_jk = sum_a Q_aj Q_ak [dh_a/dy + (dlog f_a/dy) (lam_j + lam_k - 2 h_a)],
// d^y_jk = T^y_jk / (lam_k - lam_j), and the Hellmann-Feynman force is
// F_y = -dU0/dy - sum_{j occupied} T^y_jj.
//
// Precision: FP64, or mixed (the one-coordinate model's split): FP64
// eigenpairs (the secular sums over the bath poles in double-float),
// forces, hop probabilities and rescale; FP32 coefficients, coupling
// generator, propagation (tensor cores where the trajectory fits one CTA)
// and overlap LU.
//
// One step (Sec. II B, II C in six dimensions):
//   k2_eigen      kick + drift, eigenpairs, forces, second kick, the
//                 velocity-projected scalars for the hop kernel;
//   k2_build_w    W = dt/2 (D0 + D1), D_e = v_e . d at the two ends of the step,
//                 its Gershgorin interval and the Chebyshev coefficients;
//   k_cheb        (shared with the one-coordinate model) the exponential;
//   k_hop<EXT>    determinant ratios, g_{a->m} with v . d, the selection;
//   k2_accept     the six-dimensional momentum change along d_{m, s_a},
//                 occupations, force on the new surface, counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/iesh.h"
#include "iesh_cheb.cuh"
#include "iesh_common.cuh"
#include "iesh_host.h"
#include "iesh_kernels.h"
#include "iesh_secular.cuh"
#include "iesh_syev.cuh"

using namespace iesh;

namespace {

// Model constants passed by value to the kernels.
struct Model2Dev {
    double th[16];  // eps_0, eps_1, g_{0,0..5}, g_{1,0..5}, sigma_0, sigma_1
    double vbar[2], R[6], x0[6];
    double mass, omega;
    double wsum;    // sum_k w_k of the bath
    // dense-solver models: the coupling of orbital a to bath state k is
    // vbar_a f_a(x) prof[a M + k] (prof = sqrt(w_k) times the orbital's own
    // bath profile), pnorm[a] = |prof[a]|
    const double *prof;
    double pnorm[2];
    // nested secular path: the step-1 roots of every trajectory [n][M + 1],
    // kept for the next step's warm start; prof_0k prof_1k as double-float
    // pairs (mixed path)
    double *mu;
    const float2 *ppdf;
};

// Adsorbate quantities at one geometry: levels h_a, coupling amplitudes c_a
// and kap[y] = dlog f_a/dy for the three coordinates y of orbital a.
struct Ads2 {
    double h[2], c[2], kap[6];
};

__device__ __forceinline__ Ads2 ads2_eval(const Model2Dev &md, const double *x)
{
    Ads2 o;
    for (int a = 0; a < 2; ++a) {
        double h = md.th[a];
        for (int y = 0; y < 6; ++y) h += md.th[2 + 6 * a + y] * x[y];
        const double sg = md.th[14 + a];
        double r2 = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double d = x[3 * a + q] - md.R[3 * a + q];
            r2 += d * d;
            o.kap[3 * a + q] = -d / (sg * sg);
        }
        o.h[a] = h;
        o.c[a] = md.vbar[a] * exp(-0.5 * r2 / (sg * sg));
    }
    return o;
}

// grad h_a . v and grad log f_a . v
__device__ __forceinline__ void ads2_project(const Model2Dev &md, const Ads2 &ad, const double *v,
                                             double hv[2], double kv[2])
{
    for (int a = 0; a < 2; ++a) {
        double s = 0.0;
        for (int y = 0; y < 6; ++y) s += md.th[2 + 6 * a + y] * v[y];
        hv[a] = s;
        double k = 0.0;
        for (int q = 0; q < 3; ++q) k += ad.kap[3 * a + q] * v[3 * a + q];
        kv[a] = k;
    }
}

// Velocity-projected scalars of the hop kernel: h_0, h_1, grad h_a . v,
// grad log f_a . v at momentum p.
__device__ __forceinline__ void write_geo2(const DevState &s, int64_t t, const Model2Dev &md,
                                           const Ads2 &ad, const double *p)
{
    double v[6], hv[2], kv[2];
    for (int y = 0; y < 6; ++y) v[y] = p[y] / md.mass;
    ads2_project(md, ad, v, hv, kv);
    double *g = s.geo2 + t * 8;
    g[0] = ad.h[0];
    g[1] = ad.h[1];
    g[2] = hv[0];
    g[3] = hv[1];
    g[4] = kv[0];
    g[5] = kv[1];
}

// Adsorbate quantities at x formed once per CTA by thread 0 and shared
// (an FP64 instruction costs a warp its issue slot on the FP64 pipe whatever
// its active lanes, so every thread evaluating the same exponentials would
// cost every warp that much).  Block-wide; ends with a barrier; x must be
// readable by thread 0.
__device__ __forceinline__ Ads2 ads2_block(const Model2Dev &md, const double *x, Ads2 *sh)
{
    if (threadIdx.x == 0) *sh = ads2_eval(md, x);
    __syncthreads();
    return *sh;
}

// Both ends of a step: adsorbate quantities at x_prev and x, and the
// velocity projections with v_prev and p / mass; formed once per CTA as
// ads2_block.
struct Ends2 {
    Ads2 e0, e1;
    double hv0[2], kv0[2], hv1[2], kv1[2];
};
__device__ __forceinline__ void ends2_block(const DevState &s, const Model2Dev &md, int64_t t, Ends2 *sh)
{
    if (threadIdx.x == 0) {
        double x0[6], v0[6], x1[6], v1[6];
        for (int y = 0; y < 6; ++y) {
            x0[y] = s.x_prev[t * 6 + y];
            v0[y] = s.vprev[t * 6 + y];
            x1[y] = s.x[t * 6 + y];
            v1[y] = s.p[t * 6 + y] / md.mass;
        }
        sh->e0 = ads2_eval(md, x0);
        sh->e1 = ads2_eval(md, x1);
        ads2_project(md, sh->e0, v0, sh->hv0, sh->kv0);
        ads2_project(md, sh->e1, v1, sh->hv1, sh->kv1);
    }
    __syncthreads();
}

// Force component y on the occupied surface from the occupied sums
// S_a = sum Q_aj^2 and U_a = sum Q_aj^2 (lam_j - h_a).
__device__ __forceinline__ double force2(const Model2Dev &md, const Ads2 &ad, const double *x, int y,
                                         const double S[2], const double U[2])
{
    const int a = y / 3;
    double f = -md.mass * md.omega * md.omega * (x[y] - md.x0[y]);
    f -= S[0] * md.th[2 + y] + S[1] * md.th[8 + y];
    f -= 2.0 * U[a] * ad.kap[y];
    return f;
}

// Occupied sums over the orbital list occ (block-wide; all threads call).
__device__ __forceinline__ void occ_sums(const double *lam, const double *Q0, const double *Q1,
                                         const int16_t *occ, int Ne, const Ads2 &ad, double *red,
                                         double S[2], double U[2])
{
    double s0 = 0.0, s1 = 0.0, u0 = 0.0, u1 = 0.0;
    for (int q = threadIdx.x; q < Ne; q += blockDim.x) {
        const int j = occ[q];
        const double a2 = Q0[j] * Q0[j], b2 = Q1[j] * Q1[j];
        s0 += a2;
        s1 += b2;
        u0 += a2 * (lam[j] - ad.h[0]);
        u1 += b2 * (lam[j] - ad.h[1]);
    }
    S[0] = block_sum(s0, red);
    S[1] = block_sum(s1, red);
    U[0] = block_sum(u0, red);
    U[1] = block_sum(u1, red);
}

// Per-trajectory scalars of the eigen kernel (one slot's shared record).
struct Eig2Slot {
    Ads2 ad, adp;  // at the step's end and start (mode 1)
    double x[6], p[6], xp[6];
    double c, hp, hm, tt;
    int pos, case_;  // pos: bath poles below h_-; case_: 0 general, 1 |-> decoupled, 2 no coupling
};

// mode 0: eigenpairs and forces at x (state set-up).  mode 1: a step's
// kick + drift, eigenpairs at the new x, forces and the second kick.
// tpb trajectories per CTA (slots of N threads), one thread per root; every
// barrier is reached by all threads of the CTA.  DF: the secular sums over
// the bath poles in double-float arithmetic (mixed path; the bath
// differences from the context's table, those to h_- per trajectory).
template <bool DF>
__global__ void __launch_bounds__(256, 3) k2_eigen(DevState s, Model2Dev md, double dt, int mode, int tpb)
{
    extern __shared__ double e2_sh[];
    const int N = s.N, M = s.M, Ne = s.Ne;
    const int slot = threadIdx.x / N;
    const int r = threadIdx.x - slot * N;
    const bool inslot = slot < tpb;
    const int64_t t = inslot ? traj_of(s, (int64_t)blockIdx.x * tpb + slot) : -1;
    const bool act = t >= 0 && !(s.status[t] & ST_DONE);
    const int Pw = eigen_pow2(N);                          // reduction width
    const int per = 2 * (M + 1) + 3 * N + 4 * Pw + (DF ? 2 * M + 1 : 0);
    double *eps_s = e2_sh;                                 // [M] bath energies, shared
    double *pole = eps_s + M + (inslot ? slot : 0) * per;  // [M + 1] sorted poles
    double *wt = pole + (M + 1);                           // [M + 1] their weights
    double *lam_s = wt + (M + 1);                          // [N]
    double *Q0_s = lam_s + N;                              // [N]
    double *Q1_s = Q0_s + N;                               // [N]
    double *red = Q1_s + N;                                // [4][Pw] reductions / staging
    float2 *z2df = reinterpret_cast<float2 *>(red + 4 * Pw);  // [M + 1] weights as double-float (DF)
    float2 *hdf = z2df + (M + 1);                          // [M] h_- - eps_k as double-float (DF)
    Eig2Slot *sl = reinterpret_cast<Eig2Slot *>(e2_sh + M + tpb * per) + (inslot ? slot : 0);
    for (int k = threadIdx.x; k < M; k += blockDim.x) eps_s[k] = s.eps[k];
    // warm start: the previous roots extrapolated linearly (each thread reads
    // its own entries before it overwrites them)
    double guess = 0.0, lam_old = 0.0;
    if (act) {
        if (mode == 1) {
            lam_old = s.lam[t * N + r];
            guess = 2.0 * lam_old - s.lam_prev[t * N + r];
            s.lam_prev[t * N + r] = lam_old;
            s.q0_prev[t * N + r] = s.q0[t * N + r];
            s.q2_prev[t * N + r] = s.q2[t * N + r];
        }
        if (r < 6) {
            double x = s.x[t * 6 + r], p = s.p[t * 6 + r];
            if (mode == 1) {
                s.x_prev[t * 6 + r] = x;
                sl->xp[r] = x;
                p += 0.5 * dt * s.F[t * 6 + r];
                x += dt * p / md.mass;
            }
            sl->x[r] = x;
            sl->p[r] = p;
        }
    }
    __syncthreads();
    // adsorbate quantities and the rotation of the pair (one thread per slot)
    if (act && r == 0) {
        const Ads2 ad = ads2_eval(md, sl->x);
        sl->ad = ad;
        if (mode == 1) sl->adp = ads2_eval(md, sl->xp);
        const double c0 = ad.c[0], c1 = ad.c[1], csq = c0 * c0 + c1 * c1;
        if (!(csq > 0.0)) {
            sl->case_ = 2;
        } else {
            const double hm = (c1 * c1 * ad.h[0] + c0 * c0 * ad.h[1]) / csq;
            const double tt = c0 * c1 * (ad.h[1] - ad.h[0]) / csq;
            sl->c = sqrt(csq);
            sl->hp = (c0 * c0 * ad.h[0] + c1 * c1 * ad.h[1]) / csq;
            sl->hm = hm;
            sl->tt = tt;
            sl->case_ = (tt * tt > 0.0) ? 0 : 1;
            int lo = 0, hi = M;  // bath energies below h_- (ascending: bisection)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (eps_s[mid] < hm) lo = mid + 1;
                else hi = mid;
            }
            sl->pos = lo;
        }
    }
    __syncthreads();
    const Ads2 &ad = sl->ad;
    const double c0 = ad.c[0], c1 = ad.c[1];
    const int cs = act ? sl->case_ : 2;
    const int pos = sl->pos;
    const double c = sl->c, hm = sl->hm, tt = sl->tt;
    if (act && cs != 2) {
        for (int k = r; k < M; k += N) {
            const int q = (cs == 1 || k < pos) ? k : k + 1;
            const double w = (c0 * c0 + c1 * c1) * (s.z0[k] * s.z0[k]);
            pole[q] = eps_s[k];
            wt[q] = w;
            if (DF) {
                const dfl wd = dfl_from(w);
                z2df[q] = make_float2(wd.hi, wd.lo);
                if (cs == 0) {
                    const dfl hd = dfl_from(hm - eps_s[k]);
                    hdf[k] = make_float2(hd.hi, hd.lo);
                }
            }
        }
        if (cs == 0 && r == 0) {
            pole[pos] = hm;
            wt[pos] = tt * tt;
            if (DF) {
                const dfl wd = dfl_from(tt * tt);
                z2df[pos] = make_float2(wd.hi, wd.lo);
            }
        }
    }
    __syncthreads();
    uint32_t st = 0;
    double lam = 0.0, qp = 0.0;
    if (act) {
        if (cs == 2) {
            // no coupling: diagonal Hamiltonian, sorted (ties: adsorbate first)
            const double h0 = ad.h[0], h1 = ad.h[1];
            double q0 = 0.0, q1 = 0.0;
            int idx;
            if (r < M) {
                lam = eps_s[r];
                idx = r + (h0 <= lam) + (h1 <= lam);
            } else {
                const double h = r == M ? h0 : h1;
                int below = 0;
                for (int k = 0; k < M; ++k) below += (eps_s[k] < h);
                lam = h;
                if (r == M) {
                    idx = below + (h1 < h0);
                    q0 = 1.0;
                } else {
                    idx = below + (h0 <= h1);
                    q1 = 1.0;
                }
            }
            lam_s[idx] = lam;
            Q0_s[idx] = q0;
            Q1_s[idx] = q1;
        } else {
            const int P = cs == 1 ? M : M + 1;
            // Z2 = sum of the pole weights: c^2 sum_k w_k (+ t^2)
            const double Z2 = c * c * md.wsum + (cs == 0 ? tt * tt : 0.0);
            if (r <= P) {
                int o;
                double tau;
                // an extrapolation outside the root's pole gap falls back to the last root
                const double glo = r > 0 ? pole[r - 1] : -INFINITY, ghi = r < P ? pole[r] : INFINITY;
                if (!(guess > glo && guess < ghi)) guess = lam_old;
                if (DF) {
                    const Poles<double> pp = {P, pole, wt, nullptr, s.poledf, z2df, M, cs == 0 ? pos : -1, hm, hdf};
                    secular_root<double, EV_TWO_DF>(r, pp, sl->hp, Z2, mode == 1, guess, lam, qp, st, &o, &tau);
                } else {
                    const Poles<double> pp = {P, pole, wt, nullptr, nullptr, nullptr};
                    secular_root<double>(r, pp, sl->hp, Z2, mode == 1, guess, lam, qp, st, &o, &tau);
                }
                if (cs == 0) {
                    // lam - h_-: the exact offset when the origin pole is h_- itself
                    const double lmh = (o == pos) ? tau : (pole[o] - hm) + tau;
                    const double qm = tt * qp / lmh;
                    lam_s[r] = lam;
                    Q0_s[r] = (c0 * qp - c1 * qm) / c;
                    Q1_s[r] = (c1 * qp + c0 * qm) / c;
                } else {
                    red[r] = lam;  // staged: the decoupled |-> is placed below
                }
            }
        }
        if (st) atomicOr(&s.status[t], st);
    }
    __syncthreads();
    if (act && cs == 1) {
        // M + 1 roots of the |+> arrowhead plus the decoupled |-> at h_-
        if (r <= M) {
            const int idx = r + (lam >= hm);
            lam_s[idx] = lam;
            Q0_s[idx] = c0 * qp / c;
            Q1_s[idx] = c1 * qp / c;
        } else {
            int below = 0;
            for (int k = 0; k <= M; ++k) below += (red[k] < hm);
            lam_s[below] = hm;
            // (-c_1, c_0) / c; a unit adsorbate vector (+) when one coupling vanishes
            Q0_s[below] = c0 == 0.0 ? 1.0 : (c1 == 0.0 ? 0.0 : -c1 / c);
            Q1_s[below] = c0 == 0.0 ? 0.0 : (c1 == 0.0 ? 1.0 : c0 / c);
        }
    }
    __syncthreads();
    // In a step, an eigenvector whose overlap with the previous step's is
    // decisive (|overlap| >= 1/2) keeps it non-negative (the positive |+>
    // component alone flips the |->-like eigenvector where h_0 = h_1 and t
    // changes sign); at an eigenvalue crossing within the step the positive
    // |+> component stands.  The bath rows follow from the adsorbate rows,
    // B_kj = sqrt(w_k) A_j / (lam_j - eps_k) with A_j = c_0 Q_0j + c_1 Q_1j;
    // FP32 sums (only the comparison with -1/2 is used).
    if (act && mode == 1 && cs != 2) {
        const double q0 = Q0_s[r], q1 = Q1_s[r], lj = lam_s[r];
        const double p0 = s.q0_prev[t * N + r], p1 = s.q2_prev[t * N + r], lp = s.lam_prev[t * N + r];
        const Ads2 &adp = sl->adp;
        const float Aj = (float)(c0 * q0 + c1 * q1), Ap = (float)(adp.c[0] * p0 + adp.c[1] * p1);
        const float ljf = (float)lj, lpf = (float)lp;
        float acc = 0.0f;
        for (int k = 0; k < M; ++k) {
            const float ek = (float)eps_s[k];
            const float den = (ljf - ek) * (lpf - ek);
            const float w = (float)(s.z0[k] * s.z0[k]);
            if (den != 0.0f) acc += __fdividef(w, den);
        }
        const float ov = (float)(q0 * p0 + q1 * p1) + Aj * Ap * acc;
        if (ov <= -0.5f) {
            Q0_s[r] = -q0;
            Q1_s[r] = -q1;
        }
    }
    __syncthreads();
    // occupied sums S_a = sum Q_aj^2, U_a = sum Q_aj^2 (lam_j - h_a) by a
    // fixed-order tree over the slot (thread a takes electron a)
    if (inslot) {
        double a2 = 0.0, b2 = 0.0, u0 = 0.0, u1 = 0.0;
        if (act) {
            s.lam[t * N + r] = lam_s[r];
            s.q0[t * N + r] = Q0_s[r];
            s.q2[t * N + r] = Q1_s[r];
            if (mode == 0) s.lam_prev[t * N + r] = lam_s[r];  // no extrapolation at the first step
            if (r < Ne) {
                const int j = s.occ[t * Ne + r];
                a2 = Q0_s[j] * Q0_s[j];
                b2 = Q1_s[j] * Q1_s[j];
                u0 = a2 * (lam_s[j] - ad.h[0]);
                u1 = b2 * (lam_s[j] - ad.h[1]);
            }
        }
        red[r] = a2;
        red[Pw + r] = b2;
        red[2 * Pw + r] = u0;
        red[3 * Pw + r] = u1;
        if (r < Pw - N) {
            red[N + r] = 0.0;
            red[Pw + N + r] = 0.0;
            red[2 * Pw + N + r] = 0.0;
            red[3 * Pw + N + r] = 0.0;
        }
    }
    __syncthreads();
    for (int w = Pw >> 1; w > 0; w >>= 1) {
        if (inslot && r < w) {
            red[r] += red[r + w];
            red[Pw + r] += red[Pw + r + w];
            red[2 * Pw + r] += red[2 * Pw + r + w];
            red[3 * Pw + r] += red[3 * Pw + r + w];
        }
        __syncthreads();
    }
    if (act && r < 6) {
        const double S[2] = {red[0], red[Pw]}, U[2] = {red[2 * Pw], red[3 * Pw]};
        const double F = force2(md, ad, sl->x, r, S, U);
        double p = sl->p[r];
        if (mode == 1) p += 0.5 * dt * F;
        s.x[t * 6 + r] = sl->x[r];
        s.p[t * 6 + r] = p;
        s.F[t * 6 + r] = F;
        if (mode == 0) s.vprev[t * 6 + r] = p / md.mass;
        sl->p[r] = p;
    }
    __syncthreads();
    if (act && r == 0) write_geo2(s, t, md, ad, sl->p);
}

// W[j N + k] = dt/2 (D0_jk + D1_jk), D_e = T^{v_e}_jk / (lam_k - lam_j) at
// the start (x_prev, v_prev) and the end (x, p / mass) of the step; the
// Gershgorin interval of dt diag((lam0 + lam1)/2) - i W; the Chebyshev set-up.
__global__ void __launch_bounds__(256) k2_build_w(DevState s, Model2Dev md, double dt, double tol)
{
    extern __shared__ double w2_sh[];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N;
    double *l0 = w2_sh, *a0 = l0 + N, *b0 = a0 + N, *l1 = b0 + N, *a1 = l1 + N, *b1 = a1 + N;
    double *red = b1 + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        l0[i] = s.lam_prev[t * N + i];
        a0[i] = s.q0_prev[t * N + i];
        b0[i] = s.q2_prev[t * N + i];
        l1[i] = s.lam[t * N + i];
        a1[i] = s.q0[t * N + i];
        b1[i] = s.q2[t * N + i];
    }
    __shared__ Ends2 ends;
    ends2_block(s, md, t, &ends);
    const Ads2 e0 = ends.e0, e1 = ends.e1;
    const double hv0[2] = {ends.hv0[0], ends.hv0[1]}, kv0[2] = {ends.kv0[0], ends.kv0[1]};
    const double hv1[2] = {ends.hv1[0], ends.hv1[1]}, kv1[2] = {ends.kv1[0], ends.kv1[1]};
    __syncthreads();
    const double hdt = 0.5 * dt;
    double *W = s.scratch + t * s.scratch_stride;
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double lk0 = l0[k], ak0 = a0[k], bk0 = b0[k], lk1 = l1[k], ak1 = a1[k], bk1 = b1[k];
        double Rk = 0.0;
        for (int j = 0; j < N; ++j) {
            double w = 0.0;
            if (j != k) {
                const double s0 = l0[j] + lk0, s1 = l1[j] + lk1;
                const double T0 = a0[j] * ak0 * (hv0[0] + kv0[0] * (s0 - 2.0 * e0.h[0])) +
                                  b0[j] * bk0 * (hv0[1] + kv0[1] * (s0 - 2.0 * e0.h[1]));
                const double T1 = a1[j] * ak1 * (hv1[0] + kv1[0] * (s1 - 2.0 * e1.h[0])) +
                                  b1[j] * bk1 * (hv1[1] + kv1[1] * (s1 - 2.0 * e1.h[1]));
                w = hdt * (T0 * pole_recip<double>(lk0 - l0[j]) + T1 * pole_recip<double>(lk1 - l1[j]));
            }
            W[(int64_t)j * N + k] = w;
            Rk += fabs(w);
        }
        const double Lk = hdt * (lk0 + lk1);
        lo = fmin(lo, Lk - Rk);
        hi = fmax(hi, Lk + Rk);
    }
    lo = block_min(lo, red);
    hi = block_max(hi, red);
    if (threadIdx.x == 0) cheb_setup(s, t, lo, hi, tol);
}

// Mixed precision: the same W in FP32, rows padded to Np = N rounded up to 4
// with zeros (the layout of the FP32 propagators).  Eigenvalue differences
// come from double-float eigenvalues (hi, lo), (hi_k - hi_j) + (lo_k - lo_j),
// so nearly degenerate pairs keep FP32 relative accuracy without FP64
// arithmetic per element; numerators in FP32 from lam - h_a rounded from FP64.
__global__ void __launch_bounds__(256) k2_build_w_f32(DevState s, Model2Dev md, double dt, double tol)
{
    extern __shared__ double w2_sh[];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Np = (N + 3) & ~3;
    double *red = w2_sh;                                              // [32]
    float2 *l0 = reinterpret_cast<float2 *>(red + 32), *l1 = l0 + N;  // lam as (hi, lo) per end
    float *a0 = reinterpret_cast<float *>(l1 + N), *b0 = a0 + N, *a1 = b0 + N, *b1 = a1 + N;
    float *m00 = b1 + N, *m01 = m00 + N, *m10 = m01 + N, *m11 = m10 + N;  // lam - h_a per end
    __shared__ Ends2 ends;
    ends2_block(s, md, t, &ends);
    const Ads2 e0 = ends.e0, e1 = ends.e1;
    const double hv0[2] = {ends.hv0[0], ends.hv0[1]}, kv0[2] = {ends.kv0[0], ends.kv0[1]};
    const double hv1[2] = {ends.hv1[0], ends.hv1[1]}, kv1[2] = {ends.kv1[0], ends.kv1[1]};
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double la = s.lam_prev[t * N + i], lb = s.lam[t * N + i];
        const float ha = (float)la, hb = (float)lb;
        l0[i] = make_float2(ha, (float)(la - (double)ha));
        l1[i] = make_float2(hb, (float)(lb - (double)hb));
        a0[i] = (float)s.q0_prev[t * N + i];
        b0[i] = (float)s.q2_prev[t * N + i];
        a1[i] = (float)s.q0[t * N + i];
        b1[i] = (float)s.q2[t * N + i];
        m00[i] = (float)(la - e0.h[0]);
        m01[i] = (float)(la - e0.h[1]);
        m10[i] = (float)(lb - e1.h[0]);
        m11[i] = (float)(lb - e1.h[1]);
    }
    const float hdt = (float)(0.5 * dt);
    const float H00 = (float)hv0[0], K00 = (float)kv0[0], H01 = (float)hv0[1], K01 = (float)kv0[1];
    const float H10 = (float)hv1[0], K10 = (float)kv1[0], H11 = (float)hv1[1], K11 = (float)kv1[1];
    __syncthreads();
    float *W = reinterpret_cast<float *>(s.scratch + t * s.scratch_stride);  // [N][Np]
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float2 lk0 = l0[k], lk1 = l1[k];
        const float ak0 = a0[k], bk0 = b0[k], ak1 = a1[k], bk1 = b1[k];
        const float nk00 = m00[k], nk01 = m01[k], nk10 = m10[k], nk11 = m11[k];
        float Rk = 0.0f;
        for (int j = 0; j < N; ++j) {
            float w = 0.0f;
            if (j != k) {
                const float T0 = a0[j] * ak0 * (H00 + K00 * (m00[j] + nk00)) +
                                 b0[j] * bk0 * (H01 + K01 * (m01[j] + nk01));
                const float T1 = a1[j] * ak1 * (H10 + K10 * (m10[j] + nk10)) +
                                 b1[j] * bk1 * (H11 + K11 * (m11[j] + nk11));
                const float g0 = (lk0.x - l0[j].x) + (lk0.y - l0[j].y);
                const float g1 = (lk1.x - l1[j].x) + (lk1.y - l1[j].y);
                // fast division (at most 2 ulp): the gaps are far from the range limits
                w = hdt * (__fdividef(T0, g0) + __fdividef(T1, g1));
            }
            W[(int64_t)j * Np + k] = w;
            Rk += fabsf(w);
        }
        if (k < Np - N)
            for (int j = 0; j < N; ++j) W[(int64_t)j * Np + N + k] = 0.0f;  // row padding
        // margin for the FP32 rounding of the row sum
        const double R = (double)Rk * (1.0 + 1e-5);
        const double Lk = 0.5 * dt * (s.lam_prev[t * N + k] + s.lam[t * N + k]);
        lo = fmin(lo, Lk - R);
        hi = fmax(hi, Lk + R);
    }
    lo = block_min(lo, red);
    hi = block_max(hi, red);
    if (threadIdx.x == 0) cheb_setup(s, t, lo, hi, tol);
}

// Hop acceptance: p' = p + alpha d with d = d_{m, s_a} (six components),
// alpha the energy-conserving root of smaller magnitude; occupations, the
// force on the new surface, counters, v_prev and the non-finite check.
__global__ void __launch_bounds__(64) k2_accept(DevState s, Model2Dev md)
{
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Ne = s.Ne;
    __shared__ double xs[6], ps[6], red[32];
    __shared__ int s_hopped;
    const int tid = threadIdx.x;
    if (tid < 6) {
        xs[tid] = s.x[t * 6 + tid];
        ps[tid] = s.p[t * 6 + tid];
    }
    __syncthreads();
    __shared__ Ads2 ad_sh;
    const Ads2 ad = ads2_block(md, xs, &ad_sh);
    if (tid == 0) {
        s_hopped = 0;
        const int pair = s.hop_pair[t];
        if (pair >= 0) {
            const int a = pair / N, m = pair - a * N;
            int16_t *occ = s.occ + t * Ne;
            const int sa = occ[a];
            const double *lam = s.lam + t * N, *Q0 = s.q0 + t * N, *Q1 = s.q2 + t * N;
            const double lm = lam[m], ls = lam[sa], lsum = lm + ls;
            const double A0 = Q0[m] * Q0[sa], A1 = Q1[m] * Q1[sa];
            double d[6], pd = 0.0, dd = 0.0;
            for (int y = 0; y < 6; ++y) {
                const double kp0 = y < 3 ? ad.kap[y] : 0.0, kp1 = y < 3 ? 0.0 : ad.kap[y];
                const double T = A0 * (md.th[2 + y] + kp0 * (lsum - 2.0 * ad.h[0])) +
                                 A1 * (md.th[8 + y] + kp1 * (lsum - 2.0 * ad.h[1]));
                d[y] = T / (ls - lm);
                pd += ps[y] * d[y];
                dd += d[y] * d[y];
            }
            const double dE = lm - ls;
            const double disc = pd * pd - 2.0 * md.mass * dd * dE;
            if (dd > 0.0 && disc >= 0.0) {
                const double alpha = (-pd + (pd >= 0.0 ? 1.0 : -1.0) * sqrt(disc)) / dd;
                for (int y = 0; y < 6; ++y) ps[y] += alpha * d[y];
                // replace s_a by m and keep the list ascending
                int b = a;
                occ[b] = (int16_t)m;
                while (b > 0 && occ[b - 1] > occ[b]) {
                    const int16_t tmp = occ[b - 1];
                    occ[b - 1] = occ[b];
                    occ[b] = tmp;
                    --b;
                }
                while (b < Ne - 1 && occ[b + 1] < occ[b]) {
                    const int16_t tmp = occ[b + 1];
                    occ[b + 1] = occ[b];
                    occ[b] = tmp;
                    ++b;
                }
                s.hops[t] += 1;
                s_hopped = 1;
            } else {
                s.frus[t] += 1;
            }
        }
    }
    __syncthreads();
    if (s_hopped) {  // uniform over the CTA
        double S[2], U[2];
        occ_sums(s.lam + t * N, s.q0 + t * N, s.q2 + t * N, s.occ + t * Ne, Ne, ad, red, S, U);
        if (tid < 6) s.F[t * 6 + tid] = force2(md, ad, xs, tid, S, U);
    }
    if (tid < 6) {
        s.p[t * 6 + tid] = ps[tid];
        s.vprev[t * 6 + tid] = ps[tid] / md.mass;
    }
    if (tid == 0) {
        if (s_hopped) write_geo2(s, t, md, ad, ps);  // projections at the new momentum
        s.nstep[t] += 1;
        bool bad = false;
        for (int y = 0; y < 6; ++y) bad |= !isfinite(xs[y]) || !isfinite(ps[y]);
        if (bad) atomicOr(&s.status[t], ST_NAN);
    }
}

// ------------------------------------------------ dense eigensolver path
// Two adsorbate orbitals whose couplings to the bath are not parallel (each
// orbital with its own bath profile) have no rank-two secular reduction;
// their eigenpairs come from the dense symmetric eigensolver of
// iesh_syev.cuh in three launches per step:
//   k2g_reduce  kick + drift (mode 1), H(x) built in shared memory (or in
//               the trajectory's scratch for large N), Householder reduction
//               with row 1 of the reflector product tracked;
//   k2g_ql      QL iterations, trajectories in lockstep across a warp,
//               rotating the adsorbate rows (row 0 of P is e_0, row 1
//               tracked);
//   k2g_finish  ascending order, gauge, forces, second kick.
// Everything after the eigenpairs (couplings, propagation, hops, rescale) is
// the rank-two path's: those kernels read only the eigenvalues and the two
// adsorbate rows, because the closed form of Q^T (dH/dy) Q above holds for
// any couplings of the form f_a(x) times a fixed vector over the bath.
//
// Gauge (reading R17): eigenvector j has sum_a c_a |prof_a| Q_aj >= 0, the
// rank-two path's rule; in a step, a decisive overlap with the previous
// step's eigenvector j (|overlap| >= 1/2) overrules it and is made
// non-negative.  The overlap uses the eigenvectors' bath rows, which follow
// from the adsorbate rows: B_kj = sum_a V_ak Q_aj / (lam_j - eps_k).

// Scratch of a trajectory: d[N], e[N], tracked rows Y[N][2], then the matrix
// (N x (N | 1)) when it does not fit in shared memory.
constexpr size_t kDenseSmemCap = 200 * 1024;

__host__ __device__ inline int dense_lda(int N) { return N | 1; }

__host__ __device__ inline bool dense_in_smem(int N)
{
    return (size_t)N * dense_lda(N) * 8 + (size_t)(6 * N + 8) * 8 <= kDenseSmemCap;
}

// Mode 1: the step's previous eigenpairs are kept, then the first kick and
// the drift; xs receives the geometry at which the eigenpairs are wanted.
// Block-wide; ends with a barrier.
__device__ __forceinline__ void kick_drift2(const DevState &s, const Model2Dev &md, int64_t t, double dt,
                                            int mode, double *xs)
{
    const int N = s.N, tid = threadIdx.x;
    if (mode == 1)
        for (int i = tid; i < N; i += blockDim.x) {
            s.lam_prev[t * N + i] = s.lam[t * N + i];
            s.q0_prev[t * N + i] = s.q0[t * N + i];
            s.q2_prev[t * N + i] = s.q2[t * N + i];
        }
    if (tid < 6) {
        double x = s.x[t * 6 + tid];
        if (mode == 1) {
            double p = s.p[t * 6 + tid];
            s.x_prev[t * 6 + tid] = x;
            p += 0.5 * dt * s.F[t * 6 + tid];
            x += dt * p / md.mass;
            s.x[t * 6 + tid] = x;
            s.p[t * 6 + tid] = p;
        }
        xs[tid] = x;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k2g_reduce(DevState s, Model2Dev md, double dt, int mode)
{
    extern __shared__ __align__(16) double g2_sh[];
    __shared__ double xs[6];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, M = s.M, lda = dense_lda(N), tid = threadIdx.x;
    kick_drift2(s, md, t, dt, mode, xs);
    __shared__ Ads2 ad_sh;
    const Ads2 ad = ads2_block(md, xs, &ad_sh);
    double *v = g2_sh, *w = v + N, *r1 = w + N, *d = r1 + N, *e = d + N, *tau = e + N, *sh = tau + N;
    double *out = s.scratch + t * s.scratch_stride;  // d, e, Y
    double *A = dense_in_smem(N) ? sh + 8 : out + 4 * N;
    for (int idx = tid; idx < N * lda; idx += blockDim.x) A[idx] = 0.0;
    __syncthreads();
    if (tid < 2) A[(size_t)tid * lda + tid] = ad.h[tid];
    for (int k = tid; k < M; k += blockDim.x) {
        const double v0 = ad.c[0] * md.prof[k], v1 = ad.c[1] * md.prof[M + k];
        A[(size_t)(2 + k) * lda + 2 + k] = s.eps[k];
        A[(size_t)k + 2] = v0;
        A[(size_t)(2 + k) * lda] = v0;
        A[(size_t)lda + 2 + k] = v1;
        A[(size_t)(2 + k) * lda + 1] = v1;
    }
    __syncthreads();
    householder_tridiag<double>(A, lda, N, d, e, tau, v, w, r1, sh, dense_in_smem(N));
    for (int i = tid; i < N; i += blockDim.x) {
        out[i] = d[i];
        out[N + i] = e[i];
        out[2 * N + 2 * i] = i == 0 ? 1.0 : 0.0;
        out[2 * N + 2 * i + 1] = r1[i];
    }
}

// L trajectories per warp in lockstep (ql_lockstep), four warps per CTA:
// work item (warp index) L + lane.
__global__ void __launch_bounds__(128) k2g_ql(DevState s, int L)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw * L >= s.n) return;  // the whole warp: past the batch
    const int64_t t = lane < L ? traj_of(s, gw * L + lane) : -1;
    const bool valid = t >= 0 && !(s.status[t] & ST_DONE);
    const int N = s.N;
    double *b = s.scratch + (valid ? t : 0) * s.scratch_stride;
    const bool ok = ql_lockstep<double, 2>(N, b, b + N, 1, b + 2 * N, 2, 1, valid);
    if (valid && !ok) atomicOr(&s.status[t], ST_SECULAR);
}

// sorted: the eigenvalues arrive in ascending order (the nested secular
// path), so the rank sort (N^2 FP64 comparisons) is skipped.
__global__ void __launch_bounds__(256) k2g_finish(DevState s, Model2Dev md, double dt, int mode, int sorted)
{
    extern __shared__ __align__(16) double f2_sh[];
    __shared__ double xs[6], ps[6], xp[6], red[32];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, M = s.M, Ne = s.Ne, tid = threadIdx.x;
    double *ev = f2_sh, *y0 = ev + N, *y1 = y0 + N, *lam_s = y1 + N, *Q0_s = lam_s + N, *Q1_s = Q0_s + N;
    const double *b = s.scratch + t * s.scratch_stride;
    if (tid < 6) {
        xs[tid] = s.x[t * 6 + tid];
        ps[tid] = s.p[t * 6 + tid];
        xp[tid] = s.x_prev[t * 6 + tid];
    }
    for (int i = tid; i < N; i += blockDim.x) {
        ev[i] = b[i];
        y0[i] = b[2 * N + 2 * i];
        y1[i] = b[2 * N + 2 * i + 1];
    }
    __syncthreads();
    __shared__ Ads2 ad_sh;
    const Ads2 ad = ads2_block(md, xs, &ad_sh);
    for (int i = tid; i < N; i += blockDim.x) {  // ascending, ties by index
        const double li = ev[i];
        int r = i;
        if (!sorted) {
            r = 0;
            for (int j = 0; j < N; ++j) r += (ev[j] < li) || (ev[j] == li && j < i);
        }
        lam_s[r] = li;
        Q0_s[r] = y0[i];
        Q1_s[r] = y1[i];
    }
    __syncthreads();
    {
        const double g0 = ad.c[0] * md.pnorm[0], g1 = ad.c[1] * md.pnorm[1];
        for (int j = tid; j < N; j += blockDim.x)
            if (g0 * Q0_s[j] + g1 * Q1_s[j] < 0.0) {
                Q0_s[j] = -Q0_s[j];
                Q1_s[j] = -Q1_s[j];
            }
    }
    if (mode == 1) {
        // overlap with the previous step's eigenvector j (bath rows rebuilt
        // from the adsorbate rows; FP32 sums: only the comparison with -1/2
        // is used)
        __shared__ Ads2 adp_sh;
        const Ads2 adp = ads2_block(md, xp, &adp_sh);
        for (int j = tid; j < N; j += blockDim.x) {
            const double q0 = Q0_s[j], q1 = Q1_s[j], lj = lam_s[j];
            const double p0 = s.q0_prev[t * N + j], p1 = s.q2_prev[t * N + j], lp = s.lam_prev[t * N + j];
            const float a0 = (float)(ad.c[0] * q0), a1 = (float)(ad.c[1] * q1);
            const float b0 = (float)(adp.c[0] * p0), b1 = (float)(adp.c[1] * p1);
            const float ljf = (float)lj, lpf = (float)lp;
            float ov = (float)(q0 * p0 + q1 * p1);
            for (int k = 0; k < M; ++k) {
                const float f0 = (float)md.prof[k], f1 = (float)md.prof[M + k], ek = (float)s.eps[k];
                const float den = (ljf - ek) * (lpf - ek);
                if (den != 0.0f) ov += __fdividef((a0 * f0 + a1 * f1) * (b0 * f0 + b1 * f1), den);
            }
            if (ov <= -0.5f) {
                Q0_s[j] = -q0;
                Q1_s[j] = -q1;
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < N; j += blockDim.x) {
        s.lam[t * N + j] = lam_s[j];
        s.q0[t * N + j] = Q0_s[j];
        s.q2[t * N + j] = Q1_s[j];
        if (mode == 0) s.lam_prev[t * N + j] = lam_s[j];
    }
    double S[2], U[2];
    occ_sums(lam_s, Q0_s, Q1_s, s.occ + t * Ne, Ne, ad, red, S, U);
    if (tid < 6) {
        const double F = force2(md, ad, xs, tid, S, U);
        double p = ps[tid];
        if (mode == 1) p += 0.5 * dt * F;
        s.p[t * 6 + tid] = p;
        s.F[t * 6 + tid] = F;
        if (mode == 0) s.vprev[t * 6 + tid] = p / md.mass;
        ps[tid] = p;
    }
    __syncthreads();
    if (tid == 0) write_geo2(s, t, md, ad, ps);
}

// ------------------------------------------------ nested secular path
// The same eigenpairs without the O(N^3) reduction: H is diag(h_0, h_1,
// eps) bordered by V_0k = c_0 prof_0k and V_1k = c_1 prof_1k, and a
// similarity by the eigenvectors of one bordered block leaves another
// arrowhead (two nested secular equations, one root per thread each).
//   Step 1: orbital 1 with the bath, poles eps_k and weights V_1k^2: M + 1
//     roots mu_j; eigenvector w_j has orbital-1 component s_j = 1 /
//     sqrt(f_1'(mu_j)) and bath components V_1k s_j / (mu_j - eps_k).
//   Step 2: in the basis {|0>, w_j}, H is diag(h_0, mu) bordered by c_j =
//     <0|H|w_j> = s_j sum_k V_0k V_1k / (mu_j - eps_k); its N = M + 2 roots
//     are the eigenvalues of H, the border component q_i = 1 / sqrt(f_2'(
//     lam_i)) is Q_0i, and Q_1i = sum_j <1|w_j><w_j|i> = q_i sum_j s_j c_j /
//     (lam_i - mu_j).
// Every difference between a root and a pole is formed about the root's
// origin pole (pole difference + offset) and keeps its relative accuracy;
// the step-2 pole differences mu_o - mu_k are differences of computed
// roots, which perturbs the step-2 arrowhead at the rounding level of its
// entries.  The eigenpairs go to the trajectory's scratch in the dense
// path's layout (lam[N], then Q_0i, Q_1i pairs from 2N), ascending, for
// k2g_finish (gauge, forces, second kick).
// Mode 1 starts both root searches from the previous step's roots (warm
// start, as the one-orbital kernel): the step-1 roots kept in md.mu and the
// eigenvalues.  DF (mixed path): the step-1 sums over the bath poles in
// double-float from the pole-difference table, as k_eigen<true>.
// (Without a register budget the compiler settles on 80 registers and
// spills; 128 keeps everything in registers with two 256-thread CTAs per SM.)
template <bool DF>
__global__ void __maxnreg__(128) k2n_eigen(DevState s, Model2Dev md, double dt, int mode)
{
    extern __shared__ __align__(16) double n2_sh[];
    __shared__ double xs[6], red[32];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, M = s.M, M1 = M + 1, tid = threadIdx.x;
    const bool warm = mode == 1;
    // previous roots, read before kick_drift2 moves lam to lam_prev (it
    // leaves lam itself alone)
    const double g1 = (warm && tid < M1) ? md.mu[t * M1 + tid] : 0.0;
    const double g2 = (warm && tid < N) ? s.lam[t * N + tid] : 0.0;
    kick_drift2(s, md, t, dt, mode, xs);
    __shared__ Ads2 ad_sh;
    const Ads2 ad = ads2_block(md, xs, &ad_sh);
    double *eps_s = n2_sh, *z2 = eps_s + M, *mu = z2 + M, *sv = mu + M1, *c2 = sv + M1, *cs = c2 + M1,
           *tau1 = cs + M1;
    int *o1 = reinterpret_cast<int *>(tau1 + M1);
    float2 *z2df = reinterpret_cast<float2 *>(tau1 + 2 * M1);  // [M] (DF)
    // DF: tau1, c_j^2 and s_j c_j as double-float pairs for the step-2 sums
    float2 *t1df = z2df + M, *c2df = t1df + M1, *csdf = c2df + M1;
    double z1 = 0.0;
    for (int k = tid; k < M; k += blockDim.x) {
        eps_s[k] = s.eps[k];
        const double v1 = ad.c[1] * md.prof[M + k];
        z2[k] = v1 * v1;
        if (DF) {
            const dfl zd = dfl_from(v1 * v1);
            z2df[k] = make_float2(zd.hi, zd.lo);
        }
        z1 += v1 * v1;
    }
    const double Z1 = block_sum(z1, red);  // ends with a barrier: eps_s, z2 complete
    uint32_t st = 0;
    // step 1: orbital 1 and the bath
    if (tid < M1) {
        double l, q, tau = 0.0;
        int o = 0;
        if (Z1 > 0.0) {
            if (DF) {
                const Poles<double> pp = {M, eps_s, z2, nullptr, s.poledf, z2df, 0, -1, 0.0, nullptr};
                secular_root<double, EV_DFLOAT>(tid, pp, ad.h[1], Z1, warm, g1, l, q, st, &o, &tau);
            } else {
                const Poles<double> pp = {M, eps_s, z2, nullptr, nullptr, nullptr, 0, -1, 0.0, nullptr};
                secular_root<double, EV_PLAIN>(tid, pp, ad.h[1], Z1, warm, g1, l, q, st, &o, &tau);
            }
        } else {
            // orbital 1 uncoupled: the roots are h_1 (s = 1) and the bath energies
            int pos = 0;
            for (int k = 0; k < M; ++k) pos += (eps_s[k] < ad.h[1]);
            l = tid < pos ? eps_s[tid] : (tid == pos ? ad.h[1] : eps_s[tid - 1]);
            q = tid == pos ? 1.0 : 0.0;
            o = tid < pos ? tid : (tid == pos ? -1 : tid - 1);  // bath root: its pole
        }
        mu[tid] = l;
        sv[tid] = q;
        o1[tid] = o;
        tau1[tid] = tau;
        if (DF) {
            const dfl td = dfl_from(tau);
            t1df[tid] = make_float2(td.hi, td.lo);
        }
        md.mu[t * M1 + tid] = l;
    }
    __syncthreads();
    // couplings of orbital 0 to the step-1 eigenvectors
    double zc = 0.0;
    if (tid < M1) {
        const int o = o1[tid];
        double cj;
        if (Z1 > 0.0) {
            const double tau = tau1[tid];
            double gs = 0.0;
            if (DF) {
                // sum_k prof_0k prof_1k / ((eps_o - eps_k) + tau) in double-float
                const dfl td = dfl_from(tau);
                dfl a[2] = {{0.f, 0.f}, {0.f, 0.f}};
                auto term = [&](int k, int h) {
                    const float2 dk = s.poledf[(size_t)k * M + o], pk = md.ppdf[k];
                    const dfl r = dfl_rcp(dfl_add({dk.x, dk.y}, td));
                    a[h] = dfl_add(a[h], dfl_mul({pk.x, pk.y}, r));
                };
                int k = 0;
                for (; k + 1 < M; k += 2) {
                    term(k, 0);
                    term(k + 1, 1);
                }
                if (k < M) term(k, 0);
                gs = dfl_value(dfl_add(a[0], a[1]));
            } else {
                const double eo = eps_s[o];
                for (int k = 0; k < M; ++k)
                    gs += md.prof[k] * md.prof[M + k] * pole_recip<double>((eo - eps_s[k]) + tau);
            }
            cj = ad.c[0] * ad.c[1] * sv[tid] * gs;
        } else {
            cj = o >= 0 ? ad.c[0] * md.prof[o] : 0.0;  // w_j is bath state o, or orbital 1
        }
        c2[tid] = cj * cj;
        cs[tid] = cj * sv[tid];
        if (DF) {
            const dfl a = dfl_from(cj * cj), b = dfl_from(cj * sv[tid]);
            c2df[tid] = make_float2(a.hi, a.lo);
            csdf[tid] = make_float2(b.hi, b.lo);
        }
        zc = cj * cj;
    }
    const double Z2 = block_sum(zc, red);  // ends with a barrier: mu, c2, cs complete
    // step 2: orbital 0 against the step-1 eigenvectors
    if (tid < N) {
        double l, q0, q1 = 0.0, tau = 0.0;
        int o = 0;
        if (Z2 > 0.0 && DF && Z1 > 0.0) {
            // the step-1 roots carry their bath pole: double-float sums
            const Poles<double> pp = {M1, mu, c2, nullptr, s.poledf, c2df, M, -1, 0.0, t1df, o1};
            secular_root<double, EV_NESTED>(tid, pp, ad.h[0], Z2, warm, g2, l, q0, st, &o, &tau);
            const dfl td = dfl_from(tau);
            dfl a[2] = {{0.f, 0.f}, {0.f, 0.f}};
            auto term = [&](int j, int h) {
                if (j == o) return;
                const dfl r = dfl_rcp(nested_gap(pp, o, j, td));
                const float2 cj = csdf[j];
                a[h] = dfl_add(a[h], dfl_mul({cj.x, cj.y}, r));
            };
            int j = 0;
            for (; j + 1 < M1; j += 2) {
                term(j, 0);
                term(j + 1, 1);
            }
            if (j < M1) term(j, 0);
            q1 = q0 * (dfl_value(dfl_add(a[0], a[1])) + cs[o] / tau);
        } else if (Z2 > 0.0) {
            const Poles<double> pp = {M1, mu, c2, nullptr, nullptr, nullptr, 0, -1, 0.0, nullptr};
            secular_root<double, EV_PLAIN>(tid, pp, ad.h[0], Z2, warm, g2, l, q0, st, &o, &tau);
            const double mo = mu[o];
            double ss = 0.0;
            for (int j = 0; j < M1; ++j) ss += cs[j] * pole_recip<double>((mo - mu[j]) + tau);
            q1 = q0 * ss;
        } else {
            // orbital 0 uncoupled: the roots are h_0 (Q_0 = 1) and the mu_j (Q_1 = s_j)
            int pos = 0;
            for (int j = 0; j < M1; ++j) pos += (mu[j] < ad.h[0]);
            l = tid < pos ? mu[tid] : (tid == pos ? ad.h[0] : mu[tid - 1]);
            q0 = tid == pos ? 1.0 : 0.0;
            q1 = tid < pos ? sv[tid] : (tid == pos ? 0.0 : sv[tid - 1]);
        }
        double *out = s.scratch + t * s.scratch_stride;
        out[tid] = l;
        out[2 * N + 2 * tid] = q0;
        out[2 * N + 2 * tid + 1] = q1;
    }
    if (st) atomicOr(&s.status[t], st);
}

size_t nested_smem(int M) { return (size_t)(3 * M + 9 * (M + 1)) * sizeof(double); }

size_t dense_reduce_smem(int N)
{
    return (size_t)(6 * N + 8) * sizeof(double) + (dense_in_smem(N) ? (size_t)N * dense_lda(N) * sizeof(double) : 0);
}

// Shared memory of k2_eigen with tpb slots.
size_t eigen2_smem(int N, int M, int tpb, bool df)
{
    const int per = 2 * (M + 1) + 3 * N + 4 * eigen_pow2(N) + (df ? 2 * M + 1 : 0);
    return (size_t)(M + tpb * per) * sizeof(double) + (size_t)tpb * sizeof(Eig2Slot);
}

}  // namespace

struct iesh2_ctx {
    iesh2_model model;
    int64_t max_traj = 0;
    cudaStream_t stream = nullptr;
    int N = 0, M = 0, Ne = 0;
    int skip_bound = 0;
    bool mixed = false;
    bool dense = false;  // eigenpairs from the dense symmetric eigensolver
    bool nested = false; // eigenpairs from two nested secular equations
    int sms = 1;         // SMs of the context's device
    Model2Dev md;
    DevState ds;
    std::vector<void *> allocs;
    bool have_state = false;
    std::string err;
    KernelTimer timer;
};

namespace {

iesh_status fail2(iesh2_ctx *c, iesh_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CU2(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail2(ctx, IESH_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                         __FILE__, __LINE__);                                               \
    } while (0)

template <class T>
iesh_status dalloc2(iesh2_ctx *ctx, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess)
        return fail2(ctx, IESH_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    ctx->allocs.push_back(q);
    *p = (T *)q;
    CU2(cudaMemsetAsync(q, 0, bytes, ctx->stream));
    return IESH_OK;
}

iesh_status copy_out2(iesh2_ctx *ctx, void *dst, const void *src, size_t bytes, bool &sync)
{
    if (!bytes || !dst) return IESH_OK;
    CU2(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    if (is_host_ptr(dst)) sync = true;
    return IESH_OK;
}

cudaError_t launch_eigen2(iesh2_ctx *ctx, double dt, int mode)
{
    const DevState &d = ctx->ds;
    if (d.n == 0) return cudaSuccess;
    if (ctx->nested) {
        const int threads = (d.N + 31) & ~31;
        if (ctx->mixed) k2n_eigen<true><<<(unsigned)d.n, threads, nested_smem(d.M), ctx->stream>>>(d, ctx->md, dt, mode);
        else k2n_eigen<false><<<(unsigned)d.n, threads, nested_smem(d.M), ctx->stream>>>(d, ctx->md, dt, mode);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k2g_finish<<<(unsigned)d.n, 256, (size_t)6 * d.N * sizeof(double), ctx->stream>>>(d, ctx->md, dt, mode, 1);
        return cudaGetLastError();
    }
    if (ctx->dense) {
        k2g_reduce<<<(unsigned)d.n, 256, dense_reduce_smem(d.N), ctx->stream>>>(d, ctx->md, dt, mode);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int L = ql_lockstep_lanes(d.n, ctx->sms);
        const int64_t warps = (d.n + L - 1) / L;
        k2g_ql<<<(unsigned)((warps + 3) / 4), 128, 0, ctx->stream>>>(d, L);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k2g_finish<<<(unsigned)d.n, 256, (size_t)6 * d.N * sizeof(double), ctx->stream>>>(d, ctx->md, dt, mode, 0);
        return cudaGetLastError();
    }
    const int tpb = eigen_tpb(d.N);
    const int threads = (tpb * d.N + 31) & ~31;
    const unsigned blocks = (unsigned)((d.n + tpb - 1) / tpb);
    const size_t smem = eigen2_smem(d.N, d.M, tpb, ctx->mixed);
    if (ctx->mixed) k2_eigen<true><<<blocks, threads, smem, ctx->stream>>>(d, ctx->md, dt, mode, tpb);
    else k2_eigen<false><<<blocks, threads, smem, ctx->stream>>>(d, ctx->md, dt, mode, tpb);
    return cudaGetLastError();
}

cudaError_t launch_build_w2(iesh2_ctx *ctx, double dt, double tol)
{
    const DevState &d = ctx->ds;
    if (d.n == 0) return cudaSuccess;
    const int threads = std::min(256, (d.N + 31) & ~31);
    if (ctx->mixed)
        k2_build_w_f32<<<(unsigned)d.n, threads,
                         (size_t)32 * sizeof(double) + (size_t)2 * d.N * sizeof(float2) + (size_t)8 * d.N * sizeof(float),
                         ctx->stream>>>(d, ctx->md, dt, tol);
    else
        k2_build_w<<<(unsigned)d.n, threads, (size_t)(6 * d.N + 32) * sizeof(double), ctx->stream>>>(
            d, ctx->md, dt, tol);
    return cudaGetLastError();
}

size_t coeff_bytes(const iesh2_ctx *ctx) { return ctx->mixed ? 8 : 16; }

cudaError_t launch_accept2(iesh2_ctx *ctx)
{
    const DevState &d = ctx->ds;
    if (d.n == 0) return cudaSuccess;
    k2_accept<<<(unsigned)d.n, 64, 0, ctx->stream>>>(d, ctx->md);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

const char *iesh2_last_error(const iesh2_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

iesh_status iesh2_destroy(iesh2_ctx *ctx)
{
    if (!ctx) return IESH_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->timer.release();
    for (void *p : ctx->allocs) cudaFree(p);
    delete ctx;
    return IESH_OK;
}

iesh_status iesh2_create(iesh2_ctx **out, const iesh2_model *model, int precision, int64_t max_traj,
                         int skip_bound, void *cuda_stream)
{
    if (!out) return IESH_EINVAL;
    *out = nullptr;
    if (!model || max_traj < 1) return IESH_EINVAL;
    iesh2_ctx *ctx = new iesh2_ctx();
    *out = ctx;
    ctx->model = *model;
    ctx->max_traj = max_traj;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->skip_bound = skip_bound;
    const int M = model->n_bath, Ne = model->n_elec, N = M + 2;
    if (M < 2 || N > kMaxOrbitals) return fail2(ctx, IESH_EINVAL, "n_bath %d outside 2..%d", M, kMaxOrbitals - 2);
    if (Ne < 1 || Ne > N - 1) return fail2(ctx, IESH_EINVAL, "n_elec %d outside 1..N-1", Ne);
    if (Ne > kMaxHopElectrons) return fail2(ctx, IESH_EINVAL, "n_elec %d above %d", Ne, kMaxHopElectrons);
    if (!(model->mass > 0.0)) return fail2(ctx, IESH_EINVAL, "mass must be positive");
    if (!(model->band_hi > model->band_lo)) return fail2(ctx, IESH_EINVAL, "empty band");
    if (!(model->theta[14] != 0.0 && model->theta[15] != 0.0))
        return fail2(ctx, IESH_EINVAL, "coupling widths theta[14], theta[15] must be nonzero");
    if (precision != IESH_PREC_FP64 && precision != IESH_PREC_MIXED)
        return fail2(ctx, IESH_EINVAL, "unknown precision %d", precision);
    if (model->profile != 0 && model->profile != 1)
        return fail2(ctx, IESH_EINVAL, "unknown coupling profile %d", model->profile);
    if (model->profile == 1 && !(model->prof_width[0] > 0.0 && model->prof_width[1] > 0.0))
        return fail2(ctx, IESH_EINVAL, "profile widths must be positive");
    if (model->eigensolver != 0 && model->eigensolver != 1)
        return fail2(ctx, IESH_EINVAL, "unknown eigensolver %d", model->eigensolver);
    ctx->mixed = precision == IESH_PREC_MIXED;
    ctx->dense = model->eigensolver == 1;
    ctx->nested = model->profile == 1 && model->eigensolver == 0;
    {
        int dev = 0, sms = 0;
        CU2(cudaGetDevice(&dev));
        CU2(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        ctx->sms = sms;
    }
    ctx->N = N;
    ctx->M = M;
    ctx->Ne = Ne;
    Model2Dev &k = ctx->md;
    for (int i = 0; i < 16; ++i) k.th[i] = model->theta[i];
    for (int a = 0; a < 2; ++a) k.vbar[a] = model->vbar[a];
    for (int i = 0; i < 6; ++i) {
        k.R[i] = model->R[i];
        k.x0[i] = model->x0[i];
    }
    k.mass = model->mass;
    k.omega = model->omega;
    // split Gauss-Legendre bath at mu, M/2 nodes below (Appendix A)
    std::vector<double> eps, w;
    lead_bath(IESH_DISC_GL_SPLIT, M, model->band_lo, model->band_hi, model->mu, M / 2, eps, w);
    for (int i = 1; i < M; ++i)
        if (!(eps[i] > eps[i - 1])) return fail2(ctx, IESH_EINVAL, "bath energies must be distinct");
    std::vector<double> sq(M);
    k.wsum = 0.0;
    for (int i = 0; i < M; ++i) {
        sq[i] = std::sqrt(w[i]);
        k.wsum += sq[i] * sq[i];
    }

    DevState &d = ctx->ds;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.M = M;
    d.Ne = Ne;
    const size_t T = (size_t)max_traj;
    d.scratch_stride = std::max<int64_t>((int64_t)N * N, 3LL * Ne * N + Ne);
    if (ctx->dense)  // d, e, tracked rows and the matrix when it is not in shared memory
        d.scratch_stride = std::max<int64_t>(d.scratch_stride, 4LL * N + (int64_t)N * dense_lda(N));
    d.scratch_stride = (d.scratch_stride + 31) & ~31LL;
    iesh_status st;
    double *eps_d = nullptr, *sq_d = nullptr, *Cd = nullptr, *prof_d = nullptr;
#define A2(ptr, cnt) if ((st = dalloc2(ctx, &(ptr), (cnt))) != IESH_OK) return st;
    A2(d.x, T * 6) A2(d.p, T * 6) A2(d.F, T * 6) A2(d.vprev, T * 6) A2(d.x_prev, T * 6)
    A2(d.occ, T * Ne)
    A2(Cd, T * Ne * N * 2)
    A2(d.lam, T * N) A2(d.q0, T * N) A2(d.q2, T * N)
    A2(d.lam_prev, T * N) A2(d.q0_prev, T * N) A2(d.q2_prev, T * N)
    A2(d.geo2, T * 8)
    A2(d.hop_pair, T)
    A2(d.status, T) A2(d.nstep, T) A2(d.hops, T) A2(d.frus, T)
    A2(d.scratch, T * (size_t)d.scratch_stride)
    A2(d.cheb, T * kChebStride)
    double *mu_d = nullptr;
    float2 *ppdf_d = nullptr;
    if (ctx->nested) A2(mu_d, T * (size_t)(M + 1))
    if (ctx->nested && ctx->mixed) A2(ppdf_d, (size_t)M)
    A2(eps_d, (size_t)M) A2(sq_d, (size_t)M) A2(prof_d, (size_t)2 * M)
    float2 *poledf = nullptr;
    if (ctx->mixed) A2(poledf, (size_t)M * M)
#undef A2
    d.C = Cd;
    d.eps = eps_d;
    d.z0 = sq_d;
    d.poledf = poledf;
    d.eigen_dfloat = ctx->mixed ? 1 : 0;
    configure_hop_smem();
    configure_cheb_tc();
    configure_cheb_tc16();
    // the slots of the eigen kernel can pass the 48 KiB default (N near 65)
    CU2(cudaFuncSetAttribute(k2_eigen<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)eigen2_smem(N, M, eigen_tpb(N), false)));
    CU2(cudaFuncSetAttribute(k2_eigen<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)eigen2_smem(N, M, eigen_tpb(N), true)));
    CU2(cudaMemcpyAsync(eps_d, eps.data(), M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU2(cudaMemcpyAsync(sq_d, sq.data(), M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // coupling profiles of the dense path: sqrt(w_k), times the Lorentzian
    // 1 / sqrt(1 + ((eps_k - centre_a) / width_a)^2) of each orbital (profile 1)
    std::vector<double> prof((size_t)2 * M);
    for (int a = 0; a < 2; ++a) {
        double nrm = 0.0;
        for (int i = 0; i < M; ++i) {
            double v = sq[i];
            if (model->profile == 1) {
                const double u = (eps[i] - model->prof_center[a]) / model->prof_width[a];
                v /= std::sqrt(1.0 + u * u);
            }
            prof[(size_t)a * M + i] = v;
            nrm += v * v;
        }
        k.pnorm[a] = std::sqrt(nrm);
    }
    k.prof = prof_d;
    k.mu = mu_d;
    k.ppdf = ppdf_d;
    CU2(cudaMemcpyAsync(prof_d, prof.data(), prof.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->dense && dense_reduce_smem(N) > 48 * 1024) {
        // process-wide attribute: only ever raised
        cudaFuncAttributes fa;
        CU2(cudaFuncGetAttributes(&fa, k2g_reduce));
        if (fa.maxDynamicSharedSizeBytes < (int)dense_reduce_smem(N))
            CU2(cudaFuncSetAttribute(k2g_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kDenseSmemCap + 2048)));
    }
    std::vector<float2> pf;
    if (ctx->mixed) {
        // bath pole differences eps_o - eps_k as double-float pairs, [k][o]
        pf.resize((size_t)M * M);
        for (int kk = 0; kk < M; ++kk)
            for (int o = 0; o < M; ++o) {
                const double v = eps[o] - eps[kk];
                const float hi = (float)v;
                pf[(size_t)kk * M + o] = make_float2(hi, (float)(v - (double)hi));
            }
        CU2(cudaMemcpyAsync(poledf, pf.data(), pf.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
    }
    std::vector<float2> ppf;
    if (ppdf_d) {
        // prof_0k prof_1k as double-float pairs (the nested path's couplings)
        ppf.resize((size_t)M);
        for (int kk = 0; kk < M; ++kk) {
            const double v = prof[kk] * prof[(size_t)M + kk];
            const float hi = (float)v;
            ppf[kk] = make_float2(hi, (float)(v - (double)hi));
        }
        CU2(cudaMemcpyAsync(ppdf_d, ppf.data(), ppf.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
    }
    CU2(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh2_set_state(iesh2_ctx *ctx, int64_t n_traj, const double *x, const double *p,
                            const int16_t *occ, const void *C)
{
    if (!ctx) return IESH_EINVAL;
    if (n_traj < 0 || n_traj > ctx->max_traj)
        return fail2(ctx, IESH_EINVAL, "n_traj %lld outside 0..%lld", (long long)n_traj,
                     (long long)ctx->max_traj);
    if (!x || !p || !occ || !C) return fail2(ctx, IESH_EINVAL, "set_state needs x, p, occ and C");
    DevState &d = ctx->ds;
    d.n = n_traj;
    const size_t n = (size_t)n_traj;
    if (n) {
        CU2(cudaMemsetAsync(d.status, 0, n * sizeof(uint32_t), ctx->stream));
        CU2(cudaMemsetAsync(d.nstep, 0, n * sizeof(int64_t), ctx->stream));
        CU2(cudaMemsetAsync(d.hops, 0, n * sizeof(int32_t), ctx->stream));
        CU2(cudaMemsetAsync(d.frus, 0, n * sizeof(int32_t), ctx->stream));
        CU2(cudaMemcpyAsync(d.x, x, n * 6 * sizeof(double), cudaMemcpyDefault, ctx->stream));
        CU2(cudaMemcpyAsync(d.p, p, n * 6 * sizeof(double), cudaMemcpyDefault, ctx->stream));
        CU2(cudaMemcpyAsync(d.occ, occ, n * ctx->Ne * sizeof(int16_t), cudaMemcpyDefault, ctx->stream));
        CU2(cudaMemcpyAsync(d.C, C, n * ctx->Ne * ctx->N * coeff_bytes(ctx), cudaMemcpyDefault, ctx->stream));
    }
    CU2(launch_eigen2(ctx, 0.0, 0));
    // host sources may be pageable: the copies above must finish before return
    CU2(cudaStreamSynchronize(ctx->stream));
    ctx->have_state = true;
    return IESH_OK;
}

iesh_status iesh2_get_state(iesh2_ctx *ctx, double *x, double *p, int16_t *occ, void *C, uint32_t *status)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    const size_t n = (size_t)d.n;
    bool sync = false;
    iesh_status st;
    if ((st = copy_out2(ctx, x, d.x, n * 6 * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out2(ctx, p, d.p, n * 6 * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out2(ctx, occ, d.occ, n * ctx->Ne * sizeof(int16_t), sync)) != IESH_OK) return st;
    if ((st = copy_out2(ctx, C, d.C, n * ctx->Ne * ctx->N * coeff_bytes(ctx), sync)) != IESH_OK) return st;
    if ((st = copy_out2(ctx, status, d.status, n * sizeof(uint32_t), sync)) != IESH_OK) return st;
    if (sync) CU2(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh2_get_eigen(iesh2_ctx *ctx, double *lam, double *Q, double *F)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    const size_t n = (size_t)d.n, N = (size_t)ctx->N;
    bool sync = false;
    iesh_status st;
    if ((st = copy_out2(ctx, lam, d.lam, n * N * sizeof(double), sync)) != IESH_OK) return st;
    if (Q && n) {
        // rows of [n][2][N]: orbital-0 components, then orbital-1 components
        CU2(cudaMemcpy2DAsync(Q, 2 * N * sizeof(double), d.q0, N * sizeof(double), N * sizeof(double), n,
                              cudaMemcpyDefault, ctx->stream));
        CU2(cudaMemcpy2DAsync(Q + N, 2 * N * sizeof(double), d.q2, N * sizeof(double), N * sizeof(double), n,
                              cudaMemcpyDefault, ctx->stream));
        if (is_host_ptr(Q)) sync = true;
    }
    if ((st = copy_out2(ctx, F, d.F, n * 6 * sizeof(double), sync)) != IESH_OK) return st;
    if (sync) CU2(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh2_run(iesh2_ctx *ctx, double dt, int64_t n_steps, uint64_t seed)
{
    if (!ctx) return IESH_EINVAL;
    if (!ctx->have_state) return fail2(ctx, IESH_ESTATE, "run before set_state");
    if (!(dt > 0.0) || n_steps < 0) return fail2(ctx, IESH_EINVAL, "need dt > 0 and n_steps >= 0");
    const DevState &d = ctx->ds;
    const cudaStream_t st = ctx->stream;
    const bool mx = ctx->mixed;
    // Chebyshev truncation at the rounding level of the propagation's precision
    const double tol = mx ? 1e-7 : 1e-15;
    for (int64_t k = 0; k < n_steps; ++k) {
        CU2(ctx->timer.run(st, IESH_K_EIGEN, [&] { return launch_eigen2(ctx, dt, 1); }));
        CU2(ctx->timer.run(st, IESH_K_COUPLING, [&] { return launch_build_w2(ctx, dt, tol); }));
        CU2(ctx->timer.run(st, IESH_K_PROPAGATE, [&] { return launch_cheb(d, dt, mx, st); }));
        CU2(ctx->timer.run(st, IESH_K_HOP, [&] {
            return launch_hop(d, dt, ctx->md.mass, seed, ctx->skip_bound, nullptr, st, mx, true);
        }));
        CU2(ctx->timer.run(st, IESH_K_OTHER, [&] { return launch_accept2(ctx); }));
    }
    return IESH_OK;
}

iesh_status iesh2_hop_probabilities(iesh2_ctx *ctx, double dt, double *g)
{
    if (!ctx || !g) return IESH_EINVAL;
    if (!ctx->have_state) return fail2(ctx, IESH_ESTATE, "hop_probabilities before set_state");
    const DevState &d = ctx->ds;
    const size_t bytes = (size_t)d.n * ctx->Ne * ctx->N * sizeof(double);
    if (!bytes) return IESH_OK;
    double *dst = g, *tmp = nullptr;
    const bool host = is_host_ptr(g);
    if (host) {
        CU2(cudaMallocAsync((void **)&tmp, bytes, ctx->stream));
        dst = tmp;
    }
    CU2(launch_hop(d, dt, ctx->md.mass, 0, 0, dst, ctx->stream, ctx->mixed, true));
    if (host) {
        CU2(cudaMemcpyAsync(g, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU2(cudaFreeAsync(tmp, ctx->stream));
        CU2(cudaStreamSynchronize(ctx->stream));
    }
    return IESH_OK;
}

iesh_status iesh2_get_counters(iesh2_ctx *ctx, int64_t *nstep, int32_t *hops, int32_t *frustrated)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    const size_t n = (size_t)d.n;
    bool sync = false;
    iesh_status st;
    if ((st = copy_out2(ctx, nstep, d.nstep, n * sizeof(int64_t), sync)) != IESH_OK) return st;
    if ((st = copy_out2(ctx, hops, d.hops, n * sizeof(int32_t), sync)) != IESH_OK) return st;
    if ((st = copy_out2(ctx, frustrated, d.frus, n * sizeof(int32_t), sync)) != IESH_OK) return st;
    if (sync) CU2(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh2_profile(iesh2_ctx *ctx, int enable)
{
    if (!ctx) return IESH_EINVAL;
    CU2(cudaStreamSynchronize(ctx->stream));
    ctx->timer.reset(enable != 0);
    return IESH_OK;
}

iesh_status iesh2_profile_read(iesh2_ctx *ctx, double *ms, int64_t *launches)
{
    if (!ctx) return IESH_EINVAL;
    CU2(cudaStreamSynchronize(ctx->stream));
    CU2(ctx->timer.fold());
    for (int i = 0; i < IESH_K_COUNT; ++i) {
        if (ms) ms[i] = ctx->timer.ms[i];
        if (launches) launches[i] = ctx->timer.n[i];
    }
    return IESH_OK;
}

}  // extern "C"
