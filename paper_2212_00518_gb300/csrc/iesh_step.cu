// iesh_step.cu -- kernels of one batched IESH step (sm_103a), FP64 and the
// mixed-precision variants (k_build_w_f32, k_cheb_f32t, k_hop<float2, ...>).
//
// One trajectory step (Gardner et al., arXiv:2212.00518, Sec. II B-C):
//   k_eigen     velocity-Verlet kick + drift, eigenpairs of the arrowhead
//               one-electron Hamiltonian by its secular equation, force on
//               the occupied surface, second kick;
//   k_build_w   step-averaged coupling generator W = dt/2 (v0 D0 + v1 D1),
//               D_jk = <j|d_x k>, its Gershgorin spectral interval and the
//               Chebyshev coefficients of exp(-i Abar dt);
//   k_cheb      Chebyshev action c <- exp(-i Abar dt) c on the N x Ne
//               coefficient matrix (the exponential integrator of Sec. II C);
//   k_hop       overlap matrix S, its LU factors, determinant ratios for all
//               single excitations, hop probabilities, stochastic hop and
//               momentum rescale (Sec. II B).
#include "iesh_common.cuh"
#include "iesh_kernels.h"
#include "iesh_secular.cuh"
#include "iesh_cheb.cuh"
#include "iesh_hop.cuh"

namespace iesh {

// Trajectories per CTA of k_eigen: fill warps with one thread per root.
int eigen_tpb(int N)
{
    int best = 1;
    double be = 0.0;
    for (int t = 1; t * N <= 256; ++t) {
        const int thr = t * N, thr32 = (thr + 31) & ~31;
        const double eff = (double)thr / thr32 + 1e-4 * t;
        if (eff > be) {
            be = eff;
            best = t;
        }
    }
    return best;
}

// red[0] <- sum of red[0..P) (P a power of two >= the slot width), halving
// the active range each round; every thread of the CTA must call it.
__device__ __forceinline__ void slot_tree_sum(double *red, int r, bool inslot, int P)
{
    __syncthreads();
    for (int w = P >> 1; w > 0; w >>= 1) {
        if (inslot && r < w) red[r] += red[r + w];
        __syncthreads();
    }
}

// mode 0: eigenpairs and force at the stored position (cold start);
// mode 1: full first half of a step (kick, drift, eigenpairs, force, kick).
// tpb trajectories per CTA, one thread per root.
// DF: the secular sums in double-float arithmetic (mixed path).
template <bool DF>
__global__ void __launch_bounds__(256, 3) k_eigen(DevState s, ModelDev md, double dt, int mode, int tpb)
{
    extern __shared__ double sh[];
    const int N = s.N, M = s.M, Ne = s.Ne;
    const int slot = threadIdx.x / N;
    const int r = threadIdx.x - slot * N;
    const int64_t t = slot < tpb ? traj_of(s, (int64_t)blockIdx.x * tpb + slot) : -1;
    const bool act = t >= 0 && !(s.status[t] & ST_DONE);
    const int P = eigen_pow2(N);                         // reduction width
    double *eps_s = sh;                                  // [M], shared by the slots
    const int per = M + 2 * N + P + (DF ? M : 0);
    double *z2_s = eps_s + M + (slot < tpb ? slot : 0) * per;  // [M]
    double *lam_s = z2_s + M;                            // [N]
    double *q0_s = lam_s + N;                            // [N]
    double *red_s = q0_s + N;                            // [P] slot reductions
    float2 *z2df_s = reinterpret_cast<float2 *>(red_s + P);  // [M] z_k^2 as double-float (DF)
    const bool inslot = slot < tpb;
    for (int k = threadIdx.x; k < M; k += blockDim.x) eps_s[k] = s.eps[k];
    double x = 0.0, p = 0.0, guess = 0.0;
    ModelVals mv;
    if (act) {
        x = s.x[t];
        p = s.p[t];
        if (mode == 1) {
            p += 0.5 * dt * s.F[t];
            x += dt * p / md.mass;
        }
        const double l = s.lam[t * N + r];
        guess = l;
        if (mode == 1) {
            // warm start from the linear extrapolation of the last two roots
            // (lam_prev = lam after a cold start, so the first step uses lam)
            guess = 2.0 * l - s.lam_prev[t * N + r];
            s.lam_prev[t * N + r] = l;
            s.q0_prev[t * N + r] = s.q0[t * N + r];
            s.rt_prev[t * N + r] = s.rt[t * N + r];
            s.ro_prev[t * N + r] = s.ro[t * N + r];
            if (r < 4) s.geo_prev[t * 4 + r] = s.geo[t * 4 + r];
            if (r == 0) s.fx_prev[t] = s.fx[t];
        }
        lam_s[r] = l;
        mv = model_eval(md, x);
        for (int k = r; k < M; k += N) {
            const double z = s.z0[k] * mv.f;
            z2_s[k] = z * z;
            if (DF) {
                const dfl zd = dfl_from(z * z);
                z2df_s[k] = make_float2(zd.hi, zd.lo);
            }
        }
    }
    __syncthreads();
    // Z2 = sum_k z_k^2 by a fixed-order tree over the slot's threads
    if (inslot) {
        red_s[r] = (act && r < M) ? z2_s[r] : 0.0;
        if (r < P - N) red_s[N + r] = 0.0;
    }
    slot_tree_sum(red_s, r, inslot, P);
    uint32_t st = 0;
    if (act) {
        const double Z2 = red_s[0];
        double l, q, rt_r = 0.0;
        int ro_r = 0;
        if (Z2 > 0.0) {
            // an extrapolation outside the root's pole gap falls back to lam
            const double glo = r > 0 ? eps_s[r - 1] : -INFINITY, ghi = r < M ? eps_s[r] : INFINITY;
            if (!(guess > glo && guess < ghi)) guess = lam_s[r];
            const Poles<double> pp = {M, eps_s, z2_s, s.poled, s.poledf, z2df_s};
            if (DF)
                secular_root<double, EV_DFLOAT>(r, pp, mv.h, Z2, mode == 1, guess, l, q, st, &ro_r, &rt_r);
            else
                secular_root<double, EV_TABLE>(r, pp, mv.h, Z2, mode == 1, guess, l, q, st, &ro_r, &rt_r);
        } else {
            // no coupling: the eigenvalues are h and the bath energies
            int pos = 0;
            for (int k = 0; k < M; ++k) pos += (eps_s[k] < mv.h);
            l = (r < pos) ? eps_s[r] : (r == pos ? mv.h : eps_s[r - 1]);
            q = (r == pos) ? 1.0 : 0.0;
            ro_r = (r < pos) ? r : (r == pos ? (r < M ? r : M - 1) : r - 1);
            rt_r = l - eps_s[ro_r];
        }
        s.lam[t * N + r] = l;
        s.q0[t * N + r] = q;
        s.rt[t * N + r] = rt_r;
        s.ro[t * N + r] = ro_r;
        if (mode == 0) {
            s.lam_prev[t * N + r] = l;
            s.rt_prev[t * N + r] = rt_r;
            s.ro_prev[t * N + r] = ro_r;
        }
        lam_s[r] = l;
        q0_s[r] = q;
        if (st) atomicOr(&s.status[t], st);
    }
    __syncthreads();
    // occupied-surface term of the force, sum over the occupied orbitals in
    // list order by a fixed-order tree (slot thread a takes electron a)
    const double kappa = (act && mv.f != 0.0) ? mv.df / mv.f : 0.0;
    if (inslot) {
        double c = 0.0;
        if (act && r < Ne) {
            const int i = s.occ[t * Ne + r];
            const double q = q0_s[i];
            c = q * q * (mv.dh + 2.0 * kappa * (lam_s[i] - mv.h));
        }
        red_s[r] = c;
        if (r < P - N) red_s[N + r] = 0.0;
    }
    slot_tree_sum(red_s, r, inslot, P);
    if (act && r == 0) {
        const double dl = red_s[0];
        const double F = -mv.dU0 - dl;
        if (mode == 1) p += 0.5 * dt * F;
        s.x[t] = x;
        s.p[t] = p;
        s.F[t] = F;
        s.dU0[t] = mv.dU0;
        s.geo[t * 4 + 0] = mv.h;
        s.geo[t * 4 + 1] = mv.dh;
        s.geo[t * 4 + 2] = kappa;
        s.geo[t * 4 + 3] = mv.U0;
        s.fx[t] = mv.f;
        if (mode == 0) {
            s.vprev[t] = p / md.mass;
            s.fx_prev[t] = mv.f;
        }
        if (!isfinite(x) || !isfinite(p) || !isfinite(F)) atomicOr(&s.status[t], ST_NAN);
    }
}

// Force on the occupied surface from stored eigenpairs (after occupations change).
__global__ void k_force(DevState s)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int N = s.N, Ne = s.Ne;
    const double h = s.geo[t * 4 + 0], dh = s.geo[t * 4 + 1], kap = s.geo[t * 4 + 2];
    double F = -s.dU0[t];
    for (int a = 0; a < Ne; ++a) {
        const int i = s.occ[t * Ne + a];
        const double q = s.q0[t * N + i];
        F -= q * q * (dh + 2.0 * kap * (s.lam[t * N + i] - h));
    }
    s.F[t] = F;
}

// ============================================================ couplings
// Deflation of an isolated top level (FP64 propagator).  When the top row's
// Gershgorin disc of H = dt Abar = L - i W lies above every other row's disc
// (the other rows' radii taken without the top column), exactly one
// eigenvalue mu lies in it, and by interlacing every other eigenvalue lies
// in [lo, hb]: lo the full Gershgorin minimum, hb = max_{k != top} (L_k +
// R_k - |W_top,k|).  The Chebyshev series then only needs to cover [lo, hb]
// if the component along mu's eigenvector u is propagated exactly, as e^{-i
// mu} (u^H c) u; the bulk half-width is typically a fraction of the full one
// when the adsorbate level sits far from the band (K 14 -> 9 at 1e-15 for
// the double well).  The propagators start the series from c - (u^H c) u,
// which has no u component in exact arithmetic, so no later order needs a
// projection; the u components that rounding leaves in later orders are
// carried by the series, whose value at mu is bounded by cheb_amplification
// (4 to 8 on the double well at dt = 1): with that bound above kDeflAmp64 (FP64) or
// kDeflAmp32 (FP32) the full interval is used.  u comes from a diagonally preconditioned fixed-point
// iteration (the Jacobi correction of Davidson's method): u_top = 1, mu the
// Rayleigh quotient, r = H u - mu u, u_k -= r_k / (L_k - mu) for k != top.
// At the eigenvector it is a fixed point, and it contracts by max_k R'_k /
// (mu - L_k) < 1, R'_k row k's radius without the top column, which the
// disc test bounds below 1 (on the double well the band rows barely couple
// and three iterations reach the tolerance, against about ten for the
// shifted power iteration, whose factor is the bulk half-width over mu minus
// the bulk centre).  It stops at a residual |H u - mu u| <= 1e-14 |mu -
// sigma| |u|, sigma the centre of [lo, hb]; without convergence within
// kDeflIter iterations, or when the deflated series is not at least
// kDeflGain terms shorter, the full interval is used.
constexpr int kDeflIter = 48;
constexpr int kDeflGain = 2;
constexpr double kDeflAmp64 = 1e3, kDeflAmp32 = 16.0;

// Thread 0 has set up the series over the bulk interval; it keeps the
// deflation if the series amplifies the u direction by at most amp, else it
// sets the full interval up.  Returns the block-uniform decision.
__device__ inline bool defl_keep(const DevState &s, int64_t t, bool deflate, double mu, double lo, double hi,
                                 double tol, double amp, double *df, int *flag)
{
    if (threadIdx.x == 0) {
        bool k = deflate && cheb_amplification(s.cheb + t * kChebStride, mu) <= amp;
        if (deflate && !k) cheb_setup(s, t, lo, hi, tol);
        *flag = k;
        if (df) {
            df[0] = k ? 1.0 : 0.0;
            df[1] = mu;
            if (k) sincos(mu, &df[3], &df[2]);  // once per trajectory
        }
    }
    __syncthreads();
    return *flag != 0;
}

__global__ void __launch_bounds__(256) k_build_w(DevState s, double dt, double mass, double tol)
{
    extern __shared__ double sh[];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N;
    double *l0 = sh, *q00 = l0 + N, *l1 = q00 + N, *q01 = l1 + N, *red = q01 + N;
    double *Lk_s = red + 32, *hb_s = Lk_s + N, *ur = hb_s + N, *ui = ur + N;  // deflation
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        l0[i] = s.lam_prev[t * N + i];
        q00[i] = s.q0_prev[t * N + i];
        l1[i] = s.lam[t * N + i];
        q01[i] = s.q0[t * N + i];
    }
    const double h0 = s.geo_prev[t * 4], dh0 = s.geo_prev[t * 4 + 1], k0 = s.geo_prev[t * 4 + 2];
    const double h1 = s.geo[t * 4], dh1 = s.geo[t * 4 + 1], k1 = s.geo[t * 4 + 2];
    const double a0 = 0.5 * dt * s.vprev[t], a1 = 0.5 * dt * (s.p[t] / mass);
    __syncthreads();
    double *W = s.scratch + t * s.scratch_stride;
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double lk0 = l0[k], qk0 = q00[k], lk1 = l1[k], qk1 = q01[k];
        double Rk = 0.0;
        for (int j = 0; j < N; ++j) {
            double w = 0.0;
            if (j != k)
                w = a0 * nac(l0[j], q00[j], lk0, qk0, h0, dh0, k0) +
                    a1 * nac(l1[j], q01[j], lk1, qk1, h1, dh1, k1);
            W[(int64_t)j * N + k] = w;
            Rk += fabs(w);
        }
        const double Lk = 0.5 * dt * (lk0 + lk1);
        lo = fmin(lo, Lk - Rk);
        hi = fmax(hi, Lk + Rk);
        Lk_s[k] = Lk;
        // upper end of row k's disc without the top column; for the top row
        // the lower end of its disc
        hb_s[k] = k == N - 1 ? Lk - Rk : Lk + Rk - fabs(W[(int64_t)(N - 1) * N + k]);
    }
    lo = block_min(lo, red);
    hi = block_max(hi, red);
    double *df = s.defl ? s.defl + t * defl_stride(N, s.Ne) : nullptr;
    bool deflate = false;
    double hb = hi, mu = 0.0;
    if (df && N >= 3 && N <= (int)blockDim.x) {
        const int top = N - 1;  // eigenvalues ascending at both ends: L is ascending
        double b = -__longlong_as_double(0x7ff0000000000000ll);
        for (int k = threadIdx.x; k < top; k += blockDim.x) b = fmax(b, hb_s[k]);
        b = block_max(b, red);
        // one thread takes the decision (the term counts are FP64 loops)
        __shared__ int go;
        if (threadIdx.x == 0)
            go = hb_s[top] > b && cheb_terms(0.5 * (b - lo), tol) + kDeflGain <= cheb_terms(0.5 * (hi - lo), tol);
        __syncthreads();
        if (go) {
            const double sigma = 0.5 * (lo + b);
            const int j = threadIdx.x;
            const bool rj = j < N;
            const double Lj = rj ? Lk_s[j] : 0.0;
            if (rj) {
                ur[j] = j == top ? 1.0 : 0.0;
                ui[j] = 0.0;
            }
            __syncthreads();
            for (int it = 0; it < kDeflIter; ++it) {
                double hr = 0.0, hv = 0.0;
                if (rj) {
                    // (W u)_j = -sum_k W[k N + j] u_k (W antisymmetric; column reads
                    // coalesce); the start u = e_top needs only row top (the other
                    // terms are exact zeros)
                    double wr = 0.0, wi = 0.0;
                    if (it == 0)
                        wr = -W[(int64_t)top * N + j];
                    else
                        for (int k = 0; k < N; ++k) {
                            const double w = W[(int64_t)k * N + j];
                            wr = fma(-w, ur[k], wr);
                            wi = fma(-w, ui[k], wi);
                        }
                    // H u = L u - i W u
                    hr = fma(Lj, ur[j], wi);
                    hv = fma(Lj, ui[j], -wr);
                }
                const double num = block_sum(rj ? fma(ur[j], hr, ui[j] * hv) : 0.0, red);  // u^H H u
                const double den = block_sum(rj ? fma(ur[j], ur[j], ui[j] * ui[j]) : 0.0, red);
                const double m = num / den;
                const double er = rj ? fma(-m, ur[j], hr) : 0.0, ei = rj ? fma(-m, ui[j], hv) : 0.0;
                const double res = block_sum(fma(er, er, ei * ei), red);
                const double gap = m - sigma;
                if (res <= 1e-28 * gap * gap * den) {  // uniform: every thread holds the same sums
                    deflate = gap > 0.0;
                    mu = m;
                    if (rj) {
                        const double inv = 1.0 / sqrt(den);
                        ur[j] *= inv;
                        ui[j] *= inv;
                    }
                    break;
                }
                if (rj && j != top) {
                    const double d = 1.0 / (Lj - m);
                    ur[j] = fma(-er, d, ur[j]);
                    ui[j] = fma(-ei, d, ui[j]);
                }
                __syncthreads();
            }
            if (deflate) hb = b;
        }
    }
    if (threadIdx.x == 0) cheb_setup(s, t, lo, hb, tol);
    __shared__ int keep;
    if (!defl_keep(s, t, deflate, mu, lo, hi, tol, kDeflAmp64, df, &keep)) return;
    const int Ne = s.Ne;
    double *q = df + kDeflHead;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        q[j] = ur[j];
        q[N + j] = ui[j];
    }
    // a_e = u^H c_e, one warp per electron
    const double2 *C = reinterpret_cast<const double2 *>(s.C) + t * (int64_t)Ne * N;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int e = threadIdx.x >> 5; e < Ne; e += nw) {
        double ar = 0.0, ai = 0.0;
        for (int j = lane; j < N; j += 32) {
            const double2 c = C[(int64_t)e * N + j];
            ar = fma(ur[j], c.x, fma(ui[j], c.y, ar));
            ai = fma(ur[j], c.y, fma(-ui[j], c.x, ai));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) {
            q[2 * N + e] = ar;
            q[2 * N + Ne + e] = ai;
        }
    }
}

// Mixed precision: W in FP32.  Each eigenvalue is written relative to its
// nearer bath pole o (lam = eps_o + tau); the difference of two eigenvalues
// is then the FP32 pole difference (a table rounded once from FP64) plus the
// difference of the small offsets, so nearly degenerate pairs keep FP32
// relative accuracy.  The numerators are formed in FP32.
// DFL (the mixed propagator deflates): when the top level is isolated (the
// test of k_build_w) its eigenvector u of the FP32 generator comes from the
// preconditioned iteration of k_build_w on H - sigma, in FP32 but for the
// top row (u_top = 1), whose residual is formed in FP64: in FP32 its
// rounding, about one ulp of mu, would be the floor of the whole residual.
// It stops at |H u - mu u| <= kDeflRes32 |mu - sigma| |u| (one or two
// corrections on the double well, whose top level couples weakly), so the
// eigenvector's error adds no more than about 1e-8 |u^H c| per step.  u, mu
// and a = u^H c (FP32 products and sums) go to s.defl as for FP64.
constexpr float kDeflRes32 = 1e-9f;

template <bool DFL>
__global__ void __launch_bounds__(256, 5) k_build_w_f32(DevState s, double dt, double mass, double tol)
{
    constexpr int dfl = DFL;  // a template parameter: the plain kernel keeps its registers
    extern __shared__ double sh[];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, M = s.M;
    double *red = sh;                                  // [32]
    double *Lsum = red + 32;                           // [N] dt (lam0 + lam1) / 2
    float *qf = reinterpret_cast<float *>(Lsum + N);   // [2][N]
    float *lmh = qf + 2 * N;                           // [2][N] lam - h
    float *tau = lmh + 2 * N;                          // [2][N] lam - eps_o
    int *org = reinterpret_cast<int *>(tau + 2 * N);   // [2][N] o
    double *hb_s = reinterpret_cast<double *>(org + 2 * N);  // [N] deflation: disc ends
    float *ur = reinterpret_cast<float *>(hb_s + N), *ui = ur + N;  // [N] each
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        double lsum = 0.0;
        for (int gi = 0; gi < 2; ++gi) {
            const double lam = gi ? s.lam[t * N + r] : s.lam_prev[t * N + r];
            const double q = gi ? s.q0[t * N + r] : s.q0_prev[t * N + r];
            const double h = gi ? s.geo[t * 4] : s.geo_prev[t * 4];
            int o;
            if (r == 0) o = 0;
            else if (r == M) o = M - 1;
            else o = (lam - s.eps[r - 1] <= s.eps[r] - lam) ? r - 1 : r;
            org[gi * N + r] = o;
            tau[gi * N + r] = (float)(lam - s.eps[o]);
            qf[gi * N + r] = (float)q;
            lmh[gi * N + r] = (float)(lam - h);
            lsum += lam;
        }
        Lsum[r] = 0.5 * dt * lsum;
    }
    const float dh0 = (float)s.geo_prev[t * 4 + 1], k0 = (float)s.geo_prev[t * 4 + 2];
    const float dh1 = (float)s.geo[t * 4 + 1], k1 = (float)s.geo[t * 4 + 2];
    const float a0 = (float)(0.5 * dt * s.vprev[t]), a1 = (float)(0.5 * dt * (s.p[t] / mass));
    __syncthreads();
    float *W = reinterpret_cast<float *>(s.scratch + t * s.scratch_stride);  // [N][Np]
    const int Np = (N + 3) & ~3;
    const float *__restrict__ E = s.epsdiff;  // [M][M] eps_a - eps_b
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float qk0 = qf[k], qk1 = qf[N + k], mk0 = lmh[k], mk1 = lmh[N + k];
        const float tk0 = tau[k], tk1 = tau[N + k];
        const float *E0 = E + (int64_t)org[k] * M, *E1 = E + (int64_t)org[N + k] * M;
        float Rk = 0.0f;
        for (int j = 0; j < N; ++j) {
            float w = 0.0f;
            if (j != k) {
                const float den0 = E0[org[j]] + (tk0 - tau[j]);
                const float den1 = E1[org[N + j]] + (tk1 - tau[N + j]);
                // fast division (at most 2 ulp): the gaps are far from the range limits
                const float d0 = __fdividef(qf[j] * qk0 * (dh0 + k0 * (lmh[j] + mk0)), den0);
                const float d1 = __fdividef(qf[N + j] * qk1 * (dh1 + k1 * (lmh[N + j] + mk1)), den1);
                w = a0 * d0 + a1 * d1;
            }
            W[(int64_t)j * Np + k] = w;
            Rk += fabsf(w);
        }
        // margin for the FP32 rounding of the row sum
        const double R = (double)Rk * (1.0 + 1e-5);
        if (k < Np - N)
            for (int j = 0; j < N; ++j) W[(int64_t)j * Np + N + k] = 0.0f;  // row padding
        lo = fmin(lo, Lsum[k] - R);
        hi = fmax(hi, Lsum[k] + R);
        if (dfl) hb_s[k] = k == N - 1 ? Lsum[k] - R : Lsum[k] + R - fabs((double)W[(int64_t)(N - 1) * Np + k]);
    }
    lo = block_min(lo, red);
    hi = block_max(hi, red);
    double *df = (dfl && s.defl) ? s.defl + t * defl_stride(N, s.Ne) : nullptr;
    bool deflate = false;
    double hb = hi, mu = 0.0;
    if (df && N >= 3 && N <= (int)blockDim.x) {
        const int top = N - 1;
        double b = -__longlong_as_double(0x7ff0000000000000ll);
        for (int k = threadIdx.x; k < top; k += blockDim.x) b = fmax(b, hb_s[k]);
        b = block_max(b, red);  // also orders the W stores before the reads below
        __shared__ int go;  // one thread takes the decision (the term counts are FP64 loops)
        if (threadIdx.x == 0)
            go = hb_s[top] > b && cheb_terms(0.5 * (b - lo), tol) + kDeflGain <= cheb_terms(0.5 * (hi - lo), tol);
        __syncthreads();
        if (go) {
            // the preconditioned iteration with u_top = 1 and mu taken from the
            // top row, mu = ((H - sigma) u)_top (the top thread, in FP64), so
            // that r_top vanishes and the other rows' residuals are formed
            // from small quantities in FP32
            const double sigma = 0.5 * (lo + b);
            const int j = threadIdx.x;
            const bool rj = j < N, tj = j == top;
            const float Lj = rj ? (float)(Lsum[j] - sigma) : 0.f;
            __shared__ double s_m;
            if (rj) {
                ur[j] = tj ? 1.f : 0.f;
                ui[j] = 0.f;
            }
            __syncthreads();
            for (int it = 0; it < kDeflIter; ++it) {
                float wr = 0.f, wi = 0.f;  // (W u)_j = -sum_k W[k Np + j] u_k
                if (rj && it == 0)
                    wr = -W[(int64_t)top * Np + j];  // u = e_top: the other terms are exact zeros
                else if (rj)
                    for (int k = 0; k < N; ++k) {
                        const float w = W[(int64_t)k * Np + j];
                        wr = fmaf(-w, ur[k], wr);
                        wi = fmaf(-w, ui[k], wi);
                    }
                // (H - sigma) u = (L - sigma) u - i W u; the top row gives mu
                if (tj) s_m = fma(Lsum[j] - sigma, (double)ur[j], (double)wi);
                __syncthreads();
                const double m = s_m;
                float er = 0.f, ei = 0.f;
                if (rj && !tj) {
                    er = fmaf(Lj - (float)m, ur[j], wi);
                    ei = fmaf(Lj - (float)m, ui[j], -wr);
                } else if (tj) {
                    ei = -wr;  // the imaginary part of the top row's residual
                }
                const double res = block_sum((double)fmaf(er, er, ei * ei), red);
                const double den = 1.0;  // |u|^2 >= u_top^2 = 1: the test below is conservative
                if (res <= (double)kDeflRes32 * kDeflRes32 * m * m * den) {  // uniform
                    deflate = m > 0.0;
                    mu = sigma + m;
                    const double nrm = block_sum(rj ? (double)fmaf(ur[j], ur[j], ui[j] * ui[j]) : 0.0, red);
                    if (rj) {
                        const float inv = (float)(1.0 / sqrt(nrm));
                        ur[j] *= inv;
                        ui[j] *= inv;
                    }
                    break;
                }
                if (rj && !tj) {
                    const float d = 1.f / (Lj - (float)m);
                    ur[j] = fmaf(-er, d, ur[j]);
                    ui[j] = fmaf(-ei, d, ui[j]);
                }
                __syncthreads();
            }
            if (deflate) hb = b;
        }
    }
    if (threadIdx.x == 0) cheb_setup(s, t, lo, hb, tol);
    if (!dfl) return;
    __shared__ int keep;
    if (!defl_keep(s, t, deflate, mu, lo, hi, tol, kDeflAmp32, df, &keep)) return;
    const int Ne = s.Ne;
    float *q = reinterpret_cast<float *>(df + kDeflHead);  // packed floats
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        q[j] = ur[j];
        q[N + j] = ui[j];
    }
    // a_e = u^H c_e in FP32, one warp per electron
    const float2 *C = reinterpret_cast<const float2 *>(s.C) + t * (int64_t)Ne * N;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int e = threadIdx.x >> 5; e < Ne; e += nw) {
        float ar = 0.f, ai = 0.f;
        for (int j = lane; j < N; j += 32) {
            const float2 c = C[(int64_t)e * N + j];
            ar = fmaf(ur[j], c.x, fmaf(ui[j], c.y, ar));
            ai = fmaf(ur[j], c.y, fmaf(-ui[j], c.x, ai));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) {
            q[2 * N + e] = ar;
            q[2 * N + Ne + e] = ai;
        }
    }
}

// ============================================================ propagator
// Chebyshev expansion of the exponential integrator: with the spectrum of
// H = Abar dt inside [c - rho, c + rho] (Gershgorin),
//   exp(-i H) v = e^{-ic} sum_k (2 - delta_k0) (-i)^k J_k(rho) T_k(X) v,
//   X = (H - c) / rho,  T_{k+1} = 2 X T_k - T_{k-1},
// and H v = L v - i W v with L = diag(dt (lam0 + lam1) / 2) and W the real
// antisymmetric step-averaged coupling generator.  One CTA owns G x EPT
// electrons (columns) of one trajectory; thread (g, j) owns orbital row j of
// the EPT electrons of column group g, so every warp is (nearly) full on the
// FP64 pipe, which is the bound of this kernel.
// Deflation (s.defl, flag set by k_build_w): the interval is the bulk one,
// the series starts from T_0 = c - a u (a = u^H c), and the isolated level's
// share e^{-i mu} a u is added at the end; the loop is the plain one.
template <class RT>
struct Cplx;

template <>
struct Cplx<double> {
    typedef double2 T;
};
template <>
struct Cplx<float> {
    typedef float2 T;
};

template <int EPT, class RT>
__global__ void __launch_bounds__(1024) k_cheb(DevState s, double dt, int G, int64_t t_base)
{
    typedef typename Cplx<RT>::T CT;
    extern __shared__ __align__(16) unsigned char cheb_smem[];
    RT *tk = reinterpret_cast<RT *>(cheb_smem);  // [N][2 G EPT]
    // the electron blocks of one trajectory are adjacent in launch order, so
    // they run together and share W through L2
    const int64_t t = traj_of(s, t_base + blockIdx.y);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Ne = s.Ne;
    const int NB = G * EPT, W2 = 2 * NB;
    const int g = threadIdx.x / N;
    const int j = threadIdx.x - g * N;
    const bool act = g < G;
    const int e0 = blockIdx.x * NB + g * EPT;  // first electron of this thread
    const double *cb = s.cheb + t * kChebStride;
    const double c = cb[0], rho = cb[1];
    const int K = (int)cb[2];
    const double *J = cb + 3;
    const RT inv_rho = (RT)(rho > 0.0 ? 1.0 / rho : 0.0);
    const RT *__restrict__ W = reinterpret_cast<const RT *>(s.scratch + t * s.scratch_stride);
    CT *C = reinterpret_cast<CT *>(s.C) + (int64_t)t * Ne * N;
    const RT Lc = (RT)(act ? 0.5 * dt * (s.lam_prev[t * N + j] + s.lam[t * N + j]) - c : 0.0);
    RT *myrow = tk + j * W2 + 2 * EPT * g;
    // deflation: read again after the loop (nothing of it stays in registers)
    const bool defl0 = s.defl && s.defl[t * defl_stride(N, Ne)] != 0.0;

    RT tp[2 * EPT], acc[2 * EPT];
    const RT J0 = (RT)J[0];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        CT v;
        v.x = 0;
        v.y = 0;
        if (act && e0 + e < Ne) {
            v = C[(int64_t)(e0 + e) * N + j];
            if (defl0) v = defl_start<RT>(s.defl + t * defl_stride(N, Ne), N, Ne, j, e0 + e, v);
        }
        tp[2 * e] = v.x;
        tp[2 * e + 1] = v.y;
        acc[2 * e] = J0 * v.x;
        acc[2 * e + 1] = J0 * v.y;  // single products: no contraction possible
        if (act) {
            myrow[2 * e] = v.x;
            myrow[2 * e + 1] = v.y;
        }
    }
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        RT y[2 * EPT];
#pragma unroll
        for (int q = 0; q < 2 * EPT; ++q) y[q] = 0;
        if (act) {
            const RT *col = tk + 2 * EPT * g;
#pragma unroll 4
            for (int i = 0; i < N; ++i) {
                const RT w = W[(int64_t)i * N + j];  // W_ij = -W_ji
                const RT *row = col + i * W2;
#pragma unroll
                for (int q = 0; q < 2 * EPT; ++q) y[q] = fma(w, row[q], y[q]);
            }
        }
        RT own[2 * EPT];
        if (act) {
#pragma unroll
            for (int q = 0; q < 2 * EPT; ++q) own[q] = myrow[q];
        }
        __syncthreads();
        if (act) {
            const RT cj = (RT)(2.0 * J[k + 1]);
            const int ph = (k + 1) & 3;  // (-i)^(k+1)
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                // (X t)_j = ((L_j - c) t_j - i (W t)_j) / rho and (W t)_j = -y.
                // Explicit FMAs fix the rounding independently of the CTA shape.
                const RT xr = fma(Lc, own[2 * e], -y[2 * e + 1]) * inv_rho;
                const RT xi = fma(Lc, own[2 * e + 1], y[2 * e]) * inv_rho;
                RT nr, ni;
                if (k == 0) {
                    nr = xr;
                    ni = xi;
                } else {
                    nr = fma((RT)2, xr, -tp[2 * e]);
                    ni = fma((RT)2, xi, -tp[2 * e + 1]);
                }
                tp[2 * e] = own[2 * e];
                tp[2 * e + 1] = own[2 * e + 1];
                if (ph == 0) {
                    acc[2 * e] = fma(cj, nr, acc[2 * e]);
                    acc[2 * e + 1] = fma(cj, ni, acc[2 * e + 1]);
                } else if (ph == 1) {
                    acc[2 * e] = fma(cj, ni, acc[2 * e]);
                    acc[2 * e + 1] = fma(-cj, nr, acc[2 * e + 1]);
                } else if (ph == 2) {
                    acc[2 * e] = fma(-cj, nr, acc[2 * e]);
                    acc[2 * e + 1] = fma(-cj, ni, acc[2 * e + 1]);
                } else {
                    acc[2 * e] = fma(-cj, ni, acc[2 * e]);
                    acc[2 * e + 1] = fma(cj, nr, acc[2 * e + 1]);
                }
                myrow[2 * e] = nr;
                myrow[2 * e + 1] = ni;
            }
        }
        __syncthreads();
    }
    if (act) {
        const double *df = s.defl ? s.defl + t * defl_stride(N, Ne) : nullptr;
        const bool defl = df && df[0] != 0.0;
        double scd, ccd, smd = 0.0, cmd = 1.0;
        sincos(c, &scd, &ccd);
        if (defl) {
            cmd = df[2];
            smd = df[3];
        }
        const RT sc = (RT)scd, cc = (RT)ccd;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            if (e0 + e < Ne) {
                const RT ar = acc[2 * e], ai = acc[2 * e + 1];
                CT out;
                out.x = fma(cc, ar, sc * ai);
                out.y = fma(cc, ai, -(sc * ar));
                if (defl) out = defl_end<RT>(df, N, Ne, j, e0 + e, (RT)cmd, (RT)smd, out);
                C[(int64_t)(e0 + e) * N + j] = out;
            }
        }
    }
}

// FP32 propagator, register-tiled: thread (row slot rq, column group cg)
// owns QPT row quads, rows 4q..4q+3 for q = rq + h nqh (h < QPT, nqh =
// ceil(nq / QPT) for nq row quads), and CE electrons (2 CE reals) of the
// CTA's block of G*CE electrons.  Per orbital i it loads W[i][4q..4q+3] as
// one float4 per quad (W_ji = -W_ij; W rows padded to a multiple of 4) and
// 2CE reals of t_k[i] as float4 broadcasts from shared memory, for
// 8 CE QPT FFMAs.  The quads of a thread are nqh apart so that, quad by
// quad, a warp's float4 loads of W are consecutive (conflict-free).  QPT = 2
// doubles the FFMAs per shared load and per loop instruction; its register
// tile (64 accumulators and 64 Chebyshev sums per thread) allows one CTA
// per SM.  W reaches shared memory by cp.async in chunks of kCheb32WRows
// rows, in a ring of kCheb32WRing chunks filled kCheb32WRing - 1 chunks
// ahead (one barrier per chunk), so the loop reads it at shared-memory
// latency instead of L2's.  t_k and t_(k-1) live in two shared buffers:
// t_(k+1) overwrites t_(k-1) in place (each thread rewrites only its own
// entries), so one barrier per order suffices and neither is held in
// registers.  Row j of a buffer starts at j W2 + 4 floor(j/4): the 4-float
// gap after every row quad puts the row quads of consecutive threads 4
// banks apart, so the per-thread row accesses of the recurrence are
// conflict-free float4 accesses.
__device__ __forceinline__ int cheb32_row(int j, int W2) { return j * W2 + ((j >> 2) << 2); }

template <int CE, int QPT>
__global__ void __launch_bounds__(256, QPT == 1 ? 2 : 1)
    k_cheb_f32t(DevState s, double dt, int G, int64_t t_base, int dfl)
{
    constexpr int RQ = 4 * QPT, NR = 2 * CE, NV = NR / 4;  // NV float4 per row
    extern __shared__ __align__(16) unsigned char cheb32_smem[];
    const int64_t t = traj_of(s, t_base + blockIdx.y);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Ne = s.Ne, Np = (N + 3) & ~3;
    // deflation (set up by k_build_w_f32<true>): start from c - a u, add
    // e^{-i mu} a u at the end (the flag is read again there)
    const bool defl0 = dfl && s.defl[t * defl_stride(N, Ne)] != 0.0;
    const int nq = (N + 3) / 4, nqh = (nq + QPT - 1) / QPT;
    const int W2 = NR * G;
    float *buf0 = reinterpret_cast<float *>(cheb32_smem);
    float *buf1 = buf0 + cheb32_row(Np, W2);
    const int cg = threadIdx.x / nqh, rq = threadIdx.x - cg * nqh;
    const bool act = cg < G;
    // quad h of this thread: first row j0(h); its first buffer entry mine(h)
    // (my columns); W offset wo(h), row 0 for a quad past the matrix (read,
    // never used)
    auto j0 = [&](int h) { return 4 * (rq + h * nqh); };
    auto wo = [&](int h) {
        if constexpr (QPT == 1) return 4 * rq;  // rq < nqh = nq
        return rq + h * nqh < nq ? 4 * (rq + h * nqh) : 0;
    };
    auto mine = [&](int h) { return cheb32_row(wo(h), W2) + NR * cg; };
    const int e0 = blockIdx.x * (CE * G) + cg * CE;
    const double *cb = s.cheb + t * kChebStride;
    const double c = cb[0], rho = cb[1];
    const int K = (int)cb[2];
    const double *J = cb + 3;
    // per-trajectory scalars in FP32, formed once (FP64 work costs every warp
    // that issues it): 2 J_k, 1 / rho, sin c, cos c
    __shared__ float s_cj[kChebMax], s_sc[5];
    for (int q = threadIdx.x; q <= K; q += blockDim.x) s_cj[q] = (float)(2.0 * J[q]);
    if (threadIdx.x == 0) {
        double scd, ccd;
        sincos(c, &scd, &ccd);
        s_sc[0] = (float)(rho > 0.0 ? 1.0 / rho : 0.0);
        s_sc[1] = (float)scd;
        s_sc[2] = (float)ccd;
        if (defl0) {
            s_sc[3] = (float)s.defl[t * defl_stride(N, Ne) + 3];  // e^{-i mu}
            s_sc[4] = (float)s.defl[t * defl_stride(N, Ne) + 2];
        }
    }
    const float *__restrict__ W = reinterpret_cast<const float *>(s.scratch + t * s.scratch_stride);
    float2 *C = reinterpret_cast<float2 *>(s.C) + (int64_t)t * Ne * N;
    float Lc[RQ], acc[RQ][NR];
    const float J0 = (float)J[0];
#pragma unroll
    for (int h = 0; h < QPT; ++h)
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
            const int r = 4 * h + r4, j = j0(h) + r4;
            const bool ok = act && j < N;
            Lc[r] = ok ? (float)(0.5 * dt * (s.lam_prev[t * N + j] + s.lam[t * N + j]) - c) : 0.f;
            float v[NR];
#pragma unroll
            for (int e = 0; e < CE; ++e) {
                float2 ce = make_float2(0.f, 0.f);
                if (ok && e0 + e < Ne) {
                    ce = C[(int64_t)(e0 + e) * N + j];
                    if (defl0) ce = defl_start<float>(s.defl + t * defl_stride(N, Ne), N, Ne, j, e0 + e, ce);
                }
                v[2 * e] = ce.x;
                v[2 * e + 1] = ce.y;
                acc[r][2 * e] = J0 * ce.x;
                acc[r][2 * e + 1] = J0 * ce.y;  // single products: no contraction possible
            }
            if (ok) {
                float4 *d4 = reinterpret_cast<float4 *>(buf0 + mine(h) + r4 * W2);
#pragma unroll
                for (int g = 0; g < NV; ++g) d4[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
            }
        }
    // W ring: chunk g (rows kCheb32WRows (g % nwc) ..) in slot g % kCheb32WRing,
    // one commit group each
    float *wring = buf1 + cheb32_row(Np, W2);
    const int nwc = (N + kCheb32WRows - 1) / kCheb32WRows, gtot = K * nwc;
    auto fetch = [&](int g) {
        if (g < gtot) {
            const int c = g % nwc;
            const int nv = min(kCheb32WRows, N - kCheb32WRows * c) * Np / 4;  // float4 of the chunk
            float *dst = wring + (g % kCheb32WRing) * kCheb32WRows * Np;
            const float *src = W + (int64_t)kCheb32WRows * c * Np;
            for (int v = threadIdx.x; v < nv; v += blockDim.x) cp_async16(dst + 4 * v, src + 4 * v);
        }
        cp_async_commit();
    };
    for (int g = 0; g < kCheb32WRing - 1; ++g) fetch(g);
    __syncthreads();
    const float inv_rho = s_sc[0];
    for (int k = 0; k < K; ++k) {
        const float *cur = (k & 1) ? buf1 : buf0;  // t_k
        float *nxt = (k & 1) ? buf0 : buf1;        // t_(k-1), becomes t_(k+1)
        float y[RQ][NR];
#pragma unroll
        for (int r = 0; r < RQ; ++r)
#pragma unroll
            for (int q = 0; q < NR; ++q) y[r][q] = 0.f;
        const float *col = cur + NR * cg;
        for (int c = 0; c < nwc; ++c) {
            const int g = k * nwc + c;
            // chunk g has landed for every thread (kCheb32WRing - 2 newer groups
            // may be in flight) and every thread is done with chunk g - 1,
            // whose slot takes chunk g + kCheb32WRing - 1
            cp_async_wait<kCheb32WRing - 2>();
            __syncthreads();
            fetch(g + kCheb32WRing - 1);
            if (act) {
                // row i of the chunk: W at wp + i Np, t_k at tp + i W2 (+ 4 per
                // row quad); walked by quads with the strides in registers
                const float *wp = wring + (g % kCheb32WRing) * kCheb32WRows * Np + wo(0);
                const int dwo = QPT == 2 ? wo(1) - wo(0) : 0;  // the second quad's W, relative
                const int i0 = kCheb32WRows * c, rows = min(kCheb32WRows, N - i0);
                const float *tp = col + cheb32_row(i0, W2);  // i0 is a multiple of 4
                auto row = [&](const float *wr_p, const float *tr_p) {
                    float4 w[QPT];
                    w[0] = *reinterpret_cast<const float4 *>(wr_p);
                    if constexpr (QPT == 2) w[1] = *reinterpret_cast<const float4 *>(wr_p + dwo);
                    const float4 *tr = reinterpret_cast<const float4 *>(tr_p);
                    float tv[NR];
#pragma unroll
                    for (int g4 = 0; g4 < NV; ++g4) {
                        const float4 a4 = tr[g4];
                        tv[4 * g4] = a4.x;
                        tv[4 * g4 + 1] = a4.y;
                        tv[4 * g4 + 2] = a4.z;
                        tv[4 * g4 + 3] = a4.w;
                    }
#pragma unroll
                    for (int h = 0; h < QPT; ++h) {
                        const float wr[4] = {w[h].x, w[h].y, w[h].z, w[h].w};
#pragma unroll
                        for (int r4 = 0; r4 < 4; ++r4)
#pragma unroll
                            for (int q = 0; q < NR; ++q) y[4 * h + r4][q] = fmaf(wr[r4], tv[q], y[4 * h + r4][q]);
                    }
                };
                const int Np2 = 2 * Np, Np3 = 3 * Np, Wd2 = 2 * W2, Wd3 = 3 * W2;
                int u = 0;
                for (; u + 4 <= rows; u += 4) {
                    row(wp, tp);
                    row(wp + Np, tp + W2);
                    row(wp + Np2, tp + Wd2);
                    row(wp + Np3, tp + Wd3);
                    wp += 4 * Np;
                    tp += 4 * W2 + 4;
                }
                for (int r = 0; u + r < rows; ++r) row(wp + r * Np, tp + r * W2);
            }
        }
        if (act) {
            const float cj = s_cj[k + 1];
            const int ph = (k + 1) & 3;  // (-i)^(k+1) = (1, 0), (0, -1), (-1, 0), (0, 1)
            const float ca = ph == 0 ? cj : (ph == 2 ? -cj : 0.f), cb = ph == 1 ? -cj : (ph == 3 ? cj : 0.f);
#pragma unroll
            for (int h = 0; h < QPT; ++h)
#pragma unroll
                for (int r4 = 0; r4 < 4; ++r4) {
                    const int r = 4 * h + r4;
                    if (j0(h) + r4 < N) {
                        const float4 *o4 = reinterpret_cast<const float4 *>(cur + mine(h) + r4 * W2);
                        float4 *d4 = reinterpret_cast<float4 *>(nxt + mine(h) + r4 * W2);
                        float own[NR], prv[NR], nw[NR];
#pragma unroll
                        for (int g4 = 0; g4 < NV; ++g4) {
                            const float4 a4 = o4[g4];
                            own[4 * g4] = a4.x;
                            own[4 * g4 + 1] = a4.y;
                            own[4 * g4 + 2] = a4.z;
                            own[4 * g4 + 3] = a4.w;
                            float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (k > 0) b4 = d4[g4];
                            prv[4 * g4] = b4.x;
                            prv[4 * g4 + 1] = b4.y;
                            prv[4 * g4 + 2] = b4.z;
                            prv[4 * g4 + 3] = b4.w;
                        }
#pragma unroll
                        for (int e = 0; e < CE; ++e) {
                            // (X t)_j = ((L_j - c) t_j - i (W t)_j) / rho and (W t)_j = -y
                            const float xr = fmaf(Lc[r], own[2 * e], -y[r][2 * e + 1]) * inv_rho;
                            const float xi = fmaf(Lc[r], own[2 * e + 1], y[r][2 * e]) * inv_rho;
                            float nr = xr, ni = xi;
                            if (k > 0) {
                                nr = fmaf(2.f, xr, -prv[2 * e]);
                                ni = fmaf(2.f, xi, -prv[2 * e + 1]);
                            }
                            float *a = acc[r] + 2 * e;
                            // acc += cj (-i)^(k+1) n without a branch: (ca, cb) = cj (-i)^(k+1)
                            a[0] = fmaf(ca, nr, fmaf(-cb, ni, a[0]));
                            a[1] = fmaf(ca, ni, fmaf(cb, nr, a[1]));
                            nw[2 * e] = nr;
                            nw[2 * e + 1] = ni;
                        }
#pragma unroll
                        for (int g4 = 0; g4 < NV; ++g4)
                            d4[g4] = make_float4(nw[4 * g4], nw[4 * g4 + 1], nw[4 * g4 + 2], nw[4 * g4 + 3]);
                    }
                }
        }
        __syncthreads();
    }
    cp_async_wait<0>();  // no copy outlives the CTA
    if (act) {
        const float sc = s_sc[1], cc = s_sc[2];
        const double *df = dfl ? s.defl + t * defl_stride(N, Ne) : nullptr;
        const bool defl = df && df[0] != 0.0;
#pragma unroll
        for (int h = 0; h < QPT; ++h)
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
                const int r = 4 * h + r4, j = j0(h) + r4;
#pragma unroll
                for (int e = 0; e < CE; ++e)
                    if (j < N && e0 + e < Ne) {
                        const float ar = acc[r][2 * e], ai = acc[r][2 * e + 1];
                        float2 out = make_float2(fmaf(cc, ar, sc * ai), fmaf(cc, ai, -(sc * ar)));
                        if (defl) out = defl_end<float>(df, N, Ne, j, e0 + e, s_sc[4], s_sc[3], out);
                        C[(int64_t)(e0 + e) * N + j] = out;
                    }
            }
    }
}

// Column groups of k_cheb_f32t: fill the CTA (row slots x groups <= 256)
// and waste few electron slots; with one row quad per thread two CTAs must
// fit in an SM's shared memory, with two quads one.
size_t cheb32_smem_bytes(int N, int G)
{
    const int Np = (N + 3) & ~3;
    // two buffers of padded rows and the ring of W chunks
    return ((size_t)2 * (Np * 8 * G + Np) + (size_t)kCheb32WRing * kCheb32WRows * Np) * sizeof(float);
}
bool cheb32_shape_ok(int N, int G, int qpt)
{
    const int nqh = ((N + 3) / 4 + qpt - 1) / qpt;
    return (qpt == 1 || qpt == 2) && G >= 1 && G * nqh <= 256 &&
           cheb32_smem_bytes(N, G) <= (qpt == 1 ? kCheb32MaxSmem : kCheb32WideMaxSmem);
}
void cheb32_shape(int N, int Ne, int &G, int qpt)
{
    const int nq = ((N + 3) / 4 + qpt - 1) / qpt;
    double best = -1.0;
    G = 1;
    for (int g = 1; g == 1 || cheb32_shape_ok(N, g, qpt); ++g) {
        if (g * nq > 256) break;
        const int nb = 4 * g, thr = g * nq, thr32 = (thr + 31) & ~31;
        const int blocks = (Ne + nb - 1) / nb;
        const double eff = (double)thr / thr32 * (double)Ne / (blocks * nb) + 1e-4 * g;
        if (eff > best) {
            best = eff;
            G = g;
        }
    }
}

// ================================================================= hops
// Sec. II B: the amplitude of the occupied configuration is det S with
// S_aj = C_{s_a, j}; the candidate that puts orbital m in slot a has
// amplitude det S_J = det S * (C_m S^{-1})_a.  With P S = L U, the row
// vector C_m S^{-1} is obtained by one forward substitution with U and one
// backward substitution with L, then the row permutation.  The hop
// probability is g_{a->m} = max(0, -2 dt v Re(R_ma) d_{m, s_a}).
//
// The LU uses partial pivoting without moving rows: perm[k] is the physical
// row chosen as the k-th pivot.  Each warp owns the rows r = warp (mod
// warps); per column it scales its rows, updates them, and records the
// largest candidate of the next column, so one block barrier per column
// suffices.  Complex products are written as explicit FMAs.
// Bytes of the matrix region: S / LU in FP64; in the mixed path the FP32
// factors followed by one pass of FP32 substitution rows (at most 128
// quad-lane groups).
__host__ __device__ inline size_t hop_region_bytes(int N, int Ne, bool f32)
{
    size_t a = (size_t)16 * Ne * Ne;
    if (f32) {
        const int rows = (N - Ne) < 128 ? (N - Ne) : 128;
        a = (size_t)8 * Ne * Ne + (size_t)8 * rows * Ne;
    }
    return (a + 15) & ~(size_t)15;
}

size_t hop_smem_bytes(int N, int Ne, bool f32, bool ext)
{
    return hop_region_bytes(N, Ne, f32) + (size_t)16 * Ne + (size_t)((ext ? 3 : 2) * N + 64) * 8 +
           (size_t)(64 + 64 + 4 * Ne + 2 * N) * 4;
}
size_t hop_smem_bytes(int N, int Ne) { return hop_smem_bytes(N, Ne, false, false); }

// CT: coefficient type, also the type of the factorisation.  double2: the
// FP64 path.  float2: the mixed path -- S (read from the FP32 coefficients)
// is factorised and substituted in FP32; |det S| for the skip bound and the
// hop probabilities from the ratios are formed in FP64.
// MAXT/MINB: launch bounds of the instantiation: 512 x 1 for large S;
// 256 x 3 (FP64) or 256 x 4 (mixed, 64 registers) when that many CTAs fit.
// EXT: two adsorbate orbitals over six coordinates.  The coupling that
// enters g is the velocity-projected v . d_{m, s_a} = T^v_{m s_a} /
// (lam_{s_a} - lam_m) with T^v_jk = sum_a Q_aj Q_ak [grad h_a . v +
// (grad log f_a . v) (lam_j + lam_k - 2 h_a)] (the one-orbital closed form
// per adsorbate orbital, since c_a B_k = (lam_k - h_a) Q_ak on an
// eigenvector); the kernel stops after the selection and writes the chosen
// (a, m) to hop_pair for the six-dimensional rescale.
template <class CT, int MAXT, int MINB, bool EXT = false>
__global__ void __launch_bounds__(MAXT, MINB) k_hop(DevState s, double dt, double mass, uint64_t seed,
                                                    int skip_bound, double *g_out)
{
    constexpr bool kF32 = sizeof(CT) == sizeof(float2);
    extern __shared__ __align__(16) unsigned char hop_smem[];
    const int64_t t = traj_of(s, blockIdx.x);
    if (t < 0 || (s.status[t] & ST_DONE)) return;
    const int N = s.N, Ne = s.Ne, nu = N - Ne;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const size_t abytes = hop_region_bytes(N, Ne, kF32);
    CT *A = reinterpret_cast<CT *>(hop_smem);                     // [Ne][Ne] physical rows
    CT *dinv = reinterpret_cast<CT *>(hop_smem + abytes);         // [Ne] 1/U_kk, logical k
    double *lam_s = reinterpret_cast<double *>(dinv + Ne);         // [N]
    double *q0_s = lam_s + N;                                     // [N]
    double *red = q0_s + N;                                       // [64]
    double *q2_s = red + 64;                                      // [N] (EXT)
    int *cand_v = reinterpret_cast<int *>(q2_s + (EXT ? N : 0));  // [2][32] pivot key per warp
    int *cand_i = reinterpret_cast<int *>(cand_v + 64);           // [2][32] row per warp
    int *occ_s = cand_i + 64;                                     // [Ne]
    int *perm = occ_s + Ne;                                       // [Ne] pivot k -> row
    int *rows = perm + Ne;                                        // [Ne] rows not yet pivots
    int *isocc = rows + Ne;                                       // [N]
    int *unocc = isocc + N;                                       // [N - Ne] ascending
    int *pos_of = unocc + (N - Ne);                               // [Ne] position of a row in rows
    __shared__ int s_flag, s_hop_a, s_hop_m;

    const CT *Ct = reinterpret_cast<const CT *>(s.C) + (int64_t)t * Ne * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        lam_s[i] = s.lam[t * N + i];
        q0_s[i] = s.q0[t * N + i];
        if constexpr (EXT) q2_s[i] = s.q2[t * N + i];
        isocc[i] = 0;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < Ne; a += blockDim.x) {
        occ_s[a] = s.occ[t * Ne + a];
        isocc[occ_s[a]] = 1;
    }
    if (threadIdx.x == 0) {
        s_flag = 0;
        s_hop_a = -1;
        s_hop_m = -1;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < Ne * Ne; idx += blockDim.x) {
        const int a = idx / Ne, e = idx - a * Ne;
        A[idx] = Ct[(int64_t)e * N + occ_s[a]];
    }
    if (threadIdx.x == 0) {
        int u = 0;
        for (int m = 0; m < N; ++m)
            if (!isocc[m]) unocc[u++] = m;
    }
    __syncthreads();
    // pivot candidates of column 0
    if (lane == 0) {
        int bv = -1;
        int bi = Ne;
        for (int r = warp; r < Ne; r += nwarp) {
            const int m2 = pivot_key(A[r * Ne]);
            if (m2 > bv) {
                bv = m2;
                bi = r;
            }
        }
        cand_v[warp] = bv;
        cand_i[warp] = bi;
        if (warp == 0)
            for (int r = 0; r < Ne; ++r) rows[r] = pos_of[r] = r;
    }
    __syncthreads();

    // ---- LU with partial pivoting: rows are not moved; rows[0..nr) lists the
    // rows not yet used as pivots.  Two barriers per column: multipliers,
    // then the trailing update, which also records the next column's
    // per-warp pivot candidates.
    bool singular = false;
    int nr = Ne;
    for (int kc = 0; kc < Ne; ++kc) {
        const int buf = kc & 1;
        // largest per-warp candidate (ties: lowest row), by a butterfly
        int bv = -1;
        int pr = Ne;
        if (lane < nwarp) {
            bv = cand_v[buf * 32 + lane];
            pr = cand_i[buf * 32 + lane];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, pr, o);
            if (ov > bv || (ov == bv && oi < pr)) {
                bv = ov;
                pr = oi;
            }
        }
        if (bv <= 0) {  // zero pivot column
            singular = true;
            break;
        }
        const CT pv = A[pr * Ne + kc];
        // remove pr from the row list: the last entry moves into its position
        // (thread 0 writes the list after the barrier; readers redirect)
        const int ppos = pos_of[pr];
        // multipliers of the remaining rows: only the warps that form them
        // take the FP64 reciprocal (the FP64 pipe charges every issuing warp)
        if (threadIdx.x < nr) {
            const CT pinv = crcp(pv);
            for (int q = threadIdx.x; q < nr; q += blockDim.x) {
                const int r = rows[q];
                if (r != pr) A[r * Ne + kc] = cmul(A[r * Ne + kc], pinv);
            }
            if (threadIdx.x == 0) dinv[kc] = pinv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            perm[kc] = pr;
            const int last = rows[nr - 1];
            rows[ppos] = last;
            pos_of[last] = ppos;
        }
        const int nrow = nr - 1;  // rows to update (the list without pr)
        const int ncol = Ne - kc - 1;
        int cv = -1;
        int ci = Ne;
        const int total = nrow * ncol;
        if (total > 0) {
            // flattened (row, column) walk without a division per element
            const int sq = blockDim.x / ncol, sc = blockDim.x - sq * ncol;
            int qq = threadIdx.x / ncol, cc = threadIdx.x - qq * ncol;
            for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
                const int c = kc + 1 + cc;
                // list position qq of the list without pr: entry nr-1 moved into ppos
                const int r = rows[(qq == ppos) ? nr - 1 : qq];
                const CT nv = cfms(A[r * Ne + c], A[r * Ne + kc], A[pr * Ne + c]);
                A[r * Ne + c] = nv;
                if (cc == 0) {
                    const int m2 = pivot_key(nv);
                    if (m2 > cv || (m2 == cv && r < ci)) {
                        cv = m2;
                        ci = r;
                    }
                }
                cc += sc;
                qq += sq;
                if (cc >= ncol) {
                    cc -= ncol;
                    ++qq;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ov = __shfl_xor_sync(0xffffffffu, cv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
            if (ov > cv || (ov == cv && oi < ci)) {
                cv = ov;
                ci = oi;
            }
        }
        if (lane == 0) {
            cand_v[(buf ^ 1) * 32 + warp] = cv;
            cand_i[(buf ^ 1) * 32 + warp] = ci;
        }
        nr = nrow;
        __syncthreads();
    }
    if (singular && threadIdx.x == 0) atomicOr(&s.status[t], ST_SINGULAR);
    // the six-coordinate coupling carries its velocity: v = 1 there
    const double v = EXT ? 1.0 : s.p[t] / mass;
    const double *gv = EXT ? s.geo2 + t * 8 : s.geo + t * 4;
    const double geo_h = gv[0], geo_dh = gv[1], geo_k = gv[2];
    // NAC d_{m, sa} (times v for EXT) of a candidate (target m, source sa)
    auto hop_nac = [&](int m, int sa) -> double {
        if constexpr (EXT) {
            const double lm = lam_s[m], ls = lam_s[sa], lsum = lm + ls;
            const double T = q0_s[m] * q0_s[sa] * (gv[2] + gv[4] * (lsum - 2.0 * gv[0])) +
                             q2_s[m] * q2_s[sa] * (gv[3] + gv[5] * (lsum - 2.0 * gv[1]));
            return T * pole_recip<double>(ls - lm);
        } else {
            return nac(lam_s[m], q0_s[m], lam_s[sa], q0_s[sa], geo_h, geo_dh, geo_k);
        }
    };
    const U4 rn = draw_traj(s, seed, t, kStreamHop, (uint64_t)s.nstep[t]);
    const double zeta = u53(rn.v[0], rn.v[1]);
    __syncthreads();

    bool do_ratios = !singular;
    if (do_ratios && skip_bound && g_out == nullptr) {
        // |det S| = prod |U_kk| from the stored reciprocals, as a sum of logs
        double lg = 0.0;
        for (int kc = threadIdx.x; kc < Ne; kc += blockDim.x) {
            const double2 u = to_d2(dinv[kc]);  // 1/U_kk
            lg -= 0.5 * log(u.x * u.x + u.y * u.y);
        }
        const double det_abs = exp(block_sum(lg, red));
        // upper bound of the total hop probability (Sec. II C): |<J|psi>| <= 1
        double part = 0.0;
        for (int idx = threadIdx.x; idx < Ne * nu; idx += blockDim.x) {
            const int a = idx / nu, m = unocc[idx - a * nu];
            const int sa = occ_s[a];
            part += fabs(hop_nac(m, sa));
        }
        const double sd = block_sum(part, red);
        const double bound = 2.0 * dt * fabs(v) * sd / det_abs;
        // margin for the rounding of |det S|: FP64 factors, or FP32 (mixed)
        if (bound * (kF32 ? 1.0 + 1e-5 : 1.0 + 1e-9) < zeta) do_ratios = false;
    }

    double *scr = s.scratch + t * s.scratch_stride;
    double *G = g_out ? g_out + (int64_t)t * Ne * N : scr + 2 * (int64_t)Ne * N;  // [Ne][N]
    // four lanes per unoccupied row: lane `sub` owns the entries k = sub (mod 4)
    const int sub = threadIdx.x & 3, grp = threadIdx.x >> 2, ngrp = blockDim.x >> 2;
    const unsigned quad = 0xFu << (lane & ~3);
    if (do_ratios) {
        if constexpr (kF32) {
            float2 *A32 = reinterpret_cast<float2 *>(A);  // FP32 factors
            float2 *dinv32 = reinterpret_cast<float2 *>(dinv);
            // substitution rows of one pass: group grp owns row grp (reused each pass)
            float2 *Y = reinterpret_cast<float2 *>(hop_smem + (size_t)8 * Ne * Ne);  // [min(nu, ngrp)][Ne]
            for (int u0 = 0; u0 < nu; u0 += ngrp) {
                const int u = u0 + grp;
                const bool live = u < nu;
                const int m = live ? unocc[u] : 0;
                float2 *y = Y + (size_t)(live ? grp : 0) * Ne;
                // right-hand side c_m gathered up front (all loads in flight)
                if (live)
                    for (int i = sub; i < Ne; i += 4) {
                        const CT c = Ct[(int64_t)i * N + m];
                        y[i] = make_float2(c.x, c.y);
                    }
                __syncwarp(quad);
                // y U = c_m  (U_ij = A[perm[i]][j], i <= j), in place
                for (int jc = 0; jc < Ne; ++jc) {
                    float2 acc = make_float2(0.f, 0.f);
                    if (live)
                        for (int i = sub; i < jc; i += 4) acc = cfmsf(acc, y[i], A32[perm[i] * Ne + jc]);
                    acc.x += __shfl_xor_sync(quad, acc.x, 1);
                    acc.y += __shfl_xor_sync(quad, acc.y, 1);
                    acc.x += __shfl_xor_sync(quad, acc.x, 2);
                    acc.y += __shfl_xor_sync(quad, acc.y, 2);
                    if (live && sub == (jc & 3)) {
                        const float2 c = y[jc];
                        y[jc] = cmulf(make_float2(c.x + acc.x, c.y + acc.y), dinv32[jc]);
                    }
                }
                // z L = y  (L_ij = A[perm[i]][j], i > j, unit diagonal)
                for (int jc = Ne - 2; jc >= 0; --jc) {
                    float2 acc = make_float2(0.f, 0.f);
                    if (live) {
                        int i = jc + 1 + ((sub - (jc + 1)) & 3);
                        for (; i < Ne; i += 4) acc = cfmsf(acc, y[i], A32[perm[i] * Ne + jc]);
                    }
                    acc.x += __shfl_xor_sync(quad, acc.x, 1);
                    acc.y += __shfl_xor_sync(quad, acc.y, 1);
                    acc.x += __shfl_xor_sync(quad, acc.x, 2);
                    acc.y += __shfl_xor_sync(quad, acc.y, 2);
                    if (live && sub == (jc & 3)) y[jc] = make_float2(y[jc].x + acc.x, y[jc].y + acc.y);
                }
                // R_{m, perm[i]} = z_i ; g_{a->m}
                if (live)
                    for (int i = sub; i < Ne; i += 4) {
                        const int a = perm[i];
                        const int sa = occ_s[a];
                        const double d = hop_nac(m, sa);
                        const double gam = -2.0 * dt * v * (double)y[i].x * d;
                        G[(int64_t)a * N + m] = gam > 0.0 ? gam : 0.0;
                    }
            }
        } else {
            double2 *Y = reinterpret_cast<double2 *>(scr);  // [Ne][N], column m per row
            for (int u0 = 0; u0 < nu; u0 += ngrp) {
                const int u = u0 + grp;
                const bool live = u < nu;
                const int m = live ? unocc[u] : 0;
                for (int jc = 0; jc < Ne; ++jc) {
                    double2 acc = make_double2(0.0, 0.0);
                    if (live)
                        for (int i = sub; i < jc; i += 4)
                            acc = cfms(acc, Y[(int64_t)i * N + m], A[perm[i] * Ne + jc]);
                    acc.x += __shfl_xor_sync(quad, acc.x, 1);
                    acc.y += __shfl_xor_sync(quad, acc.y, 1);
                    acc.x += __shfl_xor_sync(quad, acc.x, 2);
                    acc.y += __shfl_xor_sync(quad, acc.y, 2);
                    if (live && sub == (jc & 3)) {
                        const double2 c = to_d2(Ct[(int64_t)jc * N + m]);
                        Y[(int64_t)jc * N + m] = cmul(make_double2(c.x + acc.x, c.y + acc.y), dinv[jc]);
                    }
                }
                for (int jc = Ne - 2; jc >= 0; --jc) {
                    double2 acc = make_double2(0.0, 0.0);
                    if (live) {
                        int i = jc + 1 + ((sub - (jc + 1)) & 3);
                        for (; i < Ne; i += 4)
                            acc = cfms(acc, Y[(int64_t)i * N + m], A[perm[i] * Ne + jc]);
                    }
                    acc.x += __shfl_xor_sync(quad, acc.x, 1);
                    acc.y += __shfl_xor_sync(quad, acc.y, 1);
                    acc.x += __shfl_xor_sync(quad, acc.x, 2);
                    acc.y += __shfl_xor_sync(quad, acc.y, 2);
                    if (live && sub == (jc & 3)) {
                        const double2 yv = Y[(int64_t)jc * N + m];
                        Y[(int64_t)jc * N + m] = make_double2(yv.x + acc.x, yv.y + acc.y);
                    }
                }
                if (live)
                    for (int i = sub; i < Ne; i += 4) {
                        const int a = perm[i];
                        const int sa = occ_s[a];
                        const double d = hop_nac(m, sa);
                        const double gam = -2.0 * dt * v * Y[(int64_t)i * N + m].x * d;
                        G[(int64_t)a * N + m] = gam > 0.0 ? gam : 0.0;
                    }
            }
        }
        if (g_out)
            for (int idx = threadIdx.x; idx < Ne * Ne; idx += blockDim.x)
                G[(int64_t)(idx / Ne) * N + occ_s[idx % Ne]] = 0.0;
    } else if (g_out) {
        for (int idx = threadIdx.x; idx < Ne * N; idx += blockDim.x) G[idx] = 0.0;
    }
    __syncthreads();
    if (g_out) return;

    hop_finish<CT, EXT>(s, t, mass, zeta, do_ratios, G, red, scr, unocc, occ_s, lam_s, q0_s, geo_h, geo_dh,
                        geo_k, s_hop_a, s_hop_m, Ct);
}

// ========================================================== work list
// Stable in-place compaction of the live list: keep the trajectories that
// are neither finished nor non-finite.  One CTA of 1024 threads; the order
// of the kept entries is preserved, so results do not depend on when the
// list is compacted.
__global__ void __launch_bounds__(1024) k_compact(const uint32_t *__restrict__ status,
                                                  int32_t *__restrict__ live,
                                                  int32_t *__restrict__ n_live)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t s_base;
    const int n = *n_live;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int32_t v = -1;
        int keep = 0;
        if (i < n) {
            v = live[i];
            keep = !(status[v] & (ST_DONE | ST_NAN));
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int off = s_base, tot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) off += wsum[w];
            tot += wsum[w];
        }
        off += __popc(m & ((1u << lane) - 1u));
        __syncthreads();
        if (keep) live[off] = v;  // off <= i: earlier entries were read already
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_live = s_base;
}

__global__ void k_live_init(int64_t n, int32_t *__restrict__ live, int32_t *__restrict__ n_live)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) live[i] = (int32_t)i;
    if (i == 0) *n_live = (int32_t)n;
}

cudaError_t launch_compact(const DevState &s, int32_t *live, int32_t *n_live, cudaStream_t st)
{
    k_compact<<<1, 1024, 0, st>>>(s.status, live, n_live);
    return cudaGetLastError();
}

cudaError_t launch_live_init(int64_t n, int32_t *live, int32_t *n_live, cudaStream_t st)
{
    k_live_init<<<(unsigned)((n + 255) / 256 + 1), 256, 0, st>>>(n, live, n_live);
    return cudaGetLastError();
}

// ================================================================= init
__global__ void k_init_nuclear(DevState s, double mass, uint64_t seed, double kT, int wigner,
                               double omega, double x_eq)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const U4 o = draw_traj(s, seed, t, kStreamNuc, 0);
    const double u1 = u53(o.v[0], o.v[1]), u2 = u53(o.v[2], o.v[3]);
    const double r = sqrt(-2.0 * log(1.0 - u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    double kTe = kT;
    if (wigner && kT > 0.0) {
        const double bw = omega / kT;
        kTe = kT * (bw / (2.0 * tanh(0.5 * bw)));
    }
    s.x[t] = x_eq + sqrt(kTe / (mass * omega * omega)) * (r * cs);
    s.p[t] = sqrt(mass * kTe) * (r * sn);
}

// Exact canonical sample of the occupied orbitals at temperature kT: the
// table logZ(k, n) of the remaining orbitals k..N-1 holding n electrons is
// built backwards (threads over n), then orbitals are visited upwards and
// occupied with probability exp(-lam_k/kT) Z(k+1, n-1) / Z(k, n).
__global__ void k_sample_occ(DevState s, uint64_t seed, double kT)
{
    const int64_t t = blockIdx.x;
    if (t >= s.n) return;
    const int N = s.N, Ne = s.Ne;
    if (kT <= 0.0) {
        for (int a = threadIdx.x; a < Ne; a += blockDim.x) s.occ[t * Ne + a] = (int16_t)a;
        return;
    }
    double *LZ = s.scratch + t * s.scratch_stride;  // [(N+1)][(Ne+1)]
    const int W1 = Ne + 1;
    const double ref = s.lam[t * N];
    const double NEG = -__longlong_as_double(0x7ff0000000000000ll);
    for (int n = threadIdx.x; n <= Ne; n += blockDim.x) LZ[(int64_t)N * W1 + n] = (n == 0) ? 0.0 : NEG;
    __syncthreads();
    for (int k = N - 1; k >= 0; --k) {
        const double lw = -(s.lam[t * N + k] - ref) / kT;
        for (int n = threadIdx.x; n <= Ne; n += blockDim.x) {
            const double a = LZ[(int64_t)(k + 1) * W1 + n];
            const double b = (n > 0) ? lw + LZ[(int64_t)(k + 1) * W1 + n - 1] : NEG;
            const double mx = fmax(a, b);
            LZ[(int64_t)k * W1 + n] = (mx == NEG) ? NEG : mx + log(exp(a - mx) + exp(b - mx));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int n = Ne, cnt = 0;
        for (int k = 0; k < N && n > 0; ++k) {
            const U4 o = draw_traj(s, seed, t, kStreamElec, (uint64_t)k);
            const double u = u53(o.v[0], o.v[1]);
            const double lw = -(s.lam[t * N + k] - ref) / kT;
            const double pk = exp(lw + LZ[(int64_t)(k + 1) * W1 + n - 1] - LZ[(int64_t)k * W1 + n]);
            if (u < pk) {
                s.occ[t * Ne + cnt++] = (int16_t)k;
                --n;
            }
        }
    }
}

template <class T2>
__global__ void k_unit_coeffs(DevState s)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = s.N, Ne = s.Ne;
    const int64_t total = s.n * Ne * N;
    if (idx >= total) return;
    const int64_t t = idx / ((int64_t)Ne * N);
    const int rem = (int)(idx - t * Ne * N);
    const int e = rem / N, i = rem - e * N;
    T2 v;
    v.x = (i == s.occ[t * Ne + e]) ? 1 : 0;
    v.y = 0;
    reinterpret_cast<T2 *>(s.C)[idx] = v;
}

// ============================================================ launches
static inline int round32(int v) { return (v + 31) & ~31; }

cudaError_t launch_eigen(const DevState &s, const ModelDev &md, double dt, int mode,
                         cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    const int tpb = eigen_tpb(s.N);
    const int threads = round32(tpb * s.N);
    const bool df = s.eigen_dfloat != 0;
    const size_t smem =
        (size_t)(s.M + tpb * (s.M + 2 * s.N + eigen_pow2(s.N) + (df ? s.M : 0))) * sizeof(double);
    if (df) k_eigen<true><<<(unsigned)((s.n + tpb - 1) / tpb), threads, smem, st>>>(s, md, dt, mode, tpb);
    else k_eigen<false><<<(unsigned)((s.n + tpb - 1) / tpb), threads, smem, st>>>(s, md, dt, mode, tpb);
    return cudaGetLastError();
}

cudaError_t launch_force(const DevState &s, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    k_force<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(s);
    return cudaGetLastError();
}

// The mixed path deflates on the SIMT kernel k_cheb_f32t only: requested by
// shape (cheb_ept 4 or 32), or where neither tensor-core kernel fits.  The
// tensor-core kernels' orders are cheap enough that the eigenvector set-up
// costs more than the orders it saves (measured with a deflating FP16 split
// kernel at N = 101, Ne = 50, 4096 trajectories: coupling +0.19 ms,
// propagation -0.13 ms per step), so they keep the full interval.
static bool mixed_uses_simt(const DevState &s)
{
    if (s.cheb_ept == 16 || s.cheb_ept == 8) return false;
    if (s.cheb_ept == 4 || s.cheb_ept == 32) return true;
    return !cheb_tc16_eligible(s.N, s.Ne) && !cheb_tc_eligible(s.N, s.Ne);
}

bool mixed_deflates(const DevState &s) { return s.defl != nullptr && mixed_uses_simt(s); }

cudaError_t launch_coupling(const DevState &s, double dt, double mass, double tol, bool mixed,
                            cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    const int threads = round32(s.N < 256 ? s.N : 256);
    if (mixed) {
        // the deflation's disc ends and u only when it may run (occupancy)
        const bool dfl = mixed_deflates(s);
        const size_t smem = (size_t)(32 + (dfl ? 2 : 1) * s.N) * sizeof(double) + (size_t)(dfl ? 10 : 8) * s.N * sizeof(float);
        if (dfl) k_build_w_f32<true><<<(unsigned)s.n, threads, smem, st>>>(s, dt, mass, tol);
        else k_build_w_f32<false><<<(unsigned)s.n, threads, smem, st>>>(s, dt, mass, tol);
    } else {
        k_build_w<<<(unsigned)s.n, threads, (size_t)(8 * s.N + 32) * sizeof(double), st>>>(s, dt, mass, tol);
    }
    return cudaGetLastError();
}

// Column-group shape of k_cheb: EPT electrons per thread and G groups per
// CTA, chosen to fill warps (rows x groups close to a multiple of 32) and to
// waste no electron slots, within 1024 threads.
void cheb_shape(int N, int Ne, int &ept, int &G)
{
    double best = -1.0;
    ept = 1;
    G = 1;
    for (int e = 2; e >= 1; --e) {
        for (int g = 1; g * N <= 1024; ++g) {
            const int nb = g * e;
            if (nb > 2 * Ne + 1) break;
            const int thr = g * N, thr32 = (thr + 31) & ~31;
            const int blocks = (Ne + nb - 1) / nb;
            const double eff = (double)thr / thr32 * (double)Ne / (blocks * nb);
            // prefer larger CTAs at equal efficiency (fewer W reloads)
            const double score = eff + 1e-4 * nb;
            if (score > best) {
                best = score;
                ept = e;
                G = g;
            }
        }
    }
}

cudaError_t launch_cheb(const DevState &s, double dt, bool mixed, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    if (mixed) {
        // tensor cores (3xTF32) when the trajectory fits one CTA, unless a
        // SIMT shape was requested
        // tensor cores: FP16 split operands (two CTAs per SM) where they fit,
        // else 3xTF32 (one CTA per SM), unless a shape was requested
        if (s.cheb_ept == 16 || (s.cheb_ept == 0 && cheb_tc16_eligible(s.N, s.Ne))) return launch_cheb_tc16(s, dt, st);
        if (s.cheb_ept == 8 || (s.cheb_ept == 0 && cheb_tc_eligible(s.N, s.Ne))) return launch_cheb_tc(s, dt, st);
        // SIMT: one row quad per thread (cheb_ept 4) or two (cheb_ept 32); by
        // default two past N = 224, where its one CTA per SM measured faster
        // (N = 256: 24.5 against 29.9 ms per step at 4096 trajectories; at
        // N = 201 it measured 29.4 against 26.2 ms)
        const int qpt = s.cheb_ept == 32 || (s.cheb_ept == 0 && s.N > kCheb32WideMinN) ? 2 : 1;
        int G;
        cheb32_shape(s.N, s.Ne, G, qpt);
        if (s.cheb_G > 0 && (s.cheb_ept == 4 || s.cheb_ept == 32)) G = s.cheb_G;
        const int nb = 4 * G, nqh = ((s.N + 3) / 4 + qpt - 1) / qpt;
        const size_t smem = cheb32_smem_bytes(s.N, G);
        const int threads = (G * nqh + 31) & ~31;
        for (int64_t t0 = 0; t0 < s.n; t0 += 65535) {
            const int64_t cnt = (s.n - t0 < 65535) ? s.n - t0 : 65535;
            dim3 grid((unsigned)((s.Ne + nb - 1) / nb), (unsigned)cnt);
            const int dfl = mixed_deflates(s) ? 1 : 0;
            if (qpt == 2) k_cheb_f32t<4, 2><<<grid, threads, smem, st>>>(s, dt, G, t0, dfl);
            else k_cheb_f32t<4, 1><<<grid, threads, smem, st>>>(s, dt, G, t0, dfl);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    int ept, G;
    cheb_shape(s.N, s.Ne, ept, G);
    if (s.cheb_ept > 0 && s.cheb_G > 0) {
        ept = s.cheb_ept;
        G = s.cheb_G;
    }
    const int nb = G * ept;
    const size_t smem = (size_t)s.N * 2 * nb * sizeof(double);
    const int threads = (G * s.N + 31) & ~31;
    for (int64_t t0 = 0; t0 < s.n; t0 += 65535) {
        const int64_t cnt = (s.n - t0 < 65535) ? s.n - t0 : 65535;
        dim3 grid((unsigned)((s.Ne + nb - 1) / nb), (unsigned)cnt);
        if (ept == 2) k_cheb<2, double><<<grid, threads, smem, st>>>(s, dt, G, t0);
        else k_cheb<1, double><<<grid, threads, smem, st>>>(s, dt, G, t0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Allow the hop kernels and the tiled FP32 propagator the device's full opt-in shared memory (minus their
// static shared memory), so that later launches, including launches under
// stream capture, need no attribute change.
template <class F>
static void allow_max_smem(F *fn)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    cudaGetLastError();
}

void configure_hop_smem()
{
    allow_max_smem(k_hop<float2, 512, 1>);
    allow_max_smem(k_hop<double2, 512, 1>);
    allow_max_smem(k_hop<float2, 256, 4>);
    allow_max_smem(k_hop<double2, 256, 3>);
    allow_max_smem(k_hop<double2, 512, 1, true>);
    allow_max_smem(k_hop<double2, 256, 3, true>);
    allow_max_smem(k_hop<float2, 512, 1, true>);
    allow_max_smem(k_hop<float2, 256, 4, true>);
    allow_max_smem(k_cheb_f32t<4, 1>);
    allow_max_smem(k_cheb_f32t<4, 2>);
    configure_hop_gjl();
}

cudaError_t launch_hop(const DevState &s, double dt, double mass, uint64_t seed, int skip_bound,
                       double *g_out, cudaStream_t st, bool mixed, bool ext)
{
    if (s.n == 0) return cudaSuccess;
    // mixed path: the register-resident Gauss-Jordan kernel where it fits,
    // unless a hop CTA size was requested
    if (mixed && s.hop_threads == 0 && hop_gj_eligible(s.N, s.Ne))
        return launch_hop_gj(s, dt, mass, seed, g_out, st, ext);
    if (mixed && s.hop_threads == 0 && hop_gjl_eligible(s.N, s.Ne))
        return launch_hop_gjl(s, dt, mass, seed, g_out, st, ext);
    const size_t smem = hop_smem_bytes(s.N, s.Ne, mixed, ext);
    // 256-thread CTAs (three per SM) when two or more fit in shared memory,
    // else one CTA of 512
    int threads = (2 * smem + 2048 <= 227 * 1024) ? 256 : 512;
    if (s.hop_threads > 0) threads = s.hop_threads;
    // The shared-memory limit is a process-wide function attribute, not a
    // stream operation.  configure_hop_smem() raises it to the device's opt-in
    // maximum when a context is created; here it is only ever raised (outside
    // stream capture), never lowered, so that a small launch cannot take the
    // room away from a larger one captured later.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    auto go = [&](auto kern) {
        if (cs == cudaStreamCaptureStatusNone) {
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess &&
                fa.maxDynamicSharedSizeBytes < (int)smem)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaGetLastError();
        }
        kern<<<(unsigned)s.n, threads, smem, st>>>(s, dt, mass, seed, skip_bound, g_out);
    };
    if (ext && mixed) {
        if (threads == 256) go(k_hop<float2, 256, 4, true>);
        else go(k_hop<float2, 512, 1, true>);
    } else if (ext) {
        if (threads == 256) go(k_hop<double2, 256, 3, true>);
        else go(k_hop<double2, 512, 1, true>);
    } else if (mixed) {
        if (threads == 256) go(k_hop<float2, 256, 4>);
        else go(k_hop<float2, 512, 1>);
    } else {
        if (threads == 256) go(k_hop<double2, 256, 3>);
        else go(k_hop<double2, 512, 1>);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_nuclear(const DevState &s, double mass, uint64_t seed, double kT,
                                int wigner, double omega, double x_eq, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    k_init_nuclear<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(s, mass, seed, kT, wigner, omega, x_eq);
    return cudaGetLastError();
}

cudaError_t launch_sample_occ(const DevState &s, uint64_t seed, double kT, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    k_sample_occ<<<(unsigned)s.n, 64, 0, st>>>(s, seed, kT);
    return cudaGetLastError();
}

cudaError_t launch_unit_coeffs(const DevState &s, bool fp32, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    const int64_t total = s.n * s.Ne * s.N;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (fp32) k_unit_coeffs<float2><<<blocks, 256, 0, st>>>(s);
    else k_unit_coeffs<double2><<<blocks, 256, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace iesh
