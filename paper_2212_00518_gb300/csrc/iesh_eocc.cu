// iesh_eocc.cu -- occupied-orbital energy of a two-orbital adsorbate and its
// Hellmann-Feynman gradients (differentiable-energy workload).
//
// One-electron Hamiltonian: adsorbate orbitals a = 0, 1 with levels
// h_a = eps_a + sum_al g_{a,al} x_al, each coupled to bath state k by
// V_ak = vbar_a sqrt(w_k) f_a(x), f_a = exp(-|x_a - R_a|^2 / (2 sigma_a^2)),
// x_a = (x_{3a}, x_{3a+1}, x_{3a+2}); no direct adsorbate-adsorbate term.
// E_occ = sum of the Ne lowest eigenvalues (the classical IESH potential of
// Sec. II B at the ground-state occupation, without U0).
//
// Both border vectors are proportional to sqrt(w_k), so with c_a = vbar_a f_a
// the combination |+> = (c_0|0> + c_1|1>)/c couples to the bath with
// z_k = c sqrt(w_k) and |-> = (-c_1|0> + c_0|1>)/c does not; |-> couples
// only to |+> (through t = c_0 c_1 (h_1 - h_0) / c^2).  Eliminating |->
// leaves one arrowhead secular equation with the bath poles plus one pole at
// h_- = <-|H|-> of weight t^2:
//   lam - h_+ - sum_k z_k^2 / (lam - eps_k) - t^2 / (lam - h_-) = 0,
// whose root i has q_+ = 1/sqrt(g'(lam)), q_- = t q_+ / (lam - h_-).
// Hellmann-Feynman: dE/dy = sum_a [S_a dh_a/dy + 2 T_a dlog f_a/dy] with
// S_a = sum_{i<Ne} Q_ai^2 and T_a = sum_{i<Ne} Q_ai^2 (lam_i - h_a), because
// sum_k V_ak Q_ki = (lam_i - h_a) Q_ai on an eigenvector.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/iesh.h"
#include "iesh_common.cuh"
#include "iesh_secular.cuh"

using namespace iesh;

struct iesh_eocc_ctx {
    iesh_eocc_model model;
    cudaStream_t stream = nullptr;
    int M = 0, Ne = 0;
    double *eps_d = nullptr, *w_d = nullptr;  // bath energies, weights (FP64)
    float *eps_f = nullptr, *w_f = nullptr;   // FP32 copies
    std::string err;
};

namespace {

struct EoccConst {
    double vbar[2];
    double R[6];
};

// Per-geometry adsorbate quantities.
template <class R>
struct Ads {
    R h[2], f[2], r2[2], c[2];
};

template <class R>
__device__ __forceinline__ Ads<R> ads_eval(const EoccConst &k, const R *x, const R *th)
{
    Ads<R> o;
    for (int a = 0; a < 2; ++a) {
        R h = th[a];
        for (int al = 0; al < 6; ++al) h += th[2 + 6 * a + al] * x[al];
        R r2 = 0;
        for (int q = 0; q < 3; ++q) {
            const R d = x[3 * a + q] - (R)k.R[3 * a + q];
            r2 += d * d;
        }
        const R sg = th[14 + a];
        o.h[a] = h;
        o.r2[a] = r2;
        o.f[a] = exp(-R(0.5) * r2 / (sg * sg));
        o.c[a] = (R)k.vbar[a] * o.f[a];
    }
    return o;
}

// One CTA per geometry, one thread per needed root (the Ne lowest).
template <class R>
__global__ void k_eocc_fwd(int64_t B, int M, int Ne, EoccConst kc, const R *__restrict__ eps,
                           const R *__restrict__ w, const R *__restrict__ x, const R *__restrict__ th,
                           R *__restrict__ E, R *__restrict__ saved, uint32_t *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char eocc_smem[];
    R *pole = reinterpret_cast<R *>(eocc_smem);  // [M + 1]
    R *wt = pole + (M + 1);                      // [M + 1]
    double *red = reinterpret_cast<double *>(wt + (M + 1));  // [32], 2(M+1) values before it
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    R xs[6], ths[16];
    for (int q = 0; q < 6; ++q) xs[q] = x[b * 6 + q];
    for (int q = 0; q < 16; ++q) ths[q] = th[q];
    const Ads<R> ad = ads_eval<R>(kc, xs, ths);
    const R c2 = ad.c[0] * ad.c[0] + ad.c[1] * ad.c[1];
    const R c = sqrt(c2);
    const R hp = (ad.c[0] * ad.c[0] * ad.h[0] + ad.c[1] * ad.c[1] * ad.h[1]) / c2;
    const R hm = (ad.c[1] * ad.c[1] * ad.h[0] + ad.c[0] * ad.c[0] * ad.h[1]) / c2;
    const R tt = ad.c[0] * ad.c[1] * (ad.h[1] - ad.h[0]) / c2;
    const bool decoupled = !(tt * tt > R(0));
    // poles: bath energies, plus h_- in its sorted place unless |-> decouples
    int pos = 0;
    for (int k = 0; k < M; ++k) pos += (eps[k] < hm);
    const int P = decoupled ? M : M + 1;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const int slot = (decoupled || k < pos) ? k : k + 1;
        pole[slot] = eps[k];
        wt[slot] = c2 * w[k];
    }
    if (!decoupled && threadIdx.x == 0) {
        pole[pos] = hm;
        wt[pos] = tt * tt;
    }
    __syncthreads();
    R Z2 = 0;
    for (int k = 0; k < P; ++k) Z2 += wt[k];
    uint32_t st = 0;
    double le = 0.0, s0 = 0.0, s1 = 0.0, t0 = 0.0, t1 = 0.0;
    const int r = threadIdx.x;
    if (r < Ne) {
        R lam, qp;
        const Poles<R> pp = {P, pole, wt, nullptr, nullptr, nullptr};
        secular_root<R>(r, pp, hp, Z2, false, R(0), lam, qp, st);
        const R qm = decoupled ? R(0) : tt * qp / (lam - hm);
        const R Q0 = (ad.c[0] * qp - ad.c[1] * qm) / c;
        const R Q1 = (ad.c[1] * qp + ad.c[0] * qm) / c;
        le = (double)lam;
        s0 = (double)(Q0 * Q0);
        s1 = (double)(Q1 * Q1);
        t0 = (double)(Q0 * Q0 * (lam - ad.h[0]));
        t1 = (double)(Q1 * Q1 * (lam - ad.h[1]));
        if (decoupled && r == Ne - 1 && hm < lam) {
            // the decoupled |-> state is among the Ne lowest: it replaces root Ne-1
            le = (double)hm;
            const R P0 = -ad.c[1] / c, P1 = ad.c[0] / c;
            s0 = (double)(P0 * P0);
            s1 = (double)(P1 * P1);
            t0 = (double)(P0 * P0 * (hm - ad.h[0]));
            t1 = (double)(P1 * P1 * (hm - ad.h[1]));
        }
    }
    if (st) atomicOr(&status[b], st);
    le = block_sum(le, red);
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    t0 = block_sum(t0, red);
    t1 = block_sum(t1, red);
    if (threadIdx.x == 0) {
        E[b] = (R)le;
        saved[b * 4 + 0] = (R)s0;
        saved[b * 4 + 1] = (R)s1;
        saved[b * 4 + 2] = (R)t0;
        saved[b * 4 + 3] = (R)t1;
    }
}

// dE/dx [B][6] and per-geometry dE/dtheta [B][16], scaled by gE.
template <class R>
__global__ void k_eocc_bwd(int64_t B, EoccConst kc, const R *__restrict__ x, const R *__restrict__ th,
                           const R *__restrict__ saved, const R *__restrict__ gE, R *__restrict__ dx,
                           R *__restrict__ dth_per)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    R xs[6], ths[16];
    for (int q = 0; q < 6; ++q) xs[q] = x[b * 6 + q];
    for (int q = 0; q < 16; ++q) ths[q] = th[q];
    const Ads<R> ad = ads_eval<R>(kc, xs, ths);
    const R g = gE[b];
    const R S[2] = {saved[b * 4 + 0], saved[b * 4 + 1]};
    const R T[2] = {saved[b * 4 + 2], saved[b * 4 + 3]};
    for (int al = 0; al < 6; ++al) {
        R d = 0;
        for (int a = 0; a < 2; ++a) {
            d += S[a] * ths[2 + 6 * a + al];
            if (al / 3 == a) {
                const R sg = ths[14 + a];
                d += R(2) * T[a] * (-(xs[al] - (R)kc.R[al]) / (sg * sg));
            }
        }
        dx[b * 6 + al] = g * d;
    }
    R *o = dth_per + b * 16;
    for (int a = 0; a < 2; ++a) {
        o[a] = g * S[a];
        for (int al = 0; al < 6; ++al) o[2 + 6 * a + al] = g * S[a] * xs[al];
        const R sg = ths[14 + a];
        o[14 + a] = g * R(2) * T[a] * ad.r2[a] / (sg * sg * sg);
    }
}

// dtheta[p] = sum_b dth_per[b][p] (one CTA per parameter, fixed order).
template <class R>
__global__ void k_eocc_reduce(int64_t B, const R *__restrict__ dth_per, R *__restrict__ dth)
{
    __shared__ double red[32];
    const int p = blockIdx.x;
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) s += (double)dth_per[b * 16 + p];
    s = block_sum(s, red);
    if (threadIdx.x == 0) dth[p] = (R)s;
}

iesh_status efail(iesh_eocc_ctx *c, iesh_status s, const char *msg)
{
    if (c) c->err = msg;
    return s;
}

void gl_nodes(int n, std::vector<double> &x, std::vector<double> &w)
{
    // Newton on the Legendre polynomial (three-term recurrence)
    const double pi = 3.14159265358979323846;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p1 = z;
                p0 = 1.0;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) {
            p1 = z;
            p0 = 1.0;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

EoccConst make_const(const iesh_eocc_model &m)
{
    EoccConst k;
    for (int a = 0; a < 2; ++a) k.vbar[a] = m.vbar[a];
    for (int q = 0; q < 6; ++q) k.R[q] = m.R[q];
    return k;
}

}  // namespace

extern "C" {

iesh_status iesh_eocc_create(iesh_eocc_ctx **out, const iesh_eocc_model *model, void *cuda_stream)
{
    if (!out) return IESH_EINVAL;
    *out = nullptr;
    if (!model) return IESH_EINVAL;
    iesh_eocc_ctx *c = new iesh_eocc_ctx();
    *out = c;
    c->model = *model;
    c->stream = (cudaStream_t)cuda_stream;
    const int M = model->n_bath, Ne = model->n_elec;
    if (M < 2 || M > 4096) return efail(c, IESH_EINVAL, "n_bath outside 2..4096");
    if (Ne < 1 || Ne > M + 1 || Ne > 1024) return efail(c, IESH_EINVAL, "n_elec outside 1..min(M+1, 1024)");
    if (!(model->band_hi > model->band_lo)) return efail(c, IESH_EINVAL, "empty band");
    c->M = M;
    c->Ne = Ne;
    // split Gauss-Legendre bath at mu, M/2 nodes per half (Appendix A)
    const int nlo = M / 2, nhi = M - nlo;
    std::vector<double> x, wl, eps, w;
    gl_nodes(nlo, x, wl);
    for (int k = 0; k < nlo; ++k) {
        eps.push_back(0.5 * (model->mu - model->band_lo) * x[k] + 0.5 * (model->band_lo + model->mu));
        w.push_back(0.5 * (model->mu - model->band_lo) * wl[k]);
    }
    gl_nodes(nhi, x, wl);
    for (int k = 0; k < nhi; ++k) {
        eps.push_back(0.5 * (model->band_hi - model->mu) * x[k] + 0.5 * (model->mu + model->band_hi));
        w.push_back(0.5 * (model->band_hi - model->mu) * wl[k]);
    }
    std::vector<float> epsf(eps.begin(), eps.end()), wf(w.begin(), w.end());
    if (cudaMalloc(&c->eps_d, M * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->w_d, M * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->eps_f, M * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c->w_f, M * sizeof(float)) != cudaSuccess)
        return efail(c, IESH_ENOMEM, "cudaMalloc failed");
    if (cudaMemcpy(c->eps_d, eps.data(), M * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->w_d, w.data(), M * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->eps_f, epsf.data(), M * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->w_f, wf.data(), M * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return efail(c, IESH_ECUDA, "bath upload failed");
    return IESH_OK;
}

iesh_status iesh_eocc_destroy(iesh_eocc_ctx *c)
{
    if (!c) return IESH_OK;
    cudaFree(c->eps_d);
    cudaFree(c->w_d);
    cudaFree(c->eps_f);
    cudaFree(c->w_f);
    delete c;
    return IESH_OK;
}

const char *iesh_eocc_last_error(const iesh_eocc_ctx *c) { return c ? c->err.c_str() : "null context"; }

iesh_status iesh_eocc_forward(iesh_eocc_ctx *c, int64_t B, int precision, const void *x,
                              const void *theta, void *E, void *saved, uint32_t *status)
{
    if (!c) return IESH_EINVAL;
    if (B < 0) return efail(c, IESH_EINVAL, "B < 0");
    if (B == 0) return IESH_OK;
    if (!x || !theta || !E || !saved || !status) return efail(c, IESH_EINVAL, "null pointer");
    const int M = c->M, Ne = c->Ne;
    const int threads = (Ne + 31) & ~31;
    const EoccConst kc = make_const(c->model);
    cudaError_t e = cudaMemsetAsync(status, 0, B * sizeof(uint32_t), c->stream);
    if (e != cudaSuccess) return efail(c, IESH_ECUDA, cudaGetErrorString(e));
    if (precision == IESH_PREC_FP64) {
        const size_t smem = (size_t)2 * (M + 2) * sizeof(double) + 32 * sizeof(double);
        k_eocc_fwd<double><<<(unsigned)B, threads, smem, c->stream>>>(
            B, M, Ne, kc, c->eps_d, c->w_d, (const double *)x, (const double *)theta, (double *)E,
            (double *)saved, status);
    } else if (precision == IESH_PREC_MIXED) {
        const size_t smem = (size_t)2 * (M + 2) * sizeof(float) + 33 * sizeof(double);
        k_eocc_fwd<float><<<(unsigned)B, threads, smem, c->stream>>>(
            B, M, Ne, kc, c->eps_f, c->w_f, (const float *)x, (const float *)theta, (float *)E,
            (float *)saved, status);
    } else {
        return efail(c, IESH_EINVAL, "unknown precision");
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? IESH_OK : efail(c, IESH_ECUDA, cudaGetErrorString(e));
}

iesh_status iesh_eocc_backward(iesh_eocc_ctx *c, int64_t B, int precision, const void *x,
                               const void *theta, const void *saved, const void *gE, void *dx,
                               void *dtheta_per, void *dtheta)
{
    if (!c) return IESH_EINVAL;
    if (B < 0) return efail(c, IESH_EINVAL, "B < 0");
    if (!x || !theta || !saved || !gE || !dx || !dtheta_per || !dtheta)
        return efail(c, IESH_EINVAL, "null pointer");
    const EoccConst kc = make_const(c->model);
    const unsigned blocks = (unsigned)((B + 127) / 128);
    if (precision == IESH_PREC_FP64) {
        if (B > 0)
            k_eocc_bwd<double><<<blocks, 128, 0, c->stream>>>(
                B, kc, (const double *)x, (const double *)theta, (const double *)saved,
                (const double *)gE, (double *)dx, (double *)dtheta_per);
        k_eocc_reduce<double><<<16, 256, 0, c->stream>>>(B, (const double *)dtheta_per, (double *)dtheta);
    } else if (precision == IESH_PREC_MIXED) {
        if (B > 0)
            k_eocc_bwd<float><<<blocks, 128, 0, c->stream>>>(
                B, kc, (const float *)x, (const float *)theta, (const float *)saved,
                (const float *)gE, (float *)dx, (float *)dtheta_per);
        k_eocc_reduce<float><<<16, 256, 0, c->stream>>>(B, (const float *)dtheta_per, (float *)dtheta);
    } else {
        return efail(c, IESH_EINVAL, "unknown precision");
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IESH_OK : efail(c, IESH_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
