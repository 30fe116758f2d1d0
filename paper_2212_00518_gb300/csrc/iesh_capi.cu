// iesh_capi.cu -- C-ABI of the batched IESH library: context, bath
// discretisation, state transfer and the step loop (declared in iesh.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/iesh.h"
#include "iesh_common.cuh"
#include "iesh_host.h"
#include "iesh_kernels.h"

using namespace iesh;

struct iesh_ctx {
    iesh_model model;
    iesh_options opt;
    int64_t max_traj = 0;
    cudaStream_t stream = nullptr;
    int N = 0, M = 0, Ne = 0;
    bool mixed = false;
    std::vector<double> eps_h, z0_h;
    ModelDev md;
    DevState ds;
    std::vector<void *> allocs;
    bool have_state = false;
    std::string err;
    int32_t *live = nullptr, *n_live = nullptr;  // device work list
    int64_t steps_since_init = 0;
    KernelTimer timer;  // kernel timing
    double *obs = nullptr;        // [4][max_traj] observables
    uint32_t *summary = nullptr;  // [9] status summary
    // iesh_run_host: copy streams and per-chunk events, made on first use
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev;
};

// Launch `fn` (returning cudaError_t), bracketed by events when profiling.
template <class Fn>
static cudaError_t timed(iesh_ctx *c, int cls, Fn fn)
{
    return c->timer.run(c->stream, cls, fn);
}

static const double kPi = 3.14159265358979323846;

static iesh_status fail(iesh_ctx *c, iesh_status s, const char *fmt, ...)
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

#define CU(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, IESH_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                \
    } while (0)

// ------------------------------------------------------------ bath (host)
// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on the
// Legendre polynomial P_n (three-term recurrence), started from the
// Tricomi approximation; w = 2 / ((1 - x^2) P_n'(x)^2).
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
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
        // final derivative at the converged node
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

// One lead: n states on [a, b], split Gauss-Legendre at mu with n_lo nodes
// below it (Appendix A), or the left-endpoint trapezoid rule.
void iesh::lead_bath(int disc, int n, double a, double b, double mu, int n_lo, std::vector<double> &eps,
                     std::vector<double> &w)
{
    eps.clear();
    w.clear();
    if (disc == IESH_DISC_TRAPEZOID) {
        for (int k = 0; k < n; ++k) {
            eps.push_back(a + k * (b - a) / n);
            w.push_back((b - a) / n);
        }
        return;
    }
    if (n_lo < 0) n_lo = n / 2;
    const int n_hi = n - n_lo;
    std::vector<double> x, wl;
    if (n_lo > 0) {
        gauss_legendre(n_lo, x, wl);
        for (int k = 0; k < n_lo; ++k) {
            eps.push_back(0.5 * (mu - a) * x[k] + 0.5 * (a + mu));
            w.push_back(0.5 * (mu - a) * wl[k]);
        }
    }
    if (n_hi > 0) {
        gauss_legendre(n_hi, x, wl);
        for (int k = 0; k < n_hi; ++k) {
            eps.push_back(0.5 * (b - mu) * x[k] + 0.5 * (mu + b));
            w.push_back(0.5 * (b - mu) * wl[k]);
        }
    }
}

static iesh_status make_bath(iesh_ctx *ctx)
{
    const iesh_model &m = ctx->model;
    const double vbar = std::sqrt(m.gamma / (2.0 * kPi));
    std::vector<std::pair<double, double>> all;
    std::vector<double> e, w;
    if (m.n_leads <= 1) {
        lead_bath(m.disc, m.n_bath, m.band_lo, m.band_hi, m.mu, m.n_lo, e, w);
        for (size_t k = 0; k < e.size(); ++k) all.push_back({e[k], vbar * std::sqrt(w[k])});
    } else {
        if (m.lead_n[0] + m.lead_n[1] != m.n_bath)
            return fail(ctx, IESH_EINVAL, "lead sizes %d + %d != n_bath %d", m.lead_n[0],
                        m.lead_n[1], m.n_bath);
        for (int L = 0; L < 2; ++L) {
            lead_bath(m.disc, m.lead_n[L], m.band_lo, m.band_hi, m.lead_mu[L], m.lead_nlo[L], e, w);
            for (size_t k = 0; k < e.size(); ++k)
                all.push_back({e[k], vbar * std::sqrt(w[k] * m.lead_frac[L])});
        }
        std::stable_sort(all.begin(), all.end(),
                         [](const std::pair<double, double> &p, const std::pair<double, double> &q) {
                             return p.first < q.first;
                         });
    }
    ctx->eps_h.clear();
    ctx->z0_h.clear();
    for (auto &pr : all) {
        ctx->eps_h.push_back(pr.first);
        ctx->z0_h.push_back(pr.second);
    }
    for (size_t k = 1; k < ctx->eps_h.size(); ++k)
        if (!(ctx->eps_h[k] > ctx->eps_h[k - 1]))
            return fail(ctx, IESH_EINVAL, "bath energies must be distinct (index %zu)", k);
    return IESH_OK;
}

// ------------------------------------------------------------------ util
template <class T>
static iesh_status dalloc(iesh_ctx *ctx, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess)
        return fail(ctx, IESH_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    cudaMemsetAsync(q, 0, bytes, ctx->stream);
    ctx->allocs.push_back(q);
    *p = (T *)q;
    return IESH_OK;
}

static iesh_status copy_in(iesh_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    if (!bytes) return IESH_OK;
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    return IESH_OK;
}

static iesh_status copy_out(iesh_ctx *ctx, void *dst, const void *src, size_t bytes, bool &sync)
{
    if (!bytes || !dst) return IESH_OK;
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    if (is_host_ptr(dst)) sync = true;
    return IESH_OK;
}

// ------------------------------------------------------------- ensemble
// Condition of the ensemble's device loop: after each chunk, continue while
// some context has a live trajectory and the step cap is not reached.
__global__ void k_ensemble_cond(cudaGraphConditionalHandle h, const int32_t *const *n_live, int n_ctx,
                                int64_t *steps, const int64_t *max_steps, int64_t chunk, int64_t *live_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t live = 0;
    for (int c = 0; c < n_ctx; ++c) live += *n_live[c];
    const int64_t st = *steps + chunk;
    *steps = st;
    *live_out = live;
    cudaGraphSetConditional(h, (live > 0 && st < *max_steps) ? 1u : 0u);
}

struct iesh_ensemble {
    std::vector<iesh_ctx *> ctxs;
    cudaStream_t stream = nullptr;   // launch stream (the caller's)
    cudaStream_t capture = nullptr;  // own stream for building the loop body
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int32_t **n_live_dev = nullptr;  // [n_ctx] device pointers of the live counts
    int64_t *counters = nullptr;           // device: steps, max_steps, live
    cudaEvent_t ev = nullptr;
    int64_t chunk = 0;
    std::string err;
};

static iesh_status efail(iesh_ensemble *e, iesh_status s, const char *fmt, ...)
{
    if (e) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        e->err = buf;
    }
    return s;
}

#define CUE(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return efail(ens, IESH_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                         __FILE__, __LINE__);                                                \
    } while (0)

// ----------------------------------------------------------------- C-ABI
extern "C" {

const char *iesh_status_string(iesh_status s)
{
    switch (s) {
    case IESH_OK: return "IESH_OK";
    case IESH_EINVAL: return "IESH_EINVAL";
    case IESH_ECUDA: return "IESH_ECUDA";
    case IESH_ENOMEM: return "IESH_ENOMEM";
    case IESH_ESTATE: return "IESH_ESTATE";
    case IESH_EUNSUPPORTED: return "IESH_EUNSUPPORTED";
    case IESH_ENONCONV: return "IESH_ENONCONV";
    case IESH_ESINGULAR: return "IESH_ESINGULAR";
    case IESH_ENORM: return "IESH_ENORM";
    case IESH_ENAN: return "IESH_ENAN";
    }
    return "IESH_?";
}

const char *iesh_last_error(const iesh_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

iesh_status iesh_destroy(iesh_ctx *ctx)
{
    if (!ctx) return IESH_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (cudaStream_t s : {ctx->s_in, ctx->s_out})
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    ctx->timer.release();
    for (void *p : ctx->allocs) cudaFree(p);
    delete ctx;
    return IESH_OK;
}

iesh_status iesh_create(iesh_ctx **out, const iesh_model *model, const iesh_options *opt,
                        int64_t max_traj, void *cuda_stream)
{
    if (!out) return IESH_EINVAL;
    *out = nullptr;
    if (!model || !opt || max_traj < 1) return IESH_EINVAL;
    iesh_ctx *ctx = new iesh_ctx();
    ctx->model = *model;
    ctx->opt = *opt;
    ctx->max_traj = max_traj;
    ctx->stream = (cudaStream_t)cuda_stream;
    const int M = model->n_bath, Ne = model->n_elec, N = M + 1;
    iesh_status st = IESH_OK;
    if (model->kind < 0 || model->kind > 2) st = fail(ctx, IESH_EINVAL, "unknown model kind %d", model->kind);
    else if (M < 1 || N > kMaxOrbitals) st = fail(ctx, IESH_EINVAL, "n_bath %d outside 1..%d", M, kMaxOrbitals - 1);
    else if (Ne < 1 || Ne > N - 1) st = fail(ctx, IESH_EINVAL, "n_elec %d outside 1..N-1", Ne);
    else if (Ne > kMaxHopElectrons) st = fail(ctx, IESH_EINVAL, "n_elec %d above %d", Ne, kMaxHopElectrons);
    else if (!(model->mass > 0.0)) st = fail(ctx, IESH_EINVAL, "mass must be positive");
    else if (!(model->gamma >= 0.0)) st = fail(ctx, IESH_EINVAL, "gamma must be >= 0");
    else if (opt->precision != IESH_PREC_FP64 && opt->precision != IESH_PREC_MIXED)
        st = fail(ctx, IESH_EINVAL, "unknown precision %d", opt->precision);
    else if (opt->record_every < 0 || opt->max_records < 0) st = fail(ctx, IESH_EINVAL, "negative record sizes");
    else if (opt->compact_every < 0) st = fail(ctx, IESH_EINVAL, "negative compact_every");
    else if (opt->propagator != IESH_PROP_AVERAGED && opt->propagator != IESH_PROP_OVERLAP)
        st = fail(ctx, IESH_EINVAL, "unknown propagator %d", opt->propagator);
    else if (opt->propagator == IESH_PROP_OVERLAP && opt->precision != IESH_PREC_FP64)
        st = fail(ctx, IESH_EUNSUPPORTED, "the overlap propagator is FP64 only");
    else if (!(opt->prop_tol >= 0.0 && opt->prop_tol < 1.0))
        st = fail(ctx, IESH_EINVAL, "prop_tol must be in [0, 1)");
    else if (opt->norm_tol != opt->norm_tol) st = fail(ctx, IESH_EINVAL, "norm_tol is NaN");
    else if (opt->traj_base < 0) st = fail(ctx, IESH_EINVAL, "traj_base must be >= 0");
    if (st != IESH_OK) {
        *out = ctx;  // let the caller read the message, then destroy
        return st;
    }
    ctx->N = N;
    ctx->M = M;
    ctx->Ne = Ne;
    ctx->mixed = opt->precision == IESH_PREC_MIXED;
    if ((st = make_bath(ctx)) != IESH_OK) {
        *out = ctx;
        return st;
    }
    ctx->md.kind = model->kind;
    ctx->md.mass = model->mass;
    for (int i = 0; i < 16; ++i) ctx->md.par[i] = model->par[i];

    DevState &d = ctx->ds;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.M = M;
    d.Ne = Ne;
    d.n = 0;
    const size_t T = (size_t)max_traj;
    d.scratch_stride = std::max<int64_t>({(int64_t)N * N, 3LL * Ne * N + Ne,
                                          (int64_t)(N + 1) * (Ne + 1)});
    d.scratch_stride = (d.scratch_stride + 31) & ~31LL;
    d.record_every = opt->record_every;
    d.max_records = opt->record_every > 0 ? opt->max_records : 0;
    d.z_done = opt->z_done;
    double *eps = nullptr, *z0 = nullptr;
#define A(ptr, cnt) if ((st = dalloc(ctx, &(ptr), (cnt))) != IESH_OK) { *out = ctx; return st; }
    A(d.x, T) A(d.p, T) A(d.F, T) A(d.dU0, T) A(d.vprev, T)
    A(d.occ, T * Ne)
    double *Cd = nullptr;
    A(Cd, T * Ne * N * 2)
    d.C = Cd;
    A(d.lam, T * N) A(d.q0, T * N) A(d.lam_prev, T * N) A(d.q0_prev, T * N)
    A(d.geo, T * 4) A(d.geo_prev, T * 4)
    A(d.rt, T * N) A(d.rt_prev, T * N) A(d.ro, T * N) A(d.ro_prev, T * N)
    A(d.fx, T) A(d.fx_prev, T)
    A(d.status, T) A(d.nstep, T) A(d.hops, T) A(d.frus, T)
    A(d.scratch, T * (size_t)d.scratch_stride)
    A(d.cheb, T * kChebStride)
    if (opt->propagator == IESH_PROP_AVERAGED && !opt->no_deflation)
        A(d.defl, T * (size_t)defl_stride(N, Ne))
    A(ctx->live, T)
    A(ctx->n_live, 1)
    A(ctx->obs, 4 * T)
    A(ctx->summary, 9)
    A(d.rec_sh, std::max<size_t>(1, T * d.max_records))
    A(d.rec_wf, std::max<size_t>(1, T * d.max_records))
    A(eps, (size_t)M) A(z0, (size_t)M)
    float *epsdiff = nullptr;
    A(epsdiff, (size_t)M * M)
    double *poled = nullptr;
    A(poled, (size_t)M * M)
    float2 *poledf = nullptr;
    A(poledf, (size_t)M * M)
#undef A
    d.eps = eps;
    d.z0 = z0;
    d.epsdiff = epsdiff;
    d.poled = poled;
    d.poledf = poledf;
    d.eigen_dfloat = ctx->mixed ? 1 : 0;
    d.propagator = opt->propagator;
    d.live = (opt->compact_every > 0) ? ctx->live : nullptr;
    d.n_live = ctx->n_live;
    d.traj_base = (uint64_t)opt->traj_base;
    configure_hop_smem();
    configure_cheb_tc();
    configure_cheb_tc16();
    {
        std::vector<float> ed((size_t)M * M);
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) ed[(size_t)a * M + b] = (float)(ctx->eps_h[a] - ctx->eps_h[b]);
        std::vector<double> pd((size_t)M * M);
        std::vector<float2> pf((size_t)M * M);
        for (int k = 0; k < M; ++k)
            for (int o = 0; o < M; ++o) {
                const double v = ctx->eps_h[o] - ctx->eps_h[k];
                const float hi = (float)v;
                pd[(size_t)k * M + o] = v;
                pf[(size_t)k * M + o] = make_float2(hi, (float)(v - (double)hi));
            }
        // on the context stream, after the zero fills of dalloc (a stream created
        // non-blocking is not ordered with the legacy default stream)
        cudaError_t e0 = cudaMemcpyAsync(epsdiff, ed.data(), ed.size() * sizeof(float), cudaMemcpyHostToDevice,
                                         ctx->stream);
        if (e0 == cudaSuccess)
            e0 = cudaMemcpyAsync(poled, pd.data(), pd.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e0 == cudaSuccess)
            e0 = cudaMemcpyAsync(poledf, pf.data(), pf.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream);
        if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(ctx->stream);
        if (e0 != cudaSuccess) {
            *out = ctx;
            return fail(ctx, IESH_ECUDA, "table upload failed: %s", cudaGetErrorString(e0));
        }
    }
    cudaError_t e1 = cudaMemcpyAsync(eps, ctx->eps_h.data(), M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e2 = cudaMemcpyAsync(z0, ctx->z0_h.data(), M * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e3 = cudaStreamSynchronize(ctx->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        *out = ctx;
        return fail(ctx, IESH_ECUDA, "bath upload failed: %s",
                    cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
    }
    *out = ctx;
    return IESH_OK;
}

iesh_status iesh_bath(iesh_ctx *ctx, double *eps, double *z0)
{
    if (!ctx) return IESH_EINVAL;
    if (eps) memcpy(eps, ctx->eps_h.data(), ctx->M * sizeof(double));
    if (z0) memcpy(z0, ctx->z0_h.data(), ctx->M * sizeof(double));
    return IESH_OK;
}

static iesh_status reset_counters(iesh_ctx *ctx, int64_t n)
{
    DevState &d = ctx->ds;
    ctx->steps_since_init = 0;
    CU(launch_live_init(n, ctx->live, ctx->n_live, ctx->stream));
    CU(cudaMemsetAsync(d.status, 0, n * sizeof(uint32_t), ctx->stream));
    CU(cudaMemsetAsync(d.nstep, 0, n * sizeof(int64_t), ctx->stream));
    CU(cudaMemsetAsync(d.hops, 0, n * sizeof(int32_t), ctx->stream));
    CU(cudaMemsetAsync(d.frus, 0, n * sizeof(int32_t), ctx->stream));
    if (d.max_records > 0) {
        CU(cudaMemsetAsync(d.rec_sh, 0, (size_t)n * d.max_records * sizeof(double), ctx->stream));
        CU(cudaMemsetAsync(d.rec_wf, 0, (size_t)n * d.max_records * sizeof(double), ctx->stream));
    }
    return IESH_OK;
}

iesh_status iesh_init_state(iesh_ctx *ctx, int64_t n_traj, const double *x0, const double *p0,
                            const int16_t *occ0, double kT_nuc, double kT_el, uint64_t seed)
{
    if (!ctx) return IESH_EINVAL;
    if (n_traj < 0 || n_traj > ctx->max_traj)
        return fail(ctx, IESH_EINVAL, "n_traj %lld outside 0..%lld", (long long)n_traj, (long long)ctx->max_traj);
    if ((x0 == nullptr) != (p0 == nullptr)) return fail(ctx, IESH_EINVAL, "give both x0 and p0 or neither");
    if (!(kT_nuc >= 0.0) || !(kT_el >= 0.0)) return fail(ctx, IESH_EINVAL, "temperatures must be >= 0");
    DevState &d = ctx->ds;
    d.n = n_traj;
    iesh_status st;
    if ((st = reset_counters(ctx, n_traj)) != IESH_OK) return st;
    if (x0) {
        if ((st = copy_in(ctx, d.x, x0, n_traj * sizeof(double))) != IESH_OK) return st;
        if ((st = copy_in(ctx, d.p, p0, n_traj * sizeof(double))) != IESH_OK) return st;
    } else {
        double omega, xeq;
        int wigner;
        const double *P = ctx->model.par;
        if (ctx->model.kind == IESH_MODEL_HARMONIC) {
            omega = P[0];
            xeq = 0.0;
            wigner = 0;
        } else {  // Morse well: harmonic frequency sqrt(2 De a^2 / m) at x0, Wigner density
            omega = std::sqrt(2.0 * P[0] * P[2] * P[2] / ctx->model.mass);
            xeq = P[1];
            wigner = 1;
        }
        CU(launch_init_nuclear(d, ctx->model.mass, seed, kT_nuc, wigner, omega, xeq, ctx->stream));
    }
    // eigenpairs at x0 (occupations needed only for the force, recomputed below)
    CU(cudaMemsetAsync(d.occ, 0, (size_t)n_traj * ctx->Ne * sizeof(int16_t), ctx->stream));
    CU(launch_eigen(d, ctx->md, 0.0, 0, ctx->stream));
    if (occ0) {
        if ((st = copy_in(ctx, d.occ, occ0, (size_t)n_traj * ctx->Ne * sizeof(int16_t))) != IESH_OK) return st;
    } else {
        CU(launch_sample_occ(d, seed, kT_el, ctx->stream));
    }
    CU(launch_force(d, ctx->stream));
    CU(launch_unit_coeffs(d, ctx->mixed, ctx->stream));
    ctx->have_state = true;
    return IESH_OK;
}

iesh_status iesh_set_state(iesh_ctx *ctx, int64_t n_traj, const double *x, const double *p,
                           const int16_t *occ, const void *C)
{
    if (!ctx) return IESH_EINVAL;
    if (n_traj < 0 || n_traj > ctx->max_traj)
        return fail(ctx, IESH_EINVAL, "n_traj %lld outside 0..%lld", (long long)n_traj, (long long)ctx->max_traj);
    if (!x || !p || !occ || !C) return fail(ctx, IESH_EINVAL, "set_state needs x, p, occ and C");
    DevState &d = ctx->ds;
    d.n = n_traj;
    iesh_status st;
    if ((st = reset_counters(ctx, n_traj)) != IESH_OK) return st;
    const size_t csz = (size_t)n_traj * ctx->Ne * ctx->N * (ctx->mixed ? 8 : 16);
    if ((st = copy_in(ctx, d.x, x, n_traj * sizeof(double))) != IESH_OK) return st;
    if ((st = copy_in(ctx, d.p, p, n_traj * sizeof(double))) != IESH_OK) return st;
    if ((st = copy_in(ctx, d.occ, occ, (size_t)n_traj * ctx->Ne * sizeof(int16_t))) != IESH_OK) return st;
    if ((st = copy_in(ctx, d.C, C, csz)) != IESH_OK) return st;
    CU(launch_eigen(d, ctx->md, 0.0, 0, ctx->stream));
    ctx->have_state = true;
    return IESH_OK;
}

iesh_status iesh_get_state(iesh_ctx *ctx, double *x, double *p, int16_t *occ, void *C,
                           uint32_t *status)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    const int64_t n = d.n;
    bool sync = false;
    iesh_status st;
    if ((st = copy_out(ctx, x, d.x, n * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, p, d.p, n * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, occ, d.occ, (size_t)n * ctx->Ne * sizeof(int16_t), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, C, d.C, (size_t)n * ctx->Ne * ctx->N * (ctx->mixed ? 8 : 16), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, status, d.status, n * sizeof(uint32_t), sync)) != IESH_OK) return st;
    if (sync) CU(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh_get_eigen(iesh_ctx *ctx, double *lam, double *q0, double *force)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    bool sync = false;
    iesh_status st;
    if ((st = copy_out(ctx, lam, d.lam, (size_t)d.n * ctx->N * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, q0, d.q0, (size_t)d.n * ctx->N * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, force, d.F, (size_t)d.n * sizeof(double), sync)) != IESH_OK) return st;
    if (sync) CU(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh_get_counters(iesh_ctx *ctx, int64_t *nstep, int32_t *hops, int32_t *frustrated)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    bool sync = false;
    iesh_status st;
    if ((st = copy_out(ctx, nstep, d.nstep, d.n * sizeof(int64_t), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, hops, d.hops, d.n * sizeof(int32_t), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, frustrated, d.frus, d.n * sizeof(int32_t), sync)) != IESH_OK) return st;
    if (sync) CU(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh_get_records(iesh_ctx *ctx, double *pop_sh, double *pop_wf, int64_t *n_records)
{
    if (!ctx) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    int64_t n0 = 0;
    if (d.n > 0 && d.record_every > 0) {
        CU(cudaMemcpyAsync(&n0, d.nstep, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    const int64_t nr = d.record_every > 0 ? std::min<int64_t>(n0 / d.record_every, d.max_records) : 0;
    if (n_records) *n_records = nr;
    bool sync = false;
    iesh_status st;
    // records are stored [max_records][n] with the batch size at write time
    if ((st = copy_out(ctx, pop_sh, d.rec_sh, (size_t)nr * d.n * sizeof(double), sync)) != IESH_OK) return st;
    if ((st = copy_out(ctx, pop_wf, d.rec_wf, (size_t)nr * d.n * sizeof(double), sync)) != IESH_OK) return st;
    if (sync) CU(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

// Enqueue n_steps steps on stream st (the context's own stream for
// iesh_run, the ensemble's capture stream for iesh_ensemble_create).  With
// compact_on_cadence the work list is compacted every compact_every steps.
// The step kernels on the trajectories of d (the context's whole state, or
// a view of a range of it).
static iesh_status enqueue_steps_on(iesh_ctx *ctx, const DevState &d, double dt, int64_t n_steps, uint64_t seed,
                                    cudaStream_t st, bool compact_on_cadence)
{
    const bool mx = ctx->mixed;
    // Chebyshev truncation: FP64 rounding level, or FP32 level for the mixed path
    const double tol = ctx->opt.prop_tol > 0.0 ? ctx->opt.prop_tol : (mx ? 1e-7 : 1e-15);
    // unitarity check of the coefficient columns after each step
    const double ntol = ctx->opt.norm_tol != 0.0 ? ctx->opt.norm_tol : (mx ? 1e-3 : 1e-8);
    auto tm = [&](int cls, auto fn) { return ctx->timer.run(st, cls, fn); };
    for (int64_t k = 0; k < n_steps; ++k) {
        CU(tm(IESH_K_EIGEN, [&] { return launch_eigen(d, ctx->md, dt, 1, st); }));
        if (d.propagator == IESH_PROP_OVERLAP) {
            CU(tm(IESH_K_PROPAGATE, [&] { return launch_overlap(d, dt, st); }));
        } else {
            CU(tm(IESH_K_COUPLING, [&] { return launch_coupling(d, dt, ctx->model.mass, tol, mx, st); }));
            CU(tm(IESH_K_PROPAGATE, [&] { return launch_cheb(d, dt, mx, st); }));
        }
        CU(tm(IESH_K_HOP, [&] {
            return launch_hop(d, dt, ctx->model.mass, seed, ctx->opt.skip_bound, nullptr, st, mx);
        }));
        if (ntol > 0.0) CU(tm(IESH_K_OTHER, [&] { return launch_norm_check(d, mx, ntol, st); }));
        if (!compact_on_cadence) continue;
        ++ctx->steps_since_init;
        if (ctx->opt.compact_every > 0 && ctx->steps_since_init % ctx->opt.compact_every == 0)
            CU(tm(IESH_K_OTHER, [&] { return launch_compact(d, ctx->live, ctx->n_live, st); }));
    }
    return IESH_OK;
}

static iesh_status enqueue_steps(iesh_ctx *ctx, double dt, int64_t n_steps, uint64_t seed, cudaStream_t st,
                                 bool compact_on_cadence)
{
    return enqueue_steps_on(ctx, ctx->ds, dt, n_steps, seed, st, compact_on_cadence);
}

// View of trajectories [t0, t0 + cnt) of the context's state: every
// per-trajectory array offset by t0 rows, the Philox id base by t0.  The step
// kernels treat trajectories independently, so a range gives the same bits
// as the whole batch.  Records ([max_records][n]) and the work list are not
// trajectory-major: callers require both off.
static DevState state_view(const DevState &d, int64_t t0, int64_t cnt, size_t c_bytes)
{
    DevState v = d;
    const int64_t N = d.N, Ne = d.Ne;
    auto off = [&](auto *&ptr, int64_t per) {
        if (ptr) ptr += t0 * per;
    };
    off(v.x, 1), off(v.p, 1), off(v.F, 1), off(v.dU0, 1), off(v.vprev, 1);
    off(v.occ, Ne);
    if (v.C) v.C = static_cast<char *>(v.C) + t0 * Ne * N * (int64_t)c_bytes;
    off(v.lam, N), off(v.q0, N), off(v.lam_prev, N), off(v.q0_prev, N);
    off(v.geo, 4), off(v.geo_prev, 4);
    off(v.status, 1), off(v.nstep, 1), off(v.hops, 1), off(v.frus, 1);
    off(v.scratch, d.scratch_stride);
    off(v.cheb, kChebStride);
    off(v.defl, defl_stride(d.N, d.Ne));
    off(v.rt, N), off(v.rt_prev, N), off(v.ro, N), off(v.ro_prev, N);
    off(v.fx, 1), off(v.fx_prev, 1);
    off(v.q2, N), off(v.q2_prev, N), off(v.geo2, 8), off(v.x_prev, 6), off(v.hop_pair, 1);
    v.n = cnt;
    v.traj_base = d.traj_base + (uint64_t)t0;
    return v;
}

iesh_status iesh_run(iesh_ctx *ctx, double dt, int64_t n_steps, uint64_t seed)
{
    if (!ctx) return IESH_EINVAL;
    if (!ctx->have_state) return fail(ctx, IESH_ESTATE, "run before init_state/set_state");
    if (!(dt > 0.0) || n_steps < 0) return fail(ctx, IESH_EINVAL, "need dt > 0 and n_steps >= 0");
    return enqueue_steps(ctx, dt, n_steps, seed, ctx->stream, true);
}

iesh_status iesh_get_live(iesh_ctx *ctx, int64_t *n_live)
{
    if (!ctx || !n_live) return IESH_EINVAL;
    if (ctx->opt.compact_every <= 0) {
        *n_live = ctx->ds.n;
        return IESH_OK;
    }
    int32_t v = 0;
    CU(cudaMemcpyAsync(&v, ctx->n_live, sizeof v, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *n_live = v;
    return IESH_OK;
}

iesh_status iesh_set_kernel_shape(iesh_ctx *ctx, int cheb_ept, int cheb_G, int hop_threads)
{
    if (!ctx) return IESH_EINVAL;
    if (ctx->opt.precision == IESH_PREC_MIXED) {
        const bool simt = (cheb_ept == 4 && cheb32_shape_ok(ctx->N, cheb_G, 1)) ||
                          (cheb_ept == 32 && cheb32_shape_ok(ctx->N, cheb_G, 2));
        const bool tc = (cheb_ept == 8 && cheb_G == 1 && cheb_tc_eligible(ctx->N, ctx->Ne)) ||
                        (cheb_ept == 16 && cheb_G == 1 && cheb_tc16_eligible(ctx->N, ctx->Ne));
        if (!((cheb_ept == 0 && cheb_G == 0) || simt || tc))
            return fail(ctx, IESH_EINVAL,
                        "mixed propagator shape (%d, %d) invalid for N=%d, Ne=%d (need ept 4 with "
                        "G*ceil(N/4) <= 256, ept 32 with G*ceil(ceil(N/4)/2) <= 256, each within its "
                        "shared-memory cap, or ept 8, G 1 for the tensor-core kernel: N <= 128, Ne <= 56)",
                        cheb_ept, cheb_G, ctx->N, ctx->Ne);
    } else if (cheb_ept < 0 || cheb_ept > 2 || cheb_G < 0 || (cheb_ept > 0) != (cheb_G > 0) ||
               cheb_G * ctx->N > 1024) {
        return fail(ctx, IESH_EINVAL, "propagator shape (%d, %d) invalid for N=%d", cheb_ept, cheb_G, ctx->N);
    }
    if (hop_threads != 0 && hop_threads != 256 && hop_threads != 512)
        return fail(ctx, IESH_EINVAL, "hop_threads must be 0, 256 or 512");
    ctx->ds.cheb_ept = cheb_ept;
    ctx->ds.cheb_G = cheb_G;
    ctx->ds.hop_threads = hop_threads;
    return IESH_OK;
}

iesh_status iesh_get_kernel_shape(iesh_ctx *ctx, int *cheb_ept, int *cheb_G, int *hop_threads)
{
    if (!ctx) return IESH_EINVAL;
    int e = ctx->ds.cheb_ept, g = ctx->ds.cheb_G;
    if (e == 0) {
        if (ctx->opt.precision == IESH_PREC_MIXED && cheb_tc16_eligible(ctx->N, ctx->Ne)) {
            e = 16;
            g = 1;
        } else if (ctx->opt.precision == IESH_PREC_MIXED && cheb_tc_eligible(ctx->N, ctx->Ne)) {
            e = 8;
            g = 1;
        } else if (ctx->opt.precision == IESH_PREC_MIXED) {
            const int qpt = ctx->N > kCheb32WideMinN ? 2 : 1;
            e = qpt == 2 ? 32 : 4;
            cheb32_shape(ctx->N, ctx->Ne, g, qpt);
        } else {
            cheb_shape(ctx->N, ctx->Ne, e, g);
        }
    }
    if (cheb_ept) *cheb_ept = e;
    if (cheb_G) *cheb_G = g;
    if (hop_threads) *hop_threads = ctx->ds.hop_threads;
    return IESH_OK;
}

iesh_status iesh_get_propagator_terms(iesh_ctx *ctx, int32_t *K)
{
    if (!ctx || !K) return IESH_EINVAL;
    const DevState &d = ctx->ds;
    std::vector<double> tmp((size_t)d.n);
    if (d.n > 0) {
        CU(cudaMemcpy2DAsync(tmp.data(), sizeof(double), d.cheb + 2, kChebStride * sizeof(double),
                             sizeof(double), (size_t)d.n, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    std::vector<int32_t> k32((size_t)d.n);
    for (int64_t i = 0; i < d.n; ++i) k32[i] = (int32_t)tmp[i];
    bool sync = false;
    iesh_status st;
    if ((st = copy_out(ctx, K, k32.data(), k32.size() * sizeof(int32_t), sync)) != IESH_OK) return st;
    if (sync) CU(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh_profile(iesh_ctx *ctx, int enable)
{
    if (!ctx) return IESH_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->timer.reset(enable != 0);
    return IESH_OK;
}

iesh_status iesh_profile_read(iesh_ctx *ctx, double *ms, int64_t *launches)
{
    if (!ctx) return IESH_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    CU(ctx->timer.fold());
    for (int i = 0; i < IESH_K_COUNT; ++i) {
        if (ms) ms[i] = ctx->timer.ms[i];
        if (launches) launches[i] = ctx->timer.n[i];
    }
    return IESH_OK;
}

iesh_status iesh_hop_probabilities(iesh_ctx *ctx, double dt, double *g)
{
    if (!ctx || !g) return IESH_EINVAL;
    if (!ctx->have_state) return fail(ctx, IESH_ESTATE, "hop_probabilities before a state exists");
    const DevState &d = ctx->ds;
    const size_t bytes = (size_t)d.n * ctx->Ne * ctx->N * sizeof(double);
    double *dst = g;
    bool host = is_host_ptr(g);
    double *tmp = nullptr;
    if (host) {
        CU(cudaMallocAsync((void **)&tmp, bytes, ctx->stream));
        dst = tmp;
    }
    CU(launch_hop(d, dt, ctx->model.mass, 0, 0, dst, ctx->stream, ctx->mixed));
    if (host) {
        CU(cudaMemcpyAsync(g, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaFreeAsync(tmp, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return IESH_OK;
}

// ------------------------------------------------------------ checkpoint
// Blob layout: a 64-byte header, then every per-trajectory array of the
// first n trajectories in a fixed order, each section padded to 16 bytes,
// then the population records [max_records][n].
namespace {
struct CkptHeader {
    char magic[8];
    int32_t N, Ne, mixed, propagator;
    int64_t n, max_records, record_every, steps_since_init;
};
static_assert(sizeof(CkptHeader) <= 64, "checkpoint header");
constexpr size_t kCkptHeader = 64;
constexpr char kCkptMagic[8] = {'I', 'E', 'S', 'H', 'C', 'K', 'P', '1'};

struct Section {
    void *dev;
    size_t bytes;
};

std::vector<Section> ckpt_sections(iesh_ctx *ctx, int64_t n)
{
    DevState &d = ctx->ds;
    const size_t N = ctx->N, Ne = ctx->Ne, T = (size_t)n;
    const size_t cb = ctx->mixed ? 8 : 16;
    std::vector<Section> v = {
        {d.x, 8 * T}, {d.p, 8 * T}, {d.F, 8 * T}, {d.dU0, 8 * T}, {d.vprev, 8 * T},
        {d.occ, 2 * T * Ne}, {d.C, cb * T * Ne * N},
        {d.lam, 8 * T * N}, {d.q0, 8 * T * N}, {d.lam_prev, 8 * T * N}, {d.q0_prev, 8 * T * N},
        {d.geo, 32 * T}, {d.geo_prev, 32 * T},
        {d.rt, 8 * T * N}, {d.rt_prev, 8 * T * N}, {d.ro, 4 * T * N}, {d.ro_prev, 4 * T * N},
        {d.fx, 8 * T}, {d.fx_prev, 8 * T},
        {d.status, 4 * T}, {d.nstep, 8 * T}, {d.hops, 4 * T}, {d.frus, 4 * T},
        {d.cheb, 8 * T * kChebStride},
    };
    if (d.max_records > 0) {
        v.push_back({d.rec_sh, 8 * T * d.max_records});
        v.push_back({d.rec_wf, 8 * T * d.max_records});
    }
    return v;
}

size_t ckpt_bytes(iesh_ctx *ctx, int64_t n)
{
    size_t b = kCkptHeader;
    for (auto &s : ckpt_sections(ctx, n)) b += (s.bytes + 15) & ~(size_t)15;
    return b;
}
}  // namespace

iesh_status iesh_checkpoint_bytes(iesh_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return IESH_EINVAL;
    *bytes = ckpt_bytes(ctx, ctx->ds.n);
    return IESH_OK;
}

iesh_status iesh_checkpoint_save(iesh_ctx *ctx, void *buf, size_t bytes)
{
    if (!ctx || !buf) return IESH_EINVAL;
    if (!ctx->have_state) return fail(ctx, IESH_ESTATE, "checkpoint_save before a state exists");
    const int64_t n = ctx->ds.n;
    const size_t need = ckpt_bytes(ctx, n);
    if (bytes < need) return fail(ctx, IESH_EINVAL, "checkpoint needs %zu bytes, got %zu", need, bytes);
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kCkptMagic, 8);
    h.N = ctx->N;
    h.Ne = ctx->Ne;
    h.mixed = ctx->mixed ? 1 : 0;
    h.propagator = ctx->opt.propagator;
    h.n = n;
    h.max_records = ctx->ds.max_records;
    h.record_every = ctx->ds.record_every;
    h.steps_since_init = ctx->steps_since_init;
    char *out = (char *)buf;
    CU(cudaMemcpyAsync(out, &h, sizeof h, cudaMemcpyDefault, ctx->stream));
    size_t off = kCkptHeader;
    for (auto &s : ckpt_sections(ctx, n)) {
        if (s.bytes) CU(cudaMemcpyAsync(out + off, s.dev, s.bytes, cudaMemcpyDefault, ctx->stream));
        off += (s.bytes + 15) & ~(size_t)15;
    }
    CU(cudaStreamSynchronize(ctx->stream));  // the header copy reads a stack variable
    return IESH_OK;
}

iesh_status iesh_checkpoint_load(iesh_ctx *ctx, const void *buf, size_t bytes)
{
    if (!ctx || !buf) return IESH_EINVAL;
    if (bytes < kCkptHeader) return fail(ctx, IESH_EINVAL, "checkpoint shorter than its header");
    CkptHeader h;
    CU(cudaMemcpyAsync(&h, buf, sizeof h, cudaMemcpyDefault, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (memcmp(h.magic, kCkptMagic, 8) != 0) return fail(ctx, IESH_EINVAL, "not an IESH checkpoint");
    if (h.N != ctx->N || h.Ne != ctx->Ne || h.mixed != (ctx->mixed ? 1 : 0) ||
        h.propagator != ctx->opt.propagator || h.max_records != ctx->ds.max_records ||
        h.record_every != ctx->ds.record_every)
        return fail(ctx, IESH_EINVAL,
                    "checkpoint of N=%d, Ne=%d, mixed=%d, propagator=%d, records %lld/%lld does "
                    "not match this context", h.N, h.Ne, h.mixed, h.propagator,
                    (long long)h.max_records, (long long)h.record_every);
    if (h.n < 0 || h.n > ctx->max_traj)
        return fail(ctx, IESH_EINVAL, "checkpoint holds %lld trajectories, context at most %lld",
                    (long long)h.n, (long long)ctx->max_traj);
    if (bytes < ckpt_bytes(ctx, h.n)) return fail(ctx, IESH_EINVAL, "checkpoint truncated");
    DevState &d = ctx->ds;
    d.n = h.n;
    const char *in = (const char *)buf;
    size_t off = kCkptHeader;
    for (auto &s : ckpt_sections(ctx, h.n)) {
        if (s.bytes) CU(cudaMemcpyAsync(s.dev, in + off, s.bytes, cudaMemcpyDefault, ctx->stream));
        off += (s.bytes + 15) & ~(size_t)15;
    }
    ctx->steps_since_init = h.steps_since_init;
    // the work list is rebuilt from the restored status words (the list's
    // order never changes results)
    CU(launch_live_init(h.n, ctx->live, ctx->n_live, ctx->stream));
    if (ctx->opt.compact_every > 0) CU(launch_compact(d, ctx->live, ctx->n_live, ctx->stream));
    if (is_host_ptr(buf)) CU(cudaStreamSynchronize(ctx->stream));
    ctx->have_state = true;
    return IESH_OK;
}

iesh_status iesh_run_host(iesh_ctx *ctx, const void *in, void *out, size_t bytes, double dt, int64_t n_steps,
                          uint64_t seed, int chunks)
{
    if (!ctx || !in || !out) return IESH_EINVAL;
    if (!(dt > 0.0) || n_steps < 0) return fail(ctx, IESH_EINVAL, "need dt > 0 and n_steps >= 0");
    if (!is_host_ptr(in) || !is_host_ptr(out)) return fail(ctx, IESH_EINVAL, "run_host needs host buffers");
    if (ctx->ds.max_records > 0 || ctx->opt.compact_every > 0)
        return fail(ctx, IESH_EUNSUPPORTED, "run_host needs records and the work list off");
    if (bytes < kCkptHeader) return fail(ctx, IESH_EINVAL, "checkpoint shorter than its header");
    CkptHeader h;
    memcpy(&h, in, sizeof h);  // host memory
    if (memcmp(h.magic, kCkptMagic, 8) != 0) return fail(ctx, IESH_EINVAL, "not an IESH checkpoint");
    if (h.N != ctx->N || h.Ne != ctx->Ne || h.mixed != (ctx->mixed ? 1 : 0) ||
        h.propagator != ctx->opt.propagator || h.max_records != 0 || h.record_every != ctx->ds.record_every)
        return fail(ctx, IESH_EINVAL, "checkpoint of N=%d, Ne=%d, mixed=%d, propagator=%d does not match this context",
                    h.N, h.Ne, h.mixed, h.propagator);
    const int64_t n = h.n;
    if (n < 0 || n > ctx->max_traj)
        return fail(ctx, IESH_EINVAL, "checkpoint holds %lld trajectories, context at most %lld", (long long)n,
                    (long long)ctx->max_traj);
    if (bytes < ckpt_bytes(ctx, n)) return fail(ctx, IESH_EINVAL, "checkpoint truncated");
    const int nc = (int)std::max<int64_t>(1, std::min<int64_t>(chunks > 0 ? chunks : 4, std::max<int64_t>(n, 1)));
    if (!ctx->s_in) CU(cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking));
    if (!ctx->s_out) CU(cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
    while ((int)ctx->ev.size() < 2 * nc + 2) {
        cudaEvent_t e;
        CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->ev.push_back(e);
    }
    cudaEvent_t *ev_in = ctx->ev.data(), *ev_run = ev_in + nc, ev_start = ev_in[2 * nc], ev_end = ev_in[2 * nc + 1];
    DevState &d = ctx->ds;
    d.n = n;
    // section layout of the blob; every section is linear in the batch size
    const std::vector<Section> all = ckpt_sections(ctx, n), per = ckpt_sections(ctx, 1);
    std::vector<size_t> base(all.size());
    size_t off = kCkptHeader;
    for (size_t k = 0; k < all.size(); ++k) {
        base[k] = off;
        off += (all[k].bytes + 15) & ~(size_t)15;
    }
    const char *src = static_cast<const char *>(in);
    char *dst = static_cast<char *>(out);
    // the copies in wait for work already queued on the context's stream
    CU(cudaEventRecord(ev_start, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->s_in, ev_start, 0));
    const size_t cb = ctx->mixed ? 8 : 16;
    auto range = [&](int c, int64_t &t0, int64_t &t1) {
        t0 = n * c / nc;
        t1 = n * (c + 1) / nc;
    };
    for (int c = 0; c < nc; ++c) {
        int64_t t0, t1;
        range(c, t0, t1);
        for (size_t k = 0; k < all.size(); ++k) {
            const size_t b = per[k].bytes, len = b * (size_t)(t1 - t0);
            if (len)
                CU(cudaMemcpyAsync(static_cast<char *>(all[k].dev) + b * t0, src + base[k] + b * t0, len,
                                   cudaMemcpyHostToDevice, ctx->s_in));
        }
        CU(cudaEventRecord(ev_in[c], ctx->s_in));
    }
    for (int c = 0; c < nc; ++c) {
        int64_t t0, t1;
        range(c, t0, t1);
        CU(cudaStreamWaitEvent(ctx->stream, ev_in[c], 0));
        if (t1 > t0) {
            const DevState v = state_view(d, t0, t1 - t0, cb);
            iesh_status st = enqueue_steps_on(ctx, v, dt, n_steps, seed, ctx->stream, false);
            if (st != IESH_OK) return st;
        }
        CU(cudaEventRecord(ev_run[c], ctx->stream));
        CU(cudaStreamWaitEvent(ctx->s_out, ev_run[c], 0));
        for (size_t k = 0; k < all.size(); ++k) {
            const size_t b = per[k].bytes, len = b * (size_t)(t1 - t0);
            if (len)
                CU(cudaMemcpyAsync(dst + base[k] + b * t0, static_cast<char *>(all[k].dev) + b * t0, len,
                                   cudaMemcpyDeviceToHost, ctx->s_out));
        }
    }
    // later work on the context's stream follows the copies out
    CU(cudaEventRecord(ev_end, ctx->s_out));
    CU(cudaStreamWaitEvent(ctx->stream, ev_end, 0));
    CU(cudaStreamSynchronize(ctx->s_out));
    ctx->steps_since_init = h.steps_since_init + n_steps;
    h.steps_since_init = ctx->steps_since_init;
    memcpy(dst, &h, sizeof h);  // after the copies: out may be in
    ctx->have_state = true;
    return IESH_OK;
}

iesh_status iesh_observables(iesh_ctx *ctx, double *ke, double *epot, double *pop_sh, double *pop_wf)
{
    if (!ctx) return IESH_EINVAL;
    if (!ctx->have_state) return fail(ctx, IESH_ESTATE, "observables before a state exists");
    const DevState &d = ctx->ds;
    const int64_t n = d.n;
    CU(launch_observables(d, ctx->mixed, ctx->model.mass, ctx->obs, ctx->stream));
    bool sync = false;
    iesh_status st;
    double *outs[4] = {ke, epot, pop_sh, pop_wf};
    for (int k = 0; k < 4; ++k)
        if ((st = copy_out(ctx, outs[k], ctx->obs + k * n, n * sizeof(double), sync)) != IESH_OK) return st;
    if (sync) CU(cudaStreamSynchronize(ctx->stream));
    return IESH_OK;
}

iesh_status iesh_check(iesh_ctx *ctx, uint32_t *bits)
{
    if (!ctx) return IESH_EINVAL;
    uint32_t h[9] = {0};
    if (ctx->have_state) {
        CU(launch_status_summary(ctx->ds.status, ctx->ds.n, ctx->summary, ctx->stream));
        CU(cudaMemcpyAsync(h, ctx->summary, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    if (bits) memcpy(bits, h, sizeof h);
    if (h[0] & IESH_TRAJ_NAN) return IESH_ENAN;
    if (h[0] & IESH_TRAJ_SECULAR_NONCONV) return IESH_ENONCONV;
    if (h[0] & IESH_TRAJ_SINGULAR) return IESH_ESINGULAR;
    if (h[0] & IESH_TRAJ_NORM_DRIFT) return IESH_ENORM;
    return IESH_OK;
}

// ------------------------------------------------------------- ensemble
const char *iesh_ensemble_last_error(const iesh_ensemble *ens)
{
    return ens ? ens->err.c_str() : "null ensemble";
}

iesh_status iesh_ensemble_destroy(iesh_ensemble *ens)
{
    if (!ens) return IESH_OK;
    if (ens->stream) cudaStreamSynchronize(ens->stream);
    if (ens->capture) cudaStreamSynchronize(ens->capture);
    if (ens->exec) cudaGraphExecDestroy(ens->exec);
    if (ens->graph) cudaGraphDestroy(ens->graph);
    if (ens->n_live_dev) cudaFree(ens->n_live_dev);
    if (ens->counters) cudaFree(ens->counters);
    if (ens->ev) cudaEventDestroy(ens->ev);
    if (ens->capture) cudaStreamDestroy(ens->capture);
    delete ens;
    return IESH_OK;
}

iesh_status iesh_ensemble_create(iesh_ensemble **out, iesh_ctx *const *ctxs, int n_ctx, double dt,
                                 int64_t chunk, uint64_t seed, void *cuda_stream)
{
    if (!out) return IESH_EINVAL;
    *out = nullptr;
    iesh_ensemble *ens = new iesh_ensemble();
    *out = ens;
    ens->stream = (cudaStream_t)cuda_stream;
    ens->chunk = chunk;
    if (!ctxs || n_ctx < 1) return efail(ens, IESH_EINVAL, "need at least one context");
    if (!(dt > 0.0) || chunk < 1) return efail(ens, IESH_EINVAL, "need dt > 0 and chunk >= 1");
    for (int c = 0; c < n_ctx; ++c) {
        iesh_ctx *ctx = ctxs[c];
        if (!ctx) return efail(ens, IESH_EINVAL, "context %d is NULL", c);
        if (!ctx->have_state) return efail(ens, IESH_ESTATE, "context %d has no state", c);
        if (ctx->opt.compact_every <= 0)
            return efail(ens, IESH_EINVAL, "context %d has no work list (compact_every = 0)", c);
        if (ctx->timer.on) return efail(ens, IESH_ESTATE, "context %d has profiling on", c);
        ens->ctxs.push_back(ctx);
    }
    CUE(cudaStreamCreateWithFlags(&ens->capture, cudaStreamNonBlocking));
    CUE(cudaEventCreateWithFlags(&ens->ev, cudaEventDisableTiming));
    CUE(cudaMalloc((void **)&ens->n_live_dev, n_ctx * sizeof(int32_t *)));
    CUE(cudaMalloc((void **)&ens->counters, 3 * sizeof(int64_t)));
    std::vector<const int32_t *> nl;
    for (auto *ctx : ens->ctxs) nl.push_back(ctx->n_live);
    CUE(cudaMemcpy(ens->n_live_dev, nl.data(), n_ctx * sizeof(int32_t *), cudaMemcpyHostToDevice));
    CUE(cudaMemset(ens->counters, 0, 3 * sizeof(int64_t)));
    // graph: one while node; its body advances every context by `chunk`
    // steps, compacts every work list and sets the loop condition
    CUE(cudaGraphCreate(&ens->graph, 0));
    cudaGraphConditionalHandle h;
    CUE(cudaGraphConditionalHandleCreate(&h, ens->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CUE(cudaGraphAddNode(&node, ens->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CUE(cudaStreamBeginCaptureToGraph(ens->capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    for (auto *ctx : ens->ctxs) {
        iesh_status st = enqueue_steps(ctx, dt, chunk, seed, ens->capture, false);
        if (st == IESH_OK) {
            cudaError_t e = launch_compact(ctx->ds, ctx->live, ctx->n_live, ens->capture);
            if (e != cudaSuccess) st = fail(ctx, IESH_ECUDA, "launch_compact: %s", cudaGetErrorString(e));
        }
        if (st != IESH_OK) {
            cudaGraph_t g;
            cudaStreamEndCapture(ens->capture, &g);
            return efail(ens, st, "capturing a context's steps: %s", ctx->err.c_str());
        }
    }
    k_ensemble_cond<<<1, 32, 0, ens->capture>>>(h, ens->n_live_dev, n_ctx, ens->counters, ens->counters + 1,
                                                chunk, ens->counters + 2);
    CUE(cudaGetLastError());
    CUE(cudaStreamEndCapture(ens->capture, &body));
    CUE(cudaGraphInstantiate(&ens->exec, ens->graph, 0));
    return IESH_OK;
}

iesh_status iesh_ensemble_run(iesh_ensemble *ens, int64_t max_steps)
{
    if (!ens || !ens->exec) return IESH_EINVAL;
    if (max_steps < 1) return efail(ens, IESH_EINVAL, "max_steps must be >= 1");
    // the contexts' earlier work (set-up, copies) comes first
    for (auto *ctx : ens->ctxs) {
        CUE(cudaEventRecord(ens->ev, ctx->stream));
        CUE(cudaStreamWaitEvent(ens->stream, ens->ev, 0));
    }
    // step cap counted from the device loop's own step counter
    int64_t now = 0;
    CUE(cudaMemcpyAsync(&now, ens->counters, sizeof now, cudaMemcpyDeviceToHost, ens->stream));
    CUE(cudaStreamSynchronize(ens->stream));
    const int64_t cap = now + max_steps;
    CUE(cudaMemcpyAsync(ens->counters + 1, &cap, sizeof cap, cudaMemcpyHostToDevice, ens->stream));
    CUE(cudaStreamSynchronize(ens->stream));  // the copy reads a host stack variable
    CUE(cudaGraphLaunch(ens->exec, ens->stream));
    // later calls on the contexts come after the loop
    CUE(cudaEventRecord(ens->ev, ens->stream));
    for (auto *ctx : ens->ctxs) {
        CUE(cudaStreamWaitEvent(ctx->stream, ens->ev, 0));
        ctx->steps_since_init = 0;  // the loop compacts at the end of every chunk
    }
    return IESH_OK;
}

iesh_status iesh_ensemble_status(iesh_ensemble *ens, int64_t *steps_done, int64_t *live)
{
    if (!ens) return IESH_EINVAL;
    int64_t h[3] = {0, 0, 0};
    CUE(cudaMemcpyAsync(h, ens->counters, sizeof h, cudaMemcpyDeviceToHost, ens->stream));
    CUE(cudaStreamSynchronize(ens->stream));
    if (steps_done) *steps_done = h[0];
    if (live) *live = h[2];
    return IESH_OK;
}

}  // extern "C"
