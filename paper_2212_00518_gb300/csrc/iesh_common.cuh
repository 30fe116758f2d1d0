// iesh_common.cuh -- device-side state layout and helpers of the batched IESH
// library (sm_103a).  Internal to the library; the public C-ABI is iesh.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace iesh {

constexpr int kMaxOrbitals = 256;   // N = M + 1 limit of the step kernels
constexpr int kMaxHopElectrons = 112; // Ne limit of the in-shared-memory overlap inverse
constexpr int kChebMax = 128;       // Chebyshev terms available per step
constexpr int kChebStride = kChebMax + 8; // per-trajectory propagator record

enum : uint32_t {
    ST_SECULAR = 0x1u,
    ST_SINGULAR = 0x2u,
    ST_NAN = 0x4u,
    ST_DONE = 0x8u,
    ST_PROP = 0x10u,
    ST_TC_WAIT = 0x20u,
    ST_NORM = 0x40u,
};

// Model constants passed by value to every kernel.
struct ModelDev {
    int kind;        // 0 harmonic, 1 desorption, 2 Morse + image
    double mass;
    double par[16];
};

// Device pointers of a context's state (structure of arrays).
// Deflation record per trajectory, defl_stride doubles: [0] flag, [1] mu,
// [2] cos mu, [3] sin mu; from kDeflHead the eigenvector u (Re u[N], Im
// u[N]) and a = u^H c (Re a[Ne], Im a[Ne]), as doubles in FP64 contexts and
// as packed floats in mixed ones.
constexpr int kDeflHead = 4;
__host__ __device__ constexpr int64_t defl_stride(int N, int Ne)
{
    return kDeflHead + 2 * (int64_t)N + 2 * (int64_t)Ne;
}

struct DevState {
    int N, M, Ne;
    int64_t n;                 // trajectories in the batch
    double *x, *p, *F, *dU0, *vprev;
    int16_t *occ;              // [n][Ne] ascending
    void *C;                   // [n][Ne][N] double2 or float2
    double *lam, *q0;          // [n][N] at the current position
    double *lam_prev, *q0_prev;// [n][N] at the previous position
    double *geo, *geo_prev;    // [n][4]: h, dh/dx, kappa = f'/f, U0
    uint32_t *status;          // [n]
    int64_t *nstep;            // [n] steps taken (Philox counter)
    int32_t *hops, *frus;      // [n]
    double *scratch;           // [n][scratch_stride] per-trajectory workspace
    int64_t scratch_stride;    // doubles per trajectory
    double *cheb;              // [n][kChebStride]: c, rho, K, J_0..J_K
    // [n][defl_stride(N, Ne)] per trajectory when the propagator deflates the
    // isolated top level of the generator (null: never): a flag, its
    // eigenvalue mu, its eigenvector u (Re u[N], Im u[N]) and the components
    // a = u^H c of the electrons (Re a[Ne], Im a[Ne])
    double *defl;
    double *rec_sh, *rec_wf;   // [max_records][n]
    int record_every, max_records;
    double z_done;
    const double *eps, *z0;    // bath [M]: energies and sqrt(Gamma/2pi) sqrt(w_k)
    const float *epsdiff;      // [M][M] eps_a - eps_b rounded to FP32 (mixed path)
    const double *poled;       // [M][M] poled[k M + o] = eps_o - eps_k (secular sums)
    const float2 *poledf;      // [M][M] the same as double-float pairs (hi, lo)
    int eigen_dfloat;          // 1: secular sums in double-float (mixed path)
    // root offsets from their origin poles (lam_i = eps[ro_i] + rt_i, rt_i
    // unrounded) and the coupling factor f(x), at this and the previous step
    double *rt, *rt_prev;      // [n][N]
    int32_t *ro, *ro_prev;     // [n][N]
    double *fx, *fx_prev;      // [n]
    int propagator;            // 0 Chebyshev of the averaged generator, 1 overlap
    // work list: when live != nullptr the step kernels visit trajectory
    // live[w] for work item w < *n_live (compacted on the device)
    const int32_t *live;
    const int32_t *n_live;
    // kernel shapes (0 = built-in choice): propagator electrons per thread
    // and column groups per CTA, threads of the hop kernel
    int cheb_ept, cheb_G, hop_threads;
    // two adsorbate orbitals over six nuclear coordinates: x, p, F and vprev
    // are [n][6]; q0 holds the components Q_0j on orbital 0 and q2 the
    // components Q_1j on orbital 1; geo2 [n][8] holds h_0, h_1 and, with the
    // velocity after the second half kick, grad h_a . v and grad log f_a . v
    double *q2, *q2_prev;      // [n][N]
    double *geo2;              // [n][8]
    double *x_prev;            // [n][6] start of the step
    int32_t *hop_pair;         // [n] a N + m of the selected hop, or -1
    // global id of trajectory 0 in the Philox counters (trajectory t draws
    // with id traj_base + t), so that a batch split over several contexts
    // or devices reproduces the undivided batch
    uint64_t traj_base;
};

// 16-byte asynchronous copy global -> shared, cached in L2 only (both
// addresses 16-byte aligned); completion by commit groups.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}
// The same with src_bytes (0 or 16) read and the rest zero-filled.
__device__ __forceinline__ void cp_async16_zfill(void *smem_dst, const void *gsrc, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most `Pending` of this thread's committed groups are in flight.
template <int Pending>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(Pending) : "memory");
}

// Smallest power of two >= n (width of the fixed-order tree reductions).
__host__ __device__ inline int eigen_pow2(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Trajectory visited by work item w, or -1 when w is past the batch or the
// live count.
__device__ __forceinline__ int64_t traj_of(const DevState &s, int64_t w)
{
    if (s.live) return (w < (int64_t)*s.n_live) ? (int64_t)s.live[w] : -1;
    return (w < s.n) ? w : -1;
}

// ---------------------------------------------------------------- models
// U0, dU0/dx, h = U1 - U0, dh/dx, coupling factor f and df/dx at x.
struct ModelVals {
    double U0, dU0, h, dh, f, df;
};

__device__ __forceinline__ ModelVals model_eval(const ModelDev &md, double x)
{
    ModelVals o;
    const double *P = md.par;
    if (md.kind == 0) {
        const double mw2 = md.mass * P[0] * P[0];
        o.U0 = 0.5 * mw2 * x * x;
        o.dU0 = mw2 * x;
        // U1 - U0 = m w^2 (g^2 - 2 g x) / 2 + dG
        o.h = 0.5 * mw2 * (P[1] * P[1] - 2.0 * P[1] * x) + P[2];
        o.dh = -mw2 * P[1];
        o.f = 1.0;
        o.df = 0.0;
    } else if (md.kind == 1) {
        const double De = P[0], x0 = P[1], a = P[2], c = P[3], D1 = P[4], D2 = P[5], ap = P[6],
                     Vinf = P[7], q = P[8], at = P[9], xt = P[10];
        const double e = exp(-a * (x - x0));
        o.U0 = De * (e - 1.0) * (e - 1.0) + c;
        o.dU0 = -2.0 * a * De * (e - 1.0) * e;
        const double e1 = exp(-ap * (x - x0));
        const double U1 = D1 * e1 * e1 - D2 * e1 + Vinf;
        const double dU1 = ap * (D2 * e1 - 2.0 * D1 * e1 * e1);
        o.h = U1 - o.U0;
        o.dh = dU1 - o.dU0;
        const double th = tanh((x - xt) / at);
        o.f = 0.5 * (1.0 - q) * (1.0 - th) + q;
        o.df = -0.5 * (1.0 - q) * (1.0 - th * th) / at;
    } else {
        const double De = P[0], x0 = P[1], a = P[2], c = P[3], hinf = P[4], zim = P[5],
                     ac = P[6], zc = P[7], sg = P[8];
        const double e = exp(-a * (x - x0));
        o.U0 = De * (e - 1.0) * (e - 1.0) + c;
        o.dU0 = -2.0 * a * De * (e - 1.0) * e;
        const double dz = x - zim;
        const double r = sqrt(dz * dz + ac * ac);
        o.h = hinf - 0.25 / r;
        o.dh = 0.25 * dz / (r * r * r);
        const double u = (x - zc) / sg;
        o.f = exp(-0.5 * u * u);
        o.df = -(u / sg) * o.f;
    }
    return o;
}

// ------------------------------------------------------ counter-based RNG
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, each two 32x32 -> 64-bit
// products mixed with the key; the key advances by the Weyl constants.
struct U4 {
    uint32_t v[4];
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    U4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// 53-bit uniform in [0, 1) from two words.
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo)
{
    return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

// Streams of the counter layout (trajectory, stream, n_lo, n_hi).
constexpr uint32_t kStreamHop = 0, kStreamNuc = 1, kStreamElec = 2;

__device__ __forceinline__ U4 draw(uint64_t seed, uint32_t traj, uint32_t stream, uint64_t n)
{
    return philox4x32_10(traj, stream, (uint32_t)n, (uint32_t)(n >> 32), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// Draw of local trajectory t of a batch whose trajectory 0 has global id
// s.traj_base.  Counter (gid_lo, stream + 256 gid_hi, n_lo, n_hi): for global
// ids below 2^32 this is the layout above with traj = gid.
__device__ __forceinline__ U4 draw_traj(const DevState &s, uint64_t seed, int64_t t,
                                        uint32_t stream, uint64_t n)
{
    const uint64_t gid = s.traj_base + (uint64_t)t;
    return draw(seed, (uint32_t)gid, stream + ((uint32_t)(gid >> 32) << 8), n);
}

// ------------------------------------------------------------ reductions
// Block-wide sum / min / max of doubles; `red` is shared scratch of >= 32
// doubles, `ident` the identity of op.  All threads of the block must call.
template <class Op>
__device__ __forceinline__ double block_reduce(double v, double *red, Op op, double ident)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double w = lane < nw ? red[lane] : ident;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = op(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) red[0] = w;
    }
    __syncthreads();
    const double r = red[0];
    __syncthreads();
    return r;
}

struct OpSum {
    __device__ double operator()(double a, double b) const { return a + b; }
};
struct OpMin {
    __device__ double operator()(double a, double b) const { return fmin(a, b); }
};
struct OpMax {
    __device__ double operator()(double a, double b) const { return fmax(a, b); }
};

// Deflated propagation (the isolated top level of the generator, s.defl laid
// out as defl_stride): the start value c - a u of row j of electron e and
// the end term e^{-i mu} a u_j, in the propagator's arithmetic R (explicit
// FMAs).
template <class R, class CT>
__device__ __forceinline__ CT defl_start(const double *df, int N, int Ne, int j, int e, CT v)
{
    const R *q = reinterpret_cast<const R *>(df + kDeflHead);
    const R ur = q[j], ui = q[N + j], ar = q[2 * N + e], ai = q[2 * N + Ne + e];
    v.x -= fma(ar, ur, -(ai * ui));
    v.y -= fma(ar, ui, ai * ur);
    return v;
}
template <class R, class CT>
__device__ __forceinline__ CT defl_end(const double *df, int N, int Ne, int j, int e, R cm, R sm, CT out)
{
    const R *q = reinterpret_cast<const R *>(df + kDeflHead);
    const R ur = q[j], ui = q[N + j], ar = q[2 * N + e], ai = q[2 * N + Ne + e];
    const R br = fma(ar, ur, -(ai * ui)), bi = fma(ar, ui, ai * ur);  // a u_j
    out.x += fma(cm, br, sm * bi);                                     // e^{-i mu} a u_j
    out.y += fma(cm, bi, -(sm * br));
    return out;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    return block_reduce(v, red, OpSum(), 0.0);
}
__device__ __forceinline__ double block_min(double v, double *red)
{
    return block_reduce(v, red, OpMin(), __longlong_as_double(0x7ff0000000000000ll));
}
__device__ __forceinline__ double block_max(double v, double *red)
{
    return block_reduce(v, red, OpMax(), __longlong_as_double(0xfff0000000000000ll));
}

}  // namespace iesh
