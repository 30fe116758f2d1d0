// iesh_noalloc.cu -- hop probabilities for callers that cannot allocate
// device memory.
//
// Some callers of this library cannot call cudaMalloc: host frameworks that
// own the whole device memory through their own pool allocator (a raw
// cudaMalloc there fails or fragments the pool), and latency-critical loops
// in which an allocation, with the device synchronisation it can imply, is
// not acceptable.  For them this file provides one stateless entry point
// that computes the same hop probabilities as iesh_hop_probabilities from
// caller-owned inputs and outputs, and keeps its working memory in a
// fixed-size array that is part of the library image on each device.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/iesh.h"
#include "iesh_common.cuh"
#include "iesh_kernels.h"

using namespace iesh;

namespace {

// Working memory of iesh_hop_probabilities_noalloc.  It is part of the
// library's device module, so it is resident on every device where that
// module is loaded (with lazy module loading: from the first launch of any
// of the library's kernels on the device), whether or not this entry point
// is called, and it stays there until the process exits.  In host code the
// name is only a stand-in for the device array; the device address comes
// from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[IESH_NOALLOC_SCRATCH_BYTES / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Impurity level h, dh/dx, kappa = f'/f and U0 at each position (the
// per-trajectory quantities the hop kernel reads besides the eigenpairs).
__global__ void k_noalloc_geometry(int64_t n, ModelDev md, const double *__restrict__ x,
                                   double *__restrict__ geo)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const ModelVals mv = model_eval(md, x[t]);
    geo[t * 4 + 0] = mv.h;
    geo[t * 4 + 1] = mv.dh;
    geo[t * 4 + 2] = (mv.f != 0.0) ? mv.df / mv.f : 0.0;
    geo[t * 4 + 3] = mv.U0;
}

iesh_status report(char *err, size_t err_len, iesh_status s, const char *msg)
{
    if (err && err_len) {
        strncpy(err, msg, err_len - 1);
        err[err_len - 1] = '\0';
    }
    return s;
}

}  // namespace

extern "C" iesh_status iesh_hop_probabilities_noalloc(const iesh_model *model, int64_t n,
                                                      const double *x, const double *p,
                                                      const int16_t *occ, const void *C,
                                                      const double *lam, const double *q0,
                                                      double dt, double *g, void *cuda_stream,
                                                      char *err, size_t err_len)
{
    char buf[256];
    if (!model) return report(err, err_len, IESH_EINVAL, "model is NULL");
    const int M = model->n_bath, Ne = model->n_elec, N = M + 1;
    if (model->kind < 0 || model->kind > 2) return report(err, err_len, IESH_EINVAL, "unknown model kind");
    if (M < 1 || N > kMaxOrbitals) return report(err, err_len, IESH_EINVAL, "n_bath outside 1..255");
    if (Ne < 1 || Ne > N - 1 || Ne > kMaxHopElectrons)
        return report(err, err_len, IESH_EINVAL, "n_elec outside 1..min(N-1, 112)");
    if (!(model->mass > 0.0) || !(dt > 0.0))
        return report(err, err_len, IESH_EINVAL, "mass and dt must be positive");
    if (n < 0) return report(err, err_len, IESH_EINVAL, "n must be >= 0");
    if (n == 0) return report(err, err_len, IESH_OK, "");
    if (!x || !p || !occ || !C || !lam || !q0 || !g)
        return report(err, err_len, IESH_EINVAL, "x, p, occ, C, lam, q0 and g must be device pointers");

    // Working memory of one call: status (n x 4 B) and step counters (n x 8 B)
    // that must start at zero, the geometry (n x 32 B) and the triangular-
    // solve rows (n x Ne x N x 16 B), each section 256-byte aligned.
    const int64_t stride = ((int64_t)2 * Ne * N + 31) & ~(int64_t)31;  // doubles per trajectory
    const int64_t w_status = ((n + 1) / 2 + 31) & ~(int64_t)31;
    const int64_t w_nstep = (n + 31) & ~(int64_t)31;
    const int64_t w_geo = (4 * n + 31) & ~(int64_t)31;
    const int64_t need = w_status + w_nstep + w_geo + n * stride;
    const int64_t cap = (int64_t)(IESH_NOALLOC_SCRATCH_BYTES / sizeof(double));
    if (need > cap) {
        snprintf(buf, sizeof buf,
                 "needs %lld bytes of working memory, above the fixed %lld bytes "
                 "(IESH_NOALLOC_SCRATCH_BYTES); pass fewer trajectories per call",
                 (long long)(need * 8), (long long)(cap * 8));
        return report(err, err_len, IESH_EINVAL, buf);
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(err, err_len, IESH_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report(err, err_len, IESH_EINVAL, "device index too large");
    double *base;
    {
        // One-time set-up on this device (with the device current).
        std::lock_guard<std::mutex> lk(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess || !addr) {
                snprintf(buf, sizeof buf, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return report(err, err_len, IESH_ECUDA, buf);
            }
            // the hop kernels' shared-memory limits (process-wide function
            // attributes), set once here so that no later call changes them
            configure_hop_smem();
            g_scratch_addr[dev] = (double *)addr;
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;

    DevState s;
    memset(&s, 0, sizeof s);
    s.N = N;
    s.M = M;
    s.Ne = Ne;
    s.n = n;
    s.p = const_cast<double *>(p);
    s.occ = const_cast<int16_t *>(occ);
    s.C = const_cast<void *>(C);
    s.lam = const_cast<double *>(lam);
    s.q0 = const_cast<double *>(q0);
    s.status = reinterpret_cast<uint32_t *>(base);
    s.nstep = reinterpret_cast<int64_t *>(base + w_status);
    s.geo = base + w_status + w_nstep;
    s.scratch = base + w_status + w_nstep + w_geo;
    s.scratch_stride = stride;

    // The array keeps the previous call's contents: clear the counters.
    e = cudaMemsetAsync(base, 0, (size_t)(w_status + w_nstep) * sizeof(double), st);
    if (e != cudaSuccess) return report(err, err_len, IESH_ECUDA, cudaGetErrorString(e));
    ModelDev md;
    md.kind = model->kind;
    md.mass = model->mass;
    for (int i = 0; i < 16; ++i) md.par[i] = model->par[i];
    k_noalloc_geometry<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, md, x, s.geo);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(err, err_len, IESH_ECUDA, cudaGetErrorString(e));
    e = launch_hop(s, dt, model->mass, 0, 0, g, st);
    if (e != cudaSuccess) return report(err, err_len, IESH_ECUDA, cudaGetErrorString(e));
    return report(err, err_len, IESH_OK, "");
}
