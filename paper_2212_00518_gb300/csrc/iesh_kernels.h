// iesh_kernels.h -- host launch wrappers of the step kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "iesh_common.cuh"

namespace iesh {

cudaError_t launch_eigen(const DevState &s, const ModelDev &md, double dt, int mode,
                         cudaStream_t st);
cudaError_t launch_force(const DevState &s, cudaStream_t st);
cudaError_t launch_coupling(const DevState &s, double dt, double mass, double tol, bool mixed,
                            cudaStream_t st);
cudaError_t launch_cheb(const DevState &s, double dt, bool mixed, cudaStream_t st);
size_t hop_smem_bytes(int N, int Ne);
cudaError_t launch_hop(const DevState &s, double dt, double mass, uint64_t seed, int skip_bound,
                       double *g_out, cudaStream_t st, bool mixed = false, bool ext = false);
cudaError_t launch_init_nuclear(const DevState &s, double mass, uint64_t seed, double kT,
                                int wigner, double omega, double x_eq, cudaStream_t st);
cudaError_t launch_sample_occ(const DevState &s, uint64_t seed, double kT, cudaStream_t st);
cudaError_t launch_unit_coeffs(const DevState &s, bool fp32, cudaStream_t st);
cudaError_t launch_compact(const DevState &s, int32_t *live, int32_t *n_live, cudaStream_t st);
cudaError_t launch_live_init(int64_t n, int32_t *live, int32_t *n_live, cudaStream_t st);
void configure_hop_smem();
// mixed-path hop probabilities by Gauss-Jordan elimination in registers
// (N <= 128, Ne <= 56)
bool hop_gj_eligible(int N, int Ne);
// the same elimination with the rows past 128 in shared memory: N <= 256, Ne <= 112
bool hop_gjl_eligible(int N, int Ne);
void configure_hop_gjl();
cudaError_t launch_hop_gjl(const DevState &s, double dt, double mass, uint64_t seed, double *g_out,
                           cudaStream_t st, bool ext);
cudaError_t launch_hop_gj(const DevState &s, double dt, double mass, uint64_t seed, double *g_out,
                          cudaStream_t st, bool ext);
// Bath of one lead: energies and weights (Gauss-Legendre split at mu, or trapezoid)
void lead_bath(int disc, int n, double a, double b, double mu, int n_lo, std::vector<double> &eps,
               std::vector<double> &w);
void cheb_shape(int N, int Ne, int &ept, int &G);
// Trajectories per CTA of the eigen kernels (slots of N threads, <= 512 threads)
int eigen_tpb(int N);
// FP32 (mixed-precision) propagator: 4 electrons per thread, G column
// groups; one row quad per thread (two CTAs per SM) or two (one CTA per SM)
constexpr size_t kCheb32MaxSmem = 110 * 1024;
constexpr size_t kCheb32WideMaxSmem = 220 * 1024;
constexpr int kCheb32WideMinN = 224;  // default to two row quads per thread past this N
constexpr int kCheb32WRows = 16; // rows of W per chunk staged in shared memory
constexpr int kCheb32WRing = 3;  // chunks in the ring (filled 2 ahead)
size_t cheb32_smem_bytes(int N, int G);
void cheb32_shape(int N, int Ne, int &G, int qpt = 1);
bool cheb32_shape_ok(int N, int G, int qpt);
// the mixed SIMT propagator deflates (k_build_w_f32<true> sets the level up)
bool mixed_deflates(const DevState &s);
// FP32 propagator on the tensor cores (3xTF32), N <= 128 and Ne <= 56
constexpr size_t kChebTcMaxSmem = 224 * 1024;
size_t cheb_tc_smem_bytes(int N, int Ne);
bool cheb_tc_eligible(int N, int Ne);
void configure_cheb_tc();
cudaError_t launch_cheb_tc(const DevState &s, double dt, cudaStream_t st);
// The same on FP16 split operands, two CTAs per SM (shared memory at most
// kChebTc16MaxSmem each)
constexpr size_t kChebTc16MaxSmem = 110 * 1024;
size_t cheb_tc16_smem_bytes(int N, int Ne);
bool cheb_tc16_eligible(int N, int Ne);
void configure_cheb_tc16();
cudaError_t launch_cheb_tc16(const DevState &s, double dt, cudaStream_t st);
// unitarity check of the coefficient columns (sets ST_NORM), observables
// out[4][n] = (kinetic energy, potential energy, occupied-surface and
// wavefunction impurity populations), batch status summary out[9]
cudaError_t launch_norm_check(const DevState &s, bool fp32, double tol, cudaStream_t st);
cudaError_t launch_observables(const DevState &s, bool fp32, double mass, double *out,
                               cudaStream_t st);
cudaError_t launch_status_summary(const uint32_t *status, int64_t n, uint32_t *out, cudaStream_t st);
// diabatic-basis (overlap) propagator variant: build O^T, then apply
size_t overlap_build_smem(int N, int M);
cudaError_t launch_overlap(const DevState &s, double dt, cudaStream_t st);

}  // namespace iesh
