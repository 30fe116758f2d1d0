/*
 * iesh.h -- C-ABI of the GB300 batched independent electron surface hopping
 * (IESH) library, libiesh.so (sm_103a CUDA).
 *
 * The library advances a batch of independent IESH trajectories of a
 * Newns-Anderson adsorbate-metal model (Gardner, Corken, Janke, Habershon,
 * Maurer, arXiv:2212.00518, Sec. II).  One step of one trajectory is:
 *   1. velocity-Verlet half kick and drift of the nucleus (Sec. II C);
 *   2. eigenpairs of the arrowhead one-electron Hamiltonian H_el^1(x)
 *      (Sec. II B, single-electron Hamiltonian);
 *   3. Hellmann-Feynman force on the occupied surface (Sec. II B, classical
 *      IESH Hamiltonian) and the second half kick;
 *   4. nonadiabatic couplings d_jk = <j|d_x k> (Sec. II B) and the
 *      exponential integrator c <- exp(-i Abar dt) c for the N x Ne
 *      coefficient matrix (Sec. II C), Abar the average of the generators at
 *      the two ends of the step;
 *   5. hop probabilities g_{a->m} for every single excitation of the occupied
 *      Slater determinant from determinant ratios (Sec. II B, g, B, A and
 *      <k|psi> = det S), with the optional upper-bound skip of Sec. II C;
 *   6. stochastic hop with a Philox4x32-10 uniform and energy-conserving
 *      momentum rescaling, frustrated hops rejected (Sec. II B).
 *
 * Conventions
 *   - Units are atomic units.  N = n_bath + 1 orbitals (orbital index 0..N-1
 *     in ascending adiabatic energy), Ne electrons.
 *   - Array arguments are plain pointers that may point to host or device
 *     memory (the library copies with cudaMemcpyDefault).  They are owned by
 *     the caller, never freed by the library, and must be contiguous.
 *   - Per-trajectory arrays are trajectory-major: x[n], occ[n][Ne] (int16,
 *     ascending), C[n][Ne][N] complex interleaved (re, im) -- double for
 *     IESH_PREC_FP64, float for IESH_PREC_MIXED -- so the N coefficients of
 *     one electron are contiguous.
 *   - Every call is ordered on the stream given to iesh_create.  Calls that
 *     read into host memory synchronise that stream before returning.
 *   - Errors are returned as iesh_status; iesh_last_error(ctx) gives a
 *     message.  Numerical failures of single trajectories are reported in
 *     their status word (IESH_TRAJ_* bits) and never abort the batch.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef IESH_H
#define IESH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iesh_ctx iesh_ctx;

typedef enum {
    IESH_OK = 0,
    IESH_EINVAL = 1,   /* invalid argument (null pointer, size out of range) */
    IESH_ECUDA = 2,    /* a CUDA runtime call failed */
    IESH_ENOMEM = 3,   /* device allocation failed */
    IESH_ESTATE = 4,   /* call not allowed in the current state (e.g. run before init) */
    IESH_EUNSUPPORTED = 5, /* option combination not built */
    /* Returned only by iesh_check, which summarises the per-trajectory status
     * words of the batch (a numerical failure never aborts a batch): */
    IESH_ENONCONV = 6, /* some trajectory carries IESH_TRAJ_SECULAR_NONCONV */
    IESH_ESINGULAR = 7,/* some trajectory carries IESH_TRAJ_SINGULAR */
    IESH_ENORM = 8,    /* some trajectory carries IESH_TRAJ_NORM_DRIFT */
    IESH_ENAN = 9      /* some trajectory carries IESH_TRAJ_NAN */
} iesh_status;

/* Per-trajectory status bits (uint32). */
#define IESH_TRAJ_SECULAR_NONCONV 0x1u /* an eigenvalue iteration hit its cap */
#define IESH_TRAJ_SINGULAR 0x2u        /* overlap matrix S had a zero pivot */
#define IESH_TRAJ_NAN 0x4u             /* non-finite nucleus or force */
#define IESH_TRAJ_DONE 0x8u            /* trajectory finished (left the surface) */
#define IESH_TRAJ_PROP_RANGE 0x10u     /* propagator needed more terms than built */
#define IESH_PROP_AVERAGED 0
#define IESH_PROP_OVERLAP 1

#define IESH_TRAJ_TC_WAIT 0x20u        /* a tensor-core completion wait gave up (the
                                          step's coefficients were not updated) */
#define IESH_TRAJ_NORM_DRIFT 0x40u     /* after some step, an electron's coefficient
                                          column had | ||c_e||^2 - 1 | above
                                          iesh_options.norm_tol: the propagation
                                          (unitary in exact arithmetic, Sec. II C)
                                          lost accuracy; sticky until the next
                                          init/set_state */

/* Model kinds (Sec. II A; Sec. III B double well; Sec. III C desorption model). */
enum {
    IESH_MODEL_HARMONIC = 0,    /* par = {omega, g, dG}: U0 = m w^2 x^2/2,
                                   U1 = m w^2 (x-g)^2/2 + dG, f(x) = 1 */
    IESH_MODEL_DESORPTION = 1,  /* par = {De, x0, a, c, D1, D2, a', Vinf, q, a~, x~}:
                                   Morse U0, repulsive U1, tanh coupling f(x) */
    IESH_MODEL_MORSE_IMAGE = 2  /* par = {De, x0, a, c, h_inf, z_im, a_c, z_c, sigma}:
                                   Morse U0, h = h_inf - 1/(4 sqrt((z-z_im)^2+a_c^2)),
                                   f = exp(-(z-z_c)^2 / (2 sigma^2)) */
};
/* Coupling to bath state k: V_k(x) = sqrt(gamma / 2 pi) sqrt(w_k) f(x). */

enum { IESH_DISC_GL_SPLIT = 0, IESH_DISC_TRAPEZOID = 1 }; /* Appendix A */
enum { IESH_PREC_FP64 = 0, IESH_PREC_MIXED = 1 };

typedef struct {
    int kind;          /* IESH_MODEL_* */
    double mass;       /* nuclear mass */
    double par[16];    /* model constants, layout per kind (above) */
    double gamma;      /* wide-band hybridisation Gamma (Sec. II A) */
    double band_lo;    /* band edge a */
    double band_hi;    /* band edge b */
    double mu;         /* split point of the Gauss-Legendre discretisation */
    int n_bath;        /* M, bath states (N = M + 1 orbitals), 1 <= M <= 255 */
    int n_elec;        /* Ne electrons, 1 <= Ne <= min(N - 1, 112) */
    int disc;          /* IESH_DISC_* */
    int n_lo;          /* Gauss-Legendre nodes below mu (-1: M/2) */
    int n_leads;       /* 0 or 1: one band; 2: two leads (bias, Sec. II B end) */
    double lead_mu[2]; /* split point of each lead */
    int lead_n[2];     /* states per lead (sum = n_bath) */
    int lead_nlo[2];   /* nodes below the lead's split point */
    double lead_frac[2]; /* share of gamma per lead */
} iesh_model;

typedef struct {
    int precision;     /* IESH_PREC_FP64 or IESH_PREC_MIXED */
    int skip_bound;    /* 1: skip the ratio solve when the hop-probability upper
                          bound of Sec. II C is below the uniform (decisions unchanged) */
    int record_every;  /* record impurity populations every k steps (0: off) */
    int max_records;   /* capacity of the record buffer per trajectory */
    double z_done;     /* a trajectory is finished when x > z_done (0: never) */
    int compact_every; /* > 0: kernels visit only live trajectories (no IESH_TRAJ_DONE or
                          IESH_TRAJ_NAN) through a device work list, compacted in place
                          every compact_every steps of iesh_run (0: visit all) */
    int propagator;    /* IESH_PROP_AVERAGED (0): exponential of the step-averaged
                          adiabatic generator (Sec. II C); IESH_PROP_OVERLAP (1): the
                          diabatic-basis variant, exp(-i L1 dt/2) Q1^T Q0
                          exp(-i L0 dt/2) in the adiabatic frame (FP64 only; needs a
                          nonzero coupling factor f(x), else IESH_TRAJ_PROP_RANGE) */
    int64_t traj_base; /* global id of trajectory 0: trajectory t draws its random
                          numbers with id traj_base + t (see iesh_run), so that a
                          batch split over several contexts or GPUs, each given the
                          id of its first trajectory, reproduces the undivided batch */
    double prop_tol;   /* truncation tolerance of the Chebyshev series of the
                          propagator (0: 1e-15 for FP64, 1e-7 for the mixed path) */
    double norm_tol;   /* IESH_TRAJ_NORM_DRIFT threshold, checked after every step
                          of iesh_run (0: 1e-8 for FP64, 1e-3 for the mixed path;
                          < 0: no check) */
    int no_deflation;  /* FP64 averaged propagator: 1 runs the Chebyshev series over
                          the whole spectrum interval always; 0 (default) takes an
                          isolated top eigenvalue out of it where that shortens the
                          series by at least 2 terms, propagating its eigenvector
                          exactly (same result within the series tolerance) */
} iesh_options;

/* Create a context for up to max_traj trajectories of `model`.  Discretises
 * the bath (Appendix A), allocates all device state, and binds the CUDA
 * stream `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * On success *out holds the context; on failure *out is NULL. */
iesh_status iesh_create(iesh_ctx **out, const iesh_model *model, const iesh_options *opt,
                        int64_t max_traj, void *cuda_stream);

/* Free the context and its device memory.  NULL is accepted. */
iesh_status iesh_destroy(iesh_ctx *ctx);

/* Copy the discretised bath: eps[M] ascending bath energies and z0[M] =
 * sqrt(gamma / 2 pi) sqrt(w_k) (Appendix A). */
iesh_status iesh_bath(iesh_ctx *ctx, double *eps, double *z0);

/* Initialise n_traj trajectories (Sec. III B / III C initial conditions).
 * x0, p0 [n_traj]: given positions and momenta, or NULL to draw a thermal
 *   sample at kT_nuc (harmonic wells: Boltzmann; Morse wells: Wigner
 *   distribution of the harmonic approximation) from Philox stream 1.
 * occ0 [n_traj][Ne] ascending orbital indices, or NULL to draw an exact
 *   canonical sample at kT_el (kT_el = 0: the Ne lowest orbitals).
 * Coefficients start as unit vectors: electron j in orbital occ[j]. */
iesh_status iesh_init_state(iesh_ctx *ctx, int64_t n_traj, const double *x0, const double *p0,
                            const int16_t *occ0, double kT_nuc, double kT_el, uint64_t seed);

/* Replace the state of n_traj trajectories with (x, p, occ, C) (layouts
 * above) and recompute eigenpairs and forces there.  Step counters and
 * statistics are reset.  Used to compare with other implementations from a
 * shared state. */
iesh_status iesh_set_state(iesh_ctx *ctx, int64_t n_traj, const double *x, const double *p,
                           const int16_t *occ, const void *C);

/* Copy out the state.  Any pointer may be NULL to skip that array. */
iesh_status iesh_get_state(iesh_ctx *ctx, double *x, double *p, int16_t *occ, void *C,
                           uint32_t *status);

/* Advance every live trajectory by n_steps steps of length dt (steps 1-6
 * above).  The hop uniform of trajectory t at its step n (the count of steps
 * it has taken, kept across iesh_run calls and checkpoints) is drawn from
 * Philox4x32-10 with key = seed and counter = (g_lo, 256 g_hi, n_lo, n_hi),
 * g = traj_base + t its global id (for g < 2^32: (g, 0, n_lo, n_hi)); the
 * thermal samples of iesh_init_state use streams 1 (nuclei) and 2
 * (electrons) in the second word.  Asynchronous on the context stream. */
iesh_status iesh_run(iesh_ctx *ctx, double dt, int64_t n_steps, uint64_t seed);

/* Checkpoint / resume.  A checkpoint holds the complete per-trajectory state
 * of the context's n trajectories: x, p, occupations, coefficients, the
 * eigenpairs and model values of the current and previous step (the
 * previous step's generator enters the step average of Sec. II C), forces,
 * status words, step counters (the Philox counters of the hop uniforms),
 * hop counters and population records.  Resuming from it continues the run
 * bit for bit.  The blob is opaque and versioned; it may live in host or
 * device memory (caller-owned).
 * iesh_checkpoint_bytes: *bytes receives the size for the current batch.
 * iesh_checkpoint_save: writes it (bytes must be at least that size);
 *   returns after the copies finished.
 * iesh_checkpoint_load: restores a checkpoint written by a context of the
 *   same model sizes, precision, propagator and record layout (else
 *   IESH_EINVAL) with at most max_traj trajectories. */
iesh_status iesh_checkpoint_bytes(iesh_ctx *ctx, size_t *bytes);
iesh_status iesh_checkpoint_save(iesh_ctx *ctx, void *buf, size_t bytes);
iesh_status iesh_checkpoint_load(iesh_ctx *ctx, const void *buf, size_t bytes);

/* Advance a batch held in host memory: the same result, bit for bit, as
 * iesh_checkpoint_load(in), iesh_run(dt, n_steps, seed) and
 * iesh_checkpoint_save(out), with the copies overlapped with the steps.
 * The batch is cut into `chunks` trajectory ranges (<= 0: 4).  Range c is
 * copied in on a stream of its own, stepped on the context's stream once it
 * has landed, and copied out on a third stream while range c + 1 steps.
 * Every step kernel treats trajectories independently, so ranges give the
 * same bits as the whole batch.
 * in: a checkpoint of iesh_checkpoint_save (host memory, `bytes` long; page
 *   locked for the copies to overlap).
 * out: host buffer of the same size for the checkpoint after the steps.  It
 *   may be `in`: each range is read before it is written.
 * The context's device state then holds the advanced batch.  Returns after
 * the copies out have finished.  IESH_EUNSUPPORTED with population records
 * or the device work list on (their arrays are not trajectory-major);
 * IESH_EINVAL for device buffers, or for a checkpoint that does not match
 * the context, as iesh_checkpoint_load. */
iesh_status iesh_run_host(iesh_ctx *ctx, const void *in, void *out, size_t bytes, double dt, int64_t n_steps,
                          uint64_t seed, int chunks);

/* Observables of every trajectory at its current state (Sec. III C/D):
 * ke[n] = p^2 / 2m, epot[n] = U0(x) + sum_{i in s} lambda_i (the classical
 * IESH Hamiltonian of Sec. II B without the kinetic term), and the impurity
 * populations pop_sh[n] = sum_{i in s} q0_i^2 and pop_wf[n] =
 * sum_e |sum_i q0_i c_ie|^2.  Any pointer may be NULL. */
iesh_status iesh_observables(iesh_ctx *ctx, double *ke, double *epot, double *pop_sh,
                             double *pop_wf);

/* Summary of the batch's status words: bits[0] = OR over the trajectories,
 * bits[1 + b] = number of trajectories with bit b set (b < 8); bits may be
 * NULL.  Synchronises the context stream.  Returns IESH_ENAN, IESH_ENONCONV,
 * IESH_ESINGULAR or IESH_ENORM (checked in this order) when some trajectory
 * carries the matching bit, else IESH_OK. */
iesh_status iesh_check(iesh_ctx *ctx, uint32_t *bits);

/* Eigenvalues lam[n][N], impurity components q0[n][N] (> 0) of the
 * eigenvectors and the force F[n] at the current positions. */
iesh_status iesh_get_eigen(iesh_ctx *ctx, double *lam, double *q0, double *force);

/* Hop probabilities g[n][Ne][N] (slot a of the sorted occupation list,
 * target orbital m; zero for occupied m) of the current state at velocity
 * p/m, as used by step 5; the state is not changed. */
iesh_status iesh_hop_probabilities(iesh_ctx *ctx, double dt, double *g);

/* Per-trajectory counters: steps taken, accepted and frustrated hops. */
iesh_status iesh_get_counters(iesh_ctx *ctx, int64_t *nstep, int32_t *hops, int32_t *frustrated);

/* Recorded impurity populations [n_records][n_traj]: the occupied-surface
 * value sum_{i in s} q0_i^2 and the wavefunction value
 * sum_e |sum_i q0_i C_ie|^2.  *n_records receives the number recorded. */
iesh_status iesh_get_records(iesh_ctx *ctx, double *pop_sh, double *pop_wf, int64_t *n_records);

/* Number of live trajectories in the device work list (n_traj when the work
 * list is off).  Synchronises the context stream. */
iesh_status iesh_get_live(iesh_ctx *ctx, int64_t *n_live);

/* ---------------------------------------------------------------------
 * Uneven batches in one launch.
 *
 * Trajectories of different bath sizes (one context per model) and
 * lifetimes (a trajectory ends when it leaves the surface, Sec. III D) run
 * together: iesh_ensemble_create captures, once, a CUDA graph whose single
 * device-side loop (a conditional while node) advances every context by
 * `chunk` steps, compacts every context's work list of live trajectories
 * on the device, and decides on the device whether to go on.
 * iesh_ensemble_run enqueues one launch of that graph on cuda_stream: it
 * returns at once, and the device keeps looping until no trajectory of any
 * context is live or max_steps more steps have run (whole chunks; the
 * count is the loop's own and does not include iesh_run steps).  Finished
 * trajectories cost no work (their CTAs exit at once); results are bit
 * for bit those of iesh_run with the same seed.  Each context needs
 * compact_every > 0, a state (init_state / set_state / checkpoint_load) and
 * profiling off; the graph holds the contexts' batch sizes at creation, so
 * create the ensemble after the set-up and create it again after changing a
 * batch.  The contexts' earlier work is waited for, and their later calls
 * wait for the loop.  iesh_ensemble_status synchronises cuda_stream and
 * returns the loop's total steps and the live trajectories after the last
 * chunk; exact live trajectory-steps are the sum of iesh_get_counters'
 * step counts.  The contexts must outlive the ensemble. */
typedef struct iesh_ensemble iesh_ensemble;
iesh_status iesh_ensemble_create(iesh_ensemble **out, iesh_ctx *const *ctxs, int n_ctx, double dt,
                                 int64_t chunk, uint64_t seed, void *cuda_stream);
iesh_status iesh_ensemble_run(iesh_ensemble *ens, int64_t max_steps);
iesh_status iesh_ensemble_status(iesh_ensemble *ens, int64_t *steps_done, int64_t *live);
iesh_status iesh_ensemble_destroy(iesh_ensemble *ens);
const char *iesh_ensemble_last_error(const iesh_ensemble *ens);

/* Kernel shapes.  FP64 contexts: cheb_ept (1 or 2) electrons per thread and
 * cheb_G column groups per CTA of the propagator (cheb_G * N <= 1024).
 * Mixed contexts: cheb_ept 4 (each thread holds 4 orbitals x 4 electrons,
 * two CTAs per SM) with cheb_G * ceil(N/4) <= 256 and 8 * Np * (8 cheb_G +
 * 1) + 192 * Np bytes of shared memory (Np = N rounded up to a multiple of
 * 4; the second term stages W) at most 110 KiB; or cheb_ept 32 (8 orbitals
 * x 4 electrons per thread, one CTA per SM) with cheb_G * ceil(ceil(N/4)/2)
 * <= 256 and the same shared memory at most 220 KiB; or cheb_ept 8 with
 * cheb_G 1, the tensor-core kernel (N <= 128, Ne <= 56, 3xTF32); or
 * cheb_ept 16 with cheb_G 1, the tensor-core kernel on FP16 split operands
 * with two CTAs per SM (N <= 128, Ne <= 56, its shared memory at most 110
 * KiB).  hop_threads (256 or 512):
 * threads of the LU hop kernel; 0 restores the built-in choice, which for
 * mixed contexts is a Gauss-Jordan elimination of all determinant ratios,
 * in registers for N <= 128 and Ne <= 56 and with the rows past 128 in
 * shared memory up to N = 256, Ne = 112 (the skip bound saves no work
 * there and is not applied; its FP32 ratios round differently from the
 * LU's, about 1e-7 relative); IESH_EINVAL otherwise.  The propagator shapes do not change results
 * (each output keeps a fixed summation order).  Used by the autotuner of
 * the Python package. */
iesh_status iesh_set_kernel_shape(iesh_ctx *ctx, int cheb_ept, int cheb_G, int hop_threads);
iesh_status iesh_get_kernel_shape(iesh_ctx *ctx, int *cheb_ept, int *cheb_G, int *hop_threads);

/* Chebyshev degree K[n] used by each trajectory's propagator in its last
 * step (the number of coupling-matrix products of that step). */
iesh_status iesh_get_propagator_terms(iesh_ctx *ctx, int32_t *K);

/* Kernel timing.  With profiling on, every kernel launch of the context is
 * bracketed by CUDA events on the context stream.  iesh_profile_read
 * synchronises and returns, per kernel class (IESH_K_*), the summed device
 * time in ms and the number of launches since profiling was switched on. */
enum { IESH_K_EIGEN = 0, IESH_K_COUPLING = 1, IESH_K_PROPAGATE = 2, IESH_K_HOP = 3,
       IESH_K_OTHER = 4, IESH_K_COUNT = 5 };
iesh_status iesh_profile(iesh_ctx *ctx, int enable);
iesh_status iesh_profile_read(iesh_ctx *ctx, double *ms, int64_t *launches);

/* ---------------------------------------------------------------------
 * Hop probabilities without any device allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc: host frameworks that own all device memory through
 * their own pool allocator, and latency-critical loops that cannot afford an
 * allocation and the device synchronisation it may cause.  It computes the
 * same g[n][Ne][N] as iesh_hop_probabilities, but from caller-owned device
 * arrays and without a context: model (host pointer, read during the call),
 * x[n], p[n] positions and momenta, occ[n][Ne] (int16, ascending), C
 * [n][Ne][N] complex double coefficients, lam[n][N] and q0[n][N] the
 * eigenvalues and eigenvector impurity components at x (as returned by
 * iesh_get_eigen), dt the step length; output g[n][Ne][N] (device).  All
 * array pointers must be device memory.  Work is queued on cuda_stream
 * (a cudaStream_t, NULL = legacy default stream) and the call returns
 * without waiting.
 *
 * Working memory is a fixed array of IESH_NOALLOC_SCRATCH_BYTES inside the
 * library's device module.  It is resident on every device where that
 * module is loaded (under lazy module loading, from the first use of any
 * of the library's kernels on that device; with CUDA_MODULE_LOADING=EAGER,
 * on every device the process initialises), even in processes that never
 * call this function, and stays there until the process exits.  One call
 * needs 16 n Ne N + 48 n bytes (plus alignment), and a larger request
 * returns IESH_EINVAL before any work is queued.  The first call on a
 * device, with that device current, looks up the array's device address
 * and sets the hop kernels' shared-memory limits; make this first call
 * before any stream capture.  All calls share
 * the one array and each call overwrites it: calls that overlap on the GPU
 * (different streams or host threads without ordering) race and give wrong
 * results.  Trajectories with a singular overlap matrix get g = 0.  On error
 * a message is written to err (err_len bytes, may be NULL). */
#define IESH_NOALLOC_SCRATCH_BYTES (32u << 20)
iesh_status iesh_hop_probabilities_noalloc(const iesh_model *model, int64_t n, const double *x,
                                           const double *p, const int16_t *occ, const void *C,
                                           const double *lam, const double *q0, double dt,
                                           double *g, void *cuda_stream, char *err,
                                           size_t err_len);

/* ---------------------------------------------------------------------
 * Batched dense symmetric eigensolver.
 *
 * The paper obtains the eigenpairs of the one-electron Hamiltonian by a
 * dense symmetric diagonalisation at every step (Sec. II C, implementation
 * details); the arrowhead secular solver of iesh_run is its fast path for
 * a single adsorbate orbital.  This call is the general method: for each
 * of B symmetric n x n matrices A[b] (row-major, both triangles stored;
 * n <= 256) it computes the eigenvalues lam[b][0..n-1] in ascending order
 * and, if V is not NULL, the orthonormal eigenvectors as rows V[b][j][0..n-1]
 * (A v_j = lam_j v_j), each signed so that its component of largest
 * magnitude (the first on a tie) is positive.  Householder reduction to
 * tridiagonal form (one CTA per matrix, the matrix in shared memory up to
 * about 200 KB), implicit-shift QL iterations (one thread per matrix for
 * eigenvalues only; with eigenvectors one CTA per matrix, the rotations of
 * each sweep applied to all rows of the reflector product in parallel),
 * ordering.
 * precision: IESH_PREC_FP64 (double arrays) or IESH_PREC_MIXED (float
 * arrays, FP32 arithmetic).  info[b] (device, may be NULL) is set to 0, or
 * to 1 when an eigenvalue needed more than 60 QL iterations (the output of
 * that matrix is then unreliable).  work: caller-owned device workspace of
 * at least iesh_syev_work_bytes(B, n, precision, V != NULL) bytes.  All
 * array pointers are device memory.  Asynchronous on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream); allocates nothing.  On error
 * a message is written to err (err_len bytes, may be NULL). */
size_t iesh_syev_work_bytes(int64_t B, int n, int precision, int vectors);
iesh_status iesh_syev_batched(int64_t B, int n, int precision, const void *A, void *lam, void *V,
                              uint32_t *info, void *work, size_t work_bytes, void *cuda_stream,
                              char *err, size_t err_len);

/* ---------------------------------------------------------------------
 * Occupied-orbital energy of a two-orbital adsorbate, E_occ = sum of the Ne
 * lowest eigenvalues of the one-electron Hamiltonian (the electronic part
 * of the classical IESH Hamiltonian, Sec. II B, at ground-state occupation),
 * and its Hellmann-Feynman gradients.  Orbital a = 0, 1 has level
 * h_a = theta[a] + sum_al theta[2 + 6a + al] x[al] and couples to bath state
 * k by vbar[a] sqrt(w_k) exp(-|x_a - R_a|^2 / (2 theta[14+a]^2)), x_a =
 * (x[3a], x[3a+1], x[3a+2]); the bath is the split Gauss-Legendre
 * discretisation of [band_lo, band_hi] at mu (Appendix A). */
typedef struct iesh_eocc_ctx iesh_eocc_ctx;
typedef struct {
    int n_bath;        /* M (2..4096) */
    int n_elec;        /* Ne, orbitals summed (1..min(M+1, 1024)) */
    double band_lo, band_hi, mu;
    double vbar[2];    /* coupling amplitudes */
    double R[6];       /* coupling centres */
} iesh_eocc_model;

/* Create / destroy (the bath lives on the device in FP64 and FP32). */
iesh_status iesh_eocc_create(iesh_eocc_ctx **out, const iesh_eocc_model *model, void *cuda_stream);
iesh_status iesh_eocc_destroy(iesh_eocc_ctx *ctx);
const char *iesh_eocc_last_error(const iesh_eocc_ctx *ctx);

/* Forward for B geometries.  Device pointers; element type double for
 * precision IESH_PREC_FP64, float for IESH_PREC_MIXED.  x[B][6],
 * theta[16] -> E[B] and saved[B][4] = (S_0, S_1, T_0, T_1), S_a = sum_{i<Ne}
 * Q_ai^2, T_a = sum_{i<Ne} Q_ai^2 (lam_i - h_a); status[B] (uint32,
 * IESH_TRAJ_SECULAR_NONCONV).  Asynchronous on the context stream. */
iesh_status iesh_eocc_forward(iesh_eocc_ctx *ctx, int64_t B, int precision, const void *x,
                              const void *theta, void *E, void *saved, uint32_t *status);

/* Backward: given gE[B] = dL/dE, writes dx[B][6] = gE dE/dx, the
 * per-geometry parameter gradients dtheta_per[B][16] (caller workspace) and
 * their sum dtheta[16] (fixed summation order).  Same element type rules. */
iesh_status iesh_eocc_backward(iesh_eocc_ctx *ctx, int64_t B, int precision, const void *x,
                               const void *theta, const void *saved, const void *gE, void *dx,
                               void *dtheta_per, void *dtheta);

/* ---------------------------------------------------------------------
 * IESH dynamics of a two-orbital adsorbate over six nuclear coordinates.
 *
 * The electrons are those of the occupied-energy model above: orbital a =
 * 0, 1 with level h_a(x) = theta[a] + sum_al theta[2 + 6a + al] x[al] and
 * coupling vbar[a] sqrt(w_k) f_a(x), f_a = exp(-|x_a - R_a|^2 /
 * (2 theta[14+a]^2)), to bath state k of the split Gauss-Legendre band
 * (Appendix A, n_bath / 2 nodes below mu); N = n_bath + 2 orbitals.  The
 * nuclei move on U0 = mass omega^2 |x - x0|^2 / 2 plus the occupied
 * eigenvalues (the classical IESH Hamiltonian of Sec. II B), one mass for
 * all six coordinates.  A step is the one-coordinate step of iesh_run in
 * six dimensions (Sec. II B, II C): velocity Verlet, eigenpairs of the
 * rank-two arrowhead, Hellmann-Feynman forces, the exponential of the
 * step-averaged generator built from v . d (the NAC vectors projected on
 * the velocity at each end of the step), hop probabilities from
 * determinant ratios with v . d, and on a hop the momentum change
 * p' = p + alpha d_{m, s_a} along the NAC vector that conserves the energy
 * with the smaller |alpha|; no such alpha: the hop is frustrated.
 *
 * Eigenvector gauge: the component of eigenvector j on the coupled
 * combination c_0 |0> + c_1 |1> (c_a = vbar[a] f_a; with profile 1, c_a =
 * vbar[a] f_a |profile_a|) is >= 0, except that in a step an eigenvector
 * whose overlap with the previous step's eigenvector j is at least 1/2 in
 * magnitude keeps that overlap positive (continuity: the combination passes
 * through zero for the |->-like eigenvector where h_0 = h_1, and for
 * non-parallel couplings elsewhere too; at an eigenvalue crossing within
 * the step the overlap decides nothing and the combination rule stands).
 * Layouts: x, p, F [n][6]; occ [n][Ne] int16 ascending; C [n][Ne][N]
 * complex, double for IESH_PREC_FP64 and float for IESH_PREC_MIXED (the
 * one-coordinate split: FP64 eigenpairs, forces, hop probabilities and
 * rescale; FP32 coefficients, coupling generator, propagation and overlap
 * LU); pointers host or device as for iesh_*. */
typedef struct iesh2_ctx iesh2_ctx;
typedef struct {
    int n_bath;        /* M (2..254) */
    int n_elec;        /* Ne (1..min(M + 1, 112)) */
    double band_lo, band_hi, mu; /* band and split point of the bath */
    double mass;       /* nuclear mass (all six coordinates) */
    double omega;      /* restraint frequency */
    double x0[6];      /* restraint centres */
    double theta[16];  /* eps_0, eps_1, g_{0,0..5}, g_{1,0..5}, sigma_0, sigma_1 */
    double vbar[2];    /* coupling amplitudes */
    double R[6];       /* coupling centres */
    int profile;       /* 0: both orbitals couple to bath state k as vbar_a sqrt(w_k) f_a
                          (parallel border vectors); 1: each orbital with its own
                          Lorentzian bath profile, vbar_a sqrt(w_k) f_a / sqrt(1 +
                          ((eps_k - prof_center[a]) / prof_width[a])^2) (the border
                          vectors are not parallel) */
    double prof_center[2], prof_width[2];
    int eigensolver;   /* 0: secular equations, the rank-two arrowhead reduction for
                          profile 0, two nested arrowheads (orbital 1 with the bath,
                          then orbital 0 against those eigenvectors) for profile 1;
                          1: the dense symmetric eigensolver (as iesh_syev_batched,
                          FP64) always */
} iesh2_model;

/* Create a context for up to max_traj trajectories; precision
 * IESH_PREC_FP64 or IESH_PREC_MIXED; skip_bound as in iesh_options.  On
 * failure *out may hold a context carrying the message (destroy it). */
iesh_status iesh2_create(iesh2_ctx **out, const iesh2_model *model, int precision, int64_t max_traj,
                         int skip_bound, void *cuda_stream);
iesh_status iesh2_destroy(iesh2_ctx *ctx);
const char *iesh2_last_error(const iesh2_ctx *ctx);

/* Replace the state of n_traj trajectories and compute eigenpairs and
 * forces there; counters are reset.  Returns after the copies finished. */
iesh_status iesh2_set_state(iesh2_ctx *ctx, int64_t n_traj, const double *x, const double *p,
                            const int16_t *occ, const void *C);
iesh_status iesh2_get_state(iesh2_ctx *ctx, double *x, double *p, int16_t *occ, void *C,
                            uint32_t *status);

/* n_steps steps of length dt; the hop uniform of trajectory t at its step n
 * is Philox4x32-10 with key = seed, counter = (t, 0, n_lo, n_hi). */
iesh_status iesh2_run(iesh2_ctx *ctx, double dt, int64_t n_steps, uint64_t seed);

/* Eigenvalues lam[n][N], adsorbate components Q[n][2][N] (row a: component
 * on adsorbate orbital a of each eigenvector) and forces F[n][6] at the
 * current positions and occupations. */
iesh_status iesh2_get_eigen(iesh2_ctx *ctx, double *lam, double *Q, double *F);

/* Hop probabilities g[n][Ne][N] of the current state (velocity p / mass),
 * as used by the step; the state is not changed. */
iesh_status iesh2_hop_probabilities(iesh2_ctx *ctx, double dt, double *g);

/* Steps taken, accepted and frustrated hops per trajectory. */
iesh_status iesh2_get_counters(iesh2_ctx *ctx, int64_t *nstep, int32_t *hops, int32_t *frustrated);

/* Kernel timing, as iesh_profile / iesh_profile_read. */
iesh_status iesh2_profile(iesh2_ctx *ctx, int enable);
iesh_status iesh2_profile_read(iesh2_ctx *ctx, double *ms, int64_t *launches);

/* Diagnostic: r[i] = the reciprocal 1 / d[i] as the FP64 kernels form it
 * for pole distances and eigenvalue gaps (the PTX reciprocal estimate
 * refined by the geometric series r0 (1 + e + e^2), e = 1 - d r0), for
 * comparison with a correctly rounded division.  d, r: device arrays of n
 * doubles (normal numbers); asynchronous on cuda_stream. */
iesh_status iesh_diag_reciprocal(int64_t n, const double *d, double *r, void *cuda_stream);

/* Last error message of the context (never NULL). */
const char *iesh_last_error(const iesh_ctx *ctx);

/* Name of a status code. */
const char *iesh_status_string(iesh_status s);

#ifdef __cplusplus
}
#endif
#endif
