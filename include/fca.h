/*
 * fca.h -- C ABI of the GB300 (sm_103a) library for EM parameter estimation of two-source
 * full-rank spatial covariance analysis (FCA), in two forms:
 *
 *   conventional EM   Ito, Araki, Nakatani, "FastFCA" (arXiv 1805.06572), Sec. 2,
 *                     Eqs. (MMSE), (postquadexp), (vupdate), (Supdate): a frame-wise
 *                     M x M inverse of v1 S1 + v2 S2 at every time-frequency point;
 *   FastFCA           Sec. 3 and Algorithm 1: a per-frequency generalised eigenvector
 *                     basis P (Eq. (GEVD)) jointly diagonalises S1 and S2, so every
 *                     time-frequency point needs only scalar updates (Eqs. (MMSEtilde),
 *                     (updatePhitildeeff), (updateveff), (updateStildeeff)) and P is
 *                     updated once per frequency per iteration (Eqs. (updatePeff),
 *                     (updateLambdaeff)).
 *
 * Model (Sec. 2): y(n,f) = x1(n,f) + x2(n,f) in C^M, x_j ~ CN(0, v_j(n,f) S_j(f)), with N
 * frames and F frequency bins; both forms maximise the likelihood of Eq. (like).
 *
 * Conventions shared by every entry point:
 *   - Complex numbers are interleaved (re, im). complex64 = two floats, complex128 = two
 *     doubles. Matrices are row-major. Layouts (C order, last index fastest):
 *       y, x1, x2   [F][N][M]       complex64 (y may instead be FP16, see fca_problem)
 *       v           [2][F][N]       source powers v_j(n,f), j = 0 -> source 1
 *       S           [2][F][M][M]    spatial covariances S_j(f), Hermitian positive definite
 *   - Every call is asynchronous on the CUDA stream it is given (NULL = legacy default
 *     stream) unless stated otherwise. Argument errors are detected on the host and
 *     returned synchronously, before anything is enqueued.
 *   - Errors found by the GPU (a matrix that is not positive definite, a non-finite value,
 *     an eigensolver that does not converge) are recorded in a device status word, first
 *     error wins; fca_sync_status() waits for the stream and returns it. Once a state has
 *     failed, every later call on it returns FCA_ERR_STATE until fca_load() reloads it.
 *   - The library owns all EM state on the device (a copy of y, v, the parameters, and
 *     scratch). The caller owns every pointer it passes; input buffers are only read by
 *     work enqueued by the call, so they may be reused once that work has completed on the
 *     stream. Device pointers must be on the current CUDA device.
 *   - Sizes: 1 <= M <= 8, F >= 1, N >= 1, and F * N * M < 2^31.
 */
#ifndef FCA_H_
#define FCA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fca_state fca_state; /* opaque, allocated by fca_init, freed by fca_free */

typedef enum {
  FCA_OK = 0,
  FCA_ERR_ARG = 1,         /* invalid argument (host check)                               */
  FCA_ERR_CUDA = 2,        /* a CUDA runtime call failed                                  */
  FCA_ERR_NOMEM = 3,       /* device allocation failed                                    */
  FCA_ERR_NOT_PD = 4,      /* a covariance that must be positive definite is not          */
  FCA_ERR_EIG_NOCONV = 5,  /* the Jacobi eigensolver hit its sweep cap                    */
  FCA_ERR_NONFINITE = 6,   /* a NaN or infinity appeared in v, S, P or the log-likelihood */
  FCA_ERR_TIMEOUT = 7,     /* a bounded device wait ran out                               */
  FCA_ERR_STATE = 8,       /* the state failed earlier, or the call does not fit its form */
  FCA_ERR_SCRATCH = 9      /* fca_em_fast_noalloc: the problem needs more than its scratch  */
} fca_status;

enum { FCA_STORE_C64 = 0, FCA_STORE_F16_SCALED = 1 };
enum { FCA_MEM_DEVICE = 0, FCA_MEM_HOST = 1 };
enum { FCA_SEP_ALG1 = 0, FCA_SEP_FINAL_PARAMS = 1 };

/*
 * One mixture and its initial parameters (Algorithm 1, first step: "set initial values").
 *   storage = FCA_STORE_C64:         y is complex64 [F][N][M].
 *   storage = FCA_STORE_F16_SCALED:  y is FP16 pairs [F][N][M][2] holding g_f * y(n,f), and
 *                                    y_scale[f] = g_f > 0 (float [F]); the EM runs on the
 *                                    decoded mixture y16 / g_f.
 *                                    With y_scale = NULL (device location only), y is
 *                                    complex64 [F][N][M] and the library encodes it:
 *                                    g_f = (mean_{n,m} |y_m(n,f)|^2)^(-1/2) (FP64 sum, rounded
 *                                    to float; 1 for a silent bin) and g_f y(n,f) rounded
 *                                    to FP16 (round to nearest even, from the exact FP64
 *                                    product).
 *   v0:  double [2][F][N], initial v_j^(0)(n,f) > 0 (clamped to the positivity floor).
 *   S0:  complex128 [2][F][M][M], initial S_j^(0)(f), Hermitian positive definite.
 *   v0 = S0 = NULL: the seeded initial values, built on the device from `seed` and the mixture
 *        (as the EM sees it: decoded when stored as FP16):
 *          S_j^(0)(f) = b_j(f) b_j(f)^H + I, b_j(f) ~ CN(0, I_M),
 *          v_j^(0)(n,f) = max(|y(n,f)|^2, eps_f) / (2 tr S_j^(0)(f)),
 *          eps_f = 1e-12 mean_n |y(n,f)|^2,
 *        entry m of b_j(f) being draw t = f M + m of source j: the Philox4x64-10 block of
 *        counter (t, 0, 0, 0) under the key (seed, 1000 + j) (Salmon et al., SC 2011), whose
 *        words w0, w1 give u_k = (floor(w_k / 2^11) + 1/2) 2^-53 and
 *        b = sqrt(-ln u0) (cos 2 pi u1 + i sin 2 pi u1). One of v0, S0 without the other is
 *        an argument error.
 *   location: FCA_MEM_DEVICE or FCA_MEM_HOST, for all of y, y_scale, v0 and S0. Host
 *   buffers are copied with cudaMemcpyAsync; pinned host memory makes that asynchronous.
 *   seed: read only when v0 = S0 = NULL.
 */
typedef struct {
  int32_t M, F, N;
  int32_t storage;
  int32_t location;
  const void* y;
  const float* y_scale;
  const double* v0;
  const double* S0;
  uint64_t seed;
} fca_problem;

/* Allocate a state for the shapes in *p and load it (as fca_load). On success *out owns the
 * state; on failure *out is NULL and nothing stays allocated. */
fca_status fca_init(const fca_problem* p, void* cuda_stream, fca_state** out);

/* (fca_init and fca_load check on the device that the mixture and v0 are finite; a NaN or an
 * infinity is reported as FCA_ERR_NONFINITE by the next fca_sync_status. They also solve the
 * generalised eigenproblem of S0 (Eq. (GEVD)) in the same pass, so an S0_2 that is not
 * positive definite is reported as FCA_ERR_NOT_PD whichever EM form runs next. Device inputs
 * are read once, by that pass, which copies y and S0 into the state.) */

/* Reload a state with a new mixture and initial parameters of the same M, F and storage and
 * N frames, N at most the N the state was created with (its buffers are reused; later calls
 * work on the new N). Clears a failed status. The positivity floor of v is recomputed from the new y:
 * vfloor(f) = max(1e-12 * mean_{n,m} |y_m(n,f)|^2, 1e-30) (applied after every v update). */
fca_status fca_load(fca_state* s, const fca_problem* p, void* cuda_stream);

/* Run `iters` >= 0 iterations of conventional EM (Sec. 2, Eqs. (MMSE)-(Supdate)).
 * If the state's parameters are in the FastFCA form (P, Lambda), they are first converted
 * to S_j = P^-H T_j P^-1 (Eqs. (Sdiag), (recoverS)).
 * loglik_dev: NULL or device double [iters]; entry l receives log of Eq. (like) at the
 * parameters of iteration l (before that iteration's update), summed over all n and f. */
fca_status fca_em_conventional(fca_state* s, int32_t iters, double* loglik_dev, void* cuda_stream);

/* Run `iters` >= 0 iterations of FastFCA (Algorithm 1, steps 2-10). If the parameters are in
 * the conventional form (S1, S2), P and Lambda are first obtained from the generalised
 * eigenproblem of (S1, S2) (Eq. (GEVD)). loglik_dev as for fca_em_conventional. */
fca_status fca_em_fast(fca_state* s, int32_t iters, double* loglik_dev, void* cuda_stream);

/* FastFCA with the basis update of Eq. (recoverS) instead of Eq. (updatePeff), kept as a
 * cross-check of the efficient update (Sec. 3 derives both and proves them equal): every
 * iteration runs one FastFCA iteration, forms S_j = P^-H T_j P^-1 in the original basis
 * (Eqs. (Sdiag), (recoverS)) and takes P, Lambda from the generalised eigenproblem of
 * (S1, S2) afresh (Eq. (GEVD)). Same contract and outputs as fca_em_fast (equal up to
 * rounding); three kernel launches per iteration. */
fca_status fca_em_fast_recover(fca_state* s, int32_t iters, double* loglik_dev, void* cuda_stream);

/* Posterior means (MMSE source images, Eq. (MMSE); Algorithm 1, last step) into caller-owned
 * device buffers x1_dev, x2_dev, complex64 [F][N][M].
 *   mode FCA_SEP_ALG1:         the E-step of the last iteration run, i.e. the parameters of
 *                              iteration L-1 (the initial parameters if no iteration ran);
 *   mode FCA_SEP_FINAL_PARAMS: one more E-step with the current parameters.
 * The FastFCA form returns mu1 = P^-H mut1 and mu2 = y - mu1 (y = x1 + x2, Sec. 2); the
 * conventional form returns mu_j = v_j S_j (v1 S1 + v2 S2)^-1 y for j = 1, 2. */
fca_status fca_separate(fca_state* s, void* x1_dev, void* x2_dev, int32_t mode, void* cuda_stream);

/* Current parameters. v_dev: NULL or device float [2][F][N] (enqueued copy). S_host: NULL or
 * host complex128 [2][F][M][M]; when given, the call synchronises the stream (S is formed
 * on the device from (P, Lambda) in the FastFCA form, Eqs. (Sdiag), (recoverS)). */
fca_status fca_get_params(fca_state* s, float* v_dev, double* S_host, void* cuda_stream);

/* Per-frequency log-likelihood of the last EM call: out receives double [L][F] (L = that
 * call's iteration count), entry (l, f) being the Eq. (like) term of bin f summed over the N
 * frames at the parameters of iteration l. out may be device or host memory; a host
 * destination synchronises the stream. Returns FCA_ERR_STATE if no EM call ran since the
 * last load. *iters_out (may be NULL) receives L; with out == NULL the call only reports L. */
fca_status fca_loglik_bins(fca_state* s, double* out, int32_t* iters_out, void* cuda_stream);

/* Synchronise the stream and return the first device-side error of this state (FCA_OK if
 * none). */
fca_status fca_sync_status(fca_state* s, void* cuda_stream);

/* Precision of FastFCA's per-frequency generalised eigenproblem (Algorithm 1, step 8: the
 * Cholesky factor of St2, the Hermitian Jacobi eigensolver of L^-1 St1 L^-H and Q = L^-H U of
 * Eq. (GEVDeff5) and the Appendix), together with the cross-warp merge of the Gram sums that
 * feed it (Eq. (updateStildeeff)).
 *   FCA_GEVD_FP32:    both in FP32.
 *   FCA_GEVD_FP64:    both in FP64 (the per-warp partial sums over frames stay FP32).
 *   FCA_GEVD_REFINED: the merge as compensated FP32 pairs (about twice FP32's precision); an
 *                     FP32 solve (Newton-type steps from the identity, or the FP32 Cholesky
 *                     and Jacobi solve after a poor start), then one refinement step of Q
 *                     against the merged Grams' pairs with compensated FP32 residuals, and
 *                     a second, FP64 step after a poor start: Q^H St2 Q = I and Q^H St1 Q
 *                     diagonal to second order in the FP32 solve's residuals.
 * In the FP64 and refined modes the next basis P Q for the bin pass is a compensated FP32
 * product of P and Q each split into two FP32 parts, accurate to FP32 in every entry. The bin
 * pass is FP32 and the basis P, log-likelihood and log det S2 are kept in FP64 in every mode.
 * Batches (fca_batch_*) run the FP32 or the refined mode. */
enum { FCA_GEVD_FP32 = 0, FCA_GEVD_FP64 = 1, FCA_GEVD_REFINED = 2 };
#define FCA_GEVD_DEFAULT FCA_GEVD_REFINED /* of new states, batches, server requests and
                                             fca_em_fast_noalloc */
#define FCA_MAX_SWEEPS_LIMIT 1000

/* How the conventional EM kernel (fca_em_conventional; Sec. 2, Eqs. (MMSE)-(Supdate)) maps its
 * per-point matrix work onto threads; the arithmetic and results are the same up to rounding.
 *   FCA_CONV_THREAD: one thread per time-frequency point, every per-point matrix (the Cholesky
 *                    factor of Rx, L^-1 S_j, C) in its registers; for M >= 6 they exceed the
 *                    register file and spill to local memory.
 *   FCA_CONV_GROUP:  eight lanes per point (four for M <= 4), each owning one row or column of
 *                    those matrices; no spills at any M.
 *   FCA_CONV_AUTO:   the faster layout as measured on GB300, FCA_CONV_THREAD at every M
 *                    (the default). */
enum { FCA_CONV_AUTO = 0, FCA_CONV_THREAD = 1, FCA_CONV_GROUP = 2 };

/* Choose the conventional kernel's layout for this state's later fca_em_conventional calls.
 * Host only; returns at once. FCA_ERR_ARG for an unknown layout. */
fca_status fca_set_conv_layout(fca_state* s, int32_t layout);

/* Set the eigensolver precision (FCA_GEVD_FP32, _FP64 or _REFINED) and its cap on Jacobi sweeps
 * per eigenproblem, 0 <= max_sweeps <= FCA_MAX_SWEEPS_LIMIT (a new state has the library
 * default precision and a cap of 30). A solve that needs more sweeps stops, records
 * FCA_ERR_EIG_NOCONV in the status word and leaves the state failed (the kernel returns; no
 * wait). Applies to every later eigenproblem of the state: those of fca_em_fast,
 * fca_em_fast_recover and fca_load. A state loaded since its last EM call solves the
 * eigenproblem of S0 again, with these settings, at the next fca_em_fast. Host only;
 * returns at once. */
fca_status fca_set_eigensolver(fca_state* s, int32_t precision, int32_t max_sweeps);

/* Release the state and all its device memory. Synchronises the device first. NULL is a
 * no-op. */
void fca_free(fca_state* s);

/* Device duration (milliseconds) of the fused EM kernel launched by the last
 * fca_em_fast / fca_em_conventional call, from CUDA events recorded on that call's stream
 * just before and after the launch. Waits for the kernel to finish. FCA_ERR_STATE if no EM
 * call ran since the last load. */
fca_status fca_last_em_kernel_ms(fca_state* s, float* ms);

/* Number of CUDA kernels this library has launched in this process (all states). */
uint64_t fca_kernel_launches(void);

/* Measured arithmetic peaks of the current device, for rating the kernels against (the paper
 * has no counterpart): FP32 and FP64 fused multiply-add throughput in TFLOP/s (2 flops per
 * FMA), from a kernel of independent FMA chains on every SM timed with CUDA events (about
 * 0.3 s). Synchronous; allocates 64 bytes of device memory for the duration of the call. */
fca_status fca_measure_peaks(double* fp32_tflops, double* fp64_tflops);

/* Size of the fixed device scratch array behind fca_em_fast_noalloc (bytes). */
#define FCA_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * FastFCA without any device allocation. The paper has no counterpart: this is a way to run
 * the same kernels for callers that must not allocate device memory once running -- a
 * real-time audio loop (cudaMalloc / cudaFree may synchronise the device and take unbounded
 * time) or a host application that hands out device memory only through its own pool.
 *
 * Runs the whole job of fca_init + fca_em_fast + fca_separate(FCA_SEP_ALG1) on caller-owned
 * device buffers (complex64 storage only):
 *   y_dev       in   complex64 [F][N][M]
 *   v0_dev      in   double [2][F][N], initial v (clamped to the positivity floor)
 *   S0_dev      in   complex128 [2][F][M][M], initial S, Hermitian positive definite
 *   iters       in   number of FastFCA iterations L >= 0
 *   v_dev       out  float [2][F][N], v after the last iteration
 *   x1_dev,
 *   x2_dev      out  complex64 [F][N][M], posterior means of Algorithm 1's output
 *   loglik_dev  out  NULL or double [iters], as for fca_em_fast
 * Everything else lives in one file-scope device array of FCA_NOALLOC_SCRATCH_BYTES, which
 * every GPU that loads the library holds until the process exits. The problem must fit:
 * 256-byte-aligned regions of 4F (floor) + 2 x (16 F M^2 + 8 F M + 8 F) (basis, eigenvalues,
 * log-determinants, current and previous) + 8 F max(L, 1) (per-bin log-likelihood) + 8 F N
 * (previous v) + 16 F M^2 + 4 F M (separation) bytes, plus 256; larger problems return
 * FCA_ERR_SCRATCH before any work is enqueued (M=4, F=513, N=1000, L=50 needs about 5 MB).
 * The buffers are read and written in place, so they must be aligned: y_dev and S0_dev to
 * 16 bytes, v0_dev, x1_dev, x2_dev and loglik_dev to 8, v_dev to 4 (cudaMalloc'd buffers
 * and whole tensors are); otherwise FCA_ERR_ARG before any work is enqueued.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine). The
 * first call on a device looks up the array's device address there (cudaGetSymbolAddress,
 * with that device current); under lazy module loading (CUDA_MODULE_LOADING=LAZY, the
 * default) that first lookup may also load the library's module and place the array, which
 * allocates. Make one successful call on each device before entering a phase where
 * allocation is not allowed, and before any stream capture on that device.
 * All calls share the array, so calls whose work overlaps on the GPU (other host threads,
 * other streams) race; the call therefore synchronises `cuda_stream` before returning, and
 * returns the first device-side error of this call (FCA_OK if none).
 */
fca_status fca_em_fast_noalloc(int32_t M, int32_t F, int32_t N, const void* y_dev,
                               const double* v0_dev, const double* S0_dev, int32_t iters,
                               float* v_dev, void* x1_dev, void* x2_dev, double* loglik_dev,
                               void* cuda_stream);

/* ------------------------------------------------------------------------------------------
 * Batches: many mixtures, each with its own M, F and N, in one job.
 *
 * Every frequency bin of every mixture is an independent EM problem (all updates of Sec. 2
 * and Sec. 3 are indexed by the bin, and Eq. (like) factorises over bins and mixtures), so a
 * batch runs all bins of all mixtures together: one fused EM kernel per channel count (bins
 * ordered longest first), the channel-count groups on concurrent streams, and optionally the
 * whole job captured once as a CUDA graph and replayed with a single graph launch. Each
 * mixture's results are those of the one-mixture entry points on the same inputs (the same
 * kernels and the same fixed-order reductions; a bin's arithmetic does not depend on its
 * neighbours).
 *
 * Packed layouts (C order, mixtures back to back in the order given):
 *   y, x1, x2  complex64: mixture k's [F_k][N_k][M_k] block starts at element
 *              sum_{k' < k} F_k' N_k' M_k'
 *   v0, v      mixture k's [2][F_k][N_k] block starts at sum_{k' < k} 2 F_k' N_k'
 *   S0         complex128: mixture k's [2][F_k][M_k][M_k] starts at sum_{k' < k} 2 F_k' M_k'^2
 *   loglik     double [count][iters]
 * ------------------------------------------------------------------------------------------ */
typedef struct fca_batch fca_batch; /* opaque, allocated by fca_batch_init */

enum { FCA_FORM_FAST = 0, FCA_FORM_CONVENTIONAL = 1 };

typedef struct {
  int32_t count;        /* number of mixtures, >= 1                                          */
  const int32_t* M;     /* host int32 [count], 1..8; F, N: host int32 [count], >= 1, with   */
  const int32_t* F;     /*   F_k N_k M_k < 2^31 for every mixture                           */
  const int32_t* N;
  int32_t location;     /* FCA_MEM_DEVICE or FCA_MEM_HOST, for y, v0 and S0                 */
  const void* y;        /* complex64, packed (above)                                        */
  const double* v0;     /* initial v_j^(0)(n,f) > 0, packed                                 */
  const double* S0;     /* initial S_j^(0)(f), Hermitian positive definite, packed          */
} fca_batch_problem;

/* Allocate a batch for the shapes in *p and load it (as fca_batch_load). The device memory
 * held is about 8 sum F N M (mixture copy) + 12 sum 2 F N (source powers) bytes plus small
 * per-bin arrays. On failure *out is NULL and nothing stays allocated. */
fca_status fca_batch_init(const fca_batch_problem* p, void* cuda_stream, fca_batch** out);

/* Load new mixtures and initial parameters of the same shapes (count, M, F, N). Computes the
 * positivity floor of v from the new y as fca_load does, clears a failed status and keeps the
 * tuned launch shapes. Host v0 is staged through stream-ordered device memory. */
fca_status fca_batch_load(fca_batch* b, const fca_batch_problem* p, void* cuda_stream);

/* The whole job from the loaded initial parameters: 0 <= iters <= 65535 EM iterations of `form`
 * (FCA_FORM_FAST: Algorithm 1, from the generalised eigenproblem of S0; FCA_FORM_CONVENTIONAL:
 * Sec. 2) for every mixture, then the posterior means of Algorithm 1's output (the E-step of
 * iteration L-1; the initial parameters when iters = 0) into the packed device buffers x1_dev,
 * x2_dev. loglik_dev: NULL or device double [count][iters] (Eq. (like) at the parameters of
 * each iteration, per mixture). v_dev: NULL or device float, packed like v0: v after the last
 * iteration. The job depends only on the loaded inputs, so it can be run again.
 * use_graph != 0: the first call with given (form, iters, buffers) captures the job into a CUDA
 * graph (on an internal stream; the call must not itself be inside a stream capture) and
 * every call launches that graph on cuda_stream; other arguments re-capture. Asynchronous. */
fca_status fca_batch_run(fca_batch* b, int32_t form, int32_t iters, double* loglik_dev,
                         void* x1_dev, void* x2_dev, float* v_dev, int32_t use_graph,
                         void* cuda_stream);

/* Autotune the FastFCA launch shape of every channel-count group: threads per CTA (64 in the
 * FP32 eigensolver mode, 128, 256) and how much shared memory a CTA may take to keep its bin's mixture and source powers
 * on chip (bins that do not fit stream them from memory every iteration). Each candidate runs
 * min(iters, 4) iterations on a sample of the group's bins (at most 8192) spanning its range
 * of lengths, four times in turn with the others after a warm-up; the one with the best time
 * is kept. As the groups of a job share the GPU, the tuned set is then checked against the
 * default shapes and against all bins streaming, with whole EM passes of all groups at once,
 * and the fastest set is kept for later runs. Synchronises the stream. Overwrites the EM state (not the
 * loaded inputs) and clears the status word (the timing runs' own status is not a result), so run it
 * before fca_batch_run, not between a run and the use of its outputs. */
fca_status fca_batch_tune(fca_batch* b, int32_t iters, void* cuda_stream);

/* Launch shape of the channel-count group M: its number of bins, threads per CTA and the
 * dynamic shared memory per CTA. FCA_ERR_ARG if no mixture has M channels. */
fca_status fca_batch_shape(const fca_batch* b, int32_t M, int32_t* bins, int32_t* threads,
                           int32_t* res_bytes);

/* Set the launch shape of the channel-count group M (e.g. to reuse shapes tuned earlier):
 * threads per CTA 64 (FP32 eigensolver only), 128 or 256, and res_bytes (0..200 KB) of
 * dynamic shared memory per CTA,
 * bins needing at most that staying on chip. FCA_ERR_ARG if no mixture has M channels. */
fca_status fca_batch_set_shape(fca_batch* b, int32_t M, int32_t threads, int32_t res_bytes);

/* Parameters of mixture k (0 <= k < count) after the last fca_batch_run, into host memory:
 *   S_host    NULL or complex128 [2][F_k][M_k][M_k]: S_j(f) (FastFCA: formed from (P, Lambda)
 *             by Eqs. (Sdiag), (recoverS); conventional: the last M-step's S_j, Eq. (Supdate));
 *   llf_host  NULL or double [L][F_k], L the last run's iteration count: entry (l, f) is the
 *             Eq. (like) term of bin f summed over the mixture's frames at the parameters of
 *             iteration l (the batch's per-mixture log-likelihood is its sum over f).
 * Synchronises the stream; FCA_ERR_STATE before any run (or, for llf_host, after a run of
 * zero iterations). The FastFCA form allocates a temporary of 32 F_g M_k^2 bytes for the
 * channel-count group's F_g bins. */
fca_status fca_batch_get_params(fca_batch* b, int32_t k, double* S_host, double* llf_host,
                                void* cuda_stream);

/* Eigensolver precision of the batch's FastFCA runs (FCA_GEVD_FP32 or FCA_GEVD_REFINED; see
 * fca_set_eigensolver) and its Jacobi sweep cap (0..FCA_MAX_SWEEPS_LIMIT). A new batch has the
 * library default. The refined mode runs 128 or 256 threads per CTA (fca_batch_set_shape
 * refuses 64 there). Changing the precision resets the launch shapes to the defaults (tune
 * again) and drops the captured graph. Host only. */
fca_status fca_batch_set_eigensolver(fca_batch* b, int32_t precision, int32_t max_sweeps);

/* Synchronise the stream and return the first device-side error of this batch. After an
 * error every run returns FCA_ERR_STATE until fca_batch_load. */
fca_status fca_batch_sync_status(fca_batch* b, void* cuda_stream);

/* Release the batch (synchronises the device first). NULL is a no-op. */
void fca_batch_free(fca_batch* b);

/* ------------------------------------------------------------------------------------------
 * Serving: requests of one mixture each, arriving at any time, run concurrently.
 *
 * A server owns one device-memory arena (allocated once, at creation), a pool of CUDA streams
 * and a worker thread. Submitted requests wait in arrival order; the worker admits the oldest
 * as soon as its device memory fits in the arena and a stream is free (while the oldest waits
 * for memory, a later request that fits may be admitted ahead of it, at most 8 times per
 * waiting request, so a large request neither blocks the small ones behind it nor starves),
 * enqueues its whole job
 * on that stream (copies of the inputs to the device, the one-mixture EM kernels of Sec. 2 or
 * Sec. 3 / Algorithm 1, copies of the outputs back), and retires it when the stream's event
 * completes, returning its memory and stream to the pools. Requests admitted while others run
 * overlap them on the GPU, and each request's results equal those it gets alone (its kernels
 * are the one-mixture ones; bins and mixtures are independent). No device memory is allocated
 * per request. Every wait is on the host, with a time limit where the caller gives one.
 * ------------------------------------------------------------------------------------------ */
typedef struct fca_server fca_server; /* opaque, created by fca_server_create */

typedef struct {
  int64_t device_bytes;  /* size of the device-memory arena for requests in flight, >= 4096   */
  int32_t max_inflight;  /* requests on the GPU at once (one CUDA stream each), 1..64        */
} fca_server_config;

typedef struct {
  int32_t M, F, N;       /* 1 <= M <= 8, F >= 1, N >= 1, F N M < 2^31                           */
  int32_t form;          /* FCA_FORM_FAST or FCA_FORM_CONVENTIONAL                               */
  int32_t iters;         /* EM iterations L >= 0                                                 */
  const void* y;         /* in: complex64 [F][N][M]; host (pinned for asynchronous copies) or device */
  const double* v0;      /* in: double [2][F][N], initial v                                      */
  const double* S0;      /* in: complex128 [2][F][M][M], initial S, Hermitian positive definite  */
  void* x1;              /* out: complex64 [F][N][M], posterior means of Algorithm 1's output    */
  void* x2;
  double* loglik;        /* out: NULL or double [iters], Eq. (like) at each iteration's parameters */
  float* v;              /* out: NULL or float [2][F][N], the source powers after the last iteration */
} fca_request;           /* every buffer is the caller's and must stay valid until the wait returns */

typedef struct {
  fca_status status;     /* the request's result (device-side errors included)                   */
  double t_submit;       /* steady-clock seconds (CLOCK_MONOTONIC) of submission,                */
  double t_admit;        /*   of admission (memory and stream granted),                          */
  double t_done;         /*   and of completion (outputs copied back)                            */
} fca_request_info;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t queued, in_flight;
  int64_t max_in_flight;               /* most requests on the GPU at once so far              */
  uint64_t bytes_in_use, bytes_peak, bytes_budget;
} fca_server_counters;

/* Create a server on the current device: allocates the arena, the streams and the worker. */
fca_status fca_server_create(const fca_server_config* cfg, fca_server** out);

/* Device bytes one request of these shapes takes from the arena (0 for invalid shapes). */
size_t fca_server_request_bytes(int32_t M, int32_t F, int32_t N, int32_t iters);

/* Queue a request; *ticket identifies it. FCA_ERR_NOMEM if it could never fit the arena;
 * FCA_ERR_ARG for invalid shapes or NULL buffers. Returns at once. */
fca_status fca_server_submit(fca_server* s, const fca_request* r, uint64_t* ticket);

/* Wait for a request (timeout_ms < 0: no limit) and return its status; *info (may be NULL)
 * receives its status and times. FCA_ERR_TIMEOUT if the limit passes first (the ticket stays
 * valid); each ticket can be waited for successfully once. */
fca_status fca_server_wait(fca_server* s, uint64_t ticket, int64_t timeout_ms,
                           fca_request_info* info);

/* Counters and arena use. */
fca_status fca_server_stats(fca_server* s, fca_server_counters* out);

/* Finish every queued and running request, then release the server. NULL is a no-op. */
void fca_server_destroy(fca_server* s);

/* ------------------------------------------------------------------------------------------
 * STFT front-end: time-domain signals to the mixture y(n,f) of Sec. 2 and back.
 *
 * The analysis of the paper's experiments (Table 1): frames of W samples (W a power of two,
 * 16..8192), shift H (1 <= H <= W/2), square-root periodic Hann window w[k] = sin(pi k / W),
 * F = W/2 + 1 bins up to Nyquist (W = 1024, H = 512 gives Table 1's F = 513). Frames are
 * centred: frame n covers samples [n H - W/2, n H + W/2), zero outside the signal, so there
 * are N = T / H + 1 frames (fca_stft_frames). y(n,f) = sum_k w[k] x(n H - W/2 + k)
 * exp(-2 pi i f k / W). Synthesis is weighted overlap-add with the same window,
 * x(t) = sum_n w u_n(t) / sum_n w^2, which inverts the analysis exactly.
 * ------------------------------------------------------------------------------------------ */

/* Frames N = T / H + 1 of a T-sample signal (0 for invalid sizes). */
int64_t fca_stft_frames(int64_t T, int32_t W, int32_t H);

/* x_dev: device float [M][T] (1 <= M <= 8) -> y_dev: device complex64 [F][N][M] (the layout of
 * fca_problem.y). Asynchronous. */
fca_status fca_stft(int32_t M, int64_t T, const float* x_dev, int32_t W, int32_t H, void* y_dev,
                    void* cuda_stream);

/* y_dev: device complex64 [F][N][M] with N = fca_stft_frames(T, W, H) -> x_dev: device float
 * [M][T]; each frame is the inverse DFT of its spectrum extended by Hermitian symmetry (a real
 * frame; the imaginary parts of the DC and Nyquist bins are dropped, as a real signal has none).
 * frames_dev: caller-provided device scratch of N * M * W floats (the windowed frames
 * before the overlap-add). Each output sample is gathered from its frames in a fixed order
 * (bitwise reproducible). Asynchronous. */
fca_status fca_istft(int32_t M, int32_t N, const void* y_dev, int32_t W, int32_t H,
                     float* frames_dev, float* x_dev, int64_t T, void* cuda_stream);

/* Static description of a status code. */
const char* fca_status_string(fca_status st);

/* Library build identifier (compile-time target and version). */
const char* fca_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FCA_H_ */
