/*
 * cgl.h - C ABI of libcgl: constant-step exponential integrators for the
 * semidiscretised complex Ginzburg-Landau (CGL) equation on one GB300 GPU.
 *
 * Method: Caliari & Cassini, "Efficient simulation of complex Ginzburg-Landau
 * equations using high-order exponential-type methods" (arXiv 2403.02816).
 *
 *   u_t = (a1 + i b1) Lap u + a2 u + (a3 + i b3)|u|^2 u + (a4 + i b4)|u|^4 u
 *                                                                  (Sec. 1, eq. 1)
 * on a box (lo_1,hi_1) x ... x (lo_d,hi_d), d = 1..3, semidiscretised as
 * u' = K u + g(u) with K = A_d (+) ... (+) A_1 a Kronecker sum (Sec. 1, eq. 2).
 *   - Dirichlet/Neumann directions: 2nd-order finite differences; the linear
 *     flow exp(c tau K) is the Tucker operator U x_1 e^{c tau A_1} ... x_d
 *     e^{c tau A_d} (Sec. 3.1, eq. Tucker), one mu-mode product per direction
 *     with a dense n_mu x n_mu factor computed once per distinct c.
 *   - Periodic directions: Fourier pseudospectral; exp(c tau K) is a pointwise
 *     multiplication in Fourier space (Sec. 3.2), done with an in-house FFT.
 *
 * Conventions for every entry point:
 *   - Return value: 0 (CGL_OK) or a negative cgl_status.  Nothing throws or
 *     aborts across the ABI; cgl_last_error() gives a message for the calling
 *     thread's most recent failure.
 *   - Fields are caller-owned device buffers of N = n_1*...*n_d complex
 *     numbers, interleaved (re, im), double2 for CGL_F64 and float2 for
 *     CGL_F32, stored with index 1 fastest: the paper's vec(U) (Sec. 3.1).
 *     A PyTorch tensor of shape (n_d, ..., n_1), contiguous, has this layout.
 *   - Streams are passed as void* (a cudaStream_t; NULL = legacy default).
 *     Work is enqueued asynchronously unless an entry point says otherwise.
 *   - A plan owns its factors and workspace (device memory it allocates at
 *     creation and frees in cgl_plan_destroy).  One plan must not run on two
 *     streams at once.
 */
#ifndef CGL_H
#define CGL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cgl_plan cgl_plan;

/* Boundary condition per direction. */
enum cgl_bc { CGL_BC_DIRICHLET = 0, CGL_BC_NEUMANN = 1, CGL_BC_PERIODIC = 2 };

/* Time integrators (Sec. 2). */
enum cgl_scheme {
    CGL_STRANG = 0,   /* eq. Strang: phi_{tau/2} e^{tau K} phi_{tau/2}, order 2            */
    CGL_SPLIT4 = 1,   /* eq. Richardson: 4/3 S_{tau/2}S_{tau/2} - 1/3 S_tau, order 4        */
    CGL_LAWSON4 = 2,  /* eq. lawson4 (if4), order 4                                         */
    CGL_RK4 = 3,      /* eq. RK4 on u' = K u + g(u)                                         */
    CGL_LAWSON2 = 4,  /* eq. lawson2b (if2), order 2                                        */
    CGL_RK2 = 5,      /* eq. RK2 (Heun)                                                     */
    CGL_STRANG3T = 6, /* strang_3t (Sec. 4.3): phi^q phi^c e^{tau K} phi^c phi^q, exact      */
                      /* cubic and quintic sub-flows, order 2                                */
    CGL_SPLIT4_3T = 7 /* split4_3t (Sec. 4.3): Richardson extrapolation of strang_3t, order 4 */
};

/* Arithmetic of the state and of the time-stepping kernels.  The factors
 * exp(c tau A_mu) are always computed in FP64 and rounded once.
 *   CGL_F64    complex128 state, FP64 kernels.
 *   CGL_F32    complex64 state, FP32 kernels.
 *   CGL_BF16X3 complex64 state; the mu-mode products run on the tensor cores
 *              with each operand split into three BF16 parts and FP32
 *              accumulation (about FP32 accuracy); pointwise work in FP32.
 *              Finite differences only, every n_mu <= 256 (internally the
 *              factors are zero-padded to a multiple of 16 and the BF16
 *              planes' first direction to a multiple of 64).
 *   CGL_F64_TC complex128 state; FP64-accurate mu-mode products on the
 *              tensor cores by the Ozaki splitting: each fiber of the state
 *              and each row of the factor is scaled by a power of two and
 *              cut into seven signed 7-bit digits, exact in BF16; the 28
 *              digit products with a + b <= 6 accumulate exactly (levels
 *              0..5) in FP32 tensor memory and are combined in integer
 *              arithmetic, so a product is accurate to about 2^-46 of the
 *              scales (FP64-class).  Pointwise work in FP64.  Finite
 *              differences only, every n_mu <= 256; not for batches or the
 *              coupled system. */
enum cgl_precision { CGL_F64 = 0, CGL_F32 = 1, CGL_BF16X3 = 2, CGL_F64_TC = 3 };

enum cgl_status {
    CGL_OK = 0,
    CGL_EINVAL = -1,        /* invalid argument                                   */
    CGL_ENOMEM = -2,        /* device allocation failed                           */
    CGL_ECUDA = -3,         /* a CUDA runtime call failed (see cgl_last_error)    */
    CGL_EUNSUPPORTED = -4,  /* valid but not implemented (e.g. RK4 with FD)       */
    CGL_ETIMEOUT = -5,      /* a bounded device-side wait gave up                 */
    CGL_ENONFINITE = -6     /* a step produced Inf/NaN (finite-time blow-up)      */
};

/*
 * Create a plan: validates the problem, builds A_mu = (a1+i b1) D2_mu + a2/d
 * (Sec. 1 after eq. 2; 2nd-order FD or Fourier symbol, Sec. 3.2), computes the
 * factors exp(c tau A_mu) in FP64 on the GPU for every distinct c the scheme
 * needs (Strang/Lawson2/strang_3t: c = 1; split4/split4_3t: 1 and 1/2;
 * Lawson4: 1/2), and sizes
 * the workspace.
 *   out        receives the plan (set to NULL on failure).
 *   d          1, 2 or 3.
 *   n[d]       grid sizes, n_mu >= 2.  Periodic: n_mu <= 2048 with no prime
 *              factor above 7 (powers of two: radix-4/2 passes; others:
 *              mixed-radix 4, 2, 3, 5, 7 passes).  Finite differences:
 *              n_mu <= 1024.
 *   bc[d]      cgl_bc per direction; all periodic or none (else EUNSUPPORTED).
 *   lo[d],hi[d] domain, hi > lo.
 *   a1 > 0 (Sec. 1 assumption); b1, a2, a3, b3, a4, b4 any finite values
 *              (zeros allowed).  a4 = b4 = 0 selects the cubic model whose
 *              nonlinear flow is exact (eq. exsolcub); otherwise the flow is
 *              one RK4 step of u' = g(u) (Sec. 4.3).
 *   tau        constant step, > 0 and finite.
 *   scheme     cgl_scheme.  CGL_RK4/CGL_RK2 apply K directly: a pseudospectral
 *              multiply (periodic) or the finite-difference stencil of
 *              eq. kronsumv; explicit, so tau must respect their stability
 *              limit (about 2.8 / |lambda_max(K)| for RK4).
 *   precision  cgl_precision.
 *   stream     stream used for the set-up work; the call returns after it
 *              has completed.
 * Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA.
 */
int cgl_plan_create(cgl_plan** out, int d, const int64_t* n, const int* bc,
                    const double* lo, const double* hi,
                    double a1, double b1, double a2, double a3, double b3,
                    double a4, double b4, double tau, int scheme, int precision,
                    void* stream);

/*
 * Create a plan whose linear part K = A_d (+) ... (+) A_1 uses caller-supplied
 * direction matrices (finite differences of any order or stencil, e.g. the
 * paper's fourth-order matrices of cgl_fd4_matrix scaled by (a1 + i b1) plus
 * a2/d, Sec. 4.1.1 and 4.2); the factors exp(c tau A_mu) are computed as in
 * cgl_plan_create.
 *   A[d]       host pointers; A[mu] holds the complex n_mu x n_mu matrix in
 *              column-major order as (re, im) doubles (2 n_mu^2 doubles),
 *              copied during the call.  Finite entries.
 *   a3..b4, tau, precision, stream: as cgl_plan_create.
 *   scheme     an exponential scheme (strang, split4, lawson4, lawson2,
 *              strang_3t, split4_3t); CGL_RK4/CGL_RK2 give EUNSUPPORTED.
 * Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA.
 */
int cgl_plan_create_ex(cgl_plan** out, int d, const int64_t* n, const double* const* A,
                       double a3, double b3, double a4, double b4, double tau, int scheme,
                       int precision, void* stream);

/*
 * Create a plan for the coupled two-field system (Sec. 4.5, eq. coupled):
 *   u_t =  a0 d_x1 u + (a1+i b1) Lap u + a2 u + (a3+i b3)|u|^2 u
 *          + (a4+i b4)|u|^4 u + a5 |v|^2 u,
 *   v_t = -a0 d_x1 v + (a1+i b1) Lap v + a2 v + (a3+i b3)|v|^2 v
 *          + (a4+i b4)|v|^4 v + a5 |u|^2 v,
 * periodic in every direction (Fourier pseudospectral; sizes as for
 * cgl_plan_create).  K is block diagonal: each field has its own separable
 * symbol, the advection term i (+-a0) kappa_1 on direction 1 (0 at the
 * Nyquist mode of an even n_1, which keeps the system's mirror symmetry
 * x1 -> L - x1, u <-> v).  The nonlinear sub-flow is one RK4 step of the
 * coupled pointwise system.  scheme: CGL_STRANG, CGL_SPLIT4, CGL_LAWSON4,
 * CGL_LAWSON2 (chains of sweeps that carry u and v together), CGL_RK4 or
 * CGL_RK2 (one sweep per field and stage; explicit, so tau must respect their
 * stability limit); the three-term splittings give EUNSUPPORTED.  precision:
 * CGL_F64 or CGL_F32.
 * The field passed to cgl_step / cgl_step_host holds u (N values) followed
 * by v (N values), each in the single-field layout; cgl_linear_flow applies
 * exp(c tau K) to both.  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA.
 */
int cgl_plan_create_coupled(cgl_plan** out, int d, const int64_t* n, const double* lo, const double* hi,
                            double a0, double a1, double b1, double a2, double a3, double b3,
                            double a4, double b4, double a5, double tau, int scheme, int precision,
                            void* stream);

/*
 * The paper's fourth-order finite-difference d^2/dx^2 matrix on (lo, hi),
 * real n x n, column-major, written to host memory `out` (n*n doubles).
 *   right_bc = CGL_BC_DIRICHLET (Sec. 4.1.1): homogeneous Dirichlet at both
 *     ends, internal nodes lo + j h, j = 1..n, h = (hi - lo)/(n + 1); centred
 *     rows (-1, 16, -30, 16, -1)/(12 h^2), one-sided first row
 *     (-15, -4, 14, -6, 1)/(12 h^2) and its mirror image as the last row.
 *   right_bc = CGL_BC_NEUMANN (Sec. 4.2): Dirichlet at lo, homogeneous
 *     Neumann at hi, semi-internal nodes lo + j h, j = 1..n, h = (hi - lo)/n;
 *     first row as above, last rows (1, -6, 14, -4, -15, 10)/(12 h^2) and
 *     (1, -8/3, -6, 56, -145/3)/(12 h^2).
 * Host only (no device work).  Errors: EINVAL (n < 6, lo >= hi, other bc).
 */
int cgl_fd4_matrix(int n, double lo, double hi, int right_bc, double* out);

/*
 * Advance the caller-owned device field u (N complex values, layout above)
 * by nsteps constant steps of the plan's scheme, in place.  Asynchronous on
 * `stream`.  The step sequence is recorded once per (plan, u) pair into a
 * CUDA graph and replayed; the first call for a new u pointer therefore
 * captures on an internal stream.  nsteps >= 0.
 * Errors: EINVAL (NULL plan/u, nsteps < 0), ECUDA.
 */
int cgl_step(cgl_plan* plan, void* u, int64_t nsteps, void* stream);

/*
 * Same as cgl_step for a HOST buffer u_host (N complex values): copies it to
 * a plan-owned device field, advances nsteps, copies the result back.
 * Synchronous: returns after the result is in u_host.  u_host may be pinned
 * (fast path) or pageable.
 */
int cgl_step_host(cgl_plan* plan, void* u_host, int64_t nsteps, void* stream);

/* Destroy a plan and free its device memory.  NULL is accepted. */
int cgl_plan_destroy(cgl_plan* plan);

/*
 * Fault injection for tests (the paper has no counterpart): after `after`
 * more device allocations by plans, batches and correctors (process-wide),
 * the next one fails as if cudaMalloc had, and the call that made it
 * returns CGL_ENOMEM after freeing what it had allocated; the injection is
 * then disarmed.  after = -1 disarms it.  Errors: EINVAL (after < -1).
 */
int cgl_inject_alloc_failure(long long after);

/*
 * Apply one linear flow exp(c tau K) to the device field u in place
 * (eq. Tucker / Sec. 3.2), for c equal to one of the plan's factor values
 * (1 or 0.5; EINVAL otherwise).  Asynchronous on `stream`.
 */
int cgl_linear_flow(cgl_plan* plan, double c, void* u, void* stream);

/*
 * Copy the plan's FP64 factor for value c and direction mu (0-based) to host
 * memory: FD gives exp(c tau A_mu) as n_mu x n_mu complex (re,im) doubles in
 * column-major order (2*n_mu*n_mu doubles); periodic gives the diagonal
 * exp(c tau a_mu(kappa)) in FFT order (2*n_mu doubles).  Synchronous.
 */
int cgl_plan_factor(cgl_plan* plan, double c, int mu, double* host_out);

/* Sizes: bytes of one field, of the plan's workspace, and kernel launches
 * enqueued per time step.  Any pointer may be NULL. */
int cgl_plan_info(const cgl_plan* plan, size_t* field_bytes, size_t* workspace_bytes,
                  int* launches_per_step);

/*
 * Read (synchronising `stream`) and clear the plan's device status word:
 * returns CGL_OK, or CGL_ENONFINITE if any step since the last call wrote a
 * non-finite value.
 */
int cgl_last_device_status(cgl_plan* plan, void* stream);
/* (A bounded device-side wait that gave up is reported as CGL_ETIMEOUT.) */

/*
 * Per-kernel timing (CUDA events around every launch) of nsteps steps run
 * without the graph.  Fills up to max_kernels records, sets *count.
 * Synchronous.  flops / bytes are the algorithmic counts per launch (FFT
 * 5 n log2 n per pencil, 8 n real flops per mode-product output point, one
 * read and one write per field touched).
 */
typedef struct cgl_kernel_time {
    char name[48];
    int64_t launches;
    double total_ms;
    double flops;   /* algorithmic flops summed over the launches */
    double bytes;   /* algorithmic DRAM bytes summed over the launches */
} cgl_kernel_time;
int cgl_profile_step(cgl_plan* plan, void* u, int64_t nsteps, void* stream,
                     cgl_kernel_time* out, int max_kernels, int* count);

/*
 * Relative errors of x against y over `count` complex values of `precision`
 * (Sec. 4: relative norms against a reference): out[0] = ||x-y||_2/||y||_2,
 * out[1] = ||x-y||_inf/||y||_inf, out[2] = number of non-finite entries of x.
 * Accumulates in FP64.  Allocates its scratch with cudaMallocAsync on
 * `stream`.  Synchronous.
 */
int cgl_rel_error(const void* x, const void* y, int64_t count, int precision,
                  double* out, void* stream);

/* ------------------------------------------------------------------------
 * Batches: many independent instances of eq. 1 (each with its own grid,
 * boundary conditions and parameters) advanced together.
 * ---------------------------------------------------------------------- */

/* One problem of a batch: d, n[d], bc[d], lo[d], hi[d] and the parameters
 * exactly as in cgl_plan_create (entries beyond d are ignored). */
typedef struct cgl_problem {
    int d;
    int64_t n[3];
    int bc[3];
    double lo[3], hi[3];
    double a1, b1, a2, a3, b3, a4, b4;
} cgl_problem;

typedef struct cgl_batch cgl_batch;

/*
 * Create a batch of `count` finite-difference problems (Dirichlet/Neumann;
 * periodic -> EUNSUPPORTED) sharing one step size and scheme (strang,
 * split4, lawson4, lawson2, strang_3t, split4_3t) in CGL_F64, CGL_F32 or
 * CGL_BF16X3 (complex64 state; every n_mu <= 256).  Each instance gets its
 * own FP64 factors exp(c tau A_mu) (Sec. 3.1).  F64 / F32: the whole time
 * step is ONE persistent launch: a fixed grid of CTAs pulls (pass, instance,
 * fiber tile) items of every mode pass of every sweep from one device work
 * list, an item waiting (bounded) until its instance's previous pass is done;
 * the fibers per tile come from cgl_autotune_mode_tile.  BF16X3: per sweep
 * one grouped split prologue, one persistent tensor-core launch per mode (one
 * CTA per SM walks the pass's (instance, tile) records, its copies, MMAs and
 * epilogue overlapped across tiles) and one grouped plane epilogue.  The
 * whole time step is replayed as one CUDA graph.  Synchronous (set-up and
 * autotuning).
 * Errors: EINVAL (bad precision or scheme; per-instance validation as
 * cgl_plan_create, message names the instance), EUNSUPPORTED, ENOMEM, ECUDA.
 */
int cgl_batch_create(cgl_batch** out, int count, const cgl_problem* probs, double tau, int scheme,
                     int precision, void* stream);

/*
 * Layout of the batch's packed field: *total_points = sum of N_i; offsets
 * (count entries, may be NULL) = element offset of instance i, in instance
 * order; workspace bytes; launches per time step.  Any pointer may be NULL.
 */
int cgl_batch_info(const cgl_batch* batch, int64_t* total_points, int64_t* offsets,
                   size_t* workspace_bytes, int* launches_per_step);

/*
 * Advance every instance of the packed device field u (total_points complex
 * values; instance i at offsets[i], each in the layout of cgl_step) by nsteps
 * steps, in place.  Asynchronous on `stream`; graph captured per u pointer.
 */
int cgl_batch_step(cgl_batch* batch, void* u, int64_t nsteps, void* stream);

/* Read and clear the batch's device status word (as cgl_last_device_status). */
int cgl_batch_last_device_status(cgl_batch* batch, void* stream);

/* Destroy a batch; NULL is accepted. */
int cgl_batch_destroy(cgl_batch* batch);

/*
 * Fault injection for tests (the paper has no counterpart): with on != 0,
 * every dependency wait of an FP64 / FP32 batch's time step (an item waiting
 * for its instance's previous mode pass) waits for a count that is never
 * reached and gives up after 1024 polls (about 0.15 ms) instead of the
 * normal 2^22; the launch then stops at every CTA's next claim,
 * cgl_batch_last_device_status returns CGL_ETIMEOUT, and the field is left
 * in an unspecified state.  on = 0 restores normal waits.  Either call
 * discards the step's CUDA graph, captured again at the next cgl_batch_step.
 * Errors: EINVAL (NULL), EUNSUPPORTED (a BF16X3 batch: its tensor-core waits
 * are not injected), ECUDA.
 */
int cgl_batch_inject_wait_failure(cgl_batch* batch, int on);

/*
 * Tile-size autotuner of the mu-mode pass: times every admissible number of
 * fibers per CTA (2, 4, ..., 64, within 96 KiB of shared memory) for mode
 * length n, contiguous (mode 1) or strided fibers, precision (CGL_F64 /
 * CGL_F32) and nrhs (1 or 2) on a synthetic 2048-fiber field, and returns the
 * fastest in *tb (*ms = its time per pass, may be NULL).  Results are cached
 * per process and, when the environment variable CGL_AUTOTUNE_CACHE names a
 * file, appended to / read from that file (one line per shape).  Synchronous.
 */
int cgl_autotune_mode_tile(int n, int contiguous, int precision, int nrhs, int* tb, double* ms);

/* ------------------------------------------------------------------------
 * Learned corrector of a coarse periodic step (2D).  The corrected step is
 * u_{n+1} = C(u_n) + N(x) with C one coarse step of a plan (e.g. Lawson4,
 * eq. lawson4, in CGL_F32) and N a residual CNN: 3x3 convolutions with
 * circular padding, 9 -> hidden -> ... -> hidden -> 2 channels, ReLU between
 * layers; x = 9 planes (Re, Im of C(u_n); Re, Im of u_n; a1, b1, a2, a3, b3 as
 * constant planes).  The forward and input-gradient convolutions run on the
 * tensor cores with BF16 operands (weights, and each convolution's input
 * activations or incoming gradients rounded to nearest even) and FP32
 * accumulation; weight gradients in FP32 from the unrounded values; FP32
 * masters, Adam on the masters.  The paper has no learned part; this
 * follows the fine method (the plain integrator at a smaller step) as the
 * training target and as the reference for the corrected error.
 *
 * Field arguments are complex64 device arrays [P][H][W] (W fastest, the
 * layout of a 2D plan field with n_1 = W); `params` is float [P][5]
 * (a1, b1, a2, a3, b3); `idx` (device int[batch], may be NULL for 0..batch-1)
 * selects the samples of a batch.  Weights are a flat float array: per layer
 * w[Cout][Cin][3][3] then b[Cout].
 * ---------------------------------------------------------------------- */
typedef struct cgl_corrector cgl_corrector;

/* height, width: multiples of 16; hidden in 1..32; layers in 2..16;
 * max_batch >= 1 (sizes the activation buffers).  Weights He-uniform from
 * splitmix64(seed) (last layer x 0.1), zero biases.  Synchronous. */
int cgl_corrector_create(cgl_corrector** out, int height, int width, int hidden, int layers,
                         int max_batch, uint64_t seed, void* stream);
int cgl_corrector_num_params(const cgl_corrector* c, int64_t* count);
/* Host FP32 weights in/out (count must equal num_params); set resets Adam. */
int cgl_corrector_set_weights(cgl_corrector* c, const float* host, int64_t count);
int cgl_corrector_get_weights(const cgl_corrector* c, float* host, int64_t count);
/* N(x) into the device float array out[batch][2][H][W].  Asynchronous. */
int cgl_corrector_forward(cgl_corrector* c, const void* coarse, const void* un, const float* params,
                          const int* idx, int batch, float* out, void* stream);
/* Loss = mean over batch x 2 x H x W of ((C(u_n) + N(x) - target) / s)^2,
 * s the output scale (cgl_corrector_set_output_scale), and its
 * gradient w.r.t. the weights (host float[num_params], may be NULL); *loss
 * (may be NULL).  Synchronous when grads_host or loss is given. */
int cgl_corrector_gradients(cgl_corrector* c, const void* coarse, const void* un, const void* target,
                            const float* params, const int* idx, int batch, float* grads_host,
                            double* loss, void* stream);
/* One Adam step (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the loss
 * above; *loss (may be NULL) is the loss before the step. */
int cgl_corrector_train_step(cgl_corrector* c, const void* coarse, const void* un, const void* target,
                             const float* params, const int* idx, int batch, float lr, double* loss,
                             void* stream);
/* u_out[b] = coarse[b] + N(x_b), complex64 [batch][H][W].  Asynchronous. */
int cgl_corrector_apply(cgl_corrector* c, const void* coarse, const void* un, const float* params,
                        int batch, void* u_out, void* stream);
/* u_out[b] = coarse[b] + N(x_b) for complex128 fields [batch][H][W] (the
 * coarse step run in CGL_F64): the features are taken from the complex128
 * inputs rounded to FP32 and the correction is added in FP64.  Asynchronous. */
int cgl_corrector_apply_c128(cgl_corrector* c, const void* coarse, const void* un, const float* params,
                             int batch, void* u_out, void* stream);
/* What `target` means in cgl_corrector_gradients / train_step: mode 0
 * (default) the fine result F(u_n) (loss on C(u_n) + N(x) - target); mode 1
 * the correction F(u_n) - C(u_n) itself (loss on N(x) - target), which keeps
 * a correction far below the state's FP32 resolution intact when it is
 * formed in FP64 before it is stored.  EINVAL for other modes. */
int cgl_corrector_set_target_mode(cgl_corrector* c, int mode);
/* How N(x) is scaled: mode 0 (default) N = s a, s the output scale, a the
 * last convolution; mode 1 N_b = s r_b a_b per sample b, r_b the RMS over
 * the sample of |C(u_n) - u_n| (the coarse increment), so that the network
 * predicts the correction relative to the size of the step it corrects.
 * Applies to forward, gradients / train_step (the loss is measured in units
 * of each sample's scale) and both apply calls.  EINVAL for other modes. */
int cgl_corrector_set_scale_mode(cgl_corrector* c, int mode);
/* N(x) = scale * (last convolution); default 1.  Training sets it to the
 * typical size of the correction (fine minus coarse) so that the network's
 * own outputs stay of order one.  EINVAL unless scale > 0 and finite. */
int cgl_corrector_set_output_scale(cgl_corrector* c, float scale);
/*
 * One 3x3 convolution with circular padding on the tensor cores, the building
 * block of the corrector: y = conv(x, w) + bias, optionally ReLU.
 *   x      device float [B][Cin][H][W]; rounded to BF16 (nearest even) as the
 *          MMA operand.
 *   w      device BF16 bit patterns (uint16) [Cout][Cin][3][3].
 *   bias   device float [Cout] or NULL.
 *   y      device float [B][Cout][H][W]; must not overlap x.
 *   1 <= Cin, Cout <= 32.  Products accumulate in FP32.
 *   status optional device int; bit 1 is set if a bounded wait gave up.
 * Asynchronous on `stream`.  Errors: EINVAL, ECUDA.
 */
int cgl_conv3x3(const float* x, const uint16_t* w, const float* bias, float* y, int B, int cin,
                int cout, int H, int W, int relu, int* status, void* stream);

/*
 * Copy of one of the corrector's per-layer buffers (introspection, for
 * checking each convolution of the network separately against a
 * reference given the same inputs).  kind 0: the activation feeding layer
 * `layer` (0 = the 9 feature planes, l = the output of layer l - 1 after its
 * ReLU; layers = the network output before the output scale), float
 * [batch][C][H][W]; kind 1: the gradient of the loss w.r.t. the output of
 * layer `layer` (0..layers-1) after that layer's ReLU mask, as used by the
 * weight gradient and the input-gradient convolution.  Values are those of
 * the most recent forward / gradients / train_step / apply call.
 * dst: device or host float array of `count` values (1 <= count <=
 * max_batch * C * H * W), filled with the first `count` values.
 * Asynchronous on `stream` (synchronise before reading a host dst).
 * Errors: EINVAL (bad kind, layer or count), ECUDA.
 */
int cgl_corrector_layer_state(const cgl_corrector* c, int kind, int layer, float* dst, int64_t count,
                              void* stream);

/* Read (synchronising `stream`) and clear the corrector's device status word:
 * CGL_ETIMEOUT if a bounded tensor-core wait gave up since the last read. */
int cgl_corrector_last_device_status(cgl_corrector* c, void* stream);
int cgl_corrector_destroy(cgl_corrector* c);

/*
 * Allocation-free variant of cgl_rel_error (the paper has no counterpart:
 * this entry point exists for callers of the library, not for the method).
 *
 * Who needs it: callers that must not allocate device memory at the point
 * where they check an error norm -- code whose device memory is entirely
 * owned by another allocator (a framework's caching allocator or a fixed
 * memory budget handed out at start-up), and monitoring loops that cannot
 * afford the device-wide synchronisation cudaFree implies.  cgl_rel_error
 * allocates its scratch on every call; this variant calls no cudaMalloc,
 * cudaMallocAsync, cudaFree or allocating library routine.
 *
 * Scratch: a file-scope static __device__ array of 164 KiB (per-block
 * partial sums) that every GPU loading the library holds until the process
 * exits.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents; every slot a call reads is written by that same
 * call first, so nothing needs clearing.  Calls that overlap on the GPU
 * (concurrent streams, or threads sharing a device) race on the array:
 * serialise them.
 *
 * Arguments and results are those of cgl_rel_error.  count must satisfy
 * 1 <= count <= CGL_REL_ERROR_NOALLOC_MAX_COUNT (2^28 complex values, e.g.
 * a 512^3 field is 2^27); larger counts return CGL_EINVAL before any work is
 * enqueued.  Synchronous on `stream`.  Errors: EINVAL, ECUDA.
 */
#define CGL_REL_ERROR_NOALLOC_MAX_COUNT 268435456LL
int cgl_rel_error_noalloc(const void* x, const void* y, int64_t count, int precision,
                          double* out, void* stream);

/*
 * FMA throughput of the current device (a measurement aid, not part of the
 * method): the ALU peak that the FP64 / FP32 SIMT kernels' roofline
 * fractions are quoted against, measured rather than derived from clocks.
 *
 * precision  CGL_F64 (DFMA) or CGL_F32 (FFMA).
 * iters      rounds of 8 independent FMA chains per thread (>= 1); choose
 *            it so one launch runs for milliseconds (e.g. 4096 for FP64,
 *            65536 for FP32).  The grid is 8 blocks of 256 threads per SM.
 * tflops     out: 2 * 8 * iters * threads / seconds / 1e12, timed with CUDA
 *            events around the second of two launches on `stream`.
 * Allocates and frees a small output buffer on `stream`; synchronous.
 * Errors: EINVAL (bad precision, iters < 1, NULL tflops), ENOMEM, ECUDA.
 */
int cgl_measure_fma_peak(int precision, int iters, double* tflops, void* stream);

/* Message for a status code (static string). */
const char* cgl_strerror(int status);

/* Message of the calling thread's most recent failure ("" if none). */
const char* cgl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CGL_H */
