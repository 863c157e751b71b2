/*
 * tpcamg.h -- C ABI of the GB300 block V-cycle AMG for Toeplitz-like-plus-Cross systems.
 *
 * Method: Chen, Cao, Serra-Capizzano, "Fast algebraic multigrid for block-structured dense
 * and Toeplitz-like-plus-Cross systems arising from nonlocal diffusion problems"
 * (arXiv:2202.11288).
 *
 * The system (section 2.2): the 1-D peridynamic / nonlocal volume-constrained diffusion
 * problem -L_delta u = f on (0,1), u = g on [-delta,0] U [1,1+delta], constant kernel,
 * piecewise-quadratic collocation with N = 1/h = 2^K intervals and horizon ratio
 * r = floor(delta/h) (r = 1 when delta <= h). Its matrix is the 2x2 block matrix
 * [A B; C D] of eq. (2.9) (variant 1) or the shifted-symmetric [A B; B^T A_hat]
 * of eq. (2.10) (variant 0), of order n_K = 2N - 1.
 *
 * Vector layout everywhere (section 2.2.1, the grid function U_h): n = 2 N_k + 1 doubles,
 * first the N_k node values v, then the N_k + 1 midpoint values w. In the Cross splitting
 * of eq. (3.7), w = [w_o; w_bar]: element N_k (0-based) is w_o.
 *
 * Levels (section 3.1): level k has N_k = 2^k - 1 and n_k = 2^(k+1) - 1 unknowns; the finest
 * level is K = log2(1/h); the coarsest level kc (default 3, 15 unknowns) is solved with a
 * dense factorisation (Algorithm 2: B_1 = A_1^{-1}).
 *
 * Threading: a handle is used by one host thread at a time. All device work is ordered on
 * the stream given to tpc_setup; for NULL the handle creates its own blocking stream (which
 * is ordered with the legacy default stream), because its iterations are CUDA graphs.
 *
 * Errors: every int-returning call returns TPC_OK (0) on success, a positive status for a
 * completed call whose result is not what was asked (TPC_ENOTCONV), or a negative error.
 * tpc_last_error() returns a message for the last error of a handle (or of a failed
 * tpc_setup / host call when given NULL).
 */
#ifndef TPCAMG_H
#define TPCAMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TPC_OK = 0,
  TPC_ENOTCONV = 1,   /* solve ended at max_iters above tol; x holds the last iterate */
  TPC_EINVAL = -1,    /* bad argument: h not 2^-K, r < 1, level out of range, NULL ptr */
  TPC_ENOMEM = -2,    /* host or device allocation failed */
  TPC_ECUDA = -3,     /* a CUDA call failed; message in tpc_last_error */
  TPC_ESINGULAR = -4, /* the coarsest matrix has a zero pivot */
  TPC_ENOTSUP = -5,   /* a parameter combination this build does not implement */
  TPC_EDIVERGED = -6, /* the residual became non-finite */
  TPC_ESYNC = -7      /* a device-side wait of a stage-batched launch gave up (tpc_batch_solve) */
};

/* eq. (2.10) / eq. (2.9) of the peridynamic model (section 2.2), and the weakly
 * singular nonlocal model of section 2.1, eq. (2.3): A_h = diag(D_1, D_2) - [M Q; P N] for
 * L u = int_0^1 (u(x) - u(y)) |x - y|^{-gamma} dy on (0, 1) with gamma = kernel_a in [0, 1) (no
 * horizon: delta is ignored). Its entries are the exact element integrals of the quadratic
 * basis (the printed p_0 and boundary weights eta_{i/2}, i >= 2, are read as garbled); the
 * diagonal D is not Toeplitz and coarsens to a tridiagonal band, applied beside the FFT product. */
enum { TPC_SPD = 0, TPC_NONSYM = 1, TPC_WEAKLY = 2 };
enum { TPC_FP64 = 0, TPC_MIXED = 1 };          /* precision of the inner V-cycle */
enum { TPC_TRANSFER_PAPER = 0, TPC_TRANSFER_GEOMETRIC = 1 };  /* tpc_params.transfer */

typedef struct tpc_params {
  int variant;        /* TPC_SPD, TPC_NONSYM or TPC_WEAKLY                                */
  int kernel;         /* 0 = constant kernel gamma_delta (section 2.2); 1 = fractional
                         kernel |s|^{-(1+2a)} inside the horizon, a = kernel_a in [-1/2, 1)
                         (not defined by the paper: entries are the exact element integrals
                         of the same collocation, Hadamard finite parts for a >= 1/2, where
                         the system is indefinite and the V-cycle diverges; a = -1/2 is the
                         constant kernel; a >= 1: ENOTSUP); set-up, products and solves   */
  double kernel_a;    /* kernel = 1: a. TPC_WEAKLY: the exponent gamma in [0, 1)          */
  double gamma0;      /* kernel constant; only scales the right-hand side, not the matrix  */
  double shift;       /* sigma added to the diagonal of the finest matrix (sigma I + A)    */
  int m1, m2;         /* pre / post smoothing sweeps of Algorithm 2 (default 1, 1)         */
  double omega_pre;   /* damped Jacobi weights, eq. (7) (default 2/3, 2/3)                 */
  double omega_post;
  int coarsest_level; /* kc, 1 <= kc <= K (default 3)                                      */
  int precision;      /* TPC_FP64, or TPC_MIXED: FP32 V-cycles inside FP64 refinement      */
  int max_iters;      /* outer iterations of tpc_solve (default 100)                       */
  int inner_cycles;   /* TPC_MIXED: at most this many FP32 V-cycles per FP64 residual
                         (default 6; see tpc_solve)                                        */
  int autotune;       /* 1 (default): tpc_setup times, for every three-pass level, the
                         factorisation of its transform (m = R1 x L, log2 L the rule's value or
                         one off it) and the tile widths of the strided passes, and keeps the
                         fastest (see tpc_tune_get; results agree to rounding); 0: the rule */
  int poison;         /* checking aid, 0 (default) or 1: every device buffer of the handle
                         is filled with all-ones bytes (NaN in FP32 and FP64) when it is
                         allocated, so that a value read before it is written shows up as
                         NaN in the results; results are otherwise identical              */
  int transfer;       /* TPC_TRANSFER_PAPER (default): the 1/4 [1 2 1] restriction on the
                         concatenated vector [v; w] (section 3.1) and P = 2 R^T;
                         TPC_TRANSFER_GEOMETRIC (not in the paper): the same rows on the
                         unknowns listed by position, whose coarse unknowns are the fine
                         nodes; the V-cycle then converges at the constant kernel's rate
                         for the fractional kernel too. Not for TPC_WEAKLY (ENOTSUP)      */
  int box_residual;   /* 1 (default): when the finest level's Toeplitz generators are piecewise
                         constant (the constant kernel, eq. (2.9) / eq. (2.11), any shift),
                         the outer FP64 residual b - A u is formed from prefix sums of u, one
                         term per run of equal generator values, instead of two FFTs; 0: the
                         FFT product always. The V-cycles are not affected                 */
  int outer;          /* TPC_OUTER_VCYCLE (default): the outer iteration of section 5,
                         u <- u + B (b - A u) with B the V-cycle (TPC_MIXED: inner_cycles FP32
                         V-cycles of it per FP64 residual). TPC_OUTER_FGMRES (not in the
                         paper): each outer iteration is one restart cycle of right-
                         preconditioned flexible GMRES of at most inner_cycles steps, one
                         V-cycle per step as the preconditioner (FP32 vectors, V-cycles and
                         products in TPC_MIXED, FP64 dot products and least squares; all FP64
                         in TPC_FP64); the FP64 residual is formed anew after each cycle.
                         It converges where the stationary iteration is slow or diverges
                         (fractional kernels) and needs fewer V-cycles on the constant kernel */
} tpc_params;

enum { TPC_OUTER_VCYCLE = 0, TPC_OUTER_FGMRES = 1 };

typedef struct tpc_handle tpc_handle;
typedef struct tpc2d_handle tpc2d_handle;  /* the 2-D system: see tpc2d_setup */

/* Fill *p with the defaults: SPD, constant kernel, V(1,1), omega 2/3, kc 3, FP64, 100
 * iterations. */
void tpc_default_params(tpc_params* p);

/* Build the level hierarchy for the system with horizon delta and mesh size h.
 * h must be 2^-K with K >= coarsest_level; levels = number of levels K - kc + 1 to use,
 * or 0 for all of them (the coarsest level is then kc). The finest generators come from
 * the printed coefficients of section 2.2; coarse levels from the Galerkin product
 * A_{k-1} = R A_k P (eq. (3.6)) evaluated in generator-plus-Cross form
 * (Lemma 3.1, eq. (3.8)); the Toeplitz blocks' circulant-embedding spectra (eq. (3.4))
 * are computed on the device. cuda_stream is a cudaStream_t (NULL = default stream).
 * On success *out owns all device memory of the hierarchy until tpc_destroy; on failure
 * *out is NULL and tpc_last_error(NULL) describes the error. */
int tpc_setup(const tpc_params* p, double delta, double h, int levels, void* cuda_stream,
              tpc_handle** out);

/* Solve A_K x = b to ||b - A x||_2 / ||b - A x0||_2 < tol (section 5 stopping rule) with
 * repeated V-cycles (Algorithm 2). With precision TPC_MIXED each outer iteration runs FP32
 * V-cycle iterations on the FP64 residual (scaled to unit RMS) and adds the correction in
 * FP64; the residual and the stopping test are always FP64. The first outer iteration runs
 * inner_cycles of them, each later one the fewest (at most inner_cycles) that reach tol / 4
 * at the reduction per cycle observed in the iteration before (a deterministic function of
 * the FP64 residual norms). b_dev, x_dev: device pointers to n_K doubles (caller
 * owned; they may not alias). use_x0 != 0 starts from the values in x_dev, else from 0.
 * iters_out / relres_out (host pointers, may be NULL) receive the number of outer
 * iterations and the final relative residual. Blocks the host until the result is in
 * x_dev. Returns TPC_OK, TPC_ENOTCONV, TPC_EDIVERGED or a negative error. The solve path
 * allocates nothing. */
int tpc_solve(tpc_handle* H, const double* b_dev, double* x_dev, double tol, int use_x0,
              int* iters_out, double* relres_out);

/* One step of eq. (5.1) on a handle set up with shift = sigma (tpc_bdf4_coefficients):
 * forms b = hist_scale (4 u1 - 3 u2 + 4/3 u3 - 1/4 u4) + g_scale g on the device (u_j = U^{k-j};
 * g may be NULL for no source term) and solves (sigma I + A) u_out = b from the initial guess
 * u1, stopping as tpc_solve does (relative to the initial residual). Device pointers of n_K
 * doubles; u_out may be any of u1..u4 (they are read first). Stream-ordered on the handle's
 * stream; blocks the host like tpc_solve. Returns as tpc_solve. */
int tpc_bdf4_step(tpc_handle* H, const double* u1, const double* u2, const double* u3,
                  const double* u4, double hist_scale, const double* g, double g_scale,
                  double tol, double* u_out, int* iters_out, double* relres_out);

/* Solve count independent systems at once (instances of any sizes, variants and precisions):
 * instance i solves hs[i]'s system A x_dev[i] = b_dev[i] to tol (zero initial guess). Each
 * instance runs on its own handle's stream and the host services the instances round-robin,
 * so their iterations overlap on the GPU; every instance does exactly the arithmetic of
 * tpc_solve on its handle (results are bitwise those of solving it alone). The handles must be
 * distinct; b_dev[i], x_dev[i] are device arrays of that handle's n_K doubles. iters_out,
 * relres_out, status_out (host arrays of count entries, may be NULL) receive each instance's
 * outer iterations, final relative residual and status (TPC_OK / TPC_ENOTCONV / ...).
 * Returns TPC_OK if every instance converged, else the most severe instance status or an
 * error. Blocks until every x_dev[i] holds its result. This is the batched-instances mode of
 * the solver (not in the paper, which solves one system at a time). */
int tpc_solve_batch(tpc_handle* const* hs, int count, const double* const* b_dev,
                    double* const* x_dev, double tol, int* iters_out, double* relres_out,
                    int* status_out);

/* Stage-batched solves (the batched configuration, not in the paper). tpc_batch_create groups the
 * handles whose level structure is identical -- mixed precision, V(1,1), the single-block bottom
 * of the FP32 V-cycles, the prefix-sum residual (box_residual with the constant kernel), the
 * same finest and coarsest levels, system and inner_cycles, the stationary outer iteration,
 * every three-pass level on the general FP32 kernels (m <= 2^19), the same FFT plans -- and
 * prepares, per group, every stage's arguments for all its instances. tpc_batch_solve then runs
 * each outer iteration of a group as ONE launch per stage of Algorithm 2 over all the group's
 * instances (a three-pass product is either one persistent cooperative launch whose passes are
 * separated by grid-wide barriers on a device counter, or one launch per pass: see
 * tpc_batch_set_product_mode), captured once per inner-cycle count as a CUDA graph; the groups run
 * concurrently on their own streams, and handles outside every group are solved as by
 * tpc_solve_batch beside them. Each instance computes exactly what tpc_solve computes on its
 * handle (bitwise). A barrier's wait gives up after a bounded number of polls (about a second):
 * the launch then returns early and tpc_batch_solve returns TPC_ESYNC (results undefined, the
 * context stays usable). The handles must be distinct and outlive the batch; the batch holds
 * device memory of a few KB per instance. */
typedef struct tpc_batch tpc_batch;
int tpc_batch_create(tpc_handle* const* hs, int count, tpc_batch** out);

/* As tpc_batch_create, with count2 2-D handles (tpc2d_setup) as further instances: each runs its
 * own iteration graphs on its own stream beside the groups, exactly as tpc2d_solve would. In
 * tpc_batch_solve the vectors and outputs of the 2-D instances follow the 1-D ones (index
 * count + i). */
int tpc_batch_create_2d(tpc_handle* const* hs, int count, tpc2d_handle* const* hs2, int count2,
                        tpc_batch** out);

/* As tpc_solve_batch, on the batch's handles in their creation order. */
int tpc_batch_solve(tpc_batch* B, const double* const* b_dev, double* const* x_dev, double tol,
                    int* iters_out, double* relres_out, int* status_out);

/* How a group launches the three-pass products of its levels (a batch starts in TPC_BATCH_AUTO):
 * TPC_BATCH_COOPERATIVE, one persistent cooperative launch per product as described above;
 * TPC_BATCH_THREE_PASS, three launches per product (forward strided pass, contiguous blocks,
 * inverse strided pass), each over the tiles of all live instances; TPC_BATCH_AUTO, the choice
 * per level that measured faster (three launches on every level of the current kernels: the
 * barriers' idle blocks and the persistent kernel's two resident blocks per SM cost more than
 * the two launches they save).
 * Results are bitwise the same in every mode. Waits for the groups' work in flight and drops
 * their captured graphs. Returns TPC_EINVAL for NULL or an unknown mode. */
enum { TPC_BATCH_AUTO = 0, TPC_BATCH_COOPERATIVE = 1, TPC_BATCH_THREE_PASS = 2 };
int tpc_batch_set_product_mode(tpc_batch* B, int mode);

/* Number of stage-batched groups, and of the instances they hold (-1 for NULL). */
int tpc_batch_groups(const tpc_batch* B);
int tpc_batch_grouped_instances(const tpc_batch* B);

/* Frees the batch (not the handles); NULL-safe. */
void tpc_batch_destroy(tpc_batch* B);

/* Check of the bounded device-side wait: a cooperative launch of 4 blocks waits at a grid barrier
 * whose target nothing reaches, with max_polls polls. On return *gave_up is 1 when the wait gave
 * up and flagged it, and *passed counts the blocks that (wrongly) passed the barrier. */
int tpc_grid_wait_selftest(unsigned max_polls, int* gave_up, int* passed);

/* Same as tpc_solve with host buffers b_host / x_host (n_K doubles each): the call copies
 * b to the device, solves and copies x back before returning. */
int tpc_solve_host(tpc_handle* H, const double* b_host, double* x_host, double tol,
                   int use_x0, int* iters_out, double* relres_out);

/* y = A_level x in FP64 through the Toeplitz-plus-Cross product (eq. (3.7) and the
 * matrix-vector formula after it). level in [kc, K]; x_dev, y_dev: device pointers to
 * n_level doubles, not aliasing. Stream ordered, does not block. */
int tpc_apply(tpc_handle* H, int level, const double* x_dev, double* y_dev);

/* y = A_level x in FP32 with the FP32 hierarchy of a TPC_MIXED handle (the spectra and Cross
 * vectors are the FP64 ones rounded to FP32). Same layout and rules as tpc_apply; returns
 * TPC_EINVAL on an FP64-only handle. */
int tpc_apply_f32(tpc_handle* H, int level, const float* x_dev, float* y_dev);

/* e = B_K r: one FP64 V-cycle of Algorithm 2 with zero initial guess on the finest level.
 * r_dev, e_dev: device pointers to n_K doubles, not aliasing. Stream ordered. */
int tpc_vcycle(tpc_handle* H, const double* r_dev, double* e_dev);

/* Number of unknowns n_k of a level (0 if out of range), and the finest / coarsest level. */
long long tpc_level_size(const tpc_handle* H, int level);
int tpc_finest_level(const tpc_handle* H);
int tpc_coarsest_level(const tpc_handle* H);

/* Copy the generator-plus-Cross form of one level to host memory, as doubles:
 * [N_k, o, tA, tB, tC, tD, p, q, xi, zeta] where each t* has 2 N_k - 1 entries t[d],
 * d = i - j = -(N_k-1)..N_k-1 (T(i,j) = t_{i-j}), for the blocks A, B_bar, C_bar, D_bar of
 * eq. (3.7), and p, q, xi, zeta have N_k entries. *need receives the count
 * 2 + 4(2 N_k - 1) + 4 N_k; nothing is written if cap < *need (returns TPC_EINVAL). */
int tpc_export_level(const tpc_handle* H, int level, double* host_buf, size_t cap,
                     size_t* need);

/* Host-only (no GPU used): compute the same hierarchy as tpc_setup and write every level
 * from K down to kc, each in the tpc_export_level layout, one after another into host_buf.
 * *need receives the total count; nothing is written if cap < *need. */
int tpc_host_hierarchy(const tpc_params* p, double delta, double h, int levels,
                       double* host_buf, size_t cap, size_t* need);

/* Dense matrix of one level of the host hierarchy (generator-plus-Cross form plus the band of
 * TPC_WEAKLY), row major, n_level x n_level with n_level <= 8191: for tests against a dense
 * reference. out == NULL: only *need is set. Host only. Returns TPC_OK or a negative code. */
int tpc_host_dense_level(const tpc_params* p, double delta, double h, int levels, int level,
                         double* out, size_t cap, size_t* need);

/* ---------------------------------------------------------------------------------------
 * Time stepping (section 5): u_t = L_delta u + f on (0, 1), u = g on the interaction domain,
 * advanced by the BDF4 scheme of eq. (5.1),
 *   (25/12 I - tau L_delta) U^k = 4 U^{k-1} - 3 U^{k-2} + 4/3 U^{k-3} - 1/4 U^{k-4} + tau F^k.
 * The collocation system is A U = eta_h (-L_delta u)(x_p) - (exterior couplings of g) with
 * eta_h = 6 / (gamma h) (gamma = gamma0, or the paper's 3 / delta^3 with delta = r h when
 * gamma0 = 0; TPC_WEAKLY: eta_{h,gamma} of eq. (2.3)), so a step is the shifted solve
 *   (sigma I + A) U^k = (eta_h / tau) (4 U^{k-1} - 3 U^{k-2} + 4/3 U^{k-3} - 1/4 U^{k-4}) + b^k,
 *   sigma = 25 eta_h / (12 tau),  b^k = eta_h F^k(x_p) - (exterior couplings of g^k).
 * --------------------------------------------------------------------------------------- */

/* sigma (the shift to set in tpc_params.shift before tpc_setup) and eta_h / tau for time step
 * tau > 0. Host only. TPC_EINVAL on bad arguments (message in tpc_last_error(NULL)). */
int tpc_bdf4_coefficients(const tpc_params* p, double delta, double h, double tau,
                          double* shift_out, double* hist_scale_out);

/* Collocation right-hand side of section 2.2 (eq. (2.5) with the constrained exterior values
 * moved to the right, eqs. (2.7)-(2.8), each row with its own stencil):
 *   rhs[p] = eta_h f_colloc[p] - sum over exterior points q within the horizon of A(p, q) g(x_q).
 * f_colloc: n = 2/h - 1 values of f at the collocation points in unknown order (nodes h..1-h,
 * then midpoints h/2..1-h/2), or NULL for f = 0. g_left[j] = g(-j h/2), g_right[j] =
 * g(1 + j h/2) for j = 0..2r (r = floor(delta/h), at least 1), or NULL for zero exterior
 * values. rhs_out: n doubles. Host memory, host work O(n + r^2). Returns TPC_OK or TPC_EINVAL.
 * (SPD system: the midpoint rows use the integer-row stencil, as eq. (2.10) does.)
 * TPC_WEAKLY (no interaction domain): rhs = eta_{h,gamma} f + K0 g_left[0] + KN g_right[0] with
 * eta_{h,gamma} = (3-gamma)(2-gamma)(1-gamma)/h^{1-gamma} and K0, KN the couplings of the
 * boundary basis functions (u(0) = g_left[0], u(1) = g_right[0]; other entries unused). */
int tpc_collocation_rhs(const tpc_params* p, double delta, double h, const double* f_colloc,
                        const double* g_left, const double* g_right, double* rhs_out);

/* Process-wide tuning table of the FFT plans (tpc_params.autotune; not in the paper). For the
 * levels of size m = 2^logm of one precision (word = 4: FP32, 8: FP64) an entry holds the
 * factorisation m = R1 x L of the three-pass product (logL = log2 L), the tile width 2^logC of
 * the strided passes and whether the register-resident FP32 kernels run it (reg). The set-up
 * autotuner writes the entries it measures (the factorisation with log2 L the rule's value or
 * one off it, and every tile width); a later set-up with autotune = 1 uses an existing entry
 * instead of timing, so every handle of the process computes the same products.
 * tpc_tune_get returns 1 and fills the outputs if there is an entry, 0 if not, TPC_EINVAL for a
 * bad word or NULL. tpc_tune_set writes an entry (TPC_EINVAL unless 13 <= logm <= 23,
 * 2^7 <= L <= 2^12, 2^6 <= R1 <= 2^11, R1 x 2^logC <= 8192, 0 <= logC <= 4, and reg = 1 only
 * with word = 4 and a factorisation the register-resident kernels take: R1 = 2^10 or 2^11,
 * L = 2^10 .. 2^12); levels with the band of TPC_WEAKLY take the general kernels. Results of
 * every entry are the method's to rounding. tpc_tune_reset empties the table. */
int tpc_tune_get(int word, int logm, int* logL, int* logC, int* reg);
int tpc_tune_set(int word, int logm, int logL, int logC, int reg);
void tpc_tune_reset(void);

/* Timing of the kernels of one level's product y = f - A_level x on the handle's stream:
 * each kernel of the pipeline is launched reps times (reps >= 1) between two CUDA events,
 * after one warm-up launch. ms_out[0..2] receive the average milliseconds per launch of the
 * forward strided pass, the contiguous-block kernel (transform, spectral product, inverse
 * transform) and the inverse strided pass with its epilogue; levels small enough to use a
 * single kernel report 0 for the strided passes. x_dev, f_dev, y_dev: n_level doubles on the
 * device. Blocks the host. */
int tpc_time_level_kernels(tpc_handle* H, int level, int reps, const double* x_dev,
                           const double* f_dev, double* y_dev, double* ms_out);

/* The same timing for the FP32 copy of the level in a TPC_MIXED handle (the kernels the FP32
 * V-cycles run); x_dev, f_dev, y_dev: n_level floats on the device. TPC_EINVAL on an FP64
 * handle. */
int tpc_time_level_kernels_f32(tpc_handle* H, int level, int reps, const float* x_dev,
                               const float* f_dev, float* y_dev, double* ms_out);

/* Number of kernels this handle has launched so far (graph launches count every kernel node
 * of the graph). */
long long tpc_kernel_launches(const tpc_handle* H);

/* r = b - A_K x on the finest level, the outer residual of tpc_solve (section 5), formed the
 * way the solver forms it: from prefix sums of x over the runs of equal generator values when
 * the handle uses box_residual (see tpc_params), else with the FFT product of eq. (3.4).
 * x_dev, b_dev, r_dev: device arrays of n_K doubles; r_dev must alias neither input.
 * Stream-ordered on the handle's stream, does not block. TPC_OK or TPC_EINVAL. */
int tpc_residual(tpc_handle* H, const double* x_dev, const double* b_dev, double* r_dev);

/* 1 if the handle forms its outer residual from prefix sums (box_residual in effect), 0 if it
 * uses the FFT product; -1 for a NULL handle. */
int tpc_uses_box_residual(const tpc_handle* H);

/* V-cycles (Algorithm 2) run by the handle's latest solve: FP32 V-cycles summed over the outer
 * iterations for TPC_MIXED, one per outer iteration for TPC_FP64. Used to count the work of a
 * solve (its products per level) for measurements. -1 for a NULL handle. */
int tpc_last_solve_cycles(const tpc_handle* H);

/* y = A x for ONE level given in generator-plus-Cross form, for callers that cannot allocate
 * device memory (work recorded while a CUDA graph is captured with allocation disallowed, a
 * plugin whose host application owns every device allocation, a path that must not let
 * cudaMalloc/cudaFree synchronise the device). The paper has no counterpart of this call. It
 * allocates nothing: its work memory is one static device array of about 5.7 MB that every
 * GPU loading this library holds until the process exits.
 * N: N_k = 2^k - 1 with 2N + 2 <= 65536 (N <= 32767); larger or other N -> TPC_EINVAL.
 * tA, tB, tC, tD: device arrays of 2N - 1 doubles, the generators t[d + N - 1] = T(i, j)
 * (d = i - j) of A, B_bar, C_bar, D_bar (the tpc_export_level layout); p, q, xi, zeta: device
 * arrays of N doubles; o: the middle diagonal entry; x_dev, y_dev: device arrays of 2N + 1
 * doubles, not aliasing. Work is ordered on cuda_stream (NULL = default stream) and the call
 * does not block. All calls share the static array and it keeps the last call's contents:
 * calls that overlap on the GPU race, so order them on one stream. The first call on a device
 * sets that device up (static array address, kernel limits) and synchronises it; make it
 * before any stream capture. Levels of TPC_SPD and TPC_NONSYM handles only: the tridiagonal
 * band of a TPC_WEAKLY level is not in this layout and is not applied. Returns TPC_OK,
 * TPC_EINVAL or TPC_ECUDA (message in tpc_last_error(NULL)). */
int tpc_apply_noalloc(long long N, const double* tA, const double* tB, const double* tC,
                      const double* tD, const double* p, const double* q, const double* xi,
                      const double* zeta, double o, const double* x_dev, double* y_dev,
                      void* cuda_stream);

/* ---- 2-D Toeplitz-like-plus-Cross systems (not defined by the paper) ----
 * The reading of this library: the constant kernel on the unit square with the square horizon
 * [-delta, delta]^2 and tensor-product quadratic collocation, i.e. the 1-D unknowns of section
 * 2.2 ([v; w] per axis, n = 2N - 1 of them) on each axis, U[i][j] at (x_i, y_j) stored row by
 * row (n^2 doubles). Its matrix is A2 = A (x) I + I (x) A - (A (x) A) / (12 r), A the 1-D matrix
 * of eq. (2.9) (TPC_NONSYM) or eq. (2.10) (TPC_SPD), r = floor(delta / h): each block is block
 * Toeplitz with Toeplitz blocks plus Cross rows and columns. The V-cycle of Algorithm 2 uses the
 * section 3.1 transfers on each axis (R (x) R, P (x) P), Galerkin levels (eq. (3.2), of the form
 * A_k (x) Q_k + Q_k (x) A_k - A_k (x) A_k / (12 r)), damped Jacobi with the diagonal of each level
 * and a dense solve at the coarsest level; products are FFT products (eq. (3.4)) along rows and
 * columns. precision TPC_MIXED runs FP32 V-cycles inside FP64 refinement as tpc_solve does;
 * outer = TPC_OUTER_FGMRES runs the flexible GMRES outer iteration of tpc_params.outer. */

/* Set up on the caller's stream (NULL: a stream of the handle). Needs variant TPC_SPD or
 * TPC_NONSYM, kernel 0, the paper's transfer (else TPC_ENOTSUP), h = 2^-K with K <= 11 and
 * coarsest_level <= 3 (else TPC_EINVAL); other codes as tpc_setup. *out stays NULL on failure. */
int tpc2d_setup(const tpc_params* p, double delta, double h, void* cuda_stream,
                tpc2d_handle** out);

/* Solve A2 x = b to ||b - A2 x||_2 / ||b||_2 < tol (FP64 residual). b_dev, x_dev: device arrays
 * of n_K^2 doubles (x_dev also the initial guess when use_x0). Blocks until done. Returns TPC_OK,
 * TPC_ENOTCONV (x holds the last iterate), TPC_EDIVERGED, or a negative error. */
int tpc2d_solve(tpc2d_handle* H, const double* b_dev, double* x_dev, double tol, int use_x0,
                int* iters_out, double* relres_out);

/* y = A2_level x (FP64; levels above the coarsest), stream-ordered. n_level^2 doubles each. */
int tpc2d_apply(tpc2d_handle* H, int level, const double* x_dev, double* y_dev);

/* The same product in FP32 (TPC_MIXED handles). */
int tpc2d_apply_f32(tpc2d_handle* H, int level, const float* x_dev, float* y_dev);

/* e = B_K r: one V-cycle (FP64) from a zero initial guess, stream-ordered. */
int tpc2d_vcycle(tpc2d_handle* H, const double* r_dev, double* e_dev);

/* n_level^2 (0 for a bad level), finest and coarsest level numbers, V-cycles of the latest solve,
 * kernels launched so far (graph launches are not counted), and the last error message. */
long long tpc2d_level_size(const tpc2d_handle* H, int level);
int tpc2d_finest_level(const tpc2d_handle* H);
int tpc2d_coarsest_level(const tpc2d_handle* H);
int tpc2d_last_solve_cycles(const tpc2d_handle* H);
long long tpc2d_kernel_launches(const tpc2d_handle* H);
const char* tpc2d_last_error(const tpc2d_handle* H);

/* Frees everything; NULL-safe. */
void tpc2d_destroy(tpc2d_handle* H);

/* ---- Request server: continuous batching of independent solves (not in the paper) ----
 * A worker thread admits submitted requests while a slot (max_inflight) and device memory
 * (hbm_budget_bytes) are free, keeps level hierarchies resident keyed by (dimension, variant,
 * kernel, transfer, outer iteration, delta, h, precision) and reuses an idle one when a key repeats (evicting idle
 * ones least recently used first), and runs every admitted solve on its own stream exactly as
 * tpc_solve (1-D) or tpc2d_solve (2-D) would (the result is bitwise that of solving it alone).
 * Requests that arrive while others are on the GPU start as soon as a slot and memory free up. */
typedef struct tpc_server tpc_server;
typedef struct tpc_server_config {
  size_t hbm_budget_bytes; /* device memory the resident hierarchies may hold (default 150 GiB) */
  int max_inflight;        /* solves on the GPU at once (default 32)                        */
  int precision;           /* TPC_FP64 or TPC_MIXED (default)                                */
  int max_handles_per_key; /* hierarchies of one key (default 1: same-key requests queue, no
                              duplicate set-up); requests of other keys pass a waiting one  */
} tpc_server_config;
typedef struct tpc_request {
  int variant;             /* TPC_SPD, TPC_NONSYM or TPC_WEAKLY                              */
  double delta, h;         /* horizon and mesh size (h = 2^-K), as for tpc_setup             */
  long long n;             /* 2/h - 1 unknowns: the length of b_host and x_host              */
  const double* b_host;    /* right-hand side, host memory (pinned for speed), read once     */
  double* x_host;          /* solution, host memory; valid when the result is polled         */
  double tol;              /* relative residual target                                       */
  int kernel;              /* as tpc_params.kernel (0 constant, 1 fractional)                */
  double kernel_a;         /* as tpc_params.kernel_a                                         */
  int dim;                 /* 2: the 2-D system of tpc2d_setup (n = (2/h - 1)^2 unknowns);
                              0 or 1: the 1-D system                                         */
  int transfer;            /* TPC_REQUEST_TRANSFER_DEFAULT (0): the server's tpc_params.transfer;
                              TPC_REQUEST_TRANSFER_PAPER / _GEOMETRIC: that transfer         */
  int outer;               /* TPC_REQUEST_OUTER_DEFAULT (0): the server's tpc_params.outer;
                              TPC_REQUEST_OUTER_VCYCLE / _FGMRES: that outer iteration        */
} tpc_request;
enum { TPC_REQUEST_TRANSFER_DEFAULT = 0, TPC_REQUEST_TRANSFER_PAPER = 1,
       TPC_REQUEST_TRANSFER_GEOMETRIC = 2 };
enum { TPC_REQUEST_OUTER_DEFAULT = 0, TPC_REQUEST_OUTER_VCYCLE = 1, TPC_REQUEST_OUTER_FGMRES = 2 };
typedef struct tpc_server_result {
  long long ticket;        /* as returned by tpc_server_submit                               */
  int status;              /* TPC_OK, TPC_ENOTCONV or a negative error                       */
  int iters;               /* outer iterations                                               */
  double relres;           /* final relative residual                                        */
  double latency_s;        /* submit to result in x_host, seconds                            */
  double queue_s;          /* submit to admission, seconds                                   */
} tpc_server_result;

/* Fill *c with the defaults above. */
void tpc_server_default_config(tpc_server_config* c);
/* Start a server on the current device. p: solver parameters for its handles (NULL = the
 * defaults; precision is taken from cfg). *out owns the worker thread and every hierarchy. */
int tpc_server_create(const tpc_server_config* cfg, const tpc_params* p, tpc_server** out);
/* Queue one request (the buffers must stay valid until its result is polled). Thread-safe. */
int tpc_server_submit(tpc_server* S, const tpc_request* r, long long* ticket);
/* Move up to cap finished results into out (waiting up to wait_ms for the first); returns
 * their number. Thread-safe. */
int tpc_server_poll(tpc_server* S, tpc_server_result* out, int cap, int wait_ms);
/* Requests submitted and not yet finished. */
long long tpc_server_outstanding(tpc_server* S);
/* Occupancy of the GPU by the server's solves, accumulated by the worker since the server
 * started or since the last call with reset != 0. busy_s / elapsed_s is the fraction of the time
 * with at least one solve on the GPU; inflight_s / busy_s the mean number of solves on the GPU
 * at once while busy (their streams' work overlaps on the device). */
typedef struct tpc_server_stats {
  long long admitted;      /* requests started on the GPU                                   */
  long long setups;        /* hierarchies built                                             */
  long long evictions;     /* idle hierarchies freed to make room                           */
  double elapsed_s;        /* time covered                                                   */
  double busy_s;           /* of it, time with at least one solve on the GPU                 */
  double inflight_s;       /* integral over time of the number of solves on the GPU          */
  int max_inflight_seen;   /* most solves on the GPU at once                                 */
  size_t resident_bytes;   /* device memory the resident hierarchies hold (at the last update)*/
} tpc_server_stats;
int tpc_server_get_stats(tpc_server* S, tpc_server_stats* out, int reset);
/* Finish every outstanding request, free everything, stop the worker. NULL-safe. */
void tpc_server_destroy(tpc_server* S);

/* Release everything a handle owns. NULL-safe. */
void tpc_destroy(tpc_handle* H);

/* Message for the last error on H, or for the last failed handle-less call if H is NULL. */
const char* tpc_last_error(const tpc_handle* H);

#ifdef __cplusplus
}
#endif

#endif /* TPCAMG_H */
