/*
 * hsein.h -- C ABI of a GB300 (sm_103a) library that computes eigenvectors of
 * a real upper Hessenberg matrix H by one step of inverse iteration for many
 * shifts at once:  (H - lambda_l I) x_l = alpha_l b_l,  l = 1..m,
 * following Schwarz, "Robust level-3 BLAS Inverse Iteration from the
 * Hessenberg Matrix" (arXiv 2101.05063).
 *
 * The solve is Henry's RQ approach (Sec. 2.2, Alg. "henry") rearranged by
 * tiles (Sec. 3): every shift gets its own Givens sweep over the diagonal
 * tiles (Alg. "tiled-reduction1", "solve"), while the updates of all rows
 * above a diagonal tile read one block of H shared by every shift and run as
 * one dense matrix-matrix product over the whole block of shifts (eq.
 * "update", Alg. "tile-update"; the off-diagonal reduction of Alg.
 * "tiled-reduction2" joins the same product).  Every solution column carries
 * an exact power-of-two scale factor so that nothing overflows (Sec. 4.1,
 * eq. "robust-update"); the result is normalized with a scaled 2-norm and
 * backtransformed (Alg. "consistency-scaling"), and Varah's test flags
 * columns that did not converge (Sec. 4.2).  Complex shifts use the rotation
 * of eq. "cgivens" (Sec. 4.3).
 *
 * Conventions (all calls):
 *  - Matrices are double precision, column-major, with a leading dimension.
 *  - A real shift owns one column of B, X and Z; a complex shift (wi != 0;
 *    pass one member of each conjugate pair) owns two adjacent columns
 *    [real part, imaginary part].  Columns follow the input order of shifts.
 *  - Device pointers: memory of the current CUDA device.  The caller owns
 *    every buffer, including the workspace; the plan owns host metadata only.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and asynchronous: the returned status reports argument
 *    errors found at enqueue time and CUDA launch errors.  Errors found on the
 *    device (non-finite or reduced H, wrong shift count) are recorded in the
 *    workspace; read them with hsein_plan_sync_status.  No exception crosses
 *    this interface.  A plan is not thread-safe; distinct plans are.
 */
#ifndef HSEIN_H
#define HSEIN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsein_plan_s *hsein_plan_t;

typedef enum {
    HSEIN_OK = 0,
    HSEIN_EARG = -1,          /* invalid argument (value or pointer)                    */
    HSEIN_ENOMEM = -2,        /* host allocation failed or workspace too small           */
    HSEIN_ENOTUNREDUCED = -3, /* device: some subdiagonal entry h(k,k-1) is zero          */
    HSEIN_ENONFINITE = -4,    /* device: H or a shift contains Inf or NaN                 */
    HSEIN_ECUDA = -5,         /* a CUDA call or kernel launch failed                      */
    HSEIN_ETIMEOUT = -6,      /* device: a bounded wait of a kernel ran out (see          */
                              /* hsein_options.wait_limit_cycles)                          */
    HSEIN_ESHIFTS = -7,       /* device: the number of wi != 0 differs from m_cplx        */
    HSEIN_WNOTCONVERGED = 1   /* device: some column failed Varah's test (zeroed)         */
} hsein_status;

/* Per-shift status written by hsein_solve to dStatus[l]. */
enum {
    HSEIN_COL_OK = 0,            /* converged, column holds a unit-norm vector        */
    HSEIN_COL_NOT_CONVERGED = 1, /* failed Varah's test (Sec. 4.2), column set to 0   */
    HSEIN_COL_INVALID = 3        /* the solve did not run (device error, see above)   */
};

typedef struct {
    int br;         /* tile height b_r (Sec. 3.2), 8..128; 0 = default (64)                 */
    int precision;  /* 0 = FP64 products; 1 = split-precision products on the BF16 tensor    */
                    /*     cores with FP64 recombination (z = Q0 x), see hsein_backtransform  */
    int robust;     /* 1 = overflow protection (default); 0 = off, for tests that show       */
                    /*     what the protection prevents                                      */
    int omega_log2; /* stored solution entries stay below 2^omega_log2; 0 = default (1000).  */
                    /* Lower values (>= 16) make the scaling of Sec. 4.1 trigger on small     */
                    /* problems, for testing                                                 */
    int method;     /* 0 = the tiled level-3 solve (default); comparison baselines, one      */
                    /*     thread block per shift over the whole matrix, with the same       */
                    /*     protection, normalization and Varah test; precision must be 0:    */
                    /*   1 = Henry's RQ solve per shift, unblocked (Alg. "henry", the RQIN   */
                    /*     of Sec. 5), with the Givens backtransform;                        */
                    /*   2 = the LU approach of LAPACK's inverse iteration (Sec. 2.1):       */
                    /*     P (H - lambda I) = L U with partial pivoting, L y = P b,          */
                    /*     U x = alpha y, for the given starting vector; the packed U of     */
                    /*     every shift in flight is kept in the workspace (shifts are        */
                    /*     factored in chunks that fit in 16 GiB); n <= 14336                */
    int givens;     /* storage of the Givens rotations between the solve and its            */
                    /*     backtransform: 0 = c and s as computed (default); 1 = compact     */
                    /*     (Sec. 4.4, Stewart's scheme): one number per real rotation, two   */
                    /*     per complex rotation, the other quantities recomputed with a      */
                    /*     square root from c^2 + s^2 = 1; saves n x (m_real + m_cplx)       */
                    /*     doubles of workspace.  method must be 0                           */
    long long wait_limit_cycles;
                    /* bound of the wait of the diagonal-tile kernel for the bulk copy of   */
                    /*     its tile (SM clock cycles from the copy's issue); when it runs    */
                    /*     out the kernel records HSEIN_ETIMEOUT, still waits (bounded) for  */
                    /*     the copy in flight, and returns; the solve's statuses become      */
                    /*     HSEIN_COL_INVALID.  0 = default (2^32, about two seconds);        */
                    /*     small values make the limit expire on purpose, for testing        */
} hsein_options;

/* Fill *opt with the defaults.  Returns HSEIN_EARG for opt == NULL. */
hsein_status hsein_default_options(hsein_options *opt);

/*
 * Create a plan for n x n matrices and m_real real plus m_cplx complex shifts
 * (ncol = m_real + 2 m_cplx solution columns).  opt may be NULL (defaults).
 * *workspace_bytes receives the device workspace size hsein_solve,
 * hsein_backtransform and hsein_restart need (the last one needs a few times
 * 8n bytes beyond what the solve itself uses).  n >= 1, m_real >= 0, m_cplx >= 0,
 * m_real + m_cplx >= 1.  On error *plan is set to NULL.
 */
hsein_status hsein_plan(hsein_plan_t *plan, int n, int m_real, int m_cplx,
                        const hsein_options *opt, size_t *workspace_bytes);

/*
 * Solve (H - lambda_l I) x_l = alpha_l b_l for every shift and store unit
 * 2-norm eigenvector approximations of H in dX (Alg. "hsrq3" followed by the
 * convergence test of Sec. 4.2).
 *   dH      n x n upper Hessenberg, leading dimension ldh >= n; entries below
 *           the first subdiagonal are not read.  Every h(k,k-1) must be nonzero
 *           (H unreduced, Sec. 1).
 *   dWr,dWi m = m_real + m_cplx shifts lambda_l = wr_l + i wi_l; exactly m_cplx
 *           of them have wi != 0 (one member per conjugate pair, Sec. 4.3).
 *   dB      n x ncol starting vectors (ldb >= n) or NULL for rho*e with
 *           rho = eps ||H||_inf (Sec. 4.2; for a complex shift rho*e + 0i).
 *   dX      n x ncol output (ldx >= n); may not alias dB or dH.
 *   dStatus m per-shift codes (HSEIN_COL_*), in input order.
 *   dWork   device workspace of at least the size hsein_plan reported,
 *           256-byte aligned; contents on entry are irrelevant.
 * The eigenvectors are normalized to ||x||_2 = 1; their sign (real) or phase
 * (complex) is not normalized.  Work is enqueued on `stream`.
 */
hsein_status hsein_solve(hsein_plan_t plan, const double *dH, int ldh,
                         const double *dWr, const double *dWi,
                         const double *dB, int ldb, double *dX, int ldx,
                         int *dStatus, void *dWork, size_t work_bytes, void *stream);

/*
 * hsein_solve without a workspace argument, for callers that cannot allocate
 * device memory (plug-ins whose host framework owns all device memory and
 * forbids raw cudaMalloc, real-time paths that must not call an allocator).
 * The paper has no counterpart: this is an interface convenience.
 *   The workspace is a fixed 16 MiB array in the library's device memory,
 *   present on every device that loads the library until the process exits.
 *   Plans whose workspace (hsein_plan's *workspace_bytes) exceeds 16 MiB are
 *   rejected with HSEIN_ENOMEM; nothing is allocated, here or later.
 *   The call runs on the current device, which must be the plan's device
 *   (HSEIN_EARG otherwise).  The first call on a device looks up the array's
 *   device address (no allocation) and caches it; the cache does not survive
 *   cudaDeviceReset, so do not use this call across a reset.
 *   All calls share the array: the solve re-initializes every value it reads,
 *   but calls whose work overlaps on the GPU (other streams, other threads)
 *   race and must be serialized by the caller.  Device-side errors show in
 *   dStatus (every entry HSEIN_COL_INVALID); the other arguments and results
 *   are those of hsein_solve.
 */
hsein_status hsein_solve_noalloc(hsein_plan_t plan, const double *dH, int ldh,
                                 const double *dWr, const double *dWi,
                                 const double *dB, int ldb, double *dX, int ldx,
                                 int *dStatus, void *stream);

/*
 * z_l = Q0 x_l for every column (Sec. 1: H = Q0^T A Q0 maps eigenvectors of H
 * to eigenvectors of A).  dQ0 n x n (ldq >= n), dX n x ncol (ldx >= n), dZ
 * n x ncol output (ldz >= n, may not alias dX).  dWork as for hsein_solve
 * (the same buffer may be reused after the solve).  Stream-ordered.
 * precision 0: an FP64 product.  precision 1: every row of Q0 and column of
 * X is scaled by a power of two and cut into seven 8-bit digits, the digit
 * products with weight above the FP64 rounding level run on the BF16 tensor
 * cores with exact integer accumulation of the leading terms, and the result
 * is recombined in FP64 (error comparable to an FP64 product); dWork is used
 * and must be the size hsein_plan reported.
 */
hsein_status hsein_backtransform(hsein_plan_t plan, const double *dQ0, int ldq,
                                 const double *dX, int ldx, double *dZ, int ldz,
                                 void *dWork, size_t work_bytes, void *stream);

/*
 * The solve and z = Q0 x from host memory, end to end (Sec. 1: eigenvectors
 * of A = Q0 H Q0^T): H, the shifts and B are copied to the device on
 * `stream`; Q0 on a side stream owned by the plan meanwhile (only the
 * backtransform needs it; it waits for the previous call's backtransform to
 * have read the device copy); then hsein_solve, hsein_backtransform, and Z
 * and the statuses are copied back.  Host arrays: hH n x n (ldh >= n), hWr,
 * hWi m shifts, hB n x ncol (ldb >= n) or NULL for rho*e, hQ0 n x n
 * (ldq >= n), hZ n x ncol output (ldz >= n), hStatus m output; pinned host
 * memory lets the copies run asynchronously.  dWork: device memory of
 * hsein_host_workspace bytes (the solve's workspace followed by the device
 * copies of the operands), 256-byte aligned.  The solve on the device
 * copies runs as a CUDA graph (hsein_graph_create), captured at the first
 * call with this dWork and starting-vector choice and kept by the plan; while
 * the plan records per-launch profiling it is launched kernel by kernel.
 * Stream-ordered: hZ and hStatus are valid once `stream` has completed.  Device errors as for
 * hsein_solve (hsein_plan_sync_status on dWork).  The paper has no
 * counterpart: an interface convenience.
 */
hsein_status hsein_host_workspace(hsein_plan_t plan, size_t *workspace_bytes);
hsein_status hsein_solve_host(hsein_plan_t plan, const double *hH, int ldh,
                              const double *hWr, const double *hWi, const double *hB, int ldb,
                              const double *hQ0, int ldq, double *hZ, int ldz, int *hStatus,
                              void *dWork, size_t work_bytes, void *stream);

/*
 * One step on fixed device buffers as a CUDA graph: hsein_graph_create
 * records hsein_solve with these arguments, followed by hsein_backtransform
 * (dQ0 -> dZ from the solve's dX) when dQ0 is not NULL, into a graph (on a
 * capture stream of its own; nothing runs), and hsein_graph_launch runs
 * that graph on `stream`: the same kernels in the same order with the same
 * results as the two calls, without a host launch per kernel, which at
 * n = 4096 leaves the GPU idle between the sweep and update launches of
 * every tile column (10.41 -> 10.07 ms per step, measured).
 *   Arguments as for hsein_solve and hsein_backtransform (dZ, ldz may be
 *   NULL, 0 when dQ0 is NULL).  The buffers are used in place at every
 *   launch; refresh their contents between launches, do not free them
 *   before hsein_graph_destroy.  The plan's per-launch profiling is not
 *   recorded inside the graph.
 *   Returns HSEIN_EARG / HSEIN_ENOMEM for the arguments as the two calls
 *   would, HSEIN_ECUDA if the capture or instantiation fails.  Device errors
 *   of a launch as for hsein_solve (hsein_plan_sync_status on dWork).
 * The paper has no counterpart: a launch interface.
 */
typedef struct hsein_graph_s *hsein_graph_t;
hsein_status hsein_graph_create(hsein_plan_t plan, const double *dH, int ldh,
                                const double *dWr, const double *dWi,
                                const double *dB, int ldb, double *dX, int ldx,
                                int *dStatus, const double *dQ0, int ldq, double *dZ, int ldz,
                                void *dWork, size_t work_bytes, hsein_graph_t *graph);
hsein_status hsein_graph_launch(hsein_graph_t graph, void *stream);
hsein_status hsein_graph_destroy(hsein_graph_t graph);

/*
 * Restart loop of inverse iteration (Alg. "hsrq3in", Sec. 4.2).  Call after
 * hsein_solve with the same arguments: every shift whose status is
 * HSEIN_COL_NOT_CONVERGED is solved again, up to max_tries times, from a new
 * starting vector orthogonal to the previous choices (the given column of dB,
 * or rho*e, and the earlier trials): trial t is column n+1-t of the
 * Householder reflector whose first column is b/||b|| (real shift), or of the
 * Householder QR factor of [Re b, Im b] (complex shift; a real vector, so
 * b^H x = 0).  Converged results replace the zeroed columns of dX and their
 * status becomes HSEIN_COL_OK; the others keep HSEIN_COL_NOT_CONVERGED.
 *   max_tries >= 0 (at most n-2 are used); *n_retried (may be NULL) = the
 *   number of shifts that were retried.
 *   dWork / work_bytes as for hsein_solve; the restart uses it for
 *   sub-problems of the retried shifts (chunked when they do not fit), so
 *   hsein_margins and hsein_plan_sync_status afterwards describe the last
 *   sub-problem, not the original solve.
 * Synchronizes `stream` (which shifts to retry is decided on the host).
 * Returns HSEIN_OK when every shift has converged, HSEIN_WNOTCONVERGED if
 * some have not, HSEIN_ECUDA on a CUDA or device error, HSEIN_ENOMEM if not
 * even one retried shift fits in dWork.
 */
hsein_status hsein_restart(hsein_plan_t plan, const double *dH, int ldh,
                           const double *dWr, const double *dWi,
                           const double *dB, int ldb, double *dX, int ldx,
                           int *dStatus, int max_tries, int *n_retried,
                           void *dWork, size_t work_bytes, void *stream);

/*
 * Convergence margins of the last hsein_solve that used dWork: for every
 * shift, in input order, log2(||x||_2 / ||b||_2) - log2(1 / (10 n ||H||_inf
 * eps)), the amount (in powers of two) by which one step of inverse
 * iteration exceeded Varah's threshold (Sec. 4.2); > 0 means converged,
 * -HUGE_VAL a zero solution.  Copies m doubles to the device array dMargin,
 * stream-ordered.  The paper has no counterpart: a diagnostic of how close a
 * column came to the test.
 */
hsein_status hsein_margins(hsein_plan_t plan, const void *dWork, double *dMargin, void *stream);

/*
 * Wait for `stream`, then return the device-side status of the last
 * hsein_solve that used dWork: HSEIN_OK, HSEIN_WNOTCONVERGED, or one of the
 * device error codes.  Returns HSEIN_ECUDA if the stream reports an error.
 */
hsein_status hsein_plan_sync_status(hsein_plan_t plan, const void *dWork, void *stream);

/*
 * Per-phase device timing for measurement.  While enabled, every kernel
 * launch of hsein_solve / hsein_backtransform on this plan is bracketed by
 * CUDA events on the caller's stream (no synchronization is added).
 * hsein_plan_profile waits for the last recorded event and returns, per phase,
 * the summed milliseconds and the number of launches since the last reset:
 *   phase 0 prepare (norms, prescale, initial state)
 *   phase 1 diagonal-tile sweep and solve (one launch per tile column)
 *   phase 2 shared-H update product (one launch per tile column but the last)
 *   phase 3 normalization and Givens backtransform
 *   phase 4 z = Q0 x
 * ms and launches point to arrays of nphases (<= HSEIN_NUM_PHASES) entries;
 * reset != 0 clears the record afterwards.
 */
#define HSEIN_NUM_PHASES 5
hsein_status hsein_plan_set_profiling(hsein_plan_t plan, int enable);
hsein_status hsein_plan_profile(hsein_plan_t plan, double *ms, int *launches, int nphases,
                                int reset);

/*
 * Measurement helper, outside the method (the paper has no counterpart): the
 * FP64 rate of the GPU's CUDA cores, the denominator of the FP64 rooflines.
 * Launches count threads (a multiple of 256, at most 2^31), each running
 * eight independent chains of iters fused multiply-adds, and writes one
 * double per thread to dOut (count entries, device).  *flops (may be NULL)
 * receives the launch's flop count, 16 * iters * count; time the launch with
 * events on `stream`.  Stream-ordered.
 */
hsein_status hsein_fp64_rate(long long iters, double *dOut, long long count, double *flops,
                             void *stream);

/* Query the plan's sizes; any output pointer may be NULL. */
hsein_status hsein_plan_info(hsein_plan_t plan, int *n, int *m_real, int *m_cplx,
                             int *ncol, int *br, size_t *workspace_bytes);

/* Release the plan (NULL is accepted). */
hsein_status hsein_plan_destroy(hsein_plan_t plan);

/* Static, human-readable text for a status code. */
const char *hsein_status_string(hsein_status status);

/*
 * Householder reduction to upper Hessenberg form on the GPU: A = Q0 H Q0^T
 * (Sec. 1: H and Q0 come from A before the solve; LAPACK's DGEHRD and
 * DORGHR).  Step k (k = 1..n-2) applies P = I - 2 v v^T / (v^T v),
 * v = x - alpha e_1 for x = H(k+1:n, k) and alpha = -sign(x_1) ||x||, from the
 * left and the right and accumulates Q0 <- Q0 P; H(k+1, k) becomes alpha and
 * H(k+2:n, k) exactly 0.  dA n x n (lda >= n, not modified); dH, dQ n x n
 * outputs (ldh, ldq >= n; distinct from dA and from each other).  dWork of
 * hsein_gehrd_workspace bytes, 256-byte aligned.  Stream-ordered (n - 2 steps
 * of a few kernels each).
 */
hsein_status hsein_gehrd_workspace(int n, size_t *workspace_bytes);
hsein_status hsein_gehrd(int n, const double *dA, int lda, double *dH, int ldh, double *dQ,
                         int ldq, void *dWork, size_t work_bytes, void *stream);

/*
 * Power-of-two balancing of an upper Hessenberg matrix, so that graded inputs
 * (rows and columns of very different scale) can use the split-precision
 * products: integer exponents e with Hb = D^-1 H D, D = diag(2^e) (exact:
 * every entry is scaled by a power of two; Hb is Hessenberg with the
 * eigenvalues of H, and x eigenvector of Hb <=> D x eigenvector of H).  The
 * exponents come from sweeps over i = 1..n that scale row i and column i
 * by 2^k, k the integer nearest to log2(sqrt(r_i / c_i)) for the
 * off-diagonal 1-norms r_i (row) and c_i (column), accepted when it lowers
 * r_i + c_i by at least 5%; the sweeps stop when one changes nothing or after
 * max_sweeps (the scaling step of Parlett and Reinsch's balancing, radix 2).
 * dH n x n (ldh >= n); dHb n x n output (ldhb >= n, not aliasing dH; entries
 * below the subdiagonal are written as 0); dExp n ints.  Stream-ordered.
 */
hsein_status hsein_balance(int n, const double *dH, int ldh, double *dHb, int ldhb, int *dExp,
                           int max_sweeps, void *stream);

/*
 * Eigenvectors of the balanced matrix back to the original one: every
 * column (a complex shift's [re, im] pair jointly) becomes D x / ||D x||_2,
 * computed with exponent arithmetic so that nothing overflows (components
 * more than 2^1074 below the column's largest flush to 0); zero columns (not
 * converged) stay zero.  m shifts, dWi their imaginary parts (device; a
 * nonzero marks a two-column complex shift), dX n x (m_real + 2 m_cplx) in
 * place.  Stream-ordered.
 */
hsein_status hsein_unbalance(int n, int m, const double *dWi, const int *dExp, double *dX,
                             int ldx, void *stream);

/* ------------------------------------------------------------------------
 * Batches of independent instances (matrices of different n and shift
 * counts) in one CUDA graph.  The paper solves one matrix at a time; it
 * groups the shifts of one matrix into blocks that reuse a bounded
 * workspace (Sec. 4.4, Alg. "hsrq3infinal").  Here every instance, or every
 * block of its shifts, is a sub-problem with its own plan and slice of one
 * workspace; the sub-problems are spread over `streams` concurrent chains
 * (longest first, each to the least loaded chain) and captured once into a
 * CUDA graph, which every hsein_batch_solve replays.
 * ------------------------------------------------------------------------ */
typedef struct hsein_batch_s *hsein_batch_t;

/* one instance: the arguments of hsein_solve (device pointers; dB may be
 * NULL for rho*e).  The pointers are fixed at hsein_batch_plan; the caller
 * refreshes the data in place between solves.  Which shifts are complex
 * (dWi != 0) is read once, at hsein_batch_plan, and must not change. */
typedef struct {
    int n, m_real, m_cplx;
    const double *dH;
    int ldh;
    const double *dWr, *dWi;
    const double *dB;
    int ldb;
    double *dX;
    int ldx;
    int *dStatus;
} hsein_instance;

/* tunables of a batch (hsein_batch_autotune searches them) */
typedef struct {
    int streams;     /* concurrent chains in the graph, 1..64; 0 = 16               */
    int br_policy;   /* tile height b_r by n: 0 = 64 for every n; 1 = 32 below       */
                     /* n = 512, else 64; 2 = 16 below 256, 32 below 1024, else 64    */
    int shift_block; /* at most this many shifts per sub-problem (a complex shift     */
                     /* counts once); 0 = all shifts of an instance in one            */
    int reserved;
} hsein_batch_config;

/*
 * Plan a batch of `count` instances (host array inst, copied).  opt applies
 * to every sub-problem except its tile height, which cfg->br_policy sets (opt
 * NULL = defaults; cfg NULL = {16, 1, 0}).  Reads every instance's dWi
 * (synchronously) to lay out the shift blocks.  *workspace_bytes receives the
 * size of the one device workspace hsein_batch_solve needs for this
 * configuration and for every configuration hsein_batch_autotune may pick.
 */
hsein_status hsein_batch_plan(hsein_batch_t *batch, int count, const hsein_instance *inst,
                              const hsein_options *opt, const hsein_batch_config *cfg,
                              size_t *workspace_bytes);

/*
 * Solve every instance: the results and statuses of each instance are those
 * hsein_solve gives for it alone with the same options and tile height.  The
 * first call for a workspace address captures the CUDA graph (on `stream`,
 * with forks to the batch's own streams); later calls only launch it.
 * Stream-ordered, asynchronous.
 */
hsein_status hsein_batch_solve(hsein_batch_t batch, void *dWork, size_t work_bytes, void *stream);

/*
 * Autotuner: times the batch (graph replays, CUDA events on `stream`) under
 * the configurations of a fixed candidate set, one coordinate at a time
 * (tile-height policies 0..2, then shift block widths {all, 512, 256, 128},
 * then chain counts {4, 8, 16, 24, 32, 48}), keeps the fastest for later solves and
 * returns it in *chosen (may be NULL) and its time in *ms (may be NULL).
 * Synchronizes `stream`; the instances' outputs hold the last trial's results.
 */
hsein_status hsein_batch_autotune(hsein_batch_t batch, void *dWork, size_t work_bytes,
                                  void *stream, hsein_batch_config *chosen, double *ms);

/* the configuration in use and the number of sub-problems / chains */
hsein_status hsein_batch_info(hsein_batch_t batch, hsein_batch_config *cfg, int *subproblems);

hsein_status hsein_batch_destroy(hsein_batch_t batch);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  The paper has no
 * counterpart; it is the deployment of the solver for a stream of requests.
 * The server owns one device arena (hbm_bytes) for solve workspaces and a
 * pool of streams.  hsein_server_progress retires finished solves, then
 * admits pending requests in arrival order while a stream is free and the
 * arena can hold their workspace: requests on the same matrix (same dH, n,
 * precision, and all with or all without starting vectors) that are pending
 * together are fused into one solve of their shift sets (the shared-H
 * updates then serve all of them), up to max_merge_shifts shifts.  Work of
 * admitted solves overlaps on the device; results are scattered back to each
 * request's own dX / dStatus and equal those of hsein_solve on the request
 * alone (columns never mix).  Single-threaded: the caller drives it.
 * ------------------------------------------------------------------------ */
typedef struct hsein_server_s *hsein_server_t;

typedef struct {
    hsein_instance inst; /* the solve; its buffers stay valid until the ticket completes */
    int precision;       /* 0 FP64 products, 1 split-precision products (b_r 64)          */
    int br;              /* tile height for precision 0 (0 = 64)                          */
    const int *dExp;     /* NULL, or the exponents of hsein_balance when inst.dH is a      */
                         /* balanced matrix: the results are then mapped back with        */
                         /* hsein_unbalance before the ticket completes                    */
} hsein_request;

/*
 * hbm_bytes: device memory the server allocates once for workspaces and the
 * fused requests' gathered shifts, starting vectors and results; max_jobs:
 * solves in flight at once (1..64); max_merge_shifts: the most shifts fused
 * into one solve (>= 1).  opt: robust / omega_log2 for every solve (NULL:
 * defaults).
 */
hsein_status hsein_server_create(hsein_server_t *server, size_t hbm_bytes, int max_jobs,
                                 int max_merge_shifts, const hsein_options *opt);

/* queue a request (copied); *ticket identifies it in hsein_server_progress.
 * HSEIN_ENOMEM if its footprint alone exceeds the arena. */
hsein_status hsein_server_submit(hsein_server_t server, const hsein_request *req,
                                 long long *ticket);

/*
 * Retire finished solves and admit pending requests.  The tickets completed
 * since the last call are written to done[0 .. *n_done) (at most max_done;
 * the rest are reported by later calls).  wait != 0 blocks until at least
 * one solve finishes when solves are in flight and none has finished yet.
 */
hsein_status hsein_server_progress(hsein_server_t server, long long *done, int max_done,
                                   int *n_done, int wait);

/* requests pending admission, solves in flight, arena bytes in use,
 * requests fused into the solves admitted so far and those solves' count */
hsein_status hsein_server_stats(hsein_server_t server, int *pending, int *running,
                                size_t *bytes_in_use, long long *requests_admitted,
                                long long *solves_admitted);

/*
 * Head-of-line bypass: when the oldest pending request does not fit the
 * arena, up to max_bypass later requests (looked for among the next 64) may
 * be admitted ahead of it before admission waits for it again; each admitted
 * request still takes its own footprint.  0 (the default) keeps strict
 * arrival order.  The paper has no counterpart.
 */
hsein_status hsein_server_set_bypass(hsein_server_t server, int max_bypass);

/* waits for the solves in flight, then frees everything */
hsein_status hsein_server_destroy(hsein_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* HSEIN_H */
