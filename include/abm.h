/*
 * abm.h - C ABI of the GB300 (sm_103a) fractional Adams-Bashforth-Moulton
 * history-convolution library.
 *
 * The method (arXiv 1611.08678, Sec. 2): solve the Caputo fractional ODE
 *     D_*^alpha y(t) = f(t, y(t)),  y(0) = y0,  t in [0, T],  alpha in (0, 1]
 * (eq. (1); alpha = 0 is excluded as degenerate) on the grid t_n = n h,
 * h = T/N, with the predictor of eq. (2)
 *     y^P_{n+1} = y0 + h^alpha sum_{k=0..n} b_{n-k} f_k
 * and the corrector that follows it
 *     y_{n+1} = y0 + h^alpha (c_n f_0 + sum_{k=1..n} a_{n-k} f_k
 *                             + f(t_{n+1}, y^P_{n+1}) / Gamma(alpha+2)),
 * f_k = f(t_k, y_k), with the weights b_m, a_m, c_m defined in Sec. 2 (the
 * printed '+' inside b_m is read as '-', the product-rectangle weight).
 * Every step of the computation runs in this library's CUDA kernels; the
 * caller supplies f by choosing one of the built-in systems below.
 *
 * Conventions for every entry point:
 *  - Return value: an abm_status.  Argument errors are detected on the host
 *    and returned synchronously, before anything is launched.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and is asynchronous.  Errors found on the
 *    device (non-finite state, a bounded wait that ran out) are recorded in
 *    the plan's status word and returned by abm_plan_sync().
 *  - Device pointers must point to memory of the device that was current
 *    when the plan was created.  The caller owns every buffer it passes; the
 *    plan owns its internal workspace (weights, f history, partial sums).
 *  - A plan is not thread-safe; calls that use one plan must be serialised
 *    on one stream.
 *  - abm_last_error() returns a human-readable message for the last failure.
 */
#ifndef ABM_H_
#define ABM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ABM_OK = 0,
  ABM_ERR_INVALID_ARG = 1, /* rejected on the host, nothing launched            */
  ABM_ERR_CUDA = 2,        /* a CUDA runtime call failed                        */
  ABM_ERR_OOM = 3,         /* device allocation failed                          */
  ABM_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                */
  ABM_ERR_NONFINITE = 5,   /* a state or f value became NaN/Inf                 */
  ABM_ERR_UNSUPPORTED = 6, /* valid request this build does not implement       */
  ABM_ERR_BOUNDS = 7       /* checked build only (libabm_gb300_checked.so, compiled
                              with ABM_CHECKED): a kernel computed an index outside
                              the buffer it addresses; the access was skipped    */
} abm_status;

/* Built-in right-hand sides f(t, y) with their dimension d and parameters:
 *  LINEAR       d=1  (lam, q0, q1)            f = lam y + q0 + q1 t
 *  MANUFACTURED d=1  (q0,q1,q2,beta,gam,e0,c1,c2,c3)
 *                    f = q0 + q1 t + q2 t^2 + beta r + gam r^3,
 *                    r = y - (e0 + c1 t^a + c2 t^(1+a) + c3 t^(2+a))
 *  LORENZ       d=3  (sigma, rho, beta)  x'=sigma(y-x), y'=x(rho-z)-y, z'=xy-beta z
 *  CHEN         d=3  (a, b, c)           x'=a(y-x), y'=(c-a)x-xz+cy, z'=xy-bz
 *  ROSSLER      d=3  (a, b, c)           x'=-y-z, y'=x+ay, z'=b+z(x-c)
 *  FINANCIAL    d=3  (a, b, c)           x'=z+(y-a)x, y'=1-by-x^2, z'=-x-cz
 *  HINDMARSH_ROSE d=3 (a, b, c, d, r, s, xR, I)   the 3-D neuron model the paper
 *                    simulates (Sec. 4, CUDA simulations; Hindmarsh and Rose 1984):
 *                    x'=y-ax^3+bx^2-z+I, y'=c-dx^2-y, z'=r(s(x-xR)-z)          */
typedef enum {
  ABM_SYS_LINEAR = 0,
  ABM_SYS_MANUFACTURED = 1,
  ABM_SYS_LORENZ = 2,
  ABM_SYS_CHEN = 3,
  ABM_SYS_ROSSLER = 4,
  ABM_SYS_FINANCIAL = 5,
  ABM_SYS_HINDMARSH_ROSE = 6
} abm_system;

/* Arithmetic of the far-history part (lags older than the current time tile).
 * The weights, the j = 0 and j = n+1 terms, the near lags and the PECE state
 * update are FP64 in every mode. */
typedef enum {
  ABM_PREC_FP64 = 0,      /* far history in FP64                                 */
  ABM_PREC_FP32_FAR = 1,  /* far history: FP32 operands, FP32 products/accumulate
                             within a lag block, blocks combined in FP64         */
  ABM_PREC_BF16X3_FAR = 2, /* far history on the tensor cores (tcgen05): each
                             operand split into three BF16 pieces
                             x = hi + mid + lo, the three largest cross products
                             hi*hi + hi*mid + mid*hi, FP32 accumulation of
                             the leading product over 256 history rows, a
                             compensated FP32 sum beyond, FP64 at the end    */
  ABM_PREC_BF16X6_FAR = 3  /* as BF16X3 with all six products down to 2^-24
                             (adds hi*lo, mid*mid, lo*hi) and the leading
                             product accumulated over 128 rows: FP32-level
                             error                                            */
} abm_precision;

typedef struct abm_plan_s* abm_plan;

typedef struct {
  abm_precision prec;  /* far-history arithmetic (batched path)                 */
  int n_max;           /* largest N any call will use (workspace is sized once)  */
  int max_batch;       /* largest M for abm_solve_batched (0: single only)       */
  int tile_B;          /* time-tile length B (0 = library default)               */
  int far_ctas;        /* CTAs of the single-trajectory far kernel (0 = auto)    */
  int use_graph;       /* batched solve: 1 = capture the launch sequence in a
                          CUDA graph on the first call and replay it on calls
                          with identical arguments (same host arrays' values,
                          same device pointers); profiling events are skipped
                          inside the graph                                        */
  long long spin_timeout_cycles; /* bound of every device-side wait in clock
                          cycles (0 = default, about two seconds)                */
  int test_withhold_tile; /* testing only, 0 = off.  k > 0: in abm_solve the far
                          CTAs never publish tile k-1, so the near CTA's wait
                          runs out and the call reports ABM_ERR_TIMEOUT           */
  int profile;         /* 1: bracket every kernel launch with CUDA events on the
                          launching stream (see abm_plan_kernel_times)           */
  int near_warps;      /* batched near kernel: warps per state component, the
                          chain warp plus helpers that sum the next step's window
                          (lag slices) while the chain runs: 0 = chosen from the
                          active tiles, 1 (chain only), 2, 3 or 5                */
  int far_split;       /* tensor-core far kernel: the history of each column tile
                          may be split across CTAs while the launch takes at most
                          far_split times the waves (CTAs / SM count, rounded up)
                          of the unsplit launch; 0 = 2                           */
  int near_split;      /* batched near kernel: CTAs per column tile.  A tile's 32
                          trajectories spread over 2, 4, 8 or 16 CTAs (lanes
                          of a trajectory sum interleaved slices of the lag
                          window) so that few active tiles still use many SMs:
                          0 = the largest of 8 and 4 whose CTAs fit on the
                          SMs, else none; 1 = never; 2, 4, 8 or 16 = that
                          split for every time tile (the adjoint runs 16 as 8) */
  int corrector_passes; /* corrector passes per step: 0 or 1 = PECE, the scheme
                          of Sec. 2; m = 2..8 = P(EC)^m E: the corrector, whose
                          last term g f(t_{n+1}, y_{n+1}) makes it implicit in
                          y_{n+1}, is applied m times, each pass evaluating f at
                          the previous pass's value (not in the paper; a common
                          variant of the predictor-corrector).  Forward solves
                          only: abm_adjoint returns ABM_ERR_UNSUPPORTED for m > 1;
                          YP still receives the predictor                      */
  int test_bad_index;  /* testing only, 0 = off; accepted by the checked build
                          alone (ABM_ERR_UNSUPPORTED otherwise).  k > 0: the
                          batched near kernel offsets the output row of
                          trajectory k-1 past the end of Y, so the checked
                          kernel skips that store and the call reports
                          ABM_ERR_BOUNDS                                        */
  int reserved[5];     /* must be zero                                            */
} abm_plan_opts;

/* Fills *o with the defaults (FP64, n_max = 0, tile_B = 0 ...). */
void abm_plan_opts_default(abm_plan_opts* o);

/* Dimension d and parameter count of a system; -1 for an unknown system. */
int abm_system_dim(abm_system sys);
int abm_system_nparams(abm_system sys);

/* Creates a plan for one system.  Allocates the workspace for n_max steps and
 * max_batch trajectories on the current device.  ABM_ERR_INVALID_ARG for
 * n_max < 1, negative sizes, an unknown system or precision, an option outside
 * the values documented above or nonzero reserved fields (all checked before
 * any CUDA call; *out stays NULL); ABM_ERR_OOM when the workspace does not
 * fit; ABM_ERR_UNSUPPORTED for tile_B other than 0, 32 or 64, and for a
 * tensor-core precision (BF16X3, BF16X6) with a system of dimension 1 or with
 * tile_B = 32. */
abm_status abm_plan_create(abm_plan* out, abm_system sys, const abm_plan_opts* o);

/* Frees the plan and its workspace (synchronises the device first). */
abm_status abm_plan_destroy(abm_plan p);

/* Synchronises `stream`, then returns and clears the plan's device status
 * word (ABM_OK, ABM_ERR_NONFINITE or ABM_ERR_TIMEOUT); abm_last_error() then
 * names where it happened.  If `where` is not NULL it receives the packed
 * detail: for ABM_ERR_NONFINITE trajectory << 32 | step of the first
 * non-finite value; for ABM_ERR_TIMEOUT site << 56 | unit << 32 | position,
 * site 1 = the single-trajectory stepping CTA waiting for the far sums of
 * time tile `unit`, 2 = a single-trajectory far CTA waiting for the rows
 * before time tile `unit`, 3..5 = the tensor-core far kernel of column tile
 * `unit` (3 loader, 4 MMA issuer waiting for an accumulator, 5 MMA issuer
 * waiting for the operands of K block `position`); for ABM_ERR_BOUNDS (the
 * checked build) kernel << 52 | index of the first index found outside its
 * buffer. */
abm_status abm_plan_sync(abm_plan p, void* stream, int64_t* where);

/* Message of the last failure on this plan (owned by the plan, valid until
 * the next call on it).  Never NULL. */
const char* abm_last_error(abm_plan p);

/* A1 - weight generation (Sec. 2 weight definitions; the CUDA variant of the
 * paper's per-thread weight precompute, Sec. 4 "CUDA simulations").
 * Writes b[m], a[m], c[m] for m = 0..M (device arrays of M+1 doubles) for
 * this alpha in FP64.  Large lags use cancellation-free series, small lags a
 * 16-point Gauss-Legendre quadrature of the product-integration kernels.
 * alpha in (0, 2] (the definitions hold for every positive order), M >= 0. */
abm_status abm_weights(abm_plan p, double alpha, int M, double* b, double* a, double* c,
                       void* stream);

/* Single trajectory (the paper's ParABM problem, Sec. 3 Fig. 2 inputs
 * T = N h, N, y0).  alpha in (0, 1], h > 0 finite, 1 <= N <= n_max.
 * params: host array of abm_system_nparams(sys) doubles; y0: host array of d
 * doubles (finite).  Y: device array of (N+1)*d doubles, row n = y_n
 * (Y[0..d-1] = y0).  YP (may be NULL): device array of (N+1)*d doubles that
 * receives the predictor values y^P_n (row 0 = y0).  FP64 throughout: the
 * far history is split across the GPU's SMs, the near lags and the
 * sequential PECE steps run in one CTA. */
abm_status abm_solve(abm_plan p, double alpha, double h, int N, const double* params,
                     const double* y0, double* Y, double* YP, void* stream);

/* abm_solve with HOST buffers (the paper has no counterpart: it is the call a
 * user makes with the result in host memory).  Arguments as abm_solve; Y (and
 * YP when not NULL) are host arrays of (N+1)*d doubles, written once the
 * solve has run (the solve writes into a device copy owned by the plan,
 * allocated by the first call, then one copy per array is enqueued on
 * `stream`).  The work is complete once `stream` has passed it
 * (abm_plan_sync); page-locked host memory keeps the copies asynchronous. */
abm_status abm_solve_host(abm_plan p, double alpha, double h, int N, const double* params, const double* y0,
                          double* Y, double* YP, void* stream);

/* The general problem of eq. (1) for one trajectory: an order per state
 * component, each in (0, 2] (a non-commensurate system when they differ), and
 * for components of order above one the initial derivative y_i'(0), which
 * enters the Taylor sum of the predictor (eq. (2)) and of the corrector,
 *     sum_{k=0..ceil(alpha_i)-1} t_{n+1}^k / k! y_i^(k)(0) = y_i(0) + t_{n+1} y_i'(0);
 * component i uses the Sec. 2 weights b, a, c and h^alpha_i, 1/Gamma(alpha_i+2)
 * of its own order.  alpha: host array of d orders; y0d: host array of d
 * values or NULL (zero), read only for components with alpha_i > 1; every
 * other argument as abm_solve.  ABM_ERR_INVALID_ARG for an order outside
 * (0, 2] or a non-finite y0d. */
abm_status abm_solve_ext(abm_plan p, const double* alpha, double h, int N, const double* params,
                         const double* y0, const double* y0d, double* Y, double* YP, void* stream);

/* Batched trajectories (independent problems with their own alpha, h, N,
 * parameters and initial values).  alpha, h, N: HOST arrays of M entries
 * (they drive the scheduling: trajectories are grouped by alpha and ordered
 * by N on the host).  params: device array M x nparams; y0: device M x d.
 * Y: device array M x ldY x d with ldY >= max(N)+1; trajectory i's rows
 * 0..N[i] are written, the rest are left untouched.  YP (may be NULL) has
 * the layout of Y and receives y^P.  The plan's precision selects the
 * far-history arithmetic.  1 <= M <= max_batch, 1 <= N[i] <= n_max. */
abm_status abm_solve_batched(abm_plan p, int M, const double* alpha, const double* h,
                             const int* N, const double* params, const double* y0, double* Y,
                             long long ldY, double* YP, void* stream);

/* The general problem of eq. (1) for a batch (see abm_solve_ext): alpha is a
 * HOST array of M x d orders, each in (0, 2]; y0d a DEVICE array M x d of
 * initial derivatives or NULL (zero), read for components of order above
 * one; every other argument as abm_solve_batched.  Trajectories with equal
 * order tuples share one weight set per component.  A batch may hold at most
 * 24 distinct orders and 24 distinct order tuples (ABM_ERR_UNSUPPORTED
 * beyond).  The tensor-core precisions (BF16X3/X6) take orders that are equal
 * across the components of each trajectory (one Toeplitz operand per column
 * tile) and return ABM_ERR_UNSUPPORTED otherwise; FP64 and FP32 plans take
 * any orders. */
abm_status abm_solve_batched_ext(abm_plan p, int M, const double* alpha, const double* h, const int* N,
                                 const double* params, const double* y0, const double* y0d, double* Y,
                                 long long ldY, double* YP, void* stream);

/* abm_solve_batched with HOST buffers (the paper has no counterpart: it is
 * the call a user makes with inputs and results in host memory).  alpha, h,
 * N as above; params (M x nparams) and y0 (M x d) are read from host memory,
 * and trajectory i's rows 0..N[i] of Y (and YP when not NULL), laid out as in
 * abm_solve_batched with leading dimension ldY, are written to host memory;
 * the rest of Y is left untouched.  The inputs are copied up on `stream`
 * first.  Rows are copied down on a stream of the plan while the remaining
 * time tiles run: a trajectory's last rows right after the time tile that
 * finishes it, and, whenever the still-running trajectories form at most 32
 * runs of consecutive indices (always, when all N[i] are equal), their rows
 * of each time tile right after that tile, as 2D copies.  The call's work, copies included, is complete once `stream`
 * has passed it (abm_plan_sync).  The host arrays must stay valid until then
 * and should be page-locked (cudaHostAlloc / cudaHostRegister): with pageable
 * memory the copies still happen but stop overlapping.  The first call
 * allocates the plan's device copies of params, y0 and Y (max_batch rows of
 * n_max+1 steps each) and a copy stream; later calls reuse them, so calls on
 * one plan must not run concurrently.  Never captured in a CUDA graph. */
abm_status abm_solve_batched_host(abm_plan p, int M, const double* alpha, const double* h,
                                  const int* N, const double* params, const double* y0, double* Y,
                                  long long ldY, double* YP, void* stream);

/* Adjoint of abm_solve_batched (the discrete adjoint of exactly the scheme
 * above; the paper has no adjoint).  The arguments alpha .. ldY must be those
 * of a completed abm_solve_batched call on this plan whose outputs Y and YP
 * (both required here) are still intact.  dLdY: device array with the layout
 * of Y holding the partial derivatives of a scalar loss with respect to every
 * y_n (rows beyond N[i] ignored).  Outputs (device): dparams M x nparams and
 * dy0 M x d, the total derivatives of the loss.  The Jacobians of f are
 * recomputed from Y and YP; no Jacobian is stored. */
abm_status abm_adjoint(abm_plan p, int M, const double* alpha, const double* h, const int* N,
                       const double* params, const double* y0, const double* Y, const double* YP,
                       long long ldY, const double* dLdY, double* dparams, double* dy0,
                       void* stream);

/* Checkpoint and resume.  Every step of the scheme reads the whole history
 * (Sec. 2: y_{n+1} depends on f_0..f_n), so the state of a solve at step n is
 * y(0), y'(0) and the f history f_0..f_n; the paper has no checkpointing.
 *
 * abm_history: copies f_0..f_{rows-1} of the last single-trajectory solve on
 * this plan (abm_solve, abm_solve_ext or abm_solve_resume; rows <= its N+1)
 * to F, rows x d doubles in host or device memory, enqueued on `stream`
 * (page-locked host memory keeps the copy asynchronous). */
abm_status abm_history(abm_plan p, int rows, double* F, void* stream);

/* abm_solve_resume: continues a single-trajectory solve of the problem given
 * by alpha (d orders), h, params, y0, y0d (as abm_solve_ext) from step n0 to
 * step N (0 <= n0 <= N <= n_max): F holds f_0..f_n0 of the earlier solve
 * ((n0+1) x d doubles, host or device, as abm_history wrote them; unused when
 * n0 < 32).  Stepping restarts at the time tile (32 steps) that holds step
 * n0 + 1: rows s..N of Y (and YP) are written, where s is n0 rounded down to
 * a multiple of 32; rows s+1..n0 are recomputed with the arithmetic of an
 * uninterrupted solve, so a solve split at any n0 and resumed equals the
 * uninterrupted one bit for bit.  Rows 0..s-1 of Y are not touched. */
abm_status abm_solve_resume(abm_plan p, const double* alpha, double h, int n0, int N, const double* params,
                            const double* y0, const double* y0d, const double* F, double* Y, double* YP,
                            void* stream);

/* abm_history_batched: copies f_0..f_{min(rows, N[i]+1)-1} of every
 * trajectory of the last batched solve on this plan into F, a DEVICE array
 * M x ldF x d (ldF >= rows), row k of trajectory i at (i ldF + k) d.  The
 * arguments alpha (M x d orders, the abm_solve_batched_ext convention), h and
 * N must be those of that solve. */
abm_status abm_history_batched(abm_plan p, int M, const double* alpha, const double* h, const int* N, int rows,
                               double* F, long long ldF, void* stream);

/* abm_solve_batched_resume: continues a batched solve (arguments as
 * abm_solve_batched_ext) from step n0 (0 <= n0 <= N[i] for every i): F is a
 * DEVICE array M x ldF x d (ldF >= n0+1) holding f_0..f_n0 of each
 * trajectory, as abm_history_batched wrote them (unused when n0 < tile_B).
 * Stepping restarts at the time tile (tile_B steps, 64 by default) that holds
 * step n0 + 1: rows s+1..N[i] of Y (and YP) are written, s = n0 rounded down
 * to a multiple of tile_B, rows s+1..n0 recomputed as an uninterrupted solve
 * computes them.  With an FP64 plan the result equals the uninterrupted solve
 * bit for bit; the tensor-core plans add K-split far sums with atomics, whose
 * order (and last bit) varies from run to run.  Never captured in a graph. */
abm_status abm_solve_batched_resume(abm_plan p, int M, const double* alpha, const double* h, const int* N, int n0,
                                    const double* params, const double* y0, const double* y0d, const double* F,
                                    long long ldF, double* Y, long long ldY, double* YP, void* stream);

/* Far-history sums alone (the A2 contraction, exposed for parity tests and
 * roofline measurement).  F: device, rows x cols row-major FP64 history
 * (row k = f_k).  For targets n = s..s+B-1 and history rows k in [k_lo, k_hi)
 * with 1 <= k_lo <= k_hi <= s:
 *   P[i][col] = sum_k b_{s+i-k} F[k][col],  C[i][col] = sum_k a_{s+i-k} F[k][col]
 * (P, C: device B x cols).  Uses the plan's precision and this alpha's
 * weights. */
abm_status abm_far_history(abm_plan p, double alpha, const double* F, long long rows,
                           long long cols, long long s, int B, long long k_lo, long long k_hi,
                           double* P, double* C, void* stream);

/* Kernel kinds reported by abm_plan_kernel_times. */
typedef enum {
  ABM_KERNEL_WEIGHTS = 0,    /* A1 weight generation (and its shadows)            */
  ABM_KERNEL_FAR = 1,        /* A2 far history of the batched path                */
  ABM_KERNEL_NEAR = 2,       /* A3 near PECE steps of the batched path            */
  ABM_KERNEL_SINGLE = 3,     /* the persistent single-trajectory kernel           */
  ABM_KERNEL_ADJOINT = 4,    /* A6 adjoint kernels                                */
  ABM_KERNEL_KINDS = 5
} abm_kernel_kind;

/* Tracing.  Every call counts the kernels it launches per kind; with
 * opts.profile = 1 each launch is also bracketed by CUDA events on its
 * stream.  Synchronises `stream`, then returns the launches and the summed
 * device time in milliseconds (0 without profiling) of one kind since the
 * last reset; resets that kind's counters when reset != 0. */
abm_status abm_plan_kernel_times(abm_plan p, abm_kernel_kind kind, void* stream, int reset,
                                 long long* launches, double* total_ms);

/* abm_solve_noalloc - the single-trajectory solve (abm_solve) for callers
 * that must not allocate device memory: code whose device memory is budgeted
 * up front by a host framework or memory pool, real-time or embedded callers
 * that forbid allocation after start-up, and plug-ins that run inside another
 * process's CUDA context.  The paper has no counterpart; it exists for those
 * callers only.
 *
 * No plan is needed and nothing is allocated: the call makes no cudaMalloc,
 * cudaFree or other allocating call.  Its scratch (the f history, the
 * weights, the far-history partial sums, the wait flags and the status word)
 * lives in one static device array of about 3.2 MB compiled into this
 * library, which every GPU that loads the library holds until the process
 * exits.  That fixes the largest problem: 1 <= N <= 32768 (d <= 3); larger N
 * returns ABM_ERR_INVALID_ARG with a message saying so.
 *
 * Arguments as abm_solve (sys instead of a plan; params and y0 host arrays,
 * Y and YP device arrays of (N+1)*d doubles owned by the caller, YP may be
 * NULL), plus errbuf/errbuf_len (may be NULL/0): a message for any failure,
 * the empty string on success.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing once the library's module is
 * loaded; nothing is cached, so the address cannot go stale after a device
 * reset).  The first call on a device may load that module: make it before
 * any stream capture.  The call is synchronous: it waits for `stream` and returns the
 * device status (ABM_ERR_NONFINITE, ABM_ERR_TIMEOUT) itself.  All calls share
 * the one array, which keeps the previous call's contents (each call clears
 * what must start at zero), so calls that overlap on the GPU - from several
 * host threads or on several streams of one device at once - race and give
 * wrong results; serialise them. */
abm_status abm_solve_noalloc(abm_system sys, double alpha, double h, int N, const double* params,
                             const double* y0, double* Y, double* YP, void* stream, char* errbuf,
                             size_t errbuf_len);

#ifdef __cplusplus
}
#endif

#endif /* ABM_H_ */
