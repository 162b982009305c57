/*
 * bt.h -- C ABI of the GB300 partition-method solver for structured sparse
 * systems A x = f (Amodio & Brugnano, "Parallel Factorizations in Numerical
 * Analysis", Sec. 2, Eq. (syst)).
 *
 * The method: A is rearranged into local blocks A^(i) coupled through small
 * separator blocks a^(i) (Sec. 2, Eq. (parpart); for BABD matrices Eq.
 * (parpart1)), factored as A = F T G (Eqs. (parfact)-(parG)) with every
 * partition factored independently (Eq. (parblock)), and solved by the
 * F-solve and G-solve in parallel and the reduced system of Eq. (redmatr) /
 * (redmatr1) on the separators (Sec. 2, "the solution of the system with the
 * matrix T requires ... a reduced system").  Here each partition is a CTA (or
 * a thread, for blocks of order m <= 4) of one GPU, and the reduced system is
 * itself partitioned recursively on the device until one partition is left.
 *
 * Conventions for every entry point below:
 *  - All array pointers are DEVICE pointers (cudaMalloc'ed or
 *    torch-allocated memory on the plan's device), owned by the caller, in
 *    row-major FP64.  Right-hand sides and solutions are [rows*m][nrhs].
 *  - Calls are asynchronous on the plan's CUDA stream, except where stated.
 *    The returned status covers argument checks and launch errors; numerical
 *    failures (a zero or non-finite pivot) are recorded in a device status
 *    word and returned by the next synchronising call (bt_sync/abd_sync,
 *    bt_refine/abd_refine).
 *  - Nothing throws across the ABI.  A plan is not thread-safe: one host
 *    thread at a time may use it.
 */
#ifndef BT_H
#define BT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BT_OK = 0,
    BT_ERR_INVALID = 1,        /* bad argument or call order */
    BT_ERR_NOMEM = 2,          /* device allocation failed */
    BT_ERR_SINGULAR = 3,       /* zero pivot in a pivot block */
    BT_ERR_NONFINITE = 4,      /* inf/nan pivot */
    BT_ERR_NOT_CONVERGED = 5,  /* refinement hit maxit */
    BT_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
    BT_ERR_CUDA = 7            /* CUDA runtime error */
} bt_status;

typedef enum {
    BT_FP64 = 0,     /* every factorization step in FP64 */
    BT_FP32_IR = 1,  /* local factors in FP32, reduced system FP64; solve via FP64 refinement */
    BT_BF16_IR = 2   /* as BT_FP32_IR, with the local Schur-complement product B_j Y_{j-1}
                        taken on the tensor cores with BF16 operands and FP32 accumulation
                        (m >= 16; smaller blocks use the FP32 path) */
} bt_prec;

typedef struct bt_plan_s* bt_plan;
typedef struct bt_plan_s* abd_plan;

/* Human-readable name of a status code (static string). */
const char* bt_status_string(bt_status s);

/* ---------------------------------------------------------------------
 * Block tridiagonal systems (Sec. 2: "(block) tridiagonal"; m = 1 is the
 * scalar tridiagonal case).  Block row j (0 <= j < nblk):
 *     B_j x_{j-1} + D_j x_j + C_j x_{j+1} = f_j,
 * with B, D, C of shape [nblk][m][m]; B_0 and C_{nblk-1} are never read.
 * ------------------------------------------------------------------- */

/* Create a plan on the current CUDA device.
 *   nblk     number of block rows N (>= 1);  m block order, 1..32 (orders other
 *            than 1, 2, 4, 8, 16, 32 are embedded in the next of these with an
 *            identity tail: the caller's arrays keep order m).
 *   nrhs_max largest nrhs later passed to bt_solve/bt_refine (1..32).
 *   prec     precision of the local factors (bt_prec).
 *   p        number of top-level partitions (Sec. 2, "p processors"); 0 picks
 *            one from the device's SM count; must satisfy 1 <= p <= (nblk+1)/2.
 *   stream   cudaStream_t for every later call (NULL = legacy default stream).
 * Allocates all device workspace (factors of every recursion level).
 * Returns BT_ERR_INVALID on bad sizes, BT_ERR_NOMEM if allocation fails. */
bt_status bt_plan_create(bt_plan* plan, int64_t nblk, int m, int nrhs_max, int prec, int64_t p,
                         void* stream);

/* Partitioning parameters of plan step A0 (Sec. 2: "p processors"; here the
 * partition count of every recursion level).  Zero fields take the defaults.
 *   p0           partitions of the top level (0: ctas_per_sm x SM count,
 *                capped at nblk/4 for m >= 8 or nblk/8 for m <= 4)
 *   ctas_per_sm  level-0 partitions per SM when p0 = 0 (default 12 for m = 8,
 *                4 for m = 16, 3 for m = 32, 512 for m <= 4 where a partition is
 *                one thread)
 *   sub_rows     block rows per partition on the recursion levels (>= 2, default 4)
 *   top_rows     a level with at most this many block rows is solved by one
 *                partition (block tridiagonal) or directly (BABD); default 8
 *   reduced      solver of the top-level reduced system of a block tridiagonal
 *                plan with m >= 8: 0 = partitioned again recursively (default),
 *                1 = block cyclic reduction (the cyclic-reduction variant of
 *                Sec. 2 with one synchronisation per reduction step).  BABD
 *                plans (abd_plan_create_tuned): 1 = cyclic reduction of the
 *                whole system instead of partitions
 *   tp_block     CTA shape of the thread-per-partition kernels used for m <= 4:
 *                threads per CTA, 64, 128 or 256 (0: 128)
 *   local        local factorization of a block tridiagonal plan with m >= 8:
 *                0 = block LU with fill-in spikes (default); L >= 1 = cyclic
 *                reduction inside partitions of 2^L block rows (the
 *                cyclic-reduction factorization of Sec. 2: no fill-in spikes;
 *                the separators are the block rows at multiples of 2^L).  All
 *                partitions take their reduction steps together, one launch
 *                per step; the steps run in the plan's local precision (FP32
 *                for BT_FP32_IR and BT_BF16_IR) and the reduced system left
 *                after L steps is solved by FP64 cyclic reduction.  L is capped
 *                so that at least the last block row is FP64.  p0, ctas_per_sm,
 *                sub_rows, top_rows and reduced are then unused.
 *   pivot        1 = pivoted partitions (the variant of Sec. 2 for matrices
 *                with singular or ill-conditioned local blocks): when the
 *                local factorization of a partition meets a pivot block whose
 *                Gauss-Jordan pivot is at most tau times the largest entry of
 *                that block row (bt_plan_set_pivot_tol, default 1e-3), the
 *                factorization of the partition stops there, the row becomes
 *                one more separator and the partition is factored again as
 *                two (one pass finds every breakdown: after one the local
 *                factorization restarts at the next row); the enlarged
 *                reduced system (at most max(2 p0, nblk/16) + 15 block rows)
 *                is solved by Gaussian elimination with partial
 *                pivoting over pairs of block rows.  bt_factor then
 *                synchronises once per splitting pass; reduced and local are
 *                unused; graph capture only of solves (what = 2).  If more
 *                rows break down than the reduced system has room for,
 *                bt_factor returns BT_ERR_SINGULAR.
 *                2 = partitions factored by local QR (the variant of Sec. 2
 *                with N^(i) = Q^(i), S^(i) = R^(i)): every partition's local
 *                block is reduced by block Householder steps (one CTA per
 *                partition, FP64), so singular or ill-conditioned diagonal
 *                blocks need neither splits nor host synchronisation; the
 *                reduced system keeps p - 1 block rows and is solved by
 *                Gaussian elimination with partial pivoting.  BT_FP64 only
 *                (other precisions: BT_ERR_INVALID); reduced and local are
 *                unused; factor and solve may be captured.  A singular local
 *                block (an exactly zero R diagonal entry) is reported as
 *                BT_ERR_SINGULAR.
 *   serial       1 = captured sequences (bt_plan_capture with factor) run on
 *                one stream.  0 (default): the factorization of the levels
 *                above level 0 (and the reduced system's cyclic reduction)
 *                runs on a second stream, concurrently with the level-0
 *                forward substitution, which needs only the level-0 factors;
 *                the streams join before the reduced system's right-hand side
 *                is used.  Eager bt_factor / bt_solve calls always use the
 *                plan's stream alone. */
typedef struct {
    int64_t p0;
    int ctas_per_sm;
    int sub_rows;
    int top_rows;
    int reduced;
    int tp_block;
    int local;
    int pivot;
    int serial;
} bt_tuning;

/* bt_plan_create with explicit partitioning parameters (NULL = defaults). */
bt_status bt_plan_create_tuned(bt_plan* plan, int64_t nblk, int m, int nrhs_max, int prec,
                               const bt_tuning* tuning, void* stream);

/* Factor A = F T G (Eqs. (parfact)-(parblock)): the local block LU of every
 * partition with its fill-in spikes, the reduced matrix of Eq. (redmatr),
 * and recursively its own factorization.  Reads B, D, C; does not modify
 * them.  The plan keeps the three pointers for bt_residual/bt_refine: the
 * caller keeps the arrays alive and unchanged until the next bt_factor or
 * bt_plan_destroy.  Resets the device status word. */
bt_status bt_factor(bt_plan plan, const double* B, const double* D, const double* C);

/* Solve A X = F with the factors (the F-, T- and G-solves of Sec. 2):
 * F, X: [nblk*m][nrhs], 1 <= nrhs <= nrhs_max; X may not alias F.
 * With a BT_FP32_IR/BT_BF16_IR plan this is the low-precision solve only
 * (use bt_refine for an FP64-accurate result). */
bt_status bt_solve(bt_plan plan, const double* F, double* X, int nrhs);

/* Banded matrices (Sec. 2: a matrix with s lower and r upper off-diagonals is
 * block tridiagonal with blocks of order max(s, r)).  Converts the n x n band
 * matrix in band storage, band[(r + i - k) * n + k] = A[i][k] for
 * -r <= i - k <= s, into B, D, C of N = ceil(n/m) block rows of order m
 * (max(s, r, 1) <= m <= 32); unknowns beyond n get identity rows, so right-hand
 * sides are padded with zeros to N*m rows.  Device arrays, asynchronous. */
bt_status bt_band_to_blocks(int64_t n, int s, int r, const double* band, int m, double* B, double* D, double* C,
                            void* stream);

/* y[i] = 1/x[i] for n FP64 values (device arrays, asynchronous on `stream`)
 * with the reciprocal that every FP64 pivot step of the factorizations uses
 * instead of a division: the hardware seed rcp.approx.ftz.f64 refined by one
 * third-order Newton step, r = r0 (1 + e + e^2) with e = 1 - x r0 (within one
 * unit in the last place of 1/x); zero, subnormal, huge (|x| >= 2^1022) and
 * non-finite x take the IEEE division.  Exposed so that its accuracy can be
 * checked against IEEE 1/x.  BT_ERR_INVALID on n < 0 or null arrays. */
bt_status bt_device_rcp(int64_t n, const double* x, double* y, void* stream);

/* R = F - A X in FP64 with the matrices given to the last bt_factor. */
bt_status bt_residual(bt_plan plan, const double* F, const double* X, double* R, int nrhs);

/* R = F - A X as the plan's refinement forms it (the refinement residual of
 * Sec. 2's mixed-precision use, exposed so that it can be checked entry by
 * entry): FP64 arithmetic for BT_FP64 plans; for refined plans (BT_FP32_IR,
 * BT_BF16_IR) FP64-accurate arithmetic off the FP64 pipe -- block order 16
 * with at most 8 right-hand sides: the products on the tensor cores by an
 * error-free split into 8-bit digit planes (Ozaki, Ogita, Oishi, Rump 2012),
 * about 2^-49 of max|a_ij| max|x_j| per entry; otherwise double-float
 * (hi + lo FP32 pairs, TwoProduct and TwoSum: the compensated dot product of
 * Ogita, Rump and Oishi 2005), about sqrt(3m) 2^-48 of sum_j |a_ij||x_j| --
 * in both cases rounded to FP32 precision at the end (relative 2^-24 of
 * |R|; the correction solve is FP32).  Same arguments and errors as
 * bt_residual. */
bt_status bt_refine_residual(bt_plan plan, const double* F, const double* X, double* R, int nrhs);

/* Iterative refinement to FP64 accuracy: X = solve(F); repeat
 * { R = F - A X (FP64); stop if the normwise backward error
 *   ||R||_inf / (||A||_inf ||X||_inf + ||F||_inf) <= eta_tol (see
 *   bt_plan_set_backward_tol) or if the last correction had
 *   ||D||_F <= tol ||X||_F; else D = solve(R); X += D } for at most maxit
 * corrections.  SYNCHRONISES once per round (a few norms copied to the host).
 * iters_out (may be NULL): corrections applied; relcorr_out (may be NULL):
 * last ||D||_F/||X||_F (-1 if none).  Returns BT_ERR_NOT_CONVERGED after
 * maxit, or a recorded numerical status. */
bt_status bt_refine(bt_plan plan, const double* F, double* X, int nrhs, double tol, int maxit,
                    int* iters_out, double* relcorr_out);

/* Asynchronous refinement for schedulers that must not block: enqueue
 * X = solve(F) and exactly `sweeps` (0..30) corrections { R = F - A X (FP64);
 * D = solve(R); X += D } on the plan's stream, with no host synchronisation.
 * Works for block tridiagonal and BABD plans.  The sequence ends with a
 * residual of the result.  bt_refine_result later synchronises and reports
 * ||D||_F/||X||_F of the last correction: BT_OK if that residual's backward
 * error is below the threshold (bt_plan_set_backward_tol), if the last
 * correction is <= tol, or if the estimated forward error is below the
 * target set by bt_plan_set_forward_tol; BT_ERR_NOT_CONVERGED otherwise (or
 * a numerical status). */
bt_status bt_refine_async(bt_plan plan, const double* F, double* X, int nrhs, int sweeps);
bt_status bt_refine_result(bt_plan plan, double tol, double* relcorr_out);

/* Backward-error threshold of the refinement stopping test (default, when
 * eta_tol < 0: 4 (3m + 1) u with u = 2^-53, a few roundings per residual
 * term).  The async variant also ends with a residual of the result, and
 * bt_refine_result accepts it when that backward error is below the
 * threshold or the last correction is below tol. */
bt_status bt_plan_set_backward_tol(bt_plan plan, double eta_tol);

/* Forward-error target of the refinement stopping test, an option of the
 * mixed-precision refinement (the paper's method has no refinement step;
 * default: not used).  With fwd_tol > 0, bt_refine also stops, and
 * bt_refine_result also accepts, when after k >= 1 corrections the estimated
 * relative forward error of X,
 *   rho / (1 - rho) * ||D_k||_F / ||X||_F,  rho = ||D_k||_F / ||D_(k-1)||_F,
 * (D_0 = the first solve, taken as ||X||_F), is <= fwd_tol: the error bound
 * of a linearly converging refinement with contraction rho, the correction
 * ratio test of Demmel, Hida, Kahan, Li, Mukherjee and Riedy (2006).  No
 * estimate (never stops on it) while rho >= 1/2.  An estimate, not a bound:
 * the backward-error test above stays the certificate.  fwd_tol <= 0 turns
 * the option off; BT_ERR_INVALID for a NaN. */
bt_status bt_plan_set_forward_tol(bt_plan plan, double fwd_tol);

/* Breakdown threshold tau of a plan created with bt_tuning.pivot = 1
 * (0 <= tau < 1; default 1e-3): larger values split partitions more often
 * (more separators, smaller multipliers).  Takes effect at the next
 * bt_factor.  BT_ERR_INVALID for other plans. */
bt_status bt_plan_set_pivot_tol(bt_plan plan, double tau);

/* ||A||_inf of the matrices given to the last bt_factor / abd_factor, as the
 * stopping test uses it: FP32 row sums of the entries truncated toward zero
 * (relative error below 1e-5).  Synchronises the plan's stream.  For a plan
 * whose block order is embedded in a larger one the identity tail of the
 * padded blocks contributes rows of sum 1. */
bt_status bt_plan_anorm(bt_plan plan, double* anorm_out);

/* Plans on caller-provided device memory (e.g. from a pooling allocator), so
 * that creating a plan performs no device allocation: bt_plan_workspace_size
 * returns the bytes a plan of this shape needs (kind 0: block tridiagonal,
 * n = block rows; kind 1: BABD, n = N), bt_plan_create_in builds the plan in
 * `workspace` (256-byte aligned, at least that many bytes, owned by the
 * caller and kept alive until bt_plan_destroy, which does not free it). */
bt_status bt_plan_workspace_size(int kind, int64_t n, int m, int nrhs_max, int prec, const bt_tuning* tuning,
                                 int64_t* bytes);
bt_status bt_plan_create_in(bt_plan* plan, int kind, int64_t n, int m, int nrhs_max, int prec,
                            const bt_tuning* tuning, void* workspace, int64_t bytes, void* stream);

/* Capture one call sequence of the plan into a CUDA graph held by the plan,
 * so that later runs are one graph launch (no per-kernel launch gaps):
 *   what = 1: factor (matrices of the last bt_factor/abd_factor) + solve(F -> X)
 *   what = 2: solve(F -> X) with the current factors
 *   what = 3: factor + bt_refine_async(F -> X, sweeps)
 * The pointers are bound into the graph; bt_plan_replay re-runs it on the
 * plan's stream (new values in the same arrays are picked up).  Capture
 * synchronises the stream and replaces any earlier graph of the plan. */
bt_status bt_plan_capture(bt_plan plan, int what, const double* F, double* X, int nrhs, int sweeps);

/* Factor + solve (sweeps = -1, BT_FP64 plans) or factor + bt_refine_async
 * with `sweeps` corrections (0..30, refined plans) from HOST arrays: B, D, C
 * [N][m][m] and F [N*m][nrhs] are host memory read by the call, X
 * [N*m][nrhs] host memory written by it.  Page-locked (pinned) host memory
 * lets the copies run asynchronously; pageable memory works but the copies
 * then synchronise.  The block rows are copied in chunks of level-0
 * partitions on a copy stream of the plan, and each chunk's local
 * factorizations (Eq. (parblock)) start on their own stream as soon as their
 * rows have arrived, so the transfer overlaps the FP64 work; then the
 * right-hand side, the reduced systems, the solve (or refinement) and the
 * copy of X back, ordered on the plan's stream.  Asynchronous: bt_sync (or
 * bt_refine_result) waits and returns the numerical status; the host arrays
 * must stay valid until then.  The first call allocates device copies of the
 * arrays (3 N m^2 + 2 N m nrhs_max doubles, cudaMalloc) owned by the plan;
 * later factorizations of the plan (bt_factor) replace the bound matrices.
 * Block tridiagonal plans without padding, pivoting or local cyclic
 * reduction; BT_ERR_INVALID otherwise. */
bt_status bt_factor_solve_host(bt_plan plan, const double* B, const double* D, const double* C, const double* F,
                               double* X, int nrhs, int sweeps);

/* bt_factor_solve_host recorded into the plan's CUDA graph (as bt_plan_capture
 * does for device arrays): bt_plan_replay then re-runs the copies in, the
 * factorization, the solve (or refinement) and the copy of X out as one graph
 * launch, reading the same host arrays.  The host arrays must be page-locked
 * (BT_ERR_CUDA otherwise); synchronises the stream and replaces any earlier
 * graph of the plan. */
bt_status bt_plan_capture_host(bt_plan plan, const double* B, const double* D, const double* C, const double* F,
                               double* X, int nrhs, int sweeps);
bt_status bt_plan_replay(bt_plan plan);

/* Wait for the plan's stream; return the recorded numerical status. */
bt_status bt_sync(bt_plan plan);

/* Wait for the plan's stream and report where a numerical failure was seen:
 * recursion level, partition index (-1 for the top-level direct solve) and
 * block row of that level.  Any output pointer may be NULL. */
bt_status bt_info(bt_plan plan, int* level, int64_t* partition, int64_t* row);

/* Geometry of the recursion: number of levels with partitions (the last
 * level is solved by one partition), and for level l (l < levels) its block
 * rows and partition count.  Host call, no synchronisation. */
bt_status bt_plan_levels(bt_plan plan, int* levels, int64_t* rows, int64_t* parts, int capacity);

/* Device bytes held by the plan. */
bt_status bt_plan_bytes(bt_plan plan, int64_t* bytes);

/* Copy the top-level reduced matrix of Eq. (redmatr) out of the plan after
 * bt_factor (device-to-device, asynchronous): for the p-1 separators s,
 *   alpha[s] = T[s][s], beta[s] = T[s][s-1] (beta[0] = 0),
 *   gamma[s] = T[s][s+1] (gamma[p-2] = 0), each [p-1][m][m] in FP64.
 * For a BABD plan: alpha[i], beta[i] for the p+1 reduced rows of Eq.
 * (redmatr1) (lower block bidiagonal; beta[0] = the corner block),
 * gamma is not written.  For a plan with local cyclic reduction
 * (bt_tuning.local = L) of BT_FP64 precision: the system left on the K
 * separators (block rows 0, 2^L, 2*2^L, ... < nblk), K = nblk halved L times
 * rounding up, in the same form (alpha, beta, gamma each [K][m][m]).  Not
 * available for plans whose block order is embedded in a larger one
 * (BT_ERR_INVALID). */
bt_status bt_reduced_export(bt_plan plan, double* alpha, double* beta, double* gamma);

/* Tracing.  bt_plan_trace(plan, 1) clears the records and brackets every
 * later kernel launch of the plan with a pair of CUDA events on the plan's
 * stream; bt_plan_trace(plan, 0) stops recording.  bt_plan_trace_query
 * synchronises and returns, for kernel kind `kind` at recursion level
 * `level` (levels >= 63 are pooled into 63; level -1 sums all levels), the
 * summed event time in ms and the number of launches.  Kinds:
 * 0 local factor, 1 reduced-matrix assembly, 2 forward solve, 3 reduced
 * right-hand side, 4 back substitution, 5 top-level BABD direct solve,
 * 6 FP64 residual, 7 refinement update, 8 cyclic-reduction factor steps,
 * 9 cyclic-reduction solve steps, 10 ||A||_inf for the backward error. */
bt_status bt_plan_trace(bt_plan plan, int enable);
bt_status bt_plan_trace_query(bt_plan plan, int kind, int level, double* total_ms, int64_t* launches);

/* Number of kernels the plan has launched since it was created. */
bt_status bt_plan_launches(bt_plan plan, int64_t* count);

void bt_plan_destroy(bt_plan plan);

/* One-shot FP64 factor + solve of a block tridiagonal system that allocates
 * no device memory.  The paper has no counterpart: this entry point serves
 * callers that may not call cudaMalloc -- code inside a host application
 * that owns all device memory through its own pool or budget, or a
 * latency-critical loop that cannot accept cudaMalloc's implicit device
 * synchronisation or its possible failure.
 *   Arguments as for bt_plan_create (prec FP64, p chosen automatically),
 *   bt_factor and bt_solve: B, D, C [nblk][m][m], F, X [nblk*m][nrhs],
 *   device pointers owned by the caller; X may not alias F.
 * Every intermediate lives in one static device array of
 * BT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  If the problem needs more, the call returns
 * BT_ERR_INVALID before touching the GPU and *required_bytes (may be NULL)
 * tells how much it would need; e.g. m = 16 fits about a thousand block rows.
 * The first call on a device looks up the array's device address (with
 * cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls whose GPU work overlaps race, so callers
 * must serialise them.  Every call ends by copying the device status word to
 * host memory and synchronising `stream`, then returns the numerical status
 * (BT_ERR_SINGULAR / BT_ERR_NONFINITE). */
#define BT_NOALLOC_SCRATCH_BYTES (8u << 20)
bt_status bt_solve_noalloc(int64_t nblk, int m, const double* B, const double* D, const double* C,
                           const double* F, double* X, int nrhs, void* stream, int64_t* required_bytes);

/* ---------------------------------------------------------------------
 * Batches of independent block tridiagonal systems (the partition method
 * applied to many systems at once; every system follows Sec. 2 exactly as a
 * single plan does).  The work of all systems at the same recursion level,
 * block order and precision runs in one persistent launch over a work list of
 * (system, partition) items, and the whole run -- factor, solve, and
 * `ir_sweeps` FP64 refinement sweeps for the BT_FP32_IR/BT_BF16_IR systems --
 * is captured into one CUDA graph at creation.
 * ------------------------------------------------------------------- */
typedef struct {
    int64_t nblk;      /* block rows N */
    int m;             /* block order: 1, 2, 4, 8, 16 or 32 */
    int prec;          /* bt_prec */
    int nrhs;          /* right-hand sides, 1..32 */
    const double* B;   /* [N][m][m] device arrays, caller-owned, read-only */
    const double* D;
    const double* C;
    const double* F;   /* [N*m][nrhs] right-hand sides */
    double* X;         /* [N*m][nrhs] solutions (written by every run) */
    bt_tuning tuning;  /* partitioning (p0, ctas_per_sm, sub_rows, top_rows; `reduced` and `tp_block`
                          are not used by batches); all zero: about 32 (m >= 8) or 64 block rows
                          per top-level partition */
} bt_batch_desc;
typedef struct bt_batch_s* bt_batch;

/* Plan and capture a batch.  The arrays named by the descriptors are bound
 * into the graph: later runs re-read them (new values in the same arrays are
 * fine) and must keep them alive.  mem_cap_bytes > 0 bounds the workspace:
 * systems are split into waves that reuse it in turn (BT_ERR_NOMEM if one
 * system alone exceeds the cap).  The stream may be NULL. */
bt_status bt_batch_create(bt_batch* batch, const bt_batch_desc* systems, int count, int ir_sweeps,
                          int64_t mem_cap_bytes, void* stream);
/* One graph launch: factor and solve every system (asynchronous). */
bt_status bt_batch_run(bt_batch batch);
/* Synchronise; per-system status (may be NULL): numerical failures, and
 * BT_ERR_NOT_CONVERGED for a refined system whose last correction was larger
 * than tol relative to its solution; relcorr (may be NULL) receives that
 * ratio (0 for FP64 systems).  Returns the first failing status or BT_OK. */
bt_status bt_batch_finish(bt_batch batch, double tol, int* status, double* relcorr);
bt_status bt_batch_info(bt_batch batch, int* waves, int64_t* graph_nodes, int64_t* bytes);
void bt_batch_destroy(bt_batch batch);

/* ---------------------------------------------------------------------
 * ABD/BABD systems (Sec. 2, Eq. (parpart1) with c = 0, and Sec. 3: one-step
 * discretisations of linear BVPs).  Unknowns y_0..y_N (m each):
 *     B0 y_0 + B1 y_N = beta                       (boundary block row 0)
 *     S_j y_j + R_j y_{j+1} = r_j,  j = 0..N-1    (block rows 1..N)
 * S, R: [N][m][m]; B0, B1: [m][m].  Right-hand side and solution are
 * [(N+1)*m][nrhs] with the boundary row first.  The local factorizations
 * pivot inside each m x m block; the reduced system keeps the boundary row
 * as a separator (B0 may be singular, e.g. separated boundary conditions)
 * and the final small reduced system is solved with partial pivoting across
 * block rows.
 * ------------------------------------------------------------------- */

bt_status abd_plan_create(abd_plan* plan, int64_t N, int m, int nrhs_max, int prec, int64_t p,
                          void* stream);

/* abd_plan_create with explicit parameters (bt_tuning; NULL = defaults):
 * p0, sub_rows, top_rows and serial as for bt_plan_create_tuned; local and
 * pivot must be 0.  reduced = 1: cyclic reduction of the whole BABD system
 * instead of partitions (the method Sec. 2 recommends for ABD/BABD matrices):
 * rows 2k and 2k+1 of every level eliminate y_{2k+1} (one inverse of R_{2k} by
 * Gauss-Jordan with partial pivoting and two block products per pair, one
 * launch per level and phase), down to one row, which with the boundary row
 * is a 2m x 2m system solved by elimination with partial pivoting; about
 * log2 N levels.  Blocks of order 8, 16 or 32 and BT_FP64 only
 * (BT_ERR_INVALID otherwise). */
bt_status abd_plan_create_tuned(abd_plan* plan, int64_t N, int m, int nrhs_max, int prec, const bt_tuning* tuning,
                                void* stream);
/* Reads S, R, B0, B1 (kept by reference like bt_factor; B0 and B1 are also
 * copied into the plan). */
bt_status abd_factor(abd_plan plan, const double* S, const double* R, const double* B0,
                     const double* B1);
bt_status abd_solve(abd_plan plan, const double* RHS, double* Y, int nrhs);
bt_status abd_residual(abd_plan plan, const double* RHS, const double* Y, double* Rout, int nrhs);
/* The BABD residual as the plan's refinement forms it (bt_refine_residual:
 * FP64 for BT_FP64 plans, double-float for refined ones). */
bt_status abd_refine_residual(abd_plan plan, const double* RHS, const double* Y, double* Rout, int nrhs);
bt_status abd_refine(abd_plan plan, const double* RHS, double* Y, int nrhs, double tol, int maxit,
                     int* iters_out, double* relcorr_out);
bt_status abd_sync(abd_plan plan);
void abd_plan_destroy(abd_plan plan);

/* ---------------------------------------------------------------------
 * Circulant-like block systems (Sec. 2, Eq. (parpart1) and the remark after
 * Eq. (redmatr1)): N >= 2 unknowns y_0..y_{N-1} (m each) with
 *     S_j y_j + R_j y_{(j+1) mod N} = r_j,   j = 0..N-1,
 * a block bidiagonal matrix closed into a cycle by its corner block (periodic
 * one-step discretisations, circulant matrices with two block diagonals).
 * Moving the last block row to the top gives the BABD form above with N-1
 * steps, B0 = R_{N-1}, B1 = S_{N-1}; these calls are an abd plan on that
 * permutation (the right-hand side is rotated by one block row into plan
 * memory; the solution needs no permutation).  S, R: [N][m][m]; right-hand
 * sides and solutions [N*m][nrhs].  Errors and refinement as for abd_*;
 * cyc_residual returns the residual in the original row order. */
bt_status cyc_plan_create(abd_plan* plan, int64_t N, int m, int nrhs_max, int prec, int64_t p, void* stream);
bt_status cyc_factor(abd_plan plan, const double* S, const double* R);
bt_status cyc_solve(abd_plan plan, const double* RHS, double* Y, int nrhs);
bt_status cyc_residual(abd_plan plan, const double* RHS, const double* Y, double* Rout, int nrhs);
bt_status cyc_refine(abd_plan plan, const double* RHS, double* Y, int nrhs, double tol, int maxit,
                     int* iters_out, double* relcorr_out);

#ifdef __cplusplus
}
#endif

#endif /* BT_H */
