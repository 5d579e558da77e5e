/*
 * slqr.h -- C ABI of libslqr: in-place Householder QR in Lawson-Hanson H12
 * storage, Q^T.B application and back-substitution on one NVIDIA GB300
 * (sm_103a), for the least-squares subproblems of SLSQP.
 *
 * The operations follow the paper "Efficient Task Graph Scheduling for
 * Parallel QR Factorization in SLSQP" (Chatterjee et al.):
 *   - Alg. 2 (Section 3): in-place transform of A to upper-triangular form by
 *     the kernels update_pivot_row / update_trailing_non_pivot_row;
 *   - Task 1 / Task 2 (Alg. 3, Alg. 4): the pivot scalar `up` of each
 *     reflector is kept in a global array for later reuse, and a pivot whose
 *     reflector is undefined (zero column) is skipped;
 *   - Section 1 and the abstract: the stored reflectors are reused to apply
 *     Q^T and by the back-substitution at each SLSQP iteration.
 *
 * Storage form (H12).  A is m x n, column-major, leading dimension lda >= m,
 * FP64, with m >= n.  After slqr_factor:
 *   A[k, j] (k <= j)  = R[k, j]            (R upper triangular, R[k,k] = cl_k)
 *   A[i, k] (i >  k)  = tail of reflector k (left exactly as it was when the
 *                       reflector was built)
 *   up[k]             = pivot entry of reflector k, for k < min(m-1, n);
 *                       up[k] = 0 for a skipped pivot and for k >= min(m-1, n).
 * Reflector k is v_k = (0,..,0, up[k], A[k+1:m, k]) and
 * H_k = I + v_k v_k^T / b_k with b_k = up[k] * R[k,k] (< 0 when defined), which
 * is the Householder matrix I - 2 v v^T / (v^T v) of Alg. 1.  Q = H_0 H_1 ...
 * The sign rule is cl_k = -s when x0 > 0 and +s otherwise (s = ||x||, x the
 * column below and on the diagonal, x0 its first entry).
 *
 * Conventions for every entry point:
 *   - Pointers to matrices and vectors are DEVICE pointers owned by the
 *     caller, unless stated otherwise.  The library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; argument errors are
 *     returned synchronously and enqueue nothing.
 *   - Device-side conditions (a zero diagonal of R in slqr_solve_r, a bounded
 *     device wait that gave up) are written to a status word of the context
 *     and returned by slqr_sync().
 *   - A context serialises its calls: calls made with one context must be
 *     issued on one stream, or ordered by the caller, because they share the
 *     context's workspace.  Use one context per concurrent stream.
 *   - No C++ exception crosses this interface.
 */
#ifndef SLQR_H
#define SLQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int slqr_status;

#define SLQR_OK          0
#define SLQR_PENDING     1   /* request not finished yet (slqr_poll) */
#define SLQR_EINVAL    (-1)  /* bad argument: nothing was enqueued */
#define SLQR_ENOMEM    (-2)  /* device allocation failed */
#define SLQR_ECUDA     (-3)  /* a CUDA runtime call failed */
#define SLQR_ETIMEOUT  (-4)  /* a bounded device-side wait gave up */
#define SLQR_ERANK     (-5)  /* R has an exact zero on its diagonal */
#define SLQR_EBUSY     (-6)  /* over the HBM budget of the context */
#define SLQR_ENOTFOUND (-7)  /* unknown ticket or handle */
#define SLQR_ENOCONV   (-8)  /* iterative refinement did not reach its tolerance */
#define SLQR_ECHECK    (-9)  /* checked build (SLQR_CHECKED): a device bounds or
                                invariant check failed (the access was skipped), or
                                a workspace guard zone was overwritten */
#define SLQR_FALLBACK    2   /* slqr_lstsq_mixed_ex: the mixed-precision refinement
                                failed and x comes from the opt-in FP64 solve */

typedef struct slqr_ctx slqr_ctx;

/*
 * Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the device
 * memory the context may hold for its own workspace and, in serving, for
 * resident factorizations (0 = no cap).  On success *ctx is set and SLQR_OK
 * returned; the caller releases it with slqr_destroy.
 */
slqr_status slqr_create(slqr_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Free the context and its workspace.  Waits for work the context enqueued. */
void slqr_destroy(slqr_ctx *ctx);

/* Text of the last error recorded in `ctx` (never NULL; "" if none).  The
 * string is owned by the context and valid until its next call. */
const char *slqr_last_error(slqr_ctx *ctx);

/*
 * Wait for `stream`, then return and clear the context's device status word:
 * SLQR_OK, SLQR_ERANK (a zero diagonal met by slqr_solve_r since the last
 * sync) or SLQR_ETIMEOUT (a bounded device wait gave up).  Also returns
 * SLQR_ECUDA if the stream reports a CUDA error.
 */
slqr_status slqr_sync(slqr_ctx *ctx, void *stream);

/*
 * Diagnostic of the failure path every device-side wait of the library takes
 * (the panel's grid barrier, the tensor-core kernels' mbarrier waits): one
 * thread polls a device word that nothing sets, gives up after `polls` polls
 * (1 .. 2^20; about 0.3 us each), records SLQR_ETIMEOUT in the status word and
 * returns.  Synchronous; returns the status word it read (SLQR_ETIMEOUT when
 * the path works) and clears it, so the context stays usable.
 * Errors: SLQR_EINVAL (polls out of range), SLQR_ECUDA.
 */
slqr_status slqr_check_bounded_wait(slqr_ctx *ctx, unsigned polls, void *stream);

/*
 * Set how many polls a bounded device wait of this context makes before it
 * gives up (1 .. 2^24; 0 restores the default 2^24, about 1.5 s): the panel
 * factorization's polled exchange of per-column records and grid barrier,
 * and the grid barriers of the mixed-precision Q application and triangular
 * solves.  A wait that gives up records SLQR_ETIMEOUT in the status word
 * (slqr_sync; slqr_lstsq_mixed and slqr_lstsq_mixed_ex return it) and its
 * kernel returns, leaving that call's outputs unspecified; the context stays
 * usable.  The tensor-core kernels' mbarrier waits keep the fixed default.
 * A failure-detection aid (no counterpart in the paper): with a limit of a
 * few polls the waits run out on purpose.  Not while calls are in flight.
 * Errors: SLQR_EINVAL (polls above 2^24, NULL context).
 */
slqr_status slqr_set_spin_limit(slqr_ctx *ctx, unsigned polls);

/*
 * Panel width the factorization uses for an m x n problem (columns per
 * compact-WY block).  It depends only on (m, n).
 */
int slqr_panel_width(int m, int n);

/*
 * Size in bytes of the optional compact-WY store of an m x n factorization:
 * for each panel of slqr_panel_width(m, n) reflectors it keeps the strict
 * upper triangle of the Gram matrix V^T V, the scalars tau_k = -1/b_k (0 for a
 * skipped pivot) and the top square of V.  These are intermediate results of
 * the factorization that slqr_apply_qt can reuse instead of recomputing.
 */
size_t slqr_wy_size(int m, int n);

/*
 * In-place H12 QR of A (Alg. 2; Task 1 skip rule).  On return A holds R and
 * the reflector tails and up[0:n] the pivot entries (storage form above).
 *   m, n   sizes, m >= n >= 0, m >= 1 when n >= 1; m <= slqr_max_rows()
 *   A      device, m x n column-major, lda >= max(1, m); overwritten
 *   up     device, n doubles; written
 *   wy     device, slqr_wy_size(m, n) bytes, or NULL; when given, it receives
 *          the compact-WY store of this factorization (for slqr_apply_qt)
 * Errors: SLQR_EINVAL (sizes, lda, NULL pointers), SLQR_ENOMEM (workspace),
 * SLQR_ECUDA.  Device waits that give up are reported by slqr_sync.
 */
slqr_status slqr_factor(slqr_ctx *ctx, int m, int n, double *A, int lda, double *up,
                        double *wy, void *stream);

/*
 * Process-wide tuning knobs of the blocked factorization (no counterpart in the
 * paper; its alpha/beta task sizes play this role on the CPU):
 *   panel_width     32 or 64 forces the panel width (0: 32 for n <= 256, else 64)
 *   panel_rows_min  smallest slice of rows one panel CTA holds (0: by panel
 *                   height, 64 below 1536 rows, 128 below 6144, else 192);
 *                   larger values put fewer CTAs on each panel
 * Changing the panel width changes slqr_panel_width and slqr_wy_size: set it
 * before allocating compact-WY stores, and not while calls are in flight.
 * These overrides take precedence over the per-shape settings of
 * slqr_autotune; slqr_set_tuning(0, 0) also forgets those.
 */
void slqr_set_tuning(int panel_width, int panel_rows_min);

/*
 * Process-wide choice of the panel kernel (no counterpart in the paper):
 *   ctas  0   chosen per panel: a thread-block cluster holds the panel when it
 *             fits (FP32 panels of up to 16 x ~800 rows at width 64; FP64
 *             panels of at most 1024 rows), else the cooperative panel
 *        -1   always the cooperative panel (one grid-wide exchange of partial
 *             sums through L2 per column); this also switches the Q
 *             applications of the mixed-precision refinement to their
 *             cooperative kernel
 *         1..16  a cluster of that many CTAs wherever the panel's rows fit
 *             their shared memory, else the cooperative panel
 * The cluster panel splits the panel's rows over the CTAs of one cluster,
 * each slice in shared memory, and exchanges each column's partial sums
 * through distributed shared memory with one cluster barrier per column.
 * Both compute the same reflectors up to rounding order.  Set it while no
 * call is in flight.  Errors: SLQR_EINVAL (ctas out of range).
 */
slqr_status slqr_set_panel_cluster(int ctas);
int slqr_get_panel_cluster(void);

/*
 * Kernel of the cluster panel (a tuning and testing knob; same results up to
 * rounding order):
 *   0  chosen per panel: FP32 panels of width 64 with at most 512 rows per
 *      CTA keep the panel in registers (16 warps, 4 columns each, R / 32
 *      rows per lane), others hold it in shared memory with 16 warps
 *   1  shared memory, 16 warps     2  shared memory, 8 warps
 *   3  registers where that applies, else as 1
 * Set it while no call is in flight.  Errors: SLQR_EINVAL (out of range).
 */
slqr_status slqr_set_panel_cluster_variant(int variant);

/*
 * Look-ahead update of the FP32 factorization (the mixed-precision path):
 * after each panel of width 64, the next panel's columns X (rows k0 .. m-1)
 * become X - V T^T V^T X (the compact-WY form of the panel's reflectors,
 * Alg. 2 applied by blocks) before the next panel is factored.
 *   1  (default) one cooperative kernel: slices of V and X staged in shared
 *      memory, V^T X reduced in a fixed order, T^T W, X -= V W' (two bounded
 *      grid barriers; SLQR_ETIMEOUT if one gives up); it applies to dense
 *      matrices with at most 256 * (number of SMs) rows
 *   0  three tiled launches (V^T X partials, T^T W, X -= V W')
 * Same results up to rounding order.  A process-wide tuning and testing
 * knob: set it while no call is in flight.  Errors: SLQR_EINVAL (not 0 or 1).
 */
slqr_status slqr_set_fused_lookahead(int enable);
int slqr_get_fused_lookahead(void);

/*
 * Autotuner of those knobs for one problem shape: times slqr_factor of a
 * generic m x n scratch matrix (allocated and freed here) under panel width
 * 32 and 64 and rows-per-CTA minimum 0 (by panel height), 64, 96, 128, 192 and
 * 256, and keeps the fastest in a process-wide table keyed by (m, n): later
 * factorizations of exactly that shape (slqr_factor, slqr_factor_stacked,
 * slqr_factor_noalloc, the FP32 factorization of slqr_lstsq_mixed) use it,
 * other shapes keep the defaults.  Run it before allocating compact-WY stores
 * for that shape (the panel width sets slqr_wy_size) and not while other calls
 * are in flight.  Synchronous; takes about 24 factorizations of that shape.
 *   best_ms, best_panel_width, best_rows_min  HOST outputs, each may be NULL
 * Errors: SLQR_EINVAL (sizes), SLQR_ENOMEM (scratch), SLQR_ECUDA; on error
 * the previous tuning is kept.
 */
slqr_status slqr_autotune(slqr_ctx *ctx, int m, int n, double *best_ms, int *best_panel_width,
                          int *best_rows_min);

/*
 * The checked build (compiled with -DSLQR_CHECKED into libslqr_checked.so,
 * a stand-in for a memory checker): every workspace is filled with NaN bytes
 * (0xFF) each time an entry point takes it and is followed by a guard zone
 * whose pattern slqr_sync verifies; the cluster kernels check their launch
 * invariants and the indices they compute at run time, and a failed check
 * records SLQR_ECHECK in the status word and skips the access (nothing
 * traps).  slqr_is_checked returns 1 in that build, 0 otherwise.
 * slqr_check_selftest runs a kernel whose index check must fail on purpose
 * (the out-of-range access is skipped) and returns the status word it read:
 * SLQR_ECHECK in the checked build; SLQR_EINVAL in a normal build.
 */
int slqr_is_checked(void);
slqr_status slqr_check_selftest(slqr_ctx *ctx);

/* Largest m that slqr_factor accepts (the panel is held in shared memory). */
int slqr_max_rows(void);

/*
 * B <- Q^T B for the factorization (A, up) made by slqr_factor: the
 * reflectors H_0, H_1, ... are applied in the order they were built (the
 * reuse of the stored reflectors named in Section 1).  Reflectors with
 * b_k = up[k] * R[k,k] >= 0 are skipped.
 *   A, up  device, as left by slqr_factor (read only)
 *   nrhs   number of right-hand sides, >= 0
 *   B      device, m x nrhs column-major, ldb >= max(1, m); overwritten
 *   wy     device compact-WY store written by slqr_factor for this same
 *          (A, up), or NULL to recompute it from (A, up) (costs about
 *          panel_width/4 times the flops of one right-hand side)
 * Errors: SLQR_EINVAL, SLQR_ENOMEM, SLQR_ECUDA.
 */
slqr_status slqr_apply_qt(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                          const double *up, const double *wy, int nrhs, double *B, int ldb,
                          void *stream);

/*
 * Back-substitution R X = B[0:n, :] with R = triu(A[0:n, 0:n]); X overwrites
 * B[0:n, :] (the back-substitution that reuses the factorization, Section 1).
 * An exact zero R[i,i] sets x_i = 0 and records SLQR_ERANK in the device
 * status word (read it with slqr_sync).
 *   n      order of R, >= 0
 *   A      device, lda >= max(1, n); only its upper triangle is read
 *   nrhs   >= 0;  B device, ldb >= max(1, n)
 * Errors: SLQR_EINVAL, SLQR_ENOMEM, SLQR_ECUDA.
 */
slqr_status slqr_solve_r(slqr_ctx *ctx, int n, const double *A, int lda, int nrhs,
                         double *B, int ldb, void *stream);

/*
 * Structure-aware factorization of a stacked SLSQP least-squares matrix
 * A = [L^T; C]: an n x n upper-triangular block on top of an m_eq x n block C
 * (m = n + m_eq rows).  In Alg. 2 the reflector of column k is then zero in
 * rows k+1 .. n-1, and no reflector changes those rows of any column, so each
 * panel works on its own diagonal rows and the rows of C only: about
 * 2 m_eq n^2 flops instead of 2 m n^2 - 2 n^3 / 3.  The result is the H12
 * factorization slqr_factor computes for the same A (in exact arithmetic the
 * same reflectors; rounding differs only by the order of the sums), so
 * slqr_apply_qt, slqr_apply_qt_stacked and slqr_solve_r apply to it.
 *   n, m_eq  n >= 0, m_eq >= 0, n + m_eq <= slqr_max_rows()
 *   A      device, (n + m_eq) x n column-major, lda >= n + m_eq; the strictly
 *          lower part of the top n x n block must be zero: it is neither read
 *          nor written (it is the zero part of the reflector tails)
 *   up, wy as for slqr_factor with m = n + m_eq
 * Errors: SLQR_EINVAL, SLQR_ENOMEM, SLQR_ECUDA.
 */
slqr_status slqr_factor_stacked(slqr_ctx *ctx, int n, int m_eq, double *A, int lda,
                                double *up, double *wy, void *stream);

/*
 * B <- Q^T B for a factorization made by slqr_factor_stacked, skipping the
 * rows where the reflectors are zero (4 (m_eq + 1) n flops per right-hand side
 * instead of 4 m n - 2 n^2).  Arguments as for slqr_apply_qt with
 * m = n + m_eq; B is (n + m_eq) x nrhs, ldb >= n + m_eq.
 */
slqr_status slqr_apply_qt_stacked(slqr_ctx *ctx, int n, int m_eq, const double *A, int lda,
                                  const double *up, const double *wy, int nrhs, double *B,
                                  int ldb, void *stream);

/*
 * slqr_batch_factor -- `count` independent least-squares problems in one
 * persistent launch.  Each problem is the factorization of slqr_factor
 * (Alg. 2, Task 1 skip rule) and, when its b is given, Q^T b and the
 * back-substitution fused after it (the reuse of the stored reflectors named
 * in Section 1).  Persistent CTAs take problems from a device-side queue
 * ordered costliest first; one CTA owns one problem at a time.
 *   count        number of problems, >= 0
 *   m, n, lda    HOST arrays of count ints: 0 <= n <= m <= slqr_batch_max_rows(),
 *                lda >= max(1, m)
 *   A            HOST array of count DEVICE pointers (column-major m x n)
 *   up           HOST array of count DEVICE pointers (n doubles each)
 *   b            HOST array of count DEVICE pointers (m doubles each) or NULL
 *                (whole array) / a NULL entry: no solve for that problem
 *   prec         SLQR_FP64 or SLQR_FP32
 *   status       DEVICE array of count ints or NULL: per problem SLQR_OK,
 *                SLQR_ERANK (a zero diagonal of R) or, for SLQR_FP32,
 *                SLQR_ENOCONV (refinement stopped above its tolerance)
 *   err          DEVICE array of count doubles or NULL: for SLQR_FP32 the
 *                last refinement step ||dx||_inf / ||x||_inf of each problem
 *                (an estimate of its remaining relative error); not written
 *                for SLQR_FP64
 * Outputs, SLQR_FP64: A[i] and up[i] hold the H12 factorization (storage
 * form above); b[i][0:n] = x_i, b[i][n:m] = the residual part of Q^T b.
 * Outputs, SLQR_FP32 (b required, up may be NULL): A[i] is left unchanged;
 * the H12 factorization is computed in FP32 (reflector norm, up and b in
 * FP64) on a scratch copy, and the LS solution is refined against the FP64
 * A[i] by the augmented-system iteration [I A; A^T 0][r; x] = [b; 0] with
 * FP64 residuals (up to 12 sweeps; SLQR_OK at ||dx|| <= 1e-14 ||x||, or
 * when the steps stop contracting below 1e-10 ||x||, the FP64 noise level of
 * an ill-conditioned problem);
 * b[i][0:n] = x_i, b[i][n:m] is unspecified.
 * The host arrays are read before the call returns.  The problems must not
 * overlap in memory.  Errors: SLQR_EINVAL, SLQR_ENOMEM, SLQR_ECUDA.
 */
#define SLQR_FP64 0   /* FP64 throughout (DFMA)                                   */
#define SLQR_FP32 1   /* FP32 factorization + FP64-residual refinement            */
#define SLQR_TF32 2   /* as SLQR_FP32, the two products of the rank-NB trailing
                         update (W = V^T X and X -= V W') on the tensor cores
                         (tcgen05, TF32 operands, FP32 accumulation)
                         (slqr_lstsq_mixed only)                                  */
#define SLQR_BF16X3 3 /* as SLQR_TF32 with BF16 operands split in two,
                         x = hi + lo (about 16 significant bits), three MMAs per
                         product (hi hi + hi lo + lo hi), FP32 accumulation
                         (slqr_lstsq_mixed only)                                  */
slqr_status slqr_batch_factor(slqr_ctx *ctx, int count, const int *m, const int *n,
                              double *const *A, const int *lda, double *const *up,
                              double *const *b, int prec, int *status, double *err,
                              void *stream);
int slqr_batch_max_rows(void);

/*
 * Settings of the batched kernels and their autotuner (the batch form of the
 * paper's alpha/beta task sizes, Section 4.1).  A batched problem is factored
 * by one CTA in panels of `panel_width` reflectors (8, 16 or 32), its trailing
 * columns updated in tiles of `tile_cols` columns (16, 32 or 64); the valid
 * pairs are those with panel_width * tile_cols >= 256: (8, 32), (8, 64),
 * (16, 16), (16, 32), (16, 64), (32, 16), (32, 32), (32, 64).  The setting is
 * chosen per precision (SLQR_FP64, SLQR_FP32) and per size class of the
 * problem's row count m: class 0 m <= 64, 1 m <= 128, 2 m <= 256, 3 m <= 512
 * (slqr_batch_class_rows gives the upper bounds); (16, 32) by default.  For
 * SLQR_FP64 the classes 0 and 1 may instead take the shared-memory-resident
 * kernel (`resident` = 1, with the pair (16, 32)): the whole problem and its b
 * are copied into shared memory, factored and back-substituted there, and
 * written back once.  The
 * problems of classes that share a setting run in one persistent launch; a
 * batch whose classes use different settings makes one launch per setting,
 * one after the other on the caller's stream.  Settings are process-wide:
 * change them only while no batch or plan creation is in flight (a plan keeps
 * the settings it was created with).
 *
 * slqr_batch_set_tuning  sets the pair of one class (m_class -1: every class);
 *                        (0, 0) restores the default; resident 1 selects the
 *                        resident kernel (SLQR_FP64, class 0 or 1, pair
 *                        (16, 32) or (0, 0)).  SLQR_EINVAL for an invalid
 *                        precision, class, pair or resident request.
 * slqr_batch_get_tuning  reads it (HOST outputs, each may be NULL).
 * slqr_batch_autotune    tunes the settings of `prec` for a mixture of
 *                        shapes: count, m, n (HOST arrays) give the shapes of
 *                        the caller's batch (count 0 or m NULL: the default
 *                        law m ~ U{16..512}, n ~ U{ceil(m/4)..m}); a scratch
 *                        batch of `sample` problems (<= 0: min(count, 3000);
 *                        every (count/sample)-th shape; generic entries; fused
 *                        solve) is timed (best of two runs after a warm-up)
 *                        under each candidate.  Greedy coordinate search: the
 *                        classes costliest first, each trying every valid
 *                        pair (and, for SLQR_FP64 classes 0 and 1, the
 *                        resident kernel) with the other classes held, a
 *                        change kept only
 *                        when the whole scratch batch runs at least 1% faster
 *                        (a split into several launches must pay for itself).
 *                        Synchronous; allocates and frees its scratch.  HOST
 *                        outputs, each may be NULL: panel widths, tile widths
 *                        and resident flags per class (slqr_batch_classes()
 *                        entries), and
 *                        ms[2] = the scratch batch's time before and after.
 *                        Errors: SLQR_EINVAL, SLQR_ENOMEM, SLQR_ECUDA; on
 *                        error the previous settings are kept.
 */
int slqr_batch_classes(void);
int slqr_batch_class_rows(int m_class);
slqr_status slqr_batch_set_tuning(int prec, int m_class, int panel_width, int tile_cols,
                                  int resident);
slqr_status slqr_batch_get_tuning(int prec, int m_class, int *panel_width, int *tile_cols,
                                  int *resident);
slqr_status slqr_batch_autotune(slqr_ctx *ctx, int prec, int count, const int *m, const int *n,
                                int sample, int *panel_width, int *tile_cols, int *resident,
                                double *ms);

/*
 * slqr_batch_factor for stacked SLSQP matrices A_i = [L_i^T; C_i]: problem i
 * is (n[i] + m_eq[i]) x n[i] with an upper-triangular top n[i] x n[i] block,
 * factored with the structure of slqr_factor_stacked.  The strictly lower part
 * of the top block must be zero; SLQR_FP64 neither reads nor writes it
 * (SLQR_FP32 reads all of A for its FP64 residuals).  Other arguments and
 * outputs as for slqr_batch_factor with m[i] = n[i] + m_eq[i] <=
 * slqr_batch_max_rows().
 */
slqr_status slqr_batch_factor_stacked(slqr_ctx *ctx, int count, const int *n, const int *m_eq,
                                      double *const *A, const int *lda, double *const *up,
                                      double *const *b, int prec, int *status, double *err,
                                      void *stream);

/*
 * Batch plans: one batch launched many times (an SLSQP loop refactors
 * problems of unchanged shapes at every iteration, with new values).  The
 * arguments are those of slqr_batch_factor (ntop: NULL, or per problem the rows
 * of its upper-triangular top block as in slqr_batch_factor_stacked, 0 for a
 * dense problem); the problem table and the costliest-first order are copied
 * to the device once, and each launch replays a CUDA graph of the work-counter
 * reset and the persistent kernel.  The caller refills A[i] (and b[i]) in
 * place between launches; the pointers, sizes, status and err arrays must
 * stay valid for the plan's life.  The plan owns its device memory (the
 * FP32 plan holds a scratch of up to 1 MB per resident CTA) and counts
 * against the context's HBM budget (SLQR_EBUSY when over it).
 * slqr_batch_plan_launch is asynchronous on `stream`; one plan must not be
 * launched twice concurrently.
 */
typedef struct slqr_batch_plan slqr_batch_plan;
slqr_status slqr_batch_plan_create(slqr_ctx *ctx, int count, const int *m, const int *n,
                                   const int *ntop, double *const *A, const int *lda,
                                   double *const *up, double *const *b, int prec, int *status,
                                   double *err, slqr_batch_plan **plan);
slqr_status slqr_batch_plan_launch(slqr_batch_plan *plan, void *stream);
void slqr_batch_plan_destroy(slqr_batch_plan *plan);

/*
 * slqr_lstsq_mixed -- least squares min ||A x - b|| for one large problem in
 * mixed precision, error stated against FP64.  The H12 factorization
 * (Alg. 2) runs on an FP32 copy of A (FP32 arithmetic; up and the compact-WY
 * coefficients are stored in FP64).  The
 * FP64 solution is then recovered by iterative refinement of the augmented
 * system [I A; A^T 0][r; x] = [b; 0] with residuals computed in FP64 from A
 * and corrections through the FP32 factorization.
 *   A      device, m x n column-major FP64, lda >= m, m >= n >= 1 (read only)
 *   b      device, m doubles (read only);  x  device, n doubles (output)
 *   prec   SLQR_FP32 (trailing-update products on the FP32 FMA pipe),
 *          SLQR_TF32 (W = V^T X and X -= V W' on the tensor cores, TF32
 *          operands: refinement then converges for kappa well below 2^11) or
 *          SLQR_BF16X3 (the same products with hi + lo BF16 operands, about
 *          2^-15 per product: refinement converges for kappa well below 2^15)
 *   max_iter  refinement sweeps (<= 0: 30);  tol  stop at ||dx||_inf <=
 *          tol ||x||_inf (<= 0: 1e-14)
 *   iters, err  HOST ints/doubles or NULL: sweeps done and the last
 *          ||dx||_inf / ||x||_inf
 * Synchronous: returns when x is final.  SLQR_OK when the refinement reached
 * tol (or stopped contracting below 1e-10); SLQR_ENOCONV when it did not
 * (kappa(A) * u_fp32 too large); SLQR_ERANK for an exact zero diagonal of R;
 * SLQR_EINVAL, SLQR_ENOMEM, SLQR_ECUDA.
 */
slqr_status slqr_lstsq_mixed(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                             const double *b, double *x, int prec, int max_iter, double tol,
                             int *iters, double *err, void *stream);

/*
 * slqr_lstsq_mixed_ex -- slqr_lstsq_mixed with a choice of refinement method
 * and an opt-in FP64 fallback, so that every problem gets an answer and the
 * caller always learns how it was obtained.  The paper factors in one
 * precision only; the refinement is this library's way of reusing one
 * low-precision H12 factorization (Alg. 2) for an FP64-accurate LS solution.
 *
 * Refinement methods (opts->refine):
 *   SLQR_REFINE_AUTO    Bjorck sweeps as in slqr_lstsq_mixed; when they do
 *                       not converge, GMRES-IR from the plain solve
 *   SLQR_REFINE_BJORCK  Bjorck sweeps only (slqr_lstsq_mixed)
 *   SLQR_REFINE_GMRES   GMRES-IR only
 * GMRES-IR (Carson, Higham and Pranesh, three-precision GMRES-based iterative
 * refinement for least squares, SIAM J. Sci. Comput. 42(6), 2020): each
 * refinement step forms the residual [f; g] = [b - r - A x; -A^T r] of the
 * augmented system [I A; A^T 0][r; x] = [b; 0] in FP64 and solves for the
 * correction with GMRES (FP64 Krylov basis, at most gmres_restart vectors),
 * left-preconditioned by the augmented matrix of the low-precision QR (one
 * Bjorck correction, applied in FP64 arithmetic to the FP32 factors).  It
 * converges where kappa(A) times the factorization's backward error is above
 * 1 (where the Bjorck sweeps diverge), at the price of one preconditioner
 * application per Krylov iteration (about as much as one Bjorck sweep).  A
 * step is accepted when ||dx||_inf <= tol ||x||_inf, or when its inner solve
 * reached gmres_tol and the step is at the FP64 noise level of the problem,
 * max(1e-10, 100 kappa_est 2^-53), with kappa_est = max|R_ii| / min|R_ii|.
 *
 * Options (opts may be NULL: every field 0):
 *   refine           SLQR_REFINE_AUTO (0), _BJORCK or _GMRES
 *   max_sweeps       Bjorck sweeps (<= 0: 30)
 *   tol              stop at ||dx||_inf <= tol ||x||_inf (<= 0: 1e-14)
 *   gmres_max_iters  Krylov iterations over all GMRES-IR steps (<= 0: 300)
 *   gmres_restart    Krylov vectors per GMRES cycle, <= 512 (<= 0:
 *                    min(gmres_max_iters, 200)); the basis takes
 *                    (gmres_restart + 1) (m + n) doubles of device memory
 *   gmres_tol        relative residual of each inner GMRES solve (<= 0: 1e-10)
 *   fp64_fallback    1: when the refinement fails, solve in FP64 instead
 *                    (slqr_factor, slqr_apply_qt, slqr_solve_r on a copy of
 *                    A; m n + 2 m doubles more of device memory) and return
 *                    SLQR_FALLBACK; 0: return SLQR_ENOCONV
 *   structure        SLQR_DENSE (0), or SLQR_STACKED: A = [L^T; C] with an
 *                    upper-triangular top n x n block whose strictly lower
 *                    part is zero (it is read: the FP64 residuals use all of
 *                    A), factored with the structure of slqr_factor_stacked
 *                    (its trailing updates on the FP32 FMA pipe)
 * Report (info may be NULL), HOST struct:
 *   method       how x was obtained: SLQR_REFINE_BJORCK, SLQR_REFINE_GMRES or
 *                SLQR_REFINE_FP64 (the fallback)
 *   sweeps       Bjorck sweeps done
 *   gmres_steps  GMRES-IR refinement steps;  gmres_iters  Krylov iterations
 *   err          the last refinement step ||dx||_inf / ||x||_inf of the
 *                mixed-precision refinement (also after a fallback)
 *   kappa_est    max|R_ii| / min|R_ii| of the low-precision R (0 when
 *                GMRES-IR did not run)
 * Returns SLQR_OK (x from the mixed-precision refinement), SLQR_FALLBACK (x
 * from the FP64 solve), SLQR_ENOCONV (no fallback asked for), SLQR_ERANK, or
 * the errors of slqr_lstsq_mixed.  Synchronous.  Other arguments as for
 * slqr_lstsq_mixed.
 */
#define SLQR_REFINE_AUTO   0
#define SLQR_REFINE_BJORCK 1
#define SLQR_REFINE_GMRES  2
#define SLQR_REFINE_FP64   3   /* slqr_mixed_info.method only */

typedef struct {
  int refine;
  int max_sweeps;
  double tol;
  int gmres_max_iters;
  int gmres_restart;
  double gmres_tol;
  int fp64_fallback;
  int structure;
} slqr_mixed_opts;

typedef struct {
  int method;
  int sweeps;
  int gmres_steps;
  int gmres_iters;
  double err;
  double kappa_est;
} slqr_mixed_info;

slqr_status slqr_lstsq_mixed_ex(slqr_ctx *ctx, int m, int n, const double *A, int lda,
                                const double *b, double *x, int prec, const slqr_mixed_opts *opts,
                                slqr_mixed_info *info, void *stream);

/*
 * Request loop: continuous batching of least-squares subproblems from many
 * concurrent SLSQP runs (each one factors its QP matrix and later
 * back-substitutes with the stored factorization, Section 1).  The first
 * slqr_submit starts a worker thread in the context; slqr_destroy stops it
 * after the requests in flight finish.
 *
 * Kinds:
 *   SLQR_REQ_FACTOR        factor A (m x n, m >= n >= 1) and keep the
 *                          factorization on the device under a new handle
 *                          (returned in slqr_result.handle)
 *   SLQR_REQ_SOLVE         x = argmin ||A x - b|| with the resident
 *                          factorization of `handle` (Q^T b, back-substitution)
 *   SLQR_REQ_FACTOR_SOLVE  both, nothing kept
 *   SLQR_REQ_RELEASE       free the factorization of `handle`
 * Admission is in arrival order and by the context's HBM budget (bytes held
 * by resident factorizations and requests in flight); a request that cannot
 * fit waits until memory is freed, and one larger than the whole budget
 * fails with SLQR_EBUSY.  Admitted FP64 requests with m <= slqr_batch_max_rows()
 * share one persistent batched launch, and so do SLQR_FP32 FACTOR_SOLVE
 * requests of that size; larger FP64 ones run one per stream on a pool of
 * streams; every other mixed-precision request runs on a mixed lane (a helper
 * thread with its own stream: the low-precision factorization and the
 * automatic refinement of slqr_lstsq_mixed_ex with the FP64 fallback); all of
 * them overlap on the device.  Latency routing: while at most half of
 * those streams are busy, a batch-sized request with m * n >= 60000 also runs
 * on a stream (its factorization is spread over many SMs instead of one CTA
 * of the batched launch).  Requests that arrive while others run are
 * admitted as memory frees up.
 *
 * A, b and x are HOST pointers owned by the caller; they must stay valid
 * until slqr_poll reports the request done (A and b are copied in at
 * admission; x receives n doubles at completion).  prec: SLQR_FP64,
 * SLQR_FP32, SLQR_TF32 or SLQR_BF16X3.  A mixed-precision FACTOR_SOLVE of the
 * batch size class in SLQR_FP32 joins the batched FP32 launch (refinement as
 * in slqr_batch_factor); any other mixed-precision FACTOR_SOLVE is solved as
 * by slqr_lstsq_mixed_ex in its automatic mode with fp64_fallback = 1
 * (out->status SLQR_OK for a mixed-precision result, SLQR_FALLBACK when the
 * FP64 solve answered).  A mixed-precision FACTOR keeps the library's FP64 copy
 * of A and the low-precision factorization on the device under the handle
 * (both counted in the HBM budget: m n doubles plus about m n floats); a
 * SOLVE on it runs the refinement against that copy (SLQR_OK or
 * SLQR_FALLBACK).  Stacked mixed-precision requests use the structure-aware
 * low-precision factorization.
 * slqr_poll returns SLQR_PENDING until the request is done, then SLQR_OK with
 * *out filled (out->status is the request's own status) and forgets the
 * ticket; SLQR_ENOTFOUND for an unknown or already collected ticket.
 */
#define SLQR_REQ_FACTOR       1
#define SLQR_REQ_SOLVE        2
#define SLQR_REQ_FACTOR_SOLVE 3
#define SLQR_REQ_RELEASE      4

typedef struct {
  int kind;
  int m, n, lda;
  const double *A;      /* host, column-major m x n (FACTOR, FACTOR_SOLVE) */
  const double *b;      /* host, m doubles (SOLVE, FACTOR_SOLVE) */
  double *x;            /* host, n doubles, written at completion */
  uint64_t handle;      /* SOLVE, RELEASE */
  int prec;             /* SLQR_FP64, SLQR_FP32, SLQR_TF32 or SLQR_BF16X3 */
  int structure;        /* SLQR_DENSE, or SLQR_STACKED: A = [L^T; C] with an
                           upper-triangular top n x n block whose strictly lower
                           part is zero (factored as slqr_factor_stacked) */
} slqr_request;

#define SLQR_DENSE   0
#define SLQR_STACKED 1

typedef struct {
  int status;           /* SLQR_OK, SLQR_FALLBACK, SLQR_ERANK, SLQR_ENOCONV, SLQR_EBUSY,
                           SLQR_ENOTFOUND, ... */
  uint64_t handle;      /* FACTOR: the handle of the resident factorization */
  double residual_norm; /* solves: FP64 ||(Q^T b)[n:m]||; mixed precision ||b - A x||
                           from the caller's arrays (NaN for a SOLVE, which has no A) */
  double latency_ms;    /* from slqr_submit to completion */
  double err;           /* mixed precision: last refinement step ||dx|| / ||x|| */
} slqr_result;

slqr_status slqr_submit(slqr_ctx *ctx, const slqr_request *req, uint64_t *ticket);
slqr_status slqr_poll(slqr_ctx *ctx, uint64_t ticket, slqr_result *out);
/* Device bytes the request loop holds now (resident factorizations included). */
size_t slqr_server_bytes_in_use(slqr_ctx *ctx);

/*
 * slqr_factor_noalloc -- the factorization of slqr_factor for callers that
 * must not allocate device memory.  The paper has no counterpart: this entry
 * point exists for embedding.  Some callers cannot call cudaMalloc: a host
 * framework that has reserved all device memory for its own pool, or a
 * latency-bound loop in which cudaMalloc / cudaFree (which may synchronise the
 * whole device) are forbidden.  This call needs no context and allocates
 * nothing: the caller passes the inputs and outputs, and every other buffer
 * the factorization needs (barrier counter, reduction records, compact-WY
 * store when wy is NULL, partial sums) lives in one fixed array of about
 * 12.1 MB that the library declares in device memory.  Every GPU that loads
 * libslqr holds that array until the process exits.
 *   m, n     m >= n >= 0, m <= slqr_noalloc_max_rows() (8192),
 *            n <= slqr_noalloc_max_cols() (1024); larger sizes return
 *            SLQR_EINVAL and enqueue nothing
 *   A, lda, up, wy   as for slqr_factor (wy may be NULL)
 *   status   device int, or NULL: receives SLQR_ETIMEOUT if a bounded device
 *            wait gives up; the caller clears it before the call
 *   stream   cudaStream_t as void*; the work is enqueued on it
 * It runs on the device that is current for the calling thread.  The first
 * call on a device does a one-time set-up there (it looks up the device
 * address of the array and sets kernel attributes); make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * previous call's contents: each call clears the parts that must start at
 * zero.  Calls whose work overlaps on the GPU (other streams, other host
 * threads) race on the array and give wrong results: order them.
 * Errors: SLQR_EINVAL, SLQR_ECUDA.
 */
slqr_status slqr_factor_noalloc(int m, int n, double *A, int lda, double *up, double *wy,
                                int *status, void *stream);
int slqr_noalloc_max_rows(void);
int slqr_noalloc_max_cols(void);

/*
 * Optional CUDA-event profiler (tracing aid; no counterpart in the paper).
 * slqr_profile(ctx, 1) clears the totals and starts recording a pair of CUDA
 * events on the launching stream around every kernel the context launches;
 * slqr_profile(ctx, 0) stops.  slqr_profile_read waits for the recorded
 * events and returns, for one kernel family, the summed device time (ms), the
 * number of launches and the summed algorithmic flops of those launches
 * (Householder counts; for SLQR_KERNEL_TW and the rebuild, the blocking
 * overhead flops).  Families:
 */
#define SLQR_KERNEL_PANEL      0  /* cooperative panel factorization            */
#define SLQR_KERNEL_VTX        1  /* W = V^T X partials (trailing update, Q^T B) */
#define SLQR_KERNEL_TW         2  /* W' = T^T W                                  */
#define SLQR_KERNEL_UPD        3  /* X -= V W'                                   */
#define SLQR_KERNEL_WY_REBUILD 4  /* compact-WY rebuild inside slqr_apply_qt     */
#define SLQR_KERNEL_TRSM       5  /* back-substitution steps                     */
#define SLQR_KERNEL_BATCH      6  /* persistent batched factor (+ solve)         */
int slqr_profile(slqr_ctx *ctx, int enable);
slqr_status slqr_profile_read(slqr_ctx *ctx, int kernel, double *ms, long long *launches,
                              double *flops);

/*
 * Measured arithmetic peaks of the device (a diagnostic for rooflines; no
 * counterpart in the paper).  Synchronous: waits for the device, then times a
 * probe kernel with CUDA events (best of three launches after a warm-up) and
 * writes its rate in TFLOP/s to *tflops (HOST).
 *   SLQR_PEAK_FP64_FMA  register-resident FP64 FMA chains on every SM (the FP64
 *                       pipe that the FP64 factorization and update kernels use)
 *   SLQR_PEAK_TF32_TC   tcgen05 kind::tf32 MMAs (M = 128, N = 64, K = 8, the
 *                       shape of the TF32 trailing update) issued back to back by
 *                       one CTA per SM on shared-memory operands
 * Errors: SLQR_EINVAL (kind, NULL pointers), SLQR_ECUDA.  A probe's bounded
 * wait that gives up records SLQR_ETIMEOUT in the status word (slqr_sync).
 */
#define SLQR_PEAK_FP64_FMA 0
#define SLQR_PEAK_TF32_TC  1
slqr_status slqr_measure_peak(slqr_ctx *ctx, int kind, double *tflops);

/* Number of CUDA kernels this context has launched since it was created. */
long long slqr_launch_count(slqr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SLQR_H */
