/*
 * h12_oracle.c -- sequential CPU oracle for the in-place Householder QR kept in
 * Lawson-Hanson H12 storage, the Q^T.B application that reuses that storage, and
 * the back-substitution with R.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and the CPU-baseline legs of
 * bench.py do.  It shares no code, header, table or helper with the CUDA path.
 *
 * Precision: IEEE binary64 throughout, plain scalar loops, no BLAS, no blocking,
 * no reordering beyond what the algorithm states.
 *
 * What it follows (the paper: "Efficient Task Graph Scheduling for Parallel QR
 * Factorization in SLSQP"):
 *   - Alg. 2 (Section 3): for each pivot, update_pivot_row builds reflector i
 *     and returns (up, b); update_trailing_non_pivot_row then applies it to
 *     every later vector j > i, one vector at a time, in increasing j.
 *   - Task 1 (Alg. 3): when up or b is undefined the pivot is skipped; up is
 *     kept in global_up_array for later reuse.
 *   - Section 1 / abstract: the stored reflectors are reused to apply Q^T and
 *     for back-substitution.
 *   - Section 2.2 / Alg. 1: H_k = I - 2 u u^T / (u^T u), Q = H_1 H_2 ... .
 *
 * Readings taken where the paper is silent or garbled (each one is also listed
 * in the design notes of the repository):
 *   R1  A paper "row" is one contiguous storage vector; the matrix is m x n,
 *       column-major, and the factorization is the column QR of A.
 *   R2  min(m-1, n) reflectors; a length-1 vector gets none (up = 0 for it).
 *   R3  Sign rule: cl = -s when x0 > 0, cl = +s otherwise (x0 == 0 -> +s);
 *       R_kk = cl, up = x0 - cl.
 *   R4  The reflector vector v = (up, A[k+1:m, k]) is not normalised; the tail
 *       stays in place below the diagonal and up is stored apart.
 *   R5  The column norm is scaled by c = max|x_i| (s = c * sqrt(sum (x_i/c)^2)).
 *   R6  b is not stored; it is recomputed as b = up * R_kk.
 *   R8  Back-substitution is plain substitution; an exact zero on the diagonal
 *       of R sets that unknown to zero and reports rank deficiency.
 *
 * Parity pins: every function here is pinned by the CPU tests (hand-worked
 * exact examples, exact rational normal equations, invariants, special cases,
 * LAPACK cross-checks); see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stddef.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Number of reflectors of an m x n factorization (reading R2). */
int oracle_num_reflectors(int m, int n)
{
    int k = m - 1;
    if (n < k) k = n;
    return k < 0 ? 0 : k;
}

/*
 * update_pivot_row (Alg. 2 line 3, Task 1): builds reflector k from column k,
 * rows k..m-1.  On return A[k,k] = R_kk = cl, the tail A[k+1:m,k] is unchanged
 * (it is the reflector tail), *up_k = x0 - cl and *b_k = up_k * cl.
 * Returns 0 when the reflector is undefined (zero column: skip), 1 otherwise.
 */
static int update_pivot_row(int m, double *A, int lda, int k, double *up_k, double *b_k)
{
    double c = 0.0;
    for (int i = k; i < m; ++i) {
        double a = fabs(A[IDX(i, k, lda)]);
        if (a > c) c = a;
    }
    if (c == 0.0) {           /* "up or b undefined -> continue" */
        *up_k = 0.0;
        *b_k = 0.0;
        return 0;
    }
    double sum = 0.0;
    for (int i = k; i < m; ++i) {
        double t = A[IDX(i, k, lda)] / c;
        sum += t * t;
    }
    double s = c * sqrt(sum);
    double x0 = A[IDX(k, k, lda)];
    double cl = (x0 > 0.0) ? -s : s;
    *up_k = x0 - cl;
    A[IDX(k, k, lda)] = cl;
    *b_k = (*up_k) * cl;
    return 1;
}

/*
 * update_trailing_non_pivot_row (Alg. 2 line 5): applies reflector k, held in
 * (up_k, V[k+1:m]), to one vector c[k:m] (stride 1):
 *   sigma = (up_k c_k + sum_{i>k} v_i c_i) / b_k;  c_k += sigma up_k;
 *   c_i += sigma v_i  (i > k).
 * This is H_k c with H_k = I + v v^T / b_k; since v^T v = -2 b_k, H_k is the
 * Householder reflector I - 2 v v^T / (v^T v) of Alg. 1.
 */
static void update_trailing_non_pivot_row(int m, const double *V, int k, double up_k,
                                          double b_k, double *c)
{
    double sigma = c[k] * up_k;
    for (int i = k + 1; i < m; ++i) sigma += c[i] * V[i];
    if (sigma == 0.0) return;
    sigma /= b_k;
    c[k] += sigma * up_k;
    for (int i = k + 1; i < m; ++i) c[i] += sigma * V[i];
}

/*
 * In-place H12 QR of the m x n column-major matrix A (Alg. 2, sequential
 * order).  up must hold n doubles; up[k] for k >= min(m-1, n) is set to 0.
 * Returns the number of skipped (zero) pivots.
 */
int oracle_h12_factor(int m, int n, double *A, int lda, double *up)
{
    int K = oracle_num_reflectors(m, n);
    int skipped = 0;
    for (int k = 0; k < n; ++k) up[k] = 0.0;
    for (int k = 0; k < K; ++k) {
        double up_k, b_k;
        if (!update_pivot_row(m, A, lda, k, &up_k, &b_k)) {
            up[k] = 0.0;
            ++skipped;
            continue;
        }
        up[k] = up_k;
        const double *V = &A[IDX(0, k, lda)];
        for (int j = k + 1; j < n; ++j)
            update_trailing_non_pivot_row(m, V, k, up_k, b_k, &A[IDX(0, j, lda)]);
    }
    return skipped;
}

/*
 * Q^T . B for the factorization held in (A, up): B <- H_{K-1} ... H_1 H_0 B,
 * i.e. the reflectors are applied to every right-hand side in the order they
 * were built.  A reflector with b_k = up[k] * R_kk >= 0 (skipped pivot) is not
 * applied.  B is m x nrhs, column-major.
 */
void oracle_apply_qt(int m, int n, const double *A, int lda, const double *up, int nrhs,
                     double *B, int ldb)
{
    int K = oracle_num_reflectors(m, n);
    for (int k = 0; k < K; ++k) {
        double b_k = up[k] * A[IDX(k, k, lda)];
        if (!(b_k < 0.0)) continue;
        const double *V = &A[IDX(0, k, lda)];
        for (int r = 0; r < nrhs; ++r)
            update_trailing_non_pivot_row(m, V, k, up[k], b_k, &B[IDX(0, r, ldb)]);
    }
}

/*
 * Q . B: B <- H_0 H_1 ... H_{K-1} B (the reflectors in reverse order).  Used by
 * the tests to rebuild Q (Q . I) and Q R for the invariants of Alg. 1.
 */
void oracle_apply_q(int m, int n, const double *A, int lda, const double *up, int nrhs,
                    double *B, int ldb)
{
    int K = oracle_num_reflectors(m, n);
    for (int k = K - 1; k >= 0; --k) {
        double b_k = up[k] * A[IDX(k, k, lda)];
        if (!(b_k < 0.0)) continue;
        const double *V = &A[IDX(0, k, lda)];
        for (int r = 0; r < nrhs; ++r)
            update_trailing_non_pivot_row(m, V, k, up[k], b_k, &B[IDX(0, r, ldb)]);
    }
}

/*
 * Back-substitution R X = B[0:n, :] with R = triu(A[0:n, 0:n]) (reading R8).
 * X overwrites B[0:n, :].  x_i = (c_i - sum_{j>i} R_ij x_j) / R_ii for
 * i = n-1 .. 0.  Returns 0, or -5 when some R_ii is exactly zero (that x_i is
 * set to 0, which gives a basic solution).
 */
int oracle_solve_r(int n, const double *A, int lda, int nrhs, double *B, int ldb)
{
    int status = 0;
    for (int r = 0; r < nrhs; ++r) {
        double *x = &B[IDX(0, r, ldb)];
        for (int i = n - 1; i >= 0; --i) {
            double t = x[i];
            for (int j = i + 1; j < n; ++j) t -= A[IDX(i, j, lda)] * x[j];
            double d = A[IDX(i, i, lda)];
            if (d == 0.0) {
                x[i] = 0.0;
                status = -5;
            } else {
                x[i] = t / d;
            }
        }
    }
    return status;
}

/* Least-squares residual norm ||(Q^T b)[n:m]||_2 of one right-hand side. */
double oracle_residual_norm(int m, int n, const double *qtb)
{
    double s = 0.0;
    for (int i = n; i < m; ++i) s += qtb[i] * qtb[i];
    return sqrt(s);
}

/*
 * The whole least-squares solve of one problem, as SLSQP's subproblem runs it:
 * factor A in place, apply Q^T to b, back-substitute; b[0:n] becomes x.
 * Returns the status of the back-substitution.
 */
int oracle_lstsq(int m, int n, double *A, int lda, double *up, double *b)
{
    oracle_h12_factor(m, n, A, lda, up);
    oracle_apply_qt(m, n, A, lda, up, 1, b, m);
    return oracle_solve_r(n, A, lda, 1, b, m);
}
