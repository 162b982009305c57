/*
 * Oracle: plain, slow, sequential FP64 solvers for the structured systems
 * A x = f of Amodio & Brugnano, "Parallel Factorizations in Numerical
 * Analysis" (Sec. 2, Eq. (syst)).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no code
 * with it.
 *
 * What the partition method computes is the unique solution x = A^{-1} f of a
 * nonsingular A (Eq. (parfact): A = F T G is an exact factorization of A, so
 * solving with F, T and G in turn gives A^{-1} f up to rounding).  The oracle
 * therefore writes that definition out with the textbook sequential
 * algorithms, no blocking and no reordering:
 *
 *   oracle_tri_solve     scalar tridiagonal: Thomas (LU without pivoting).
 *   oracle_btri_solve    block tridiagonal: block Thomas, every m x m pivot
 *                        block applied through LU with partial pivoting.
 *   oracle_babd_solve    lower block bidiagonal with an upper-right corner
 *                        (the BABD form of Sec. 2, Eq. (parpart1) with c = 0):
 *                        Gaussian elimination with partial pivoting restricted
 *                        to the rows that are nonzero in the pivot column.
 *   oracle_dense_solve   dense Gaussian elimination with partial pivoting.
 *   oracle_*_residual    r = f - A x, the plain definition.
 *
 * All arrays are row-major host arrays in FP64; the right-hand sides are
 * stored as [rows][nrhs].  Functions return 0 on success, -1 on a zero pivot
 * (singular input) and -2 on invalid sizes.  Compiled with -ffp-contract=off
 * so that every product and sum is rounded on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- m x m Gaussian elimination with partial pivoting (first max |.|) ---- */

/* In-place LU with partial pivoting of the n x n row-major matrix a:
 * P a = L U with unit-lower L stored below the diagonal, U on and above it.
 * piv[k] is the row swapped with row k at step k. */
static int lu_factor(int n, double *a, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(a[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; j++) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        }
        double piv_val = a[(size_t)k * n + k];
        for (int i = k + 1; i < n; i++) {
            double l = a[(size_t)i * n + k] / piv_val;
            a[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++)
                a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    return 0;
}

/* Solve (LU) x = P b for the nc columns of the n x nc row-major b, in place. */
static void lu_solve(int n, const double *lu, const int *piv, double *b, int nc)
{
    for (int k = 0; k < n; k++) {
        int p = piv[k];
        if (p != k) {
            for (int c = 0; c < nc; c++) {
                double t = b[(size_t)k * nc + c];
                b[(size_t)k * nc + c] = b[(size_t)p * nc + c];
                b[(size_t)p * nc + c] = t;
            }
        }
    }
    for (int i = 0; i < n; i++)
        for (int k = 0; k < i; k++) {
            double l = lu[(size_t)i * n + k];
            for (int c = 0; c < nc; c++) b[(size_t)i * nc + c] -= l * b[(size_t)k * nc + c];
        }
    for (int i = n - 1; i >= 0; i--) {
        for (int k = i + 1; k < n; k++) {
            double u = lu[(size_t)i * n + k];
            for (int c = 0; c < nc; c++) b[(size_t)i * nc + c] -= u * b[(size_t)k * nc + c];
        }
        double d = lu[(size_t)i * n + i];
        for (int c = 0; c < nc; c++) b[(size_t)i * nc + c] /= d;
    }
}

/* ---- dense GEPP ---- */

int oracle_dense_solve(int n, const double *A, const double *F, double *X, int nrhs)
{
    if (n < 0 || nrhs < 1) return -2;
    if (n == 0) return 0;
    double *lu = (double *)malloc(sizeof(double) * (size_t)n * n);
    int *piv = (int *)malloc(sizeof(int) * (size_t)n);
    memcpy(lu, A, sizeof(double) * (size_t)n * n);
    int rc = lu_factor(n, lu, piv);
    if (rc == 0) {
        memcpy(X, F, sizeof(double) * (size_t)n * nrhs);
        lu_solve(n, lu, piv, X, nrhs);
    }
    free(lu);
    free(piv);
    return rc;
}

/* ---- scalar tridiagonal: Thomas ---- */

/* Rows i = 0..n-1:  dl[i] x[i-1] + d[i] x[i] + du[i] x[i+1] = f[i]
 * (dl[0] and du[n-1] are ignored).  LU without pivoting: u_0 = d_0,
 * l_i = dl_i / u_{i-1}, u_i = d_i - l_i du_{i-1}; forward g_i = f_i - l_i g_{i-1};
 * backward x_i = (g_i - du_i x_{i+1}) / u_i. */
int oracle_tri_solve(int64_t n, const double *dl, const double *d, const double *du,
                     const double *f, double *x, int nrhs)
{
    if (n < 0 || nrhs < 1) return -2;
    if (n == 0) return 0;
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *l = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = 0;
    u[0] = d[0];
    l[0] = 0.0;
    if (u[0] == 0.0) rc = -1;
    for (int64_t i = 1; i < n && rc == 0; i++) {
        l[i] = dl[i] / u[i - 1];
        u[i] = d[i] - l[i] * du[i - 1];
        if (u[i] == 0.0) rc = -1;
    }
    if (rc == 0) {
        for (int c = 0; c < nrhs; c++) {
            x[c] = f[c];
            for (int64_t i = 1; i < n; i++)
                x[(size_t)i * nrhs + c] = f[(size_t)i * nrhs + c] - l[i] * x[(size_t)(i - 1) * nrhs + c];
            x[(size_t)(n - 1) * nrhs + c] /= u[n - 1];
            for (int64_t i = n - 2; i >= 0; i--)
                x[(size_t)i * nrhs + c] =
                    (x[(size_t)i * nrhs + c] - du[i] * x[(size_t)(i + 1) * nrhs + c]) / u[i];
        }
    }
    free(u);
    free(l);
    return rc;
}

int oracle_tri_residual(int64_t n, const double *dl, const double *d, const double *du,
                        const double *x, const double *f, double *r, int nrhs)
{
    if (n < 0 || nrhs < 1) return -2;
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < nrhs; c++) {
            double ax = d[i] * x[(size_t)i * nrhs + c];
            if (i > 0) ax += dl[i] * x[(size_t)(i - 1) * nrhs + c];
            if (i + 1 < n) ax += du[i] * x[(size_t)(i + 1) * nrhs + c];
            r[(size_t)i * nrhs + c] = f[(size_t)i * nrhs + c] - ax;
        }
    return 0;
}

/* ---- block tridiagonal: block Thomas ---- */

/* Block rows j = 0..N-1 (m x m blocks, row-major, block j at offset j*m*m):
 *   B_j x_{j-1} + D_j x_j + C_j x_{j+1} = f_j      (B_0, C_{N-1} ignored).
 * Forward: D'_0 = D_0; Y_j = D'_j^{-1} C_j; h_j = D'_j^{-1} g_j;
 *          D'_{j+1} = D_{j+1} - B_{j+1} Y_j;  g_{j+1} = f_{j+1} - B_{j+1} h_j.
 * Backward: x_{N-1} = h_{N-1};  x_j = h_j - Y_j x_{j+1}.
 * Each D'_j^{-1} is applied through its LU with partial pivoting. */
int oracle_btri_solve(int64_t N, int m, const double *B, const double *D, const double *C,
                      const double *F, double *X, int nrhs)
{
    if (N < 0 || m < 1 || nrhs < 1) return -2;
    if (N == 0) return 0;
    const size_t mm = (size_t)m * m, mr = (size_t)m * nrhs;
    double *Y = (double *)malloc(sizeof(double) * mm * (size_t)N); /* Y_j */
    double *lu = (double *)malloc(sizeof(double) * mm);
    int *piv = (int *)malloc(sizeof(int) * (size_t)m);
    int rc = 0;
    /* X holds g_j, then h_j, then x_j */
    memcpy(X, F, sizeof(double) * mr * (size_t)N);
    for (int64_t j = 0; j < N && rc == 0; j++) {
        memcpy(lu, D + mm * (size_t)j, sizeof(double) * mm);
        if (j > 0) {
            const double *Bj = B + mm * (size_t)j;
            const double *Yp = Y + mm * (size_t)(j - 1);
            const double *hp = X + mr * (size_t)(j - 1);
            double *gj = X + mr * (size_t)j;
            for (int r = 0; r < m; r++)
                for (int k = 0; k < m; k++) {
                    double b = Bj[(size_t)r * m + k];
                    for (int c = 0; c < m; c++) lu[(size_t)r * m + c] -= b * Yp[(size_t)k * m + c];
                    for (int c = 0; c < nrhs; c++) gj[(size_t)r * nrhs + c] -= b * hp[(size_t)k * nrhs + c];
                }
        }
        if (lu_factor(m, lu, piv) != 0) { rc = -1; break; }
        lu_solve(m, lu, piv, X + mr * (size_t)j, nrhs);
        if (j + 1 < N) {
            memcpy(Y + mm * (size_t)j, C + mm * (size_t)j, sizeof(double) * mm);
            lu_solve(m, lu, piv, Y + mm * (size_t)j, m);
        }
    }
    if (rc == 0) {
        for (int64_t j = N - 2; j >= 0; j--) {
            const double *Yj = Y + mm * (size_t)j;
            const double *xn = X + mr * (size_t)(j + 1);
            double *xj = X + mr * (size_t)j;
            for (int r = 0; r < m; r++)
                for (int k = 0; k < m; k++) {
                    double yv = Yj[(size_t)r * m + k];
                    for (int c = 0; c < nrhs; c++) xj[(size_t)r * nrhs + c] -= yv * xn[(size_t)k * nrhs + c];
                }
        }
    }
    free(Y);
    free(lu);
    free(piv);
    return rc;
}

int oracle_btri_residual(int64_t N, int m, const double *B, const double *D, const double *C,
                         const double *X, const double *F, double *R, int nrhs)
{
    if (N < 0 || m < 1 || nrhs < 1) return -2;
    const size_t mm = (size_t)m * m, mr = (size_t)m * nrhs;
    for (int64_t j = 0; j < N; j++)
        for (int r = 0; r < m; r++)
            for (int c = 0; c < nrhs; c++) {
                double ax = 0.0;
                for (int k = 0; k < m; k++) {
                    if (j > 0) ax += B[mm * (size_t)j + (size_t)r * m + k] * X[mr * (size_t)(j - 1) + (size_t)k * nrhs + c];
                    ax += D[mm * (size_t)j + (size_t)r * m + k] * X[mr * (size_t)j + (size_t)k * nrhs + c];
                    if (j + 1 < N) ax += C[mm * (size_t)j + (size_t)r * m + k] * X[mr * (size_t)(j + 1) + (size_t)k * nrhs + c];
                }
                R[mr * (size_t)j + (size_t)r * nrhs + c] = F[mr * (size_t)j + (size_t)r * nrhs + c] - ax;
            }
    return 0;
}

/* ---- BABD: lower block bidiagonal with an upper-right corner ---- */

/* Unknowns y_0..y_N (m each).  Block row 0:  B0 y_0 + B1 y_N = beta;
 * block row j+1 (j = 0..N-1):  S_j y_j + R_j y_{j+1} = r_j.
 * RHS is [(N+1) m][nrhs] with beta first; Y has the same shape.
 *
 * Gaussian elimination with partial pivoting, column block by column block.
 * Before eliminating the column block of y_j the only rows with nonzeros in
 * it are m rows carried over from the previous step (at j = 0: the boundary
 * rows; they also hold the corner fill-in in the y_N columns) and the m rows
 * of block row j+1.  Partial pivoting over these 2m rows eliminates y_j; the
 * m pivot rows are kept for back substitution and the other m rows carry on.
 * When j + 1 = N the columns of y_{j+1} and y_N coincide and are merged; the
 * final m x m system in y_N is solved by GEPP. */
int oracle_babd_solve(int64_t N, int m, const double *S, const double *R, const double *B0,
                      const double *B1, const double *RHS, double *Y, int nrhs)
{
    if (N < 1 || m < 1 || nrhs < 1) return -2;
    const size_t mm = (size_t)m * m, mr = (size_t)m * nrhs;
    const int W = 3 * m + nrhs;                   /* columns: y_j | y_{j+1} | y_N | rhs */
    double *work = (double *)malloc(sizeof(double) * (size_t)(2 * m) * W);
    /* kept pivot rows per step: m x W each (U in the y_j columns) */
    double *keep = (double *)malloc(sizeof(double) * (size_t)N * m * W);
    double *shift = (double *)malloc(sizeof(double) * (size_t)W);
    int rc = 0;
    /* carried rows, stored in work rows 0..m-1 */
    memset(work, 0, sizeof(double) * (size_t)(2 * m) * W);
    for (int r = 0; r < m; r++) {
        for (int c = 0; c < m; c++) {
            work[(size_t)r * W + c] = B0[(size_t)r * m + c];
            work[(size_t)r * W + 2 * m + c] = B1[(size_t)r * m + c];
        }
        for (int c = 0; c < nrhs; c++) work[(size_t)r * W + 3 * m + c] = RHS[(size_t)r * nrhs + c];
    }
    for (int64_t j = 0; j < N && rc == 0; j++) {
        const int last = (j + 1 == N);
        /* rows m..2m-1: block row j+1 of A */
        for (int r = 0; r < m; r++) {
            double *w = work + (size_t)(m + r) * W;
            memset(w, 0, sizeof(double) * W);
            for (int c = 0; c < m; c++) {
                w[c] = S[mm * (size_t)j + (size_t)r * m + c];
                w[(last ? 2 * m : m) + c] = R[mm * (size_t)j + (size_t)r * m + c];
            }
            for (int c = 0; c < nrhs; c++) w[3 * m + c] = RHS[mr * (size_t)(j + 1) + (size_t)r * nrhs + c];
        }
        /* eliminate the y_j columns with partial pivoting over the 2m rows */
        for (int k = 0; k < m; k++) {
            int p = k;
            double best = fabs(work[(size_t)k * W + k]);
            for (int i = k + 1; i < 2 * m; i++) {
                double v = fabs(work[(size_t)i * W + k]);
                if (v > best) { best = v; p = i; }
            }
            if (best == 0.0) { rc = -1; break; }
            if (p != k)
                for (int c = 0; c < W; c++) {
                    double t = work[(size_t)k * W + c];
                    work[(size_t)k * W + c] = work[(size_t)p * W + c];
                    work[(size_t)p * W + c] = t;
                }
            double pv = work[(size_t)k * W + k];
            for (int i = k + 1; i < 2 * m; i++) {
                double l = work[(size_t)i * W + k] / pv;
                work[(size_t)i * W + k] = 0.0;
                for (int c = k + 1; c < W; c++) work[(size_t)i * W + c] -= l * work[(size_t)k * W + c];
            }
        }
        if (rc) break;
        memcpy(keep + (size_t)j * m * W, work, sizeof(double) * (size_t)m * W);
        /* rows m..2m-1 now have zeros in the y_j columns: they carry on, their
         * y_{j+1} columns become the y_j columns of the next step */
        for (int r = 0; r < m; r++) {
            double *dst = work + (size_t)r * W;
            const double *src = work + (size_t)(m + r) * W;
            memset(shift, 0, sizeof(double) * W);
            for (int c = 0; c < m; c++) { shift[c] = src[m + c]; shift[2 * m + c] = src[2 * m + c]; }
            for (int c = 0; c < nrhs; c++) shift[3 * m + c] = src[3 * m + c];
            memcpy(dst, shift, sizeof(double) * W);
        }
    }
    if (rc == 0) {
        /* final m x m system in y_N: the carried rows' y_N columns */
        double *a = (double *)malloc(sizeof(double) * mm);
        double *b = (double *)malloc(sizeof(double) * mr);
        int *piv = (int *)malloc(sizeof(int) * (size_t)m);
        for (int r = 0; r < m; r++) {
            for (int c = 0; c < m; c++) a[(size_t)r * m + c] = work[(size_t)r * W + 2 * m + c];
            for (int c = 0; c < nrhs; c++) b[(size_t)r * nrhs + c] = work[(size_t)r * W + 3 * m + c];
        }
        if (lu_factor(m, a, piv) != 0) rc = -1;
        else {
            lu_solve(m, a, piv, b, nrhs);
            memcpy(Y + mr * (size_t)N, b, sizeof(double) * mr);
            /* back substitution: U_j y_j = rhs - P_j y_{j+1} - Q_j y_N */
            for (int64_t j = N - 1; j >= 0; j--) {
                const double *kp = keep + (size_t)j * m * W;
                const int last = (j + 1 == N);
                const double *yn = Y + mr * (size_t)N;
                const double *y1 = Y + mr * (size_t)(j + 1);
                double *yj = Y + mr * (size_t)j;
                for (int r = m - 1; r >= 0; r--)
                    for (int c = 0; c < nrhs; c++) {
                        double s = kp[(size_t)r * W + 3 * m + c];
                        for (int k = r + 1; k < m; k++) s -= kp[(size_t)r * W + k] * yj[(size_t)k * nrhs + c];
                        if (!last)
                            for (int k = 0; k < m; k++) s -= kp[(size_t)r * W + m + k] * y1[(size_t)k * nrhs + c];
                        for (int k = 0; k < m; k++) s -= kp[(size_t)r * W + 2 * m + k] * yn[(size_t)k * nrhs + c];
                        yj[(size_t)r * nrhs + c] = s / kp[(size_t)r * W + r];
                    }
            }
        }
        free(a);
        free(b);
        free(piv);
    }
    free(work);
    free(keep);
    free(shift);
    return rc;
}

int oracle_babd_residual(int64_t N, int m, const double *S, const double *R, const double *B0,
                         const double *B1, const double *Y, const double *RHS, double *Rout, int nrhs)
{
    if (N < 1 || m < 1 || nrhs < 1) return -2;
    const size_t mm = (size_t)m * m, mr = (size_t)m * nrhs;
    for (int r = 0; r < m; r++)
        for (int c = 0; c < nrhs; c++) {
            double ax = 0.0;
            for (int k = 0; k < m; k++) {
                ax += B0[(size_t)r * m + k] * Y[(size_t)k * nrhs + c];
                ax += B1[(size_t)r * m + k] * Y[mr * (size_t)N + (size_t)k * nrhs + c];
            }
            Rout[(size_t)r * nrhs + c] = RHS[(size_t)r * nrhs + c] - ax;
        }
    for (int64_t j = 0; j < N; j++)
        for (int r = 0; r < m; r++)
            for (int c = 0; c < nrhs; c++) {
                double ax = 0.0;
                for (int k = 0; k < m; k++) {
                    ax += S[mm * (size_t)j + (size_t)r * m + k] * Y[mr * (size_t)j + (size_t)k * nrhs + c];
                    ax += R[mm * (size_t)j + (size_t)r * m + k] * Y[mr * (size_t)(j + 1) + (size_t)k * nrhs + c];
                }
                Rout[mr * (size_t)(j + 1) + (size_t)r * nrhs + c] = RHS[mr * (size_t)(j + 1) + (size_t)r * nrhs + c] - ax;
            }
    return 0;
}
