/*
 * Plain FP64 CPU oracle for the Chebyshev filter of ChFSI (test infrastructure).
 *
 * This file is the reference the CUDA path is checked against.  Only tests/,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the product
 * library never does.  It shares no code with the CUDA sources.
 *
 * Everything is written the slow, obvious way:
 *   - CSR sparse x dense products row by row, summing each row's terms in stored
 *     column order, compiled with -ffp-contract=off (no fused multiply-add);
 *   - the filter is the three-term Chebyshev recurrence of Algorithm 1, step 1
 *     (Sec. 3.4), with its coefficients derived from T_{k+1} = 2x T_k - T_{k-1};
 *   - the adjoint is plain reverse-mode differentiation of that loop with every
 *     iterate stored (no checkpointing), using the transpose product H^T.
 * OpenMP splits rows (or column slices) across threads; every output element is
 * produced by one thread in a fixed order, so results do not depend on the
 * thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Y = H X for CSR H (N x N), dense row-major X (N x n, leading dim ldx). */
void oracle_spmm(int64_t N, const int64_t* row_ptr, const int32_t* col, const double* val,
                 int64_t n, const double* X, int64_t ldx, double* Y, int64_t ldy) {
    int64_t r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < N; r++) {
        double* y = Y + r * ldy;
        for (int64_t j = 0; j < n; j++) y[j] = 0.0;
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; p++) {
            const double h = val[p];
            const double* x = X + (int64_t)col[p] * ldx;
            for (int64_t j = 0; j < n; j++) y[j] = y[j] + h * x[j];
        }
    }
}

/* Y = H^T X by scattering each stored entry H[r, col] into row col of Y.
 * Threads own disjoint column slices of Y, so there are no write conflicts. */
void oracle_spmm_t(int64_t N, const int64_t* row_ptr, const int32_t* col, const double* val,
                   int64_t n, const double* X, int64_t ldx, double* Y, int64_t ldy) {
    const int64_t slice = 16;
    const int64_t nslices = (n + slice - 1) / slice;
    int64_t s;
#pragma omp parallel for schedule(static)
    for (s = 0; s < nslices; s++) {
        const int64_t j0 = s * slice, j1 = (j0 + slice < n) ? j0 + slice : n;
        for (int64_t r = 0; r < N; r++)
            for (int64_t j = j0; j < j1; j++) Y[r * ldy + j] = 0.0;
        for (int64_t r = 0; r < N; r++) {
            const double* x = X + r * ldx;
            for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; p++) {
                const double h = val[p];
                double* y = Y + (int64_t)col[p] * ldy;
                for (int64_t j = j0; j < j1; j++) y[j] = y[j] + h * x[j];
            }
        }
    }
}

/* Copy a dense N x n block between leading dimensions. */
static void copy_block(int64_t N, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb) {
    for (int64_t r = 0; r < N; r++) memcpy(B + r * ldb, A + r * lda, (size_t)n * sizeof(double));
}

/*
 * Coefficients of the scaled Chebyshev filter of Algorithm 1, step 1 (Sec. 3.4),
 * derived here from the textbook three-term recurrence T_{k+1}(x) = 2x T_k(x) - T_{k-1}(x).
 *
 * The affine map t -> (t - c)/e with c = (b + a)/2 and half-width e = (b - a)/2 sends
 * the unwanted interval [a, b] onto [-1, 1]; the filter polynomial of degree k is
 * p_k(t) = T_k((t - c)/e) / T_k(tau) with tau = (a0 - c)/e, so that p_k(a0) = 1.
 * With the ratio r_k = T_{k-1}(tau)/T_k(tau) (r_1 = 1/tau) the Chebyshev recurrence
 * divided by T_{k+1}(tau) gives
 *     r_{k+1} = 1/(2 tau - r_k),
 *     Y_1     = (r_1/e)(H - c) Y_0,
 *     Y_{k+1} = (2 r_{k+1}/e)(H - c) Y_k - r_k r_{k+1} Y_{k-1},
 * i.e. Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2} with alpha_1 = r_1/e,
 * alpha_k = 2 r_k/e and beta_k = r_{k-1} r_k (k >= 2).  The paper's sigma_k is this
 * ratio r_k.  Inputs a = eps_ub^w, b = eps_ub^uw, a0 = eps_0.
 * alpha and beta have m+1 entries (index 0 unused, beta_1 = 0).
 */
void oracle_coefficients(int32_t m, double a, double b, double a0, double* alpha, double* beta,
                         double* c_out) {
    const double half_width = (b - a) / 2.0;
    const double centre = (b + a) / 2.0;
    const double tau = (a0 - centre) / half_width;
    double r = 1.0 / tau;                    /* r_1 */
    alpha[0] = 0.0; beta[0] = 0.0;
    alpha[1] = r / half_width; beta[1] = 0.0;
    for (int32_t k = 2; k <= m; k++) {
        const double r_next = 1.0 / (2.0 * tau - r);
        alpha[k] = 2.0 * r_next / half_width;
        beta[k] = r * r_next;
        r = r_next;
    }
    *c_out = centre;
}

/*
 * Y = Y_m of the scaled Chebyshev filter (Algorithm 1, step 1; Sec. 3.4): the
 * newest iterate of the three-term recurrence whose coefficients
 * oracle_coefficients gives,
 *     Y_0 = X,  Y_k = alpha_k (H Y_{k-1} - c Y_{k-1}) - beta_k Y_{k-2}  (beta_1 = 0).
 * The product H Y_{k-1} is formed first (oracle_spmm), then each element is
 * combined in that order.  work holds 3 * N * n doubles (Y_{k-2}, Y_{k-1}, H Y_{k-1}).
 * Returns 0, or -1 for m < 1.
 */
int oracle_filter(int64_t N, const int64_t* row_ptr, const int32_t* col, const double* val,
                  int64_t n, const double* X_in, int64_t ldx, int32_t m,
                  double a, double b, double a0, double* Y, int64_t ldy, double* work) {
    if (m < 1) return -1;
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double* beta = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double c;
    oracle_coefficients(m, a, b, a0, alpha, beta, &c);

    double* older = work;               /* Y_{k-2}; becomes Y_k in place */
    double* newer = work + N * n;       /* Y_{k-1}                       */
    double* prod = work + 2 * N * n;    /* H Y_{k-1}                     */
    copy_block(N, n, X_in, ldx, newer, n);   /* Y_0 */
    for (int64_t q = 0; q < N * n; q++) older[q] = 0.0;

    for (int32_t k = 1; k <= m; k++) {
        oracle_spmm(N, row_ptr, col, val, n, newer, n, prod, n);
        const double ak = alpha[k], bk = beta[k];
        int64_t r;
#pragma omp parallel for schedule(static)
        for (r = 0; r < N; r++)
            for (int64_t j = 0; j < n; j++) {
                const int64_t q = r * n + j;
                double v = ak * (prod[q] - c * newer[q]);
                if (k >= 2) v = v - bk * older[q];
                older[q] = v;             /* Y_k overwrites Y_{k-2} after reading it */
            }
        double* t = older; older = newer; newer = t;   /* (Y_{k-1}, Y_k) */
    }
    copy_block(N, n, newer, n, Y, ldy);
    free(alpha);
    free(beta);
    return 0;
}

/*
 * Reverse-mode derivative of the filter for a loss with dL/dY_m = G.
 *   Ybar_m = G
 *   Ybar_{k-1} += alpha_k (H^T - c) Ybar_k,   Ybar_{k-2} -= beta_k Ybar_k   (k = m..1)
 *   dH[p] += alpha_k * <Ybar_k[row p, :], Y_{k-1}[col p, :]>   for every stored entry p
 *   dX = Ybar_0
 * All iterates Y_0..Y_m are kept.  work holds (m + 4) * N * n doubles.
 * dH may be NULL (skipped).  Returns 0, or -1 for m < 1.
 */
int oracle_filter_adjoint(int64_t N, const int64_t* row_ptr, const int32_t* col, const double* val,
                          int64_t n, const double* X_in, int64_t ldx, int32_t m,
                          double a, double b, double a0, const double* G, int64_t ldg,
                          double* dX, int64_t lddx, double* dH, double* work) {
    if (m < 1) return -1;
    double* alpha = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double* beta = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double c;
    oracle_coefficients(m, a, b, a0, alpha, beta, &c);
    const int64_t Nn = N * n;
    double* Ys = work;                        /* Y_0..Y_m, (m+1) blocks */
    double* Bk = work + (int64_t)(m + 1) * Nn;  /* Ybar_k     */
    double* Bk1 = Bk + Nn;                    /* Ybar_{k-1} */
    double* T = Bk1 + Nn;                     /* H^T Ybar_k */
    int64_t r;

    /* forward pass, storing every iterate */
    copy_block(N, n, X_in, ldx, Ys, n);
    for (int32_t k = 1; k <= m; k++) {
        const double* Yp = Ys + (int64_t)(k - 1) * Nn;
        const double* Ypp = (k >= 2) ? Ys + (int64_t)(k - 2) * Nn : NULL;
        double* Yk = Ys + (int64_t)k * Nn;
        oracle_spmm(N, row_ptr, col, val, n, Yp, n, T, n);
#pragma omp parallel for schedule(static)
        for (r = 0; r < N; r++)
            for (int64_t j = 0; j < n; j++) {
                const int64_t q = r * n + j;
                double v = alpha[k] * (T[q] - c * Yp[q]);
                if (Ypp) v = v - beta[k] * Ypp[q];
                Yk[q] = v;
            }
    }

    /* reverse pass: Bk = Ybar_k, Bk1 accumulates Ybar_{k-1}; the pending
     * -beta term for Ybar_{k-2} is folded in when that block becomes current. */
    if (dH) for (int64_t p = 0; p < row_ptr[N]; p++) dH[p] = 0.0;
    copy_block(N, n, G, ldg, Bk, n);          /* Ybar_m */
    double* Bprev = NULL;                     /* Ybar_{k+1}, for the beta term */
    double* spare = (double*)malloc(sizeof(double) * (size_t)Nn);
    for (int32_t k = m; k >= 1; k--) {
        const double* Ykm1 = Ys + (int64_t)(k - 1) * Nn;
        /* dH contribution of step k */
        if (dH) {
#pragma omp parallel for schedule(static)
            for (r = 0; r < N; r++)
                for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; p++) {
                    const double* yb = Bk + r * n;
                    const double* yv = Ykm1 + (int64_t)col[p] * n;
                    double s = 0.0;
                    for (int64_t j = 0; j < n; j++) s = s + yb[j] * yv[j];
                    dH[p] = dH[p] + alpha[k] * s;
                }
        }
        /* Ybar_{k-1} = alpha_k (H^T Ybar_k - c Ybar_k) - beta_{k+1} Ybar_{k+1} */
        oracle_spmm_t(N, row_ptr, col, val, n, Bk, n, T, n);
        const double bnext = (k + 1 <= m) ? beta[k + 1] : 0.0;
#pragma omp parallel for schedule(static)
        for (r = 0; r < N; r++)
            for (int64_t j = 0; j < n; j++) {
                const int64_t q = r * n + j;
                double v = alpha[k] * (T[q] - c * Bk[q]);
                if (Bprev) v = v - bnext * Bprev[q];
                Bk1[q] = v;
            }
        /* rotate: Ybar_{k+1} <- Ybar_k, Ybar_k <- Ybar_{k-1} */
        if (!Bprev) Bprev = spare;
        memcpy(Bprev, Bk, sizeof(double) * (size_t)Nn);
        memcpy(Bk, Bk1, sizeof(double) * (size_t)Nn);
    }
    copy_block(N, n, Bk, n, dX, lddx);        /* dX = Ybar_0 */
    free(spare);
    free(alpha);
    free(beta);
    return 0;
}
