/*
 * FP64 CPU oracle for the loop nests that loop internalization (paper Sec. VI-C)
 * and array-reduction detection (paper Sec. VI-B) speed up: GEMM, a chain of
 * two GEMMs (polybench 2mm), three chained products (polybench 3mm),
 * covariance, correlation, SYRK and SYR2K, plus the vector-Jacobian products of
 * the chain, 3mm, covariance and correlation, and Gram-Schmidt QR (polybench
 * gramschmidt).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain definition of what the GPU
 * library computes, written as straightforward FP64 loops with no blocking, no
 * fusion and no reordering beyond the definition. Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or constant with the CUDA library and includes nothing from it.
 *
 * Conventions: every matrix is row-major and contiguous (leading dimension =
 * number of columns); every value is an FP64 number (FP32 inputs are widened
 * exactly by the caller). Summations run in the natural index order.
 *
 * Loop internalization and reduction detection only change where operands live
 * and how often an accumulator is written back; the value they compute is the
 * plain loop nest's value (paper Sec. VI-B, Sec. VI-C, Listings 5 and 6), so
 * the oracle is that loop nest.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - alpha/beta placement: C = alpha*A*B + beta*C (polybench GEMM form);
 *    beta == 0 means the input C is never read (BLAS convention).
 *  - covariance divisor: n - 1 (sample covariance).
 *  - correlation: corr_ii = 1 exactly; corr_ij = 0 when a column has zero
 *    variance (no division by zero).
 *  - SYRK/SYR2K fill: LOWER/UPPER read and write only that triangle of C;
 *    FULL computes the lower triangle from C's lower triangle and writes the
 *    value to both (i,j) and (j,i).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_FILL_FULL 0
#define ORACLE_FILL_LOWER 1
#define ORACLE_FILL_UPPER 2

/* Number of host threads the loops may use (OpenMP over output rows). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * GEMM, polybench form: C_out[i][j] = alpha * sum_k A[i][k] * B[k][j] + beta * C_in[i][j].
 * A is MxK, B is KxN, C is MxN. The k-loop is the per-work-item loop of the
 * paper's loop-internalization candidate (Sec. VI-C, Listing 5); the scalar
 * accumulator is the array-reduction form of Sec. VI-B. C_in may equal C_out.
 */
void oracle_gemm(int M, int N, int K, double alpha, const double *A, const double *B,
                 double beta, const double *C_in, double *C_out) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < N; ++j) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += A[(size_t)i * K + k] * B[(size_t)k * N + j];
            double c = (beta == 0.0) ? 0.0 : beta * C_in[(size_t)i * N + j];
            C_out[(size_t)i * N + j] = alpha * acc + c;
        }
    }
}

/*
 * Chained product (polybench 2mm, paper Sec. VIII): T = A*B, E = T*C,
 * F = alpha*E + beta*D. A is ni x nk, B is nk x nj, C is nj x nl, D/E/F are
 * ni x nl. T (ni x nj) is kept in FP64 and returned when T_out is not NULL.
 */
void oracle_gemm_chain(int ni, int nj, int nk, int nl, double alpha, const double *A,
                       const double *B, const double *C, double beta, const double *D,
                       double *T_out, double *E, double *F) {
    double *T = T_out ? T_out : (double *)malloc(sizeof(double) * (size_t)ni * nj + 1);
    oracle_gemm(ni, nj, nk, 1.0, A, B, 0.0, NULL, T);
    oracle_gemm(ni, nl, nj, 1.0, T, C, 0.0, NULL, E);
    for (size_t p = 0; p < (size_t)ni * nl; ++p)
        F[p] = alpha * E[p] + ((beta == 0.0) ? 0.0 : beta * D[p]);
    if (!T_out) free(T);
}

/*
 * Column statistics of a data matrix X (n samples x m features), two passes:
 * mean_j = (1/n) sum_s X[s][j]; ss_j = sum_s (X[s][j] - mean_j)^2.
 * These are the array reductions of polybench covariance/correlation.
 */
void oracle_col_stats(int n, int m, const double *X, double *mean, double *ss) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += X[(size_t)r * m + j];
        double mu = (n > 0) ? s / n : 0.0;
        double q = 0.0;
        for (int r = 0; r < n; ++r) {
            double d = X[(size_t)r * m + j] - mu;
            q += d * d;
        }
        mean[j] = mu;
        ss[j] = q;
    }
}

/*
 * Covariance (polybench covariance): cov[i][j] = sum_s Xc[s][i] * Xc[s][j] / (n - 1)
 * with Xc = X - 1*mean^T from the two-pass mean. n >= 2.
 */
void oracle_covariance(int n, int m, const double *X, double *cov) {
    double *mean = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *ss = (double *)malloc(sizeof(double) * (size_t)m + 1);
    oracle_col_stats(n, m, X, mean, ss);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j <= i; ++j) {
            double acc = 0.0;
            for (int r = 0; r < n; ++r)
                acc += (X[(size_t)r * m + i] - mean[i]) * (X[(size_t)r * m + j] - mean[j]);
            double v = acc / (double)(n - 1);
            cov[(size_t)i * m + j] = v;
            cov[(size_t)j * m + i] = v;
        }
    }
    free(mean);
    free(ss);
}

/*
 * Correlation (polybench correlation): corr[i][j] =
 * sum_s Xc[s][i] Xc[s][j] / (sqrt(ss_i) * sqrt(ss_j)) for i != j, corr[i][i] = 1,
 * and corr[i][j] = 0 (i != j) when ss_i or ss_j is zero.
 */
void oracle_correlation(int n, int m, const double *X, double *corr) {
    double *mean = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *ss = (double *)malloc(sizeof(double) * (size_t)m + 1);
    oracle_col_stats(n, m, X, mean, ss);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < m; ++i) {
        corr[(size_t)i * m + i] = 1.0;
        for (int j = 0; j < i; ++j) {
            double v = 0.0;
            if (ss[i] > 0.0 && ss[j] > 0.0) {
                double acc = 0.0;
                for (int r = 0; r < n; ++r)
                    acc += (X[(size_t)r * m + i] - mean[i]) * (X[(size_t)r * m + j] - mean[j]);
                v = acc / (sqrt(ss[i]) * sqrt(ss[j]));
            }
            corr[(size_t)i * m + j] = v;
            corr[(size_t)j * m + i] = v;
        }
    }
    free(mean);
    free(ss);
}

/*
 * Three chained products (polybench 3mm, paper Sec. VIII, one of the kernels
 * loop internalization speeds up): E = A*B, F = C*D, G = E*F, no scaling.
 * A is ni x nk, B is nk x nj, C is nj x nm, D is nm x nl; E is ni x nj,
 * F is nj x nl, G is ni x nl. E and F are kept in FP64 and returned when the
 * pointers are not NULL.
 */
void oracle_3mm(int ni, int nj, int nk, int nl, int nm, const double *A, const double *B,
                const double *C, const double *D, double *E_out, double *F_out, double *G) {
    double *E = E_out ? E_out : (double *)malloc(sizeof(double) * (size_t)ni * nj + 1);
    double *F = F_out ? F_out : (double *)malloc(sizeof(double) * (size_t)nj * nl + 1);
    oracle_gemm(ni, nj, nk, 1.0, A, B, 0.0, NULL, E);
    oracle_gemm(nj, nl, nm, 1.0, C, D, 0.0, NULL, F);
    oracle_gemm(ni, nl, nj, 1.0, E, F, 0.0, NULL, G);
    if (!E_out) free(E);
    if (!F_out) free(F);
}

/*
 * X_out = P * Q^T (P is r x c, Q is s x c, X_out is r x s), the contraction
 * over the shared trailing index that the 3mm adjoint uses.
 */
static void oracle_mm_nt(int r, int s, int c, const double *Pm, const double *Qm, double *X_out) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < s; ++j) {
            double acc = 0.0;
            for (int q = 0; q < c; ++q) acc += Pm[(size_t)i * c + q] * Qm[(size_t)j * c + q];
            X_out[(size_t)i * s + j] = acc;
        }
}

/* X_out = P^T * Q (P is c x r, Q is c x s, X_out is r x s). */
static void oracle_mm_tn(int r, int s, int c, const double *Pm, const double *Qm, double *X_out) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < s; ++j) {
            double acc = 0.0;
            for (int q = 0; q < c; ++q) acc += Pm[(size_t)q * r + i] * Qm[(size_t)q * s + j];
            X_out[(size_t)i * s + j] = acc;
        }
}

/*
 * Vector-Jacobian product of 3mm, G = (A B)(C D), for an upstream gradient
 * Gb = dL/dG (ni x nl). With E = A B and F = C D: dE = Gb F^T, dF = E^T Gb,
 * dA = dE B^T, dB = A^T dE, dC = dF D^T, dD = C^T dF.
 */
void oracle_3mm_vjp(int ni, int nj, int nk, int nl, int nm, const double *A, const double *B, const double *C,
                    const double *D, const double *Gb, double *dA, double *dB, double *dC, double *dD) {
    double *E = (double *)malloc(sizeof(double) * (size_t)ni * nj + 1);
    double *F = (double *)malloc(sizeof(double) * (size_t)nj * nl + 1);
    double *dE = (double *)malloc(sizeof(double) * (size_t)ni * nj + 1);
    double *dF = (double *)malloc(sizeof(double) * (size_t)nj * nl + 1);
    oracle_gemm(ni, nj, nk, 1.0, A, B, 0.0, NULL, E);
    oracle_gemm(nj, nl, nm, 1.0, C, D, 0.0, NULL, F);
    oracle_mm_nt(ni, nj, nl, Gb, F, dE);
    oracle_mm_tn(nj, nl, ni, E, Gb, dF);
    oracle_mm_nt(ni, nk, nj, dE, B, dA);
    oracle_mm_tn(nk, nj, ni, A, dE, dB);
    oracle_mm_nt(nj, nm, nl, dF, D, dC);
    oracle_mm_tn(nm, nl, nj, C, dF, dD);
    free(E);
    free(F);
    free(dE);
    free(dF);
}

static int in_fill(int fill, int i, int j) {
    if (fill == ORACLE_FILL_UPPER) return i <= j;
    return i >= j; /* LOWER, and FULL computes the lower triangle */
}

/*
 * SYRK (polybench syrk): on the selected triangle,
 * C_out[i][j] = alpha * sum_k A[i][k] * A[j][k] + beta * C_in[i][j]; A is n x k.
 * Entries outside the triangle are copied from C_in (LOWER/UPPER) or mirrored
 * from the computed lower triangle (FULL). C_in may equal C_out.
 */
void oracle_syrk(int fill, int n, int k, double alpha, const double *A, double beta,
                 const double *C_in, double *C_out) {
    if (C_out != C_in && fill != ORACLE_FILL_FULL)
        memcpy(C_out, C_in, sizeof(double) * (size_t)n * n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            if (!in_fill(fill, i, j)) continue;
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += A[(size_t)i * k + q] * A[(size_t)j * k + q];
            double c = (beta == 0.0) ? 0.0 : beta * C_in[(size_t)i * n + j];
            C_out[(size_t)i * n + j] = alpha * acc + c;
        }
    }
    if (fill == ORACLE_FILL_FULL)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) C_out[(size_t)j * n + i] = C_out[(size_t)i * n + j];
}

/*
 * SYR2K (polybench syr2k): on the selected triangle,
 * C_out[i][j] = alpha * sum_k (A[i][k] * B[j][k] + B[i][k] * A[j][k]) + beta * C_in[i][j];
 * A and B are n x k. Fill handling as for oracle_syrk.
 */
void oracle_syr2k(int fill, int n, int k, double alpha, const double *A, const double *B,
                  double beta, const double *C_in, double *C_out) {
    if (C_out != C_in && fill != ORACLE_FILL_FULL)
        memcpy(C_out, C_in, sizeof(double) * (size_t)n * n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            if (!in_fill(fill, i, j)) continue;
            double acc = 0.0;
            for (int q = 0; q < k; ++q)
                acc += A[(size_t)i * k + q] * B[(size_t)j * k + q] +
                       B[(size_t)i * k + q] * A[(size_t)j * k + q];
            double c = (beta == 0.0) ? 0.0 : beta * C_in[(size_t)i * n + j];
            C_out[(size_t)i * n + j] = alpha * acc + c;
        }
    }
    if (fill == ORACLE_FILL_FULL)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) C_out[(size_t)j * n + i] = C_out[(size_t)i * n + j];
}

/*
 * Vector-Jacobian product of E = (A*B)*C with upstream gradient G = dL/dE
 * (ni x nl). By the product rule on the two matrix products:
 *   dA = G * (B*C)^T,  dB = A^T * G * C^T,  dC = (A*B)^T * G.
 * Each factor is formed explicitly with plain loops.
 */
void oracle_gemm_chain_vjp(int ni, int nj, int nk, int nl, const double *A, const double *B,
                           const double *C, const double *G, double *dA, double *dB, double *dC) {
    double *BC = (double *)malloc(sizeof(double) * (size_t)nk * nl + 1);  /* B*C,   nk x nl */
    double *T = (double *)malloc(sizeof(double) * (size_t)ni * nj + 1);   /* A*B,   ni x nj */
    double *GCt = (double *)malloc(sizeof(double) * (size_t)ni * nj + 1); /* G*C^T, ni x nj */
    oracle_gemm(nk, nl, nj, 1.0, B, C, 0.0, NULL, BC);
    oracle_gemm(ni, nj, nk, 1.0, A, B, 0.0, NULL, T);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < ni; ++i)
        for (int j = 0; j < nj; ++j) {
            double acc = 0.0;
            for (int l = 0; l < nl; ++l) acc += G[(size_t)i * nl + l] * C[(size_t)j * nl + l];
            GCt[(size_t)i * nj + j] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < ni; ++i)
        for (int k = 0; k < nk; ++k) {
            double acc = 0.0;
            for (int l = 0; l < nl; ++l) acc += G[(size_t)i * nl + l] * BC[(size_t)k * nl + l];
            dA[(size_t)i * nk + k] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j) {
            double acc = 0.0;
            for (int i = 0; i < ni; ++i) acc += A[(size_t)i * nk + k] * GCt[(size_t)i * nj + j];
            dB[(size_t)k * nj + j] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nj; ++j)
        for (int l = 0; l < nl; ++l) {
            double acc = 0.0;
            for (int i = 0; i < ni; ++i) acc += T[(size_t)i * nj + j] * G[(size_t)i * nl + l];
            dC[(size_t)j * nl + l] = acc;
        }
    free(BC);
    free(T);
    free(GCt);
}

/*
 * Vector-Jacobian product of cov(X) with upstream gradient W = dL/dcov (m x m).
 * cov = Xc^T Xc / (n-1) gives dL/dXc = Xc (W + W^T) / (n-1); the centring
 * Xc = X - 1 mean^T contributes dX = dXc - 1 (1^T dXc) / n.
 */
void oracle_covariance_vjp(int n, int m, const double *X, const double *W, double *dX) {
    double *mean = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *ss = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *colsum = (double *)calloc((size_t)m + 1, sizeof(double));
    oracle_col_stats(n, m, X, mean, ss);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int i = 0; i < m; ++i)
                acc += (X[(size_t)r * m + i] - mean[i]) * (W[(size_t)i * m + j] + W[(size_t)j * m + i]);
            dX[(size_t)r * m + j] = acc / (double)(n - 1);
        }
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) colsum[j] += dX[(size_t)r * m + j];
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) dX[(size_t)r * m + j] -= colsum[j] / n;
    free(mean);
    free(ss);
    free(colsum);
}

/*
 * Vector-Jacobian product of corr(X) with upstream gradient W = dL/dcorr.
 * With s_j = sqrt(ss_j), Z = Xc diag(1/s) and R = Z^T Z (off-diagonal = corr):
 *   dZ = Z (W' + W'^T), W' = W with its diagonal zeroed (corr_ii = 1 is constant);
 *   dXc_j = (dZ_j - Z_j (Z_j . dZ_j)) / s_j  (adjoint of the column normalisation);
 *   dX = dXc - 1 (1^T dXc) / n               (adjoint of the centring).
 * Columns with s_j = 0 have corr_ij = 0 for all i != j and get dX_j = 0.
 */
void oracle_correlation_vjp(int n, int m, const double *X, const double *W, double *dX) {
    double *mean = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *ss = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *s = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * m + 1);
    double *dZ = (double *)malloc(sizeof(double) * (size_t)n * m + 1);
    double *dot = (double *)calloc((size_t)m + 1, sizeof(double));
    double *colsum = (double *)calloc((size_t)m + 1, sizeof(double));
    oracle_col_stats(n, m, X, mean, ss);
    for (int j = 0; j < m; ++j) s[j] = sqrt(ss[j]);
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j)
            Z[(size_t)r * m + j] = (s[j] > 0.0) ? (X[(size_t)r * m + j] - mean[j]) / s[j] : 0.0;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int i = 0; i < m; ++i) {
                if (i == j) continue;
                acc += Z[(size_t)r * m + i] * (W[(size_t)i * m + j] + W[(size_t)j * m + i]);
            }
            dZ[(size_t)r * m + j] = acc;
        }
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) dot[j] += Z[(size_t)r * m + j] * dZ[(size_t)r * m + j];
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) {
            double v = (s[j] > 0.0) ? (dZ[(size_t)r * m + j] - Z[(size_t)r * m + j] * dot[j]) / s[j] : 0.0;
            dX[(size_t)r * m + j] = v;
            colsum[j] += v;
        }
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < m; ++j) dX[(size_t)r * m + j] -= colsum[j] / n;
    free(mean);
    free(ss);
    free(s);
    free(Z);
    free(dZ);
    free(dot);
    free(colsum);
}

/*
 * Selected rows of the covariance (corr == 0) or correlation (corr != 0)
 * matrix, by the same definitions as oracle_covariance / oracle_correlation:
 * out[q][j] for q < nrows is entry (rows[q], j). Lets a test check sampled
 * outputs of a full-size matrix without forming all of it.
 */
void oracle_cov_rows(int n, int m, const double *X, int corr, int nrows, const int *rows, double *out) {
    double *mean = (double *)malloc(sizeof(double) * (size_t)m + 1);
    double *ss = (double *)malloc(sizeof(double) * (size_t)m + 1);
    oracle_col_stats(n, m, X, mean, ss);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < nrows; ++q) {
        const int i = rows[q];
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int r = 0; r < n; ++r)
                acc += (X[(size_t)r * m + i] - mean[i]) * (X[(size_t)r * m + j] - mean[j]);
            double v;
            if (!corr) v = acc / (double)(n - 1);
            else if (i == j) v = 1.0;
            else if (ss[i] > 0.0 && ss[j] > 0.0) v = acc / (sqrt(ss[i]) * sqrt(ss[j]));
            else v = 0.0;
            out[(size_t)q * m + j] = v;
        }
    }
    free(mean);
    free(ss);
}

/*
 * Gram-Schmidt QR (polybench gramschmidt, paper Sec. VIII; the kernel whose
 * candidate loop sits in a divergent region, Sec. VI-C and Sec. VIII). For
 * the m x n matrix A, modified Gram-Schmidt one column at a time, with W a
 * working copy of A that is overwritten as in the benchmark:
 *   for k = 0 .. n-1:
 *     R[k][k] = sqrt(sum_i W[i][k]^2)
 *     Q[i][k] = W[i][k] / R[k][k]
 *     for j = k+1 .. n-1:
 *       R[k][j] = sum_i Q[i][k] * W[i][j]
 *       W[i][j] = W[i][j] - Q[i][k] * R[k][j]
 * Q is m x n, R is n x n with its strictly lower triangle set to zero.
 * Reading where the benchmark would divide by zero: a column whose norm is
 * exactly zero gets R[k][k] = 0 and a zero column of Q (so R[k][j] = 0 for
 * j > k and the later columns are left as they are).
 */
void oracle_gramschmidt(int m, int n, const double *A, double *Q, double *R) {
    double *W = (double *)malloc(sizeof(double) * (size_t)m * n + 1);
    memcpy(W, A, sizeof(double) * (size_t)m * n);
    memset(R, 0, sizeof(double) * (size_t)n * n);
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += W[(size_t)i * n + k] * W[(size_t)i * n + k];
        const double rkk = sqrt(nrm);
        R[(size_t)k * n + k] = rkk;
        for (int i = 0; i < m; ++i) Q[(size_t)i * n + k] = rkk > 0.0 ? W[(size_t)i * n + k] / rkk : 0.0;
#pragma omp parallel for schedule(static)
        for (int j = k + 1; j < n; ++j) {
            double acc = 0.0;
            for (int i = 0; i < m; ++i) acc += Q[(size_t)i * n + k] * W[(size_t)i * n + j];
            R[(size_t)k * n + j] = acc;
            for (int i = 0; i < m; ++i) W[(size_t)i * n + j] -= Q[(size_t)i * n + k] * acc;
        }
    }
    free(W);
}
