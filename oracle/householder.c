/*
 * CPU oracle (test infrastructure only): plain FP64 Householder QR least squares.
 *
 * This file is the oracle's statement of the direct least-squares method of
 * Sec. 2.2 (Alg. 1: QR factorization, b <- Q^T b, x = R^{-1} b) for
 * min ||Ax - b||_2 (Eq. opt:lls), written for clarity rather than speed:
 * unblocked Householder reflections, one column at a time. It shares no code
 * with the GPU library. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.
 *
 * Storage: column-major, leading dimension lda >= m. All arithmetic FP64.
 * The trailing-column loop of each reflector application is split across
 * OpenMP threads; every column's arithmetic is independent and in a fixed
 * order, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define COL(A, lda, j) ((A) + (size_t)(j) * (size_t)(lda))

/* Householder QR in place (Sec. 2.2, Alg. 1 step "qr(A)").
 * On return the upper triangle of A holds R, the entries below the diagonal of
 * column k hold the reflector v_k (v_k[k] = 1 implicit), tau[k] its scale, so
 * that H_k = I - tau_k v_k v_k^T and Q = H_0 H_1 ... H_{n-1}.
 * Returns 0, or -1 for bad sizes. */
int oracle_householder_qr(int m, int n, double* A, int lda, double* tau)
{
    if (m < 1 || n < 1 || n > m || lda < m) return -1;
    for (int k = 0; k < n; ++k) {
        double* a = COL(A, lda, k);
        double alpha = a[k];
        double sigma = 0.0;
        for (int i = k + 1; i < m; ++i) sigma += a[i] * a[i];
        if (sigma == 0.0) {            /* column already upper triangular */
            tau[k] = 0.0;
            continue;
        }
        double norm = sqrt(alpha * alpha + sigma);
        double beta = (alpha <= 0.0) ? norm : -norm;   /* -sign(alpha)*||a||, no cancellation */
        double v0 = alpha - beta;
        for (int i = k + 1; i < m; ++i) a[i] /= v0;
        tau[k] = (beta - alpha) / beta;
        a[k] = beta;
        const double t = tau[k];
        #pragma omp parallel for schedule(static)
        for (int j = k + 1; j < n; ++j) {
            double* c = COL(A, lda, j);
            double w = c[k];
            for (int i = k + 1; i < m; ++i) w += a[i] * c[i];
            w *= t;
            c[k] -= w;
            for (int i = k + 1; i < m; ++i) c[i] -= w * a[i];
        }
    }
    return 0;
}

/* y <- Q^T y for the factored form above (Alg. 1 step "b = Q'*b"). */
void oracle_apply_qt(int m, int n, const double* QR, int lda, const double* tau, double* y)
{
    for (int k = 0; k < n; ++k) {
        if (tau[k] == 0.0) continue;
        const double* v = COL(QR, lda, k);
        double w = y[k];
        for (int i = k + 1; i < m; ++i) w += v[i] * y[i];
        w *= tau[k];
        y[k] -= w;
        for (int i = k + 1; i < m; ++i) y[i] -= w * v[i];
    }
}

/* Explicit m x n Q (ldq >= m) from the factored form: Q = H_0 ... H_{n-1} I[:, :n]. */
void oracle_form_q(int m, int n, const double* QR, int lda, const double* tau, double* Q, int ldq)
{
    for (int j = 0; j < n; ++j) {
        double* q = COL(Q, ldq, j);
        memset(q, 0, sizeof(double) * (size_t)m);
        q[j] = 1.0;
    }
    for (int k = n - 1; k >= 0; --k) {
        if (tau[k] == 0.0) continue;
        const double* v = COL(QR, lda, k);
        const double t = tau[k];
        #pragma omp parallel for schedule(static)
        for (int j = k; j < n; ++j) {
            double* c = COL(Q, ldq, j);
            double w = c[k];
            for (int i = k + 1; i < m; ++i) w += v[i] * c[i];
            w *= t;
            c[k] -= w;
            for (int i = k + 1; i < m; ++i) c[i] -= w * v[i];
        }
    }
}

/* Solve R x = y by back substitution (Alg. 1 step "x = inv(R)*b"); R is the
 * upper triangle of the n x n leading block of QR. Returns -2 if a diagonal
 * entry is zero. */
int oracle_back_substitute(int n, const double* QR, int lda, const double* y, double* x)
{
    for (int k = n - 1; k >= 0; --k) {
        double s = y[k];
        for (int j = k + 1; j < n; ++j) s -= COL(QR, lda, j)[k] * x[j];
        double d = COL(QR, lda, k)[k];
        if (d == 0.0) return -2;
        x[k] = s / d;
    }
    return 0;
}

/* Whole direct solve of Alg. 1 on a private copy: x = argmin ||A x - b||.
 * A: m x n FP64 column-major (lda), b: m, x: n. Returns 0, -1 (args), -2 (singular R). */
int oracle_lls(int m, int n, const double* A, int lda, const double* b, double* x)
{
    if (m < 1 || n < 1 || n > m || lda < m) return -1;
    double* W = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* tau = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)m);
    if (!W || !tau || !y) { free(W); free(tau); free(y); return -1; }
    for (int j = 0; j < n; ++j) memcpy(COL(W, m, j), COL(A, lda, j), sizeof(double) * (size_t)m);
    memcpy(y, b, sizeof(double) * (size_t)m);
    int rc = oracle_householder_qr(m, n, W, m, tau);
    if (rc == 0) {
        oracle_apply_qt(m, n, W, m, tau, y);
        rc = oracle_back_substitute(n, W, m, y, x);
    }
    free(W); free(tau); free(y);
    return rc;
}

/* ---- error-free transformations (Knuth TwoSum, Dekker/FMA TwoProduct) ---- */
static inline void two_sum(double a, double b, double* s, double* e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static inline void two_prod(double a, double b, double* p, double* e)
{
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

/* r = b - A x with A given in FP32, computed with the compensated dot product
 * (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005, Dot2), i.e. as
 * if in twice FP64 precision and rounded once. Used to evaluate residuals of
 * nearly compatible systems without the FP64 cancellation floor. */
void oracle_residual_f32(int m, int n, const float* A, int lda, const double* x,
                         const double* b, double* r)
{
    double* c = (double*)calloc((size_t)m, sizeof(double));
    for (int i = 0; i < m; ++i) r[i] = b[i];
    for (int j = 0; j < n; ++j) {
        const float* a = A + (size_t)j * (size_t)lda;
        const double xj = x[j];
        for (int i = 0; i < m; ++i) {
            double p, e1, s, e2;
            two_prod(-(double)a[i], xj, &p, &e1);
            two_sum(r[i], p, &s, &e2);
            r[i] = s;
            c[i] += e1 + e2;
        }
    }
    for (int i = 0; i < m; ++i) r[i] += c[i];
    free(c);
}

/* u = A^T r for FP32 A with the same compensated dot product. */
void oracle_atr_f32(int m, int n, const float* A, int lda, const double* r, double* u)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
        const float* a = A + (size_t)j * (size_t)lda;
        double s = 0.0, c = 0.0;
        for (int i = 0; i < m; ++i) {
            double p, e1, e2;
            two_prod((double)a[i], r[i], &p, &e1);
            two_sum(s, p, &s, &e2);
            c += e1 + e2;
        }
        u[j] = s + c;
    }
}
