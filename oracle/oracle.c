/*
 * CPU oracle, plain C, FP64.  TEST INFRASTRUCTURE ONLY: imported by tests/, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline leg; never by the product path.
 *
 *  fo_spmm    Y = A X for a 0/1 pattern CSR A (the paper's SpMM, Section 3.3: every
 *             non-zero adds one row of the dense input to one row of the output).  The plain
 *             definition: rows in order, non-zeros of a row in stored order, FP64 accumulate.
 *             OpenMP splits rows between threads, which does not change any row's arithmetic.
 *  fo_jacobi  eigen-decomposition of a small dense symmetric matrix by the cyclic-by-row
 *             Jacobi method (Golub & Van Loan, Matrix Computations, Section 8.5: the 2x2
 *             symmetric Schur decomposition and the cyclic sweep).  It solves the projected
 *             m x m problem of Algorithm 1 step (2), which the paper hands to LAPACK.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Y[i, :] = sum_{p = rowptr[i]}^{rowptr[i+1]-1} X[colidx[p], :], row-major n x b. */
void fo_spmm(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* X, int b,
             double* Y) {
  #pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    double acc[64];
    for (int c = 0; c < b; ++c) acc[c] = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const double* x = X + (int64_t)colidx[p] * b;
      for (int c = 0; c < b; ++c) acc[c] += x[c];
    }
    for (int c = 0; c < b; ++c) Y[i * b + c] = acc[c];
  }
}

/* Same, for a sampled set of rows: Y[t, :] = (A X)[rows[t], :]. */
void fo_spmm_rows(const int64_t* rowptr, const int32_t* colidx, const double* X, int b,
                  int64_t nrows, const int64_t* rows, double* Y) {
  #pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < nrows; ++t) {
    int64_t i = rows[t];
    double acc[64];
    for (int c = 0; c < b; ++c) acc[c] = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const double* x = X + (int64_t)colidx[p] * b;
      for (int c = 0; c < b; ++c) acc[c] += x[c];
    }
    for (int c = 0; c < b; ++c) Y[t * b + c] = acc[c];
  }
}

static double off_norm(int m, const double* A) {
  double s = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      if (i != j) s += A[i * m + j] * A[i * m + j];
  return sqrt(s);
}

/*
 * A (m x m, row-major, symmetric) is overwritten; on return evals[i] = A[i][i] and column i
 * of V (row-major m x m) is the matching unit eigenvector.  Sweeps until off(A) <= tol*||A||_F
 * or max_sweeps.  Returns the number of sweeps, or -1 if it did not converge.
 */
int fo_jacobi(int m, double* A, double* evals, double* V, double tol, int max_sweeps) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < m * m; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  int sweep = 0;
  int ok = 0;
  while (sweep <= max_sweeps) {
    if (off_norm(m, A) <= tol * fro) { ok = 1; break; }
    if (sweep == max_sweeps) break;
    ++sweep;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        double apq = A[p * m + q];
        if (apq == 0.0) continue;
        /* 2x2 symmetric Schur decomposition: choose (c, s) so that the rotated (p, q)
         * entry vanishes; t is the smaller root of t^2 + 2 tau t - 1 = 0. */
        double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        /* A <- J^T A J with J = identity except J[p][p]=c, J[p][q]=s, J[q][p]=-s, J[q][q]=c */
        for (int k = 0; k < m; ++k) {  /* columns p, q */
          double akp = A[k * m + p], akq = A[k * m + q];
          A[k * m + p] = c * akp - s * akq;
          A[k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  /* rows p, q */
          double apk = A[p * m + k], aqk = A[q * m + k];
          A[p * m + k] = c * apk - s * aqk;
          A[q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {  /* V <- V J */
          double vkp = V[k * m + p], vkq = V[k * m + q];
          V[k * m + p] = c * vkp - s * vkq;
          V[k * m + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < m; ++i) evals[i] = A[i * m + i];
  return ok ? sweep : -1;
}
