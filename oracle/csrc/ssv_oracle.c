/*
 * CPU oracle for the shifted m-Hessenberg solver (Bosner, Bujanovic, Drmac,
 * "Parallel solver for shifted systems in a hybrid CPU-GPU framework").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * Everything is IEEE double / double complex, column-major unless stated.
 * Parallel loops (OpenMP) only split independent work (columns of an update,
 * independent shifts); no blocking, fusion or reordering of the arithmetic.
 *
 * Functions:
 *   ora_dense_solve   : X = (A - sigma I)^{-1} B by LU with partial pivoting on
 *                       the full matrix A - sigma I (the plain definition of the
 *                       solve of Sec. 1, eq. for (A - sigma I)X = B).
 *   ora_dense_solve_vec: one right-hand side per shift, x = (A - sigma I)^{-1} b
 *                       or, transposed, x = (A - sigma I)^{-T} c (plain
 *                       transpose, not conjugate): the systems with different
 *                       right-hand sides for different shifts of Sec. 3.3,
 *                       b = B bhat, c = C^T chat.  Same LU as ora_dense_solve.
 *   ora_reduce        : controller-Hessenberg form of (A, B, C) by unblocked
 *                       Householder reflectors, following Algorithm 1 (Sec. 2):
 *                       QR of B, similarity with Q_B, m-Hessenberg reduction,
 *                       C <- C Q.  Optionally accumulates Q.
 *   ora_reduced_solve : Xhat = (H - sigma I)^{-1} R in reduced coordinates by
 *                       Gaussian elimination with partial pivoting (rows) that
 *                       skips the structural zeros of the m-Hessenberg H; the
 *                       "tier 2" oracle.  Optionally G = Ct Xhat and a Hager
 *                       estimate of the 1-norm condition number of H - sigma I.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

#define ORA_OK 0
#define ORA_SINGULAR 1

static double cabs1(zc z) { return fabs(creal(z)) + fabs(cimag(z)); }

/* ------------------------------------------------------------------------ */
/* Dense complex LU with partial pivoting, in place (column-major, ld = n).   */
/* Returns 0, or k+1 if the k-th pivot is exactly zero (factorization stops). */
/* Pivot = largest |re|+|im| in the column, lowest row index on ties.        */
/* ------------------------------------------------------------------------ */
static int zgetrf_plain(int n, zc* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = cabs1(a[k + (size_t)k * n]);
    for (int i = k + 1; i < n; ++i) {
      double v = cabs1(a[i + (size_t)k * n]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        zc t = a[k + (size_t)j * n];
        a[k + (size_t)j * n] = a[p + (size_t)j * n];
        a[p + (size_t)j * n] = t;
      }
    }
    zc d = a[k + (size_t)k * n];
    for (int i = k + 1; i < n; ++i) a[i + (size_t)k * n] /= d;
    /* rank-1 update of the trailing block, one column at a time */
#pragma omp parallel for schedule(static) if (n - k > 256)
    for (int j = k + 1; j < n; ++j) {
      zc akj = a[k + (size_t)j * n];
      if (akj != 0) {
        zc* colj = a + (size_t)j * n;
        const zc* colk = a + (size_t)k * n;
        for (int i = k + 1; i < n; ++i) colj[i] -= colk[i] * akj;
      }
    }
  }
  return 0;
}

/* Solve with the factors: b (n x nrhs, ld = n) overwritten by the solution. */
static void zgetrs_plain(int n, const zc* a, const int* piv, int nrhs, zc* b) {
  for (int r = 0; r < nrhs; ++r) {
    zc* x = b + (size_t)r * n;
    for (int k = 0; k < n; ++k) {
      if (piv[k] != k) { zc t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    }
    for (int k = 0; k < n; ++k)            /* L y = P b, unit lower */
      for (int i = k + 1; i < n; ++i) x[i] -= a[i + (size_t)k * n] * x[k];
    for (int k = n - 1; k >= 0; --k) {     /* U x = y */
      x[k] /= a[k + (size_t)k * n];
      for (int i = 0; i < k; ++i) x[i] -= a[i + (size_t)k * n] * x[k];
    }
  }
}

/*
 * X(:, :, j) = (A - sigma_j I)^{-1} B for j = 0..ns-1.
 * A n x n real (lda), B n x m real (ldb), sigma ns complex, X n x m x ns
 * complex (column-major, X + j*n*m), status[j] = 0 or 1 (exact zero pivot).
 */
int ora_dense_solve(int n, int m, const double* A, int lda, const double* B, int ldb, int ns,
                    const zc* sigma, zc* X, int* status) {
  zc* M = (zc*)malloc(sizeof(zc) * (size_t)n * n);
  int* piv = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!M || !piv) { free(M); free(piv); return -1; }
  for (int s = 0; s < ns; ++s) {
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) M[i + (size_t)j * n] = A[i + (size_t)j * lda];
    for (int i = 0; i < n; ++i) M[i + (size_t)i * n] -= sigma[s];
    zc* Xs = X + (size_t)s * n * m;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < n; ++i) Xs[i + (size_t)j * n] = B[i + (size_t)j * ldb];
    int info = zgetrf_plain(n, M, piv);
    if (info) {
      status[s] = ORA_SINGULAR;
      for (size_t t = 0; t < (size_t)n * m; ++t) Xs[t] = NAN;
      continue;
    }
    zgetrs_plain(n, M, piv, m, Xs);
    status[s] = ORA_OK;
  }
  free(M);
  free(piv);
  return 0;
}

/* One complex right-hand side per shift: column s of rhs (ld ldr) solved with
 * M = A - sigma_s I (trans = 0) or M = (A - sigma_s I)^T (trans = 1) into
 * column s of X (ld n).  status[s] = ORA_SINGULAR on an exactly zero pivot. */
int ora_dense_solve_vec(int n, const double* A, int lda, int ns, const zc* sigma, int trans,
                        const zc* rhs, int ldr, zc* X, int* status) {
  zc* M = (zc*)malloc(sizeof(zc) * (size_t)n * n);
  int* piv = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!M || !piv) { free(M); free(piv); return -1; }
  for (int s = 0; s < ns; ++s) {
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        M[i + (size_t)j * n] = trans ? A[j + (size_t)i * lda] : A[i + (size_t)j * lda];
    for (int i = 0; i < n; ++i) M[i + (size_t)i * n] -= sigma[s];
    zc* xs = X + (size_t)s * n;
    for (int i = 0; i < n; ++i) xs[i] = rhs[i + (size_t)s * ldr];
    int info = zgetrf_plain(n, M, piv);
    if (info) {
      status[s] = ORA_SINGULAR;
      for (int i = 0; i < n; ++i) xs[i] = NAN;
      continue;
    }
    zgetrs_plain(n, M, piv, 1, xs);
    status[s] = ORA_OK;
  }
  free(M);
  free(piv);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Householder reflector (LAPACK dlarfg convention, written out):            */
/*   given x = [alpha; x2] (length len), find beta, tau, v = [1; v2] with    */
/*   (I - tau v v^T) x = [beta; 0],  beta = -sign(alpha) ||x||.              */
/* x is overwritten by [beta; v2].  Returns tau (0 if x2 == 0).             */
/* ------------------------------------------------------------------------ */
static double house(int len, double* x, int incx) {
  if (len <= 1) return 0.0;
  double alpha = x[0];
  double ss = 0.0;
  for (int i = 1; i < len; ++i) ss += x[(size_t)i * incx] * x[(size_t)i * incx];
  if (ss == 0.0) return 0.0;
  double nrm = sqrt(alpha * alpha + ss);
  double beta = alpha >= 0.0 ? -nrm : nrm;
  double tau = (beta - alpha) / beta;
  double scal = 1.0 / (alpha - beta);
  for (int i = 1; i < len; ++i) x[(size_t)i * incx] *= scal;
  x[0] = beta;
  return tau;
}

/* Apply H = I - tau v v^T from the left to rows r0..r0+len-1 of the
 * columns c0..c1-1 of a (ld), v[0] = 1 implied by the caller's copy. */
static void apply_left(double* a, int ld, int r0, int len, int c0, int c1, const double* v,
                       double tau) {
  if (tau == 0.0) return;
#pragma omp parallel for schedule(static) if ((size_t)(c1 - c0) * len > 65536)
  for (int j = c0; j < c1; ++j) {
    double* col = a + (size_t)j * ld + r0;
    double w = 0.0;
    for (int i = 0; i < len; ++i) w += v[i] * col[i];
    w *= tau;
    for (int i = 0; i < len; ++i) col[i] -= v[i] * w;
  }
}

/* Apply H = I - tau v v^T from the right to rows 0..nr-1 and columns
 * c0..c0+len-1 of a (ld):  w = a(:, c0:) v  (w_i accumulated over j in
 * ascending order), then a(:, c0+j) -= tau * v_j * w.  Rows are split into
 * contiguous chunks across threads; each row's arithmetic is unchanged. */
static void apply_right(double* a, int ld, int nr, int c0, int len, const double* v, double tau) {
  if (tau == 0.0 || nr <= 0) return;
  int nchunk = (nr + 255) / 256;
#pragma omp parallel for schedule(static) if ((size_t)nr * len > 65536)
  for (int ch = 0; ch < nchunk; ++ch) {
    int i0 = ch * 256, i1 = i0 + 256 < nr ? i0 + 256 : nr;
    double w[256];
    for (int i = i0; i < i1; ++i) w[i - i0] = 0.0;
    for (int j = 0; j < len; ++j) {
      const double* col = a + (size_t)(c0 + j) * ld;
      double vj = v[j];
      for (int i = i0; i < i1; ++i) w[i - i0] += col[i] * vj;
    }
    for (int i = i0; i < i1; ++i) w[i - i0] *= tau;
    for (int j = 0; j < len; ++j) {
      double* col = a + (size_t)(c0 + j) * ld;
      double vj = v[j];
      for (int i = i0; i < i1; ++i) col[i] -= w[i - i0] * vj;
    }
  }
}

/*
 * Controller-Hessenberg reduction (Algorithm 1, Sec. 2), unblocked.
 *   In : A n x n (lda), B n x m (ldb), C p x n (ldc), all real.
 *   Out: H n x n (ld n)   = Q^T A Q, zero below the m-th subdiagonal (stored 0)
 *        R n x m (ld n)   = Q^T B, zero below the diagonal (stored 0)
 *        Ct p x n (ld p)  = C Q
 *        Q n x n (ld n)   = Q_B Q_A if Q != NULL.
 * Step 1: QR of B by Householder reflectors on columns i = 0..min(m, n-1)-1,
 *         each acting on rows i..n-1.
 * Step 2: each reflector is applied to A from both sides and to C.
 * Step 3: for column j = 0..n-m-2, a reflector acting on rows j+m..n-1
 *         annihilates A(j+m+1 : n-1, j); applied from the left to the
 *         trailing columns, from the right to all rows, and to C.
 */
int ora_reduce(int n, int m, int p, const double* A, int lda, const double* B, int ldb,
               const double* C, int ldc, double* H, double* R, double* Ct, double* Q) {
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!v) return -1;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) H[i + (size_t)j * n] = A[i + (size_t)j * lda];
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < n; ++i) R[i + (size_t)j * n] = B[i + (size_t)j * ldb];
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < p; ++i) Ct[i + (size_t)j * p] = C[i + (size_t)j * ldc];
  if (Q) {
    memset(Q, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) Q[i + (size_t)i * n] = 1.0;
  }

  /* Step 1 + 2: QR of B; each reflector applied to R, A (both sides), C, Q. */
  int kb = m < n - 1 ? m : n - 1;
  for (int i = 0; i < kb; ++i) {
    int len = n - i;
    double* x = R + i + (size_t)i * n;
    double tau = house(len, x, 1);
    v[0] = 1.0;
    for (int t = 1; t < len; ++t) v[t] = x[t];
    for (int t = 1; t < len; ++t) x[t] = 0.0;               /* R(i+1:n, i) = 0 */
    apply_left(R, n, i, len, i + 1, m, v, tau);              /* rest of B */
    apply_left(H, n, i, len, 0, n, v, tau);                  /* A <- H_i A */
    apply_right(H, n, n, i, len, v, tau);                    /* A <- A H_i */
    apply_right(Ct, p, p, i, len, v, tau);                   /* C <- C H_i */
    if (Q) apply_right(Q, n, n, i, len, v, tau);             /* Q <- Q H_i */
  }

  /* Step 3 + 4: m-Hessenberg reduction of A, C updated alongside. */
  for (int j = 0; j + m + 1 < n; ++j) {
    int r0 = j + m, len = n - r0;
    double* x = H + r0 + (size_t)j * n;
    double tau = house(len, x, 1);
    v[0] = 1.0;
    for (int t = 1; t < len; ++t) v[t] = x[t];
    for (int t = 1; t < len; ++t) x[t] = 0.0;               /* H(j+m+1:n, j) = 0 */
    apply_left(H, n, r0, len, j + 1, n, v, tau);
    apply_right(H, n, n, r0, len, v, tau);
    apply_right(Ct, p, p, r0, len, v, tau);
    if (Q) apply_right(Q, n, n, r0, len, v, tau);
  }
  free(v);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tier-2: (H - sigma I) Xhat = R by Gaussian elimination with row partial   */
/* pivoting.  Column k of an upper m-Hessenberg matrix is nonzero only in    */
/* rows <= k+m, and row interchanges among rows k..k+m keep that property    */
/* for the columns to the right, so row k's elimination touches rows         */
/* k+1..min(k+m, n-1) only.  U is kept row-major (row k = entries k..n-1).  */
/* ------------------------------------------------------------------------ */

/* Solve U x = y (upper triangular, row-major, ld n) in place. */
static void utri_solve(int n, const zc* U, zc* x) {
  for (int k = n - 1; k >= 0; --k) {
    zc s = x[k];
    const zc* row = U + (size_t)k * n;
    for (int j = k + 1; j < n; ++j) s -= row[j] * x[j];
    x[k] = s / row[k];
  }
}

/* Solve U^H x = y in place. */
static void utri_solve_h(int n, const zc* U, zc* x) {
  for (int k = 0; k < n; ++k) {
    x[k] /= conj(U[(size_t)k * n + k]);
    const zc* row = U + (size_t)k * n;
    for (int j = k + 1; j < n; ++j) x[j] -= conj(row[j]) * x[k];
  }
}

/*
 * For every shift: factor P (H - sigma I) = L U with band-limited elimination,
 * then Xhat = U^{-1} L^{-1} P R.
 *   mode 0: out = Xhat (n x m per shift, ld n, shift s at out + s*n*m)
 *   mode 1: out = G = Ct Xhat (p x m per shift, ld p, at out + s*p*m)
 *   cond1 (may be NULL): Hager's estimate of ||(H - sigma I)^{-1}||_1 times
 *   ||H - sigma I||_1 (Hager 1984, as refined by Higham 1988: alternate
 *   solves with M and M^H starting from the all-ones/n vector, at most 5
 *   iterations).
 */
int ora_reduced_solve(int n, int m, int p, const double* H, int ldh, const double* R, int ldr,
                      const double* Ct, int ldc, int ns, const zc* sigma, int mode, zc* out,
                      int* status, double* cond1) {
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < ns; ++s) {
    zc* U = (zc*)malloc(sizeof(zc) * (size_t)n * n);
    zc* Lm = (zc*)malloc(sizeof(zc) * (size_t)n * (m + 1)); /* multipliers per row k */
    int* piv = (int*)malloc(sizeof(int) * (size_t)n);
    zc* X = (zc*)malloc(sizeof(zc) * (size_t)n * m);
    zc* w = (zc*)malloc(sizeof(zc) * (size_t)n);
    if (!U || !Lm || !piv || !X || !w) {
      free(U); free(Lm); free(piv); free(X); free(w);
#pragma omp atomic write
      fail = 1;
      continue;
    }
    /* U := H - sigma I, row-major */
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) U[(size_t)i * n + j] = H[i + (size_t)j * ldh];
    for (int i = 0; i < n; ++i) U[(size_t)i * n + i] -= sigma[s];
    double anorm = 0.0;
    for (int j = 0; j < n; ++j) {
      double cs = 0.0;
      for (int i = 0; i < n; ++i) cs += cabs(U[(size_t)i * n + j]);
      if (cs > anorm) anorm = cs;
    }
    int singular = 0;
    for (int k = 0; k < n; ++k) {
      int last = k + m < n - 1 ? k + m : n - 1;
      int pr = k;
      double best = cabs1(U[(size_t)k * n + k]);
      for (int i = k + 1; i <= last; ++i) {
        double v = cabs1(U[(size_t)i * n + k]);
        if (v > best) { best = v; pr = i; }
      }
      piv[k] = pr;
      if (best == 0.0) { singular = 1; break; }
      if (pr != k)
        for (int j = k; j < n; ++j) {
          zc t = U[(size_t)k * n + j];
          U[(size_t)k * n + j] = U[(size_t)pr * n + j];
          U[(size_t)pr * n + j] = t;
        }
      zc d = U[(size_t)k * n + k];
      for (int i = k + 1; i <= last; ++i) {
        zc l = U[(size_t)i * n + k] / d;
        Lm[(size_t)k * (m + 1) + (i - k)] = l;
        U[(size_t)i * n + k] = 0.0;
        for (int j = k + 1; j < n; ++j) U[(size_t)i * n + j] -= l * U[(size_t)k * n + j];
      }
    }
    if (singular) {
      status[s] = ORA_SINGULAR;
      size_t cnt = mode == 0 ? (size_t)n * m : (size_t)p * m;
      zc* o = out + (size_t)s * cnt;
      for (size_t t = 0; t < cnt; ++t) o[t] = NAN;
      if (cond1) cond1[s] = INFINITY;
    } else {
      status[s] = ORA_OK;
      for (int j = 0; j < m; ++j) {
        zc* x = X + (size_t)j * n;
        for (int i = 0; i < n; ++i) x[i] = R[i + (size_t)j * ldr];
        for (int k = 0; k < n; ++k) {             /* apply P and L^{-1} */
          int last = k + m < n - 1 ? k + m : n - 1;
          if (piv[k] != k) { zc t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
          for (int i = k + 1; i <= last; ++i) x[i] -= Lm[(size_t)k * (m + 1) + (i - k)] * x[k];
        }
        utri_solve(n, U, x);
      }
      if (mode == 0) {
        memcpy(out + (size_t)s * n * m, X, sizeof(zc) * (size_t)n * m);
      } else {
        zc* G = out + (size_t)s * p * m;
        for (int j = 0; j < m; ++j)
          for (int i = 0; i < p; ++i) {
            zc acc = 0.0;
            for (int k = 0; k < n; ++k) acc += Ct[i + (size_t)k * ldc] * X[k + (size_t)j * n];
            G[i + (size_t)j * p] = acc;
          }
      }
      if (cond1) {
        /* Hager / Higham 1-norm estimator of ||M^{-1}||_1. */
        for (int i = 0; i < n; ++i) w[i] = 1.0 / n;
        double est = 0.0;
        int jlast = -1;
        for (int it = 0; it < 5; ++it) {
          /* y = M^{-1} w */
          for (int k = 0; k < n; ++k) {
            int last = k + m < n - 1 ? k + m : n - 1;
            if (piv[k] != k) { zc t = w[k]; w[k] = w[piv[k]]; w[piv[k]] = t; }
            for (int i = k + 1; i <= last; ++i) w[i] -= Lm[(size_t)k * (m + 1) + (i - k)] * w[k];
          }
          utri_solve(n, U, w);
          double ynorm = 0.0;
          for (int i = 0; i < n; ++i) ynorm += cabs(w[i]);
          if (it > 0 && ynorm <= est) break;
          est = ynorm;
          /* xi = sign(y); z = M^{-H} xi */
          for (int i = 0; i < n; ++i) {
            double a = cabs(w[i]);
            w[i] = a > 0 ? w[i] / a : 1.0;
          }
          utri_solve_h(n, U, w);
          for (int k = n - 1; k >= 0; --k) {       /* L^{-H} then P^T */
            int last = k + m < n - 1 ? k + m : n - 1;
            for (int i = k + 1; i <= last; ++i) w[k] -= conj(Lm[(size_t)k * (m + 1) + (i - k)]) * w[i];
            if (piv[k] != k) { zc t = w[k]; w[k] = w[piv[k]]; w[piv[k]] = t; }
          }
          int jmax = 0;
          double zmax = -1.0;
          for (int i = 0; i < n; ++i)
            if (cabs(w[i]) > zmax) { zmax = cabs(w[i]); jmax = i; }
          if (jmax == jlast) break;
          jlast = jmax;
          for (int i = 0; i < n; ++i) w[i] = 0.0;
          w[jmax] = 1.0;
        }
        cond1[s] = est * anorm;
      }
    }
    free(U); free(Lm); free(piv); free(X); free(w);
  }
  return fail ? -1 : 0;
}
