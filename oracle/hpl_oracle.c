/*
 * hpl_oracle.c -- plain, slow, obviously correct CPU oracle for the HPL hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker that the CUDA library is
 * compared against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the library's compute path never does.  It
 * shares no code, header, table or helper with the CUDA sources.
 *
 * Method (paper: "Optimizing High-Performance Linpack for Exascale Accelerated
 * Architectures", rocHPL):
 *   Sec. II   -- a random N x N FP64 system A x = b (b appended as column N of an
 *                augmented system) is solved by Gaussian elimination with partial
 *                pivoting, A = P L U, followed by the triangular solves.
 *   Sec. I    -- FACT picks, per column, the pivot row of largest magnitude;
 *                RS applies the pivots to the rest of the matrix; UPDATE is the
 *                triangular solve (DTRSM) and the rank-NB Schur update (DGEMM).
 * A blocked, right-looking schedule of those phases reaches the same factors as
 * the unblocked right-looking elimination below, up to rounding order; the
 * oracle therefore is that unblocked elimination, written out.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - generator: 64-bit LCG s' = a s + c (mod 2^64), Knuth's MMIX constants;
 *     element t = i + j*N of A, t = N*N + i of b; value = (s_{t+1} >> 11) 2^-53 - 1/2.
 *   - pivot ties go to the smallest row index (strict '>' while scanning down).
 *   - zero pivot: LAPACK info convention (first zero pivot, 1-based), continue.
 *   - residual: ||Ax-b||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) N), eps = 2^-53.
 *   - LAPACK row-interchange convention: swaps run across all N columns.
 *
 * Compiled with -ffp-contract=off so that every product and sum is rounded as
 * written (fma() is used only where it is called by name, for exact products).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LCG_A 6364136223846793005ULL
#define ORC_LCG_C 1442695040888963407ULL

/* ---------------------------------------------------------------- generator */

/* One LCG step. */
static inline uint64_t orc_step(uint64_t s) { return ORC_LCG_A * s + ORC_LCG_C; }

/* Map a 64-bit state to a double in [-0.5, 0.5): top 53 bits scaled by 2^-53,
 * minus one half.  Both operations are exact in FP64. */
double orc_value(uint64_t s) { return (double)(s >> 11) * 0x1p-53 - 0.5; }

/* State after t steps from seed, by composing the affine map x -> a x + c with
 * itself (repeated squaring; Brown 1994, "Random number generation with
 * arbitrary strides").  (A1,C1) is the map for 2^k steps, (A,C) the
 * accumulated map. */
uint64_t orc_lcg_skip(uint64_t seed, uint64_t t) {
  uint64_t A = 1, C = 0, A1 = ORC_LCG_A, C1 = ORC_LCG_C;
  while (t) {
    if (t & 1) { A = A1 * A; C = A1 * C + C1; }
    C1 = A1 * C1 + C1;
    A1 = A1 * A1;
    t >>= 1;
  }
  return A * seed + C;
}

/* The random system of Sec. II: A(i,j) for i,j < n in column-major order, then
 * b(i) as column n of the augmented system.  Plain sequential stepping. */
void orc_generate(int64_t n, uint64_t seed, double* A, int64_t lda, double* b) {
  uint64_t s = seed;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      s = orc_step(s);
      A[i + j * lda] = orc_value(s);
    }
  for (int64_t i = 0; i < n; ++i) {
    s = orc_step(s);
    if (b) b[i] = orc_value(s);
  }
}

/* Diagonally dominant variant used by the mixed-precision solve: off-diagonals
 * and b as in orc_generate, then A(i,i) = sum_{j != i} |A(i,j)| accumulated in
 * ascending j with plain FP64 additions (this fixed order defines the value). */
void orc_generate_dd(int64_t n, uint64_t seed, double* A, int64_t lda, double* b) {
  orc_generate(n, seed, A, lda, b);
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t j = 0; j < n; ++j)
      if (j != i) d = d + fabs(A[i + j * lda]);
    A[i + i * lda] = d;
  }
}

/* ------------------------------------------------------------------- getrf */

/* Unblocked right-looking LU with partial pivoting of an m x n matrix (Sec. I
 * FACT/RS/UPDATE with NB = 1; Sec. II A = P L U).  For j = 0..min(m,n)-1:
 *   p = argmax_{i >= j} |A(i,j)|, first maximum wins (ties -> smallest i);
 *   ipiv[j] = p + 1;
 *   if A(p,j) == 0: record info (first only) and skip the elimination step;
 *   else swap rows j and p across all n columns, divide the subdiagonal of
 *   column j by A(j,j), and subtract A(i,j) A(j,c) from A(i,c) for i, c > j.
 * The square system of the benchmark is m = n; a panel (FACT) is m >= n.
 *
 * Pivot replay: when `replay` is not NULL it holds another factorization's
 * 1-based pivots (an entry 0 means: no replay for that column).  Where
 * replay[j]-1 = g differs from p the replayed row is accepted only if
 * ||A(g,j)| - |A(p,j)|| < rtol * max(|A(g,j)|, |A(p,j)|) (both magnitudes taken
 * from this elimination's step-j values); accepted columns are logged in
 * mism[] and the elimination continues with g, so later steps stay
 * comparable.  A rejected replay stops the elimination and returns -(j+1).
 * Returns 0 otherwise; *info gets the LAPACK singularity code. */
static int getrf_core(int64_t m, int64_t n, int64_t steps, double* A, int64_t lda, int32_t* ipiv,
                      int32_t* info, const int32_t* replay, double rtol, int64_t* mism,
                      int64_t mism_cap, int64_t* n_mism) {
  int32_t inf = 0;
  int64_t nm = 0;
  int64_t kmax = m < n ? m : n;
  if (steps >= 0 && steps < kmax) kmax = steps;
  for (int64_t j = 0; j < kmax; ++j) {
    int64_t p = j;
    double best = fabs(A[j + j * lda]);
    for (int64_t i = j + 1; i < m; ++i) {
      double v = fabs(A[i + j * lda]);
      if (v > best) { best = v; p = i; }
    }
    if (replay && replay[j] != 0) {
      int64_t g = (int64_t)replay[j] - 1;
      if (g != p) {
        if (g < j || g >= m) { *info = inf; if (n_mism) *n_mism = nm; return (int)-(j + 1); }
        double ag = fabs(A[g + j * lda]);
        double mx = ag > best ? ag : best;
        if (!(fabs(ag - best) < rtol * mx)) { *info = inf; if (n_mism) *n_mism = nm; return (int)-(j + 1); }
        if (mism && nm < mism_cap) mism[nm] = j;
        ++nm;
        p = g;
      }
    }
    ipiv[j] = (int32_t)(p + 1);
    if (A[p + j * lda] == 0.0) {
      if (inf == 0) inf = (int32_t)(j + 1);
      continue;
    }
    if (p != j)
      for (int64_t c = 0; c < n; ++c) {
        double t = A[j + c * lda];
        A[j + c * lda] = A[p + c * lda];
        A[p + c * lda] = t;
      }
    double piv = A[j + j * lda];
    for (int64_t i = j + 1; i < m; ++i) A[i + j * lda] = A[i + j * lda] / piv;
    /* rank-1 update; each element is written by one iteration, so the result
     * does not depend on the thread count */
#pragma omp parallel for schedule(static) if ((m - j) * (n - j) > 65536)
    for (int64_t c = j + 1; c < n; ++c) {
      double u = A[j + c * lda];
      for (int64_t i = j + 1; i < m; ++i) A[i + c * lda] = A[i + c * lda] - A[i + j * lda] * u;
    }
  }
  *info = inf;
  if (n_mism) *n_mism = nm;
  return 0;
}

int orc_getrf_mn(int64_t m, int64_t n, double* A, int64_t lda, int32_t* ipiv, int32_t* info,
                 const int32_t* replay, double rtol, int64_t* mism, int64_t mism_cap,
                 int64_t* n_mism) {
  return getrf_core(m, n, -1, A, lda, ipiv, info, replay, rtol, mism, mism_cap, n_mism);
}

/* The first `steps` elimination steps of orc_getrf_mn only (a bounded sample
 * of a factorization, used to time the oracle on systems it cannot finish). */
int orc_getrf_steps(int64_t m, int64_t n, int64_t steps, double* A, int64_t lda, int32_t* ipiv,
                    int32_t* info) {
  return getrf_core(m, n, steps, A, lda, ipiv, info, NULL, 0.0, NULL, 0, NULL);
}

/* Square system (m = n). */
int orc_getrf(int64_t n, double* A, int64_t lda, int32_t* ipiv, int32_t* info,
              const int32_t* replay, double rtol, int64_t* mism, int64_t mism_cap,
              int64_t* n_mism) {
  return orc_getrf_mn(n, n, A, lda, ipiv, info, replay, rtol, mism, mism_cap, n_mism);
}

/* RS of Sec. I: apply the interchanges k = k1..k2-1 (row k <-> row ipiv[k]-1,
 * in increasing k) to the ncols columns of A. */
void orc_laswp(int64_t ncols, double* A, int64_t lda, int64_t k1, int64_t k2, const int32_t* ipiv) {
  for (int64_t k = k1; k < k2; ++k) {
    int64_t p = ipiv[k] - 1;
    if (p == k) continue;
    for (int64_t c = 0; c < ncols; ++c) {
      double t = A[k + c * lda];
      A[k + c * lda] = A[p + c * lda];
      A[p + c * lda] = t;
    }
  }
}

/* DTRSM of the UPDATE phase (Sec. I): B <- L^-1 B with L the unit-lower m x m
 * triangle of A; forward substitution, one column of B at a time. */
void orc_trsm_llnu(int64_t m, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb) {
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < m; ++i) {
      double s = B[i + c * ldb];
      for (int64_t k = 0; k < i; ++k) s = s - A[i + k * lda] * B[k + c * ldb];
      B[i + c * ldb] = s;
    }
}

/* DGEMM of the UPDATE phase (Sec. I): C <- alpha op(A) op(B) + beta C with
 * op(X) = X or X^T; plain triple loop, sum in increasing k; beta = 0 does
 * not read C. */
void orc_gemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  int TA = (ta == 'T' || ta == 't'), TB = (tb == 'T' || tb == 't');
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t q = 0; q < k; ++q) {
        double a = TA ? A[q + i * lda] : A[i + q * lda];
        double b = TB ? B[j + q * ldb] : B[q + j * ldb];
        s = s + a * b;
      }
      C[i + j * ldc] = (beta == 0.0) ? alpha * s : alpha * s + beta * C[i + j * ldc];
    }
}

/* LU without pivoting (the mixed-precision variant factors a diagonally
 * dominant matrix, for which elimination needs no interchanges).  Same update
 * as orc_getrf with p = j.  *info = first zero pivot (1-based), elimination
 * continues past it. */
void orc_getrf_nopiv(int64_t n, double* A, int64_t lda, int32_t* info) {
  int32_t inf = 0;
  for (int64_t j = 0; j < n; ++j) {
    double piv = A[j + j * lda];
    if (piv == 0.0) { if (inf == 0) inf = (int32_t)(j + 1); continue; }
    for (int64_t i = j + 1; i < n; ++i) A[i + j * lda] = A[i + j * lda] / piv;
#pragma omp parallel for schedule(static) if (n - j > 256)
    for (int64_t c = j + 1; c < n; ++c) {
      double u = A[j + c * lda];
      for (int64_t i = j + 1; i < n; ++i) A[i + c * lda] = A[i + c * lda] - A[i + j * lda] * u;
    }
  }
  *info = inf;
}

/* ------------------------------------------------------------------- getrs */

/* Solve with the factors of orc_getrf (Sec. II: U x = L^-1 P^-1 b, then U^-1).
 * trans 'N': B <- A^-1 B: apply the interchanges in order j = 0..n-1, forward
 *            substitution with unit-lower L, backward substitution with U.
 * trans 'T': B <- A^-T B: forward substitution with U^T, backward with unit
 *            L^T, then the interchanges in reverse order j = n-1..0.
 * ipiv may be NULL (no interchanges: factors from orc_getrf_nopiv). */
void orc_getrs(char trans, int64_t n, int64_t nrhs, const double* LU, int64_t lda,
               const int32_t* ipiv, double* B, int64_t ldb) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double* x = B + r * ldb;
    if (trans == 'N' || trans == 'n') {
      if (ipiv)
        for (int64_t j = 0; j < n; ++j) {
          int64_t p = ipiv[j] - 1;
          double t = x[j]; x[j] = x[p]; x[p] = t;
        }
      for (int64_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int64_t k = 0; k < i; ++k) s = s - LU[i + k * lda] * x[k];
        x[i] = s;
      }
      for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s = s - LU[i + k * lda] * x[k];
        x[i] = s / LU[i + i * lda];
      }
    } else {
      /* U^T y = x: row i of U^T is column i of U */
      for (int64_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int64_t k = 0; k < i; ++k) s = s - LU[k + i * lda] * x[k];
        x[i] = s / LU[i + i * lda];
      }
      /* L^T z = y, unit diagonal: row i of L^T is column i of L */
      for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s = s - LU[k + i * lda] * x[k];
        x[i] = s;
      }
      if (ipiv)
        for (int64_t j = n - 1; j >= 0; --j) {
          int64_t p = ipiv[j] - 1;
          double t = x[j]; x[j] = x[p]; x[p] = t;
        }
    }
  }
}

/* ---------------------------------------------------------------- residual */

/* Error-free transformations (Ogita, Rump, Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 2005): TwoSum (Knuth) and TwoProduct via a
 * fused multiply-add.  Dot2 accumulates (hi, lo) so a dot product is computed
 * as if in twice the working precision, which keeps the residual b - Ax
 * accurate although it is of the order of rounding errors. */
static inline void orc_two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static inline void orc_dot2_add(double* hi, double* lo, double a, double x) {
  double p = a * x;
  double pe = fma(a, x, -p);
  double s, se;
  orc_two_sum(*hi, p, &s, &se);
  *hi = s;
  *lo = *lo + (se + pe);
}

static void orc_residual_finish(int64_t n, const double* rhi, const double* rlo,
                                const double* rowabs, const double* x, const double* b,
                                double* out5) {
  double rn = 0, an = 0, xn = 0, bn = 0;
  for (int64_t i = 0; i < n; ++i) {
    double hi = rhi[i], lo = rlo[i];
    double r = hi + lo;
    double ar = fabs(r);
    if (ar > rn || isnan(ar)) rn = ar;
    if (rowabs[i] > an || isnan(rowabs[i])) an = rowabs[i];
    double ax = fabs(x[i]);
    if (ax > xn || isnan(ax)) xn = ax;
    double ab = fabs(b[i]);
    if (ab > bn || isnan(ab)) bn = ab;
  }
  const double eps = 0x1p-53;
  out5[0] = rn / (eps * (an * xn + bn) * (double)(n > 0 ? n : 1));
  out5[1] = rn;
  out5[2] = an;
  out5[3] = xn;
  out5[4] = bn;
}

/* HPL scaled residual from a stored matrix:
 *   out5 = { ||Ax-b||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) N),
 *            ||Ax-b||_inf, ||A||_inf, ||x||_inf, ||b||_inf },  eps = 2^-53.
 * r = A x - b per row with Dot2. */
void orc_residual_dense(int64_t n, const double* A, int64_t lda, const double* x,
                        const double* b, double* out5) {
  double* rhi = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* rlo = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* rowabs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double hi = -b[i], lo = 0.0, ra = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      orc_dot2_add(&hi, &lo, A[i + j * lda], x[j]);
      ra = ra + fabs(A[i + j * lda]);
    }
    rhi[i] = hi; rlo[i] = lo; rowabs[i] = ra;
  }
  orc_residual_finish(n, rhi, rlo, rowabs, x, b, out5);
  free(rhi); free(rlo); free(rowabs);
}

/* Same residual with A and b regenerated from the seed column by column, so
 * that no N x N copy is held (N = 131072 does not fit in host memory).  Each
 * thread takes a contiguous range of columns, jumps the generator to its first
 * element and keeps its own per-row Dot2 accumulators; the per-thread partial
 * sums are merged with TwoSum at the end.  dd != 0 selects the diagonally
 * dominant matrix of orc_generate_dd; its diagonal is the ascending-j plain sum
 * of the row's off-diagonal magnitudes, which is rebuilt exactly by a second
 * sequential pass per row block.  b_out (may be NULL) receives b. */
void orc_residual_seeded(int64_t n, uint64_t seed, int dd, const double* x,
                         double* b_out, double* out5) {
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  size_t nn = (size_t)(n > 0 ? n : 1);
  double* hi = (double*)calloc(nn * (size_t)nt, sizeof(double));
  double* lo = (double*)calloc(nn * (size_t)nt, sizeof(double));
  double* ra = (double*)calloc(nn * (size_t)nt, sizeof(double));
  double* b = (double*)calloc(nn, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int64_t j0 = (n * tid) / nt, j1 = (n * (tid + 1)) / nt;
    double* h = hi + (size_t)tid * nn;
    double* l = lo + (size_t)tid * nn;
    double* a = ra + (size_t)tid * nn;
    uint64_t s = orc_lcg_skip(seed, (uint64_t)j0 * (uint64_t)n);
    for (int64_t j = j0; j < j1; ++j)
      for (int64_t i = 0; i < n; ++i) {
        s = orc_step(s);
        double v = orc_value(s);
        if (dd && i == j) continue; /* diagonal added below */
        orc_dot2_add(&h[i], &l[i], v, x[j]);
        a[i] = a[i] + fabs(v);
      }
  }
  {
    uint64_t s = orc_lcg_skip(seed, (uint64_t)n * (uint64_t)n);
    for (int64_t i = 0; i < n; ++i) { s = orc_step(s); b[i] = orc_value(s); }
  }
  double* rhi = (double*)calloc(nn, sizeof(double));
  double* rlo = (double*)calloc(nn, sizeof(double));
  double* rowabs = (double*)calloc(nn, sizeof(double));
  double* diag = NULL;
  if (dd) {
    /* exact diagonal: ascending-j plain sum of |A(i,j)|, j != i */
    diag = (double*)calloc(nn, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t ib = 0; ib < n; ib += 256) {
      int64_t ie = ib + 256 < n ? ib + 256 : n;
      double acc[256];
      for (int64_t i = ib; i < ie; ++i) acc[i - ib] = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        uint64_t s = orc_lcg_skip(seed, (uint64_t)j * (uint64_t)n + (uint64_t)ib);
        for (int64_t i = ib; i < ie; ++i) {
          s = orc_step(s);
          if (i != j) acc[i - ib] = acc[i - ib] + fabs(orc_value(s));
        }
      }
      for (int64_t i = ib; i < ie; ++i) diag[i] = acc[i - ib];
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double h = -b[i], l = 0.0, a = 0.0;
    for (int t = 0; t < nt; ++t) {
      double s, e;
      orc_two_sum(h, hi[(size_t)t * nn + i], &s, &e);
      h = s;
      l = l + e + lo[(size_t)t * nn + i];
      a = a + ra[(size_t)t * nn + i];
    }
    if (dd) {
      orc_dot2_add(&h, &l, diag[i], x[i]);
      a = a + diag[i];
    }
    rhi[i] = h; rlo[i] = l; rowabs[i] = a;
  }
  orc_residual_finish(n, rhi, rlo, rowabs, x, b, out5);
  if (b_out) memcpy(b_out, b, nn * sizeof(double));
  free(hi); free(lo); free(ra); free(b); free(rhi); free(rlo); free(rowabs); free(diag);
}

/* ------------------------------------------------------------ factor check */

/* ||P A - L U||_F / (||A||_F * n * eps), eps = 2^-53, with L unit-lower and U
 * upper taken from the packed factors and P the product of the interchanges
 * ipiv (applied in order j = 0..n-1 to the rows of A0). */
double orc_factor_error(int64_t n, const double* A0, int64_t lda0, const double* LU,
                        int64_t lda, const int32_t* ipiv) {
  if (n <= 0) return 0.0;
  int64_t* perm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  if (ipiv)
    for (int64_t j = 0; j < n; ++j) {
      int64_t p = ipiv[j] - 1;
      int64_t t = perm[j]; perm[j] = perm[p]; perm[p] = t;
    }
  double num = 0.0, den = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : num, den)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = 0; i < n; ++i) {
      /* (L U)(i,c) = sum_{k <= min(i,c)} L(i,k) U(k,c), L(i,i) = 1 */
      int64_t kmax = i < c ? i : c;
      double s = 0.0;
      for (int64_t k = 0; k <= kmax; ++k) {
        double l = (k == i) ? 1.0 : LU[i + k * lda];
        s = s + l * LU[k + c * lda];
      }
      double a = A0[perm[i] + c * lda0];
      double d = a - s;
      num += d * d;
      den += a * a;
    }
  }
  free(perm);
  return sqrt(num) / (sqrt(den) * (double)n * 0x1p-53);
}

/* Randomized (Freivalds-style) estimate of ||P A - L U||_F for systems too
 * large for orc_factor_error: for v with i.i.d. unit-variance entries,
 * E ||E v||_2^2 = ||E||_F^2, so ||P (A v) - L (U v)||_2 estimates ||PA - LU||_F.
 * A is regenerated from the seed (orc_generate order) column by column; A v,
 * U v and L (U v) are accumulated with Dot2 so the difference is not swamped
 * by the rounding of the products.  Returns the estimate divided by
 * (||A||_F n eps), eps = 2^-53 (||A||_F computed exactly on the same pass,
 * up to rounding). */
double orc_factor_probe(int64_t n, uint64_t seed, const double* LU, int64_t lda,
                        const int32_t* ipiv, const double* v) {
  if (n <= 0) return 0.0;
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  size_t nn = (size_t)n;
  double* hi = (double*)calloc(nn * (size_t)nt, sizeof(double));
  double* lo = (double*)calloc(nn * (size_t)nt, sizeof(double));
  double* fro = (double*)calloc((size_t)nt, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int64_t j0 = (n * tid) / nt, j1 = (n * (tid + 1)) / nt;
    double* h = hi + (size_t)tid * nn;
    double* l = lo + (size_t)tid * nn;
    double f = 0.0;
    uint64_t s = orc_lcg_skip(seed, (uint64_t)j0 * (uint64_t)n);
    for (int64_t j = j0; j < j1; ++j)
      for (int64_t i = 0; i < n; ++i) {
        s = orc_step(s);
        double a = orc_value(s);
        orc_dot2_add(&h[i], &l[i], a, v[j]);
        f = f + a * a;
      }
    fro[tid] = f;
  }
  double* y = (double*)calloc(nn, sizeof(double));  /* A v */
  double fa = 0.0;
  for (int t = 0; t < nt; ++t) fa = fa + fro[t];
  for (int64_t i = 0; i < n; ++i) {
    double h = 0.0, l = 0.0;
    for (int t = 0; t < nt; ++t) {
      double s2, e;
      orc_two_sum(h, hi[(size_t)t * nn + i], &s2, &e);
      h = s2;
      l = l + e + lo[(size_t)t * nn + i];
    }
    y[i] = h + l;
  }
  /* P (A v): the interchanges in order */
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = ipiv[j] - 1;
    double t = y[j]; y[j] = y[p]; y[p] = t;
  }
  /* w = U v, row i = sum_{j >= i} U(i,j) v_j; then z = L w, row i = w_i + sum_{j < i} L(i,j) w_j */
  double* w = (double*)calloc(nn, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double h = 0.0, l = 0.0;
    for (int64_t j = i; j < n; ++j) orc_dot2_add(&h, &l, LU[i + j * lda], v[j]);
    w[i] = h + l;
  }
  double num = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : num)
  for (int64_t i = 0; i < n; ++i) {
    double h = w[i], l = 0.0;
    for (int64_t j = 0; j < i; ++j) orc_dot2_add(&h, &l, LU[i + j * lda], w[j]);
    /* (P A v)_i - (L U v)_i with one more error-free step */
    double d_h = 0.0, d_l = 0.0;
    orc_two_sum(y[i], -h, &d_h, &d_l);
    double d = d_h + (d_l - l);
    num += d * d;
  }
  free(hi); free(lo); free(fro); free(y); free(w);
  return sqrt(num) / (sqrt(fa) * (double)n * 0x1p-53);
}

/* ----------------------------------------------------------------- adjoint */

/* Adjoint of X = A^-1 B for the loss sum(W .* X): dB = A^-T W and
 * dA = -dB X^T (closed form; reuses the factors, nothing is refactored).
 * dB (n x k, ldb) and dA (n x n, ldda) are outputs. */
void orc_solve_adjoint(int64_t n, int64_t k, const double* LU, int64_t lda,
                       const int32_t* ipiv, const double* X, int64_t ldx,
                       const double* W, int64_t ldw, double* dB, int64_t ldb,
                       double* dA, int64_t ldda) {
  for (int64_t r = 0; r < k; ++r)
    for (int64_t i = 0; i < n; ++i) dB[i + r * ldb] = W[i + r * ldw];
  orc_getrs('T', n, k, LU, lda, ipiv, dB, ldb);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t r = 0; r < k; ++r) s = s + dB[i + r * ldb] * X[c + r * ldx];
      dA[i + c * ldda] = -s;
    }
}

/* ------------------------------------------------ mixed-precision variant */
/* Not in the paper (it only names HPL-MxP, Sec. I).  The variant factors a
 * diagonally dominant system without pivoting: the panel and the U12 solve in
 * FP32, the trailing update with BF16 or FP8-E4M3 operands that carry one
 * power-of-two scale per 128-row tile of L21 (spanning the panel width) and per
 * 128-column tile of U12, products accumulated at (at least) FP32, and the
 * trailing matrix kept in FP32.  The oracle follows those steps in order;
 * its update sums the exact products of the quantized values in FP64. */

/* BF16 from FP32, round to nearest even (IEEE 754 binary32 -> the 16-bit
 * format that keeps the binary32 exponent and 7 fraction bits). */
uint16_t orc_f32_to_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x0040u); /* quiet NaN */
  uint32_t rest = u & 0xffffu, keep = u >> 16;
  if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
  return (uint16_t)keep;
}

float orc_bf16_to_f32(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* OCP FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 fraction bits; no
 * infinities; S.1111.111 is NaN; largest finite 448; subnormals k 2^-9).
 * Round to nearest even; magnitudes beyond 448 saturate to 448. */
uint8_t orc_f32_to_e4m3(float x) {
  uint8_t sign = signbit(x) ? 0x80 : 0x00;
  double a = fabs((double)x);
  if (isnan(x)) return (uint8_t)(sign | 0x7f);
  if (a < 0x1p-6) { /* subnormal range: k 2^-9, k = 0..8 (8 is the smallest normal) */
    double k = rint(a * 0x1p9);
    return (uint8_t)(sign | (uint8_t)k);
  }
  int E;
  frexp(a, &E);          /* a = f 2^E, f in [0.5, 1) */
  int ex = E - 1;        /* a = m 2^ex, m in [1, 2) */
  double m = ldexp(a, -ex);
  double q = rint((m - 1.0) * 8.0);
  if (q == 8.0) { q = 0.0; ex += 1; }
  int biased = ex + 7;
  if (biased > 15 || (biased == 15 && q == 7.0)) return (uint8_t)(sign | 0x7e); /* saturate to 448 */
  return (uint8_t)(sign | (uint8_t)(biased << 3) | (uint8_t)q);
}

float orc_e4m3_to_f32(uint8_t c) {
  double s = (c & 0x80) ? -1.0 : 1.0;
  int e = (c >> 3) & 0xf, m = c & 7;
  if (e == 15 && m == 7) return NAN;
  if (e == 0) return (float)(s * ldexp((double)m, -9));
  return (float)(s * ldexp(1.0 + m / 8.0, e - 7));
}

/* Largest integer e with amax 2^e <= qmax, computed exactly from the binary
 * exponents; 0 for amax == 0 or non-finite; clamped to [-126, 126]. */
int orc_scale_exp(double amax, double qmax) {
  if (!(amax > 0.0) || isinf(amax)) return 0;
  int Ea, Eq;
  double fa = frexp(amax, &Ea), fq = frexp(qmax, &Eq);
  int e = Eq - Ea - (fa > fq ? 1 : 0);
  if (e > 126) e = 126;
  if (e < -126) e = -126;
  return e;
}

/* Quantized value (as the exact FP32 it encodes) of x 2^e in format prec
 * (0 = BF16, 1 = E4M3). */
static double orc_quant_value(float x, int e, int prec) {
  float y = ldexpf(x, e); /* exact: a power-of-two scaling within range */
  if (prec == 0) return (double)orc_bf16_to_f32(orc_f32_to_bf16(y));
  return (double)orc_e4m3_to_f32(orc_f32_to_e4m3(y));
}

double orc_qmax(int prec) { return prec == 0 ? 1.0 : 448.0; }

/* Tile scale exponents of an FP32 block X (rows x cols, ldx): tiles of 128
 * rows spanning all columns when by_rows != 0, else tiles of 128 columns
 * spanning all rows.  exps[t] for t = 0..ceil(extent/128)-1. */
void orc_tile_exps(int64_t rows, int64_t cols, const float* X, int64_t ldx, int by_rows, int prec,
                   int32_t* exps) {
  int64_t ext = by_rows ? rows : cols;
  for (int64_t t = 0; t * 128 < ext; ++t) {
    int64_t a0 = t * 128, a1 = a0 + 128 < ext ? a0 + 128 : ext;
    double amax = 0.0;
    for (int64_t j = 0; j < cols; ++j)
      for (int64_t i = 0; i < rows; ++i) {
        int64_t a = by_rows ? i : j;
        if (a < a0 || a >= a1) continue;
        double v = fabs((double)X[i + j * ldx]);
        if (v > amax) amax = v;
      }
    exps[t] = orc_scale_exp(amax, orc_qmax(prec));
  }
}

/* Codes of X 2^e (e from the tile of each element): out[i + j rows] holds the
 * BF16 (prec 0) or E4M3 (prec 1) code of element (i, j), stored in uint16. */
void orc_quantize(int64_t rows, int64_t cols, const float* X, int64_t ldx, int by_rows, int prec,
                  const int32_t* exps, uint16_t* out) {
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i) {
      int e = exps[(by_rows ? i : j) / 128];
      float y = ldexpf(X[i + j * ldx], e);
      out[i + j * rows] = prec == 0 ? orc_f32_to_bf16(y) : (uint16_t)orc_f32_to_e4m3(y);
    }
}

/* Steps 2 to 4 of the mixed-precision LU for the panel at columns k0 .. k0+jb-1
 * (factored in W): U12 by FP32 forward substitution, the tile exponents and
 * codes of L21 and U12 taken from Q (W itself, or the factors being replayed),
 * and the trailing update from the exact products of the decoded codes. */
static void mxp_trailing(int64_t n, int64_t k0, int64_t jb, int prec, float* W, int64_t ldw, const float* Q,
                         int64_t ldq) {
  const int64_t e = k0 + jb, m2 = n - e;
  if (m2 <= 0) return;
  /* 2. U12 */
#pragma omp parallel for schedule(static)
  for (int64_t c = e; c < n; ++c)
    for (int64_t i = k0; i < e; ++i) {
      float s = W[i + c * ldw];
      for (int64_t k = k0; k < i; ++k) s = s - W[i + k * ldw] * W[k + c * ldw];
      W[i + c * ldw] = s;
    }
  /* 3. scales and quantized operands (as exact doubles) */
  int64_t nt = (m2 + 127) / 128;
  int32_t* eL = (int32_t*)malloc((size_t)nt * sizeof(int32_t));
  int32_t* eU = (int32_t*)malloc((size_t)nt * sizeof(int32_t));
  orc_tile_exps(m2, jb, Q + e + k0 * ldq, ldq, 1, prec, eL);
  orc_tile_exps(jb, m2, Q + k0 + e * ldq, ldq, 0, prec, eU);
  double* qL = (double*)malloc((size_t)m2 * (size_t)jb * sizeof(double));
  double* qU = (double*)malloc((size_t)m2 * (size_t)jb * sizeof(double));
  for (int64_t k = 0; k < jb; ++k)
    for (int64_t i = 0; i < m2; ++i) {
      qL[i + k * m2] = orc_quant_value(Q[e + i + (k0 + k) * ldq], eL[i / 128], prec);
      qU[k + i * jb] = orc_quant_value(Q[k0 + k + (e + i) * ldq], eU[i / 128], prec);
    }
  /* 4. update */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < m2; ++c)
    for (int64_t i = 0; i < m2; ++i) {
      double p = 0.0;
      for (int64_t k = 0; k < jb; ++k) p = p + qL[i + k * m2] * qU[k + c * jb];
      p = ldexp(p, -(eL[i / 128] + eU[c / 128]));
      W[e + i + (e + c) * ldw] = (float)((double)W[e + i + (e + c) * ldw] - p);
    }
  free(eL); free(eU); free(qL); free(qU);
}

/* Mixed-precision LU without pivoting of the n x n FP64 matrix A64 into the
 * FP32 factors LU (ldl), panels of nb columns.  Per panel:
 *   1. FP32 right-looking LU of the m x jb panel (no interchanges);
 *   2. U12 <- L11^-1 A12 by FP32 forward substitution;
 *   3. per-tile scale exponents eL (128-row tiles of L21) and eU (128-column
 *      tiles of U12), quantization of L21 2^eL and U12 2^eU to prec;
 *   4. A22 <- fl32(A22 - 2^-(eL+eU) sum_k qL(i,k) qU(k,j)), the sum of exact
 *      products taken in FP64.
 * *info = first zero pivot (1-based) or 0.
 *
 * Two options serve the parity tests (both off in orc_mxp_getrf):
 *   - replay R (ldr), the final factors of another implementation: step 3
 *     takes the exponents and codes from R's L21 and U12 of the panel instead
 *     of its own.  Those blocks are final once their panel is done, so the
 *     oracle's trailing matrix then follows the same quantized products as R's
 *     did, and each panel of W can be compared with R's in isolation: what is
 *     left between them is FP32 arithmetic of one panel and the FP32 rounding
 *     of the updates, no quantization decision (a value near a rounding
 *     boundary of the format would otherwise make the two pick different
 *     codes, an error of one code step that no rounding bound covers).
 *   - plant (panel plant_panel, relative size plant_rel): after step 1 of that
 *     panel, L21 is multiplied by (1 + plant_rel) in FP32, a planted error in
 *     the panel's product L21 = A21 U11^-1, for the test that checks that the
 *     comparison catches it. */
void orc_mxp_getrf_ex(int64_t n, int64_t nb, int prec, const double* A64, int64_t lda, float* W,
                      int64_t ldw, int32_t* info, const float* R, int64_t ldr, int64_t plant_panel,
                      double plant_rel) {
  int32_t inf = 0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) W[i + j * ldw] = (float)A64[i + j * lda];
  for (int64_t k0 = 0; k0 < n; k0 += nb) {
    int64_t jb = nb < n - k0 ? nb : n - k0;
    int64_t e = k0 + jb;
    /* 1. panel */
    for (int64_t j = k0; j < e; ++j) {
      float piv = W[j + j * ldw];
      if (piv == 0.0f) { if (inf == 0) inf = (int32_t)(j + 1); continue; }
      for (int64_t i = j + 1; i < n; ++i) W[i + j * ldw] = W[i + j * ldw] / piv;
      for (int64_t c = j + 1; c < e; ++c) {
        float u = W[j + c * ldw];
        for (int64_t i = j + 1; i < n; ++i) W[i + c * ldw] = W[i + c * ldw] - W[i + j * ldw] * u;
      }
    }
    if (k0 / nb == plant_panel && plant_rel != 0.0)
      for (int64_t j = k0; j < e; ++j)
        for (int64_t i = e; i < n; ++i) W[i + j * ldw] = (float)((double)W[i + j * ldw] * (1.0 + plant_rel));
    mxp_trailing(n, k0, jb, prec, W, ldw, R ? R : W, R ? ldr : ldw); /* R: whose L21 and U12 are quantized */
  }
  *info = inf;
}

void orc_mxp_getrf(int64_t n, int64_t nb, int prec, const double* A64, int64_t lda, float* W,
                   int64_t ldw, int32_t* info) {
  orc_mxp_getrf_ex(n, nb, prec, A64, lda, W, ldw, info, NULL, 0, -1, 0.0);
}

/* Solve with FP32 unpivoted factors, arithmetic in FP64: x <- U^-1 L^-1 x. */
void orc_mxp_getrs(int64_t n, const float* LU, int64_t ldl, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double s = x[i];
    for (int64_t k = 0; k < i; ++k) s = s - (double)LU[i + k * ldl] * x[k];
    x[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t k = i + 1; k < n; ++k) s = s - (double)LU[i + k * ldl] * x[k];
    x[i] = s / (double)LU[i + i * ldl];
  }
}

/* Mixed-precision LU WITH partial pivoting of the n x n FP64 matrix A64 into
 * FP32 factors W (ldw) and pivots ipiv (1-based, LAPACK), panels of nb
 * columns: the steps of orc_mxp_getrf with step 1 pivoted as FACT is in
 * Sec. I: at column j of the panel the row p >= j of largest |W(p,j)| (first
 * maximum on ties) is chosen, ipiv[j] = p + 1, and rows j and p are swapped
 * across all n columns (the columns left of the panel, the panel and the
 * trailing columns, so that P A = L U holds for the packed factors); then
 * the column is scaled and the panel's columns right of it are updated, in
 * FP32.  Steps 2 to 4 (U12, quantization, the trailing update) are those of
 * the unpivoted variant.  *info = first zero pivot (1-based) or 0. */
void orc_mxp_getrf_piv(int64_t n, int64_t nb, int prec, const double* A64, int64_t lda, float* W, int64_t ldw,
                       int32_t* ipiv, int32_t* info) {
  int32_t inf = 0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) W[i + j * ldw] = (float)A64[i + j * lda];
  for (int64_t k0 = 0; k0 < n; k0 += nb) {
    int64_t jb = nb < n - k0 ? nb : n - k0;
    int64_t e = k0 + jb;
    for (int64_t j = k0; j < e; ++j) {
      int64_t p = j;
      float best = fabsf(W[j + j * ldw]);
      for (int64_t i = j + 1; i < n; ++i)
        if (fabsf(W[i + j * ldw]) > best) { best = fabsf(W[i + j * ldw]); p = i; }
      ipiv[j] = (int32_t)(p + 1);
      if (p != j)
        for (int64_t c = 0; c < n; ++c) {
          float t = W[j + c * ldw];
          W[j + c * ldw] = W[p + c * ldw];
          W[p + c * ldw] = t;
        }
      float piv = W[j + j * ldw];
      if (piv == 0.0f) { if (inf == 0) inf = (int32_t)(j + 1); continue; }
      for (int64_t i = j + 1; i < n; ++i) W[i + j * ldw] = W[i + j * ldw] / piv;
      for (int64_t c = j + 1; c < e; ++c) {
        float u = W[j + c * ldw];
        for (int64_t i = j + 1; i < n; ++i) W[i + c * ldw] = W[i + c * ldw] - W[i + j * ldw] * u;
      }
    }
    mxp_trailing(n, k0, jb, prec, W, ldw, W, ldw);
  }
  *info = inf;
}

/* Solve with FP32 pivoted factors, arithmetic in FP64: x <- U^-1 L^-1 P x
 * (the interchanges of ipiv applied in order, then orc_mxp_getrs). */
void orc_mxp_getrs_piv(int64_t n, const float* LU, int64_t ldl, const int32_t* ipiv, double* x) {
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = (int64_t)ipiv[j] - 1;
    if (p != j) { double t = x[j]; x[j] = x[p]; x[p] = t; }
  }
  orc_mxp_getrs(n, LU, ldl, x);
}

/* ------------------------------------------- emulated FP64 trailing update */
/* Not the paper's method (rocHPL runs the trailing update as an FP64 DGEMM,
 * Sec. I): the Schur update C <- C - A B of Sec. I computed from products of
 * low-precision slices, after Ozaki, Ogita, Oishi and Rump ("Error-free
 * transformations of matrix multiplication by using fast routines of matrix
 * multiplication and its applications", Numer. Algorithms 59, 2012).
 *
 * Splitting (error-free): row r of A (m x k) has mu_r = max_c |A(r,c)| and E_r
 * with mu_r < 2^E_r (E_r = 0 for a zero row); every entry is scaled to
 * a' = A(r,c) 2^-E_r in (-1, 1) and peeled into s integer slices of beta bits:
 * t = a' 2^beta, q_i = nearest integer to t (ties to even), a' = t - q_i,
 * so that A(r,c) = 2^E_r (sum_i q_i 2^(-i beta) + rest), |q_1| <= 2^beta,
 * |q_i| <= 2^(beta-1) for i >= 2, |rest| <= 2^(-s beta - 1).  Every step is
 * exact in FP64.  Columns of B (k x n) are split the same way with their own
 * exponents F_c.
 *
 * Products: for each level d = i + j = 2 .. s+1 the integer matrix
 * P_d = sum_{i+j=d} Q_i Q'_j, exact (the oracle sums it in FP64 well inside
 * 2^53).  The pairs with i + j > s + 1 are the ones the scheme drops.
 *
 * Sum, smallest level first: the levels d >= d0 = max(2, s + 1 -
 * floor(37 / beta)) are summed exactly in 64-bit integers,
 * T = sum_{d >= d0} P_d 2^((s + 1 - d) beta) (|P_d| <= 2^24, so |T| < 2^63),
 * and rounded once to FP64, S = fl(T) 2^-((s + 1 - d0) beta); the levels
 * below follow in FP64, S = P_d + 2^-beta S for d = d0 - 1 .. 2 (the scaling
 * exact, one rounding each); then C(r,c) <- C(r,c) - 2^(E_r + F_c - 2 beta) S,
 * the product exact and the difference rounded once.  (The levels may be
 * summed in any order; the exact integer part spares FP64 roundings and the
 * FP64 work of a GPU whose FP64 pipe is its slowest.) */

/* The lowest level d0 of the exact integer part of the level sum. */
int orc_ozaki_int_level(int s, int beta) {
  int d0 = s + 1 - 37 / beta;
  return d0 < 2 ? 2 : d0;
}

/* E with mu < 2^E for mu > 0 (the binary exponent of frexp); 0 for mu == 0. */
static int orc_slice_exp(double mu) {
  if (!(mu > 0.0)) return 0;
  int E;
  frexp(mu, &E);
  return E;
}

/* The s slices of x (|x| < 2^E): q[i] for i = 0 .. s-1 (slice i + 1). */
static void orc_split_value(double x, int E, int s, int beta, double* q) {
  double a = ldexp(x, -E);
  for (int i = 0; i < s; ++i) {
    double t = ldexp(a, beta);
    double qi = nearbyint(t); /* round to nearest, ties to even (default mode) */
    q[i] = qi;
    a = t - qi;
  }
}

/* Row exponents and slices of A (m x k): QA[(i * m + r) * k + c] = slice i+1
 * of A(r, c); ER[r]. */
void orc_ozaki_split_rows(int64_t m, int64_t k, const double* A, int64_t lda, int s, int beta, int32_t* ER,
                          double* QA) {
  for (int64_t r = 0; r < m; ++r) {
    double mu = 0.0;
    for (int64_t c = 0; c < k; ++c) {
      double v = fabs(A[r + c * lda]);
      if (v > mu) mu = v;
    }
    int E = orc_slice_exp(mu);
    ER[r] = E;
    double q[64];
    for (int64_t c = 0; c < k; ++c) {
      orc_split_value(A[r + c * lda], E, s, beta, q);
      for (int i = 0; i < s; ++i) QA[((int64_t)i * m + r) * k + c] = q[i];
    }
  }
}

/* Column exponents and slices of B (k x n): QB[(j * n + c) * k + r] = slice
 * j+1 of B(r, c); FC[c]. */
void orc_ozaki_split_cols(int64_t k, int64_t n, const double* B, int64_t ldb, int s, int beta, int32_t* FC,
                          double* QB) {
  for (int64_t c = 0; c < n; ++c) {
    double mu = 0.0;
    for (int64_t r = 0; r < k; ++r) {
      double v = fabs(B[r + c * ldb]);
      if (v > mu) mu = v;
    }
    int F = orc_slice_exp(mu);
    FC[c] = F;
    double q[64];
    for (int64_t r = 0; r < k; ++r) {
      orc_split_value(B[r + c * ldb], F, s, beta, q);
      for (int j = 0; j < s; ++j) QB[((int64_t)j * n + c) * k + r] = q[j];
    }
  }
}

/* C (m x n, ldc) <- C - A B with A (m x k, lda) and B (k x n, ldb) by the
 * slice products above; 1 <= s <= 64, 1 <= beta <= 26.  Returns 0, or -1 if
 * a level sum could leave the range where FP32 accumulation of the slice
 * products is exact (k sum_{i+j=d} max|q_i| max|q_j| > 2^24): the GPU kernel
 * relies on that exactness, so the oracle refuses the same cases. */
int orc_ozaki_gemm(int64_t m, int64_t n, int64_t k, int s, int beta, const double* A, int64_t lda,
                   const double* B, int64_t ldb, double* C, int64_t ldc) {
  if (s < 1 || s > 64 || beta < 1 || beta > 26) return -1;
  for (int d = 2; d <= s + 1; ++d) {
    double bound = 0.0;
    for (int i = 1; i < d; ++i) {
      int j = d - i;
      if (i > s || j > s) continue;
      bound += ldexp(1.0, i == 1 ? beta : beta - 1) * ldexp(1.0, j == 1 ? beta : beta - 1);
    }
    if ((double)k * bound > 16777216.0) return -1;
  }
  if (m <= 0 || n <= 0) return 0;
  int32_t* ER = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* FC = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  double* QA = (double*)malloc((size_t)s * (size_t)m * (size_t)(k > 0 ? k : 1) * sizeof(double));
  double* QB = (double*)malloc((size_t)s * (size_t)n * (size_t)(k > 0 ? k : 1) * sizeof(double));
  orc_ozaki_split_rows(m, k, A, lda, s, beta, ER, QA);
  orc_ozaki_split_cols(k, n, B, ldb, s, beta, FC, QB);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    double P[66];
    for (int64_t r = 0; r < m; ++r) {
      for (int d = 2; d <= s + 1; ++d) {
        double p = 0.0;
        for (int i = 1; i < d; ++i) {
          int j = d - i;
          if (i > s || j > s) continue;
          const double* qa = QA + ((int64_t)(i - 1) * m + r) * k;
          const double* qb = QB + ((int64_t)(j - 1) * n + c) * k;
          for (int64_t t = 0; t < k; ++t) p = p + qa[t] * qb[t];
        }
        P[d] = p;
      }
      const int d0 = orc_ozaki_int_level(s, beta);
      int64_t T = 0;
      for (int d = d0; d <= s + 1; ++d) T = T * ((int64_t)1 << beta) + (int64_t)P[d];  /* P_d0 weighs most */
      double S = ldexp((double)T, -(s + 1 - d0) * beta); /* (double) of an int64: nearest, ties to even */
      for (int d = d0 - 1; d >= 2; --d) S = P[d] + ldexp(S, -beta);
      double scale = ldexp(1.0, ER[r] + FC[c] - 2 * beta);
      C[r + c * ldc] = C[r + c * ldc] - scale * S;
    }
  }
  free(ER); free(FC); free(QA); free(QB);
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
