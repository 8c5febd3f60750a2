/*
 * Plain, slow, FP64 CPU oracle for the factorization-based DPP sampler of
 * Poulson, "High-performance sampling of generic Determinantal Point
 * Processes" (arXiv:1905.00165).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * helper with the CUDA library; the CUDA path never calls it.
 *
 * What is computed, and where the paper fixes it:
 *   - Algorithm 1 ("Unblocked, right-looking, non-Hermitian DPP sampling"),
 *     Theorem 1: for j = 0..n-1 the pivot A_jj is the conditional inclusion
 *     probability of index j; index j is kept by a Bernoulli draw with that
 *     probability, otherwise 1 is subtracted from the pivot (Prop. 4, element
 *     exclusion); the column below the pivot is divided by the pivot and the
 *     trailing block receives the rank-1 Schur-complement update (Prop. 3/4).
 *   - The likelihood of the sample is the product of the absolute values of
 *     the final pivots (Theorem 1, and the proof of Prop. 1 that follows it):
 *     log P(Y) = sum_j log|d_j|.
 *   - The Hermitian specialisation (Section 3, "the same specializations that
 *     exist for modifying an unpivoted LU factorization into ... LDL^H"): only
 *     the lower triangle is referenced, L is unit lower triangular and D is
 *     real diagonal.
 *
 * Readings where the paper is silent (they are the library's documented
 * conventions as well, but implemented here independently):
 *   - Bernoulli(d): keep iff u_j < Re(d_j), u_j in (0,1).
 *   - u_j comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC'11) with key = (seed lo, seed hi) and
 *     counter = (j, instance lo, instance hi, 0); the 53-bit uniform is
 *     u = ((x0 << 21 | x1 >> 11) + 0.5) * 2^-53.
 *   - Hermitian pivots are real: the imaginary part is discarded.
 *
 * Parallelism: the rank-1 update loops over independent columns with OpenMP;
 * each matrix entry receives exactly the operations of the definition, in the
 * same order, so the result does not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon et al., SC'11).       */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(PHILOX_M0, c0, &hi0, &lo0);
    mulhilo32(PHILOX_M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double oracle_uniform(uint64_t seed, uint64_t instance, uint64_t j) {
  uint32_t ctr[4] = {(uint32_t)j, (uint32_t)instance, (uint32_t)(instance >> 32), 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  oracle_philox4x32_10(ctr, key, x);
  uint64_t bits53 = ((uint64_t)x[0] << 21) | (uint64_t)(x[1] >> 11);
  return ((double)bits53 + 0.5) * 0x1.0p-53;
}

void oracle_uniforms(uint64_t seed, uint64_t instance, int64_t n, double* u) {
  for (int64_t j = 0; j < n; ++j) u[j] = oracle_uniform(seed, instance, (uint64_t)j);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: unblocked right-looking non-Hermitian sampler (real).          */
/* A: column-major n x n with leading dimension ld, overwritten with the       */
/* in-place LU factors of K - 1_{Y^c}. u: n uniforms. keep: n bytes (0/1).     */
/* pivots: n final pivots d_j (after the -1 of a rejection). Returns |Y|.      */
/* ------------------------------------------------------------------------- */
int64_t oracle_dpp_lu_r64(int64_t n, double* A, int64_t ld, const double* u,
                          uint8_t* keep, double* pivots, double* logp) {
  double lp = 0.0;
  int64_t kept = 0;
  for (int64_t j = 0; j < n; ++j) {
    double d = A[j + j * ld];
    if (u[j] < d) {
      keep[j] = 1;
      ++kept;
    } else {
      keep[j] = 0;
      d -= 1.0;
      A[j + j * ld] = d;
    }
    pivots[j] = d;
    lp += log(fabs(d));
    for (int64_t i = j + 1; i < n; ++i) A[i + j * ld] /= d;
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      const double ajk = A[j + k * ld];
      for (int64_t i = j + 1; i < n; ++i) A[i + k * ld] -= A[i + j * ld] * ajk;
    }
  }
  *logp = lp;
  return kept;
}

/* Algorithm 1, complex: keep iff u_j < Re(d_j); log|d_j| uses the modulus. */
int64_t oracle_dpp_lu_c128(int64_t n, double complex* A, int64_t ld,
                           const double* u, uint8_t* keep,
                           double complex* pivots, double* logp) {
  double lp = 0.0;
  int64_t kept = 0;
  for (int64_t j = 0; j < n; ++j) {
    double complex d = A[j + j * ld];
    if (u[j] < creal(d)) {
      keep[j] = 1;
      ++kept;
    } else {
      keep[j] = 0;
      d -= 1.0;
      A[j + j * ld] = d;
    }
    pivots[j] = d;
    lp += log(cabs(d));
    for (int64_t i = j + 1; i < n; ++i) A[i + j * ld] /= d;
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      const double complex ajk = A[j + k * ld];
      for (int64_t i = j + 1; i < n; ++i) A[i + k * ld] -= A[i + j * ld] * ajk;
    }
  }
  *logp = lp;
  return kept;
}

/* ------------------------------------------------------------------------- */
/* Hermitian specialisation (LDL^H): only the lower triangle of A is read and  */
/* written. On return the strictly-lower part holds L (unit diagonal implied)  */
/* and the diagonal holds D, the final real pivots.                            */
/* ------------------------------------------------------------------------- */
int64_t oracle_dpp_ldl_r64(int64_t n, double* A, int64_t ld, const double* u,
                           uint8_t* keep, double* pivots, double* logp) {
  double lp = 0.0;
  int64_t kept = 0;
  for (int64_t j = 0; j < n; ++j) {
    double d = A[j + j * ld];
    if (u[j] < d) {
      keep[j] = 1;
      ++kept;
    } else {
      keep[j] = 0;
      d -= 1.0;
      A[j + j * ld] = d;
    }
    pivots[j] = d;
    lp += log(fabs(d));
    for (int64_t i = j + 1; i < n; ++i) A[i + j * ld] /= d; /* L_ij */
    /* A_ik -= L_ij * d_j * L_kj for i >= k > j (lower triangle) */
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      const double c = d * A[k + j * ld];
      for (int64_t i = k; i < n; ++i) A[i + k * ld] -= A[i + j * ld] * c;
    }
  }
  *logp = lp;
  return kept;
}

int64_t oracle_dpp_ldl_c128(int64_t n, double complex* A, int64_t ld,
                            const double* u, uint8_t* keep, double* pivots,
                            double* logp) {
  double lp = 0.0;
  int64_t kept = 0;
  for (int64_t j = 0; j < n; ++j) {
    double d = creal(A[j + j * ld]); /* D is real for Hermitian K */
    if (u[j] < d) {
      keep[j] = 1;
      ++kept;
    } else {
      keep[j] = 0;
      d -= 1.0;
    }
    A[j + j * ld] = d;
    pivots[j] = d;
    lp += log(fabs(d));
    for (int64_t i = j + 1; i < n; ++i) A[i + j * ld] /= d; /* L_ij */
    /* A_ik -= L_ij * d_j * conj(L_kj) for i >= k > j */
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      const double complex c = d * conj(A[k + j * ld]);
      for (int64_t i = k; i < n; ++i) A[i + k * ld] -= A[i + j * ld] * c;
    }
  }
  *logp = lp;
  return kept;
}

/* ------------------------------------------------------------------------- */
/* Greedy maximum-likelihood variant (the remark after the proof of Prop. 1):  */
/* each Bernoulli draw is replaced by its more likely outcome. Reading: keep   */
/* iff Re(d_j) > 1/2 (a tie rejects). Real Hermitian form.                     */
/* ------------------------------------------------------------------------- */
int64_t oracle_dpp_ldl_greedy_r64(int64_t n, double* A, int64_t ld,
                                  uint8_t* keep, double* pivots, double* logp) {
  double lp = 0.0;
  int64_t kept = 0;
  for (int64_t j = 0; j < n; ++j) {
    double d = A[j + j * ld];
    if (d > 0.5) {
      keep[j] = 1;
      ++kept;
    } else {
      keep[j] = 0;
      d -= 1.0;
      A[j + j * ld] = d;
    }
    pivots[j] = d;
    lp += log(fabs(d));
    for (int64_t i = j + 1; i < n; ++i) A[i + j * ld] /= d;
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      const double c = d * A[k + j * ld];
      for (int64_t i = k; i < n; ++i) A[i + k * ld] -= A[i + j * ld] * c;
    }
  }
  *logp = lp;
  return kept;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 (Theorem 2): elementary (projection) DPP sampling by k steps of */
/* left-looking, diagonally-pivoted Cholesky. K (real symmetric, an orthogonal */
/* projection of rank k) is copied into A (n x n, column-major, ld n) and     */
/* factored in place with symmetric row/column swaps; d holds the remaining   */
/* diagonal by position, perm the original index at each position.            */
/* Step j: S = sum over positions p >= j of max(d_p, 0) (= k - j in exact    */
/* arithmetic); the position t is the first p >= j whose running sum of       */
/* max(d, 0) exceeds u_j S (the last position with d > 0 if rounding leaves   */
/* none); positions j and t are swapped in A (rows and columns), d and perm;  */
/* A_jj = sqrt(d_j); then A[j+1:n, j] -= A[j+1:n, 0:j] A[j, 0:j]^T, the       */
/* column is divided by A_jj and each d_i loses A_ij^2.                       */
/* Outputs: sample[0:k] = perm[0:k] (selection order), chol (k x k, ld k) the */
/* lower-triangular Cholesky factor of K_Y in that order, logp = 2 sum_j      */
/* log A_jj (Theorem 2: P(Y) = product of the squared pivots). margin (k or   */
/* NULL) receives, per step, the distance of u_j S to the nearest running sum */
/* divided by S: where it is tiny, another summation order may pick the      */
/* neighbouring position. Returns 0, or -1 if a pivot was not positive.       */
/* ------------------------------------------------------------------------- */
int oracle_dpp_elementary_r64(int64_t n, const double* K, int64_t ldk, int64_t k,
                              const double* u, int64_t* sample, double* chol,
                              double* logp, double* margin) {
  double* A = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int bad = 0;
  double lp = 0.0;
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < n; ++i) A[i + c * n] = K[i + c * ldk];
  for (int64_t i = 0; i < n; ++i) {
    d[i] = A[i + i * n];
    perm[i] = i;
  }
  for (int64_t j = 0; j < k; ++j) {
    /* draw the position */
    double S = 0.0;
    for (int64_t p = j; p < n; ++p) S += d[p] > 0.0 ? d[p] : 0.0;
    const double target = u[j] * S;
    int64_t t = -1, last = -1;
    double acc = 0.0;
    for (int64_t p = j; p < n; ++p) {
      if (d[p] > 0.0) last = p;
      acc += d[p] > 0.0 ? d[p] : 0.0;
      if (acc > target) {
        t = p;
        break;
      }
    }
    if (t < 0) t = last >= 0 ? last : j;
    if (margin) {
      double m = fabs(target), run = 0.0;
      for (int64_t p = j; p < n; ++p) {
        run += d[p] > 0.0 ? d[p] : 0.0;
        const double dist = fabs(run - target);
        if (dist < m) m = dist;
      }
      margin[j] = S > 0.0 ? m / S : 0.0;
    }
    /* symmetric swap of positions j and t */
    if (t != j) {
      for (int64_t c = 0; c < n; ++c) {
        const double x = A[j + c * n];
        A[j + c * n] = A[t + c * n];
        A[t + c * n] = x;
      }
      for (int64_t i = 0; i < n; ++i) {
        const double x = A[i + j * n];
        A[i + j * n] = A[i + t * n];
        A[i + t * n] = x;
      }
      const double dx = d[j];
      d[j] = d[t];
      d[t] = dx;
      const int64_t px = perm[j];
      perm[j] = perm[t];
      perm[t] = px;
    }
    if (!(d[j] > 0.0)) bad = 1;
    const double ajj = sqrt(d[j] > 0.0 ? d[j] : 0.0);
    A[j + j * n] = ajj;
    lp += 2.0 * log(ajj);
    if (j == k - 1) break;
    /* new column (left-looking) and diagonal downdate */
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double v = A[i + j * n];
      for (int64_t s = 0; s < j; ++s) v -= A[i + s * n] * A[j + s * n];
      v /= ajj;
      A[i + j * n] = v;
      d[i] -= v * v;
    }
  }
  for (int64_t j = 0; j < k; ++j) {
    sample[j] = perm[j];
    for (int64_t i = 0; i < k; ++i) chol[i + j * k] = i >= j ? A[i + j * n] : 0.0;
  }
  *logp = lp;
  free(A);
  free(d);
  free(perm);
  return bad ? -1 : 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
