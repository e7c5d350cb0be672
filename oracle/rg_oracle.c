/*
 * rg_oracle.c -- plain, slow, single-threaded FP64 rank-Greville (TEST INFRASTRUCTURE).
 *
 * This file is the CPU oracle that the CUDA path is checked against. Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it. It shares no code,
 * header or constant with the CUDA library.
 *
 * What it computes: Algorithm 1 ("UpdateLeastSquares", Section 3), one row at a time,
 * in the paper's order and notation, with plain left-to-right loops and no BLAS:
 *
 *   gamma   = Ct Gamma                              (Eq. label_eq_gnplusoneproj)
 *   Gamma_r = Gamma - C^T gamma                     (rejection, Section 2.1)
 *   if Gamma_r != 0 (threshold test, Eq. label_eq_eps):
 *       K   = Gamma_r / ||Gamma_r||^2               (Theorem 4)
 *       C   = [C ; Gamma^T]                         (Eq. label_eq_Cnplusone_indep_update)
 *       Ct  = [Ct - gamma K^T ; K^T]                (Eq. label_eq_Cnplusonetilde_indep_update)
 *       P^-1 = diag(P^-1, 1)                        (Eq. label_eq_Pnplusoneinv_indep_update)
 *   else:
 *       zeta = P^-1 gamma                           (Eq. label_eq_znplusone)
 *       K    = Ct^T zeta / (1 + gamma^T zeta)       (Theorem 5)
 *       P^-1 = P^-1 - zeta zeta^T / (1 + gamma^T zeta)  (Eq. label_eq_Pnplusoneinv_lindep_update)
 *   X = X + K (y - Gamma^T X)                       (Eq. label_eq_recursive_least_squares)
 *
 * Orthonormal variant (Section 2.2, Eqs. label_eq_Cnplusone_indep_update_orthog,
 * label_eq_Cnplusonetilde_indep_update_orthog, label_eq_Pnplusoneinv_indep_update_orthog
 * with alpha = 1 / ||Gamma_r||): an independent row instead stores
 *       C    = [C ; alpha Gamma_r^T],   Ct = [Ct ; Gamma_r^T / (alpha ||Gamma_r||^2)]
 *       P^-1 = [[P^-1, -alpha zeta], [-alpha zeta^T, alpha^2 (1 + gamma^T zeta)]],
 *              zeta = P^-1 gamma
 * (so the rows of C are orthonormal and Ct = C); K, the dependent case and the X update
 * are unchanged, since Theorems 4 and 5 hold for any rank factorization. The orthogonal
 * variant of the same section takes alpha = 1: C stores the raw rejections (orthogonal,
 * not normalised) and Ct the same rows divided by their squared norms.
 *
 * Readings of the paper taken here (each listed in the design notes):
 *  - Threshold (Eq. label_eq_eps). Two modes. REL (default): independent iff
 *    ||Gamma_r|| > eps ||Gamma||. PAPER: dependent iff ||Gamma_r|| < eps or
 *    ||Gamma_r|| < eps ||Gamma||. Both are evaluated in squared form in FP64
 *    (s = ||Gamma_r||^2, t = ||Gamma||^2; monotone, so equivalent up to rounding).
 *  - eps = tol when tol > 0, else the paper's default (m^2 r + m r + m) eps_M with r the
 *    rank before the row and eps_M = 2^-52 (Section 4.2 states eps_M = 2.22e-16).
 *  - P^-1 is updated as a full matrix exactly as printed, with no symmetrisation.
 *  - A row that would make the rank exceed r_max stops the stream with status 4
 *    (capacity) and leaves the state as it was before that row.
 *
 * The `mutation` argument of rgo_solve_mut plants one deliberate mistake (a dropped
 * term, a wrong sign, a wrong index or a transposed operand) so that the tests can show
 * that the oracle's pins catch it. rgo_solve always runs with mutation 0.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define RGO_TEST_REL 0
#define RGO_TEST_PAPER 2

typedef struct {
  int64_t m, r_max, r;
  double tol;
  int test_mode;
  int mutation;
  int variant;  /* 0: general (Algorithm 1), 1: orthonormal, 2: orthogonal (Section 2.2) */
  double *C;    /* r_max x m, row i = i-th basis row (a selected input row)      */
  double *Ct;   /* r_max x m, row i = i-th dual basis row                          */
  double *Pinv; /* r_max x r_max, leading r x r block is P^-1 = (B^T B)^-1         */
  double *X;    /* m, current minimum-norm least-squares solution                  */
  double *gamma, *Gr, *zeta, *K;
  int64_t *basis_rows;
  int64_t rows_seen;
} rgo_state;

static int rgo_alloc(rgo_state *st, int64_t m, int64_t r_max, double tol, int test_mode) {
  memset(st, 0, sizeof(*st));
  st->m = m;
  st->r_max = r_max;
  st->tol = tol;
  st->test_mode = test_mode;
  st->C = (double *)calloc((size_t)(r_max * m), sizeof(double));
  st->Ct = (double *)calloc((size_t)(r_max * m), sizeof(double));
  st->Pinv = (double *)calloc((size_t)(r_max * r_max + 1), sizeof(double));
  st->X = (double *)calloc((size_t)m, sizeof(double));
  st->gamma = (double *)calloc((size_t)(r_max + 1), sizeof(double));
  st->zeta = (double *)calloc((size_t)(r_max + 1), sizeof(double));
  st->Gr = (double *)calloc((size_t)m, sizeof(double));
  st->K = (double *)calloc((size_t)m, sizeof(double));
  st->basis_rows = (int64_t *)calloc((size_t)(r_max + 1), sizeof(int64_t));
  if (!st->C || !st->Ct || !st->Pinv || !st->X || !st->gamma || !st->zeta || !st->Gr ||
      !st->K || !st->basis_rows)
    return 2;
  return 0;
}

static void rgo_release(rgo_state *st) {
  free(st->C); free(st->Ct); free(st->Pinv); free(st->X); free(st->gamma);
  free(st->zeta); free(st->Gr); free(st->K); free(st->basis_rows);
  memset(st, 0, sizeof(*st));
}

#define CM(i, c) st->C[(i) * st->m + (c)]
#define CT(i, c) st->Ct[(i) * st->m + (c)]
#define PI(i, j) st->Pinv[(i) * st->r_max + (j)]

/* Threshold of Eq. label_eq_eps in squared form: returns 1 iff the row is independent. */
static int rgo_is_independent(const rgo_state *st, double s, double t) {
  double eps = st->tol;
  if (!(eps > 0.0)) {
    double m = (double)st->m, r = (double)st->r;
    eps = (m * m * r + m * r + m) * DBL_EPSILON;
  }
  double e2 = eps * eps;
  if (st->test_mode == RGO_TEST_PAPER) return !(s < e2 || s < e2 * t);
  return s > e2 * t;
}

/* One call of UpdateLeastSquares(Gamma, y, X, C, Ct, P^-1). Returns 1 if the row was
 * independent, 0 if dependent, -4 on capacity overflow (state untouched). */
static int rgo_update(rgo_state *st, const double *G, double y) {
  const int64_t m = st->m, r = st->r;
  const int mut = st->mutation;
  /* gamma <- Ct Gamma */
  for (int64_t i = 0; i < r; ++i) {
    double acc = 0.0;
    for (int64_t c = 0; c < m; ++c) acc += (mut == 5 ? CM(i, c) : CT(i, c)) * G[c];
    st->gamma[i] = acc;
  }
  /* Gamma_r <- Gamma - C^T gamma */
  for (int64_t c = 0; c < m; ++c) {
    double acc = 0.0;
    for (int64_t i = 0; i < r; ++i) acc += CM(i, c) * st->gamma[i];
    st->Gr[c] = (mut == 1 ? G[c] + acc : G[c] - acc);
  }
  double s = 0.0, t = 0.0;
  for (int64_t c = 0; c < m; ++c) {
    s += st->Gr[c] * st->Gr[c];
    t += G[c] * G[c];
  }
  int indep = rgo_is_independent(st, s, t);
  if (indep && (st->variant == 1 || st->variant == 2)) {
    if (r >= st->r_max) return -4;
    /* orthonormal: alpha = 1 / ||Gamma_r||; orthogonal: alpha = 1 (the raw rejection) */
    const double alpha = (st->variant == 2) ? 1.0 : 1.0 / sqrt(s);
    /* zeta <- P^-1 gamma (for the bordered P^-1) */
    for (int64_t i = 0; i < r; ++i) {
      double acc = 0.0;
      for (int64_t j = 0; j < r; ++j) acc += PI(i, j) * st->gamma[j];
      st->zeta[i] = acc;
    }
    double gz = 0.0;
    for (int64_t i = 0; i < r; ++i) gz += st->gamma[i] * st->zeta[i];
    /* K <- Gamma_r / ||Gamma_r||^2 */
    for (int64_t c = 0; c < m; ++c) st->K[c] = st->Gr[c] / s;
    /* C <- [C ; alpha Gamma_r^T], Ct <- [Ct ; Gamma_r^T / (alpha ||Gamma_r||^2)] */
    for (int64_t c = 0; c < m; ++c) {
      CM(r, c) = alpha * st->Gr[c];
      CT(r, c) = st->Gr[c] / (alpha * s);
    }
    /* P^-1 <- [[P^-1, -alpha zeta], [-alpha zeta^T, alpha^2 (1 + gamma^T zeta)]] */
    const double sg = (mut == 9 ? 1.0 : -1.0);
    for (int64_t i = 0; i < r; ++i) {
      PI(i, r) = sg * alpha * st->zeta[i];
      PI(r, i) = sg * alpha * st->zeta[i];
    }
    PI(r, r) = (mut == 8 ? 1.0 + gz : alpha * alpha * (1.0 + gz));
    st->basis_rows[r] = st->rows_seen;
    st->r = r + 1;
  } else if (indep) {
    if (r >= st->r_max) return -4;
    /* K <- Gamma_r / ||Gamma_r||^2 */
    for (int64_t c = 0; c < m; ++c) st->K[c] = st->Gr[c] / s;
    /* Ct <- [Ct - gamma K^T ; K^T] */
    for (int64_t i = 0; i < r; ++i)
      for (int64_t c = 0; c < m; ++c)
        CT(i, c) -= (mut == 2 ? 0.0 : st->gamma[i] * st->K[c]);
    for (int64_t c = 0; c < m; ++c) CT(r, c) = st->K[c];
    /* C <- [C ; Gamma^T] */
    for (int64_t c = 0; c < m; ++c) CM(r, c) = G[c];
    /* P^-1 <- diag(P^-1, 1) */
    for (int64_t i = 0; i < r; ++i) {
      PI(i, r) = 0.0;
      PI(r, i) = 0.0;
    }
    PI(r, r) = 1.0;
    st->basis_rows[r] = st->rows_seen;
    st->r = r + 1;
  } else {
    /* zeta <- P^-1 gamma */
    for (int64_t i = 0; i < r; ++i) {
      double acc = 0.0;
      for (int64_t j = 0; j < r; ++j) acc += PI(i, j) * st->gamma[mut == 6 ? (j + 1) % r : j];
      st->zeta[i] = acc;
    }
    double gz = 0.0;
    for (int64_t i = 0; i < r; ++i) gz += st->gamma[i] * st->zeta[i];
    double d = (mut == 3 ? gz : 1.0 + gz);
    /* K <- Ct^T zeta / (1 + gamma^T zeta) */
    for (int64_t c = 0; c < m; ++c) {
      double acc = 0.0;
      for (int64_t i = 0; i < r; ++i) acc += CT(i, c) * st->zeta[i];
      st->K[c] = acc / d;
    }
    /* P^-1 <- P^-1 - zeta zeta^T / (1 + gamma^T zeta) */
    for (int64_t i = 0; i < r; ++i)
      for (int64_t j = 0; j < r; ++j)
        PI(i, j) -= (mut == 4 ? 0.0 : st->zeta[i] * st->zeta[j] / d);
  }
  /* X <- X + K (y - Gamma^T X) */
  double gx = 0.0;
  for (int64_t c = 0; c < m; ++c) gx += G[c] * st->X[c];
  double dy = (mut == 7 ? y + gx : y - gx);
  for (int64_t c = 0; c < m; ++c) st->X[c] += st->K[c] * dy;
  st->rows_seen += 1;
  return indep;
}

/*
 * Solve one stream from scratch (Corollary label_th_full_lstsq): feed the n rows of
 * A (n x m, row-major) with targets Y in order.
 *
 * Outputs (any may be NULL): X (m), rank_out (1), basis_rows (r_max; the input row
 * index of each basis row), indep (n bytes, 1 = row grew the rank), Ct_out (r_max x m),
 * Pinv_out (r_max x r_max), C_out (r_max x m), rows_done (1).
 * Returns 0, 1 (bad arguments), 2 (out of memory) or 4 (rank would exceed r_max; rows
 * before the offending row are applied, rows_done says how many).
 */
int rgo_solve_var(int64_t n, int64_t m, const double *A, const double *Y, double tol,
                  int test_mode, int64_t r_max, int variant, int mutation, double *X,
                  int64_t *rank_out, int64_t *basis_rows, uint8_t *indep, double *Ct_out,
                  double *Pinv_out, double *C_out, int64_t *rows_done) {
  if (n < 0 || m <= 0 || (n > 0 && (!A || !Y)) || tol != tol) return 1;
  if (r_max <= 0) r_max = m;
  if (r_max > m) r_max = m;
  rgo_state st;
  if (rgo_alloc(&st, m, r_max, tol, test_mode)) {
    rgo_release(&st);
    return 2;
  }
  st.mutation = mutation;
  st.variant = variant;
  int status = 0;
  int64_t i = 0;
  for (; i < n; ++i) {
    int res = rgo_update(&st, A + i * m, Y[i]);
    if (res == -4) {
      status = 4;
      break;
    }
    if (indep) indep[i] = (uint8_t)res;
  }
  if (rows_done) *rows_done = i;
  if (X) memcpy(X, st.X, (size_t)m * sizeof(double));
  if (rank_out) *rank_out = st.r;
  if (basis_rows) memcpy(basis_rows, st.basis_rows, (size_t)st.r * sizeof(int64_t));
  if (Ct_out) memcpy(Ct_out, st.Ct, (size_t)(st.r * m) * sizeof(double));
  if (C_out) memcpy(C_out, st.C, (size_t)(st.r * m) * sizeof(double));
  if (Pinv_out) {
    for (int64_t a = 0; a < st.r; ++a)
      for (int64_t b = 0; b < st.r; ++b) Pinv_out[a * st.r + b] = st.Pinv[a * st.r_max + b];
  }
  rgo_release(&st);
  return status;
}

int rgo_solve_mut(int64_t n, int64_t m, const double *A, const double *Y, double tol,
                  int test_mode, int64_t r_max, int mutation, double *X, int64_t *rank_out,
                  int64_t *basis_rows, uint8_t *indep, double *Ct_out, double *Pinv_out,
                  double *C_out, int64_t *rows_done) {
  return rgo_solve_var(n, m, A, Y, tol, test_mode, r_max, 0, mutation, X, rank_out, basis_rows,
                       indep, Ct_out, Pinv_out, C_out, rows_done);
}

int rgo_solve(int64_t n, int64_t m, const double *A, const double *Y, double tol,
              int test_mode, int64_t r_max, double *X, int64_t *rank_out,
              int64_t *basis_rows, uint8_t *indep, double *Ct_out, double *Pinv_out,
              double *C_out, int64_t *rows_done) {
  return rgo_solve_mut(n, m, A, Y, tol, test_mode, r_max, 0, X, rank_out, basis_rows, indep,
                       Ct_out, Pinv_out, C_out, rows_done);
}

/*
 * Pseudoinverse update (Theorems label_th_pinv_indep and label_th_pinv_lindep): feed the
 * n rows of A (n x m, row-major) in order and keep A_n^+ (m x n) explicitly. Per row,
 * with the general factorization of Algorithm 1 before the row (C, Ct, P^-1 and B_n):
 *   gamma = Ct Gamma, zeta = P^-1 gamma, b = B_n zeta (Eq. label_eq_znplusone),
 *   K = Gamma_r / ||Gamma_r||^2 (independent) or Ct^T zeta / (1 + gamma^T zeta)
 *   (dependent), exactly the K of Algorithm 1 (rgo_update forms it),
 *   A_{n+1}^+ = [A_n^+ - K b^T, K],
 * and B grows as the factorizations of the two theorems' proofs state:
 *   dependent: B_{n+1} = [B_n; gamma^T]; independent: B_{n+1} = [[B_n, 0], [0, 1]].
 * Output Apinv (m x n row-major: Apinv[c * n + i] is entry (c, i) of A^+); rank_out and
 * indep (n) may be NULL. mutation plants a mistake for the pins: 10 drops the -K b^T
 * term, 11 adds it with the wrong sign, 12 appends gamma^T to B for an independent row.
 * Returns 0, 1 (bad arguments), 2 (out of memory) or 4 (a row would make the rank exceed m).
 */
int rgo_pinv_mut(int64_t n, int64_t m, const double *A, double tol, int test_mode, int mutation,
                 double *Apinv, int64_t *rank_out, uint8_t *indep) {
  if (n < 0 || m <= 0 || (n > 0 && !A) || !Apinv || tol != tol) return 1;
  const int64_t r_max = m;
  rgo_state sto;
  rgo_state *st = &sto;
  double *Bm = (double *)calloc((size_t)((n > 0 ? n : 1) * r_max), sizeof(double));
  double *gam = (double *)calloc((size_t)r_max + 1, sizeof(double));
  double *zet = (double *)calloc((size_t)r_max + 1, sizeof(double));
  double *b = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (rgo_alloc(st, m, r_max, tol, test_mode) || !Bm || !gam || !zet || !b) {
    rgo_release(st);
    free(Bm); free(gam); free(zet); free(b);
    return 2;
  }
  for (int64_t e = 0; e < m * n; ++e) Apinv[e] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double *G = A + i * m;
    const int64_t r = st->r;
    /* gamma = Ct Gamma, zeta = P^-1 gamma, b = B_n zeta (state before the row) */
    for (int64_t k = 0; k < r; ++k) {
      double acc = 0.0;
      for (int64_t c = 0; c < m; ++c) acc += CT(k, c) * G[c];
      gam[k] = acc;
    }
    for (int64_t k = 0; k < r; ++k) {
      double acc = 0.0;
      for (int64_t l = 0; l < r; ++l) acc += st->Pinv[k * st->r_max + l] * gam[l];
      zet[k] = acc;
    }
    for (int64_t j = 0; j < i; ++j) {
      double acc = 0.0;
      for (int64_t k = 0; k < r; ++k) acc += Bm[j * r_max + k] * zet[k];
      b[j] = acc;
    }
    /* Algorithm 1 on the row: decides it, forms K and updates C, Ct, P^-1 */
    int res = rgo_update(st, G, 0.0);
    if (res < 0) { /* rank would exceed m: only a breakdown of the rank test gets here */
      rgo_release(st);
      free(Bm); free(gam); free(zet); free(b);
      return 4;
    }
    if (indep) indep[i] = (uint8_t)res;
    /* A^+ <- [A^+ - K b^T, K] */
    for (int64_t c = 0; c < m; ++c) {
      const double kc = st->K[c];
      for (int64_t j = 0; j < i; ++j) {
        if (mutation == 10) break;
        Apinv[c * n + j] += (mutation == 11 ? kc * b[j] : -kc * b[j]);
      }
      Apinv[c * n + i] = kc;
    }
    /* B_{n+1} */
    if (res == 1 && mutation != 12) {
      for (int64_t k = 0; k < r_max; ++k) Bm[i * r_max + k] = 0.0;
      Bm[i * r_max + r] = 1.0;
    } else {
      for (int64_t k = 0; k < r_max; ++k) Bm[i * r_max + k] = (k < r) ? gam[k] : 0.0;
    }
  }
  if (rank_out) *rank_out = st->r;
  rgo_release(st);
  free(Bm); free(gam); free(zet); free(b);
  return 0;
}

int rgo_pinv(int64_t n, int64_t m, const double *A, double tol, int test_mode, double *Apinv,
             int64_t *rank_out, uint8_t *indep) {
  return rgo_pinv_mut(n, m, A, tol, test_mode, 0, Apinv, rank_out, indep);
}

/*
 * Batched form: B independent streams in the packed layout (instance b: rows
 * A[elem_off[b] .. elem_off[b+1]) as n_b x m_b, targets Y[row_off[b] ..], solution
 * X[x_off[b] .. x_off[b] + m_b)). Instances run in parallel over `threads` OpenMP
 * threads (<= 0: all available). ranks (B) and status (B) may be NULL.
 */
/*
 * Batched form: B independent streams (OpenMP over instances, one thread per instance).
 * Instance b's rows are A[elem_off[b] .. elem_off[b+1]) viewed as n_b x m_b row-major with
 * n_b = row_off[b+1] - row_off[b], m_b = x_off[b+1] - x_off[b]; its targets are
 * Y[row_off[b] ..]. Outputs: X at x_off[b], ranks[b], status[b] and, when indep is not
 * NULL, the per-row flags at indep[row_off[b] ..] (rows after a capacity stop keep 0xFF).
 * variant as rgo_solve_var. Each instance runs rgo_solve_var unchanged, with r_max = m_b.
 */
int rgo_solve_batch_var(int64_t B, const int64_t *row_off, const int64_t *elem_off,
                        const int64_t *x_off, const double *A, const double *Y, double tol,
                        int test_mode, int variant, int threads, double *X, int64_t *ranks,
                        int *status, uint8_t *indep) {
  if (B < 0 || !row_off || !elem_off || !x_off) return 1;
  int bad = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
  for (int64_t b = 0; b < B; ++b) {
    int64_t n = row_off[b + 1] - row_off[b];
    int64_t m = x_off[b + 1] - x_off[b];
    int64_t rk = 0;
    int st = 1;
    uint8_t *ind = indep ? indep + row_off[b] : NULL;
    if (ind)
      for (int64_t i = 0; i < n; ++i) ind[i] = 0xFF;
    if (m > 0 && (elem_off[b + 1] - elem_off[b]) == n * m)
      st = rgo_solve_var(n, m, A + elem_off[b], Y + row_off[b], tol, test_mode, m, variant, 0,
                         X + x_off[b], &rk, NULL, ind, NULL, NULL, NULL, NULL);
    if (ranks) ranks[b] = rk;
    if (status) status[b] = st;
    bad |= (st != 0);
  }
  return bad ? 1 : 0;
}

int rgo_solve_batch(int64_t B, const int64_t *row_off, const int64_t *elem_off,
                    const int64_t *x_off, const double *A, const double *Y, double tol,
                    int test_mode, int threads, double *X, int64_t *ranks, int *status) {
  return rgo_solve_batch_var(B, row_off, elem_off, x_off, A, Y, tol, test_mode, 0, threads, X,
                             ranks, status, NULL);
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int rgo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
