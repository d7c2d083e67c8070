/* Plain C restatement of the oracle's two leapfrog loops, for timing on the host cores.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests (cross-checked against oracle/online.py and
 * oracle/fine.py) and by the CPU-baseline / reference legs of bench.py; nothing in the product
 * links or calls it.  FP64, OpenMP over cells (ROM) or rows (fine grid), no blocking or fusion
 * beyond the steps below.
 *
 * oracle_rom_leapfrog: on-line stage of Algorithm alg1red (stage 2) without the Appendix D
 * correction.  Per step n, with U^1_i the cell's face unknowns stacked in its face order and
 * U^{m_i+1}_i = 0:
 *   r_n = sum_f q~_f^T u~_f                                        (Eq. solatrec, before the update)
 *   F^k_i = Gamma^k_i (U^{k+1}_i - U^k_i),  k = 1..m_i             (Eq. intrtstep_td)
 *   U^k_i <- 2 U^k_i - U^k_i,old + tau^2 Gamma-hat^k_i (F^k_i - F^{k-1}_i),  k = 2..m_i
 *   u~_f <- 2 u~_f - u~_f,old + tau^2 M_f^{-1} (sum_{i in f} F^1_i|_f - g~_f w(t_n))   (Eq. bdrytstep)
 * the face sums taken over the face's cells in ascending cell order.
 *
 * oracle_fine_leapfrog: u^{n+1} = 2 u^n - u^{n-1} + tau^2 B^{-1} (A u^n - g w(t_n)), r_n = q u^n
 * (Section 1, Eq. wave_fll), A and q in CSR.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Y (K x S) = G (K x K, row-major) X (K x S) */
static void block_product(const double *restrict G, const double *restrict X, double *restrict Y, int K, int S) {
  for (int r = 0; r < K; ++r) {
    double *y = Y + (size_t)r * S;
    for (int s = 0; s < S; ++s) y[s] = 0.0;
    const double *g = G + (size_t)r * K;
    for (int c = 0; c < K; ++c) {
      const double a = g[c];
      const double *x = X + (size_t)c * S;
      for (int s = 0; s < S; ++s) y[s] += a * x[s];
    }
  }
}

/* Sizes and layout (all row-major, sources fastest):
 *   cell_m[i], cell_K[i]; cell_face_ptr[n_cells+1] / cell_faces: the faces of cell i in order;
 *   face_M[f], face_row[n_faces+1]: first row of face f in the stacked face state;
 *   face_cell_ptr[n_faces+1] / face_cell / face_cell_off: the cells of face f (ascending) and the
 *     offset of f's block inside that cell's boundary vector;
 *   coef_off[i]: offset of cell i's blocks in gamma and gamma_hat (m_i blocks of K_i x K_i each);
 *   minv, minv_off[f]: M_f^{-1} (M_f x M_f);  state_off[i]: first row of cell i's hidden layers
 *     ((m_i - 1) K_i rows);  g: face rows x S;  q: R x face rows;  traces: n_steps x R x S.
 * Returns 0, or -1 when scratch memory cannot be had. */
int oracle_rom_leapfrog(int n_cells, int n_faces, int S, int R, const int32_t *cell_m, const int32_t *cell_K,
                        const int64_t *cell_face_ptr, const int32_t *cell_faces, const int32_t *face_M,
                        const int64_t *face_row, const int64_t *face_cell_ptr, const int32_t *face_cell,
                        const int32_t *face_cell_off, const double *gamma, const double *gamma_hat,
                        const int64_t *coef_off, const double *minv, const int64_t *minv_off,
                        const int64_t *state_off, const double *g, const double *q, const double *w,
                        double tau, int n_steps, double *traces) {
  const int64_t rows = face_row[n_faces];
  int64_t srows = 0, frows = 0;
  int maxK = 1, maxm = 1;
  int64_t *f1_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells + 1));
  if (!f1_off) return -1;
  for (int i = 0; i < n_cells; ++i) {
    f1_off[i] = frows;
    frows += cell_K[i];
    srows += (int64_t)(cell_m[i] - 1) * cell_K[i];
    if (cell_K[i] > maxK) maxK = cell_K[i];
    if (cell_m[i] > maxm) maxm = cell_m[i];
  }
  f1_off[n_cells] = frows;
  double *fu = (double *)calloc((size_t)(rows * S), sizeof(double));
  double *fo = (double *)calloc((size_t)(rows * S), sizeof(double));
  double *cu = (double *)calloc((size_t)(srows * S) + 1, sizeof(double));
  double *co = (double *)calloc((size_t)(srows * S) + 1, sizeof(double));
  double *f1 = (double *)calloc((size_t)(frows * S), sizeof(double));
  int nt = oracle_threads();
  const size_t per = (size_t)(2 * maxm + 2) * maxK * S + (size_t)maxK * S;
  double *scr = (double *)malloc(sizeof(double) * per * (size_t)nt);
  if (!fu || !fo || !cu || !co || !f1 || !scr) {
    free(f1_off); free(fu); free(fo); free(cu); free(co); free(f1); free(scr);
    return -1;
  }
  const double t2 = tau * tau;
  for (int n = 0; n < n_steps; ++n) {
    double *out = traces + (size_t)n * R * S;
    for (int r = 0; r < R; ++r) {
      double *o = out + (size_t)r * S;
      for (int s = 0; s < S; ++s) o[s] = 0.0;
      for (int64_t j = 0; j < rows; ++j) {      /* rows of q are mostly zero: skip those terms */
        const double a = q[(size_t)r * rows + j];
        if (a == 0.0) continue;
        const double *x = fu + (size_t)j * S;
        for (int s = 0; s < S; ++s) o[s] += a * x[s];
      }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n_cells; ++i) {
#ifdef _OPENMP
      double *ws = scr + per * (size_t)omp_get_thread_num();
#else
      double *ws = scr;
#endif
      const int K = cell_K[i], m = cell_m[i];
      const size_t KS = (size_t)K * S;
      double *U = ws;                      /* U^1..U^{m+1}: (m+1) K x S */
      double *F = U + (size_t)(m + 1) * KS; /* F^1..F^m */
      double *D = F + (size_t)m * KS;       /* one K x S work block */
      int64_t o = 0;
      for (int64_t e = cell_face_ptr[i]; e < cell_face_ptr[i + 1]; ++e) {
        const int f = cell_faces[e];
        memcpy(U + (size_t)o * S, fu + (size_t)face_row[f] * S, sizeof(double) * (size_t)face_M[f] * S);
        o += face_M[f];
      }
      const double *cs = cu + (size_t)state_off[i] * S;
      double *cso = co + (size_t)state_off[i] * S;
      if (m > 1) memcpy(U + KS, cs, sizeof(double) * (size_t)(m - 1) * KS);
      memset(U + (size_t)m * KS, 0, sizeof(double) * KS);
      for (int k = 0; k < m; ++k) {
        for (size_t e = 0; e < KS; ++e) D[e] = U[(size_t)(k + 1) * KS + e] - U[(size_t)k * KS + e];
        block_product(gamma + coef_off[i] + (size_t)k * K * K, D, F + (size_t)k * KS, K, S);
      }
      memcpy(f1 + (size_t)f1_off[i] * S, F, sizeof(double) * KS);
      for (int k = 1; k < m; ++k) {
        for (size_t e = 0; e < KS; ++e) D[e] = F[(size_t)k * KS + e] - F[(size_t)(k - 1) * KS + e];
        double *A = U + (size_t)m * KS;    /* reuse the zero block as the acceleration */
        block_product(gamma_hat + coef_off[i] + (size_t)k * K * K, D, A, K, S);
        const double *now = cs + (size_t)(k - 1) * KS;
        double *old = cso + (size_t)(k - 1) * KS;
        for (size_t e = 0; e < KS; ++e) old[e] = 2.0 * now[e] - old[e] + t2 * A[e];
      }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int f = 0; f < n_faces; ++f) {
#ifdef _OPENMP
      double *ws = scr + per * (size_t)omp_get_thread_num();
#else
      double *ws = scr;
#endif
      const int M = face_M[f];
      double *sum = ws, *a = ws + (size_t)M * S;
      memset(sum, 0, sizeof(double) * (size_t)M * S);
      for (int64_t e = face_cell_ptr[f]; e < face_cell_ptr[f + 1]; ++e) {
        const double *src = f1 + (size_t)(f1_off[face_cell[e]] + face_cell_off[e]) * S;
        for (size_t x = 0; x < (size_t)M * S; ++x) sum[x] += src[x];
      }
      const double *gf = g + (size_t)face_row[f] * S;
      for (size_t x = 0; x < (size_t)M * S; ++x) sum[x] -= gf[x] * w[n];
      block_product(minv + minv_off[f], sum, a, M, S);
      const double *now = fu + (size_t)face_row[f] * S;
      double *old = fo + (size_t)face_row[f] * S;
      for (size_t x = 0; x < (size_t)M * S; ++x) old[x] = 2.0 * now[x] - old[x] + t2 * a[x];
    }
    double *t;
    t = fu; fu = fo; fo = t;
    t = cu; cu = co; co = t;
  }
  free(f1_off); free(fu); free(fo); free(cu); free(co); free(f1); free(scr);
  return 0;
}

/* A (N x N) and q (R x N) in CSR; B the diagonal; g: N x S; traces: n_steps x R x S. */
int oracle_fine_leapfrog(int64_t N, int S, int R, const int64_t *a_ptr, const int64_t *a_col, const double *a_val,
                         const double *B, const double *g, const int64_t *q_ptr, const int64_t *q_col,
                         const double *q_val, const double *w, double tau, int n_steps, double *traces) {
  double *u = (double *)calloc((size_t)(N * S), sizeof(double));
  double *uo = (double *)calloc((size_t)(N * S), sizeof(double));
  if (!u || !uo) { free(u); free(uo); return -1; }
  const double t2 = tau * tau;
  for (int n = 0; n < n_steps; ++n) {
    double *out = traces + (size_t)n * R * S;
    for (int r = 0; r < R; ++r)
      for (int s = 0; s < S; ++s) {
        double acc = 0.0;
        for (int64_t e = q_ptr[r]; e < q_ptr[r + 1]; ++e) acc += q_val[e] * u[(size_t)q_col[e] * S + s];
        out[(size_t)r * S + s] = acc;
      }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      for (int s = 0; s < S; ++s) {
        double au = 0.0;
        for (int64_t e = a_ptr[i]; e < a_ptr[i + 1]; ++e) au += a_val[e] * u[(size_t)a_col[e] * S + s];
        const size_t x = (size_t)i * S + s;
        uo[x] = 2.0 * u[x] - uo[x] + t2 * (au - g[x] * w[n]) / B[i];
      }
    }
    double *t = u; u = uo; uo = t;
  }
  free(u); free(uo);
  return 0;
}
