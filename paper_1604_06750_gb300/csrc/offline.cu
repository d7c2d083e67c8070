// Off-line stage on the GPU, FP64 (Algorithm alg1red, stage 1), batched over cells.
//
// Per cell i (cells are independent, Section 4.2):
//   C   = P^Gamma S_i, block-diagonal face bases on the boundary rows (Section 4.1);
//   V_0 = B-orthonormal basis of B^{-1} C                         (zero-power block, Remark Sinsubspace)
//   V_j = B-orthonormal basis of (A + sB)^{-1} B V_{j-1}, made B-orthogonal to V_0..V_{j-1}
//         by two passes of block Gram-Schmidt (Eq. npks, pencil form), j = 1..m-1;
//         the shifted solves use Jacobi-preconditioned CG on -(A + sB) (SPD for s < 0), batched
//         over (cell, column);
//   A^m = V^T A V, S^m = V^T C                                       (Eq. tfprj, B^m = I)
//   block Lanczos on (A^m, S^m) with full reorthogonalisation        (Appendix C, Eq. NtDtri)
//   Gamma^k, Gamma-hat^k by the symmetric change of variables         (Eq. GammaTrans)
// Dense per-cell blocks are row-major N_i x K_i with a common row stride W; cells of a chunk are
// stacked along the rows.  Host C++ builds the split cell matrices and the face bases; the face
// masses M_f = sum (Gamma-hat^1_{i,f})^{-1} (Eq. bdrytstep) and the Appendix D data are
// assembled on the host from the device results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "cuda_util.h"

namespace mss {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int cell_of_row(const int64_t *row0, int nc, int64_t r) {
  int lo = 0, hi = nc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row0[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// X[r][j] = (r < K_c) ? Cb_c[r][j] / b_r : 0, j < Kt_c; zero elsewhere in the stride.
__global__ void k_expand_c(double *X, const double *Cb, const int64_t *cb_off, const int64_t *row0, const int32_t *Kb,
                           const int32_t *Kt, const double *B, int nc, int64_t rows, int W, int scale_by_binv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * W) return;
  const int64_t r = i / W;
  const int j = (int)(i - r * W);
  const int c = cell_of_row(row0, nc, r);
  const int64_t lr = r - row0[c];
  double v = 0.0;
  if (j < Kt[c] && lr < Kb[c]) {
    v = Cb[cb_off[c] + lr * Kt[c] + j];
    if (scale_by_binv) v /= B[r];
  }
  X[i] = v;
}

// Y = op(X) row-wise: mode 0: Y = A X; mode 1: Y = -(A + s B) X; mode 2: Y = B X.
__global__ void k_spmm(double *Y, const double *X, const int64_t *ptr, const int64_t *col, const double *val,
                       const double *B, double s, const int64_t *row0, const int32_t *Kt, int nc, int64_t rows, int W,
                       int mode) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * W) return;
  const int64_t r = i / W;
  const int j = (int)(i - r * W);
  const int c = cell_of_row(row0, nc, r);
  if (j >= Kt[c]) { Y[i] = 0.0; return; }
  if (mode == 2) { Y[i] = B[r] * X[i]; return; }
  double acc = 0.0;
  for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) acc += val[k] * X[col[k] * W + j];
  if (mode == 1) acc = -(acc + s * B[r] * X[i]);
  Y[i] = acc;
}

// out[c*W + j] = sum_{r in cell c} X[r][j] * Y[r][j] (* B[r] if B); optionally out2 = sum X^2.
__global__ void k_coldot(double *out, double *out2, const double *X, const double *Y, const double *B, const int64_t *row0,
                         const int32_t *Kt, int W) {
  const int c = blockIdx.x;
  const int64_t r0 = row0[c], r1 = row0[c + 1];
  for (int j = threadIdx.x; j < W; j += blockDim.x) {
    double a = 0.0, a2 = 0.0;
    if (j < Kt[c]) {
      for (int64_t r = r0; r < r1; ++r) {
        const double x = X[r * W + j];
        const double y = Y[r * W + j];
        a += (B ? B[r] : 1.0) * x * y;
        if (out2) a2 += x * x;
      }
    }
    out[(int64_t)c * W + j] = a;
    if (out2) out2[(int64_t)c * W + j] = a2;
  }
}

// CG pieces (per (cell, column) scalars in [c*W + j]).
__global__ void k_cg_init(double *y, double *r, double *z, double *p, const double *b, const double *dinv, const int64_t *row0,
                          const int32_t *Kt, int nc, int64_t rows, int W) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * W) return;
  const int64_t row = i / W;
  y[i] = 0.0;
  r[i] = b[i];
  z[i] = b[i] * dinv[row];
  p[i] = z[i];
}

__global__ void k_cg_xr(double *y, double *r, double *z, const double *p, const double *q, const double *dinv,
                        const double *rz, const double *pq, const int64_t *row0, int nc, int64_t rows, int W) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * W) return;
  const int64_t row = i / W;
  const int j = (int)(i - row * W);
  const int c = cell_of_row(row0, nc, row);
  const double num = rz[(int64_t)c * W + j], den = pq[(int64_t)c * W + j];
  const double al = (den > 0.0 && num > 0.0) ? num / den : 0.0;
  y[i] += al * p[i];
  r[i] -= al * q[i];
  z[i] = r[i] * dinv[row];
}

__global__ void k_cg_p(double *p, const double *z, const double *rz_new, const double *rz_old, const int64_t *row0, int nc,
                       int64_t rows, int W) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * W) return;
  const int64_t row = i / W;
  const int j = (int)(i - row * W);
  const int c = cell_of_row(row0, nc, row);
  const double o = rz_old[(int64_t)c * W + j];
  const double be = o > 0.0 ? rz_new[(int64_t)c * W + j] / o : 0.0;
  p[i] = z[i] + be * p[i];
}

// max over (cell, column) of rr / bb (squared relative residual); single block.
__global__ void k_maxratio(double *out, const double *rr, const double *bb, const int32_t *Kt, int nc, int W) {
  __shared__ double sm[kThreads];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < (int64_t)nc * W; i += blockDim.x) {
    const int c = (int)(i / W), j = (int)(i - (int64_t)c * W);
    if (j < Kt[c] && bb[i] > 0.0) m = fmax(m, rr[i] / bb[i]);
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// Per cell: G = sum_r P[r][a] Q[r][b] (w[r]), a < na, b < nb (na = nb = Kt_c), written at G + c*W*W (ld W).
// Tiles of 16 x 16 outputs, rows streamed through shared memory 32 at a time.
__global__ void k_gram(double *G, const double *P, const double *Q, const double *w, const int64_t *row0, const int32_t *Kt,
                       int W) {
  const int c = blockIdx.x;
  const int K = Kt[c];
  const int a0 = blockIdx.y * 16, b0 = blockIdx.z * 16;
  if (a0 >= K || b0 >= K) return;
  __shared__ double Ps[32][17], Qs[32][17];
  const int ta = threadIdx.x / 16, tb = threadIdx.x % 16;
  double acc = 0.0;
  const int64_t r0 = row0[c], r1 = row0[c + 1];
  for (int64_t rb = r0; rb < r1; rb += 32) {
    for (int t = threadIdx.x; t < 32 * 16; t += blockDim.x) {
      const int rr = t / 16, cc = t % 16;
      const int64_t r = rb + rr;
      const bool ok = r < r1;
      const double wr = (ok && w) ? w[r] : 1.0;
      Ps[rr][cc] = (ok && a0 + cc < K) ? P[r * W + a0 + cc] * wr : 0.0;
      Qs[rr][cc] = (ok && b0 + cc < K) ? Q[r * W + b0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) acc += Ps[rr][ta] * Qs[rr][tb];
    __syncthreads();
  }
  if (a0 + ta < K && b0 + tb < K) G[(int64_t)c * W * W + (int64_t)(a0 + ta) * W + b0 + tb] = acc;
}

// X[r][b] (op)= sum_a P[r][a] G_c[a][b] (trans: G_c[b][a]); op 0: assign, 1: subtract.
__global__ void k_rowmul(double *X, const double *P, const double *G, int trans, int op, const int64_t *row0,
                         const int32_t *Kt, int nc, int64_t rows, int W) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * W) return;
  const int64_t r = i / W;
  const int b = (int)(i - r * W);
  const int c = cell_of_row(row0, nc, r);
  const int K = Kt[c];
  if (b >= K) { if (op == 0) X[i] = 0.0; return; }
  const double *Gc = G + (int64_t)c * W * W;
  double acc = 0.0;
  for (int a = 0; a < K; ++a) acc += P[r * W + a] * (trans ? Gc[(int64_t)b * W + a] : Gc[(int64_t)a * W + b]);
  if (op == 0) X[i] = acc; else X[i] -= acc;
}

// ------------------------------------------------------------------ block-cooperative dense FP64 helpers
// Matrices in global memory, row-major with leading dimension ld.

// C = alpha op(A) op(B) + beta C, op(A): M x Kd, op(B): Kd x N.
__device__ void bgemm(double *C, int ldc, const double *A, int lda, bool ta, const double *B, int ldb, bool tb, int M, int N,
                      int Kd, double alpha, double beta) {
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    double acc = 0.0;
    for (int k = 0; k < Kd; ++k) {
      const double a = ta ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k];
      const double b = tb ? B[(int64_t)j * ldb + k] : B[(int64_t)k * ldb + j];
      acc += a * b;
    }
    C[(int64_t)i * ldc + j] = alpha * acc + (beta == 0.0 ? 0.0 : beta * C[(int64_t)i * ldc + j]);
  }
  __syncthreads();
}

__device__ void bcopy(double *D, int ldd, const double *S, int lds, int M, int N, double alpha) {
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    D[(int64_t)i * ldd + j] = alpha * S[(int64_t)i * lds + j];
  }
  __syncthreads();
}

__device__ void bsym(double *A, int lda, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    if (i < j) {
      const double v = 0.5 * (A[(int64_t)i * lda + j] + A[(int64_t)j * lda + i]);
      A[(int64_t)i * lda + j] = v;
      A[(int64_t)j * lda + i] = v;
    }
  }
  __syncthreads();
}

// In-place Cholesky A = L L^T (lower part holds L, upper cleared). Returns false if a pivot <= tol.
__device__ bool bchol(double *A, int lda, int n, double tol) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(int64_t)j * lda + j];
      if (!(d > tol)) { ok = 0; A[(int64_t)j * lda + j] = 1.0; }
      else A[(int64_t)j * lda + j] = sqrt(d);
    }
    __syncthreads();
    const double piv = A[(int64_t)j * lda + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * lda + j] /= piv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < (n - j - 1) * (n - j - 1); idx += blockDim.x) {
      const int i = j + 1 + idx / (n - j - 1), k = j + 1 + idx % (n - j - 1);
      if (k <= i) A[(int64_t)i * lda + k] -= A[(int64_t)i * lda + j] * A[(int64_t)k * lda + j];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx - i * n;
    if (k > i) A[(int64_t)i * lda + k] = 0.0;
  }
  __syncthreads();
  return ok != 0;
}

// Linv = L^{-1} for lower-triangular L (columns solved in parallel).
__device__ void btrinv_lower(double *Linv, int ldi, const double *L, int ldl, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      if (i < j) { Linv[(int64_t)i * ldi + j] = 0.0; continue; }
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) s -= L[(int64_t)i * ldl + k] * Linv[(int64_t)k * ldi + j];
      Linv[(int64_t)i * ldi + j] = s / L[(int64_t)i * ldl + i];
    }
  }
  __syncthreads();
}

// Ainv = A^{-1} by Gauss-Jordan with partial pivoting; A is overwritten.  Returns false if singular.
__device__ bool binverse(double *A, int lda, double *Ainv, int ldi, int n) {
  __shared__ int piv_row, ok;
  if (threadIdx.x == 0) ok = 1;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    Ainv[(int64_t)i * ldi + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double best = fabs(A[(int64_t)c * lda + c]);
      for (int r = c + 1; r < n; ++r) {
        const double v = fabs(A[(int64_t)r * lda + c]);
        if (v > best) { best = v; p = r; }
      }
      piv_row = p;
      if (best == 0.0) ok = 0;
    }
    __syncthreads();
    if (!ok) return false;
    const int p = piv_row;
    if (p != c) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t = A[(int64_t)p * lda + k]; A[(int64_t)p * lda + k] = A[(int64_t)c * lda + k]; A[(int64_t)c * lda + k] = t;
        t = Ainv[(int64_t)p * ldi + k]; Ainv[(int64_t)p * ldi + k] = Ainv[(int64_t)c * ldi + k]; Ainv[(int64_t)c * ldi + k] = t;
      }
    }
    __syncthreads();
    const double d = A[(int64_t)c * lda + c];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      A[(int64_t)c * lda + k] /= d;
      Ainv[(int64_t)c * ldi + k] /= d;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, k = idx - r * n;
      if (r == c) continue;
      const double f = A[(int64_t)r * lda + c];
      if (k != c) A[(int64_t)r * lda + k] -= f * A[(int64_t)c * lda + k];
      Ainv[(int64_t)r * ldi + k] -= f * Ainv[(int64_t)c * ldi + k];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != c) A[(int64_t)r * lda + c] = 0.0;
    __syncthreads();
  }
  return true;
}

// Cholesky factor + inverse of a K x K Gram matrix per cell: Rinv^T stored so that X Rinv = rowmul(X, Linv, trans).
// pre: squared B-norms of the block's columns before Gram-Schmidt (the deflation scale);
// blocks j >= m_c of a cell are not part of its basis and never report deflation.
__global__ void k_chol_inv(double *Linv, double *G, const double *pre, const int32_t *Kt, const int32_t *mc, int j, int W,
                           double rel_tol, int *status) {
  const int c = blockIdx.x;
  const int K = Kt[c];
  double *Gc = G + (int64_t)c * W * W;
  __shared__ double scale;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < K; ++i) s = fmax(s, fmax(Gc[(int64_t)i * W + i], pre[(int64_t)c * W + i]));
    scale = s;
  }
  __syncthreads();
  bsym(Gc, W, K);
  if (!bchol(Gc, W, K, rel_tol * scale)) {
    if (threadIdx.x == 0 && j < mc[c]) atomicExch(status, MSS_ERR_KRYLOV_DEFLATION);
  }
  btrinv_lower(Linv + (int64_t)c * W * W, W, Gc, W, K);
}

// Block Lanczos (Appendix C) + symmetric GammaTrans on A^m (n x n, n = m K) and S^m (n x K), one
// block per cell.  Workspace per cell: n^2 + 3 n K + 8 K^2 doubles.
__global__ void k_lanczos_gamma(const double *Am, const int64_t *am_off, const double *Sm, const int64_t *sm_off,
                                const int32_t *Kt, const int32_t *mc, double *work, const int64_t *work_off, double *gam,
                                double *gh, const int64_t *coef_off, int *status) {
  const int c = blockIdx.x;
  const int K = Kt[c], m = mc[c], n = m * K;
  const double *A = Am + am_off[c];
  const double *S = Sm + sm_off[c];
  double *w = work + work_off[c];
  double *Q = w;                          // n x n : columns block k = Q[:, kK:(k+1)K]
  double *Wk = Q + (int64_t)n * n;        // n x K
  double *W2 = Wk + (int64_t)n * K;       // n x K
  double *T = W2 + (int64_t)n * K;        // n x K
  double *k1 = T + (int64_t)n * K;        // K x K scratch x 8
  double *k2 = k1 + K * K, *k3 = k2 + K * K, *k4 = k3 + K * K, *Gm = k4 + K * K, *Gp = Gm + K * K;
  double *alpha = Gp + K * K, *beta = alpha + K * K;
  double *G = gam + coef_off[c], *H = gh + coef_off[c];
  __shared__ double anorm;
  __shared__ int bad;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < n; ++i) {
      double r = 0;
      for (int j = 0; j < n; ++j) r += fabs(A[(int64_t)i * n + j]);
      s = fmax(s, r);
    }
    anorm = s;
    bad = 0;
  }
  __syncthreads();
  // QR (CholeskyQR2, positive diagonal) of X (n x K) into Qblk (ld n) and R (K x K upper, in Rout)
  auto qr = [&](const double *X, double *Qblk, double *Rout) -> bool {
    bgemm(k1, K, X, K, true, X, K, false, K, K, n, 1.0, 0.0);            // X^T X
    if (!bchol(k1, K, K, 1e-300)) return false;                          // L1 L1^T
    btrinv_lower(k2, K, k1, K, K);                                        // L1^{-1}
    bgemm(T, K, X, K, false, k2, K, true, n, K, K, 1.0, 0.0);            // X L1^{-T}
    bgemm(k3, K, T, K, true, T, K, false, K, K, n, 1.0, 0.0);            // second pass
    if (!bchol(k3, K, K, 1e-300)) return false;
    btrinv_lower(k4, K, k3, K, K);
    bgemm(W2, K, T, K, false, k4, K, true, n, K, K, 1.0, 0.0);           // Q = T L2^{-T}
    bcopy(Qblk, n, W2, K, n, K, 1.0);
    bgemm(Rout, K, k3, K, true, k1, K, true, K, K, K, 1.0, 0.0);          // R = L2^T L1^T
    return true;
  };
  // beta_1: S^m = Q_1 beta_1
  bcopy(Wk, K, S, K, n, K, 1.0);
  if (!qr(Wk, Q, beta)) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_LANCZOS_BREAKDOWN); return; }
  // G_1 = beta_1^T, Gamma^0 = 0
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int i = idx / K, j = idx - i * K;
    Gm[idx] = beta[j * K + i];
    Gp[idx] = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    const double *Qk = Q + (int64_t)k * K;
    // Wk = A Q_k - Q_{k-1} beta_k^T
    bgemm(Wk, K, A, n, false, Qk, n, false, n, K, n, 1.0, 0.0);
    if (k > 0) bgemm(Wk, K, Q + (int64_t)(k - 1) * K, n, false, beta, K, true, n, K, K, -1.0, 1.0);
    // alpha_k = Q_k^T Wk (symmetrised)
    bgemm(alpha, K, Qk, n, true, Wk, K, false, K, K, n, 1.0, 0.0);
    bsym(alpha, K, K);
    // GammaTrans for layer k+1: Gamma-hat = G G^T, Gamma = -G^{-T} alpha G^{-1} - Gamma_prev
    bgemm(H + (int64_t)k * K * K, K, Gm, K, false, Gm, K, true, K, K, K, 1.0, 0.0);
    bcopy(k1, K, Gm, K, K, K, 1.0);
    if (!binverse(k1, K, k2, K, K)) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD); return; }
    bgemm(k3, K, alpha, K, false, k2, K, false, K, K, K, 1.0, 0.0);       // alpha G^{-1}
    bgemm(G + (int64_t)k * K * K, K, k2, K, true, k3, K, false, K, K, K, -1.0, 0.0);
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) G[(int64_t)k * K * K + idx] -= Gp[idx];
    __syncthreads();
    bsym(G + (int64_t)k * K * K, K, K);
    bsym(H + (int64_t)k * K * K, K, K);
    bcopy(Gp, K, G + (int64_t)k * K * K, K, K, K, 1.0);
    if (k + 1 == m) break;
    // Wk -= Q_k alpha_k; full reorthogonalisation against Q_1..Q_k (two passes)
    bgemm(Wk, K, Qk, n, false, alpha, K, false, n, K, K, -1.0, 1.0);
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j <= k; ++j) {
        bgemm(k1, K, Q + (int64_t)j * K, n, true, Wk, K, false, K, K, n, 1.0, 0.0);
        bgemm(Wk, K, Q + (int64_t)j * K, n, false, k1, K, false, n, K, K, -1.0, 1.0);
      }
    // Q_{k+1} beta_{k+1} = Wk
    if (!qr(Wk, Q + (int64_t)(k + 1) * K, beta)) {
      if (threadIdx.x == 0) atomicExch(status, MSS_ERR_LANCZOS_BREAKDOWN);
      return;
    }
    if (threadIdx.x == 0) {
      double dmin = 1e300;
      for (int i = 0; i < K; ++i) dmin = fmin(dmin, fabs(beta[i * K + i]));
      if (dmin < 1e-13 * anorm) bad = 1;
    }
    __syncthreads();
    if (bad) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_LANCZOS_BREAKDOWN); return; }
    // G_{k+1} = (G_k^T Gamma^k)^{-1} beta_{k+1}^T
    bgemm(k1, K, Gm, K, true, G + (int64_t)k * K * K, K, false, K, K, K, 1.0, 0.0);
    if (!binverse(k1, K, k2, K, K)) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD); return; }
    bgemm(Gm, K, k2, K, false, beta, K, true, K, K, K, 1.0, 0.0);
  }
  // SPD checks of all coefficients (Eq. S-fraction: symmetric positive definite)
  for (int k = 0; k < m; ++k) {
    bcopy(k1, K, G + (int64_t)k * K * K, K, K, K, 1.0);
    if (!bchol(k1, K, K, 0.0)) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD); return; }
    bcopy(k1, K, H + (int64_t)k * K * K, K, K, K, 1.0);
    if (!bchol(k1, K, K, 0.0)) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD); return; }
  }
}

// Pack per-cell blocks Am[j1][j2] = V_j1^T (A V_j2) (from Gram tiles at ld W) into the n x n matrix.
__global__ void k_pack_block(double *Am, const int64_t *am_off, const double *Gt, const int32_t *Kt, const int32_t *mc, int W,
                             int j1, int j2) {
  const int c = blockIdx.x;
  const int K = Kt[c], m = mc[c], n = m * K;
  if (j1 >= m || j2 >= m) return;
  const double *g = Gt + (int64_t)c * W * W;
  double *a = Am + am_off[c];
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int i = idx / K, j = idx - i * K;
    if (j1 == j2) {
      a[(int64_t)(j1 * K + i) * n + j1 * K + j] = 0.5 * (g[(int64_t)i * W + j] + g[(int64_t)j * W + i]);
    } else {
      const double v = g[(int64_t)i * W + j];
      a[(int64_t)(j1 * K + i) * n + j2 * K + j] = v;
      a[(int64_t)(j2 * K + j) * n + j1 * K + i] = v;
    }
  }
}

// Sm rows of block j: V_j[0:Kb]^T Cb  (K x K), written at rows j*K.. of the n x K matrix.
__global__ void k_pack_sm(double *Sm, const int64_t *sm_off, const double *V, const double *Cb, const int64_t *cb_off,
                          const int64_t *row0, const int32_t *Kb, const int32_t *Kt, const int32_t *mc, int W, int j) {
  const int c = blockIdx.x;
  const int K = Kt[c];
  if (j >= mc[c]) return;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int a = idx / K, b = idx - a * K;
    double acc = 0.0;
    for (int r = 0; r < Kb[c]; ++r) acc += V[(row0[c] + r) * W + a] * Cb[cb_off[c] + (int64_t)r * K + b];
    Sm[sm_off[c] + (int64_t)(j * K + a) * K + b] = acc;
  }
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

// Chunk of cells processed together on the device.
static void build_chunk(const Partition &P, const std::vector<int> &cells, const std::vector<int> &Kt_all,
                        const std::vector<int> &m_all, const std::vector<std::vector<double>> &Cb_all, double shift,
                        double cg_tol, int cg_maxit, Rom &R, cudaStream_t st) {
  const int nc = (int)cells.size();
  int W = 0, mmax = 0;
  for (int c : cells) {
    W = std::max(W, Kt_all[c]);
    mmax = std::max(mmax, m_all[c]);
  }
  std::vector<int64_t> row0(nc + 1, 0), ptr, col;
  std::vector<double> val, Bv, Cb;
  std::vector<int64_t> cb_off(nc, 0);
  std::vector<int32_t> Kb(nc), Kt(nc), mc(nc);
  ptr.push_back(0);
  for (int i = 0; i < nc; ++i) {
    const Cell &cl = P.cells[cells[i]];
    row0[i + 1] = row0[i] + (int64_t)cl.nodes.size();
    for (int64_t r = 0; r < cl.A.n; ++r) {
      for (int64_t k = cl.A.ptr[r]; k < cl.A.ptr[r + 1]; ++k) {
        col.push_back(row0[i] + cl.A.col[k]);
        val.push_back(cl.A.val[k]);
      }
      ptr.push_back((int64_t)col.size());
    }
    Bv.insert(Bv.end(), cl.B.begin(), cl.B.end());
    cb_off[i] = (int64_t)Cb.size();
    Cb.insert(Cb.end(), Cb_all[cells[i]].begin(), Cb_all[cells[i]].end());
    Kb[i] = (int32_t)cl.K;
    Kt[i] = Kt_all[cells[i]];
    mc[i] = m_all[cells[i]];
  }
  const int64_t rows = row0[nc];
  const int64_t NW = rows * W;
  DevMem d_row0, d_ptr, d_col, d_val, d_B, d_dinv, d_Cb, d_cboff, d_Kb, d_Kt, d_mc, d_status;
  upload(d_row0, row0);
  upload(d_ptr, ptr);
  upload(d_col, col);
  upload(d_val, val);
  upload(d_B, Bv);
  std::vector<double> dinv(rows);
  for (int i = 0; i < nc; ++i) {
    const Cell &cl = P.cells[cells[i]];
    for (int64_t r = 0; r < cl.A.n; ++r) {
      double diag = 0;
      for (int64_t k = cl.A.ptr[r]; k < cl.A.ptr[r + 1]; ++k)
        if (cl.A.col[k] == r) diag = cl.A.val[k];
      dinv[row0[i] + r] = 1.0 / (-diag - shift * cl.B[r]);
    }
  }
  upload(d_dinv, dinv);
  upload(d_Cb, Cb);
  upload(d_cboff, cb_off);
  upload(d_Kb, Kb);
  upload(d_Kt, Kt);
  upload(d_mc, mc);
  upload(d_status, std::vector<int>(1, 0));
  std::vector<DevMem> V(mmax);
  for (auto &v : V) v.alloc(NW * 8);
  DevMem X, Y, cr, cz, cp, cq, G, Linv, sb1, sb2, sb3, sb4, sb5, sb6, mx;
  for (DevMem *b : {&X, &Y, &cr, &cz, &cp, &cq}) b->alloc(NW * 8);
  G.alloc((size_t)nc * W * W * 8);
  Linv.alloc((size_t)nc * W * W * 8);
  for (DevMem *b : {&sb1, &sb2, &sb3, &sb4, &sb5, &sb6}) b->alloc((size_t)nc * W * 8);
  double *s1 = sb1.as<double>(), *s2 = sb2.as<double>(), *s3 = sb3.as<double>(), *s4 = sb4.as<double>(),
         *s5 = sb5.as<double>(), *pre = sb6.as<double>();
  mx.alloc(8);
  const int64_t *r0 = d_row0.as<int64_t>();
  const int32_t *kt = d_Kt.as<int32_t>();
  int *status = d_status.as<int>();
  const dim3 ggram(nc, (W + 15) / 16, (W + 15) / 16);
  // B-orthonormalise block X against previous blocks (two passes) into V[j]
  auto orth = [&](int j) {
    k_coldot<<<nc, 128, 0, st>>>(pre, nullptr, X.as<double>(), X.as<double>(), d_B.as<double>(), r0, kt, W);
    for (int pass = 0; pass < 2; ++pass)
      for (int p = 0; p < j; ++p) {
        k_gram<<<ggram, kThreads, 0, st>>>(G.as<double>(), V[p].as<double>(), X.as<double>(), d_B.as<double>(), r0, kt, W);
        k_rowmul<<<nblk(NW), kThreads, 0, st>>>(X.as<double>(), V[p].as<double>(), G.as<double>(), 0, 1, r0, kt, nc, rows, W);
      }
    k_gram<<<ggram, kThreads, 0, st>>>(G.as<double>(), X.as<double>(), X.as<double>(), d_B.as<double>(), r0, kt, W);
    k_chol_inv<<<nc, kThreads, 0, st>>>(Linv.as<double>(), G.as<double>(), pre, kt, d_mc.as<int32_t>(), j, W, 1e-20,
                                        status);
    k_rowmul<<<nblk(NW), kThreads, 0, st>>>(V[j].as<double>(), X.as<double>(), Linv.as<double>(), 1, 0, r0, kt, nc, rows, W);
  };
  // V_0 from B^{-1} C
  k_expand_c<<<nblk(NW), kThreads, 0, st>>>(X.as<double>(), d_Cb.as<double>(), d_cboff.as<int64_t>(), r0, d_Kb.as<int32_t>(), kt,
                                           d_B.as<double>(), nc, rows, W, 1);
  orth(0);
  for (int j = 1; j < mmax; ++j) {
    // rhs = B V_{j-1}; solve -(A + sB) y = rhs by CG (cells with m_c <= j carry along harmlessly)
    k_spmm<<<nblk(NW), kThreads, 0, st>>>(Y.as<double>(), V[j - 1].as<double>(), d_ptr.as<int64_t>(), d_col.as<int64_t>(),
                                         d_val.as<double>(), d_B.as<double>(), shift, r0, kt, nc, rows, W, 2);
    k_coldot<<<nc, 128, 0, st>>>(s5, nullptr, Y.as<double>(), Y.as<double>(), nullptr, r0, kt, W);  // |b|^2
    k_cg_init<<<nblk(NW), kThreads, 0, st>>>(X.as<double>(), cr.as<double>(), cz.as<double>(), cp.as<double>(), Y.as<double>(),
                                            d_dinv.as<double>(), r0, kt, nc, rows, W);
    k_coldot<<<nc, 128, 0, st>>>(s1, nullptr, cr.as<double>(), cz.as<double>(), nullptr, r0, kt, W);  // rz
    bool conv = false;
    for (int it = 0; it < cg_maxit; ++it) {
      k_spmm<<<nblk(NW), kThreads, 0, st>>>(cq.as<double>(), cp.as<double>(), d_ptr.as<int64_t>(), d_col.as<int64_t>(),
                                           d_val.as<double>(), d_B.as<double>(), shift, r0, kt, nc, rows, W, 1);
      k_coldot<<<nc, 128, 0, st>>>(s2, nullptr, cp.as<double>(), cq.as<double>(), nullptr, r0, kt, W);  // pq
      k_cg_xr<<<nblk(NW), kThreads, 0, st>>>(X.as<double>(), cr.as<double>(), cz.as<double>(), cp.as<double>(), cq.as<double>(),
                                            d_dinv.as<double>(), s1, s2, r0, nc, rows, W);
      k_coldot<<<nc, 128, 0, st>>>(s3, s4, cr.as<double>(), cz.as<double>(), nullptr, r0, kt, W);
      k_cg_p<<<nblk(NW), kThreads, 0, st>>>(cp.as<double>(), cz.as<double>(), s3, s1, r0, nc, rows, W);
      std::swap(s1, s3);
      if (it % 10 == 9 || it + 1 == cg_maxit) {
        k_maxratio<<<1, kThreads, 0, st>>>(mx.as<double>(), s4, s5, kt, nc, W);
        double h = 0;
        MSS_CUDA(cudaMemcpyAsync(&h, mx.p, 8, cudaMemcpyDeviceToHost, st));
        MSS_CUDA(cudaStreamSynchronize(st));
        if (h <= cg_tol * cg_tol) { conv = true; break; }
      }
    }
    MSS_REQUIRE(conv, MSS_ERR_NOT_CONVERGED, "shifted CG did not reach the tolerance");
    orth(j);
  }
  int h_status = 0;
  MSS_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MSS_CUDA(cudaStreamSynchronize(st));
  MSS_REQUIRE(h_status == 0, h_status, "Krylov basis is (numerically) rank deficient (Assumption ass1)");
  // A^m = V^T A V (blockwise), S^m = V^T C
  std::vector<int64_t> am_off(nc + 1, 0), sm_off(nc + 1, 0), work_off(nc + 1, 0), coef_off(nc + 1, 0);
  for (int i = 0; i < nc; ++i) {
    const int64_t n = (int64_t)mc[i] * Kt[i];
    am_off[i + 1] = am_off[i] + n * n;
    sm_off[i + 1] = sm_off[i] + n * Kt[i];
    work_off[i + 1] = work_off[i] + n * n + 3 * n * Kt[i] + 8 * (int64_t)Kt[i] * Kt[i];
    coef_off[i + 1] = coef_off[i] + (int64_t)mc[i] * Kt[i] * Kt[i];
  }
  DevMem d_am, d_sm, d_work, d_gam, d_gh, d_amoff, d_smoff, d_workoff, d_coefoff;
  d_am.alloc(am_off[nc] * 8);
  d_sm.alloc(sm_off[nc] * 8);
  d_work.alloc(work_off[nc] * 8);
  d_gam.alloc(coef_off[nc] * 8);
  d_gh.alloc(coef_off[nc] * 8);
  upload(d_amoff, am_off);
  upload(d_smoff, sm_off);
  upload(d_workoff, work_off);
  upload(d_coefoff, coef_off);
  for (int j2 = 0; j2 < mmax; ++j2) {
    k_spmm<<<nblk(NW), kThreads, 0, st>>>(Y.as<double>(), V[j2].as<double>(), d_ptr.as<int64_t>(), d_col.as<int64_t>(),
                                         d_val.as<double>(), d_B.as<double>(), shift, r0, kt, nc, rows, W, 0);
    for (int j1 = 0; j1 <= j2; ++j1) {
      k_gram<<<ggram, kThreads, 0, st>>>(G.as<double>(), V[j1].as<double>(), Y.as<double>(), nullptr, r0, kt, W);
      k_pack_block<<<nc, kThreads, 0, st>>>(d_am.as<double>(), d_amoff.as<int64_t>(), G.as<double>(), kt, d_mc.as<int32_t>(),
                                            W, j1, j2);
    }
    k_pack_sm<<<nc, kThreads, 0, st>>>(d_sm.as<double>(), d_smoff.as<int64_t>(), V[j2].as<double>(), d_Cb.as<double>(),
                                       d_cboff.as<int64_t>(), r0, d_Kb.as<int32_t>(), kt, d_mc.as<int32_t>(), W, j2);
  }
  // the per-cell Am blocks from k_gram are V_j1^T A V_j2; symmetrise is done inside the Lanczos kernel
  k_lanczos_gamma<<<nc, kThreads, 0, st>>>(d_am.as<double>(), d_amoff.as<int64_t>(), d_sm.as<double>(), d_smoff.as<int64_t>(),
                                           kt, d_mc.as<int32_t>(), d_work.as<double>(), d_workoff.as<int64_t>(),
                                           d_gam.as<double>(), d_gh.as<double>(), d_coefoff.as<int64_t>(), status);
  MSS_CUDA(cudaGetLastError());
  MSS_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<double> gam(coef_off[nc]), gh(coef_off[nc]);
  MSS_CUDA(cudaMemcpyAsync(gam.data(), d_gam.p, gam.size() * 8, cudaMemcpyDeviceToHost, st));
  MSS_CUDA(cudaMemcpyAsync(gh.data(), d_gh.p, gh.size() * 8, cudaMemcpyDeviceToHost, st));
  MSS_CUDA(cudaStreamSynchronize(st));
  MSS_REQUIRE(h_status == 0, h_status, "block Lanczos / S-fraction extraction failed");
  for (int i = 0; i < nc; ++i) {
    const int c = cells[i];
    std::copy(gam.begin() + coef_off[i], gam.begin() + coef_off[i + 1], R.gamma.begin() + R.coef_off[c]);
    std::copy(gh.begin() + coef_off[i], gh.begin() + coef_off[i + 1], R.gamma_hat.begin() + R.coef_off[c]);
  }
}

static void invert_spd_host(const double *A, int n, double *out) {
  // Cholesky-based inverse (FP64, host) of a small SPD matrix
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    MSS_REQUIRE(s > 0, MSS_ERR_COEF_NOT_SPD, "Gamma-hat^1 face block not SPD");
    L[(size_t)j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / L[(size_t)j * n + j];
    }
  }
  for (int col = 0; col < n; ++col) {
    std::vector<double> y(n, 0.0);
    for (int i = 0; i < n; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
      y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * out[(size_t)k * n + col];
      out[(size_t)i * n + col] = s / L[(size_t)i * n + i];
    }
  }
}

static void build_roms(const Partition &Pc, const mss_rom_params &prm, const int32_t *cell_m, cudaStream_t st, Rom &R) {
  Partition &P = const_cast<Partition &>(Pc);
  MSS_REQUIRE(prm.n_modes >= 1 && prm.shift < 0 && prm.cg_tol > 0 && prm.cg_maxit > 0, MSS_ERR_INVALID_ARG,
              "bad ROM parameters (n_modes >= 1, shift < 0, cg_tol > 0, cg_maxit > 0)");
  const int nc = P.n_cells, nf = (int)P.faces.size();
  // face bases and topology
  R.n_cells = nc;
  R.n_faces = nf;
  R.face_M.assign(nf, 0);
  R.face_K.assign(nf, 0);
  R.basis_off.assign(nf + 1, 0);
  R.bases.clear();
  R.face_cells.assign(2 * nf, -1);
  for (int f = 0; f < nf; ++f) {
    std::vector<double> S;
    int M = 0;
    face_basis(P.faces[f], prm.n_modes, S, M);
    R.face_M[f] = M;
    R.face_K[f] = (int32_t)P.faces[f].nodes.size();
    R.bases.insert(R.bases.end(), S.begin(), S.end());
    R.basis_off[f + 1] = (int64_t)R.bases.size();
    R.face_cells[2 * f] = P.faces[f].cells[0];
    R.face_cells[2 * f + 1] = P.faces[f].cells[1];
  }
  R.cell_m.assign(nc, prm.m);
  if (cell_m)
    for (int c = 0; c < nc; ++c) R.cell_m[c] = cell_m[c];
  R.cell_face_ptr.assign(nc + 1, 0);
  R.cell_faces.clear();
  for (int c = 0; c < nc; ++c) {
    R.cell_faces.insert(R.cell_faces.end(), P.cells[c].faces.begin(), P.cells[c].faces.end());
    R.cell_face_ptr[c + 1] = (int32_t)R.cell_faces.size();
  }
  R.finalize_topology();
  R.gamma.assign(R.coef_off[nc], 0.0);
  R.gamma_hat.assign(R.coef_off[nc], 0.0);
  // per cell: split matrices and the boundary block of C = P^Gamma S_c (K_c rows x Kt_c)
  std::vector<int> Kt(nc), mv(nc);
  std::vector<std::vector<double>> Cb(nc);
  int64_t maxbytes = 0;
  for (int c = 0; c < nc; ++c) {
    P.build_cell(c);
    const Cell &cl = P.cells[c];
    Kt[c] = R.cell_K[c];
    mv[c] = R.cell_m[c];
    MSS_REQUIRE(mv[c] >= 1, MSS_ERR_INVALID_ARG, "m must be >= 1");
    MSS_REQUIRE((int64_t)mv[c] * Kt[c] <= (int64_t)cl.nodes.size(), MSS_ERR_KRYLOV_DEFLATION,
                "m * K exceeds the cell size (Assumption ass1)");
    Cb[c].assign((size_t)cl.K * Kt[c], 0.0);
    int64_t rr = 0;
    int oc = 0;
    for (int f : cl.faces) {
      const int Kf = R.face_K[f], M = R.face_M[f];
      const double *S = R.bases.data() + R.basis_off[f];
      for (int r = 0; r < Kf; ++r)
        for (int j = 0; j < M; ++j) Cb[c][(size_t)(rr + r) * Kt[c] + oc + j] = S[(size_t)r * M + j];
      rr += Kf;
      oc += M;
    }
    maxbytes = std::max<int64_t>(maxbytes, (int64_t)cl.nodes.size());
  }
  // chunks bounded by device memory (~ (mmax + 6) dense N x W arrays)
  size_t free_b = 0, total_b = 0;
  MSS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const int Wmax = *std::max_element(Kt.begin(), Kt.end());
  const int mmax = *std::max_element(mv.begin(), mv.end());
  const double budget = std::min<double>(0.5 * (double)free_b, 48e9);
  std::vector<int> chunk;
  double used = 0;
  for (int c = 0; c < nc; ++c) {
    const double need = (double)P.cells[c].nodes.size() * Wmax * 8.0 * (mmax + 7) +
                        8.0 * ((double)mv[c] * Kt[c]) * ((double)mv[c] * Kt[c]) * 3;
    if (!chunk.empty() && used + need > budget) {
      build_chunk(P, chunk, Kt, mv, Cb, prm.shift, prm.cg_tol, prm.cg_maxit, R, st);
      chunk.clear();
      used = 0;
    }
    chunk.push_back(c);
    used += need;
  }
  if (!chunk.empty()) build_chunk(P, chunk, Kt, mv, Cb, prm.shift, prm.cg_tol, prm.cg_maxit, R, st);
  // face masses M_f = sum_i (Gamma-hat^1_{i,f})^{-1}
  R.face_mass.assign(R.fmass_off[nf], 0.0);
  for (int f = 0; f < nf; ++f) {
    const int M = R.face_M[f];
    std::vector<double> blk((size_t)M * M), inv((size_t)M * M);
    for (int s = 0; s < 2; ++s) {
      const int c = R.face_cells[2 * f + s];
      if (c < 0) continue;
      int o = 0;
      for (int k = R.cell_face_ptr[c]; k < R.cell_face_ptr[c + 1]; ++k) {
        if (R.cell_faces[k] == f) break;
        o += R.face_M[R.cell_faces[k]];
      }
      const int K = R.cell_K[c];
      const double *H1 = R.gamma_hat.data() + R.coef_off[c];
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) blk[(size_t)i * M + j] = 0.5 * (H1[(size_t)(o + i) * K + o + j] + H1[(size_t)(o + j) * K + o + i]);
      invert_spd_host(blk.data(), M, inv.data());
      for (size_t t = 0; t < inv.size(); ++t) R.face_mass[R.fmass_off[f] + t] += inv[t];
    }
    for (int i = 0; i < M; ++i)
      for (int j = i + 1; j < M; ++j) {
        const double v = 0.5 * (R.face_mass[R.fmass_off[f] + (size_t)i * M + j] + R.face_mass[R.fmass_off[f] + (size_t)j * M + i]);
        R.face_mass[R.fmass_off[f] + (size_t)i * M + j] = v;
        R.face_mass[R.fmass_off[f] + (size_t)j * M + i] = v;
      }
  }
  // Appendix D data: per corner-set node, (face, S_f row of its hanging copy, b_{k_f}/b_k)
  R.cg_ptr.assign(1, 0);
  R.cg_face.clear();
  R.cg_rows.clear();
  R.cg_weight.clear();
  for (int64_t u : P.corner_set) {
    const int32_t *lst;
    const int n = P.faces_of(u, &lst);
    std::vector<double> mass(n);
    double tot = 0;
    for (int k = 0; k < n; ++k) tot += (mass[k] = P.hanging_mass(u, lst[k]));
    for (int k = 0; k < n; ++k) {
      const int f = lst[k];
      const Face &F = P.faces[f];
      const int64_t h = P.hang_first[u] + k;
      const int row = (int)(std::find(F.nodes.begin(), F.nodes.end(), h) - F.nodes.begin());
      const int M = R.face_M[f];
      const double *S = R.bases.data() + R.basis_off[f];
      R.cg_face.push_back(f);
      R.cg_rows.insert(R.cg_rows.end(), S + (size_t)row * M, S + (size_t)(row + 1) * M);
      R.cg_weight.push_back(mass[k] / tot);
    }
    R.cg_ptr.push_back((int32_t)R.cg_face.size());
  }
  if (R.cg_ptr.size() == 1) R.cg_ptr.clear();
  R.source = &Pc;
}

}  // namespace mss

using namespace mss;

extern "C" mss_status mss_build_roms(const mss_partition *p, const mss_rom_params *prm, const int32_t *cell_m, void *stream,
                                     mss_rom **out) {
  return guard([&] {
    MSS_REQUIRE(p && prm && out, MSS_ERR_INVALID_ARG, "null argument");
    auto h = std::make_unique<mss_rom>();
    build_roms(p->p, *prm, cell_m, (cudaStream_t)stream, h->r);
    *out = h.release();
  });
}
