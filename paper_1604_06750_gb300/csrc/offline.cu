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
#include <thread>

#include "cuda_util.h"

namespace mss {

namespace {

constexpr int kThreads = 256;
// The last S-fraction coefficient may be positive semidefinite (a cell without a Dirichlet node keeps
// the constant mode): pivot floor of its Cholesky factor and the most negative pivot still taken as
// rounding, both relative to its largest diagonal entry.
constexpr double kPsdFloor = 1e-13;
constexpr double kPsdNegTol = 1e-8;

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

// Cholesky factor of a positive semidefinite matrix (the last S-fraction coefficient of a cell that
// holds no Dirichlet node, where the constant mode makes it singular up to rounding): as bchol, but a
// pivot d <= floor_rel * s (s = largest diagonal entry) is raised to floor_rel * s, and a pivot below
// -neg_rel * s means the matrix is indefinite.  Returns the number of raised pivots, or -1 if
// indefinite (or without a positive diagonal).  A holds L in its lower part, upper part cleared.
__device__ int bchol_psd(double *A, int lda, int n, double floor_rel, double neg_rel) {
  __shared__ int floored;
  __shared__ double scale;
  if (threadIdx.x == 0) {
    double sc = 0;
    for (int i = 0; i < n; ++i) sc = fmax(sc, A[(int64_t)i * lda + i]);
    scale = sc;
    floored = sc > 0 ? 0 : -1;
  }
  __syncthreads();
  if (floored < 0) return -1;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = A[(int64_t)j * lda + j];
      if (!(d > floor_rel * scale)) {
        if (!(d >= -neg_rel * scale)) floored = -1;
        else if (floored >= 0) ++floored;
        d = floor_rel * scale;
      }
      A[(int64_t)j * lda + j] = sqrt(d);
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
  return floored;
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
// Lift rows (optional): cell c owns rows lift_ptr[c] .. lift_ptr[c+1]-1, row l holds V^T e_n (n values,
// the cell's Krylov basis at one interior node) and receives the lift weights w_k = G_k^{-T} Q_k^T V^T e_n,
// k = 1..m, as m blocks of K values (Remark MFEM: the value at node n is sum_k w_k . U^k).
__global__ void k_lanczos_gamma(const double *Am, const int64_t *am_off, const double *Sm, const int64_t *sm_off,
                                const int32_t *Kt, const int32_t *mc, double *work, const int64_t *work_off, double *gam,
                                double *gh, const int64_t *coef_off, int *status, const int32_t *lift_ptr,
                                const double *lift_v, double *lift_w, const int64_t lift_ld) {
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
  double *tl = beta + K * K;              // K: Q_k^T v of one lift row
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
    // lift weights of layer k+1: w = G_k^{-T} (Q_k^T v), with k2 = G_k^{-1} still in place
    if (lift_ptr)
      for (int l = lift_ptr[c]; l < lift_ptr[c + 1]; ++l) {
        const double *v = lift_v + (int64_t)l * lift_ld;
        for (int i = threadIdx.x; i < K; i += blockDim.x) {
          double t = 0;
          for (int r = 0; r < n; ++r) t += Qk[(int64_t)r * n + i] * v[r];
          tl[i] = t;
        }
        __syncthreads();
        double *wl = lift_w + (int64_t)l * lift_ld + (int64_t)k * K;
        for (int i = threadIdx.x; i < K; i += blockDim.x) {
          double t = 0;
          for (int j = 0; j < K; ++j) t += k2[(int64_t)j * K + i] * tl[j];
          wl[i] = t;
        }
        __syncthreads();
      }
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
  // SPD checks of all coefficients (Eq. S-fraction: symmetric positive definite), except that the
  // last Gamma^m may be positive semidefinite: it is factored with floored pivots and, if a pivot
  // was raised, replaced by L L^T, which must stay within 10 (floor + neg) s of it elementwise.
  for (int k = 0; k < m; ++k) {
    double *Gk = G + (int64_t)k * K * K;
    bcopy(k1, K, Gk, K, K, K, 1.0);
    if (k + 1 < m) {
      if (!bchol(k1, K, K, 0.0)) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD); return; }
    } else {
      const int fl = bchol_psd(k1, K, K, kPsdFloor, kPsdNegTol);
      if (fl < 0) { if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD); return; }
      if (fl > 0) {
        bgemm(k2, K, k1, K, false, k1, K, true, K, K, K, 1.0, 0.0);      // L L^T
        bsym(k2, K, K);
        __shared__ double gap, gsc;
        if (threadIdx.x == 0) {
          double g = 0, sc = 0;
          for (int i = 0; i < K; ++i) sc = fmax(sc, Gk[(int64_t)i * K + i]);
          for (int i = 0; i < K * K; ++i) g = fmax(g, fabs(k2[i] - Gk[i]));
          gap = g;
          gsc = sc;
        }
        __syncthreads();
        if (!(gap <= 10.0 * (kPsdFloor + kPsdNegTol) * gsc)) {
          if (threadIdx.x == 0) atomicExch(status, MSS_ERR_COEF_NOT_SPD);
          return;
        }
        bcopy(Gk, K, k2, K, K, K, 1.0);
      }
    }
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

// Transfer function of the three-point scheme (Eqs. GammaU1st, GammaUrem, tfgamma) at a real
// Laplace point z, per cell: Z_m = D_m, Z_k = D_k - Gamma^k Z_{k+1}^{-1} Gamma^k, U^1 = Z_1^{-1},
// D_k = -Gamma^k - Gamma^{k-1} + z (Gamma-hat^k)^{-1}; then the relative Frobenius distance
// of U^1 to F (the exact cell transfer function at z).  Workspace: 6 K x K per cell.
__global__ void k_sfrac_err(const double *gam, const double *gh, const int64_t *coef_off, const int32_t *Kt,
                            const int32_t *mc, double z, const double *F, const int64_t *f_off, double *work,
                            const int64_t *w_off, double *err) {
  const int c = blockIdx.x;
  const int K = Kt[c], m = mc[c];
  const double *G = gam + coef_off[c], *H = gh + coef_off[c];
  double *w = work + w_off[c];
  double *Z = w, *T1 = w + (size_t)K * K, *T2 = T1 + (size_t)K * K, *Hi = T2 + (size_t)K * K,
         *T3 = Hi + (size_t)K * K;
  __shared__ double num, den;
  for (int k = m - 1; k >= 0; --k) {
    // D_k (0-based layer k): -Gamma^k - Gamma^{k-1} + z (Gamma-hat^k)^{-1}
    bcopy(T1, K, H + (size_t)k * K * K, K, K, K, 1.0);
    if (!binverse(T1, K, Hi, K, K)) { if (threadIdx.x == 0) err[c] = 1e300; return; }
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
      double v = -G[(size_t)k * K * K + idx] + z * Hi[idx];
      if (k > 0) v -= G[(size_t)(k - 1) * K * K + idx];
      T2[idx] = v;
    }
    __syncthreads();
    if (k < m - 1) {
      // T2 -= Gamma^k Z^{-1} Gamma^k   (Z holds Z_{k+1})
      bcopy(T1, K, Z, K, K, K, 1.0);
      if (!binverse(T1, K, Hi, K, K)) { if (threadIdx.x == 0) err[c] = 1e300; return; }
      bgemm(T3, K, Hi, K, false, G + (size_t)k * K * K, K, false, K, K, K, 1.0, 0.0);
      bgemm(T2, K, G + (size_t)k * K * K, K, false, T3, K, false, K, K, K, -1.0, 1.0);
    }
    bcopy(Z, K, T2, K, K, K, 1.0);
  }
  bcopy(T1, K, Z, K, K, K, 1.0);
  if (!binverse(T1, K, Hi, K, K)) { if (threadIdx.x == 0) err[c] = 1e300; return; }
  if (threadIdx.x == 0) { num = 0; den = 0; }
  __syncthreads();
  double a = 0, b = 0;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const double f = F[f_off[c] + idx];
    const double d = Hi[idx] - f;
    a += d * d;
    b += f * f;
  }
  atomicAdd(&num, a);
  atomicAdd(&den, b);
  __syncthreads();
  if (threadIdx.x == 0) err[c] = sqrt(num / fmax(den, 1e-300));
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

// ------------------------------------------------------------------ per-cell layer-count rule
// Inputs of the rule of the dipping-layer workload (reading R22), and its per-cell answers.
struct LayerRule {
  int m_lo, m_hi, n_freq;
  double omega_max, tol;
  int32_t *cell_m;   // per cell of the partition
  double *err;       // per cell (may be null)
};

struct cplx {
  double re, im;
};
static inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// X (K x K, complex, row-major) <- X^{-1} by Gauss-Jordan elimination with partial pivoting; false
// if a pivot vanishes.  work: K x K.
static bool cinvert(std::vector<cplx> &X, int K, std::vector<cplx> &work) {
  work.assign((size_t)K * K, cplx{0, 0});
  for (int i = 0; i < K; ++i) work[(size_t)i * K + i] = {1, 0};
  for (int c = 0; c < K; ++c) {
    int piv = c;
    double best = 0;
    for (int r = c; r < K; ++r) {
      const cplx v = X[(size_t)r * K + c];
      const double a = v.re * v.re + v.im * v.im;
      if (a > best) { best = a; piv = r; }
    }
    if (!(best > 0)) return false;
    if (piv != c)
      for (int j = 0; j < K; ++j) {
        std::swap(X[(size_t)piv * K + j], X[(size_t)c * K + j]);
        std::swap(work[(size_t)piv * K + j], work[(size_t)c * K + j]);
      }
    const cplx d = X[(size_t)c * K + c];
    const double dn = d.re * d.re + d.im * d.im;
    const cplx inv = {d.re / dn, -d.im / dn};
    for (int j = 0; j < K; ++j) {
      X[(size_t)c * K + j] = cmul(X[(size_t)c * K + j], inv);
      work[(size_t)c * K + j] = cmul(work[(size_t)c * K + j], inv);
    }
    for (int r = 0; r < K; ++r) {
      if (r == c) continue;
      const cplx f = X[(size_t)r * K + c];
      if (f.re == 0 && f.im == 0) continue;
      for (int j = 0; j < K; ++j) {
        const cplx a = cmul(f, X[(size_t)c * K + j]), b = cmul(f, work[(size_t)c * K + j]);
        X[(size_t)r * K + j].re -= a.re;
        X[(size_t)r * K + j].im -= a.im;
        work[(size_t)r * K + j].re -= b.re;
        work[(size_t)r * K + j].im -= b.im;
      }
    }
  }
  X.swap(work);
  return true;
}

// C (p x q) -= A (p x r) B (r x q), complex row-major with leading dimensions; transB: B given as
// its transpose (q x r, element (k, j) at Bt[j * ldb + k]).
static void cgemm_sub(cplx *C, int ldc, const cplx *A, int lda, const cplx *B, int ldb, bool transB, int p, int q, int r) {
  for (int i = 0; i < p; ++i)
    for (int k = 0; k < r; ++k) {
      const cplx a = A[(size_t)i * lda + k];
      if (a.re == 0 && a.im == 0) continue;
      for (int j = 0; j < q; ++j) {
        const cplx b = transB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j];
        C[(size_t)i * ldc + j].re -= a.re * b.re - a.im * b.im;
        C[(size_t)i * ldc + j].im -= a.re * b.im + a.im * b.re;
      }
    }
}

// The rule for one cell from its m_hi-layer projection A (n x n), S (n x K), n = m_hi K: the ROM
// transfer function of m layers is F^m(z) = S_m^T (A_m + z I)^{-1} S_m with A_m, S_m the leading
// m K rows and columns (nested Krylov spaces).  Per test point, one block LDL^T of A + z I by K x K
// blocks (complex symmetric; every leading block A_m + z I is nonsingular since Im z > 0 and A_m is
// real symmetric) gives every m at once: with Y = L^{-1} S, F^m = sum_{b < m} Y_b^T D_b^{-1} Y_b.
// errs[m] = max over the points of ||F^m - F^{m_hi}||_F / ||F^{m_hi}||_F.  False if a pivot block
// is singular.
static bool layer_rule_cell(const double *A, const double *S, int K, const LayerRule &lr, std::vector<double> &errs) {
  const int mh = lr.m_hi, n = mh * K;
  errs.assign(mh + 1, 0.0);
  std::vector<cplx> M((size_t)n * n), Y((size_t)n * K), D, Dinv, work, T((size_t)K * K), Lib((size_t)K * K);
  std::vector<std::vector<cplx>> F(mh + 1, std::vector<cplx>((size_t)K * K));
  for (int jz = 1; jz <= lr.n_freq; ++jz) {
    const double w = jz * lr.omega_max / lr.n_freq;
    const cplx z = {-w * w, w * lr.omega_max / 10.0};
    for (size_t i = 0; i < (size_t)n * n; ++i) M[i] = {A[i], 0.0};
    for (int i = 0; i < n; ++i) {
      M[(size_t)i * n + i].re += z.re;
      M[(size_t)i * n + i].im += z.im;
    }
    for (size_t i = 0; i < (size_t)n * K; ++i) Y[i] = {S[i], 0.0};
    std::vector<cplx> Fc((size_t)K * K, cplx{0, 0});
    for (int b = 0; b < mh; ++b) {
      cplx *Mbb = M.data() + (size_t)b * K * n + (size_t)b * K;
      Dinv.resize((size_t)K * K);
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) Dinv[(size_t)i * K + j] = Mbb[(size_t)i * n + j];
      if (!cinvert(Dinv, K, work)) return false;
      // F^{b+1} = F^b + Y_b^T D_b^{-1} Y_b
      const cplx *Yb = Y.data() + (size_t)b * K * K;
      std::fill(T.begin(), T.end(), cplx{0, 0});
      cgemm_sub(T.data(), K, Dinv.data(), K, Yb, K, false, K, K, K);     // T = -D^{-1} Y_b
      for (int i = 0; i < K; ++i)
        for (int k = 0; k < K; ++k) {
          const cplx yt = Yb[(size_t)k * K + i];                           // (Y_b^T)_{ik}
          for (int j = 0; j < K; ++j) {
            const cplx t = T[(size_t)k * K + j];
            Fc[(size_t)i * K + j].re -= yt.re * t.re - yt.im * t.im;
            Fc[(size_t)i * K + j].im -= yt.re * t.im + yt.im * t.re;
          }
        }
      F[b + 1] = Fc;
      // eliminate block column b below the diagonal (lower triangle of blocks kept current)
      for (int i = b + 1; i < mh; ++i) {
        const cplx *Mib = M.data() + (size_t)i * K * n + (size_t)b * K;
        std::fill(Lib.begin(), Lib.end(), cplx{0, 0});
        cgemm_sub(Lib.data(), K, Mib, n, Dinv.data(), K, false, K, K, K);  // Lib = -M_ib D^{-1}
        for (int i2 = 0; i2 < K * K; ++i2) Lib[i2] = {-Lib[i2].re, -Lib[i2].im};
        for (int jj = b + 1; jj <= i; ++jj)                                  // M_ij -= L_ib M_jb^T
          cgemm_sub(M.data() + (size_t)i * K * n + (size_t)jj * K, n, Lib.data(), K,
                    M.data() + (size_t)jj * K * n + (size_t)b * K, n, true, K, K, K);
        cgemm_sub(Y.data() + (size_t)i * K * K, K, Lib.data(), K, Yb, K, false, K, K, K);
      }
    }
    double nref = 0;
    for (const cplx &v : F[mh]) nref += v.re * v.re + v.im * v.im;
    nref = std::sqrt(nref);
    for (int m = lr.m_lo; m < mh; ++m) {
      double d = 0;
      for (size_t i = 0; i < (size_t)K * K; ++i) {
        const double a = F[m][i].re - F[mh][i].re, c = F[m][i].im - F[mh][i].im;
        d += a * a + c * c;
      }
      errs[m] = std::max(errs[m], std::sqrt(d) / std::max(nref, 1e-300));
    }
  }
  return true;
}

// Chunk of cells processed together on the device.
static void build_chunk(const Partition &P, const std::vector<int> &cells, const std::vector<int> &Kt_all,
                        const std::vector<int> &m_all, const std::vector<std::vector<double>> &Cb_all, double shift,
                        double cg_tol, int cg_maxit, Rom &R, cudaStream_t st, const LayerRule *rule = nullptr) {
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
    work_off[i + 1] = work_off[i] + n * n + 3 * n * Kt[i] + 8 * (int64_t)Kt[i] * Kt[i] + Kt[i];
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
  if (rule) {
    // the layer-count rule on the host from the projections (cells on host threads), then done
    std::vector<double> am(am_off[nc]), sm(sm_off[nc]);
    MSS_CUDA(cudaMemcpyAsync(am.data(), d_am.p, am.size() * 8, cudaMemcpyDeviceToHost, st));
    MSS_CUDA(cudaMemcpyAsync(sm.data(), d_sm.p, sm.size() * 8, cudaMemcpyDeviceToHost, st));
    MSS_CUDA(cudaStreamSynchronize(st));
    const int nt = std::max(1, std::min<int>(nc, (int)std::min(32u, std::max(1u, std::thread::hardware_concurrency()))));
    std::vector<int> bad(nt, 0);
    std::vector<std::thread> pool;
    for (int th = 0; th < nt; ++th)
      pool.emplace_back([&, th] {
        std::vector<double> errs;
        for (int i = th; i < nc; i += nt) {
          if (!layer_rule_cell(am.data() + am_off[i], sm.data() + sm_off[i], Kt[i], *rule, errs)) {
            bad[th] = 1;
            continue;
          }
          int mpick = rule->m_hi;
          for (int m = rule->m_lo; m <= rule->m_hi; ++m)
            if (errs[m] <= rule->tol) { mpick = m; break; }
          rule->cell_m[cells[i]] = mpick;
          if (rule->err) rule->err[cells[i]] = errs[mpick];
        }
      });
    for (auto &t : pool) t.join();
    for (int b : bad) MSS_REQUIRE(b == 0, MSS_ERR_LANCZOS_BREAKDOWN, "singular pivot block in the layer-count rule");
    return;
  }
  // lift rows: V^T e_n of every lift node of these cells (m blocks of the node's row of V_j)
  std::vector<int32_t> lptr(nc + 1, 0);
  std::vector<int> lnode;                    // index into P.lift_* per lift row
  {
    std::vector<int> chunk_pos(P.n_cells, -1);
    for (int i = 0; i < nc; ++i) chunk_pos[cells[i]] = i;
    std::vector<std::vector<int>> per(nc);
    for (size_t l = 0; l < P.lift_cell.size(); ++l)
      if (chunk_pos[P.lift_cell[l]] >= 0) per[chunk_pos[P.lift_cell[l]]].push_back((int)l);
    for (int i = 0; i < nc; ++i) {
      lptr[i + 1] = lptr[i] + (int32_t)per[i].size();
      lnode.insert(lnode.end(), per[i].begin(), per[i].end());
    }
  }
  DevMem d_lptr, d_lv, d_lw;
  int64_t lw_stride = 0;
  for (int i = 0; i < nc; ++i) lw_stride = std::max<int64_t>(lw_stride, (int64_t)mc[i] * Kt[i]);
  if (!lnode.empty()) {
    // one row per lift node, padded to the longest basis of the chunk; row l uses its cell's n
    upload(d_lptr, lptr);
    d_lv.alloc((size_t)lnode.size() * lw_stride * 8);
    d_lw.alloc((size_t)lnode.size() * lw_stride * 8);
    for (int i = 0; i < nc; ++i)
      for (int l = lptr[i]; l < lptr[i + 1]; ++l) {
        const int64_t row = row0[i] + P.lift_local[lnode[l]];
        for (int j = 0; j < mc[i]; ++j)
          MSS_CUDA(cudaMemcpyAsync(d_lv.as<double>() + (int64_t)l * lw_stride + (int64_t)j * Kt[i],
                                   V[j].as<double>() + row * W, (size_t)Kt[i] * 8, cudaMemcpyDeviceToDevice, st));
      }
  }
  // the per-cell Am blocks from k_gram are V_j1^T A V_j2; symmetrise is done inside the Lanczos kernel
  k_lanczos_gamma<<<nc, kThreads, 0, st>>>(d_am.as<double>(), d_amoff.as<int64_t>(), d_sm.as<double>(), d_smoff.as<int64_t>(),
                                           kt, d_mc.as<int32_t>(), d_work.as<double>(), d_workoff.as<int64_t>(),
                                           d_gam.as<double>(), d_gh.as<double>(), d_coefoff.as<int64_t>(), status,
                                           lnode.empty() ? nullptr : d_lptr.as<int32_t>(), d_lv.as<double>(),
                                           d_lw.as<double>(), lw_stride);
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
  if (!lnode.empty()) {
    std::vector<double> lw((size_t)lnode.size() * lw_stride);
    MSS_CUDA(cudaMemcpyAsync(lw.data(), d_lw.p, lw.size() * 8, cudaMemcpyDeviceToHost, st));
    MSS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < nc; ++i)
      for (int l = lptr[i]; l < lptr[i + 1]; ++l) {
        const int g = lnode[l];
        const int64_t n = (int64_t)mc[i] * Kt[i];
        std::copy(lw.begin() + (int64_t)l * lw_stride, lw.begin() + (int64_t)l * lw_stride + n,
                  R.lift_w.begin() + R.lift_off[g]);
      }
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

// Topology, face bases and C = P^Gamma S blocks of every cell (host); coefficients left zero.
static void rom_topology(Partition &P, const mss_rom_params &prm, const int32_t *cell_m, Rom &R,
                         std::vector<int> &Kt, std::vector<int> &mv, std::vector<std::vector<double>> &Cb) {
  MSS_REQUIRE(prm.n_modes >= 1 && prm.shift < 0 && prm.cg_tol > 0 && prm.cg_maxit > 0, MSS_ERR_INVALID_ARG,
              "bad ROM parameters (n_modes >= 1, shift < 0, cg_tol > 0, cg_maxit > 0)");
  const int nc = P.n_cells, nf = (int)P.faces.size();
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
    if (f < (int)P.user_bases.size() && !P.user_bases[f].empty()) {
      S = P.user_bases[f];
      M = P.user_M[f];
    } else {
      face_basis(P.faces[f], prm.n_modes, S, M);
    }
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
  Kt.assign(nc, 0);
  mv.assign(nc, 0);
  // Galerkin lift of the partition's lift nodes: m_c K_c weights each, filled by the exact build
  R.lift_unknown = P.lift_unknown;
  R.lift_cell = P.lift_cell;
  R.lift_off.assign(P.lift_cell.size() + 1, 0);
  for (size_t l = 0; l < P.lift_cell.size(); ++l)
    R.lift_off[l + 1] = R.lift_off[l] + (int64_t)R.cell_m[P.lift_cell[l]] * R.cell_K[P.lift_cell[l]];
  R.lift_w.assign(R.lift_off.back(), 0.0);
  Cb.assign(nc, std::vector<double>());
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
  }
}

// Exact off-line construction of the listed cells on the device (chunks bounded by memory).
static void rom_exact_cells(const Partition &P, const std::vector<int> &cells, const std::vector<int> &Kt,
                            const std::vector<int> &mv, const std::vector<std::vector<double>> &Cb,
                            const mss_rom_params &prm, Rom &R, cudaStream_t st) {
  if (cells.empty()) return;
  size_t free_b = 0, total_b = 0;
  MSS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  int Wmax = 0, mmax = 0;
  for (int c : cells) {
    Wmax = std::max(Wmax, Kt[c]);
    mmax = std::max(mmax, mv[c]);
  }
  const double budget = std::min<double>(0.5 * (double)free_b, 48e9);
  std::vector<int> chunk;
  double used = 0;
  for (int c : cells) {
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
}

// Exact Markov parameter Gamma-hat^1 = S^T P^T B^{-1} P S (block-diagonal over the faces;
// Remark Sinsubspace) of the listed cells, written as layer 1 of gamma_hat.
static void rom_exact_markov(const Partition &P, const std::vector<int> &cells, Rom &R) {
  for (int c : cells) {
    const Cell &cl = P.cells[c];
    const int K = R.cell_K[c];
    double *H = R.gamma_hat.data() + R.coef_off[c];
    std::fill(H, H + (size_t)K * K, 0.0);
    int64_t rr = 0;
    int oc = 0;
    for (int f : cl.faces) {
      const int Kf = R.face_K[f], M = R.face_M[f];
      const double *S = R.bases.data() + R.basis_off[f];
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
          double acc = 0;
          for (int r = 0; r < Kf; ++r) acc += S[(size_t)r * M + i] * S[(size_t)r * M + j] / cl.B[rr + r];
          H[(size_t)(oc + i) * K + oc + j] = acc;
        }
      rr += Kf;
      oc += M;
    }
  }
}

// Face masses from Gamma-hat^1 and the Appendix D groups.
static void rom_faces(const Partition &Pc, Rom &R) {
  Partition &P = const_cast<Partition &>(Pc);
  const int nf = R.n_faces;
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

static void build_roms(const Partition &Pc, const mss_rom_params &prm, const int32_t *cell_m, cudaStream_t st, Rom &R) {
  Partition &P = const_cast<Partition &>(Pc);
  std::vector<int> Kt, mv;
  std::vector<std::vector<double>> Cb;
  rom_topology(P, prm, cell_m, R, Kt, mv, Cb);
  std::vector<int> all(P.n_cells);
  std::iota(all.begin(), all.end(), 0);
  rom_exact_cells(P, all, Kt, mv, Cb, prm, R, st);
  rom_faces(Pc, R);
  R.prm = prm;
}


// Exact cell transfer functions F(s) = C^T (A + sB)^{-1} C of the listed cells (batched CG on
// -(A + sB)), compared with the S-fraction transfer functions of the ROM's current coefficients.
static void screen_cells(const Partition &P, const std::vector<int> &cells, const std::vector<int> &Kt,
                         const std::vector<std::vector<double>> &Cb, const Rom &R, double shift, double cg_tol,
                         int cg_maxit, double *err_out, cudaStream_t st) {
  const int nc = (int)cells.size();
  if (nc == 0) return;
  int W = 0;
  for (int c : cells) W = std::max(W, Kt[c]);
  std::vector<int64_t> row0(nc + 1, 0), ptr(1, 0), col, cb_off(nc, 0);
  std::vector<double> val, Bv, Cbv, dinv;
  std::vector<int32_t> Kb(nc), K(nc), mc(nc);
  for (int i = 0; i < nc; ++i) {
    const Cell &cl = P.cells[cells[i]];
    row0[i + 1] = row0[i] + (int64_t)cl.nodes.size();
    for (int64_t r = 0; r < cl.A.n; ++r) {
      double diag = 0;
      for (int64_t k = cl.A.ptr[r]; k < cl.A.ptr[r + 1]; ++k) {
        col.push_back(row0[i] + cl.A.col[k]);
        val.push_back(cl.A.val[k]);
        if (cl.A.col[k] == r) diag = cl.A.val[k];
      }
      ptr.push_back((int64_t)col.size());
      dinv.push_back(1.0 / (-diag - shift * cl.B[r]));
    }
    Bv.insert(Bv.end(), cl.B.begin(), cl.B.end());
    cb_off[i] = (int64_t)Cbv.size();
    Cbv.insert(Cbv.end(), Cb[cells[i]].begin(), Cb[cells[i]].end());
    Kb[i] = (int32_t)cl.K;
    K[i] = Kt[cells[i]];
    mc[i] = R.cell_m[cells[i]];
  }
  const int64_t rows = row0[nc], NW = rows * W;
  DevMem d_row0, d_ptr, d_col, d_val, d_B, d_dinv, d_Cb, d_cboff, d_Kb, d_Kt, d_mc;
  upload(d_row0, row0);
  upload(d_ptr, ptr);
  upload(d_col, col);
  upload(d_val, val);
  upload(d_B, Bv);
  upload(d_dinv, dinv);
  upload(d_Cb, Cbv);
  upload(d_cboff, cb_off);
  upload(d_Kb, Kb);
  upload(d_Kt, K);
  upload(d_mc, mc);
  DevMem X, Y, cr, cz, cp, cq, G, sb1, sb2, sb3, sb4, sb5, mx;
  for (DevMem *b : {&X, &Y, &cr, &cz, &cp, &cq}) b->alloc(NW * 8);
  G.alloc((size_t)nc * W * W * 8);
  for (DevMem *b : {&sb1, &sb2, &sb3, &sb4, &sb5}) b->alloc((size_t)nc * W * 8);
  mx.alloc(8);
  double *s1 = sb1.as<double>(), *s2 = sb2.as<double>(), *s3 = sb3.as<double>(), *s4 = sb4.as<double>(),
         *s5 = sb5.as<double>();
  const int64_t *r0 = d_row0.as<int64_t>();
  const int32_t *kt = d_Kt.as<int32_t>();
  // X = C; solve -(A + sB) Y = C
  k_expand_c<<<nblk(NW), kThreads, 0, st>>>(X.as<double>(), d_Cb.as<double>(), d_cboff.as<int64_t>(), r0,
                                           d_Kb.as<int32_t>(), kt, d_B.as<double>(), nc, rows, W, 0);
  k_coldot<<<nc, 128, 0, st>>>(s5, nullptr, X.as<double>(), X.as<double>(), nullptr, r0, kt, W);
  k_cg_init<<<nblk(NW), kThreads, 0, st>>>(Y.as<double>(), cr.as<double>(), cz.as<double>(), cp.as<double>(), X.as<double>(),
                                          d_dinv.as<double>(), r0, kt, nc, rows, W);
  k_coldot<<<nc, 128, 0, st>>>(s1, nullptr, cr.as<double>(), cz.as<double>(), nullptr, r0, kt, W);
  bool conv = false;
  for (int it = 0; it < cg_maxit; ++it) {
    k_spmm<<<nblk(NW), kThreads, 0, st>>>(cq.as<double>(), cp.as<double>(), d_ptr.as<int64_t>(), d_col.as<int64_t>(),
                                         d_val.as<double>(), d_B.as<double>(), shift, r0, kt, nc, rows, W, 1);
    k_coldot<<<nc, 128, 0, st>>>(s2, nullptr, cp.as<double>(), cq.as<double>(), nullptr, r0, kt, W);
    k_cg_xr<<<nblk(NW), kThreads, 0, st>>>(Y.as<double>(), cr.as<double>(), cz.as<double>(), cp.as<double>(), cq.as<double>(),
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
  MSS_REQUIRE(conv, MSS_ERR_NOT_CONVERGED, "shifted CG of the screen did not reach the tolerance");
  // F = -C^T Y, packed K x K per cell
  const dim3 ggram(nc, (W + 15) / 16, (W + 15) / 16);
  k_gram<<<ggram, kThreads, 0, st>>>(G.as<double>(), X.as<double>(), Y.as<double>(), nullptr, r0, kt, W);
  std::vector<double> Gh((size_t)nc * W * W);
  MSS_CUDA(cudaMemcpyAsync(Gh.data(), G.p, Gh.size() * 8, cudaMemcpyDeviceToHost, st));
  MSS_CUDA(cudaStreamSynchronize(st));
  std::vector<int64_t> f_off(nc + 1, 0), c_off(nc + 1, 0), w_off(nc + 1, 0);
  std::vector<double> Fv, gam, gh;
  for (int i = 0; i < nc; ++i) {
    const int k = K[i], c = cells[i];
    f_off[i + 1] = f_off[i] + (int64_t)k * k;
    for (int a = 0; a < k; ++a)
      for (int bb = 0; bb < k; ++bb) Fv.push_back(-Gh[(size_t)i * W * W + (size_t)a * W + bb]);
    const int64_t n = (int64_t)mc[i] * k * k;
    c_off[i + 1] = c_off[i] + n;
    gam.insert(gam.end(), R.gamma.begin() + R.coef_off[c], R.gamma.begin() + R.coef_off[c] + n);
    gh.insert(gh.end(), R.gamma_hat.begin() + R.coef_off[c], R.gamma_hat.begin() + R.coef_off[c] + n);
    w_off[i + 1] = w_off[i] + 6LL * k * k;
  }
  DevMem d_F, d_foff, d_gam, d_gh, d_coff, d_work, d_woff, d_err;
  upload(d_F, Fv);
  upload(d_foff, f_off);
  upload(d_gam, gam);
  upload(d_gh, gh);
  upload(d_coff, c_off);
  d_work.alloc(w_off[nc] * 8);
  upload(d_woff, w_off);
  d_err.alloc(nc * 8);
  k_sfrac_err<<<nc, kThreads, 0, st>>>(d_gam.as<double>(), d_gh.as<double>(), d_coff.as<int64_t>(), kt, d_mc.as<int32_t>(),
                                       shift, d_F.as<double>(), d_foff.as<int64_t>(), d_work.as<double>(),
                                       d_woff.as<int64_t>(), d_err.as<double>());
  MSS_CUDA(cudaGetLastError());
  MSS_CUDA(cudaMemcpyAsync(err_out, d_err.p, nc * 8, cudaMemcpyDeviceToHost, st));
  MSS_CUDA(cudaStreamSynchronize(st));
}

// Slot of each boundary row of cell c in the fixed surrogate layout: face on the low / high side
// of axis a -> slot 2a / 2a+1 (slot_modes rows each), I/O face -> rows after the 6 slots.
static void cell_slots(const Partition &P, const Rom &R, int c, int slot_modes, int io_slots, std::vector<int> &row_of,
                       float *feat) {
  row_of.clear();
  const Cell &cl = P.cells[c];
  if (feat)
    for (int j = 0; j < 7; ++j) feat[j] = 0.f;
  for (int f : cl.faces) {
    const Face &F = P.faces[f];
    const int M = R.face_M[f];
    int base;
    if (F.kind == 1) {
      MSS_REQUIRE(M <= io_slots, MSS_ERR_INVALID_ARG, "I/O face larger than the surrogate's I/O slots");
      base = 6 * slot_modes;
      if (feat) feat[6] = (float)M / (float)io_slots;
    } else {
      MSS_REQUIRE(M <= slot_modes, MSS_ERR_INVALID_ARG, "face has more modes than the surrogate's slots");
      const int slot = 2 * F.axis + (F.cells[0] == c ? 1 : 0);
      base = slot * slot_modes;
      if (feat) feat[slot] = 1.f;
    }
    for (int j = 0; j < M; ++j) row_of.push_back(base + j);
  }
}

// In-place lower Cholesky factor of an SPD n x n row-major matrix (upper part zeroed); false if
// a pivot is not positive.
static bool cholesky_lower(double *A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = v / d;
    }
    for (int k = j + 1; k < n; ++k) A[(size_t)j * n + k] = 0.0;
  }
  return true;
}

// Row-major lower-triangle position of (a, b), a >= b.
static inline int64_t tri_index(int a, int b) { return (int64_t)a * (a + 1) / 2 + b; }

// Packed factors -> Gamma^k (k = 1..m) and Gamma-hat^k (k = 2..m) = L L^T of the listed cells.
static void unpack_cells(Rom &R, const Partition &P, const std::vector<int> &cells, int slot_modes, int io_slots,
                         const double *packed) {
  const int Kp = 6 * slot_modes + io_slots;
  const int64_t tri = (int64_t)Kp * (Kp + 1) / 2;
  std::vector<int> row_of;
  std::vector<double> L;
  for (size_t i = 0; i < cells.size(); ++i) {
    const int c = cells[i];
    MSS_REQUIRE(c >= 0 && c < R.n_cells, MSS_ERR_INVALID_ARG, "cell out of range");
    const int m = R.cell_m[c], K = R.cell_K[c];
    const int64_t D = (int64_t)(2 * m - 1) * tri;
    cell_slots(P, R, c, slot_modes, io_slots, row_of, nullptr);
    const double *t = packed + (int64_t)i * D;
    L.assign((size_t)K * K, 0.0);
    for (int q = 0; q < 2 * m - 1; ++q) {
      for (int a = 0; a < K; ++a)
        for (int b2 = 0; b2 <= a; ++b2) {
          const double v = t[(int64_t)q * tri + tri_index(row_of[a], row_of[b2])];
          L[(size_t)a * K + b2] = a == b2 ? std::exp(v) : v;
        }
      double *Mq = q < m ? R.gamma.data() + R.coef_off[c] + (size_t)q * K * K
                         : R.gamma_hat.data() + R.coef_off[c] + (size_t)(q - m + 1) * K * K;
      for (int a = 0; a < K; ++a)
        for (int b2 = 0; b2 <= a; ++b2) {
          double acc = 0;
          for (int k = 0; k <= b2; ++k) acc += L[(size_t)a * K + k] * L[(size_t)b2 * K + k];
          Mq[(size_t)a * K + b2] = acc;
          Mq[(size_t)b2 * K + a] = acc;
        }
    }
  }
}

}  // namespace mss

using namespace mss;

extern "C" {

mss_status mss_rom_skeleton(const mss_partition *p, const mss_rom_params *prm, const int32_t *cell_m, mss_rom **out) {
  return guard([&] {
    const Range nvtx_range("mss_rom_skeleton");
    MSS_REQUIRE(p && prm && out, MSS_ERR_INVALID_ARG, "null argument");
    auto h = std::make_unique<mss_rom>();
    Partition &P = const_cast<Partition &>(p->p);
    std::vector<int> Kt, mv;
    std::vector<std::vector<double>> Cb;
    rom_topology(P, *prm, cell_m, h->r, Kt, mv, Cb);
    std::vector<int> all(P.n_cells);
    std::iota(all.begin(), all.end(), 0);
    rom_exact_markov(P, all, h->r);
    rom_faces(p->p, h->r);
    h->r.prm = *prm;
    *out = h.release();
  });
}

mss_status mss_rom_rebuild_cells(mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells, void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_rom_rebuild_cells");
    MSS_REQUIRE(r && p && n >= 0 && (n == 0 || cells), MSS_ERR_INVALID_ARG, "bad argument");
    Rom &R = r->r;
    MSS_REQUIRE(R.source == &p->p, MSS_ERR_STATE, "ROM was not built from this partition");
    Partition &P = const_cast<Partition &>(p->p);
    std::vector<int> list(cells, cells + n);
    for (int c : list) MSS_REQUIRE(c >= 0 && c < R.n_cells, MSS_ERR_INVALID_ARG, "cell out of range");
    Rom tmp = R;   // topology recomputation below must not disturb the ROM's face bases
    std::vector<int> Kt, mv;
    std::vector<std::vector<double>> Cb;
    rom_topology(P, R.prm, R.cell_m.data(), tmp, Kt, mv, Cb);
    tmp.gamma = R.gamma;
    tmp.gamma_hat = R.gamma_hat;
    rom_exact_cells(P, list, Kt, mv, Cb, R.prm, tmp, (cudaStream_t)stream);
    rom_exact_markov(P, list, tmp);   // keep Gamma-hat^1 (and so the face masses) exact
    R.gamma.swap(tmp.gamma);
    R.gamma_hat.swap(tmp.gamma_hat);
  });
}

mss_status mss_surrogate_cell_inputs(const mss_partition *p, int32_t n, const int32_t *cells, int32_t slot_modes,
                                     int32_t io_slots, float *x, float *feat) {
  return guard([&] {
    MSS_REQUIRE(p && n >= 1 && cells && x && feat && slot_modes >= 1 && io_slots >= 0, MSS_ERR_INVALID_ARG,
                "bad argument");
    const Partition &P = p->p;
    const mss_grid &g = P.op->g;
    MSS_REQUIRE(P.d == 3 && P.cs[0] == P.cs[1] && P.cs[1] == P.cs[2], MSS_ERR_INVALID_ARG, "cubic 3D cells required");
    const int c3 = P.cs[0];
    Rom dummy;
    dummy.face_M.assign(P.faces.size(), 0);
    for (size_t f = 0; f < P.faces.size(); ++f)
      dummy.face_M[f] = P.faces[f].kind == 1 ? (int)P.faces[f].nodes.size()
                                               : std::min<int>(slot_modes, (int)P.faces[f].nodes.size());
    std::vector<int> row_of;
    for (int i = 0; i < n; ++i) {
      const int c = cells[i];
      MSS_REQUIRE(c >= 0 && c < P.n_cells, MSS_ERR_INVALID_ARG, "cell out of range");
      const int *C = P.cells[c].coords;
      float *xs = x + (int64_t)i * 2 * c3 * c3 * c3, *xr = xs + (int64_t)c3 * c3 * c3;
      for (int a = 0; a < c3; ++a)
        for (int b2 = 0; b2 < c3; ++b2)
          for (int d2 = 0; d2 < c3; ++d2) {
            const int64_t v = (((int64_t)(C[0] * c3 + a) * g.n[1]) + C[1] * c3 + b2) * g.n[2] + C[2] * c3 + d2;
            const int64_t o = ((int64_t)a * c3 + b2) * c3 + d2;
            xs[o] = (float)std::log(P.sigma[v]);
            xr[o] = (float)std::log(P.rho[v]);
          }
      cell_slots(P, dummy, c, slot_modes, io_slots, row_of, feat + (int64_t)i * 7);
    }
  });
}

mss_status mss_surrogate_pack(const mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells, int32_t slot_modes,
                              int32_t io_slots, double *targets, float *mask) {
  return guard([&] {
    MSS_REQUIRE(r && p && n >= 1 && cells && targets && slot_modes >= 1, MSS_ERR_INVALID_ARG, "bad argument");
    const Rom &R = r->r;
    const int Kp = 6 * slot_modes + io_slots;
    const int64_t tri = (int64_t)Kp * (Kp + 1) / 2;
    const int m = R.cell_m[cells[0]];
    const int64_t D = (int64_t)(2 * m - 1) * tri;
    std::vector<int> row_of;
    std::vector<double> L;
    for (int i = 0; i < n; ++i) {
      const int c = cells[i];
      MSS_REQUIRE(c >= 0 && c < R.n_cells && R.cell_m[c] == m, MSS_ERR_INVALID_ARG, "cells must share m");
      cell_slots(p->p, R, c, slot_modes, io_slots, row_of, nullptr);
      const int K = R.cell_K[c];
      double *t = targets + (int64_t)i * D;
      std::fill(t, t + D, 0.0);
      if (mask) std::fill(mask + (int64_t)i * D, mask + (int64_t)(i + 1) * D, 0.f);
      for (int q = 0; q < 2 * m - 1; ++q) {
        const double *Mq = q < m ? R.gamma.data() + R.coef_off[c] + (size_t)q * K * K
                                 : R.gamma_hat.data() + R.coef_off[c] + (size_t)(q - m + 1) * K * K;
        L.assign(Mq, Mq + (size_t)K * K);
        MSS_REQUIRE(cholesky_lower(L.data(), K), MSS_ERR_COEF_NOT_SPD, "a coefficient block is not SPD");
        for (int a = 0; a < K; ++a)
          for (int b2 = 0; b2 <= a; ++b2) {
            const int64_t o = (int64_t)q * tri + tri_index(row_of[a], row_of[b2]);
            t[o] = a == b2 ? std::log(L[(size_t)a * K + a]) : L[(size_t)a * K + b2];
            if (mask) mask[(int64_t)i * D + o] = 1.f;
          }
      }
    }
  });
}

mss_status mss_surrogate_unpack(mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells, int32_t slot_modes,
                                int32_t io_slots, const double *packed) {
  return guard([&] {
    MSS_REQUIRE(r && p && n >= 1 && cells && packed, MSS_ERR_INVALID_ARG, "bad argument");
    unpack_cells(r->r, p->p, std::vector<int>(cells, cells + n), slot_modes, io_slots, packed);
  });
}

mss_status mss_surrogate_screen(const mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells, double *err,
                                void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_surrogate_screen");
    MSS_REQUIRE(r && p && n >= 1 && cells && err, MSS_ERR_INVALID_ARG, "bad argument");
    const Rom &R = r->r;
    MSS_REQUIRE(R.source == &p->p, MSS_ERR_STATE, "ROM was not built from this partition");
    Partition &P = const_cast<Partition &>(p->p);
    Rom tmp;
    std::vector<int> Kt, mv;
    std::vector<std::vector<double>> Cb;
    rom_topology(P, R.prm, R.cell_m.data(), tmp, Kt, mv, Cb);
    std::vector<int> list(cells, cells + n);
    screen_cells(P, list, Kt, Cb, R, R.prm.shift, R.prm.cg_tol, R.prm.cg_maxit, err, (cudaStream_t)stream);
  });
}

mss_status mss_surrogate_infer(mss_surrogate *sur, mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells,
                               int32_t slot_modes, int32_t io_slots, double tol, double *err, int32_t *fallback,
                               void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_surrogate_infer");
    MSS_REQUIRE(sur && r && p && n >= 1 && cells && err && fallback && tol > 0, MSS_ERR_INVALID_ARG, "bad argument");
    Rom &R = r->r;
    MSS_REQUIRE(R.source == &p->p, MSS_ERR_STATE, "ROM was not built from this partition");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t info[4];
    mss_status e = mss_surrogate_info(sur, info);
    MSS_REQUIRE(e == MSS_OK, e, "surrogate info");
    const int Kp = 6 * slot_modes + io_slots;
    const int64_t tri = (int64_t)Kp * (Kp + 1) / 2;
    const int m = R.cell_m[cells[0]];
    for (int i = 0; i < n; ++i)
      MSS_REQUIRE(cells[i] >= 0 && cells[i] < R.n_cells && R.cell_m[cells[i]] == m, MSS_ERR_INVALID_ARG,
                  "cells must exist and share m");
    MSS_REQUIRE(info[2] == 7 && info[3] == (2 * m - 1) * tri, MSS_ERR_INVALID_ARG,
                "surrogate outputs do not match the slot layout");
    const int64_t nx = info[1];
    std::vector<float> x((size_t)n * nx), f((size_t)n * 7);
    e = mss_surrogate_cell_inputs(p, n, cells, slot_modes, io_slots, x.data(), f.data());
    MSS_REQUIRE(e == MSS_OK, e, "surrogate inputs");
    DevMem dx, df, dy;
    upload(dx, x);
    upload(df, f);
    dy.alloc((size_t)n * info[3] * 4);
    e = mss_surrogate_predict(sur, n, dx.as<float>(), df.as<float>(), dy.as<float>(), stream);
    MSS_REQUIRE(e == MSS_OK, e, "surrogate forward");
    std::vector<float> yh((size_t)n * info[3]);
    MSS_CUDA(cudaMemcpyAsync(yh.data(), dy.p, yh.size() * 4, cudaMemcpyDeviceToHost, st));
    MSS_CUDA(cudaStreamSynchronize(st));
    std::vector<double> yd(yh.begin(), yh.end());
    std::vector<int> list(cells, cells + n);
    unpack_cells(R, p->p, list, slot_modes, io_slots, yd.data());
    Partition &P = const_cast<Partition &>(p->p);
    Rom tmp;
    std::vector<int> Kt, mv;
    std::vector<std::vector<double>> Cb;
    rom_topology(P, R.prm, R.cell_m.data(), tmp, Kt, mv, Cb);
    screen_cells(P, list, Kt, Cb, R, R.prm.shift, R.prm.cg_tol, R.prm.cg_maxit, err, st);
    std::vector<int> bad;
    for (int i = 0; i < n; ++i) {
      fallback[i] = !(err[i] <= tol);
      if (fallback[i]) bad.push_back(cells[i]);
    }
    rom_exact_cells(P, bad, Kt, mv, Cb, R.prm, R, st);
    rom_exact_markov(P, bad, R);
  });
}

}  // extern "C"

namespace mss {
}  // namespace mss

using namespace mss;

extern "C" mss_status mss_layer_rule_cell(const double *A, const double *S, int32_t K, int32_t m_lo, int32_t m_hi,
                                          double omega_max, double tol, int32_t n_freq, int32_t *m_out, double *errs) {
  return guard([&] {
    MSS_REQUIRE(A && S && m_out && errs && K >= 1, MSS_ERR_INVALID_ARG, "null argument or K < 1");
    MSS_REQUIRE(m_lo >= 1 && m_hi >= m_lo && omega_max > 0 && tol > 0 && n_freq >= 1, MSS_ERR_INVALID_ARG,
                "need 1 <= m_lo <= m_hi, omega_max > 0, tol > 0, n_freq >= 1");
    const LayerRule rule{m_lo, m_hi, n_freq, omega_max, tol, nullptr, nullptr};
    std::vector<double> e;
    MSS_REQUIRE(layer_rule_cell(A, S, K, rule, e), MSS_ERR_LANCZOS_BREAKDOWN, "singular pivot block");
    int mpick = m_hi;
    for (int m = m_lo; m <= m_hi; ++m)
      if (e[m] <= tol) { mpick = m; break; }
    for (int m = 0; m <= m_hi; ++m) errs[m] = m >= m_lo ? e[m] : 0.0;
    *m_out = mpick;
  });
}

extern "C" mss_status mss_layer_rule(const mss_partition *p, const mss_rom_params *prm, int32_t m_lo, int32_t m_hi,
                                     double omega_max, double tol, int32_t n_freq, int32_t *cell_m, double *err,
                                     void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_layer_rule");
    MSS_REQUIRE(p && prm && cell_m, MSS_ERR_INVALID_ARG, "null argument");
    MSS_REQUIRE(m_lo >= 1 && m_hi >= m_lo && omega_max > 0 && tol > 0 && n_freq >= 1, MSS_ERR_INVALID_ARG,
                "need 1 <= m_lo <= m_hi, omega_max > 0, tol > 0, n_freq >= 1");
    Partition &P = const_cast<Partition &>(p->p);
    const LayerRule rule{m_lo, m_hi, n_freq, omega_max, tol, cell_m, err};
    // the m_hi-layer projection of every cell, as mss_build_roms makes it (chunks bounded by memory)
    std::vector<int32_t> mh(P.n_cells, m_hi);
    Rom R;
    std::vector<int> Kt, mv;
    std::vector<std::vector<double>> Cb;
    rom_topology(P, *prm, mh.data(), R, Kt, mv, Cb);
    size_t free_b = 0, total_b = 0;
    MSS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    int Wmax = 0;
    for (int c = 0; c < P.n_cells; ++c) Wmax = std::max(Wmax, Kt[c]);
    const double budget = std::min<double>(0.5 * (double)free_b, 48e9);
    const cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> chunk;
    double used = 0;
    for (int c = 0; c < P.n_cells; ++c) {
      const double need = (double)P.cells[c].nodes.size() * Wmax * 8.0 * (m_hi + 7) +
                          8.0 * ((double)m_hi * Kt[c]) * ((double)m_hi * Kt[c]) * 3;
      if (!chunk.empty() && used + need > budget) {
        build_chunk(P, chunk, Kt, mv, Cb, prm->shift, prm->cg_tol, prm->cg_maxit, R, st, &rule);
        chunk.clear();
        used = 0;
      }
      chunk.push_back(c);
      used += need;
    }
    if (!chunk.empty()) build_chunk(P, chunk, Kt, mv, Cb, prm->shift, prm->cg_tol, prm->cg_maxit, R, st, &rule);
  });
}

extern "C" mss_status mss_build_roms(const mss_partition *p, const mss_rom_params *prm, const int32_t *cell_m, void *stream,
                                     mss_rom **out) {
  return guard([&] {
    const Range nvtx_range("mss_build_roms");
    MSS_REQUIRE(p && prm && out, MSS_ERR_INVALID_ARG, "null argument");
    auto h = std::make_unique<mss_rom>();
    build_roms(p->p, *prm, cell_m, (cudaStream_t)stream, h->r);
    *out = h.release();
  });
}
