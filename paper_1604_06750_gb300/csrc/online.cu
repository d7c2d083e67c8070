// On-line stage of the multiscale S-fraction ROM (Algorithm alg1red, stage 2).
//
// One time step is two or three kernels:
//   k_cell   -- per (cell, source tile): F^k = Gamma^k (U^{k+1} - U^k), k = 1..m (fluxes of
//               Eq. intrtstep_td), the face slices of F^1 published to the flux buffer (the
//               exchange of step 2.1), and the hidden-layer leapfrog
//               U^k <- 2U^k - U^k_old + tau^2 Gamma-hat^k (F^k - F^{k-1}), k = 2..m (step 2.2);
//   k_face   -- per (face, source tile): u~_f <- 2u~_f - u~_f,old + tau^2 M_f^{-1}(sum of the
//               cells' F^1 slices - g~_f w(t_n)) (Eq. bdrytstep, step 2.3); extra blocks sample
//               the receivers (Eq. solatrec) from the state before the update;
//   k_corner -- optional Appendix D correction of the new face level, on the faces that carry
//               hanging nodes (their values u^ are computed by k_face).
// U^1 of a cell is gathered from the face state (Eq. contred: one state per face, shared by
// both cells).  Coefficient matrices are symmetric; the thread that owns output row r reads
// Gamma[c][r] for c = 0..K-1, so the threads of a warp read consecutive addresses.
// The time loop can be captured as a CUDA graph (cached per call signature).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <thread>
#include <type_traits>

#include "cuda_util.h"

namespace mss {

template <typename T>
struct StepArgs {
  // cells
  const int32_t *cell_K, *cell_m;
  const int64_t *cell_coef, *cell_ghat, *cell_state, *cell_row;
  const int64_t *row_face_row;   // per cell boundary row: global face row
  const int8_t *row_side;        // 0 = lower cell of the face, 1 = upper cell
  // faces
  const int32_t *face_M, *face_two;
  const int64_t *face_row, *face_minv;
  const int32_t *fsrc_ptr, *fsrc_index;
  const int64_t *fsrc_val;
  // receivers
  const int32_t *rcv_ptr, *rcv_face;
  const int64_t *rcv_off;
  // receivers read off hidden layers (Galerkin lift of nodes inside cells; null when none): per
  // receiver entries rh_ptr[r]..rh_ptr[r+1]-1 of rh_cnt values at rh_val + rh_off, dotted with the
  // current cell state rows rh_row0 .. rh_row0 + rh_cnt - 1
  const int32_t *rh_ptr, *rh_cnt;
  const int64_t *rh_row0, *rh_off;
  const T *rh_val;
  // corners: members listed per face (fm_*), per corner group (grp_ptr), member data (mem_*),
  // faces that carry members (cfaces)
  const int32_t *fm_ptr, *fm_member, *mem_group, *mem_face, *grp_ptr, *cfaces;
  const int64_t *mem_row;
  // per face, its members' rows of S_f laid out contiguously (fm_rows from fm_roff[f]), and per
  // member entry (member, first and past-last member of its group): one load, no index chains
  const int64_t *fm_roff;
  const int4 *fm_info;
  // values
  const T *coef, *minv, *src_val, *rcv_val, *cg_rows, *cg_w, *fm_rows;
  T *fstate0, *fstate1, *cstate0, *cstate1, *flux, *uhat;
  int S, n_cells, n_faces, n_rcv, corners, n_cfaces;
  // 1: the block of Gamma^m in coef holds W = L + L^T - diag(L), L the lower Cholesky factor of
  // Gamma^m, and F^m = L (L^T D^m) is formed from it in two triangular passes
  int factor_last;
  T tau2;
};

constexpr int kCellThreads = 256;
constexpr int kFaceThreads = 128;
constexpr int kChunk = 8;      // coefficients loaded ahead per thread (register pipeline)

// Bulk prefetch of [p, p + bytes) into L2 (cp.async.bulk.prefetch), trimmed inward to 16-byte
// boundaries, in 32 KB pieces issued by the first threads of the block.  Nothing outside the range
// is touched.
__device__ __forceinline__ void prefetch_l2_range(const void *p, size_t bytes) {
  constexpr uintptr_t kPiece = 32768;
  const uintptr_t lo = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t hi = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  const uintptr_t at = lo + (uintptr_t)threadIdx.x * kPiece;
  if (lo < hi && at < hi) {
    const unsigned n = (unsigned)(hi - at < kPiece ? hi - at : kPiece);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(at), "r"(n) : "memory");
  }
}


// d0 += a b0, d1 += a b1 as one paired FP32 FMA (fma.rn.f32x2): each lane rounds exactly like
// a scalar FMA, half the instructions.
__device__ __forceinline__ void fma2(float &d0, float &d1, float a, float b0, float b1) {
  asm("{\n .reg .b64 pa, pb, pc;\n mov.b64 pa, {%2, %2};\n mov.b64 pb, {%3, %4};\n mov.b64 pc, {%0, %1};\n"
      " fma.rn.f32x2 pc, pa, pb, pc;\n mov.b64 {%0, %1}, pc;\n}"
      : "+f"(d0), "+f"(d1)
      : "f"(a), "f"(b0), "f"(b1));
}

// acc[s] = sum_c G[c*K] * X[c*ST + s] for the thread's output row (G already offset by the row).
// The column stream of G is software-pipelined in registers: the next kChunk loads are issued
// before the current kChunk values are consumed; the caller has bulk-prefetched the whole matrix
// into L2, so each register load waits on L2 rather than on HBM.
template <typename T, int ST>
__device__ __forceinline__ void row_times_block(const T *__restrict__ G, int K, const T *__restrict__ X,
                                                T (&acc)[ST]) {
#pragma unroll
  for (int s = 0; s < ST; ++s) acc[s] = T(0);
  T g[kChunk], gn[kChunk];
#pragma unroll
  for (int j = 0; j < kChunk; ++j) g[j] = j < K ? __ldg(G + (size_t)j * K) : T(0);
  for (int c0 = 0; c0 < K; c0 += kChunk) {
    const int c1 = c0 + kChunk;
#pragma unroll
    for (int j = 0; j < kChunk; ++j) gn[j] = (c1 + j < K) ? __ldg(G + (size_t)(c1 + j) * K) : T(0);
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      if (c0 + j < K) {
        const T *x = X + (c0 + j) * ST;
        if constexpr (std::is_same<T, float>::value && ST % 2 == 0) {
#pragma unroll
          for (int s = 0; s < ST; s += 2) fma2(acc[s], acc[s + 1], g[j], x[s], x[s + 1]);
        } else {
#pragma unroll
          for (int s = 0; s < ST; ++s) acc[s] += g[j] * x[s];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kChunk; ++j) g[j] = gn[j];
  }
}

// acc[s] += sum over c = c1-1 down to c0 of G[c*K] * X[c*ST + s]: the column stream of
// row_times_block over a column range in descending order (one triangle of a factored
// coefficient; the streamed kernels meet the rows of that matrix in the same order), accumulating.
template <typename T, int ST>
__device__ __forceinline__ void row_times_range_desc(const T *__restrict__ G, int K, const T *__restrict__ X, int c0,
                                                     int c1, T (&acc)[ST]) {
  T g[kChunk], gn[kChunk];
#pragma unroll
  for (int j = 0; j < kChunk; ++j) g[j] = c1 - 1 - j >= c0 ? __ldg(G + (size_t)(c1 - 1 - j) * K) : T(0);
  for (int cb = c1 - 1; cb >= c0; cb -= kChunk) {
    const int cn = cb - kChunk;
#pragma unroll
    for (int j = 0; j < kChunk; ++j) gn[j] = (cn - j >= c0) ? __ldg(G + (size_t)(cn - j) * K) : T(0);
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      if (cb - j >= c0) {
        const T *x = X + (cb - j) * ST;
        if constexpr (std::is_same<T, float>::value && ST % 2 == 0) {
#pragma unroll
          for (int s = 0; s < ST; s += 2) fma2(acc[s], acc[s + 1], g[j], x[s], x[s + 1]);
        } else {
#pragma unroll
          for (int s = 0; s < ST; ++s) acc[s] += g[j] * x[s];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kChunk; ++j) g[j] = gn[j];
  }
}

// 16-byte vector type of T (4 floats or 2 doubles)
template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };
__device__ __forceinline__ float4 pack_vec(const float (&d)[4]) { return make_float4(d[0], d[1], d[2], d[3]); }
__device__ __forceinline__ double2 pack_vec(const double (&d)[2]) { return make_double2(d[0], d[1]); }

// One (cell, source tile) of the cell phase with the CUDA cores; any block size.
template <typename T, int ST, int FAC = -1>   // FAC: 0/1 fixes the factored-last flag at compile time, -1 reads it
__device__ __forceinline__ void cell_item(const StepArgs<T> &a, const int cur, const int cell, const int tile,
                                          unsigned char *smem_raw) {
  const int s0 = tile * ST;
  const int K = a.cell_K[cell], m = a.cell_m[cell];
  const int ns = min(ST, a.S - s0);
  T *X = reinterpret_cast<T *>(smem_raw);        // U (layers 1..m, [k][r][s]), then F^k
  T *D = X + (size_t)m * K * ST;                 // U^{k+1} - U^k, then F^k - F^{k-1}
  T *Y = D + (size_t)m * K * ST;                 // factored last coefficient: L^T D^m (even length)
  const bool fac = FAC < 0 ? a.factor_last != 0 : FAC != 0;
  const size_t ylen = fac ? (((size_t)K * ST + 1) & ~(size_t)1) : 0;
  int64_t *rows = reinterpret_cast<int64_t *>(Y + ylen);   // K boundary rows: face row*2+side
  const T *fs = cur ? a.fstate1 : a.fstate0;
  const T *cs = cur ? a.cstate1 : a.cstate0;
  T *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t rp = a.cell_row[cell];
  const int64_t so = a.cell_state[cell];
  const int S = a.S;
  if (tile == 0) prefetch_l2_range(a.coef + a.cell_coef[cell], sizeof(T) * (size_t)(2 * m - 1) * K * K);
  for (int r = threadIdx.x; r < K; r += blockDim.x) rows[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
  __syncthreads();
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  // vector path needs whole vectors of sources inside the tile and aligned rows
  const bool vec = (ST >= VN) && (ST % VN == 0) && (ns == ST) && (S % VN == 0) && (s0 % VN == 0);
  if (vec) {
    constexpr int NV = ST >= VN ? ST / VN : 1;
    for (int i = threadIdx.x; i < K * NV; i += blockDim.x) {
      const int r = i / NV, v = i - r * NV;
      reinterpret_cast<V *>(X)[i] = *reinterpret_cast<const V *>(fs + (rows[r] >> 1) * S + s0 + v * VN);
    }
    for (int i = threadIdx.x; i < (m - 1) * K * NV; i += blockDim.x) {
      const int r = i / NV, v = i - r * NV;
      reinterpret_cast<V *>(X + (size_t)K * ST)[i] = *reinterpret_cast<const V *>(cs + (so + r) * S + s0 + v * VN);
    }
  } else {
    for (int i = threadIdx.x; i < K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      X[i] = s < ns ? fs[(rows[r] >> 1) * S + s0 + s] : T(0);
    }
    for (int i = threadIdx.x; i < (m - 1) * K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      X[(size_t)K * ST + i] = s < ns ? cs[(so + r) * S + s0 + s] : T(0);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m * K * ST; i += blockDim.x) {
    const int k = i / (K * ST);
    D[i] = (k + 1 < m ? X[i + (size_t)K * ST] : T(0)) - X[i];
  }
  __syncthreads();
  // fluxes F^k = Gamma^k D^k into X (U is not needed any more: the "now" level is re-read below)
  const T *G = a.coef + a.cell_coef[cell];
  if (!fac) {
    for (int it = threadIdx.x; it < m * K; it += blockDim.x) {
      const int k = it / K, r = it - k * K;
      T acc[ST];
      row_times_block<T, ST>(G + (size_t)k * K * K + r, K, D + (size_t)k * K * ST, acc);
#pragma unroll
      for (int s = 0; s < ST; ++s) X[(size_t)k * K * ST + r * ST + s] = acc[s];
    }
    __syncthreads();
  } else {
    // F^1..F^{m-1} as above; F^m = L (L^T D^m) with W = L + L^T - diag(L) read column by column:
    // y_r = sum_{c >= r} W[c][r] D^m_c (L^T), then F^m_r = sum_{c <= r} W[c][r] y_c (L), both
    // summed over c in descending order.  Rows r and K-1-r share an item, so every item streams
    // K+1 coefficients of the triangle pair.
    const T *W = G + (size_t)(m - 1) * K * K;
    const T *Dm = D + (size_t)(m - 1) * K * ST;
    const int full = (m - 1) * K, pairs = (K + 1) / 2;
    for (int it = threadIdx.x; it < full + pairs; it += blockDim.x) {
      if (it < full) {
        const int k = it / K, r = it - k * K;
        T acc[ST];
        row_times_block<T, ST>(G + (size_t)k * K * K + r, K, D + (size_t)k * K * ST, acc);
#pragma unroll
        for (int s = 0; s < ST; ++s) X[(size_t)k * K * ST + r * ST + s] = acc[s];
      } else {
        const int p = it - full;
        for (int h = 0; h < 2; ++h) {
          const int r = h ? K - 1 - p : p;
          if (h && r == p) break;
          T acc[ST];
#pragma unroll
          for (int s = 0; s < ST; ++s) acc[s] = T(0);
          row_times_range_desc<T, ST>(W + r, K, Dm, r, K, acc);
#pragma unroll
          for (int s = 0; s < ST; ++s) Y[r * ST + s] = acc[s];
        }
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
      for (int h = 0; h < 2; ++h) {
        const int r = h ? K - 1 - p : p;
        if (h && r == p) break;
        T acc[ST];
#pragma unroll
        for (int s = 0; s < ST; ++s) acc[s] = T(0);
        row_times_range_desc<T, ST>(W + r, K, Y, 0, r + 1, acc);
#pragma unroll
        for (int s = 0; s < ST; ++s) X[(size_t)(m - 1) * K * ST + r * ST + s] = acc[s];
      }
    }
    __syncthreads();
  }
  // exchange: this cell's F^1 on each of its faces; E^k = F^k - F^{k-1} into D
  if (vec) {
    constexpr int NV = ST >= VN ? ST / VN : 1;
    for (int i = threadIdx.x; i < K * NV; i += blockDim.x) {
      const int r = i / NV, v = i - r * NV;
      *reinterpret_cast<V *>(a.flux + rows[r] * S + s0 + v * VN) = reinterpret_cast<const V *>(X)[i];
    }
  } else {
    for (int i = threadIdx.x; i < K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      if (s < ns) a.flux[rows[r] * S + s0 + s] = X[i];
    }
  }
  for (int i = threadIdx.x; i < (m - 1) * K * ST; i += blockDim.x) {
    const size_t j = (size_t)K * ST + i;
    D[j] = X[j] - X[j - (size_t)K * ST];
  }
  __syncthreads();
  const T *H = a.coef + a.cell_ghat[cell];
  const T tau2 = a.tau2;
  for (int it = threadIdx.x; it < (m - 1) * K; it += blockDim.x) {
    const int k = 1 + it / K, r = it - (k - 1) * K;
    T acc[ST];
    row_times_block<T, ST>(H + (size_t)(k - 1) * K * K + r, K, D + (size_t)k * K * ST, acc);
    const int64_t base = (so + (int64_t)(k - 1) * K + r) * S + s0;
    if (vec) {
#pragma unroll
      for (int v = 0; v < (ST >= VN ? ST / VN : 0); ++v) {
        const V now = *reinterpret_cast<const V *>(cs + base + v * VN);
        V old = *reinterpret_cast<const V *>(cso + base + v * VN);
        T *o = reinterpret_cast<T *>(&old);
        const T *nw = reinterpret_cast<const T *>(&now);
#pragma unroll
        for (int e = 0; e < VN; ++e) o[e] = T(2) * nw[e] - o[e] + tau2 * acc[v * VN + e];
        *reinterpret_cast<V *>(cso + base + v * VN) = old;
      }
    } else {
#pragma unroll
      for (int s = 0; s < ST; ++s)
        if (s < ns) cso[base + s] = T(2) * cs[base + s] - cso[base + s] + tau2 * acc[s];
    }
  }
}

// FAC: the factored last coefficient (a separate instantiation, so that the plain kernel keeps
// its register budget)
template <typename T, int ST, bool FAC = false>
__global__ void __launch_bounds__(kCellThreads, sizeof(T) == 4 ? 4 : 2) k_cell(const StepArgs<T> a, const int cur) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 1-D grid, source tiles of a cell adjacent so that they share its coefficients in L2
  const int tiles = (a.S + ST - 1) / ST;
  cell_item<T, ST, FAC ? 1 : 0>(a, cur, blockIdx.x / tiles, blockIdx.x % tiles, smem_raw);
}

// Item b of the face phase: b < n_faces is a face update, the rest are receiver blocks of
// blockDim.x / ST receivers each (sampled before the state advances).
template <typename T, int ST>
__device__ __forceinline__ void face_item(const StepArgs<T> &a, const int cur, const int b, const int tile,
                                          const double *w, T *traces, unsigned char *smem_raw) {
  const int s0 = tile * ST;
  const int ns = min(ST, a.S - s0);
  const int S = a.S;
  const T *fs = cur ? a.fstate1 : a.fstate0;
  if (b < a.n_faces) {
    const int f = b, M = a.face_M[f];
    const int j0 = a.corners ? a.fm_ptr[f] : 0, nm = a.corners ? a.fm_ptr[f + 1] - j0 : 0;
    T *sum = reinterpret_cast<T *>(smem_raw);    // M x ST flux sums
    T *nv = sum + (size_t)M * ST;                // M x ST new face values (corner correction only)
    T *mi = nv + (size_t)M * ST;                 // M x M inverse face mass
    T *rw = mi + (size_t)M * M;                  // nm x M rows of S_f of the face's hanging nodes
    const int64_t row0 = a.face_row[f];
    const bool two = a.face_two[f] != 0;
    const T wn = (T)(*w);
    // stage everything the face needs in one round of independent loads
    for (int i = threadIdx.x; i < M * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      T v = T(0);
      if (s < ns) {
        v = a.flux[((row0 + r) * 2) * S + s0 + s];
        if (two) v += a.flux[((row0 + r) * 2 + 1) * S + s0 + s];
        for (int e = a.fsrc_ptr[f]; e < a.fsrc_ptr[f + 1]; ++e)
          if (a.fsrc_index[e] == s0 + s) v -= a.src_val[a.fsrc_val[e] + r] * wn;
      }
      sum[i] = v;
    }
    const T *Mi = a.minv + a.face_minv[f];
    for (int i = threadIdx.x; i < M * M; i += blockDim.x) mi[i] = Mi[i];
    if (nm > 0) {
      const T *src = a.fm_rows + a.fm_roff[f];
      for (int i = threadIdx.x; i < nm * M; i += blockDim.x) rw[i] = src[i];
    }
    __syncthreads();
    T *dst = cur ? a.fstate0 : a.fstate1;        // the old level becomes the new one
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::n;
    constexpr int NV = ST % VN == 0 ? ST / VN : 1;
    const bool vec = (ST % VN == 0) && (ns == ST) && (S % VN == 0);
    if (vec) {
      // same products in the same order as the scalar loops below, VN sources per thread
      for (int i = threadIdx.x; i < M * NV; i += blockDim.x) {
        const int r = i / NV, v = i - r * NV;
        T acc[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) acc[e] = T(0);
        for (int c = 0; c < M; ++c) {
          const T mv = mi[r * M + c];
          const V x = *reinterpret_cast<const V *>(sum + c * ST + v * VN);
          const T *xe = reinterpret_cast<const T *>(&x);
#pragma unroll
          for (int e = 0; e < VN; ++e) acc[e] += mv * xe[e];
        }
        const int64_t idx = (row0 + r) * S + s0 + v * VN;
        const V fv = *reinterpret_cast<const V *>(fs + idx);
        V dv = *reinterpret_cast<const V *>(dst + idx);
        const T *fe = reinterpret_cast<const T *>(&fv);
        T *de = reinterpret_cast<T *>(&dv);
#pragma unroll
        for (int e = 0; e < VN; ++e) de[e] = T(2) * fe[e] - de[e] + a.tau2 * acc[e];
        *reinterpret_cast<V *>(dst + idx) = dv;
        if (a.corners) *reinterpret_cast<V *>(nv + r * ST + v * VN) = dv;
      }
      if (nm > 0) {
        __syncthreads();
        for (int i = threadIdx.x; i < nm * NV; i += blockDim.x) {
          const int j = i / NV, v = i - j * NV;
          const int l = a.fm_member[j0 + j];
          T d[VN];
#pragma unroll
          for (int e = 0; e < VN; ++e) d[e] = T(0);
          for (int c = 0; c < M; ++c) {
            const T rv = rw[j * M + c];
            const V x = *reinterpret_cast<const V *>(nv + c * ST + v * VN);
            const T *xe = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int e = 0; e < VN; ++e) d[e] += rv * xe[e];
          }
          *reinterpret_cast<V *>(a.uhat + (int64_t)l * S + s0 + v * VN) = pack_vec(d);
        }
      }
      return;
    }
    for (int i = threadIdx.x; i < M * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      T acc = T(0);
      for (int c = 0; c < M; ++c) acc += mi[r * M + c] * sum[c * ST + s];
      if (s < ns) {
        const int64_t idx = (row0 + r) * S + s0 + s;
        const T v = T(2) * fs[idx] - dst[idx] + a.tau2 * acc;
        dst[idx] = v;
        if (a.corners) nv[i] = v;
      } else if (a.corners) {
        nv[i] = T(0);
      }
    }
    if (nm > 0) {
      // values of this face's hanging nodes, u^_l = s_l . u~_f (Appendix D step 1), pre-correction
      __syncthreads();
      for (int i = threadIdx.x; i < nm * ST; i += blockDim.x) {
        const int j = i / ST, s = i - j * ST;
        if (s >= ns) continue;
        const int l = a.fm_member[j0 + j];
        T d = T(0);
        for (int c = 0; c < M; ++c) d += rw[j * M + c] * nv[c * ST + s];
        a.uhat[(int64_t)l * S + s0 + s] = d;
      }
    }
  } else {
    // receivers: sample the state at this step, before it is advanced
    const int per = (int)blockDim.x / ST;
    const int r = (b - a.n_faces) * per + (int)threadIdx.x / ST;
    const int s = (int)threadIdx.x % ST;
    if (r >= a.n_rcv || s >= ns) return;
    T acc = T(0);
    for (int e = a.rcv_ptr[r]; e < a.rcv_ptr[r + 1]; ++e) {
      const int f = a.rcv_face[e];
      const int M = a.face_M[f];
      const int64_t row0 = a.face_row[f];
      const T *q = a.rcv_val + a.rcv_off[e];
      for (int c = 0; c < M; ++c) acc += q[c] * fs[(row0 + c) * S + s0 + s];
    }
    if (a.rh_ptr) {
      const T *cs = cur ? a.cstate1 : a.cstate0;
      for (int e = a.rh_ptr[r]; e < a.rh_ptr[r + 1]; ++e) {
        const int64_t row0 = a.rh_row0[e];
        const T *q = a.rh_val + a.rh_off[e];
        for (int c = 0; c < a.rh_cnt[e]; ++c) acc += q[c] * cs[(row0 + c) * S + s0 + s];
      }
    }
    traces[(int64_t)r * S + s0 + s] = acc;
  }
}

// Appendix D steps 2-3 on the faces that carry hanging nodes: delta_l = sum_{l' in g} w_l' u^_l'
// - u^_l from the pre-correction values u^ (computed by k_face), then u~_f += sum_l s_l delta_l,
// in place on the new level (each block touches only its own face's rows).
template <typename T, int ST>
__global__ void __launch_bounds__(kFaceThreads) k_face(const StepArgs<T> a, const int cur, const double *w,
                                                       T *traces) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  face_item<T, ST>(a, cur, blockIdx.x, blockIdx.y, w, traces, smem_raw);
}

template <typename T, int ST>
__device__ __forceinline__ void corner_item(const StepArgs<T> &a, const int cur, const int ci, const int tile,
                                            unsigned char *smem_raw) {
  const int f = a.cfaces[ci];
  const int s0 = tile * ST;
  const int ns = min(ST, a.S - s0);
  const int S = a.S;
  const int M = a.face_M[f];
  const int64_t row0 = a.face_row[f];
  T *dst = cur ? a.fstate0 : a.fstate1;
  const int j0 = a.fm_ptr[f], nm = a.fm_ptr[f + 1] - j0;
  T *delta = reinterpret_cast<T *>(smem_raw);   // nm x ST
  T *rowsm = delta + (size_t)nm * ST;           // nm x M member rows of S_f
  {
    const T *src = a.fm_rows + a.fm_roff[f];
    for (int i = threadIdx.x; i < nm * M; i += blockDim.x) rowsm[i] = src[i];
  }
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  constexpr int NV = ST % VN == 0 ? ST / VN : 1;
  if ((ST % VN == 0) && (ns == ST) && (S % VN == 0)) {
    // same products in the same order as the scalar loops below, VN sources per thread
    for (int i = threadIdx.x; i < nm * NV; i += blockDim.x) {
      const int j = i / NV, v = i - j * NV;
      const int4 info = a.fm_info[j0 + j];
      const int l = info.x;
      T mean[VN];
#pragma unroll
      for (int e = 0; e < VN; ++e) mean[e] = T(0);
#pragma unroll 4
      for (int l2 = info.y; l2 < info.z; ++l2) {
        const T wv = a.cg_w[l2];
        const V x = *reinterpret_cast<const V *>(a.uhat + (int64_t)l2 * S + s0 + v * VN);
        const T *xe = reinterpret_cast<const T *>(&x);
#pragma unroll
        for (int e = 0; e < VN; ++e) mean[e] += wv * xe[e];
      }
      const V self = *reinterpret_cast<const V *>(a.uhat + (int64_t)l * S + s0 + v * VN);
      const T *se = reinterpret_cast<const T *>(&self);
      T d[VN];
#pragma unroll
      for (int e = 0; e < VN; ++e) d[e] = mean[e] - se[e];
      *reinterpret_cast<V *>(delta + j * ST + v * VN) = pack_vec(d);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M * NV; i += blockDim.x) {
      const int r = i / NV, v = i - r * NV;
      T acc[VN];
#pragma unroll
      for (int e = 0; e < VN; ++e) acc[e] = T(0);
      for (int j = 0; j < nm; ++j) {
        const T rv = rowsm[j * M + r];
        const V x = *reinterpret_cast<const V *>(delta + j * ST + v * VN);
        const T *xe = reinterpret_cast<const T *>(&x);
#pragma unroll
        for (int e = 0; e < VN; ++e) acc[e] += rv * xe[e];
      }
      T *o = dst + (row0 + r) * S + s0 + v * VN;
      V ov = *reinterpret_cast<const V *>(o);
      T *oe = reinterpret_cast<T *>(&ov);
#pragma unroll
      for (int e = 0; e < VN; ++e) oe[e] += acc[e];
      *reinterpret_cast<V *>(o) = ov;
    }
    return;
  }
  for (int i = threadIdx.x; i < nm * ST; i += blockDim.x) {
    const int j = i / ST, s = i - j * ST;
    T d = T(0);
    if (s < ns) {
      const int4 info = a.fm_info[j0 + j];
      const int l = info.x;
      T mean = T(0);
#pragma unroll 4
      for (int l2 = info.y; l2 < info.z; ++l2) mean += a.cg_w[l2] * a.uhat[(int64_t)l2 * S + s0 + s];
      d = mean - a.uhat[(int64_t)l * S + s0 + s];
    }
    delta[i] = d;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < M * ST; i += blockDim.x) {
    const int r = i / ST, s = i - r * ST;
    if (s >= ns) continue;
    T v = T(0);
    for (int j = 0; j < nm; ++j) v += rowsm[j * M + r] * delta[j * ST + s];
    dst[(row0 + r) * S + s0 + s] += v;
  }
}

template <typename T, int ST>
__global__ void __launch_bounds__(kFaceThreads) k_corner(const StepArgs<T> a, const int cur) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  corner_item<T, ST>(a, cur, blockIdx.x, blockIdx.y, smem_raw);
}

}  // namespace mss

#include "cell_tc.cuh"
#include "cell_stream.cuh"
#include "cell_wide.cuh"
#include "cell_split.cuh"
#include "cell_tc_split.cuh"
#include "cell_tc_pipe.cuh"
#include "cell_tw.cuh"

namespace mss {

// ------------------------------------------------------------------ simulation object
struct SimDev {
  DevMem cell_K, cell_m, cell_coef, cell_ghat, cell_state, cell_row, row_face_row, row_side;
  DevMem face_M, face_two, face_row, face_minv, fsrc_ptr, fsrc_index, fsrc_val;
  DevMem rcv_ptr, rcv_face, rcv_off, rh_ptr, rh_cnt, rh_row0, rh_off, rh_val;
  DevMem fm_ptr, fm_member, mem_group, mem_face, grp_ptr, mem_row, fm_roff, fm_info, fm_rows;
  DevMem coef, minv, src_val, rcv_val, cg_rows, cg_w;
  DevMem fstate[2], cstate[2], flux, uhat, cfaces, wbuf, tbuf;
  DevMem tc_blob, tc_off, tc_Kp, tc_Kr, tc_err;
  DevMem tw_blob, tw_off;               // wide tensor-core (TF32) cell kernel blob
  DevMem sc_coef, sc_off, sc_Kq, bar;   // streamed cell kernel blob, grid barrier words
  DevMem flux_items, accel_items, f_off, F;   // split cell phase
};

struct GraphKey {
  int64_t n;
  const void *w, *t;
  int cur, sched, variant;
  bool operator<(const GraphKey &o) const {
    return std::tie(n, w, t, cur, sched, variant) < std::tie(o.n, o.w, o.t, o.cur, o.sched, o.variant);
  }
};

}  // namespace mss

struct mss_sim {
  int prec = MSS_FP64;
  int tc = 0, tc_terms = 3, tc_nt = 16;       // tensor-core cell kernel
  size_t tc_smem = 0;
  int tcs_nt = 16;                             // split tensor-core kernels: sources per CTA
  size_t tcs_smem = 0;
  size_t tcp_smem = 0;                         // pipelined split tensor-core kernels
  int tcp_krmax = 8, tcp_slots = 1;
  int tcq_nt = 0, tcq_grid = 1;                // warp-specialised persistent tensor-core kernel
  size_t tcq_smem = 0;
  int tc_kpmax = 16, st_max = 1, dev_smem = 0;
  bool stream_blob = false;                    // streamed-kernel coefficient copy present
  bool wide_blob = false, wide_ok = false;     // wide streamed kernel (K_i up to 384) usable
  size_t wide_smem = 0, wide_smem8 = 0;       // with 16- and 8-source tiles
  int wide_var = 0;                            // its variant: bit 0 unroll 4 (else 2), bit 1 two rows per
                                               // thread (else 4), bit 2 8-source tiles (else 16)
  mss::TcArgs tca{};
  int tw = 0;                                  // MSS_TF32_TC: the wide tensor-core cell kernel
  int tw_ring_max = 2;                         // its copy-ring slots: the most that fit; twa.ring in use
  size_t tw_smem = 0;
  mss::TwArgs twa{};
  int n_cells = 0, n_faces = 0, n_src = 0, n_rcv = 0, ST = 1, tiles = 1;
  int corners = 0, max_K = 0, max_m = 0, max_M = 0, max_nm = 0, n_cfaces = 0;
  int factor_last = 0;                         // FP32: Gamma^m applied as L (L^T .)
  int n_rh = 0;                                // receiver entries on hidden layers
  int64_t face_rows = 0, cell_rows = 0;
  int64_t steps = 0;
  int cur = 0;
  double tau = 0;
  size_t cell_smem = 0, face_smem = 0, corner_smem = 0;
  // schedule of the step: MSS_SCHED_* (graph-captured kernels, plain or streamed cell kernel,
  // or the persistent time-block kernel with either cell body)
  int sched = MSS_SCHED_GRAPH;
  bool stream_ok = false;
  int stream_groups = 4;             // column groups (128 threads each) of the streamed cell kernel
  size_t stream_smem = 0;
  mss::StreamArgs sca{};
  int persist_block = 512;           // steps per persistent launch
  int n_flux_items = 0, n_accel_items = 0;
  size_t split_smem = 0;
  int64_t dev_bytes = 0;
  mss::SimDev d;
  std::map<mss::GraphKey, cudaGraphExec_t> graphs;
  int device = 0;
  cudaStream_t cap = nullptr;          // capture/replay stream, joined to the caller's stream by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ~mss_sim() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace mss {

template <typename T>
static StepArgs<T> make_args(const mss_sim &s) {
  const SimDev &d = s.d;
  StepArgs<T> a;
  a.cell_K = d.cell_K.as<int32_t>();
  a.cell_m = d.cell_m.as<int32_t>();
  a.cell_coef = d.cell_coef.as<int64_t>();
  a.cell_ghat = d.cell_ghat.as<int64_t>();
  a.cell_state = d.cell_state.as<int64_t>();
  a.cell_row = d.cell_row.as<int64_t>();
  a.row_face_row = d.row_face_row.as<int64_t>();
  a.row_side = d.row_side.as<int8_t>();
  a.face_M = d.face_M.as<int32_t>();
  a.face_two = d.face_two.as<int32_t>();
  a.face_row = d.face_row.as<int64_t>();
  a.face_minv = d.face_minv.as<int64_t>();
  a.fsrc_ptr = d.fsrc_ptr.as<int32_t>();
  a.fsrc_index = d.fsrc_index.as<int32_t>();
  a.fsrc_val = d.fsrc_val.as<int64_t>();
  a.rcv_ptr = d.rcv_ptr.as<int32_t>();
  a.rcv_face = d.rcv_face.as<int32_t>();
  a.rcv_off = d.rcv_off.as<int64_t>();
  a.rh_ptr = s.n_rh ? d.rh_ptr.as<int32_t>() : nullptr;
  a.rh_cnt = d.rh_cnt.as<int32_t>();
  a.rh_row0 = d.rh_row0.as<int64_t>();
  a.rh_off = d.rh_off.as<int64_t>();
  a.rh_val = d.rh_val.as<T>();
  a.fm_ptr = d.fm_ptr.as<int32_t>();
  a.fm_member = d.fm_member.as<int32_t>();
  a.mem_group = d.mem_group.as<int32_t>();
  a.mem_face = d.mem_face.as<int32_t>();
  a.grp_ptr = d.grp_ptr.as<int32_t>();
  a.mem_row = d.mem_row.as<int64_t>();
  a.fm_roff = d.fm_roff.as<int64_t>();
  a.fm_info = d.fm_info.as<int4>();
  a.fm_rows = d.fm_rows.as<T>();
  a.coef = d.coef.as<T>();
  a.minv = d.minv.as<T>();
  a.src_val = d.src_val.as<T>();
  a.rcv_val = d.rcv_val.as<T>();
  a.cg_rows = d.cg_rows.as<T>();
  a.cg_w = d.cg_w.as<T>();
  a.fstate0 = d.fstate[0].as<T>();
  a.fstate1 = d.fstate[1].as<T>();
  a.cstate0 = d.cstate[0].as<T>();
  a.cstate1 = d.cstate[1].as<T>();
  a.flux = d.flux.as<T>();
  a.uhat = d.uhat.as<T>();
  a.cfaces = d.cfaces.as<int32_t>();
  a.S = s.n_src;
  a.n_cells = s.n_cells;
  a.n_faces = s.n_faces;
  a.n_rcv = s.n_rcv;
  a.corners = s.corners;
  a.n_cfaces = s.n_cfaces;
  a.factor_last = s.factor_last;
  a.tau2 = (T)(s.tau * s.tau);
  return a;
}

template <typename T, int ST>
static void set_smem_attrs(const mss_sim &s) {
  if (s.tc && s.tcq_nt) {
    MSS_CUDA(cudaFuncSetAttribute(k_cell_tcp<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tcq_smem));
    MSS_CUDA(cudaFuncSetAttribute(k_cell_tcp<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tcq_smem));
  }
  if (s.tc) {
    for (const void *kf : {(const void *)k_tc_split<16, true>, (const void *)k_tc_split<16, false>,
                           (const void *)k_tc_split<32, true>, (const void *)k_tc_split<32, false>,
                           (const void *)k_tc_split<64, true>, (const void *)k_tc_split<64, false>,
                           (const void *)k_tc_split<128, true>, (const void *)k_tc_split<128, false>})
      MSS_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tcs_smem));
    for (const void *kf : {(const void *)k_tc_pipe<16, true>, (const void *)k_tc_pipe<16, false>,
                           (const void *)k_tc_pipe<32, true>, (const void *)k_tc_pipe<32, false>,
                           (const void *)k_tc_pipe<64, true>, (const void *)k_tc_pipe<64, false>,
                           (const void *)k_tc_pipe<128, true>, (const void *)k_tc_pipe<128, false>})
      MSS_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tcp_smem));
    MSS_CUDA(cudaFuncSetAttribute(k_cell_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tc_smem));
    MSS_CUDA(cudaFuncSetAttribute(k_cell_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tc_smem));
    MSS_CUDA(cudaFuncSetAttribute(k_cell_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tc_smem));
  }
  MSS_CUDA(cudaFuncSetAttribute(k_cell<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.cell_smem));
  if (s.tw) MSS_CUDA(cudaFuncSetAttribute(k_cell_tw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tw_smem));
  if (s.factor_last)
    MSS_CUDA(cudaFuncSetAttribute(k_cell<T, ST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.cell_smem));
  if (s.wide_ok) {
    for (const void *kf : {(const void *)k_cell_w<2, 4, 16>, (const void *)k_cell_w<4, 4, 16>,
                           (const void *)k_cell_w<2, 2, 16>, (const void *)k_cell_w<4, 2, 16>})
      MSS_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.wide_smem));
    for (const void *kf : {(const void *)k_cell_w<2, 4, 8>, (const void *)k_cell_w<4, 4, 8>,
                           (const void *)k_cell_w<2, 2, 8>, (const void *)k_cell_w<4, 2, 8>})
      MSS_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.wide_smem8));
  }
  if (s.stream_ok)
  {
    MSS_CUDA(cudaFuncSetAttribute(k_cell_s<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.stream_smem));
    MSS_CUDA(cudaFuncSetAttribute(k_cell_s<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.stream_smem));
  }
  MSS_CUDA(cudaFuncSetAttribute(k_flux<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.split_smem));
  MSS_CUDA(cudaFuncSetAttribute(k_accel<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.split_smem));
  MSS_CUDA(cudaFuncSetAttribute(k_face<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.face_smem));
  MSS_CUDA(cudaFuncSetAttribute(k_corner<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.corner_smem));
}

template <int NT>
static void launch_tcp(const mss_sim &s, const StepArgs<float> &a, int cur, cudaStream_t st) {
  const int total = s.n_cells * ((s.n_src + NT - 1) / NT);
  k_cell_tcp<NT><<<std::min(total, s.tcq_grid), kTcpThreads, s.tcq_smem, st>>>(a, s.tca, cur, s.tcp_krmax, s.max_m);
}

template <int NT>
static void launch_tc(const mss_sim &s, const StepArgs<float> &a, int cur, cudaStream_t st) {
  const dim3 g(s.n_cells * ((s.n_src + NT - 1) / NT));
  k_cell_tc<NT><<<g, kTcThreads, s.tc_smem, st>>>(a, s.tca, cur);
}

template <typename T, int ST>
static void launch_cell(const mss_sim &s, const StepArgs<T> &a, int cur, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (s.tw) {
      k_cell_tw<<<s.n_cells * ((s.n_src + kTwNT - 1) / kTwNT), kTwThreads, s.tw_smem, st>>>(a, s.twa, cur);
      return;
    }
    if (s.tc && s.sched == MSS_SCHED_PERSIST_STREAM) {
      if (s.tcq_nt == 32) launch_tcp<32>(s, a, cur, st);
      else launch_tcp<16>(s, a, cur, st);
      return;
    }
    if (s.tc) {
      switch (s.tc_nt) {
        case 16: launch_tc<16>(s, a, cur, st); return;
        case 32: launch_tc<32>(s, a, cur, st); return;
        default: launch_tc<64>(s, a, cur, st); return;
      }
    }
  }
  const dim3 gc(s.n_cells * s.tiles);
  if constexpr (std::is_same<T, float>::value && ST == kStreamST) {
    if (s.sched == MSS_SCHED_GRAPH_STREAM) {
      if (!s.stream_ok) {
        const dim3 g8(s.n_cells * ((s.n_src + 7) / 8));
        switch (s.wide_var) {
          case 1: k_cell_w<4, 4, 16><<<gc, wide_threads(4, 16), s.wide_smem, st>>>(a, s.sca, cur); break;
          case 2: k_cell_w<2, 2, 16><<<gc, wide_threads(2, 16), s.wide_smem, st>>>(a, s.sca, cur); break;
          case 3: k_cell_w<4, 2, 16><<<gc, wide_threads(2, 16), s.wide_smem, st>>>(a, s.sca, cur); break;
          case 4: k_cell_w<2, 4, 8><<<g8, wide_threads(4, 8), s.wide_smem8, st>>>(a, s.sca, cur); break;
          case 5: k_cell_w<4, 4, 8><<<g8, wide_threads(4, 8), s.wide_smem8, st>>>(a, s.sca, cur); break;
          case 6: k_cell_w<2, 2, 8><<<g8, wide_threads(2, 8), s.wide_smem8, st>>>(a, s.sca, cur); break;
          case 7: k_cell_w<4, 2, 8><<<g8, wide_threads(2, 8), s.wide_smem8, st>>>(a, s.sca, cur); break;
          default: k_cell_w<2, 4, 16><<<gc, wide_threads(4, 16), s.wide_smem, st>>>(a, s.sca, cur); break;
        }
      }
      else if (s.stream_groups == 4) k_cell_s<4><<<gc, 512, s.stream_smem, st>>>(a, s.sca, cur);
      else k_cell_s<2><<<gc, 256, s.stream_smem, st>>>(a, s.sca, cur);
      return;
    }
  }
  if (s.factor_last) k_cell<T, ST, true><<<gc, kCellThreads, s.cell_smem, st>>>(a, cur);
  else k_cell<T, ST><<<gc, kCellThreads, s.cell_smem, st>>>(a, cur);
}

template <typename T>
static SplitArgs<T> make_split(const mss_sim &s) {
  SplitArgs<T> p;
  p.flux_items = s.d.flux_items.as<int2>();
  p.accel_items = s.d.accel_items.as<int2>();
  p.f_off = s.d.f_off.as<int64_t>();
  p.F = s.d.F.as<T>();
  return p;
}

template <int NT>
static void launch_tc_split(const mss_sim &s, const StepArgs<float> &a, const SplitArgs<float> &p, int cur,
                            cudaStream_t st) {
  const int tiles = (s.n_src + NT - 1) / NT;
  k_tc_split<NT, true><<<dim3(s.n_flux_items * tiles), kTcsThreads, s.tcs_smem, st>>>(a, p, s.tca, cur);
  if (s.n_accel_items > 0)
    k_tc_split<NT, false><<<dim3(s.n_accel_items * tiles), kTcsThreads, s.tcs_smem, st>>>(a, p, s.tca, cur);
}

template <int NT>
static void launch_tc_pipe(const mss_sim &s, const StepArgs<float> &a, const SplitArgs<float> &p, int cur,
                           cudaStream_t st) {
  const int tiles = (s.n_src + NT - 1) / NT;
  for (int ph = 0; ph < 2; ++ph) {
    const int n_items = ph == 0 ? s.n_flux_items : s.n_accel_items;
    if (n_items == 0) continue;
    const int total = n_items * tiles;
    const int grid = std::min(total, s.tcp_slots);
    if (ph == 0)
      k_tc_pipe<NT, true><<<grid, kTcsThreads, s.tcp_smem, st>>>(a, p, s.tca, cur, n_items, s.tcp_krmax);
    else
      k_tc_pipe<NT, false><<<grid, kTcsThreads, s.tcp_smem, st>>>(a, p, s.tca, cur, n_items, s.tcp_krmax);
  }
}

template <typename T, int ST>
static void launch_split(const mss_sim &s, const StepArgs<T> &a, const SplitArgs<T> &p, int cur, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (s.tc && s.sched == MSS_SCHED_PERSIST) {
      switch (s.tcs_nt) {
        case 16: launch_tc_pipe<16>(s, a, p, cur, st); return;
        case 32: launch_tc_pipe<32>(s, a, p, cur, st); return;
        case 64: launch_tc_pipe<64>(s, a, p, cur, st); return;
        default: launch_tc_pipe<128>(s, a, p, cur, st); return;
      }
    }
    if (s.tc) {
      switch (s.tcs_nt) {
        case 16: launch_tc_split<16>(s, a, p, cur, st); return;
        case 32: launch_tc_split<32>(s, a, p, cur, st); return;
        case 64: launch_tc_split<64>(s, a, p, cur, st); return;
        default: launch_tc_split<128>(s, a, p, cur, st); return;
      }
    }
  }
  k_flux<T, ST><<<dim3(s.n_flux_items * s.tiles), kSplitThreads, s.split_smem, st>>>(a, p, cur);
  if (s.n_accel_items > 0)
    k_accel<T, ST><<<dim3(s.n_accel_items * s.tiles), kSplitThreads, s.split_smem, st>>>(a, p, cur);
}

// Shared memory of the persistent kernel: the largest of its phases.
template <typename T, int ST>
static size_t persist_smem(const mss_sim &s, bool stream) {
  const size_t aux = stream ? (size_t)kStreamSlots * kStreamChunk + 64 : 0;
  return std::max({stream ? s.stream_smem : s.cell_smem, aux + s.face_smem, aux + s.corner_smem});
}

// n steps as persistent launches of at most persist_block steps each (cooperative: the driver
// refuses a grid that cannot be resident at once).
template <typename T, int ST>
static void launch_persist(mss_sim &s, int64_t n, const double *w, T *traces, cudaStream_t st) {
  const bool stream = s.sched == MSS_SCHED_PERSIST_STREAM;
  StepArgs<T> a = make_args<T>(s);
  const size_t smem = persist_smem<T, ST>(s, stream);
  void (*kern)(const StepArgs<T>, const StreamArgs, const int, const int, const double *, T *, unsigned *, const int);
  if constexpr (std::is_same<T, float>::value && ST == kStreamST) {
    kern = stream ? k_persist<T, ST, true> : k_persist<T, ST, false>;
  } else {
    MSS_REQUIRE(!stream, MSS_ERR_INVALID_ARG, "the streamed cell body needs FP32 and 16-source tiles");
    kern = k_persist<T, ST, false>;
  }
  MSS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  MSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCellThreads, smem));
  MSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device));
  MSS_REQUIRE(per_sm >= 1, MSS_ERR_INVALID_ARG, "persistent kernel does not fit on an SM");
  const int per = kCellThreads / ST;
  int n_rcv_items = (s.n_rcv + per - 1) / per;
  const int64_t items = (int64_t)std::max(s.n_cells, s.n_faces + n_rcv_items) * s.tiles;
  int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, std::max<int64_t>(1, items));
  StreamArgs t = s.sca;
  t.err = s.d.tc_err.as<int>();
  unsigned *bar = s.d.bar.as<unsigned>();
  int cur = s.cur;
  for (int64_t j0 = 0; j0 < n; j0 += s.persist_block) {
    int nb = (int)std::min<int64_t>(s.persist_block, n - j0);
    const double *wj = w + j0;
    T *tj = traces + j0 * (int64_t)s.n_rcv * s.n_src;
    MSS_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    void *args[] = {&a, &t, &cur, &nb, &wj, &tj, &bar, &n_rcv_items};
    MSS_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kCellThreads), args, smem, st));
    cur ^= (nb & 1);
  }
}

template <typename T, int ST>
static void launch_steps(mss_sim &s, int64_t n, const double *w, T *traces, cudaStream_t st) {
  const StepArgs<T> a = make_args<T>(s);
  const int per = kFaceThreads / ST;
  const int rcv_blocks = (s.n_rcv + per - 1) / per;
  const dim3 gc(s.n_cells, s.tiles), gf(s.n_faces + rcv_blocks, s.tiles), gk(std::max(1, s.n_cfaces), s.tiles);
  int cur = s.cur;
  const SplitArgs<T> sp = make_split<T>(s);
  for (int64_t j = 0; j < n; ++j) {
    if (s.sched == MSS_SCHED_GRAPH_SPLIT || (s.tc && s.sched == MSS_SCHED_PERSIST)) launch_split<T, ST>(s, a, sp, cur, st);
    else launch_cell<T, ST>(s, a, cur, st);
    k_face<T, ST><<<gf, kFaceThreads, s.face_smem, st>>>(a, cur, w + j, traces + j * (int64_t)s.n_rcv * s.n_src);
    if (s.corners) k_corner<T, ST><<<gk, kFaceThreads, s.corner_smem, st>>>(a, cur);
    cur ^= 1;
  }
  MSS_CUDA(cudaGetLastError());
}

template <typename T, int ST>
static void step_impl(mss_sim &s, int64_t n, const double *w, void *traces, int use_graph, cudaStream_t st) {
  set_smem_attrs<T, ST>(s);
  if (!s.tc && (s.sched == MSS_SCHED_PERSIST || s.sched == MSS_SCHED_PERSIST_STREAM)) {
    launch_persist<T, ST>(s, n, w, (T *)traces, st);
  } else if (!use_graph) {
    launch_steps<T, ST>(s, n, w, (T *)traces, st);
  } else {
    // capture and replay on the sim's own stream (the legacy stream cannot be captured)
    MSS_CUDA(cudaEventRecord(s.ev_in, st));
    MSS_CUDA(cudaStreamWaitEvent(s.cap, s.ev_in, 0));
    GraphKey key{n, w, traces, s.cur, s.sched,
                 s.stream_groups + 8 * s.ST + 4096 * s.tcs_nt + 65536 * s.wide_var + (1 << 20) * s.twa.ring};
    auto it = s.graphs.find(key);
    if (it == s.graphs.end()) {
      cudaGraph_t g = nullptr;
      MSS_CUDA(cudaStreamBeginCapture(s.cap, cudaStreamCaptureModeThreadLocal));
      try {
        launch_steps<T, ST>(s, n, w, (T *)traces, s.cap);
      } catch (...) {
        cudaStreamEndCapture(s.cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      MSS_CUDA(cudaStreamEndCapture(s.cap, &g));
      cudaGraphExec_t ge;
      cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      MSS_CUDA(e);
      it = s.graphs.emplace(key, ge).first;
    }
    MSS_CUDA(cudaGraphLaunch(it->second, s.cap));
    MSS_CUDA(cudaEventRecord(s.ev_out, s.cap));
    MSS_CUDA(cudaStreamWaitEvent(st, s.ev_out, 0));
  }
  s.cur = (int)((s.cur + n) & 1);
  s.steps += n;
}

template <typename T, int ST>
static void profile_impl(mss_sim &s, int64_t n, const double *w, T *traces, double ms[3], cudaStream_t st) {
  set_smem_attrs<T, ST>(s);
  const StepArgs<T> a = make_args<T>(s);
  const int per = kFaceThreads / ST;
  const int rcv_blocks = (s.n_rcv + per - 1) / per;
  const dim3 gc(s.n_cells, s.tiles), gf(s.n_faces + rcv_blocks, s.tiles), gk(std::max(1, s.n_cfaces), s.tiles);
  const SplitArgs<T> sp = make_split<T>(s);
  cudaEvent_t ev[4];
  for (auto &e : ev) MSS_CUDA(cudaEventCreate(&e));
  double acc[3] = {0, 0, 0};
  int cur = s.cur;
  try {
    for (int64_t j = 0; j < n; ++j) {
      MSS_CUDA(cudaEventRecord(ev[0], st));
      if (s.sched == MSS_SCHED_GRAPH_SPLIT || (s.tc && s.sched == MSS_SCHED_PERSIST)) launch_split<T, ST>(s, a, sp, cur, st);
      else launch_cell<T, ST>(s, a, cur, st);
      MSS_CUDA(cudaEventRecord(ev[1], st));
      k_face<T, ST><<<gf, kFaceThreads, s.face_smem, st>>>(a, cur, w + j, traces + j * (int64_t)s.n_rcv * s.n_src);
      MSS_CUDA(cudaEventRecord(ev[2], st));
      if (s.corners) k_corner<T, ST><<<gk, kFaceThreads, s.corner_smem, st>>>(a, cur);
      MSS_CUDA(cudaEventRecord(ev[3], st));
      MSS_CUDA(cudaEventSynchronize(ev[3]));
      for (int k = 0; k < 3; ++k) {
        float t = 0;
        MSS_CUDA(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
        acc[k] += t;
      }
      cur ^= 1;
    }
    MSS_CUDA(cudaGetLastError());
  } catch (...) {
    for (auto &e : ev) cudaEventDestroy(e);
    throw;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  for (int k = 0; k < 3; ++k) ms[k] = n > 0 ? acc[k] / (double)n : 0.0;
  if (!s.corners) ms[2] = 0.0;
  s.cur = (int)((s.cur + n) & 1);
  s.steps += n;
}

template <typename T>
static void profile_dispatch(mss_sim &s, int64_t n, const double *w, void *traces, double ms[3], cudaStream_t st) {
  switch (s.ST) {
    case 1: profile_impl<T, 1>(s, n, w, (T *)traces, ms, st); break;
    case 2: profile_impl<T, 2>(s, n, w, (T *)traces, ms, st); break;
    case 4: profile_impl<T, 4>(s, n, w, (T *)traces, ms, st); break;
    case 8: profile_impl<T, 8>(s, n, w, (T *)traces, ms, st); break;
    default: profile_impl<T, 16>(s, n, w, (T *)traces, ms, st); break;
  }
}

template <typename T>
static void step_dispatch(mss_sim &s, int64_t n, const double *w, void *traces, int use_graph, cudaStream_t st) {
  switch (s.ST) {
    case 1: step_impl<T, 1>(s, n, w, traces, use_graph, st); break;
    case 2: step_impl<T, 2>(s, n, w, traces, use_graph, st); break;
    case 4: step_impl<T, 4>(s, n, w, traces, use_graph, st); break;
    case 8: step_impl<T, 8>(s, n, w, traces, use_graph, st); break;
    default: step_impl<T, 16>(s, n, w, traces, use_graph, st); break;
  }
}

template <typename T>
static void upload_as(DevMem &m, const std::vector<double> &v) {
  std::vector<T> t(v.begin(), v.end());
  upload(m, t);
}

// Invert the SPD face masses on the host (Gauss-Jordan with partial pivoting, FP64).
static std::vector<double> inverse(const double *A, int n) {
  std::vector<double> a(A, A + (size_t)n * n), inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    MSS_REQUIRE(a[(size_t)p * n + c] != 0, MSS_ERR_COEF_NOT_SPD, "singular face mass");
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)p * n + k], a[(size_t)c * n + k]);
        std::swap(inv[(size_t)p * n + k], inv[(size_t)c * n + k]);
      }
    const double piv = a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      a[(size_t)c * n + k] /= piv;
      inv[(size_t)c * n + k] /= piv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  return inv;
}

static inline uint16_t host_bf16(float f) {   // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
static inline float host_bf16_to_f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Coefficients of every cell in the tensor-core kernel's layout: per cell the 2m-1 matrices
// Gamma^1..Gamma^m, Gamma-hat^2..Gamma-hat^m, each as BF16 hi then lo, Kr x Kp, K-major core
// matrices (see cell_tc.cuh).
static void build_tc_blob(const Rom &R, std::vector<uint16_t> &blob, std::vector<int64_t> &off, std::vector<int32_t> &Kp,
                          std::vector<int32_t> &Kr) {
  blob.clear();
  off.assign(R.n_cells, 0);
  Kp.assign(R.n_cells, 0);
  Kr.assign(R.n_cells, 0);
  for (int c = 0; c < R.n_cells; ++c) {
    const int K = R.cell_K[c], m = R.cell_m[c];
    const int kp = (K + 15) / 16 * 16, kr = (K + 7) / 8 * 8;
    Kp[c] = kp;
    Kr[c] = kr;
    off[c] = (int64_t)blob.size() * 2;
    const size_t half = (size_t)kr * kp;
    for (int p = 0; p < 2 * m - 1; ++p) {
      const double *A = p < m ? R.gamma.data() + R.coef_off[c] + (size_t)p * K * K
                              : R.gamma_hat.data() + R.coef_off[c] + (size_t)(p - m + 1) * K * K;
      const size_t base = blob.size();
      blob.resize(base + 2 * half, 0);
      for (int r = 0; r < K; ++r)
        for (int k = 0; k < K; ++k) {
          const float v = (float)A[(size_t)r * K + k];
          const uint16_t h = host_bf16(v);
          const uint16_t l = host_bf16(v - host_bf16_to_f(h));
          const size_t o = ((size_t)(r >> 3) * (16 * kp) + (size_t)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) / 2;
          blob[base + o] = h;
          blob[base + half + o] = l;
        }
    }
  }
}

// Coefficients of every cell in the wide tensor-core kernel's layout (cell_tw.cuh): per cell, the
// A blocks of its 2m products in the order the kernel consumes them -- Gamma^1..Gamma^{m-1}, the
// factored last coefficient twice (L^T: W's upper triangle, L: its lower triangle, W = L + L^T -
// diag(L) at matrix m-1 of coef), Gamma-hat^2..Gamma-hat^m; within a product by k chunk, then M
// tile -- each block 128 rows (fewer in the last M tile) x 32 columns (fewer in the last chunk),
// FP32, K-major core-matrix layout.
static void build_tw_blob(const Rom &R, const std::vector<double> &coef, const std::vector<int64_t> &cell_coef,
                          std::vector<float> &blob, std::vector<int64_t> &off) {
  blob.clear();
  off.assign(R.n_cells, 0);
  for (int c = 0; c < R.n_cells; ++c) {
    const int K = R.cell_K[c], m = R.cell_m[c], K8 = (K + 7) & ~7, MT = tw_mt(K);
    off[c] = (int64_t)blob.size();
    for (int j = 0; j < 2 * m; ++j) {
      const int q = j < m - 1 ? j : (j <= m ? m - 1 : j - 1);
      const double *A = coef.data() + cell_coef[c] + (size_t)q * K * K;
      const int nch = (K8 + 31) / 32;
      for (int ch = 0; ch < nch; ++ch) {
        for (int t = 0; t < MT; ++t) {
          int c0, c1;
          tw_chunks(j, t, m, K, c0, c1);
          if (ch < c0 || ch >= c1) continue;
          const int rows = std::min(128, K8 - 128 * t);
          const int kc = std::min(32, K8 - 32 * ch);
          const size_t base = blob.size();
          blob.resize(base + (size_t)rows * kc, 0.f);
          for (int row = 0; row < rows; ++row)
            for (int k = 0; k < kc; ++k) {
              const int gi = 128 * t + row, gk = 32 * ch + k;
              if (gi >= K || gk >= K) continue;
              if ((j == m - 1 && gk < gi) || (j == m && gk > gi)) continue;   // the other triangle
              blob[base + (size_t)(row >> 3) * (8 * kc) + (size_t)(k >> 2) * 32 + (row & 7) * 4 + (k & 3)] =
                  (float)A[(size_t)gi * K + gk];
            }
        }
      }
    }
  }
}

// Shared memory of the CUDA-core cell kernel: U and D (m K ST values each), the factored last
// coefficient's intermediate (K ST values, rounded up to even), and the K boundary-row indices.
static size_t cell_smem_bytes(int max_m, int max_K, int ST, size_t es, int factor_last) {
  const size_t y = factor_last ? (((size_t)max_K * ST + 1) & ~(size_t)1) : 0;
  return (2 * (size_t)max_m * max_K * ST + y) * es + 8 * (size_t)max_K;
}

// Lower Cholesky factor of a positive semidefinite n x n matrix (row-major, FP64): pivots at or
// below 1e-13 of the largest diagonal entry are raised to that floor; a pivot below -1e-8 of it
// means the matrix is indefinite (returns false).
static bool psd_cholesky_host(const double *M, int n, std::vector<double> &L) {
  double sc = 0;
  for (int i = 0; i < n; ++i) sc = std::max(sc, M[(size_t)i * n + i]);
  if (!(sc > 0)) return false;
  L.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 1e-13 * sc)) {
      if (!(d >= -1e-8 * sc)) return false;
      d = 1e-13 * sc;
    }
    const double piv = std::sqrt(d);
    L[(size_t)j * n + j] = piv;
    for (int i = j + 1; i < n; ++i) {
      double v = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = v / piv;
    }
  }
  return true;
}

// Sizes that depend on the CUDA-core source tile ST (every per-column result is independent of
// the tiling, so changing ST leaves the arithmetic of each source unchanged).
static void apply_tile(mss_sim &s, int ST) {
  const size_t es = s.prec == MSS_FP64 ? 8 : 4;
  s.ST = ST;
  s.tiles = (s.n_src + ST - 1) / ST;
  s.cell_smem = cell_smem_bytes(s.max_m, s.max_K, ST, es, s.factor_last);
  s.corner_smem = std::max<size_t>(16, (size_t)s.max_nm * (ST + s.max_M) * es);
  s.face_smem = std::max<size_t>(16, (2 * (size_t)s.max_M * ST + (size_t)s.max_M * s.max_M +
                                      (s.corners ? (size_t)s.max_nm * s.max_M : 0)) * es);
  s.split_smem = (size_t)s.max_K * ST * es + 8 * (size_t)s.max_K;
  s.stream_ok = s.stream_blob && ST == kStreamST;
  s.wide_ok = s.wide_blob && ST == kStreamST;
}

// Sizes and residency of the split / pipelined tensor-core kernels with NT sources per CTA.
static void apply_tcs_nt(mss_sim &s, int nt) {
  s.tcs_nt = nt;
  s.tcs_smem = tcs_smem_bytes(nt, s.tc_kpmax);
  s.tcp_smem = tcp_smem_bytes(nt, s.tc_kpmax, s.tcp_krmax);
  int sms = 0, per = 0;
  MSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device));
  const void *kf = nt == 16 ? (const void *)k_tc_pipe<16, true>
                   : nt == 32 ? (const void *)k_tc_pipe<32, true>
                   : nt == 64 ? (const void *)k_tc_pipe<64, true>
                              : (const void *)k_tc_pipe<128, true>;
  MSS_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.tcp_smem));
  MSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kf, kTcsThreads, s.tcp_smem));
  // at most 2 resident CTAs per SM keeps TMEM at <= 2 x 128 columns
  s.tcp_slots = std::max(1, std::min(per, 2)) * sms;
}

static void sim_create(mss_sim &s, const Rom &R, int prec, double tau, int flags) {
  MSS_REQUIRE((flags & ~(MSS_SIM_CORNERS | MSS_SIM_FACTOR_LAST)) == 0, MSS_ERR_INVALID_ARG, "unknown sim flags");
  const int corners = flags & MSS_SIM_CORNERS;
  MSS_REQUIRE(!(flags & MSS_SIM_FACTOR_LAST) || prec == MSS_FP32 || prec == MSS_TF32_TC, MSS_ERR_INVALID_ARG,
              "the factored last coefficient is an option of MSS_FP32 (MSS_TF32_TC always applies it)");
  s.factor_last = ((flags & MSS_SIM_FACTOR_LAST) || prec == MSS_TF32_TC) ? 1 : 0;
  MSS_REQUIRE(prec == MSS_FP64 || prec == MSS_FP32 || prec == MSS_FP32_TC || prec == MSS_BF16_TC || prec == MSS_TF32_TC,
              MSS_ERR_INVALID_ARG, "precision must be MSS_FP64, MSS_FP32, MSS_FP32_TC, MSS_BF16_TC or MSS_TF32_TC");
  MSS_REQUIRE(tau > 0 && std::isfinite(tau), MSS_ERR_CFL, "tau must be positive");
  MSS_REQUIRE(R.has_io, MSS_ERR_STATE, "ROM has no sources/receivers (mss_rom_set_io*)");
  MSS_CUDA(cudaGetDevice(&s.device));
  MSS_CUDA(cudaStreamCreateWithFlags(&s.cap, cudaStreamNonBlocking));
  MSS_CUDA(cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming));
  MSS_CUDA(cudaEventCreateWithFlags(&s.ev_out, cudaEventDisableTiming));
  s.prec = prec;
  s.tau = tau;
  s.n_cells = R.n_cells;
  s.n_faces = R.n_faces;
  s.n_src = R.n_src;
  s.n_rcv = R.n_rcv;
  s.corners = (corners && !R.cg_ptr.empty()) ? 1 : 0;
  const int S = s.n_src;
  s.ST = S <= 1 ? 1 : S <= 2 ? 2 : S <= 4 ? 4 : S <= 8 ? 8 : 16;
  const size_t es = prec == MSS_FP64 ? 8 : 4;
  // shrink the source tile until the cell kernel fits shared memory
  s.max_K = *std::max_element(R.cell_K.begin(), R.cell_K.end());
  s.max_m = *std::max_element(R.cell_m.begin(), R.cell_m.end());
  s.max_M = *std::max_element(R.face_M.begin(), R.face_M.end());
  int dev_smem = 0;
  MSS_CUDA(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, s.device));
  auto cell_smem = [&](int st) { return cell_smem_bytes(s.max_m, s.max_K, st, es, s.factor_last); };
  while (s.ST > 1 && cell_smem(s.ST) > (size_t)dev_smem) s.ST /= 2;
  s.cell_smem = cell_smem(s.ST);
  MSS_REQUIRE(s.cell_smem <= (size_t)dev_smem, MSS_ERR_INVALID_ARG, "cell too large for shared memory");
  s.face_smem = std::max<size_t>(16, 2 * (size_t)s.max_M * s.ST * es);
  s.tiles = (S + s.ST - 1) / s.ST;
  if (prec == MSS_FP32_TC || prec == MSS_BF16_TC) {
    MSS_REQUIRE(s.max_K <= 128, MSS_ERR_INVALID_ARG, "tensor-core precisions need K_i <= 128");
    s.tc = 1;
    s.tc_terms = prec == MSS_FP32_TC ? 3 : 1;
    int kpmax = 0;
    for (int K : R.cell_K) kpmax = std::max(kpmax, (K + 15) / 16 * 16);
    int nt = S <= 16 ? 16 : S <= 32 ? 32 : 64;
    int krmax = 8;
    for (int K : R.cell_K) krmax = std::max(krmax, (K + 7) / 8 * 8);
    // two A slots of KrMax rows, max_m B buffers, rows, barriers, and a tail so that the 128-row
    // reads of the last slot stay inside the allocation
    auto smem_of = [&](int ntv) {
      return (size_t)2 * (2 * krmax * kpmax * 2) + (size_t)s.max_m * (2 * ntv * kpmax * 2) + 128 * 8 + 8 * 8 +
             (size_t)128 * kpmax * 2;
    };
    auto cols_of = [&](int ntv) {
      unsigned c = 32;
      while (c < (unsigned)(s.max_m * ntv)) c <<= 1;
      return c;
    };
    while (nt > 16 && (smem_of(nt) > (size_t)dev_smem || cols_of(nt) > 512)) nt /= 2;
    MSS_REQUIRE(smem_of(nt) <= (size_t)dev_smem && cols_of(nt) <= 512, MSS_ERR_INVALID_ARG,
                "cells too large for the tensor-core kernel");
    s.tc_nt = nt;
    s.tc_smem = smem_of(nt);
    s.tc_kpmax = kpmax;
    for (int K : R.cell_K) s.tcp_krmax = std::max(s.tcp_krmax, (K + 7) / 8 * 8);
    apply_tcs_nt(s, S <= 16 ? 16 : S <= 32 ? 32 : S <= 64 ? 64 : 128);
    {
      int sms = 0;
      MSS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.device));
      // warp-specialised persistent kernel: 32-source tiles when they fit, else 16
      for (int ntv : {32, 16}) {
        if (ntv == 32 && S <= 16) continue;
        const size_t need = tcp_smem(ntv, kpmax, s.tcp_krmax, s.max_m, s.max_K);
        if (need <= (size_t)dev_smem && (size_t)s.max_m * ntv <= 512) {
          s.tcq_nt = ntv;
          s.tcq_smem = need;
          break;
        }
      }
      s.tcq_grid = sms;
    }
    std::vector<uint16_t> blob;
    std::vector<int64_t> off;
    std::vector<int32_t> kp, kr;
    build_tc_blob(R, blob, off, kp, kr);
    upload(s.d.tc_blob, blob);
    upload(s.d.tc_off, off);
    upload(s.d.tc_Kp, kp);
    upload(s.d.tc_Kr, kr);
    upload(s.d.tc_err, std::vector<int>(1, 0));
    s.tca.blob = s.d.tc_blob.as<unsigned char>();
    s.tca.blob_off = s.d.tc_off.as<int64_t>();
    s.tca.Kp = s.d.tc_Kp.as<int32_t>();
    s.tca.Kr = s.d.tc_Kr.as<int32_t>();
    s.tca.err = s.d.tc_err.as<int>();
    s.tca.slot_bytes = 2 * krmax * kpmax * 2;
    s.tca.kpmax = kpmax;
    s.tca.krmax = krmax;
    s.tca.bbuf_bytes = 2 * nt * kpmax * 2;
    s.tca.max_m = s.max_m;
    s.tca.terms = s.tc_terms;
    s.tca.tmem_cols = cols_of(nt);
  }
  // topology
  std::vector<int64_t> face_row(R.n_faces + 1, 0), face_minv(R.n_faces, 0);
  std::vector<int32_t> face_two(R.n_faces, 0);
  for (int f = 0; f < R.n_faces; ++f) {
    face_row[f + 1] = face_row[f] + R.face_M[f];
    face_minv[f] = R.fmass_off[f];
    face_two[f] = R.face_cells[2 * f + 1] >= 0 ? 1 : 0;
  }
  s.face_rows = face_row[R.n_faces];
  std::vector<int64_t> cell_coef(R.n_cells), cell_ghat(R.n_cells), cell_state(R.n_cells), cell_row(R.n_cells);
  std::vector<int64_t> row_face_row;
  std::vector<int8_t> row_side;
  std::vector<double> coef;
  int64_t srows = 0;
  for (int c = 0; c < R.n_cells; ++c) {
    const int K = R.cell_K[c], m = R.cell_m[c];
    cell_coef[c] = (int64_t)coef.size();
    const double *g = R.gamma.data() + R.coef_off[c];
    coef.insert(coef.end(), g, g + (int64_t)m * K * K);
    cell_ghat[c] = (int64_t)coef.size();
    const double *h = R.gamma_hat.data() + R.coef_off[c] + (int64_t)K * K;
    coef.insert(coef.end(), h, h + (int64_t)(m - 1) * K * K);
    cell_state[c] = srows;
    srows += (int64_t)(m - 1) * K;
    cell_row[c] = (int64_t)row_face_row.size();
    for (int k = R.cell_face_ptr[c]; k < R.cell_face_ptr[c + 1]; ++k) {
      const int f = R.cell_faces[k];
      const int8_t side = R.face_cells[2 * f] == c ? 0 : 1;
      for (int r = 0; r < R.face_M[f]; ++r) {
        row_face_row.push_back(face_row[f] + r);
        row_side.push_back(side);
      }
    }
  }
  s.cell_rows = srows;
  if (s.factor_last) {
    // Gamma^m of every cell -> W = L + L^T - diag(L), L its (floored) lower Cholesky factor;
    // cells are independent, factored on the host threads
    const int nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<int> bad(nt, -1);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
      pool.emplace_back([&, t] {
        std::vector<double> L;
        for (int c = t; c < R.n_cells; c += nt) {
          const int K = R.cell_K[c], m = R.cell_m[c];
          double *Wc = coef.data() + cell_coef[c] + (size_t)(m - 1) * K * K;
          if (!psd_cholesky_host(Wc, K, L)) {
            if (bad[t] < 0) bad[t] = c;
            continue;
          }
          for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) Wc[(size_t)i * K + j] = i >= j ? L[(size_t)i * K + j] : L[(size_t)j * K + i];
        }
      });
    for (auto &th : pool) th.join();
    for (int b : bad)
      MSS_REQUIRE(b < 0, MSS_ERR_COEF_NOT_SPD, "last coefficient of cell " + std::to_string(b) + " is indefinite");
  }
  if (prec == MSS_TF32_TC) {
    // wide tensor-core kernel: K_i <= 384, 2m accumulators of 16 columns per M tile in TMEM, the
    // largest copy ring (2..8 slots of 16 KB) that fits beside the stages and B buffers
    MSS_REQUIRE(s.max_K <= kTwMaxK, MSS_ERR_INVALID_ARG, "MSS_TF32_TC needs K_i <= 384");
    unsigned cols = 32;
    for (int c = 0; c < R.n_cells; ++c)
      while (cols < (unsigned)(2 * R.cell_m[c] * tw_mt(R.cell_K[c]) * kTwNT)) cols <<= 1;
    MSS_REQUIRE(cols <= 512, MSS_ERR_INVALID_ARG, "MSS_TF32_TC: 2 m_i ceil(K_i / 128) x 16 accumulator columns exceed TMEM");
    const int k8max = (s.max_K + 7) & ~7;
    int ring = kTwMaxRing;
    while (ring > 2 && tw_smem_bytes(ring, k8max) > (size_t)dev_smem) --ring;
    MSS_REQUIRE(tw_smem_bytes(ring, k8max) <= (size_t)dev_smem, MSS_ERR_INVALID_ARG,
                "MSS_TF32_TC: cells too large for shared memory");
    std::vector<float> blob;
    std::vector<int64_t> off;
    build_tw_blob(R, coef, cell_coef, blob, off);
    upload(s.d.tw_blob, blob);
    upload(s.d.tw_off, off);
    s.tw = 1;
    s.tw_smem = tw_smem_bytes(ring, k8max);
    s.twa.blob = s.d.tw_blob.as<float>();
    s.twa.blob_off = s.d.tw_off.as<int64_t>();
    s.twa.ring = ring;
    s.tw_ring_max = ring;
    s.twa.k8max = k8max;
    s.twa.tmem_cols = cols;
  }
  {
    // split cell phase: one item per (cell, matrix) and an F scratch block of m K rows per cell
    std::vector<int2> fi, ai;
    std::vector<int64_t> foff(R.n_cells);
    int64_t frows = 0;
    for (int c = 0; c < R.n_cells; ++c) {
      foff[c] = frows;
      frows += (int64_t)R.cell_m[c] * R.cell_K[c];
      for (int k = 0; k < R.cell_m[c]; ++k) fi.push_back(make_int2(c, k));
      for (int k = 1; k < R.cell_m[c]; ++k) ai.push_back(make_int2(c, k));
    }
    upload(s.d.flux_items, fi);
    upload(s.d.accel_items, ai.empty() ? std::vector<int2>(1, make_int2(0, 1)) : ai);
    upload(s.d.f_off, foff);
    s.d.F.alloc((size_t)frows * S * es);
    s.n_flux_items = (int)fi.size();
    s.n_accel_items = (int)ai.size();
    s.split_smem = (size_t)s.max_K * s.ST * es + 8 * (size_t)s.max_K;
  }
  // streamed cell kernels: FP32 CUDA-core path with 16-source tiles; the same matrices as coef,
  // each row padded to Kq = K rounded up to 4 floats (16-byte rows).  k_cell_s takes K_i <= 128
  // (not the factored last coefficient), the wide kernel K_i <= 512; in the wide kernel's copy the
  // factored last coefficient's rows are stored in descending order.
  if (prec == MSS_FP32 && !s.tc && s.ST == kStreamST) {
    const size_t need = (size_t)kStreamSlots * kStreamChunk + 64 + 2 * (size_t)s.max_m * s.max_K * kStreamST * 4 +
                        8 * (size_t)s.max_K;
    const bool narrow = !s.factor_last && s.max_K <= 128 && need <= (size_t)dev_smem;
    const size_t wneed = wide_smem_bytes(s.max_m, s.max_K, s.factor_last, 16);
    const bool wide = s.max_K <= kWideMaxK && wneed <= (size_t)dev_smem;
    if (narrow || wide) {
      std::vector<float> blob;
      std::vector<int64_t> soff(R.n_cells);
      std::vector<int32_t> kq(R.n_cells);
      for (int c = 0; c < R.n_cells; ++c) {
        const int K = R.cell_K[c], m = R.cell_m[c], Kq = (K + 3) / 4 * 4;
        kq[c] = Kq;
        soff[c] = (int64_t)blob.size();
        const double *src = coef.data() + cell_coef[c];
        for (int q = 0; q < 2 * m - 1; ++q)
          for (int jj = 0; jj < K; ++jj) {
            const int j = (s.factor_last && q == m - 1) ? K - 1 - jj : jj;
            for (int r = 0; r < K; ++r) blob.push_back((float)src[(size_t)q * K * K + (size_t)j * K + r]);
            for (int r = K; r < Kq; ++r) blob.push_back(0.f);
          }
      }
      upload(s.d.sc_coef, blob);
      upload(s.d.sc_off, soff);
      upload(s.d.sc_Kq, kq);
      s.sca.coef = s.d.sc_coef.as<float>();
      s.sca.coef_off = s.d.sc_off.as<int64_t>();
      s.sca.Kq = s.d.sc_Kq.as<int32_t>();
      if (narrow) {
        s.stream_smem = need;
        s.stream_blob = true;
        s.stream_ok = true;
      } else {
        s.wide_smem = wneed;
        s.wide_smem8 = wide_smem_bytes(s.max_m, s.max_K, s.factor_last, 8);
        s.wide_blob = true;
        s.wide_ok = true;
      }
    }
  }
  if (!s.tc) upload(s.d.tc_err, std::vector<int>(1, 0));   // error word of the bounded waits
  s.sca.err = s.d.tc_err.as<int>();
  s.twa.err = s.d.tc_err.as<int>();
  upload(s.d.bar, std::vector<unsigned>(2, 0u));
  std::vector<double> minv(R.fmass_off[R.n_faces]);
  for (int f = 0; f < R.n_faces; ++f) {
    auto inv = inverse(R.face_mass.data() + R.fmass_off[f], R.face_M[f]);
    std::copy(inv.begin(), inv.end(), minv.begin() + R.fmass_off[f]);
  }
  // sources grouped per face
  std::vector<int32_t> fsrc_ptr(R.n_faces + 1, 0), fsrc_index;
  std::vector<int64_t> fsrc_val;
  std::vector<int64_t> src_off(R.src_face.size() + 1, 0);
  for (size_t e = 0; e < R.src_face.size(); ++e) src_off[e + 1] = src_off[e] + R.face_M[R.src_face[e]];
  for (int f = 0; f < R.n_faces; ++f) {
    for (size_t e = 0; e < R.src_face.size(); ++e)
      if (R.src_face[e] == f) {
        fsrc_index.push_back(R.src_index[e]);
        fsrc_val.push_back(src_off[e]);
      }
    fsrc_ptr[f + 1] = (int32_t)fsrc_index.size();
  }
  // receivers grouped per receiver
  std::vector<int32_t> rcv_ptr(R.n_rcv + 1, 0), rcv_face;
  std::vector<int64_t> rcv_off, rv_off(R.rcv_face.size() + 1, 0);
  for (size_t e = 0; e < R.rcv_face.size(); ++e) rv_off[e + 1] = rv_off[e] + R.face_M[R.rcv_face[e]];
  for (int r = 0; r < R.n_rcv; ++r) {
    for (size_t e = 0; e < R.rcv_face.size(); ++e)
      if (R.rcv_index[e] == r) {
        rcv_face.push_back(R.rcv_face[e]);
        rcv_off.push_back(rv_off[e]);
      }
    rcv_ptr[r + 1] = (int32_t)rcv_face.size();
  }
  // receivers on hidden layers (lifted nodes inside cells), grouped per receiver
  std::vector<int32_t> rh_ptr(R.n_rcv + 1, 0), rh_cnt;
  std::vector<int64_t> rh_row0, rh_off;
  std::vector<double> rh_val;
  for (int r = 0; r < R.n_rcv; ++r) {
    int64_t o = 0;
    for (size_t e = 0; e < R.rcv_h_index.size(); ++e) {
      const int c = R.rcv_h_cell[e], K = R.cell_K[c];
      if (R.rcv_h_index[e] == r) {
        rh_row0.push_back(cell_state[c] + (int64_t)(R.rcv_h_layer[e] - 2) * K);
        rh_cnt.push_back(K);
        rh_off.push_back((int64_t)rh_val.size());
        rh_val.insert(rh_val.end(), R.rcv_h_vals.begin() + o, R.rcv_h_vals.begin() + o + K);
      }
      o += K;
    }
    rh_ptr[r + 1] = (int32_t)rh_row0.size();
  }
  s.n_rh = (int)rh_row0.size();
  // corner groups
  std::vector<int32_t> fm_ptr(R.n_faces + 1, 0), fm_member, mem_group, mem_face, grp_ptr, cfaces;
  std::vector<int64_t> mem_row, fm_roff;
  std::vector<int4> fm_info;
  std::vector<double> fm_rows;
  if (s.corners) {
    const int G = (int)R.cg_ptr.size() - 1;
    grp_ptr = R.cg_ptr;
    mem_face = R.cg_face;
    int64_t o = 0;
    for (size_t l = 0; l < R.cg_face.size(); ++l) {
      mem_row.push_back(o);
      o += R.face_M[R.cg_face[l]];
    }
    mem_group.assign(R.cg_face.size(), 0);
    for (int g = 0; g < G; ++g)
      for (int l = R.cg_ptr[g]; l < R.cg_ptr[g + 1]; ++l) mem_group[l] = g;
    std::vector<std::vector<int32_t>> per(R.n_faces);
    for (size_t l = 0; l < R.cg_face.size(); ++l) per[R.cg_face[l]].push_back((int32_t)l);
    for (int f = 0; f < R.n_faces; ++f) {
      fm_member.insert(fm_member.end(), per[f].begin(), per[f].end());
      fm_ptr[f + 1] = (int32_t)fm_member.size();
      s.max_nm = std::max<int>(s.max_nm, (int)per[f].size());
      if (!per[f].empty()) cfaces.push_back(f);
    }
    fm_roff.assign(R.n_faces + 1, 0);
    for (int f = 0; f < R.n_faces; ++f) {
      for (int32_t l : per[f]) {
        const double *row = R.cg_rows.data() + mem_row[l];
        fm_rows.insert(fm_rows.end(), row, row + R.face_M[f]);
        const int g = mem_group[l];
        fm_info.push_back(make_int4(l, R.cg_ptr[g], R.cg_ptr[g + 1], 0));
      }
      fm_roff[f + 1] = (int64_t)fm_rows.size();
    }
  }
  s.n_cfaces = (int)cfaces.size();
  s.corner_smem = std::max<size_t>(16, (size_t)s.max_nm * (s.ST + s.max_M) * es);
  s.dev_smem = dev_smem;
  s.st_max = s.ST;
  apply_tile(s, s.ST);
  SimDev &d = s.d;
  upload(d.cell_K, R.cell_K);
  upload(d.cell_m, R.cell_m);
  upload(d.cell_coef, cell_coef);
  upload(d.cell_ghat, cell_ghat);
  upload(d.cell_state, cell_state);
  upload(d.cell_row, cell_row);
  upload(d.row_face_row, row_face_row);
  upload(d.row_side, row_side);
  upload(d.face_M, R.face_M);
  upload(d.face_two, face_two);
  upload(d.face_row, face_row);
  upload(d.face_minv, face_minv);
  upload(d.fsrc_ptr, fsrc_ptr);
  upload(d.fsrc_index, fsrc_index);
  upload(d.fsrc_val, fsrc_val);
  upload(d.rcv_ptr, rcv_ptr);
  upload(d.rcv_face, rcv_face);
  upload(d.rcv_off, rcv_off);
  upload(d.rh_ptr, rh_ptr);
  upload(d.rh_cnt, rh_cnt);
  upload(d.rh_row0, rh_row0);
  upload(d.rh_off, rh_off);
  upload(d.fm_ptr, fm_ptr);
  upload(d.fm_member, fm_member);
  upload(d.mem_group, mem_group);
  upload(d.mem_face, mem_face);
  upload(d.grp_ptr, grp_ptr);
  upload(d.mem_row, mem_row);
  upload(d.fm_roff, fm_roff);
  upload(d.fm_info, fm_info);
  upload(d.cfaces, cfaces);
  auto up = [&](DevMem &m, const std::vector<double> &v) {
    if (prec == MSS_FP64) upload_as<double>(m, v);
    else upload_as<float>(m, v);
  };
  up(d.coef, (s.tc || s.tw) ? std::vector<double>() : coef);
  up(d.minv, minv);
  up(d.src_val, R.src_vals);
  up(d.rcv_val, R.rcv_vals);
  up(d.rh_val, rh_val);
  up(d.cg_rows, s.corners ? R.cg_rows : std::vector<double>());
  up(d.cg_w, s.corners ? R.cg_weight : std::vector<double>());
  up(d.fm_rows, fm_rows);
  for (int l = 0; l < 2; ++l) {
    d.fstate[l].alloc((size_t)s.face_rows * S * es);
    d.cstate[l].alloc((size_t)std::max<int64_t>(1, s.cell_rows) * S * es);
  }
  d.flux.alloc((size_t)s.face_rows * 2 * S * es);
  d.uhat.alloc(s.corners ? R.cg_face.size() * (size_t)S * es : 16);
  MSS_CUDA(cudaMemset(d.flux.p, 0, d.flux.bytes));
  int64_t bytes = 0;
  for (DevMem *m : {&d.cell_K, &d.cell_m, &d.cell_coef, &d.cell_ghat, &d.cell_state, &d.cell_row, &d.row_face_row,
                    &d.row_side, &d.face_M, &d.face_two, &d.face_row, &d.face_minv, &d.fsrc_ptr, &d.fsrc_index,
                    &d.fsrc_val, &d.rcv_ptr, &d.rcv_face, &d.rcv_off, &d.fm_ptr, &d.fm_member, &d.mem_group,
                    &d.mem_face, &d.grp_ptr, &d.mem_row, &d.coef, &d.minv, &d.src_val, &d.rcv_val, &d.cg_rows,
                    &d.cg_w, &d.fm_rows, &d.fm_roff, &d.fm_info, &d.fstate[0], &d.fstate[1], &d.cstate[0], &d.cstate[1], &d.flux, &d.uhat, &d.cfaces})
    bytes += (int64_t)m->bytes;
  s.dev_bytes = bytes;
}

static void sim_reset(mss_sim &s, cudaStream_t st) {
  for (int l = 0; l < 2; ++l) {
    MSS_CUDA(cudaMemsetAsync(s.d.fstate[l].p, 0, s.d.fstate[l].bytes, st));
    MSS_CUDA(cudaMemsetAsync(s.d.cstate[l].p, 0, s.d.cstate[l].bytes, st));
  }
  s.cur = 0;
  s.steps = 0;
}

// Host FP64 <-> device state of precision T.
static void state_io(mss_sim &s, double *now, double *old, const double *inow, const double *iold) {
  const size_t es = s.prec == MSS_FP64 ? 8 : 4;
  const int64_t nf = s.face_rows * s.n_src, nc = s.cell_rows * s.n_src;
  std::vector<unsigned char> buf((size_t)(nf + nc) * es);
  for (int lv = 0; lv < 2; ++lv) {
    const int slot = lv == 0 ? s.cur : (s.cur ^ 1);
    if (now || old) {
      double *dst = lv == 0 ? now : old;
      MSS_CUDA(cudaMemcpy(buf.data(), s.d.fstate[slot].p, nf * es, cudaMemcpyDeviceToHost));
      if (nc) MSS_CUDA(cudaMemcpy(buf.data() + nf * es, s.d.cstate[slot].p, nc * es, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < nf + nc; ++i)
        dst[i] = es == 8 ? reinterpret_cast<double *>(buf.data())[i] : reinterpret_cast<float *>(buf.data())[i];
    } else {
      const double *src = lv == 0 ? inow : iold;
      for (int64_t i = 0; i < nf + nc; ++i) {
        if (es == 8) reinterpret_cast<double *>(buf.data())[i] = src[i];
        else reinterpret_cast<float *>(buf.data())[i] = (float)src[i];
      }
      MSS_CUDA(cudaMemcpy(s.d.fstate[slot].p, buf.data(), nf * es, cudaMemcpyHostToDevice));
      if (nc) MSS_CUDA(cudaMemcpy(s.d.cstate[slot].p, buf.data() + nf * es, nc * es, cudaMemcpyHostToDevice));
    }
  }
}

}  // namespace mss

// ------------------------------------------------------------------ stepping without allocation
// The flux exchange of the allocation-free step lives in this fixed file-scope array; host code
// must not pass the symbol itself to a kernel (in host code it names a host-side stand-in), so
// its device address is looked up once per device and cached.  The cache is not invalidated:
// after cudaDeviceReset on a device the cached address is stale, so a process that resets a
// device must not call the allocation-free step on it again.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MSS_NOALLOC_SCRATCH_BYTES];

namespace mss {

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];

static void *noalloc_scratch() {
  int dev = 0;
  MSS_CUDA(cudaGetDevice(&dev));
  MSS_REQUIRE(dev >= 0 && dev < 256, MSS_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    MSS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

template <typename T, int ST>
static void noalloc_impl(mss_step_buffers &b, int64_t n, const double *w, T *traces, cudaStream_t st, void *scratch) {
  StepArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.cell_K = b.cell_K;
  a.cell_m = b.cell_m;
  a.cell_coef = b.cell_coef;
  a.cell_ghat = b.cell_ghat;
  a.cell_state = b.cell_state;
  a.cell_row = b.cell_row;
  a.row_face_row = b.row_face_row;
  a.row_side = b.row_side;
  a.face_M = b.face_M;
  a.face_two = b.face_two;
  a.face_row = b.face_row;
  a.face_minv = b.face_minv;
  a.fsrc_ptr = b.fsrc_ptr;
  a.fsrc_index = b.fsrc_index;
  a.fsrc_val = b.fsrc_val;
  a.rcv_ptr = b.rcv_ptr;
  a.rcv_face = b.rcv_face;
  a.rcv_off = b.rcv_off;
  a.coef = (const T *)b.coef;
  a.minv = (const T *)b.minv;
  a.src_val = (const T *)b.src_val;
  a.rcv_val = (const T *)b.rcv_val;
  a.fstate0 = (T *)b.face_state[0];
  a.fstate1 = (T *)b.face_state[1];
  a.cstate0 = (T *)b.cell_state_buf[0];
  a.cstate1 = (T *)b.cell_state_buf[1];
  a.flux = (T *)scratch;
  a.uhat = nullptr;
  a.cfaces = nullptr;
  a.S = b.n_src;
  a.n_cells = b.n_cells;
  a.n_faces = b.n_faces;
  a.n_rcv = b.n_rcv;
  a.corners = 0;
  a.tau2 = (T)(b.tau * b.tau);
  const size_t es = sizeof(T);
  const int tiles = (b.n_src + ST - 1) / ST;
  const size_t cell_smem = 2 * (size_t)b.max_m * b.max_K * ST * es + 8 * (size_t)b.max_K;
  const size_t face_smem = std::max<size_t>(16, (2 * (size_t)b.max_M * ST + (size_t)b.max_M * b.max_M) * es);
  int dev = 0, dev_smem = 0;
  MSS_CUDA(cudaGetDevice(&dev));
  MSS_CUDA(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  MSS_REQUIRE(cell_smem <= (size_t)dev_smem, MSS_ERR_INVALID_ARG, "cell too large for shared memory");
  MSS_CUDA(cudaFuncSetAttribute(k_cell<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem));
  MSS_CUDA(cudaFuncSetAttribute(k_face<T, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)face_smem));
  const int per = kFaceThreads / ST;
  const int rcv_blocks = (b.n_rcv + per - 1) / per;
  const dim3 gc(b.n_cells * tiles), gf(b.n_faces + rcv_blocks, tiles);
  int cur = b.cur & 1;
  for (int64_t j = 0; j < n; ++j) {
    k_cell<T, ST><<<gc, kCellThreads, cell_smem, st>>>(a, cur);
    k_face<T, ST><<<gf, kFaceThreads, face_smem, st>>>(a, cur, w + j, traces + j * (int64_t)b.n_rcv * b.n_src);
    cur ^= 1;
  }
  MSS_CUDA(cudaGetLastError());
  b.cur = cur;
}

template <typename T>
static void noalloc_dispatch(mss_step_buffers &b, int64_t n, const double *w, void *traces, cudaStream_t st,
                             void *scratch) {
  const int S = b.n_src;
  const size_t es = sizeof(T);
  int ST = S <= 1 ? 1 : S <= 2 ? 2 : S <= 4 ? 4 : S <= 8 ? 8 : 16;
  int dev = 0, dev_smem = 0;
  MSS_CUDA(cudaGetDevice(&dev));
  MSS_CUDA(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  while (ST > 1 && 2 * (size_t)b.max_m * b.max_K * ST * es + 8 * (size_t)b.max_K > (size_t)dev_smem) ST /= 2;
  switch (ST) {
    case 1: noalloc_impl<T, 1>(b, n, w, (T *)traces, st, scratch); break;
    case 2: noalloc_impl<T, 2>(b, n, w, (T *)traces, st, scratch); break;
    case 4: noalloc_impl<T, 4>(b, n, w, (T *)traces, st, scratch); break;
    case 8: noalloc_impl<T, 8>(b, n, w, (T *)traces, st, scratch); break;
    default: noalloc_impl<T, 16>(b, n, w, (T *)traces, st, scratch); break;
  }
}

}  // namespace mss

using namespace mss;

extern "C" {

mss_status mss_step_noalloc(mss_step_buffers *b, int64_t n_steps, const double *waveform, void *traces,
                            void *stream) {
  return guard([&] {
    MSS_REQUIRE(b && waveform && traces && n_steps >= 0, MSS_ERR_INVALID_ARG, "bad argument");
    MSS_REQUIRE(b->precision == MSS_FP64 || b->precision == MSS_FP32, MSS_ERR_INVALID_ARG,
                "precision must be FP64 or FP32");
    MSS_REQUIRE(b->n_cells >= 1 && b->n_faces >= 1 && b->n_src >= 1 && b->n_rcv >= 0 && b->max_K >= 1 &&
                    b->max_m >= 1 && b->max_M >= 1 && b->face_rows >= 1 && b->tau > 0,
                MSS_ERR_INVALID_ARG, "bad sizes in mss_step_buffers");
    MSS_REQUIRE(b->cell_K && b->cell_m && b->cell_coef && b->cell_ghat && b->cell_state && b->cell_row &&
                    b->row_face_row && b->row_side && b->face_M && b->face_two && b->face_row && b->face_minv &&
                    b->fsrc_ptr && b->fsrc_index && b->fsrc_val && b->rcv_ptr && b->rcv_face && b->rcv_off &&
                    b->coef && b->minv && b->src_val && b->rcv_val && b->face_state[0] && b->face_state[1] &&
                    b->cell_state_buf[0] && b->cell_state_buf[1],
                MSS_ERR_INVALID_ARG, "null pointer in mss_step_buffers");
    for (const void *q : {b->face_state[0], b->face_state[1], b->cell_state_buf[0], b->cell_state_buf[1]})
      MSS_REQUIRE(((uintptr_t)q & 15) == 0, MSS_ERR_INVALID_ARG, "state buffers must be 16-byte aligned");
    const size_t es = b->precision == MSS_FP64 ? 8 : 4;
    // rows the fixed scratch can hold for this source count; compared without forming the
    // product face_rows * 2 * n_src * es, which could wrap around for a huge face_rows
    const size_t row_bytes = 2 * (size_t)b->n_src * es;
    const size_t max_rows = (size_t)MSS_NOALLOC_SCRATCH_BYTES / row_bytes;
    MSS_REQUIRE((uint64_t)b->face_rows <= (uint64_t)max_rows, MSS_ERR_INVALID_ARG,
                "flux exchange of " + std::to_string(b->face_rows) + " face rows x " + std::to_string(b->n_src) +
                    " sources needs more than the fixed scratch of " +
                    std::to_string((size_t)MSS_NOALLOC_SCRATCH_BYTES) + " bytes (at most " +
                    std::to_string(max_rows) + " face rows)");
    if (n_steps == 0) return;
    void *scratch = noalloc_scratch();
    cudaStream_t st = (cudaStream_t)stream;
    if (b->precision == MSS_FP64) noalloc_dispatch<double>(*b, n_steps, waveform, traces, st, scratch);
    else noalloc_dispatch<float>(*b, n_steps, waveform, traces, st, scratch);
  });
}

mss_status mss_sim_create(const mss_rom *r, int32_t precision, double tau, int32_t flags, mss_sim **out) {
  return guard([&] {
    const Range nvtx_range("mss_sim_create");
    MSS_REQUIRE(r && out, MSS_ERR_INVALID_ARG, "null argument");
    auto s = std::make_unique<mss_sim>();
    sim_create(*s, r->r, precision, tau, flags);
    sim_reset(*s, 0);
    MSS_CUDA(cudaStreamSynchronize(0));
    *out = s.release();
  });
}

mss_status mss_sim_info(const mss_sim *s, int64_t info[8]) {
  return guard([&] {
    MSS_REQUIRE(s && info, MSS_ERR_INVALID_ARG, "null argument");
    {
      int e = 0;
      MSS_CUDA(cudaMemcpy(&e, s->d.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
      MSS_REQUIRE(e == 0, MSS_ERR_TIMEOUT, "a bounded wait in a cell kernel or grid barrier gave up");
    }
    info[0] = s->n_src;
    info[1] = s->n_rcv;
    info[2] = s->prec;
    info[3] = s->steps;
    info[4] = (s->face_rows + s->cell_rows) * s->n_src;
    info[5] = s->dev_bytes;
    info[6] = s->corners ? 3 : 2;
    info[7] = s->ST;
  });
}

mss_status mss_sim_reset(mss_sim *s, void *stream) {
  return guard([&] {
    MSS_REQUIRE(s, MSS_ERR_INVALID_ARG, "null sim");
    sim_reset(*s, (cudaStream_t)stream);
  });
}

mss_status mss_step(mss_sim *s, int64_t n_steps, const double *waveform, void *traces, int32_t use_graph,
                    void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_step");
    MSS_REQUIRE(s && waveform && traces && n_steps >= 0, MSS_ERR_INVALID_ARG, "bad argument");
    if (n_steps == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->prec == MSS_FP64) step_dispatch<double>(*s, n_steps, waveform, traces, use_graph, st);
    else step_dispatch<float>(*s, n_steps, waveform, traces, use_graph, st);
  });
}

mss_status mss_step_profile(mss_sim *s, int64_t n_steps, const double *waveform, void *traces, double ms[3],
                            void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_step_profile");
    MSS_REQUIRE(s && waveform && traces && ms && n_steps > 0, MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (s->prec == MSS_FP64) profile_dispatch<double>(*s, n_steps, waveform, traces, ms, st);
    else profile_dispatch<float>(*s, n_steps, waveform, traces, ms, st);
  });
}

static bool sched_allowed(const mss_sim &s, int sched) {
  if (s.tw) return sched == MSS_SCHED_GRAPH;
  if (s.factor_last)
    return sched == MSS_SCHED_GRAPH || sched == MSS_SCHED_PERSIST || (sched == MSS_SCHED_GRAPH_STREAM && s.wide_ok);
  switch (sched) {
    case MSS_SCHED_GRAPH: return true;
    case MSS_SCHED_GRAPH_STREAM: return s.stream_ok || s.wide_ok;
    case MSS_SCHED_PERSIST: return true;   // tensor-core precisions: pipelined split kernels
    case MSS_SCHED_PERSIST_STREAM: return s.tc ? s.tcq_nt > 0 : s.stream_ok;
    case MSS_SCHED_GRAPH_SPLIT: return s.tc ? true : s.split_smem <= 48 * 1024;
    default: return false;
  }
}

mss_status mss_sim_set_schedule(mss_sim *s, int32_t sched) {
  return guard([&] {
    MSS_REQUIRE(s, MSS_ERR_INVALID_ARG, "null argument");
    MSS_REQUIRE(sched_allowed(*s, sched), MSS_ERR_INVALID_ARG, "schedule not available for this sim");
    s->sched = sched;
  });
}

mss_status mss_sim_debug(mss_sim *s, int32_t knob, int32_t value) {
  return guard([&] {
    MSS_REQUIRE(s && value >= 0, MSS_ERR_INVALID_ARG, "bad argument");
    switch (knob) {
      case MSS_DEBUG_GRID_EXTRA_ARRIVALS: s->sca.extra_arrivals = value; break;
      case MSS_DEBUG_TC_EXTRA_TX:
        s->tca.extra_tx = (unsigned)value;
        s->sca.extra_tx = (unsigned)value;
        s->twa.extra_tx = (unsigned)value;
        break;
      default: MSS_REQUIRE(false, MSS_ERR_INVALID_ARG, "unknown debug knob");
    }
  });
}

mss_status mss_sim_clear_error(mss_sim *s, void *stream) {
  return guard([&] {
    MSS_REQUIRE(s, MSS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    MSS_CUDA(cudaMemsetAsync(s->d.tc_err.p, 0, sizeof(int), st));
    MSS_CUDA(cudaMemsetAsync(s->d.bar.p, 0, 2 * sizeof(unsigned), st));
    MSS_CUDA(cudaStreamSynchronize(st));
  });
}

mss_status mss_sim_set_tile(mss_sim *s, int32_t source_tile, int32_t tc_sources, int32_t groups) {
  return guard([&] {
    MSS_REQUIRE(s, MSS_ERR_INVALID_ARG, "null argument");
    if (source_tile > 0) {
      MSS_REQUIRE(source_tile <= s->st_max && (source_tile & (source_tile - 1)) == 0, MSS_ERR_INVALID_ARG,
                  "source tile must be a power of two up to the sim's largest");
      apply_tile(*s, source_tile);
      if (!sched_allowed(*s, s->sched)) s->sched = MSS_SCHED_GRAPH;
    }
    if (tc_sources > 0) {
      MSS_REQUIRE(s->tc, MSS_ERR_INVALID_ARG, "tensor-core tile on a CUDA-core sim");
      MSS_REQUIRE(tc_sources == 16 || tc_sources == 32 || tc_sources == 64 || tc_sources == 128, MSS_ERR_INVALID_ARG,
                  "tensor-core tile must be 16, 32, 64 or 128 sources");
      MSS_REQUIRE(tcs_smem_bytes(tc_sources, s->tc_kpmax) <= (size_t)s->dev_smem, MSS_ERR_INVALID_ARG,
                  "tensor-core tile too large for shared memory");
      apply_tcs_nt(*s, tc_sources);
    }
    if (groups > 0) {
      if (s->tw) {
        MSS_REQUIRE(groups >= 2 && groups <= s->tw_ring_max, MSS_ERR_INVALID_ARG,
                    "copy-ring slots of the wide tensor-core kernel must be 2 .. the most that fit");
        s->twa.ring = groups;
      } else if (s->wide_ok && !s->stream_ok) {
        MSS_REQUIRE(groups <= 8, MSS_ERR_INVALID_ARG, "wide streamed kernel variant must be 1..8");
        s->wide_var = groups - 1;
      } else {
        MSS_REQUIRE(groups == 2 || groups == 4, MSS_ERR_INVALID_ARG, "thread groups must be 2 or 4");
        s->stream_groups = groups;
      }
    }
  });
}

mss_status mss_sim_get_schedule(const mss_sim *s, int32_t *sched, int32_t *available, int32_t *tile) {
  return guard([&] {
    MSS_REQUIRE(s && sched, MSS_ERR_INVALID_ARG, "null argument");
    *sched = s->sched;
    if (available)
      for (int k = 0; k < MSS_SCHED_COUNT; ++k) available[k] = sched_allowed(*s, k) ? 1 : 0;
    if (tile) {
      tile[0] = s->ST;
      tile[1] = s->tc ? s->tcs_nt : 0;
      tile[2] = s->tw ? s->twa.ring : s->wide_ok && !s->stream_ok ? s->wide_var + 1 : s->stream_groups;
    }
  });
}

mss_status mss_sim_autotune(mss_sim *s, int32_t n_steps, void *stream, double *ms, int32_t *chosen) {
  return guard([&] {
    const Range nvtx_range("mss_sim_autotune");
    MSS_REQUIRE(s && n_steps >= 2, MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = n_steps + (n_steps & 1);   // even: the time-level parity returns, graphs are reused
    const size_t es = s->prec == MSS_FP64 ? 8 : 4;
    const int64_t nf = s->face_rows * s->n_src, nc = std::max<int64_t>(1, s->cell_rows) * s->n_src;
    DevMem keep[4], w, tr;
    DevMem *lv[4] = {&s->d.fstate[0], &s->d.fstate[1], &s->d.cstate[0], &s->d.cstate[1]};
    const int64_t cnt[4] = {nf, nf, nc, nc};
    MSS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < 4; ++i) {
      keep[i].alloc(cnt[i] * es);
      MSS_CUDA(cudaMemcpy(keep[i].p, lv[i]->p, cnt[i] * es, cudaMemcpyDeviceToDevice));
    }
    w.alloc((size_t)n * 8);
    MSS_CUDA(cudaMemset(w.p, 0, (size_t)n * 8));
    tr.alloc((size_t)n * std::max(1, s->n_rcv) * s->n_src * es);
    const int cur0 = s->cur, sched0 = s->sched;
    const int st_keep = s->ST, nt_keep = s->tcs_nt, g_keep = s->stream_groups, wv_keep = s->wide_var;
    const int ring_keep = s->twa.ring;
    const int64_t steps0 = s->steps;
    cudaEvent_t e0, e1;
    MSS_CUDA(cudaEventCreate(&e0));
    MSS_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int best_k = sched0;
    auto restore = [&]() {
      for (int i = 0; i < 4; ++i)
        MSS_CUDA(cudaMemcpyAsync(lv[i]->p, keep[i].p, cnt[i] * es, cudaMemcpyDeviceToDevice, st));
      s->cur = cur0;
      s->steps = steps0;
    };
    try {
      // candidates: every available schedule x its tile variants (CUDA-core source tile ST,
      // tensor-core split N, streamed-kernel thread groups); every variant computes each source's
      // columns with the same operations, so the choice does not change the arithmetic
      struct Cand { int sched, st, nt, groups, wv; };
      std::vector<Cand> cands;
      const int st0 = s->ST, nt0 = s->tcs_nt, g0 = s->stream_groups;
      for (int k = 0; k < MSS_SCHED_COUNT; ++k) {
        if (ms) ms[k] = -1.0;
        if (!sched_allowed(*s, k)) continue;
        if (s->tw) {
          // the wide tensor-core kernel: its copy-ring depth (groups field)
          for (int ring = 2; ring <= s->tw_ring_max; ++ring) cands.push_back({k, st0, nt0, ring, s->wide_var});
        } else if (!s->tc) {
          const bool streamed = k == MSS_SCHED_GRAPH_STREAM || k == MSS_SCHED_PERSIST_STREAM;
          for (int st : {s->st_max, s->st_max / 2}) {
            if (st < 8 && st != s->st_max) continue;
            if (streamed && st != kStreamST) continue;
            if (k == MSS_SCHED_GRAPH_STREAM && !s->stream_ok) {
              for (int wv = 0; wv < 8; ++wv) cands.push_back({k, st, nt0, g0, wv});
            } else if (k == MSS_SCHED_GRAPH_STREAM) {
              for (int gv : {4, 2}) cands.push_back({k, st, nt0, gv, s->wide_var});
            } else {
              cands.push_back({k, st, nt0, g0, s->wide_var});
            }
          }
        } else if (k == MSS_SCHED_GRAPH_SPLIT || k == MSS_SCHED_PERSIST) {
          for (int nt : {16, 32, 64, 128}) {
            if (nt > 16 && nt / 2 >= s->n_src) continue;
            if (tcs_smem_bytes(nt, s->tc_kpmax) > (size_t)s->dev_smem) continue;
            cands.push_back({k, st0, nt, g0, s->wide_var});
          }
        } else {
          cands.push_back({k, st0, nt0, g0, s->wide_var});
        }
      }
      const int wv0 = s->wide_var;
      Cand best_c{sched0, st0, nt0, g0, wv0};
      for (const Cand &c : cands) {
        s->sched = c.sched;
        if (c.st != s->ST) apply_tile(*s, c.st);
        if (s->tc && c.nt != s->tcs_nt) apply_tcs_nt(*s, c.nt);
        if (s->tw) s->twa.ring = c.groups;
        else s->stream_groups = c.groups;
        s->wide_var = c.wv;
        auto run = [&]() {
          if (s->prec == MSS_FP64) step_dispatch<double>(*s, n, w.as<double>(), tr.p, 1, st);
          else step_dispatch<float>(*s, n, w.as<double>(), tr.p, 1, st);
        };
        run();   // warm-up (and graph capture)
        MSS_CUDA(cudaEventRecord(e0, st));
        run();
        MSS_CUDA(cudaEventRecord(e1, st));
        MSS_CUDA(cudaEventSynchronize(e1));
        float t = 0;
        MSS_CUDA(cudaEventElapsedTime(&t, e0, e1));
        int err = 0;
        MSS_CUDA(cudaMemcpy(&err, s->d.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        MSS_REQUIRE(err == 0, MSS_ERR_TIMEOUT, "a bounded wait gave up during autotuning");
        const double per = t / (double)n;
        if (ms && (ms[c.sched] < 0 || per < ms[c.sched])) ms[c.sched] = per;
        if (per < best) {
          best = per;
          best_k = c.sched;
          best_c = c;
        }
        restore();
      }
      if (best_c.st != s->ST) apply_tile(*s, best_c.st);
      if (s->tc && best_c.nt != s->tcs_nt) apply_tcs_nt(*s, best_c.nt);
      const int best_groups = best_c.groups;
      if (s->tw) s->twa.ring = best_groups;
      else s->stream_groups = best_groups;
      s->wide_var = best_c.wv;
    } catch (...) {
      restore();
      s->sched = sched0;
      if (s->ST != st_keep) apply_tile(*s, st_keep);
      if (s->tc && s->tcs_nt != nt_keep) apply_tcs_nt(*s, nt_keep);
      s->stream_groups = g_keep;
      s->wide_var = wv_keep;
      s->twa.ring = ring_keep;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MSS_CUDA(cudaStreamSynchronize(st));
    // graphs recorded on the scratch buffers are dropped with them
    for (auto it = s->graphs.begin(); it != s->graphs.end();) {
      if (it->first.w == w.p) {
        cudaGraphExecDestroy(it->second);
        it = s->graphs.erase(it);
      } else {
        ++it;
      }
    }
    s->sched = best_k;
    if (chosen) *chosen = best_k;
  });
}

mss_status mss_run_host(mss_sim *s, int64_t n_steps, const double *waveform_host, void *traces_host, void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_run_host");
    MSS_REQUIRE(s && waveform_host && traces_host && n_steps > 0, MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = s->prec == MSS_FP64 ? 8 : 4;
    const size_t tb = (size_t)n_steps * s->n_rcv * s->n_src * es;
    if (s->d.wbuf.bytes < (size_t)n_steps * 8) s->d.wbuf.alloc((size_t)n_steps * 8);
    if (s->d.tbuf.bytes < tb) s->d.tbuf.alloc(tb);
    MSS_CUDA(cudaMemcpyAsync(s->d.wbuf.p, waveform_host, (size_t)n_steps * 8, cudaMemcpyHostToDevice, st));
    sim_reset(*s, st);
    if (s->prec == MSS_FP64) step_dispatch<double>(*s, n_steps, s->d.wbuf.as<double>(), s->d.tbuf.p, 1, st);
    else step_dispatch<float>(*s, n_steps, s->d.wbuf.as<double>(), s->d.tbuf.p, 1, st);
    MSS_CUDA(cudaMemcpyAsync(traces_host, s->d.tbuf.p, tb, cudaMemcpyDeviceToHost, st));
    MSS_CUDA(cudaStreamSynchronize(st));
    if (s->tc || s->tw) {
      int e = 0;
      MSS_CUDA(cudaMemcpy(&e, s->d.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
      MSS_REQUIRE(e == 0, MSS_ERR_TIMEOUT, "a tensor-core cell kernel's bounded wait gave up");
    }
  });
}

mss_status mss_sim_save_state(const mss_sim *s, double *now, double *old, int64_t *steps_taken) {
  return guard([&] {
    MSS_REQUIRE(s && now && old, MSS_ERR_INVALID_ARG, "null argument");
    MSS_CUDA(cudaDeviceSynchronize());
    state_io(const_cast<mss_sim &>(*s), now, old, nullptr, nullptr);
    if (steps_taken) *steps_taken = s->steps;
  });
}

mss_status mss_sim_load_state(mss_sim *s, const double *now, const double *old, int64_t steps_taken) {
  return guard([&] {
    MSS_REQUIRE(s && now && old && steps_taken >= 0, MSS_ERR_INVALID_ARG, "bad argument");
    MSS_CUDA(cudaDeviceSynchronize());
    state_io(*s, nullptr, nullptr, now, old);
    s->steps = steps_taken;
  });
}

void mss_sim_destroy(mss_sim *s) { delete s; }

}  // extern "C"
