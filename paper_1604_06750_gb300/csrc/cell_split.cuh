// Cell phase split into one small CTA per (cell, matrix): the flux kernel computes
//   F^k = Gamma^k (U^{k+1} - U^k)           for every (cell, k), k = 1..m    (Eq. GammaUremi)
// into a per-cell scratch block (F^1 also into the face flux buffer), and the acceleration kernel
//   U^k <- 2U^k - U^k_old + tau^2 Gamma-hat^k (F^k - F^{k-1})   for every (cell, k), k = 2..m.
// Each CTA stages its K x ST operand block in shared memory (a few KB) and its 128 threads stream
// the matrix rows straight from HBM (thread r reads G[j][r] = G[r][j], coalesced across the warp,
// register-pipelined), so up to 8 CTAs share an SM and hide the load latency with occupancy
// instead of a staging ring.  Arithmetic order per row equals the fused cell kernel's.
#pragma once

namespace mss {

constexpr int kSplitThreads = 128;

template <typename T>
struct SplitArgs {
  const int2 *flux_items;    // (cell, k - 1), k = 1..m
  const int2 *accel_items;   // (cell, k - 1), k = 2..m
  const int64_t *f_off;      // per cell: first row of its F scratch block (m K rows of S values)
  T *F;
};

template <typename T, int ST>
__global__ void __launch_bounds__(kSplitThreads, 8) k_flux(const StepArgs<T> a, const SplitArgs<T> p, const int cur) {
  const int tiles = (a.S + ST - 1) / ST;          // 1-D grid, tiles of an item adjacent
  const int2 it = p.flux_items[blockIdx.x / tiles];
  const int cell = it.x, q = it.y;
  const int s0 = (blockIdx.x % tiles) * ST;
  const int K = a.cell_K[cell], m = a.cell_m[cell];
  const int ns = min(ST, a.S - s0);
  const int S = a.S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *D = reinterpret_cast<T *>(smem_raw);                               // K x ST
  int64_t *rows = reinterpret_cast<int64_t *>(D + (size_t)K * ST);      // q == 0 only
  const T *fs = cur ? a.fstate1 : a.fstate0;
  const T *cs = cur ? a.cstate1 : a.cstate0;
  const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
  const T *G = a.coef + a.cell_coef[cell] + (size_t)q * K * K;
  if (s0 == 0) prefetch_l2_range(G, sizeof(T) * (size_t)K * K);
  if (q == 0)
    for (int r = threadIdx.x; r < K; r += blockDim.x) rows[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
  __syncthreads();
  // D = U_{q+1} - U_q with U_0 the face values, U_l (l >= 1) hidden layer l, U_m = 0
  for (int i = threadIdx.x; i < K * ST; i += blockDim.x) {
    const int r = i / ST, s = i - r * ST;
    T v = T(0);
    if (s < ns) {
      const T up = q + 1 < m ? cs[(so + (int64_t)q * K + r) * S + s0 + s] : T(0);
      const T lo = q == 0 ? fs[(rows[r] >> 1) * S + s0 + s] : cs[(so + (int64_t)(q - 1) * K + r) * S + s0 + s];
      v = up - lo;
    }
    D[i] = v;
  }
  __syncthreads();
  T *Fo = p.F + (p.f_off[cell] + (int64_t)q * K) * S + s0;
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    T acc[ST];
    row_times_block<T, ST>(G + r, K, D, acc);
#pragma unroll
    for (int s = 0; s < ST; ++s)
      if (s < ns) Fo[(int64_t)r * S + s] = acc[s];
    if (q == 0) {
#pragma unroll
      for (int s = 0; s < ST; ++s)
        if (s < ns) a.flux[rows[r] * S + s0 + s] = acc[s];
    }
  }
}

template <typename T, int ST>
__global__ void __launch_bounds__(kSplitThreads, 8) k_accel(const StepArgs<T> a, const SplitArgs<T> p, const int cur) {
  const int tiles = (a.S + ST - 1) / ST;
  const int2 it = p.accel_items[blockIdx.x / tiles];
  const int cell = it.x, k = it.y;   // hidden layer k (0-based), k >= 1
  const int s0 = (blockIdx.x % tiles) * ST;
  const int K = a.cell_K[cell];
  const int ns = min(ST, a.S - s0);
  const int S = a.S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *E = reinterpret_cast<T *>(smem_raw);                               // K x ST
  const T *cs = cur ? a.cstate1 : a.cstate0;
  T *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t so = a.cell_state[cell];
  const T *Fk = p.F + (p.f_off[cell] + (int64_t)k * K) * S + s0;
  const T *H = a.coef + a.cell_ghat[cell] + (size_t)(k - 1) * K * K;
  if (s0 == 0) prefetch_l2_range(H, sizeof(T) * (size_t)K * K);
  for (int i = threadIdx.x; i < K * ST; i += blockDim.x) {
    const int r = i / ST, s = i - r * ST;
    E[i] = s < ns ? Fk[(int64_t)r * S + s] - Fk[(int64_t)(r - K) * S + s] : T(0);
  }
  __syncthreads();
  const T tau2 = a.tau2;
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    T acc[ST];
    row_times_block<T, ST>(H + r, K, E, acc);
    const int64_t base = (so + (int64_t)(k - 1) * K + r) * S + s0;
#pragma unroll
    for (int s = 0; s < ST; ++s)
      if (s < ns) cso[base + s] = T(2) * cs[base + s] - cso[base + s] + tau2 * acc[s];
  }
}

}  // namespace mss
