// Cell phase with the coefficient stream staged by TMA, and the persistent time-block kernel.
//
// Streamed cell item (FP32, CUDA cores, 16-source tiles, K_i <= 128).  The coefficients a cell
// needs in one step -- Gamma^1..Gamma^m then Gamma-hat^2..Gamma-hat^m (Eq. intrtstep_td) -- are
// stored contiguously per cell, each matrix as K rows of Kq = K rounded up to 4 floats, so the
// whole per-cell stream is one 16-byte-aligned byte range.  One thread issues 1-D bulk copies
// (cp.async.bulk) of fixed-size chunks of whole rows into a ring of shared-memory slots, each
// guarded by an mbarrier with a transaction count; the 256 threads consume the chunks in order
// while the next ones are in flight.  Row j of a stored symmetric matrix is also its column j, so
// thread (g, r) -- r = tid % 128, g = tid / 128 -- accumulates
//   acc[e] += G[j][r] * D[j][8g + e],  e = 0..7,
// with G[j][r] read conflict-free from the slot and D[j][.] a broadcast read of the operand block.
// At the end of matrix q the thread holds row r of F^{q+1} (flux) or of Gamma-hat^k E^k (then
// it advances U^k by leapfrog).  Every wait is bounded (globaltimer); on timeout the CTA records
// an error, waits (bounded) for its own copies in flight and returns.
//
// Persistent kernel (cooperative launch, all CTAs resident): each CTA loops over T time steps
// and, per step, over the items of three phases -- cells, then faces and receivers, then the
// Appendix D corner correction -- separated by a grid barrier (count + generation word in
// global memory, thread 0 spins with a time limit and stops on the error flag).
#pragma once

namespace mss {

constexpr int kStreamSlots = 4;
constexpr int kStreamChunk = 16384;  // bytes per ring slot
constexpr int kStreamST = 16;
constexpr unsigned long long kGridWaitNs = 1000000000ull;   // 1 s per grid barrier

struct StreamArgs {
  const float *coef;        // per cell: 2m-1 matrices of K x Kq floats
  const int64_t *coef_off;  // per cell, floats
  const int32_t *Kq;
  int *err;                 // 1: an mbarrier wait timed out; 2: a grid barrier timed out
  int extra_arrivals;       // failure-path test hook: arrivals a grid barrier waits for beyond the grid
  unsigned extra_tx;        // failure-path test hook: bytes the wide kernel's chunk barriers wait for
                            // beyond their copies
};

// Wait for chunk c's slot; uniform over the CTA.  On failure the caller drains and returns.
__device__ __forceinline__ bool stream_wait(const uint64_t *full, unsigned gc, const int *err) {
  const unsigned slot = gc % kStreamSlots, par = (gc / kStreamSlots) & 1u;
  const bool ok = mbar_wait(smem_u32(full + slot), par, err);
  return __syncthreads_and(ok) != 0;
}

// Wait (bounded, ignoring the error flag) for every chunk issued but not consumed, so that no
// copy is still writing shared memory when the CTA leaves.
__device__ __forceinline__ void stream_drain(const uint64_t *full, unsigned gc_consumed, unsigned gc_issued) {
  if (threadIdx.x == 0)
    for (unsigned c = gc_consumed; c < gc_issued; ++c)
      mbar_wait(smem_u32(full + c % kStreamSlots), (c / kStreamSlots) & 1u, nullptr);
  __syncthreads();
}

// Streamed cell item, for 128 G threads (G column groups of 16 / G sources).  gc: chunks this
// CTA has consumed so far (slot and parity bookkeeping that persists across items); returns false
// if a wait timed out (error recorded, copies drained).
template <int G>
__device__ bool cell_stream_item(const StepArgs<float> &a, const StreamArgs &t, const int cur, const int cell,
                                 const int tile, unsigned char *smem, unsigned &gc) {
  static_assert(G == 1 || G == 2 || G == 4, "16 sources split into 1, 2 or 4 column groups");
  constexpr int CP = kStreamST / G;   // sources per thread
  constexpr int ST = kStreamST;
  const int s0 = tile * ST;
  const int K = a.cell_K[cell], m = a.cell_m[cell], Kq = t.Kq[cell];
  const int ns = min(ST, a.S - s0);
  const int S = a.S;
  const int tid = threadIdx.x;
  unsigned char *ring = smem;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStreamSlots * kStreamChunk);
  float *X = reinterpret_cast<float *>(smem + kStreamSlots * kStreamChunk + 64);
  float *D = X + (size_t)m * K * ST;
  int64_t *rows = reinterpret_cast<int64_t *>(D + (size_t)m * K * ST);
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
  // chunk geometry: whole rows of Kq floats
  const int row_bytes = Kq * 4;
  const int CR = kStreamChunk / row_bytes;
  const int total_rows = (2 * m - 1) * K;
  const int nch = (total_rows + CR - 1) / CR;
  const unsigned gc0 = gc;
  const float *src = t.coef + t.coef_off[cell];
  auto issue = [&](int c) {   // thread 0 only
    const unsigned g = gc0 + (unsigned)c, slot = g % kStreamSlots;
    const int r0 = c * CR, nr = min(CR, total_rows - r0);
    const unsigned bytes = (unsigned)(nr * row_bytes);
    fence_async_smem();
    mbar_expect_tx(smem_u32(full + slot), bytes);
    bulk_g2s(smem_u32(ring + (size_t)slot * kStreamChunk), src + (size_t)r0 * Kq, bytes, smem_u32(full + slot));
  };
  if (tid == 0)
    for (int c = 0; c < min(nch, kStreamSlots); ++c) issue(c);
  // operands: U (face rows gathered, then interior layers), then D^k = U^{k+1} - U^k
  for (int r = tid; r < K; r += blockDim.x) rows[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
  __syncthreads();
  const bool vec = (ns == ST) && (S % 4 == 0);
  if (vec) {
    for (int i = tid; i < K * (ST / 4); i += blockDim.x) {
      const int r = i / (ST / 4), v = i - r * (ST / 4);
      reinterpret_cast<float4 *>(X)[i] = *reinterpret_cast<const float4 *>(fs + (rows[r] >> 1) * S + s0 + v * 4);
    }
    for (int i = tid; i < (m - 1) * K * (ST / 4); i += blockDim.x) {
      const int r = i / (ST / 4), v = i - r * (ST / 4);
      reinterpret_cast<float4 *>(X + (size_t)K * ST)[i] = *reinterpret_cast<const float4 *>(cs + (so + r) * S + s0 + v * 4);
    }
  } else {
    for (int i = tid; i < K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      X[i] = s < ns ? fs[(rows[r] >> 1) * S + s0 + s] : 0.f;
    }
    for (int i = tid; i < (m - 1) * K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      X[(size_t)K * ST + i] = s < ns ? cs[(so + r) * S + s0 + s] : 0.f;
    }
  }
  __syncthreads();
  for (int i = tid; i < m * K * ST; i += blockDim.x) {
    const int k = i / (K * ST);
    D[i] = (k + 1 < m ? X[i + (size_t)K * ST] : 0.f) - X[i];
  }
  __syncthreads();
  const int r = tid & 127, g = tid >> 7;          // row, column group
  const bool act = r < K && g < G;
  const float tau2 = a.tau2;
  auto fail = [&](int c) {
    if (tid == 0) atomicExch(t.err, 1);
    stream_drain(full, gc0 + (unsigned)c, gc0 + (unsigned)min(nch, c + kStreamSlots));
    gc = gc0 + (unsigned)nch;   // bookkeeping only; the caller stops
  };
  int c = 0;                                      // chunk being read
  if (!stream_wait(full, gc0, t.err)) {
    fail(0);
    return false;
  }
  for (int q = 0; q < 2 * m - 1; ++q) {
    if (q == m) {
      // all fluxes are in X: publish F^1, then E^k = F^k - F^{k-1} into D
      __syncthreads();
      if (vec) {
        for (int i = tid; i < K * (ST / 4); i += blockDim.x) {
          const int rr = i / (ST / 4), v = i - rr * (ST / 4);
          *reinterpret_cast<float4 *>(a.flux + rows[rr] * S + s0 + v * 4) = reinterpret_cast<const float4 *>(X)[i];
        }
      } else {
        for (int i = tid; i < K * ST; i += blockDim.x) {
          const int rr = i / ST, s = i - rr * ST;
          if (s < ns) a.flux[rows[rr] * S + s0 + s] = X[i];
        }
      }
      for (int i = tid; i < (m - 1) * K * ST; i += blockDim.x) {
        const size_t jj = (size_t)K * ST + i;
        D[jj] = X[jj] - X[jj - (size_t)K * ST];
      }
      __syncthreads();
    }
    const int layer = q < m ? q : q - m + 1;
    float acc[CP];
#pragma unroll
    for (int e = 0; e < CP; ++e) acc[e] = 0.f;
    for (int j0 = 0; j0 < K;) {
      const int fr = q * K + j0;
      if (fr >= (c + 1) * CR) {
        // chunk c consumed by every thread: refill its slot, move to the next chunk
        __syncthreads();
        if (tid == 0 && c + kStreamSlots < nch) issue(c + kStreamSlots);
        ++c;
        if (!stream_wait(full, gc0 + (unsigned)c, t.err)) {
          fail(c);
          return false;
        }
      }
      const int j1 = min(K, (c + 1) * CR - q * K);
      if (act) {
        const float *sp = reinterpret_cast<const float *>(ring + (size_t)((gc0 + c) % kStreamSlots) * kStreamChunk) +
                          (size_t)(fr - c * CR) * Kq + r;
        const float4 *dp = reinterpret_cast<const float4 *>(D + ((size_t)layer * K + j0) * ST) + (CP / 4) * g;
        const int n = j1 - j0;
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
          const float gv = sp[(size_t)i * Kq];
#pragma unroll
          for (int h = 0; h < CP / 4; ++h) {
            const float4 d = dp[4 * i + h];
            fma2(acc[4 * h + 0], acc[4 * h + 1], gv, d.x, d.y);
            fma2(acc[4 * h + 2], acc[4 * h + 3], gv, d.z, d.w);
          }
        }
      }
      j0 = j1;
    }
    // end of matrix q: row r of F^{q+1}, or leapfrog of U^k with Gamma-hat^k E^k
    if (act) {
      if (q < m) {
        float4 *o = reinterpret_cast<float4 *>(X + ((size_t)q * K + r) * ST + CP * g);
#pragma unroll
        for (int h = 0; h < CP / 4; ++h)
          o[h] = make_float4(acc[4 * h], acc[4 * h + 1], acc[4 * h + 2], acc[4 * h + 3]);
      } else {
        const int k = q - m + 1;
        const int64_t base = (so + (int64_t)(k - 1) * K + r) * S + s0 + CP * g;
        if (vec) {
#pragma unroll
          for (int h = 0; h < CP / 4; ++h) {
            const float4 nw = *reinterpret_cast<const float4 *>(cs + base + 4 * h);
            float4 od = *reinterpret_cast<const float4 *>(cso + base + 4 * h);
            od.x = 2.f * nw.x - od.x + tau2 * acc[4 * h + 0];
            od.y = 2.f * nw.y - od.y + tau2 * acc[4 * h + 1];
            od.z = 2.f * nw.z - od.z + tau2 * acc[4 * h + 2];
            od.w = 2.f * nw.w - od.w + tau2 * acc[4 * h + 3];
            *reinterpret_cast<float4 *>(cso + base + 4 * h) = od;
          }
        } else {
#pragma unroll
          for (int e = 0; e < CP; ++e)
            if (CP * g + e < ns) cso[base + e] = 2.f * cs[base + e] - cso[base + e] + tau2 * acc[e];
        }
      }
    }
  }
  __syncthreads();   // last chunk consumed (its slot may be refilled by the next item)
  if (m == 1) {
    // no interior layers: publish F^1 here
    for (int i = tid; i < K * ST; i += blockDim.x) {
      const int rr = i / ST, s = i - rr * ST;
      if (s < ns) a.flux[rows[rr] * S + s0 + s] = X[i];
    }
  }
  gc = gc0 + (unsigned)nch;
  return true;
}

__device__ __forceinline__ void stream_init(unsigned char *smem) {
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStreamSlots * kStreamChunk);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStreamSlots; ++i) mbar_init(smem_u32(full + i), 1);
    fence_mbar_init();
  }
  __syncthreads();
}

template <int G>
__global__ void __launch_bounds__(128 * G, G == 4 ? 1 : 2) k_cell_s(const StepArgs<float> a, const StreamArgs t,
                                                                     const int cur) {
  extern __shared__ __align__(128) unsigned char smem_s[];
  if (*(volatile const int *)t.err) return;
  stream_init(smem_s);
  unsigned gc = 0;
  const int tiles = (a.S + kStreamST - 1) / kStreamST;   // 1-D grid, tiles of a cell adjacent
  cell_stream_item<G>(a, t, cur, blockIdx.x / tiles, blockIdx.x % tiles, smem_s, gc);
}

// Grid barrier for a cooperative launch.  bar[0] counts arrivals, bar[1] is the generation.
// Returns false (uniformly over the CTA) if the wait exceeded kGridWaitNs or another CTA
// recorded an error.
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *err, int extra = 0) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1 + (unsigned)extra) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      for (unsigned it = 1; *vgen == gen; ++it) {
        if ((it & 63) == 0) {
          if (*(volatile int *)err) { ok = 0; break; }
          if (globaltimer_ns() - t0 > kGridWaitNs) {
            atomicExch(err, 2);
            ok = 0;
            break;
          }
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// n_steps time steps in one launch: per step the cell items (streamed or plain), the face and
// receiver items (receiver items hold blockDim.x / ST receivers), then the corner items.
template <typename T, int ST, bool STREAM>
__global__ void __launch_bounds__(kCellThreads, sizeof(T) == 4 ? 3 : 2) k_persist(const StepArgs<T> a, const StreamArgs t, const int cur0,
                                                             const int n_steps, const double *w, T *traces,
                                                             unsigned *bar, const int n_rcv_items) {
  extern __shared__ __align__(128) unsigned char smem_p[];
  if constexpr (STREAM) stream_init(smem_p);
  // face and corner scratch: after the ring and its mbarriers when the cell body streams
  unsigned char *aux = STREAM ? smem_p + kStreamSlots * kStreamChunk + 64 : smem_p;
  unsigned gc = 0;
  const int tiles = (a.S + ST - 1) / ST;
  const int n_cell_items = a.n_cells * tiles;
  const int n_face_items = (a.n_faces + n_rcv_items) * tiles;
  int n_corner = 0;
  if (a.corners) n_corner = a.n_cfaces * tiles;
  int cur = cur0;
  for (int step = 0; step < n_steps; ++step) {
    for (int it = blockIdx.x; it < n_cell_items; it += gridDim.x) {
      if constexpr (STREAM) {
        if (!cell_stream_item<kCellThreads / 128>(a, t, cur, it / tiles, it % tiles, smem_p, gc)) return;
      } else {
        cell_item<T, ST>(a, cur, it / tiles, it % tiles, smem_p);
      }
      __syncthreads();
    }
    if (!grid_sync(bar, t.err, t.extra_arrivals)) return;
    const int nfb = a.n_faces + n_rcv_items;
    for (int it = blockIdx.x; it < n_face_items; it += gridDim.x) {
      face_item<T, ST>(a, cur, it % nfb, it / nfb, w + step, traces + (int64_t)step * a.n_rcv * a.S, aux);
      __syncthreads();
    }
    if (n_corner > 0) {
      if (!grid_sync(bar, t.err, t.extra_arrivals)) return;
      for (int it = blockIdx.x; it < n_corner; it += gridDim.x) {
        corner_item<T, ST>(a, cur, it % a.n_cfaces, it / a.n_cfaces, aux);
        __syncthreads();
      }
    }
    if (!grid_sync(bar, t.err, t.extra_arrivals)) return;
    cur ^= 1;
  }
}

}  // namespace mss
