// Wide streamed cell kernel: the cell phase for large boundary dimensions (K_i up to 384), FP32 on
// the CUDA cores, 16-source tiles, the coefficient stream staged by TMA.
//
// At the paper's operating point (cells about one wavelength across, K~ = 180-294, Section 7) a
// cell's 2m-1 coefficient matrices hold about 2 MB per step, more than the L2 share of the CTAs
// resident at once, so the stream is moved by the copy engine, not by thread loads: one thread
// issues 1-D bulk copies (cp.async.bulk) of whole stored rows into a ring of 16 KB shared-memory
// slots (eight per SM), each guarded by an mbarrier with a transaction count, and the threads
// consume them.  Thread (q, g): g = tid % 4 picks 4 of the 16 sources, q = tid / 4 the R
// consecutive output rows Rq .. Rq+R-1 (R = 4 or 2).  Row j of a stored symmetric matrix is also
// its column j, so
//   acc[i][e] += G[j][Rq + i] * D[j][4g + e]
// takes one 16-byte (or 8-byte) load of the slot and one broadcast 16-byte load of D per row j for
// 4R fused multiply-adds (2R paired instructions).  R = 4 halves the instructions per multiply-add
// against one row per thread; R = 2 doubles the warps that hide the shared-memory latency.
//
// Factored last coefficient (Gamma^m = L L^T, the stored matrix W = L + L^T - diag(L) with its rows
// in descending order): F^m = L (L^T D^m) in one pass over the stream.  Rows j arrive from K-1 down
// to 0.  In each ring segment, y_r += W[j][r] D^m_j for r <= j (the L^T product; y_j is complete
// once row j has passed), the segment's complete y_j go to shared memory, and after a barrier
// F_r += W[j][r] y_j for r >= j (the L product) reuses the same rows from the slot.  Per element
// this is the same sequence of fused multiply-adds as the plain cell kernel's descending
// triangular passes, so both give identical bits.
//
// Chunks advance per warp: each warp waits on the next chunk's barrier itself, and the last warp
// to release a chunk (a count in shared memory) refills its slot, so no block-wide barrier is taken
// per chunk.  Every wait is bounded (globaltimer); on timeout the error is recorded, the warps keep
// the block's control flow without waiting, and the CTA waits (bounded) for its copies in flight
// before it returns.
#pragma once

namespace mss {

constexpr int kWideMaxK = 384;     // largest K_i of the wide kernel
constexpr int kWideCP = 4;          // sources per thread (four 4-source groups per 16-source tile)
// threads of the wide kernel with R consecutive rows per thread and NS-source tiles: NS / 4 source
// groups x K_max / R
__host__ __device__ constexpr int wide_threads(int R, int NS) { return NS / 4 * kWideMaxK / R; }
// ring slots of the wide kernel: eight 16 KB slots with 16-source tiles; four with 8-source tiles,
// whose smaller operand block then lets two CTAs share an SM (eight slots per SM either way)
__host__ __device__ constexpr int wide_slots(int NS) { return NS == 16 ? 8 : 4; }

// Shared memory of the wide kernel with NS-source tiles: ring, a 128-byte header (the slots'
// barriers, release counts and issue count), one operand block of m K NS floats (U, then D^k,
// then F^k, then E^k, each in place), the factored product's y (K NS floats), the K boundary-row
// indices.
inline size_t wide_smem_bytes(int max_m, int max_K, int factor_last, int NS) {
  return (size_t)wide_slots(NS) * kStreamChunk + 128 +
         ((size_t)max_m * max_K * NS + (factor_last ? (size_t)max_K * NS : 0)) * 4 + 8 * (size_t)max_K;
}

// R consecutive floats of a slot row (16-byte or 8-byte aligned: Kq and r4 are multiples of R)
template <int R>
__device__ __forceinline__ void load_rows(float (&gv)[R], const float *p) {
  if constexpr (R == 4) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    gv[0] = q.x; gv[1] = q.y; gv[2] = q.z; gv[3] = q.w;
  } else {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    gv[0] = q.x; gv[1] = q.y;
  }
}

__device__ __forceinline__ void fma4(float (&acc)[kWideCP], float gv, const float4 d) {
  fma2(acc[0], acc[1], gv, d.x, d.y);
  fma2(acc[2], acc[3], gv, d.z, d.w);
}

// One (cell, 16-source tile) of the cell phase.  gc: chunks this CTA has consumed so far; returns
// false if a wait timed out (error recorded, copies drained).  U: unroll depth of the row loops
// (the autotuner picks 2 or 4); R: consecutive rows per thread (4, or 2 for twice the warps); the
// arithmetic depends on neither.
template <int U, int R, int NS>
__device__ bool cell_wide_item(const StepArgs<float> &a, const StreamArgs &t, const int cur, const int cell,
                               const int tile, unsigned char *smem, unsigned &gc) {
  constexpr int ST = NS, CP = kWideCP, SL = wide_slots(NS), G = NS / CP;
  const int s0 = tile * ST;
  const int K = a.cell_K[cell], m = a.cell_m[cell], Kq = t.Kq[cell];
  const int ns = min(ST, a.S - s0);
  const int S = a.S;
  const int tid = threadIdx.x;
  const bool fac = a.factor_last != 0;
  unsigned char *ring = smem;
  // header: the slots' barriers, per-slot release counts of the warps, the chunks issued so far
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + SL * kStreamChunk);
  unsigned *released = reinterpret_cast<unsigned *>(smem + SL * kStreamChunk + 64);
  unsigned *issued = released + SL;
  float *D = reinterpret_cast<float *>(smem + SL * kStreamChunk + 128);
  float *Ys = D + (size_t)m * K * ST;
  int64_t *rows = reinterpret_cast<int64_t *>(Ys + (fac ? (size_t)K * ST : 0));
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
  const int row_bytes = Kq * 4;
  const int CR = kStreamChunk / row_bytes;
  const int total_rows = (2 * m - 1) * K;
  const int nch = (total_rows + CR - 1) / CR;
  const unsigned gc0 = gc;
  const float *src = t.coef + t.coef_off[cell];
  auto issue = [&](int c) {   // thread 0 only
    const unsigned g = gc0 + (unsigned)c, slot = g % SL;
    const int r0 = c * CR, nr = min(CR, total_rows - r0);
    const unsigned bytes = (unsigned)(nr * row_bytes);
    fence_async_smem();
    mbar_expect_tx(smem_u32(full + slot), bytes + t.extra_tx);
    bulk_g2s(smem_u32(ring + (size_t)slot * kStreamChunk), src + (size_t)r0 * Kq, bytes, smem_u32(full + slot));
  };
  if (tid == 0) {
    for (int i = 0; i < SL; ++i) released[i] = 0;
    *issued = (unsigned)min(nch, SL);
    for (int c = 0; c < min(nch, SL); ++c) issue(c);
  }
  // operand block: U (face rows gathered, then interior layers), then D^k = U^{k+1} - U^k in place
  for (int r = tid; r < K; r += blockDim.x) rows[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
  __syncthreads();
  const bool vec = (ns == ST) && (S % 4 == 0);
  if (vec) {
    for (int i = tid; i < K * (ST / 4); i += blockDim.x) {
      const int r = i / (ST / 4), v = i - r * (ST / 4);
      reinterpret_cast<float4 *>(D)[i] = *reinterpret_cast<const float4 *>(fs + (rows[r] >> 1) * S + s0 + v * 4);
    }
    for (int i = tid; i < (m - 1) * K * (ST / 4); i += blockDim.x) {
      const int r = i / (ST / 4), v = i - r * (ST / 4);
      reinterpret_cast<float4 *>(D + (size_t)K * ST)[i] = *reinterpret_cast<const float4 *>(cs + (so + r) * S + s0 + v * 4);
    }
  } else {
    for (int i = tid; i < K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      D[i] = s < ns ? fs[(rows[r] >> 1) * S + s0 + s] : 0.f;
    }
    for (int i = tid; i < (m - 1) * K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      D[(size_t)K * ST + i] = s < ns ? cs[(so + r) * S + s0 + s] : 0.f;
    }
  }
  __syncthreads();
  // one thread per (row, source) position walks the layers upwards, so U^{k+1} is read before
  // its own difference overwrites it
  for (int p = tid; p < K * ST; p += blockDim.x) {
    float u = D[p];
    for (int k = 0; k < m; ++k) {
      const float un = k + 1 < m ? D[(size_t)(k + 1) * K * ST + p] : 0.f;
      D[(size_t)k * K * ST + p] = un - u;
      u = un;
    }
  }
  __syncthreads();
  // consecutive threads share a row quad (one broadcast 16-byte coefficient load) and take its four
  // 4-source groups; the quads of a small K are then packed into the first warps, and the warps
  // beyond 4 K threads have no rows at all (no partially filled warps)
  const int g = tid % G, r4 = R * (tid / G);
  const bool actq = r4 < K;                      // rows r4 .. r4+R-1 (those >= K read zero padding)
  int rr[R];
  bool act[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    rr[i] = r4 + i;
    act[i] = rr[i] < K;
  }
  const float tau2 = a.tau2;
  const int lane = tid & 31;
  const unsigned nwarps = blockDim.x >> 5;
  // Chunks advance per warp, not per block: a warp waits for the next chunk's barrier on its own,
  // and the last warp to release a chunk refills its slot (release counts in shared memory), so no
  // block-wide barrier is taken per chunk.  A wait that runs out records the error; the warp then
  // stops waiting (its results are void, the state of a failed step is undefined) but keeps the
  // block's control flow, and the copies in flight are drained at the end.
  bool bad = false;
  auto wait_chunk = [&](int cc) {
    const unsigned gg = gc0 + (unsigned)cc;
    const bool ok = mbar_wait(smem_u32(full + gg % SL), (gg / SL) & 1u, t.err);
    if (__all_sync(0xffffffffu, ok)) return;
    if (lane == 0) atomicExch(t.err, 1);
    bad = true;
  };
  int c = 0;                                      // chunk being read
  wait_chunk(0);
  for (int q = 0; q < 2 * m - 1; ++q) {
    if (q == m) {
      // all fluxes are in the operand block: publish F^1, then E^k = F^k - F^{k-1} in place
      __syncthreads();
      if (vec) {
        for (int i = tid; i < K * (ST / 4); i += blockDim.x) {
          const int r = i / (ST / 4), v = i - r * (ST / 4);
          *reinterpret_cast<float4 *>(a.flux + rows[r] * S + s0 + v * 4) = reinterpret_cast<const float4 *>(D)[i];
        }
      } else {
        for (int i = tid; i < K * ST; i += blockDim.x) {
          const int r = i / ST, s = i - r * ST;
          if (s < ns) a.flux[rows[r] * S + s0 + s] = D[i];
        }
      }
      // layers downwards per position, so F^{k-1} is read before it becomes E^{k-1}
      for (int p = tid; p < K * ST; p += blockDim.x)
        for (int k = m - 1; k >= 1; --k) D[(size_t)k * K * ST + p] -= D[(size_t)(k - 1) * K * ST + p];
      __syncthreads();
    }
    const int layer = q < m ? q : q - m + 1;
    const bool tri = fac && q == m - 1;           // the factored last coefficient, rows descending
    float acc[R][CP], yv[R][CP];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int e = 0; e < CP; ++e) acc[i][e] = yv[i][e] = 0.f;
    const float *Dl = D + (size_t)layer * K * ST + CP * g;
    for (int j0 = 0; j0 < K;) {
      const int fr = q * K + j0;
      if (fr >= (c + 1) * CR) {
        // this warp is done with chunk c; the last warp to release it refills the slot
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          const unsigned slot = (gc0 + (unsigned)c) % SL;
          if (atomicAdd(released + slot, 1u) == nwarps - 1) {
            atomicExch(released + slot, 0u);
            __threadfence_block();
            if (c + SL < nch) {
              issue(c + SL);
              atomicMax(issued, (unsigned)(c + SL + 1));
            }
          }
        }
        __syncwarp();
        ++c;
        if (!bad) wait_chunk(c);
      }
      const int j1 = min(K, (c + 1) * CR - q * K);
      const int n = j1 - j0;
      const float *sp = reinterpret_cast<const float *>(ring + (size_t)((gc0 + c) % SL) * kStreamChunk) +
                        (size_t)(fr - c * CR) * Kq;
      if (!tri) {
        // acc[i] += G[j][r4 + i] D^layer_j, j = j0 .. j1-1 ascending
        if (actq) {
#pragma unroll U
          for (int h = 0; h < n; ++h) {
            const float4 d = *reinterpret_cast<const float4 *>(Dl + (size_t)(j0 + h) * ST);
            float gv[R];
            load_rows<R>(gv, sp + (size_t)h * Kq + r4);
#pragma unroll
            for (int i = 0; i < R; ++i) fma4(acc[i], gv[i], d);
          }
        }
      } else {
        // stored position p holds row K-1-p: the segment covers rows jt = K-1-j0 down to jb
        const int jt = K - 1 - j0, jb = K - j1;
#pragma unroll U
        for (int h = 0; h < n && actq; ++h) {
          const int j = jt - h;
          const float4 d = *reinterpret_cast<const float4 *>(Dl + (size_t)j * ST);
          float gv[R];
          load_rows<R>(gv, sp + (size_t)h * Kq + r4);
#pragma unroll
          for (int i = 0; i < R; ++i)
            if (rr[i] <= j) fma4(yv[i], gv[i], d);
        }
        // the y of this segment's rows are complete: share them
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (act[i] && rr[i] >= jb && rr[i] <= jt)
            *reinterpret_cast<float4 *>(Ys + (size_t)rr[i] * ST + CP * g) =
                make_float4(yv[i][0], yv[i][1], yv[i][2], yv[i][3]);
        __syncthreads();
#pragma unroll U
        for (int h = 0; h < n && actq; ++h) {
          const int j = jt - h;
          const float4 y = *reinterpret_cast<const float4 *>(Ys + (size_t)j * ST + CP * g);
          float gv[R];
          load_rows<R>(gv, sp + (size_t)h * Kq + r4);
#pragma unroll
          for (int i = 0; i < R; ++i)
            if (rr[i] >= j) fma4(acc[i], gv[i], y);
        }
      }
      j0 = j1;
    }
    // end of matrix q: rows of F^{q+1} (over D^{q+1}, once every warp has passed it), or leapfrog of
    // U^k with Gamma-hat^k E^k
    if (q < m) __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if (!act[i]) continue;
      const int r = rr[i];
      if (q < m) {
        *reinterpret_cast<float4 *>(D + ((size_t)q * K + r) * ST + CP * g) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      } else {
        const int k = q - m + 1;
        const int64_t base = (so + (int64_t)(k - 1) * K + r) * S + s0 + CP * g;
        if (vec) {
#pragma unroll
          for (int h = 0; h < CP / 4; ++h) {
            const float4 nw = *reinterpret_cast<const float4 *>(cs + base + 4 * h);
            float4 od = *reinterpret_cast<const float4 *>(cso + base + 4 * h);
            od.x = 2.f * nw.x - od.x + tau2 * acc[i][4 * h + 0];
            od.y = 2.f * nw.y - od.y + tau2 * acc[i][4 * h + 1];
            od.z = 2.f * nw.z - od.z + tau2 * acc[i][4 * h + 2];
            od.w = 2.f * nw.w - od.w + tau2 * acc[i][4 * h + 3];
            *reinterpret_cast<float4 *>(cso + base + 4 * h) = od;
          }
        } else {
#pragma unroll
          for (int e = 0; e < CP; ++e)
            if (CP * g + e < ns) cso[base + e] = 2.f * cs[base + e] - cso[base + e] + tau2 * acc[i][e];
        }
      }
    }
  }
  __syncthreads();   // last chunk consumed (its slot may be refilled by the next item)
  if (*(volatile int *)t.err) {
    // a wait ran out somewhere: let the copies still in flight (only the last SL issued
    // can be) land before the CTA leaves
    if (tid == 0) {
      const unsigned iss = *issued;
      for (unsigned cc = iss > (unsigned)SL ? iss - SL : 0u; cc < iss; ++cc) {
        const unsigned gg = gc0 + cc;
        mbar_wait(smem_u32(full + gg % SL), (gg / SL) & 1u, nullptr);
      }
    }
    __syncthreads();
    gc = gc0 + (unsigned)nch;
    return false;
  }
  if (m == 1) {
    // no interior layers: publish F^1 here
    for (int i = tid; i < K * ST; i += blockDim.x) {
      const int r = i / ST, s = i - r * ST;
      if (s < ns) a.flux[rows[r] * S + s0 + s] = D[i];
    }
  }
  gc = gc0 + (unsigned)nch;
  return true;
}

template <int U, int R, int NS>
__global__ void __launch_bounds__(wide_threads(R, NS), NS == 16 ? 1 : 2)
    k_cell_w(const StepArgs<float> a, const StreamArgs t, const int cur) {
  extern __shared__ __align__(128) unsigned char smem_w[];
  if (*(volatile const int *)t.err) return;
  constexpr int SL = wide_slots(NS);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_w + SL * kStreamChunk);
  if (threadIdx.x == 0) {
    for (int i = 0; i < SL; ++i) mbar_init(smem_u32(full + i), 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned gc = 0;
  const int tiles = (a.S + NS - 1) / NS;   // 1-D grid, tiles of a cell adjacent
  cell_wide_item<U, R, NS>(a, t, cur, blockIdx.x / tiles, blockIdx.x % tiles, smem_w, gc);
}

}  // namespace mss
