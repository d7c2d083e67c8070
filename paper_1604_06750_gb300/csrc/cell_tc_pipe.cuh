// Cell phase on the tensor cores as a warp-specialised persistent kernel (one CTA per SM).
//
// Warp 0 (producer, one lane) streams the coefficient matrices of the CTA's (cell, source tile)
// items -- Gamma^1..Gamma^m then Gamma-hat^2..Gamma-hat^m of each cell, BF16 hi/lo in the
// core-matrix layout -- through a ring of shared-memory slots with 1-D bulk copies, gated by
// per-slot "empty" mbarriers that the tensor core arrives on when the products reading the slot
// have completed.  Warps 1-8 (two per TMEM lane quarter, one per column half) do, per item:
//   stage B = U^{k+1} - U^k (all k)  ->  one thread issues the m flux products into TMEM
//   (F^k in columns k NT), commit  ->  publish F^1, E^k = F^k - F^{k-1} into the B buffers
//   (8x8 lane transposes)  ->  the m-1 acceleration products (Gamma-hat^k E^k), commit  ->
//   hidden-layer leapfrog (Eq. intrtstep_td).
// The matrices of the next items are already in flight while an item's staging and epilogues
// run, so the coefficient stream (the dominant bytes) is not serialised behind them.  Products
// and epilogue arithmetic are those of the fused tensor-core kernel (same values, same order).
// Every wait is bounded (globaltimer) and stops on the error word; on error the CTA waits
// (bounded) for its copies and products in flight, frees its TMEM and returns.
#pragma once

namespace mss {

constexpr int kTcpCompute = 256;   // warps 1..8 compute: warp w reads TMEM lane quarter w % 4, column half (w-1) / 4
constexpr int kTcpThreads = 32 + kTcpCompute;   // warp 0 producer
constexpr int kTcpSlots = 4;

__device__ __forceinline__ void compute_bar() { asm volatile("bar.sync 1, %0;\n" ::"n"(kTcpCompute) : "memory"); }

// Bytes of shared memory of k_cell_tcp: barriers, ring of kTcpSlots matrices (Kr_max rows, hi
// then lo), max_m B buffers (hi, lo) of NT x Kp_max, K_max boundary rows, and a tail so that the
// 128-row A reads of the last slot stay inside the allocation.
__host__ __device__ constexpr size_t tcp_smem(int NT, int kpmax, int krmax, int max_m, int max_K) {
  return 256 + (size_t)kTcpSlots * 2 * krmax * kpmax * 2 + (size_t)max_m * 2 * NT * kpmax * 2 + 8 * (size_t)max_K +
         (size_t)128 * kpmax * 2 + 64;
}

template <int NT>
__global__ void __launch_bounds__(kTcpThreads, 1) k_cell_tcp(const StepArgs<float> a, const TcArgs t, const int cur,
                                                             const int krmax, const int max_m) {
  const int tiles = (a.S + NT - 1) / NT;
  const int total = a.n_cells * tiles;
  const int S = a.S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(128) unsigned char smem[];
  const int kpmax = t.kpmax;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);      // full[4] empty[4] mdone
  int *ctl = reinterpret_cast<int *>(smem + 128);              // [0] tmem base, [1] ok, [2] copies issued,
                                                               // [3] copies consumed, [4] commits, [5] waited
  const size_t half = (size_t)krmax * kpmax * 2;
  unsigned char *ring = smem + 256;
  unsigned char *bbuf = ring + (size_t)kTcpSlots * 2 * half;
  const size_t bstride = (size_t)2 * NT * kpmax * 2;          // one B buffer: hi then lo
  int64_t *rows = reinterpret_cast<int64_t *>(bbuf + (size_t)max_m * bstride);
  unsigned full[kTcpSlots], empty[kTcpSlots];
#pragma unroll
  for (int i = 0; i < kTcpSlots; ++i) {
    full[i] = smem_u32(bars + i);
    empty[i] = smem_u32(bars + kTcpSlots + i);
  }
  const unsigned mdone = smem_u32(bars + 2 * kTcpSlots);
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  unsigned cols = 32;
  while (cols < (unsigned)(max_m * NT)) cols <<= 1;

  __shared__ int bail;
  if (tid == 0) bail = *(volatile const int *)t.err;
  __syncthreads();
  if (bail || (int)blockIdx.x >= total) return;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(ctl)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * kTcpSlots + 1; ++i) mbar_init(smem_u32(bars + i), 1);
    ctl[1] = 1;
    ctl[2] = ctl[3] = ctl[4] = ctl[5] = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = (unsigned)ctl[0];

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      unsigned g = 0;
      for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int cell = it / tiles;
        const int m = a.cell_m[cell];
        const unsigned mh = (unsigned)t.Kr[cell] * t.Kp[cell] * 2;
        const unsigned char *src = t.blob + t.blob_off[cell];
        bool stop = false;
        for (int p = 0; p < 2 * m - 1; ++p, ++g) {
          const unsigned slot = g % kTcpSlots, use = g / kTcpSlots;
          if (use > 0 && !mbar_wait(empty[slot], (use - 1) & 1, t.err)) {
            atomicExch(t.err, 1);
            stop = true;
            break;
          }
          unsigned char *dst = ring + (size_t)slot * 2 * half;
          mbar_expect_tx(full[slot], t.terms == 3 ? 2 * mh : mh);
          bulk_g2s(smem_u32(dst), src + (size_t)p * 2 * mh, mh, full[slot]);
          if (t.terms == 3) bulk_g2s(smem_u32(dst + half), src + (size_t)p * 2 * mh + mh, mh, full[slot]);
          ctl[2] = (int)(g + 1);
        }
        if (stop) break;
      }
    }
    __syncwarp();   // the other producer lanes wait for lane 0 before the final barrier
  } else {
    // ---------------------------------------------------------------- compute warps
    const int ct = tid - 32, cw = ct >> 5;
    const int q = warp & 3;                             // TMEM lane quarter of this warp
    const int r = 32 * q + lane;                        // accumulator row
    const unsigned lane_addr = (unsigned)(32 * q) << 16;
    constexpr int CH = NT / 2;                          // columns of this warp's half
    const int c0 = (cw >> 2) * CH;
    const uint32_t idesc = idesc_bf16(128, NT);
    unsigned gm = 0, nmd = 0;                           // matrices consumed, mdone commits (issuer)
    const bool vec_ok = (S % 4) == 0;
    const float tau2 = a.tau2;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
      const int cell = it / tiles;
      const int s0 = (it % tiles) * NT;
      const int K = a.cell_K[cell], m = a.cell_m[cell], Kp = t.Kp[cell];
      const int ns = min(NT, S - s0);
      const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
      for (int i = ct; i < K; i += kTcpCompute) rows[i] = a.row_face_row[rp + i] * 2 + a.row_side[rp + i];
      compute_bar();
      // stage B^k = U^{k+1} - U^k, k = 0..m-1
      tc_stage_layers<NT>(fs, cs, rows, so, S, s0, ns, K, Kp, m, bbuf, bstride, (size_t)NT * kpmax * 2, cw,
                          kTcpCompute / 32, lane);
      fence_async_smem();
      tc_fence_before();
      compute_bar();
      tc_fence_after();
      const unsigned lbo = 128, sbo = 16u * Kp;
      auto issue_products = [&](int p0, int p1) -> bool {   // issuer thread only
        for (int p = p0; p < p1; ++p, ++gm) {
          const unsigned slot = gm % kTcpSlots;
          if (!mbar_wait(full[slot], (gm / kTcpSlots) & 1, t.err)) return false;
          ctl[3] = (int)(gm + 1);
          tc_fence_after();
          const int bi = p < m ? p : p - m;                 // B buffer: D^p, or E^{p-m+1} in buffer p-m
          const unsigned ah = smem_u32(ring + (size_t)slot * 2 * half), al = ah + (unsigned)half;
          const unsigned bh = smem_u32(bbuf + (size_t)bi * bstride), bl = bh + (unsigned)(NT * kpmax * 2);
          const unsigned dcol = tmem + (unsigned)(bi * NT);
          for (int kk = 0; kk < Kp / 16; ++kk) {
            const unsigned o = kk * 256;
            mma_bf16(dcol, sdesc(ah + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, kk > 0 ? 1u : 0u);
            if (t.terms == 3) {
              mma_bf16(dcol, sdesc(ah + o, lbo, sbo), sdesc(bl + o, lbo, sbo), idesc, 1u);
              mma_bf16(dcol, sdesc(al + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, 1u);
            }
          }
          tc_commit(empty[slot]);
        }
        return true;
      };
      // ---- flux products
      if (ct == 0) {
        bool ok = issue_products(0, m);
        if (ok) {
          tc_commit(mdone);
          ++nmd;
          ctl[4] = (int)nmd;
          ok = mbar_wait(mdone, (nmd - 1) & 1, t.err);
          if (ok) ctl[5] = (int)nmd;
        }
        if (!ok) {
          atomicExch(t.err, 1);
          ctl[1] = 0;
        }
      }
      compute_bar();
      if (!ctl[1]) break;
      tc_fence_after();
      // ---- publish F^1; E^k = F^k - F^{k-1} into B buffer k-1
      for (int ch = 0; ch < CH; ch += 8) {
        const int cc = c0 + ch;
        float prev[8], curv[8];
        const bool full8 = vec_ok && cc + 8 <= ns;
        for (int k = 0; k < m; ++k) {
          __syncwarp();
          tc_ld8(tmem + lane_addr + (unsigned)(k * NT + cc), curv);
          if (k == 0) {
            if (r < K) {
              float *o = a.flux + rows[r] * S + s0 + cc;
              if (full8) {
                reinterpret_cast<float4 *>(o)[0] = make_float4(curv[0], curv[1], curv[2], curv[3]);
                reinterpret_cast<float4 *>(o)[1] = make_float4(curv[4], curv[5], curv[6], curv[7]);
              } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                  if (cc + j < ns) o[j] = curv[j];
              }
            }
          } else {
            float e8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) e8[j] = r < K ? curv[j] - prev[j] : 0.f;
            transpose8(e8, lane);
            const int r0 = r & ~7;
            if (r0 < Kp) {
              unsigned char *h = bbuf + (size_t)(k - 1) * bstride;
              store_core8(h, h + NT * kpmax * 2, core_off(cc + (lane & 7), r0, Kp), e8);
            }
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) prev[j] = curv[j];
        }
      }
      fence_async_smem();
      tc_fence_before();
      compute_bar();
      tc_fence_after();
      // ---- acceleration products
      if (ct == 0 && m > 1) {
        bool ok = issue_products(m, 2 * m - 1);
        if (ok) {
          tc_commit(mdone);
          ++nmd;
          ctl[4] = (int)nmd;
          ok = mbar_wait(mdone, (nmd - 1) & 1, t.err);
          if (ok) ctl[5] = (int)nmd;
        }
        if (!ok) {
          atomicExch(t.err, 1);
          ctl[1] = 0;
        }
      }
      compute_bar();
      if (!ctl[1]) break;
      tc_fence_after();
      // ---- hidden-layer leapfrog
      tc_leapfrog<NT, CH>(tmem, lane_addr, cs, cso, so, K, S, s0, ns, m, r, c0, tau2);
      tc_fence_before();
      compute_bar();   // TMEM columns, B buffers and rows are free for the next item
    }
  }
  __syncthreads();
  if (tid == 0 && !ctl[1]) {
    // wait (bounded) for this CTA's copies and products still in flight
    for (int c = ctl[3]; c < ctl[2]; ++c) mbar_wait(full[c % kTcpSlots], (c / kTcpSlots) & 1, nullptr);
    if (ctl[4] > ctl[5]) mbar_wait(mdone, (ctl[4] - 1) & 1, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
  }
}

}  // namespace mss
