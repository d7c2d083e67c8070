// Cell phase on the tensor cores, split into one CTA per (cell, matrix, source tile):
//   flux:         F^k = Gamma^k (U^{k+1} - U^k)                       (CTA per (cell, k), k = 1..m)
//   acceleration: U^k <- 2U^k - U^k_old + tau^2 Gamma-hat^k (F^k - F^{k-1})  (k = 2..m)
// (Eq. intrtstep_td).  Each CTA makes one product D = A B on tcgen05 (kind::f16, M = 128,
// N = NT sources, FP32 accumulators in TMEM): A is one coefficient matrix brought in by two 1-D
// bulk copies (BF16 hi and lo, core layout, as stored by the fused tensor-core kernel), B is
// staged by the threads from FP32 state (lanes over sources, 16-byte core rows, hi/lo split).
// With no product-to-product dependency inside a CTA, two CTAs share an SM and overlap each
// other's copies, staging and epilogues.  The products and the arithmetic of the epilogues are
// the fused kernel's, in the same order.  Every wait is bounded; on timeout the CTA records an
// error, drains its copies (bounded), frees its TMEM and returns.
#pragma once

namespace mss {

constexpr int kTcsThreads = 128;   // 4 warps = the 128 TMEM lanes (accumulator rows)

// Shared-memory bytes of one split tensor-core CTA with NT sources and KpMax columns.
__host__ __device__ constexpr size_t tcs_smem_bytes(int NT, int kpmax) {
  return (size_t)2 * 128 * kpmax * 2 + (size_t)2 * NT * kpmax * 2 + 64;
}

template <int NT, bool FLUX>
__global__ void __launch_bounds__(kTcsThreads, 2) k_tc_split(const StepArgs<float> a, const SplitArgs<float> p,
                                                             const TcArgs t, const int cur) {
  const int tiles = (a.S + NT - 1) / NT;           // 1-D grid, tiles of an item adjacent
  const int2 it = FLUX ? p.flux_items[blockIdx.x / tiles] : p.accel_items[blockIdx.x / tiles];
  const int cell = it.x, k = it.y;
  const int s0 = (blockIdx.x % tiles) * NT;
  const int K = a.cell_K[cell], m = a.cell_m[cell];
  const int Kp = t.Kp[cell], Kr = t.Kr[cell];
  const int S = a.S, ns = min(NT, S - s0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(128) unsigned char smem[];
  // layout: A hi (128 x KpMax), A lo, B hi (NT x KpMax), B lo, then barriers; the A halves and
  // the B halves are KpMax-strided so that one allocation serves every cell
  const int kpmax = (t.slot_bytes / 2) / (128 * 2);
  unsigned char *Ah = smem, *Al = smem + 128 * kpmax * 2;
  unsigned char *Bh = smem + 2 * 128 * kpmax * 2, *Bl = Bh + NT * kpmax * 2;
  uint64_t *bars = reinterpret_cast<uint64_t *>(Bl + NT * kpmax * 2);   // full, done
  unsigned *tmem_sm = reinterpret_cast<unsigned *>(bars + 2);
  const unsigned full = smem_u32(bars + 0), done = smem_u32(bars + 1);
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
  const int mat = FLUX ? k : m + k - 1;              // Gamma^{k+1} or Gamma-hat^{k+1} in the blob
  const unsigned mat_half = (unsigned)Kr * Kp * 2;
  const unsigned char *src = t.blob + t.blob_off[cell] + (size_t)mat * 2 * mat_half;
  unsigned cols = 32;
  while (cols < (unsigned)NT) cols <<= 1;

  __shared__ int bail;
  if (tid == 0) bail = *(volatile const int *)t.err;
  __syncthreads();
  if (bail) return;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_sm)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(done, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(full, 2 * mat_half);
    bulk_g2s(smem_u32(Ah), src, mat_half, full);
    bulk_g2s(smem_u32(Al), src + mat_half, mat_half, full);
  }
  // A rows Kr..127 are zero (the copies write rows 0..Kr-1 only)
  {
    const int pad0 = Kr * Kp * 2, pad1 = 128 * Kp * 2;
    for (int i = pad0 / 16 + tid; i < pad1 / 16; i += kTcsThreads) {
      reinterpret_cast<int4 *>(Ah)[i] = make_int4(0, 0, 0, 0);
      reinterpret_cast<int4 *>(Al)[i] = make_int4(0, 0, 0, 0);
    }
  }
  // B: D^k = U^{k+1} - U^k (flux) or E^k = F^k - F^{k-1} (acceleration), rows >= K zero
  const float *Fk = p.F + (p.f_off[cell] + (int64_t)k * K) * S + s0;
  {
    constexpr int CPW = NT < 32 ? NT : 32;
    constexpr int RPW = 32 / CPW;
    const int NR8 = Kp / 8, ngp = (NR8 + RPW - 1) / RPW, cblocks = NT / CPW;
    const int cl = lane % CPW, sub = lane / CPW;
    for (int tt = warp; tt < ngp * cblocks; tt += kTcsThreads / 32) {
      const int cb = tt % cblocks, gp = tt / cblocks;
      const int g8 = gp * RPW + sub, c = cb * CPW + cl;
      if (g8 >= NR8) continue;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = g8 * 8 + i;
        float x = 0.f;
        if (r < K && c < ns) {
          if (FLUX) {
            const float u0 = k == 0 ? fs[(a.row_face_row[rp + r]) * S + s0 + c]
                                    : cs[(so + (int64_t)(k - 1) * K + r) * S + s0 + c];
            const float u1 = k + 1 < m ? cs[(so + (int64_t)k * K + r) * S + s0 + c] : 0.f;
            x = u1 - u0;
          } else {
            x = Fk[(int64_t)r * S + c] - Fk[(int64_t)(r - K) * S + c];
          }
        }
        v[i] = x;
      }
      store_core8(Bh, Bl, core_off(c, g8 * 8, Kp), v);
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_sm;
  __shared__ int ok_sm, issued_sm;
  if (tid == 0) {
    int ok = mbar_wait(full, 0, t.err) ? 1 : 0;
    issued_sm = 0;
    if (ok) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128, NT);
      const unsigned lbo = 128, sbo = 16u * Kp;
      const unsigned ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
      for (int kk = 0; kk < Kp / 16; ++kk) {
        const unsigned o = kk * 256;
        mma_bf16(tmem, sdesc(ah + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, kk > 0 ? 1u : 0u);
        if (t.terms == 3) {
          mma_bf16(tmem, sdesc(ah + o, lbo, sbo), sdesc(bl + o, lbo, sbo), idesc, 1u);
          mma_bf16(tmem, sdesc(al + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, 1u);
        }
      }
      tc_commit(done);
      issued_sm = 1;
      ok = mbar_wait(done, 0, t.err) ? 1 : 0;
    }
    ok_sm = ok;
  }
  __syncthreads();
  const bool go = ok_sm != 0;
  tc_fence_after();
  if (go) {
    const int r = 32 * warp + lane;                  // accumulator row = TMEM lane
    const unsigned lane_addr = (unsigned)(32 * warp) << 16;
    const bool vec_ok = (S % 4) == 0;
    const float tau2 = a.tau2;
    for (int cc = 0; cc < NT; cc += 8) {
      float acc[8];
      __syncwarp();
      tc_ld8(tmem + lane_addr + (unsigned)cc, acc);   // every lane loads; stores are predicated
      if (r < K) {
      const bool full8 = vec_ok && cc + 8 <= ns;
      if (FLUX) {
        float *o = p.F + (p.f_off[cell] + (int64_t)k * K + r) * S + s0 + cc;
        float *fo = k == 0 ? a.flux + (a.row_face_row[rp + r] * 2 + a.row_side[rp + r]) * S + s0 + cc : nullptr;
        if (full8) {
          const float4 v0 = make_float4(acc[0], acc[1], acc[2], acc[3]);
          const float4 v1 = make_float4(acc[4], acc[5], acc[6], acc[7]);
          reinterpret_cast<float4 *>(o)[0] = v0;
          reinterpret_cast<float4 *>(o)[1] = v1;
          if (fo) {
            reinterpret_cast<float4 *>(fo)[0] = v0;
            reinterpret_cast<float4 *>(fo)[1] = v1;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (cc + j < ns) {
              o[j] = acc[j];
              if (fo) fo[j] = acc[j];
            }
        }
      } else {
        const int64_t base = (so + (int64_t)(k - 1) * K + r) * S + s0 + cc;
        if (full8) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
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
          for (int j = 0; j < 8; ++j)
            if (cc + j < ns) cso[base + j] = 2.f * cs[base + j] - cso[base + j] + tau2 * acc[j];
        }
      }
      }
    }
  } else if (tid == 0) {
    atomicExch(t.err, 1);
    // the A copies must land, and issued products finish, before shared memory and TMEM go away
    mbar_wait(full, 0, nullptr);
    if (issued_sm) mbar_wait(done, 0, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
  }
}

}  // namespace mss
