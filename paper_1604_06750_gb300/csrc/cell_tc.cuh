// Cell phase of the on-line step on the 5th-generation tensor cores (sm_103a).
//
// Per (cell, source tile of NT sources), one CTA of 256 threads computes what k_cell computes:
//   F^k = Gamma^k (U^{k+1} - U^k), k = 1..m;  publish F^1;  E^k = F^k - F^{k-1};
//   U^k <- 2U^k - U^k_old + tau^2 Gamma-hat^k E^k, k = 2..m            (Eq. intrtstep_td)
// with every matrix product on tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in TMEM).
// FP32 accuracy is kept by splitting both operands into BF16 hi + lo parts and summing three
// products, A_hi B_hi + A_hi B_lo + A_lo B_hi (terms = 3); terms = 1 is plain BF16.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout of 8-row x 16-byte
// core matrices: element (row, k) of a tile with Kp columns sits at
//   (row/8) * (16 Kp) + (k/8) * 128 + (row%8) * 16 + (k%8) * 2 bytes,
// i.e. leading (K-direction) core stride 128 B, stride (row-direction) core stride 16 Kp B.
// The coefficient matrices are stored in HBM already in this layout (rows rounded up to 8,
// columns to 16, zero padded, hi then lo), so each one is a single 1-D TMA bulk copy
// (cp.async.bulk) into a two-slot ring of KrMax-row slots.  The MMA reads 128 rows from a slot;
// rows at and beyond the cell's Kr are whatever follows in shared memory and only feed
// accumulator rows >= K, which are never stored (E rows >= K are written as zero).
// B = U^{k+1} - U^k (then E^k) is staged by the threads from FP32 state, split into hi/lo.
// The MMA issuer is one thread; TMEM holds m accumulators of NT columns.  Every wait on an
// mbarrier is bounded; on timeout the CTA records an error, drains its own copies (bounded),
// frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>

namespace mss {

struct TcArgs {
  const unsigned char *blob;   // per cell: 2m-1 matrices, each hi (Kr x Kp bf16) then lo, core layout
  const int64_t *blob_off;     // per cell, bytes
  const int32_t *Kp, *Kr;      // columns rounded up to 16, rows rounded up to 8
  int *err;                    // set to 1 by a CTA whose wait timed out
  int slot_bytes;              // one A slot of the fused kernel: hi + lo of KrMax rows x KpMax
  int kpmax, krmax;            // largest K rounded to 16 (columns) and to 8 (rows) over the cells
  int bbuf_bytes;              // one B buffer: hi + lo of NT rows x KpMax
  int max_m;
  int terms;                   // 3: split BF16 (FP32-class products), 1: plain BF16
  unsigned tmem_cols;
  unsigned extra_tx;           // failure-path test hook: bytes a split kernel's matrix barrier waits
                               // for beyond its copies (the wait then runs out)
};

constexpr int kTcThreads = 256;
constexpr int kStageRounds = 4;   // row groups per warp whose staging loads are in flight together
constexpr unsigned long long kWaitNs = 100000000ull;   // 100 ms: a wait longer than this is declared hung

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
// Bounded wait: false after kWaitNs, or (err != nullptr) as soon as any CTA has recorded an error.
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity, const int *err) {
  if (mbar_try_wait(a, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(a, parity)) return true;
    if ((it & 255) == 0) {
      if (err && *(volatile const int *)err) return false;
      if (globaltimer_ns() - t0 > kWaitNs) return false;
    }
    if (it > 32) __nanosleep(64);
  }
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, leading (K) core stride lbo, row core stride sbo
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(unsigned dtmem, uint64_t a, uint64_t b, uint32_t idesc, unsigned accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_ld8(unsigned taddr, float (&v)[8]) {
  unsigned r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ unsigned core_off(int row, int k, int Kp) {
  return (unsigned)((row >> 3) * (16 * Kp) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_store(unsigned char *hi, unsigned char *lo, unsigned off, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  *reinterpret_cast<__nv_bfloat16 *>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat16 *>(lo + off) = l;
}

// BF16 hi/lo split of a pair, packed as two 32-bit words (element 0 in the low half)
__device__ __forceinline__ void split_pack2(float v0, float v1, uint32_t &hw, uint32_t &lw) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
  const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
  const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
  hw = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
  lw = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
}

// Eight consecutive K-direction values (k0..k0+7, k0 % 8 == 0) of B row c, split into hi and lo:
// one 16-byte core-matrix row each.
__device__ __forceinline__ void store_core8(unsigned char *hi, unsigned char *lo, unsigned off, const float (&v)[8]) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_pack2(v[2 * i], v[2 * i + 1], hw[i], lw[i]);
  *reinterpret_cast<uint4 *>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4 *>(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// 8 x 8 transpose across each group of 8 consecutive lanes: on entry v[j] = M[lane % 8][j], on
// return v[j] = M[j][lane % 8].  Three butterfly rounds; every lane of the warp must call it.
__device__ __forceinline__ void transpose8(float (&v)[8], int lane) {
#pragma unroll
  for (int s = 1; s < 8; s <<= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if ((j & s) == 0) {
        const float send = up ? v[j] : v[j + s];
        const float recv = __shfl_xor_sync(0xffffffffu, send, s);
        if (up) v[j] = recv;
        else v[j + s] = recv;
      }
    }
  }
}

// B^k = U^{k+1} - U^k, k = 0..m-1 (U^0 = the cell's face rows, U^m = 0) of one (cell, source
// tile) into the K-major core layout, split hi/lo: buffer k at bb + k * bstride, its lo half
// lo_off bytes after the hi half; rows >= K zero.  Warp wi of nwarps stagers; lanes run over
// sources (coalesced loads), each lane fills one 16-byte core row of 8 k values.  Branch-free:
// every element of a round of kStageRounds row groups is loaded (masked-off ones from a safe
// address, dropped by a select) before any is converted, so the round's loads are in flight
// together.  rows[r] = face row * 2 + side of the cell's boundary row r.
template <int NT>
__device__ __forceinline__ void tc_stage_layers(const float *fs, const float *cs, const int64_t *rows, int64_t so,
                                                int S, int s0, int ns, int K, int Kp, int m, unsigned char *bb,
                                                size_t bstride, size_t lo_off, int wi, int nwarps, int lane) {
  constexpr int CPW = NT < 32 ? NT : 32;        // sources per warp pass
  constexpr int RPW = 32 / CPW;                 // 8-row groups per warp pass
  const int NR8 = Kp / 8, ngp = (NR8 + RPW - 1) / RPW, cblocks = NT / CPW;
  const int cl = lane % CPW, sub = lane / CPW;
  const int passes = m * ngp * cblocks;
  const float *dummy = cs;
  auto load8 = [&](int tt, float (&x0)[8], float (&x1)[8], unsigned &mask, int &kb, int &off) -> bool {
    if (tt >= passes) return false;
    const int cb = tt % cblocks, t2 = tt / cblocks;
    const int gp = t2 % ngp, k = t2 / ngp;
    const int g8 = gp * RPW + sub, c = cb * CPW + cl;
    if (g8 >= NR8) return false;
    const int r0 = g8 * 8;
    mask = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) mask |= (r0 + i < K && c < ns) ? 1u << i : 0u;
    const bool has_hi = k + 1 < m;
    const bool all = mask == 0xFFu;   // whole group inside the block: no address selects
    if (k == 0) {
      if (all) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x0[i] = fs[(rows[r0 + i] >> 1) * S + s0 + c];
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x0[i] = *(((mask >> i) & 1u) ? fs + (rows[r0 + i] >> 1) * S + s0 + c : dummy);
      }
    } else {
      const float *lo = cs + (so + (int64_t)(k - 1) * K + r0) * S + s0 + c;
      if (all) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x0[i] = lo[(int64_t)i * S];
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x0[i] = *(((mask >> i) & 1u) ? lo + (int64_t)i * S : dummy);
      }
    }
    if (has_hi) {
      const float *hi = cs + (so + (int64_t)k * K + r0) * S + s0 + c;
      if (all) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x1[i] = hi[(int64_t)i * S];
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x1[i] = *(((mask >> i) & 1u) ? hi + (int64_t)i * S : dummy);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) x1[i] = 0.f;
      mask |= 1u << 8;   // upper level is zero
    }
    kb = k;
    off = (int)core_off(c, r0, Kp);
    return true;
  };
  for (int t0 = wi; t0 < passes; t0 += kStageRounds * nwarps) {
    float x0[kStageRounds][8], x1[kStageRounds][8];
    unsigned mask[kStageRounds];
    int kb[kStageRounds], off[kStageRounds];
    bool has[kStageRounds];
#pragma unroll
    for (int u = 0; u < kStageRounds; ++u) has[u] = load8(t0 + u * nwarps, x0[u], x1[u], mask[u], kb[u], off[u]);
#pragma unroll
    for (int u = 0; u < kStageRounds; ++u)
      if (has[u]) {
        float v[8];
        const bool zero_hi = (mask[u] >> 8) & 1u;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = ((mask[u] >> i) & 1u) ? (zero_hi ? 0.f : x1[u][i]) - x0[u][i] : 0.f;
        unsigned char *h = bb + (size_t)kb[u] * bstride;
        store_core8(h, h + lo_off, (unsigned)off[u], v);
      }
  }
}

// Hidden-layer leapfrog U^k <- 2 U^k - U^k_old + tau^2 (Gamma-hat^k E^k), k = 2..m, from the
// accumulators of acceleration product k-1 at TMEM columns (k-2) NT.. : accumulator row r (the
// thread's TMEM lane), columns c0 .. c0 + CH - 1 of the tile.  TMEM loads in every lane; up to four
// 8-column chunks per iteration keep their global loads in flight together.
template <int NT, int CH>
__device__ __forceinline__ void tc_leapfrog(unsigned tmem, unsigned lane_addr, const float *cs, float *cso,
                                            int64_t so, int K, int S, int s0, int ns, int m, int r, int c0,
                                            float tau2) {
  constexpr int U = CH >= 32 ? 4 : CH / 8;
  const bool vec_ok = (S % 4) == 0;
  for (int k = 1; k < m; ++k) {
    const int64_t base = (so + (int64_t)(k - 1) * K + r) * S + s0 + c0;
    for (int cb = 0; cb < CH; cb += 8 * U) {
      float acc[U][8];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        __syncwarp();
        tc_ld8(tmem + lane_addr + (unsigned)((k - 1) * NT + c0 + cb + 8 * u), acc[u]);
      }
      if (r >= K) continue;
      const float *nrow = cs + base + cb;
      float *crow = cso + base + cb;
      if (vec_ok && c0 + cb + 8 * U <= ns) {
        float4 nw[U][2], od[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            nw[u][h] = *reinterpret_cast<const float4 *>(nrow + 8 * u + 4 * h);
            od[u][h] = *reinterpret_cast<const float4 *>(crow + 8 * u + 4 * h);
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float4 o = od[u][h];
            const float4 n = nw[u][h];
            o.x = 2.f * n.x - o.x + tau2 * acc[u][4 * h + 0];
            o.y = 2.f * n.y - o.y + tau2 * acc[u][4 * h + 1];
            o.z = 2.f * n.z - o.z + tau2 * acc[u][4 * h + 2];
            o.w = 2.f * n.w - o.w + tau2 * acc[u][4 * h + 3];
            *reinterpret_cast<float4 *>(crow + 8 * u + 4 * h) = o;
          }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (c0 + cb + 8 * u + j < ns) {
              const int e = 8 * u + j;
              crow[e] = 2.f * nrow[e] - crow[e] + tau2 * acc[u][j];
            }
      }
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(kTcThreads, 2) k_cell_tc(const StepArgs<float> a, const TcArgs t, const int cur) {
  const int tiles = (a.S + NT - 1) / NT;           // 1-D grid, tiles of a cell adjacent (L2 reuse)
  const int cell = blockIdx.x / tiles;
  const int s0 = (blockIdx.x % tiles) * NT;
  const int K = a.cell_K[cell], m = a.cell_m[cell];
  const int Kp = t.Kp[cell], Kr = t.Kr[cell];
  const int S = a.S;
  const int ns = min(NT, S - s0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *slot[2] = {smem, smem + t.slot_bytes};
  const unsigned lo_off = (unsigned)t.krmax * t.kpmax * 2;   // lo half of a slot
  unsigned char *bb = smem + 2 * t.slot_bytes;                 // B buffers: max_m x bbuf_bytes
  // rows and barriers sit after a 128-row gap so that no 128-row A read reaches them
  int64_t *rows = reinterpret_cast<int64_t *>(bb + (size_t)t.max_m * t.bbuf_bytes + (size_t)128 * t.kpmax * 2);
  uint64_t *bars = reinterpret_cast<uint64_t *>(rows + 128);   // full0 full1 empty0 empty1 done
  unsigned *tmem_base_sm = reinterpret_cast<unsigned *>(bars + 5);
  int *abort_sm = reinterpret_cast<int *>(tmem_base_sm + 1);
  const unsigned full[2] = {smem_u32(bars + 0), smem_u32(bars + 1)};
  const unsigned empty[2] = {smem_u32(bars + 2), smem_u32(bars + 3)};
  const unsigned done = smem_u32(bars + 4);
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
  const int nmat = 2 * m - 1;
  const unsigned mat_half = (unsigned)Kr * Kp * 2;             // bytes of hi (or lo) of one matrix in HBM
  const unsigned char *cblob = t.blob + t.blob_off[cell];
  const uint32_t idesc = idesc_bf16(128, NT);

  __shared__ int bail;
  if (tid == 0) bail = *(volatile const int *)t.err;
  __syncthreads();
  if (bail) return;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_base_sm)),
                 "r"(t.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(smem_u32(bars + i), 1);
    *abort_sm = 0;
    fence_mbar_init();
  }
  for (int r = tid; r < K; r += kTcThreads) rows[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_base_sm;
  // producer: first two matrices into the ring
  int issued = 0;     // matrices whose copy has been issued (thread 0 only)
  int consumed = 0;   // matrices whose copy has landed and been waited for (thread 0 only)
  auto issue = [&](int p) {
    const int sl = p & 1;
    const unsigned char *src = cblob + (size_t)p * 2 * mat_half;
    mbar_expect_tx(full[sl], 2 * mat_half);
    bulk_g2s(smem_u32(slot[sl]), src, mat_half, full[sl]);
    bulk_g2s(smem_u32(slot[sl] + lo_off), src + mat_half, mat_half, full[sl]);
  };
  if (tid == 0) {
    issue(0);
    issued = 1;
    if (nmat > 1) { issue(1); issued = 2; }
  }
  // stage B^k = U^{k+1} - U^k, k = 0..m-1 (U^0 = faces, U^m = 0)
  tc_stage_layers<NT>(fs, cs, rows, so, S, s0, ns, K, Kp, m, bb, t.bbuf_bytes, (size_t)NT * Kp * 2, warp,
                      kTcThreads / 32, lane);
  fence_async_smem();
  __syncthreads();
  const unsigned lbo = 128, sbo = 16u * Kp;
  const int ksteps = Kp / 16;
  // products p = 0..nmat-1: fluxes (p < m, B = buffer p, D column p*NT), then accelerations
  // (p >= m, B = buffer p-m, D column (p-m)*NT); the B buffers of the second group are written
  // by the first epilogue.
  auto run_products = [&](int p0, int p1) {
    for (int p = p0; p < p1; ++p) {
      const int sl = p & 1;
      const int bi = p < m ? p : p - m;
      if (!mbar_wait(full[sl], (p >> 1) & 1, t.err)) { *abort_sm = 1; break; }
      consumed = p + 1;
      tc_fence_after();
      const unsigned ah = smem_u32(slot[sl]), al = ah + lo_off;
      const unsigned bh = smem_u32(bb + (size_t)bi * t.bbuf_bytes), bl = bh + NT * Kp * 2;
      const unsigned dcol = tmem + (unsigned)(bi * NT);
      for (int kk = 0; kk < ksteps; ++kk) {
        const unsigned o = kk * 256;
        mma_bf16(dcol, sdesc(ah + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, kk > 0 ? 1u : 0u);
        if (t.terms == 3) {
          mma_bf16(dcol, sdesc(ah + o, lbo, sbo), sdesc(bl + o, lbo, sbo), idesc, 1u);
          mma_bf16(dcol, sdesc(al + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, 1u);
        }
      }
      tc_commit(empty[sl]);
      // refill the slot of the previous product (its MMAs were queued before this one's)
      const int q = p - 1;
      if (q >= 0 && q + 2 < nmat && issued == q + 2) {
        if (!mbar_wait(empty[q & 1], (q >> 1) & 1, t.err)) { *abort_sm = 1; break; }
        issue(q + 2);
        issued = q + 3;
      }
    }
    tc_commit(done);
  };
  if (tid == 0) run_products(0, m);
  const int q = warp & 3, half = warp >> 2;
  const int r = 32 * q + lane;                     // accumulator row = TMEM lane
  const unsigned lane_addr = (unsigned)(32 * q) << 16;
  const int c0 = half * (NT / 2);
  bool ok = mbar_wait(done, 0, t.err);
  tc_fence_after();
  // all flux MMAs are complete, so the slot of the last one can take the next matrix now
  if (tid == 0 && ok && !*abort_sm && issued == m + 1 && m + 1 < nmat) {
    issue(m + 1);
    issued = m + 2;
  }
  // epilogue 1: publish F^1; E^k = F^k - F^{k-1} (k = 1..m-1) into B buffer k-1.
  // tcgen05.ld is warp-wide: the decision is made uniform over the CTA first.
  const bool go1 = __syncthreads_and(ok && !*abort_sm) != 0;
  const bool vec_ok = (S % 4) == 0;
  if (go1) {
    for (int cc = 0; cc < NT / 2; cc += 8) {
      float prev[8], curv[8];
      const bool full8 = vec_ok && (c0 + cc + 8 <= ns);
      for (int k = 0; k < m; ++k) {
        tc_ld8(tmem + lane_addr + (unsigned)(k * NT + c0 + cc), curv);
        if (k == 0) {
          if (r < K) {
            float *o = a.flux + rows[r] * S + s0 + c0 + cc;
            if (full8) {
              reinterpret_cast<float4 *>(o)[0] = make_float4(curv[0], curv[1], curv[2], curv[3]);
              reinterpret_cast<float4 *>(o)[1] = make_float4(curv[4], curv[5], curv[6], curv[7]);
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (c0 + cc + j < ns) o[j] = curv[j];
            }
          }
        } else {
          // E^k row r, 8 sources -> transpose in groups of 8 rows -> one core row per source
          float e8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) e8[j] = r < K ? curv[j] - prev[j] : 0.f;
          transpose8(e8, lane);
          const int r0 = r & ~7;
          if (r0 < Kp) {
            unsigned char *h = bb + (size_t)(k - 1) * t.bbuf_bytes;
            store_core8(h, h + NT * Kp * 2, core_off(c0 + cc + (lane & 7), r0, Kp), e8);
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) prev[j] = curv[j];
      }
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!go1 && tid == 0) *abort_sm = 1;
  if (tid == 0 && go1 && m > 1) run_products(m, nmat);
  ok = (go1 && m > 1) ? mbar_wait(done, 1, t.err) : go1;
  tc_fence_after();
  // epilogue 2: hidden-layer leapfrog
  const bool go2 = __syncthreads_and(ok && !*abort_sm) != 0;
  if (go2) {
    tc_leapfrog<NT, NT / 2>(tmem, lane_addr, cs, cso, so, K, S, s0, ns, m, r, c0, a.tau2);
  } else if (tid == 0) {
    *abort_sm = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_sm) {
    atomicExch(t.err, 1);
    // drain this CTA's own copies still in flight (bounded) before the shared memory goes away
    for (int p = consumed; p < issued; ++p) mbar_wait(full[p & 1], (p >> 1) & 1, nullptr);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(t.tmem_cols) : "memory");
  }
}

}  // namespace mss
