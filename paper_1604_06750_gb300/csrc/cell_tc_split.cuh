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

constexpr int kTcsThreads = 256;   // 8 warps: warp w reads TMEM lanes 32 (w % 4).. (accumulator rows),
                                   // columns split in two halves by w / 4

// Shared-memory bytes of one split tensor-core CTA with NT sources and KpMax columns.
__host__ __device__ constexpr size_t tcs_smem_bytes(int NT, int kpmax) {
  return (size_t)2 * 128 * kpmax * 2 + (size_t)2 * NT * kpmax * 2 + 64;
}

// B operand of one split product into the core layout (hi, lo): D^k = U^{k+1} - U^k for the
// flux, E^k = F^k - F^{k-1} for the acceleration; rows >= K zero.  Lanes run over sources
// (coalesced loads); each warp takes kStageRounds 8-row groups per round and issues all their
// loads (two per element, 64 per thread) before any conversion.  rows_sm holds
// the cell's face rows (face row * 2 + side) and is read for the flux of k = 0 only.
template <int NT, bool FLUX>
__device__ __forceinline__ void tcs_stage_b(const StepArgs<float> &a, const float *Fk, const float *fs, const float *cs,
                                            const int64_t *rows_sm, int64_t so, int k, int m, int K, int Kp, int s0,
                                            int ns, unsigned char *Bh, unsigned char *Bl) {
  constexpr int CPW = NT < 32 ? NT : 32;
  constexpr int RPW = 32 / CPW;
  const int S = a.S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int NR8 = Kp / 8, ngp = (NR8 + RPW - 1) / RPW, cblocks = NT / CPW;
  const int cl = lane % CPW, sub = lane / CPW;
  const int passes = ngp * cblocks;
  // Branch-free loads: every element of a round is loaded (masked-off ones from a safe address
  // and dropped by a select) before any is converted, so all the round's loads are in flight.
  const float *dummy = cs;
  auto load8 = [&](int tt, float (&x0)[8], float (&x1)[8], unsigned &mask, int &off) -> bool {
    const int cb = tt % cblocks, gp = tt / cblocks;
    const int g8 = gp * RPW + sub, c = cb * CPW + cl;
    if (tt >= passes || g8 >= NR8) return false;
    const int r0 = g8 * 8;
    mask = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) mask |= (r0 + i < K && c < ns) ? 1u << i : 0u;
    // 8 rows from base with row stride S: unmasked when the whole group is inside the block
    // (the common case, no address selects), else masked elements read the safe address
    const bool all = mask == 0xFFu;
    auto rows8 = [&](float (&x)[8], const float *base) {
      if (all) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = base[(int64_t)i * S];
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = *(((mask >> i) & 1u) ? base + (int64_t)i * S : dummy);
      }
    };
    if (FLUX) {
      // lower level U^k (face rows for k = 0) and upper level U^{k+1} (zero past the last layer);
      // k and the upper layer's presence are uniform over the CTA
      const bool has_hi = k + 1 < m;
      if (k == 0) {
        if (all) {
#pragma unroll
          for (int i = 0; i < 8; ++i) x0[i] = fs[(rows_sm[r0 + i] >> 1) * S + s0 + c];
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            x0[i] = *(((mask >> i) & 1u) ? fs + (rows_sm[r0 + i] >> 1) * S + s0 + c : dummy);
        }
      } else {
        rows8(x0, cs + (so + (int64_t)(k - 1) * K + r0) * S + s0 + c);
      }
      if (has_hi) {
        rows8(x1, cs + (so + (int64_t)k * K + r0) * S + s0 + c);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x1[i] = 0.f;
        mask |= 1u << 8;   // upper level is zero
      }
    } else {
      const float *f1 = Fk + (int64_t)r0 * S + c;
      rows8(x1, f1);
      rows8(x0, f1 - (int64_t)K * S);
    }
    off = (int)core_off(c, r0, Kp);
    return true;
  };
  for (int t0 = warp; t0 < passes; t0 += kStageRounds * nw) {
    float x0[kStageRounds][8], x1[kStageRounds][8];
    unsigned mask[kStageRounds];
    int off[kStageRounds];
    bool has[kStageRounds];
#pragma unroll
    for (int u = 0; u < kStageRounds; ++u) has[u] = load8(t0 + u * nw, x0[u], x1[u], mask[u], off[u]);
#pragma unroll
    for (int u = 0; u < kStageRounds; ++u)
      if (has[u]) {
        float v[8];
        const bool zero_hi = (mask[u] >> 8) & 1u;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = ((mask[u] >> i) & 1u) ? (zero_hi ? 0.f : x1[u][i]) - x0[u][i] : 0.f;
        store_core8(Bh, Bl, (unsigned)off[u], v);
      }
  }
}

// Epilogue of one split product: warp w reads TMEM lanes 32 (w % 4).. for the columns of half
// w / 4; flux -> F scratch rows from f_row (and the face flux buffer for k = 0, rows from
// rows_sm), acceleration -> leapfrog of the hidden layer.  Up to four 8-column chunks per
// iteration keep their global loads in flight together; the row pointers are formed once.
template <int NT, bool FLUX>
__device__ __forceinline__ void tcs_epilogue(const StepArgs<float> &a, const SplitArgs<float> &p, unsigned tmem,
                                             int k, int K, int s0, int ns, int64_t f_row, const int64_t *rows_sm,
                                             int64_t so, const float *cs, float *cso) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, half = warp >> 2;
  const int r = 32 * q + lane;
  const unsigned lane_addr = (unsigned)(32 * q) << 16;
  constexpr int CH = NT / 2;                        // columns per half (8 .. 64)
  const int c0 = half * CH;
  const int S = a.S;
  const bool vec_ok = (S % 4) == 0;
  const float tau2 = a.tau2;
  const bool live = r < K;
  float *orow = nullptr, *frow = nullptr;
  const float *nrow = nullptr;
  float *crow = nullptr;
  if (live) {
    if (FLUX) {
      orow = p.F + (f_row + r) * S + s0;
      if (k == 0) frow = a.flux + rows_sm[r] * S + s0;
    } else {
      const int64_t b = (so + (int64_t)(k - 1) * K + r) * S + s0;
      nrow = cs + b;
      crow = cso + b;
    }
  }
  // U chunks of 8 columns per iteration: their TMEM loads, then all their global loads in flight
  // together, then the arithmetic and the stores
  constexpr int U = CH >= 32 ? 4 : CH / 8;
  for (int cb = 0; cb < CH; cb += 8 * U) {
    float acc[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      __syncwarp();
      tc_ld8(tmem + lane_addr + (unsigned)(c0 + cb + 8 * u), acc[u]);   // every lane loads
    }
    if (!live) continue;
    if (FLUX) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int col = c0 + cb + 8 * u;
        float *o = orow + col;
        float *fo = frow ? frow + col : nullptr;
        if (vec_ok && col + 8 <= ns) {
          const float4 v0 = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
          const float4 v1 = make_float4(acc[u][4], acc[u][5], acc[u][6], acc[u][7]);
          reinterpret_cast<float4 *>(o)[0] = v0;
          reinterpret_cast<float4 *>(o)[1] = v1;
          if (fo) {
            reinterpret_cast<float4 *>(fo)[0] = v0;
            reinterpret_cast<float4 *>(fo)[1] = v1;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (col + e < ns) {
              o[e] = acc[u][e];
              if (fo) fo[e] = acc[u][e];
            }
        }
      }
    } else {
      const int cc = c0 + cb;
      if (vec_ok && cc + 8 * U <= ns) {
        float4 nw[U][2], od[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            nw[u][h] = *reinterpret_cast<const float4 *>(nrow + cc + 8 * u + 4 * h);
            od[u][h] = *reinterpret_cast<const float4 *>(crow + cc + 8 * u + 4 * h);
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
            *reinterpret_cast<float4 *>(crow + cc + 8 * u + 4 * h) = o;
          }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int col = cc + 8 * u + e;
            if (col < ns) crow[col] = 2.f * nrow[col] - crow[col] + tau2 * acc[u][e];
          }
      }
    }
  }
}

// Epilogue through shared memory (k_tc_split, whose A and B buffers are free once its products
// are done): the accumulator tile (K rows, NT sources) goes TMEM -> tile (row pitch NT + 4
// floats: conflict-free 16-byte stores from lanes over rows), then the global traffic runs with
// lanes over sources, coalesced along each row and four 16-byte vectors per thread in flight:
// flux -> F scratch rows (and the face flux buffer for k = 0), acceleration -> leapfrog of the
// hidden layer.  Same per-element arithmetic as tcs_epilogue.
template <int NT, bool FLUX>
__device__ __forceinline__ void tcs_epilogue_staged(const StepArgs<float> &a, const SplitArgs<float> &p,
                                                    unsigned tmem, int k, int K, int s0, int ns, int64_t f_row,
                                                    const int64_t *rows_sm, int64_t so, const float *cs, float *cso,
                                                    float *tile) {
  constexpr int LD = NT + 4;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, half = warp >> 2;
  const int r = 32 * q + lane;
  const unsigned lane_addr = (unsigned)(32 * q) << 16;
  constexpr int CH = NT / 2;
  const int c0 = half * CH;
  constexpr int U = CH >= 32 ? 4 : CH / 8;
  fence_async_smem();   // the tile overwrites operands the tensor cores have finished reading
  for (int cb = 0; cb < CH; cb += 8 * U) {
    float acc[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      __syncwarp();
      tc_ld8(tmem + lane_addr + (unsigned)(c0 + cb + 8 * u), acc[u]);
    }
    if (r < K) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float4 *d = reinterpret_cast<float4 *>(tile + r * LD + c0 + cb + 8 * u);
        d[0] = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
        d[1] = make_float4(acc[u][4], acc[u][5], acc[u][6], acc[u][7]);
      }
    }
  }
  __syncthreads();
  const int S = a.S;
  const float tau2 = a.tau2;
  if ((S % 4) == 0 && ns == NT) {
    constexpr int VR = NT / 4;   // 16-byte vectors per row
    constexpr int B4 = 4;        // vectors per thread in flight
    const int total = K * VR;
    for (int i0 = tid; i0 < total; i0 += B4 * kTcsThreads) {
      if (FLUX) {
#pragma unroll
        for (int b = 0; b < B4; ++b) {
          const int i = i0 + b * kTcsThreads;
          if (i < total) {
            const int rr = i / VR, v = i - rr * VR;
            const float4 x = reinterpret_cast<const float4 *>(tile + rr * LD)[v];
            reinterpret_cast<float4 *>(p.F + (f_row + rr) * S + s0)[v] = x;
            if (k == 0) reinterpret_cast<float4 *>(a.flux + rows_sm[rr] * S + s0)[v] = x;
          }
        }
      } else {
        float4 nw[B4], od[B4];
        int64_t at[B4];
#pragma unroll
        for (int b = 0; b < B4; ++b) {
          const int i = i0 + b * kTcsThreads;
          const bool ok = i < total;
          const int rr = ok ? i / VR : 0, v = i - rr * VR;
          at[b] = ok ? (so + (int64_t)(k - 1) * K + rr) * S + s0 + 4 * v : -1;
          nw[b] = *reinterpret_cast<const float4 *>(ok ? cs + at[b] : cs);
          od[b] = *reinterpret_cast<const float4 *>(ok ? cso + at[b] : cso);
        }
#pragma unroll
        for (int b = 0; b < B4; ++b) {
          const int i = i0 + b * kTcsThreads;
          if (at[b] < 0) continue;
          const int rr = i / VR, v = i - rr * VR;
          const float4 x = reinterpret_cast<const float4 *>(tile + rr * LD)[v];
          float4 o = od[b];
          const float4 n = nw[b];
          o.x = 2.f * n.x - o.x + tau2 * x.x;
          o.y = 2.f * n.y - o.y + tau2 * x.y;
          o.z = 2.f * n.z - o.z + tau2 * x.z;
          o.w = 2.f * n.w - o.w + tau2 * x.w;
          *reinterpret_cast<float4 *>(cso + at[b]) = o;
        }
      }
    }
  } else {
    // ragged source tile or rows not 16-byte aligned: one element per thread and step
    for (int i = tid; i < K * NT; i += kTcsThreads) {
      const int rr = i / NT, c = i - rr * NT;
      if (c >= ns) continue;
      const float x = tile[rr * LD + c];
      if (FLUX) {
        p.F[(f_row + rr) * S + s0 + c] = x;
        if (k == 0) a.flux[rows_sm[rr] * S + s0 + c] = x;
      } else {
        const int64_t at = (so + (int64_t)(k - 1) * K + rr) * S + s0 + c;
        cso[at] = 2.f * cs[at] - cso[at] + tau2 * x;
      }
    }
  }
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
  const int tid = threadIdx.x, warp = tid >> 5;
  extern __shared__ __align__(128) unsigned char smem[];
  // layout: A hi (128 x KpMax), A lo, B hi (NT x KpMax), B lo, then barriers; the A halves and
  // the B halves are KpMax-strided so that one allocation serves every cell
  const int kpmax = t.kpmax;
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
  __shared__ int64_t rows_sm[128];                   // face rows of the cell (flux of k = 0)
  if (tid == 0) bail = *(volatile const int *)t.err;
  if (FLUX && k == 0)
    for (int r = tid; r < K; r += kTcsThreads) rows_sm[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
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
    mbar_expect_tx(full, 2 * mat_half + t.extra_tx);
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
  const int64_t f_row = p.f_off[cell] + (int64_t)k * K;
  const float *Fk = p.F + f_row * S + s0;
  tcs_stage_b<NT, FLUX>(a, Fk, fs, cs, rows_sm, so, k, m, K, Kp, s0, ns, Bh, Bl);
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
    tcs_epilogue_staged<NT, FLUX>(a, p, tmem, k, K, s0, ns, f_row, rows_sm, so, cs, cso,
                                  reinterpret_cast<float *>(smem));
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

namespace mss {

// Shared memory of the pipelined split kernel: barriers, two A slots of Kr_max rows (hi, lo),
// one B buffer (hi, lo) and a tail so that the 128-row A reads of the last slot stay inside the
// allocation (rows >= Kr of a product only feed accumulator rows that are never stored).
__host__ __device__ constexpr size_t tcp_smem_bytes(int NT, int kpmax, int krmax) {
  return 64 + (size_t)4 * krmax * kpmax * 2 + (size_t)2 * NT * kpmax * 2 + (size_t)(128 - krmax) * kpmax * 2 + 64;
}

// Pipelined form of k_tc_split: a resident grid loops over the (item, tile) list; while item j is
// staged, multiplied and written back, the bulk copy of item j+1's matrix is already in flight
// into the other A slot.  Same products and epilogues as k_tc_split (bit-identical).
template <int NT, bool FLUX>
__global__ void __launch_bounds__(kTcsThreads, 1) k_tc_pipe(const StepArgs<float> a, const SplitArgs<float> p,
                                                            const TcArgs t, const int cur, const int n_items,
                                                            const int krmax) {
  const int tiles = (a.S + NT - 1) / NT;
  const int total = n_items * tiles;
  const int S = a.S;
  const int tid = threadIdx.x, warp = tid >> 5;
  extern __shared__ __align__(128) unsigned char smem[];
  const int kpmax = t.kpmax;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);    // full0, full1, done
  unsigned *tmem_sm = reinterpret_cast<unsigned *>(bars + 3);
  const size_t half = (size_t)krmax * kpmax * 2;
  unsigned char *A0 = smem + 64;                             // slot s: hi at A0 + 2s half, lo after it
  unsigned char *Bh = A0 + 4 * half, *Bl = Bh + (size_t)NT * kpmax * 2;
  const unsigned full[2] = {smem_u32(bars + 0), smem_u32(bars + 1)};
  const unsigned done = smem_u32(bars + 2);
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  unsigned cols = 32;
  while (cols < (unsigned)NT) cols <<= 1;

  __shared__ int bail, ok_sm;
  __shared__ int64_t rows_sm[128];                   // face rows of the item's cell (flux of k = 0)
  if (tid == 0) bail = *(volatile const int *)t.err;
  __syncthreads();
  if (bail || (int)blockIdx.x >= total) return;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_sm)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(full[0], 1);
    mbar_init(full[1], 1);
    mbar_init(done, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_sm;
  // thread 0 bookkeeping: copies issued / waited for, products committed / waited for
  int n_issued = 0, n_landed = 0, n_committed = 0, n_done = 0;
  auto issue_A = [&](int it, int slot) {
    const int2 itm = FLUX ? p.flux_items[it / tiles] : p.accel_items[it / tiles];
    const int c = itm.x, mm = a.cell_m[c];
    const int mat = FLUX ? itm.y : mm + itm.y - 1;
    const unsigned mh = (unsigned)t.Kr[c] * t.Kp[c] * 2;
    const unsigned char *src = t.blob + t.blob_off[c] + (size_t)mat * 2 * mh;
    unsigned char *dst = A0 + (size_t)2 * slot * half;
    mbar_expect_tx(full[slot], t.terms == 3 ? 2 * mh : mh);
    bulk_g2s(smem_u32(dst), src, mh, full[slot]);
    if (t.terms == 3) bulk_g2s(smem_u32(dst + half), src + mh, mh, full[slot]);
    ++n_issued;
  };
  if (tid == 0) issue_A(blockIdx.x, 0);
  bool ok = true;
  int j = 0;
  for (int it = blockIdx.x; it < total; it += gridDim.x, ++j) {
    const int slot = j & 1;
    if (tid == 0 && it + (int)gridDim.x < total) issue_A(it + gridDim.x, slot ^ 1);
    const int2 itm = FLUX ? p.flux_items[it / tiles] : p.accel_items[it / tiles];
    const int cell = itm.x, k = itm.y;
    const int s0 = (it % tiles) * NT;
    const int K = a.cell_K[cell], m = a.cell_m[cell], Kp = t.Kp[cell];
    const int ns = min(NT, S - s0);
    const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
    const int64_t f_row = p.f_off[cell] + (int64_t)k * K;
    const float *Fk = p.F + f_row * S + s0;
    if (FLUX && k == 0) {   // uniform over the CTA; the previous item's epilogue has synchronised
      for (int r = tid; r < K; r += kTcsThreads) rows_sm[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
      __syncthreads();
    }
    tcs_stage_b<NT, FLUX>(a, Fk, fs, cs, rows_sm, so, k, m, K, Kp, s0, ns, Bh, Bl);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      int good = mbar_wait(full[slot], (j >> 1) & 1, t.err) ? 1 : 0;
      if (good) {
        ++n_landed;
        tc_fence_after();
        const uint32_t idesc = idesc_bf16(128, NT);
        const unsigned lbo = 128, sbo = 16u * Kp;
        const unsigned ah = smem_u32(A0 + (size_t)2 * slot * half), al = ah + (unsigned)half;
        const unsigned bh = smem_u32(Bh), bl = smem_u32(Bl);
        for (int kk = 0; kk < Kp / 16; ++kk) {
          const unsigned o = kk * 256;
          mma_bf16(tmem, sdesc(ah + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, kk > 0 ? 1u : 0u);
          if (t.terms == 3) {
            mma_bf16(tmem, sdesc(ah + o, lbo, sbo), sdesc(bl + o, lbo, sbo), idesc, 1u);
            mma_bf16(tmem, sdesc(al + o, lbo, sbo), sdesc(bh + o, lbo, sbo), idesc, 1u);
          }
        }
        tc_commit(done);
        ++n_committed;
        good = mbar_wait(done, j & 1, t.err) ? 1 : 0;
        if (good) ++n_done;
      }
      ok_sm = good;
    }
    __syncthreads();
    if (!ok_sm) {
      ok = false;
      break;
    }
    tc_fence_after();
    tcs_epilogue<NT, FLUX>(a, p, tmem, k, K, s0, ns, f_row, rows_sm, so, cs, cso);
    tc_fence_before();
    __syncthreads();   // TMEM, the B buffer and this item's A slot are free again
  }
  if (!ok && tid == 0) {
    atomicExch(t.err, 1);
    // wait (bounded) for this CTA's copies and products still in flight
    for (int c = n_landed; c < n_issued; ++c) mbar_wait(full[c & 1], (c >> 1) & 1, nullptr);
    if (n_committed > n_done) mbar_wait(done, (n_committed - 1) & 1, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
  }
}

}  // namespace mss
