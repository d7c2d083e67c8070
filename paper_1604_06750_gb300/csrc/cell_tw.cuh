// Wide tensor-core cell kernel: the cell phase for K_i up to 384 on the 5th-generation tensor
// cores with FP32-class products (sm_103a).
//
// Per (cell, 16-source tile) one CTA computes what the factored FP32 cell kernels compute,
//   F^k = Gamma^k D^k (k < m),  y = L^T D^m,  F^m = L y,  publish F^1,  E^k = F^k - F^{k-1},
//   U^k <- 2 U^k - U^k_old + tau^2 Gamma-hat^k E^k  (k = 2..m)                  (Eq. intrtstep_td)
// with D^k = U^{k+1} - U^k and Gamma^m = L L^T (the floored Cholesky factor of the semidefinite
// last coefficient), every product on tcgen05.mma kind::tf32: M = 128 coefficient rows, N = 16
// sources, 8 k per instruction, FP32 accumulators in TMEM.  TF32 keeps 10 explicit mantissa bits,
// so both operands are split, x = hi + lo, hi = x with its low 13 mantissa bits cleared and lo =
// (x - hi) cleared the same way, and every product is A_hi B_hi + A_hi B_lo + A_lo B_hi: each term
// then carries about 21 bits, against FP32's 24, and the dropped A_lo B_lo is below both.  The
// coefficient's hi part is the landed FP32 block itself: the tensor core reads a TF32 operand from
// a 32-bit container and ignores its low 13 bits, which is the same truncation (the parity tests
// against the FP64 oracle would fail by orders of magnitude otherwise: a coefficient rounded to TF32
// without its lo part makes the stepping unstable).
//
// The coefficients stream from HBM as FP32 (the algorithm's own bytes), in 128-row x 32-column
// blocks, each stored in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
// matrix: element (row, k) at (row/8) (32 kc) + (k/4) 128 + (row%8) 16 + (k%4) 4 bytes, kc the
// block's columns) and all of a cell's blocks laid out in the order they are consumed, so the
// producer walks the cell's blob front to back with one 1-D bulk copy (cp.async.bulk) per block.
// Only the rows of the cell are stored (the last M tile is short) and, for the two triangular
// products, only blocks that meet the triangle (with the other triangle stored as zeros).
//
// Warp roles (320 threads), around a ring of slots (a 16 KB block and its 16 KB lo part each):
//   warp 0     producer: one bulk copy per block into the next free slot (mbarrier with
//              transaction count);
//   warps 2-5  converters: the lo part of a landed block (rows past the block zero);
//   warp 1     one thread issues the block's MMAs and commits them to the slot's barrier, which
//              frees the slot for the producer, and commits each product to a B-buffer barrier;
//   warps 6-9  epilogue (warp w reads TMEM lanes 32 (w % 4) ..): stage each product's B operand
//              (D^k from the state, y and E^k from TMEM) into a double buffer, publish F^1, and
//              apply the hidden-layer leapfrog once the last product is complete.
// Every wait is bounded (globaltimer) and stops on the error word; on error the CTA records it,
// lets its copies and products in flight finish (bounded), frees its TMEM and returns.
#pragma once

namespace mss {

constexpr int kTwMaxK = 384;                 // three M tiles of 128 rows
constexpr int kTwNT = 16;                    // sources per CTA (MMA N)
constexpr int kTwThreads = 320;
constexpr int kTwBlock = 128 * 32 * 4;       // bytes of one FP32 A block (128 rows x 32 k)
constexpr int kTwMaxRing = 6;                // 3 x 6 + 5 barriers stay below the control words at byte 240

struct TwArgs {
  const float *blob;          // per cell: the A blocks of every product, in consumption order
  const int64_t *blob_off;    // per cell, in floats
  int *err;                   // error word of the bounded waits
  int ring;                   // 16 KB slots of the copy ring
  int k8max;                  // largest K rounded up to 8 (B operand extent)
  unsigned tmem_cols;
  unsigned extra_tx;          // failure-path test hook: bytes a slot's barrier waits for beyond its copy
};

__host__ __device__ inline int tw_mt(int K) { return (K + 127) / 128; }

// k chunks [c0, c1) of product j (0..2m-1), M tile t: all chunks, except for y = L^T D^m (j = m-1:
// chunks reaching the diagonal or right of it) and F^m = L y (j = m: chunks reaching the diagonal
// or left of it).
__host__ __device__ inline void tw_chunks(int j, int t, int m, int K, int &c0, int &c1) {
  const int K8 = (K + 7) & ~7;
  const int nch = (K8 + 31) / 32;
  c0 = 0;
  c1 = nch;
  if (j == m - 1) c0 = 4 * t;
  if (j == m) c1 = (((128 * t + 127) < (K - 1) ? (128 * t + 127) : (K - 1)) >> 5) + 1;
}

// Bytes of shared memory: barriers and control words, the ring (block and lo part per slot), the
// double-buffered B operand (hi, lo of 16 x K8 each), the K boundary-row indices.
inline size_t tw_smem_bytes(int ring, int k8max) {
  return 256 + (size_t)ring * 2 * kTwBlock + (size_t)4 * kTwNT * k8max * 4 + 8 * (size_t)k8max;
}

// instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(unsigned dtmem, uint64_t a, uint64_t b, uint32_t idesc, unsigned accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}

// TF32 split: hi keeps the sign, exponent and 10 leading mantissa bits of x; lo the same of x - hi
// (exact in FP32, since x and hi agree in all but the low 13 bits)
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = __uint_as_float(__float_as_uint(x - hi) & 0xFFFFE000u);
}

// 4 x 4 transpose across each group of 4 consecutive lanes: on entry a[j] = M[lane % 4][j], on
// return a[j] = M[j][lane % 4].  Every lane of the warp must call it.
__device__ __forceinline__ void transpose4(float (&a)[4], int lane) {
#pragma unroll
  for (int s = 1; s < 4; s <<= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((j & s) == 0) {
        const float send = up ? a[j] : a[j + s];
        const float recv = __shfl_xor_sync(0xffffffffu, send, s);
        if (up) a[j] = recv;
        else a[j + s] = recv;
      }
    }
  }
}

// B operand row k = r (this thread's row) for sources 0..15, split into the hi and lo buffers of
// the core layout (source n, k) at (n/8) sbo + (k/4) 128 + (n%8) 16 + (k%4) 4.  Lanes 4g..4g+3 hold
// rows 4g..4g+3 (r is 4-aligned per lane quad), so after a 4 x 4 transpose per source quad each
// lane writes one 16-byte core row per buffer.  store: rows inside the buffer (quad-uniform).
__device__ __forceinline__ void tw_store_b(unsigned char *bh, unsigned char *bl, int r, const float (&v)[16],
                                           unsigned sbo, int lane, bool store) {
#pragma unroll
  for (int nb = 0; nb < 4; ++nb) {
    float q[4] = {v[4 * nb], v[4 * nb + 1], v[4 * nb + 2], v[4 * nb + 3]};
    transpose4(q, lane);
    if (store) {
      const int n = 4 * nb + (lane & 3);
      const unsigned off = (unsigned)(n >> 3) * sbo + (unsigned)(r >> 2) * 128u + (unsigned)(n & 7) * 16u;
      float h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) tf32_split(q[i], h[i], l[i]);
      *reinterpret_cast<float4 *>(bh + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4 *>(bl + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// 16 accumulator columns (the 16 sources) of TMEM lane quarter `lane_addr` at column col
__device__ __forceinline__ void tw_ld16(unsigned taddr, float (&v)[16]) {
  float a[8], b[8];
  tc_ld8(taddr, a);
  tc_ld8(taddr + 8, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = a[i];
    v[8 + i] = b[i];
  }
}

// The cell's A blocks in consumption order: product j, then k chunk c, then the M tiles t whose
// chunk range holds c, so consecutive blocks feed different accumulators.
struct TwIter {
  int m, K, K8, MT, NP, nch;
  int j, c, t, cfirst;   // cfirst: first chunk of (j, t), whose first MMA starts the accumulator
  int64_t off;           // bytes from the start of the cell's blob
  __device__ void begin(int m_, int K_) {
    m = m_;
    K = K_;
    K8 = (K + 7) & ~7;
    MT = tw_mt(K);
    NP = 2 * m;
    nch = (K8 + 31) / 32;
    j = 0;
    c = 0;
    t = -1;
    off = 0;
    advance();
  }
  // the next (j, c, t) whose chunk range holds c; every (j, c) has one (tile 0 for j != m, the last
  // tile for j = m)
  __device__ void advance() {
    for (;;) {
      if (++t >= MT) {
        t = 0;
        if (++c >= nch) {
          c = 0;
          if (++j >= NP) return;
        }
      }
      int a, b;
      tw_chunks(j, t, m, K, a, b);
      if (c >= a && c < b) {
        cfirst = a;
        return;
      }
    }
  }
  __device__ bool valid() const { return j < NP; }
  __device__ int rows() const { return min(128, K8 - 128 * t); }
  __device__ int kc() const { return min(32, K8 - 32 * c); }
  __device__ unsigned bytes() const { return (unsigned)(rows() * kc() * 4); }
  __device__ void next() {
    off += bytes();
    advance();
  }
};

__global__ void __launch_bounds__(kTwThreads, 1) k_cell_tw(const StepArgs<float> a, const TwArgs t, const int cur) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tiles = (a.S + kTwNT - 1) / kTwNT;   // 1-D grid, tiles of a cell adjacent
  const int cell = blockIdx.x / tiles;
  const int s0 = (blockIdx.x % tiles) * kTwNT;
  const int K = a.cell_K[cell], m = a.cell_m[cell], S = a.S;
  const int K8 = (K + 7) & ~7, MT = tw_mt(K), NP = 2 * m;
  const int ns = min(kTwNT, S - s0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = t.ring;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  // barriers: copy landed[R], lo part ready[R], slot free[R] (MMAs done), B ready[2], B free[2], done
  const int TF = 0, SF = R, SE = 2 * R, BR = 3 * R, BF = 3 * R + 2, DN = 3 * R + 4;
  auto bar = [&](int i) { return smem_u32(bars + i); };
  volatile int *ctl = reinterpret_cast<volatile int *>(smem + 240);   // [0] TMEM base, [1] abort, [2] copies issued
  unsigned char *ring = smem + 256;
  unsigned char *bbuf = ring + (size_t)R * 2 * kTwBlock;              // hi0 lo0 hi1 lo1
  const size_t bhalf = (size_t)kTwNT * t.k8max * 4;
  int64_t *rows = reinterpret_cast<int64_t *>(bbuf + 4 * bhalf);
  const float *fs = cur ? a.fstate1 : a.fstate0;
  const float *cs = cur ? a.cstate1 : a.cstate0;
  float *cso = cur ? a.cstate0 : a.cstate1;
  const int64_t rp = a.cell_row[cell], so = a.cell_state[cell];
  const unsigned sbo_b = (unsigned)K8 * 32u;

  __shared__ int bail;
  if (tid == 0) bail = *(volatile const int *)t.err;
  __syncthreads();
  if (bail) return;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32((void *)ctl)),
                 "r"(t.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < R; ++i) {
      mbar_init(bar(TF + i), 1);
      mbar_init(bar(SF + i), 128);
      mbar_init(bar(SE + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(BR + i), 128);
      mbar_init(bar(BF + i), 1);
    }
    mbar_init(bar(DN), 1);
    ctl[1] = 0;
    ctl[2] = 0;
    fence_mbar_init();
  }
  for (int r = tid; r < K; r += kTwThreads) rows[r] = a.row_face_row[rp + r] * 2 + a.row_side[rp + r];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = (unsigned)ctl[0];
  auto fail = [&]() {
    ctl[1] = 1;
    atomicExch(t.err, 1);
  };

  if (warp == 0) {
    // ---- producer
    if (lane == 0) {
      const unsigned char *src = reinterpret_cast<const unsigned char *>(t.blob + t.blob_off[cell]);
      TwIter it;
      it.begin(m, K);
      for (int b = 0; it.valid(); it.next(), ++b) {
        const int s = b % R;
        if (b >= R && !mbar_wait(bar(SE + s), ((b / R) - 1) & 1, t.err)) { fail(); break; }
        if (ctl[1]) break;
        const unsigned bytes = it.bytes();
        mbar_expect_tx(bar(TF + s), bytes + t.extra_tx);
        bulk_g2s(smem_u32(ring + (size_t)s * 2 * kTwBlock), src + it.off, bytes, bar(TF + s));
        ctl[2] = b + 1;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, kTwNT);
      TwIter it;
      it.begin(m, K);
      int b = 0;
      bool ok = true;
      while (ok && it.valid()) {
        const int j = it.j;
        if (!mbar_wait(bar(BR + (j & 1)), (j >> 1) & 1, t.err)) { ok = false; break; }
        tc_fence_after();
        const unsigned bh = smem_u32(bbuf + (size_t)(j & 1) * 2 * bhalf), bl = bh + (unsigned)bhalf;
        while (it.valid() && it.j == j) {
          const int s = b % R;
          if (!mbar_wait(bar(SF + s), (b / R) & 1, t.err)) { ok = false; break; }
          tc_fence_after();
          const unsigned ah = smem_u32(ring + (size_t)s * 2 * kTwBlock);
          const int kc = it.kc();
          const unsigned sbo_a = (unsigned)kc * 32u;
          const unsigned dcol = tmem + (unsigned)((j * MT + it.t) * kTwNT);
          // descriptors of the block's first k step; each further step of 8 k advances both operands
          // by two core matrices (256 bytes, 16 in the descriptor's address field, which cannot carry
          // out: shared addresses stay below 256 KB)
          const uint64_t dah = sdesc(ah, 128, sbo_a), dal = sdesc(ah + kTwBlock, 128, sbo_a);
          const uint64_t dbh = sdesc(bh + (unsigned)it.c * 1024u, 128, sbo_b);
          const uint64_t dbl = sdesc(bl + (unsigned)it.c * 1024u, 128, sbo_b);
          const unsigned acc0 = it.c == it.cfirst ? 0u : 1u;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            if (kk * 8 < kc) {
              const uint64_t o = (uint64_t)(16 * kk);
              mma_tf32(dcol, dah + o, dbh + o, idesc, kk == 0 ? acc0 : 1u);
              mma_tf32(dcol, dah + o, dbl + o, idesc, 1u);
              mma_tf32(dcol, dal + o, dbh + o, idesc, 1u);
            }
          }
          tc_commit(bar(SE + s));
          it.next();
          ++b;
        }
        if (!ok) break;
        tc_commit(bar(BF + (j & 1)));
      }
      if (!ok) fail();
      tc_commit(bar(DN));   // arrives once every MMA issued above has completed
    }
  } else if (warp < 6) {
    // ---- converters: lo part of each landed FP32 block, 128 rows (the block's own rows as the MMA
    // reads them; rows past a short block read stale values there, which reach only accumulator
    // rows past the cell, never stored, so their lo part is simply zero)
    const int ct = tid - 64;
    TwIter it;
    it.begin(m, K);
    for (int b = 0; it.valid(); it.next(), ++b) {
      const int s = b % R;
      const bool ok = mbar_wait(bar(TF + s), (b / R) & 1, t.err);
      if (!ok || ctl[1]) {
        if (!ok) fail();
        break;
      }
      const unsigned real = it.bytes(), full = 128u * (unsigned)it.kc() * 4u;
      const unsigned char *src = ring + (size_t)s * 2 * kTwBlock;
      unsigned char *dl = ring + (size_t)s * 2 * kTwBlock + kTwBlock;
      // four 16-byte pieces per thread per round, their loads issued together
      for (unsigned o0 = (unsigned)ct * 16u; o0 < full; o0 += 4u * 128u * 16u) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned o = o0 + (unsigned)u * 128u * 16u;
          v[u] = o < real ? *reinterpret_cast<const float4 *>(src + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned o = o0 + (unsigned)u * 128u * 16u;
          float4 h, l;
          tf32_split(v[u].x, h.x, l.x);
          tf32_split(v[u].y, h.y, l.y);
          tf32_split(v[u].z, h.z, l.z);
          tf32_split(v[u].w, h.w, l.w);
          if (o < full) *reinterpret_cast<float4 *>(dl + o) = l;
        }
      }
      fence_async_smem();
      mbar_arrive(bar(SF + s));
    }
  } else {
    // ---- epilogue: B operands, F^1, leapfrog
    const int q = warp & 3;
    const int rl = 32 * q + lane;                          // accumulator row in an M tile = TMEM lane
    const unsigned lane_addr = (unsigned)(32 * q) << 16;
    const bool vec = ns == kTwNT && (S % 4) == 0;
    auto acc16 = [&](int j, int tt, float (&v)[16]) { tw_ld16(tmem + lane_addr + (unsigned)((j * MT + tt) * kTwNT), v); };
    // U^k row r (paper layer k = 1..m+1; U^1 the cell's face rows, U^{m+1} = 0), sources 0..15
    auto load_u = [&](int k, int r, float (&u)[16]) {
#pragma unroll
      for (int n = 0; n < 16; ++n) u[n] = 0.f;
      if (k > m || r >= K) return;
      const float *p = k == 1 ? fs + (rows[r] >> 1) * S + s0 : cs + (so + (int64_t)(k - 2) * K + r) * S + s0;
      if (vec) {
#pragma unroll
        for (int v4 = 0; v4 < 4; ++v4) {
          const float4 x = *reinterpret_cast<const float4 *>(p + 4 * v4);
          u[4 * v4] = x.x;
          u[4 * v4 + 1] = x.y;
          u[4 * v4 + 2] = x.z;
          u[4 * v4 + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int n = 0; n < 16; ++n)
          if (n < ns) u[n] = p[n];
      }
    };
    // B operand of product j into buffer j % 2
    auto stage_b = [&](int j) {
      unsigned char *bh = bbuf + (size_t)(j & 1) * 2 * bhalf, *bl = bh + bhalf;
      for (int tt = 0; tt < MT; ++tt) {
        const int r = 128 * tt + rl;
        float v[16];
        if (j < m) {
          // D^{j+1} = U^{j+2} - U^{j+1}
          float u0[16], u1[16];
          load_u(j + 1, r, u0);
          load_u(j + 2, r, u1);
#pragma unroll
          for (int n = 0; n < 16; ++n) v[n] = u1[n] - u0[n];
        } else if (j == m) {
          acc16(m - 1, tt, v);                             // y = L^T D^m
        } else {
          // E^k = F^k - F^{k-1}, k = j - m + 1 (F^k in product k-1, F^m in product m)
          const int k = j - m + 1;
          float f0[16];
          acc16(k == m ? m : k - 1, tt, v);
          acc16(k - 2, tt, f0);
#pragma unroll
          for (int n = 0; n < 16; ++n) v[n] -= f0[n];
        }
        if (r >= K) {
#pragma unroll
          for (int n = 0; n < 16; ++n) v[n] = 0.f;
        }
        tw_store_b(bh, bl, r, v, sbo_b, lane, r < K8);
      }
    };
    auto publish_f1 = [&](int j) {
      for (int tt = 0; tt < MT; ++tt) {
        const int r = 128 * tt + rl;
        float v[16];
        acc16(j, tt, v);
        if (r >= K) continue;
        float *o = a.flux + rows[r] * S + s0;
        if (vec) {
#pragma unroll
          for (int v4 = 0; v4 < 4; ++v4)
            reinterpret_cast<float4 *>(o)[v4] = make_float4(v[4 * v4], v[4 * v4 + 1], v[4 * v4 + 2], v[4 * v4 + 3]);
        } else {
#pragma unroll
          for (int n = 0; n < 16; ++n)
            if (n < ns) o[n] = v[n];
        }
      }
    };
    bool ok = true;
    for (int j = 0; j < NP; ++j) {
      // buffer j % 2 is free once product j-2 has completed; y (j = m) and E^2 (j = m+1) also need
      // product j-1 (L^T D^m, resp. F^m)
      if (j >= 2) ok = mbar_wait(bar(BF + (j & 1)), ((j - 2) >> 1) & 1, t.err);
      if (ok && (j == m || j == m + 1) && j >= 1) ok = mbar_wait(bar(BF + ((j - 1) & 1)), ((j - 1) >> 1) & 1, t.err);
      ok = __all_sync(0xffffffffu, ok) && !ctl[1];
      if (!ok) break;
      tc_fence_after();
      stage_b(j);
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(bar(BR + (j & 1)));
      if (j == 2) publish_f1(0);                           // product 0 (F^1) completed before j = 2
    }
    if (ok) ok = __all_sync(0xffffffffu, mbar_wait(bar(BF + ((NP - 1) & 1)), ((NP - 1) >> 1) & 1, t.err));
    if (ok && !ctl[1]) {
      tc_fence_after();
      if (m == 1) publish_f1(1);                           // F^1 = L y
      const float tau2 = a.tau2;
      for (int k = 2; k <= m; ++k) {
        const int j = m + k - 1;
        for (int tt = 0; tt < MT; ++tt) {
          const int r = 128 * tt + rl;
          float v[16];
          acc16(j, tt, v);
          if (r >= K) continue;
          const int64_t base = (so + (int64_t)(k - 2) * K + r) * S + s0;
          if (vec) {
#pragma unroll
            for (int v4 = 0; v4 < 4; ++v4) {
              const float4 nw = *reinterpret_cast<const float4 *>(cs + base + 4 * v4);
              float4 od = *reinterpret_cast<const float4 *>(cso + base + 4 * v4);
              od.x = 2.f * nw.x - od.x + tau2 * v[4 * v4 + 0];
              od.y = 2.f * nw.y - od.y + tau2 * v[4 * v4 + 1];
              od.z = 2.f * nw.z - od.z + tau2 * v[4 * v4 + 2];
              od.w = 2.f * nw.w - od.w + tau2 * v[4 * v4 + 3];
              *reinterpret_cast<float4 *>(cso + base + 4 * v4) = od;
            }
          } else {
#pragma unroll
            for (int n = 0; n < 16; ++n)
              if (n < ns) cso[base + n] = 2.f * cs[base + n] - cso[base + n] + tau2 * v[n];
          }
        }
      }
    } else if (lane == 0) {
      fail();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 32) mbar_wait(bar(DN), 0, nullptr);           // every issued MMA has completed
  if (tid == 0 && ctl[1]) {
    // let the copies still in flight (at most the last R issued) land before the memory goes away
    const int iss = ctl[2];
    for (int b = iss > R ? iss - R : 0; b < iss; ++b) mbar_wait(bar(TF + b % R), (b / R) & 1, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(t.tmem_cols) : "memory");
  }
}

}  // namespace mss
