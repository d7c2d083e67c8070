// Learned surrogate of the off-line stage: a small 3D CNN mapping a coarse cell's sigma/rho
// patch (plus features describing which faces the cell has) to its S-fraction coefficients,
// trained on cells whose coefficients the exact off-line stage produced.  The paper has no such
// component; it replaces the Krylov/Lanczos construction for repeated media, with the exact
// construction kept as the fallback for every cell its screen rejects.
//
// Network (channels C, hidden H, cell of c^3 voxels, c a power of two >= 4):
//   conv3d 3x3x3 pad 1: 2 -> C stride 2, then (log2 c - 2) more stride-2 convs C -> C, then one
//   stride-1 conv C -> C (spatial 2^3 at the end), ReLU after each;
//   dense (8C + F) -> H ReLU, dense H -> D (linear), F = per-cell features appended to the
//   flattened conv output.
// Weights are kept as FP32 masters (Adam) and used in BF16 by the forward and backward passes;
// activations and accumulation are FP32.  Loss: mean squared error over batch x outputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <random>

#include "cuda_util.h"

namespace mss {

namespace {

constexpr int kT = 256;
inline unsigned nb(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

struct LayerDesc {
  int conv;         // 1 conv3d, 0 dense
  int cin, cout;
  int din, dout;    // spatial edge in/out (conv); 1 for dense
  int stride;
  int relu;
  int64_t woff, boff;   // offsets (elements) into the parameter vector
  int64_t in_off, out_off;   // offsets (elements per sample) into the activation arena
};

// conv3d forward: out[b][co][z][y][x] = bias[co] + sum W[co][ci][dz][dy][dx] in[b][ci][...]
__global__ void k_conv_fwd(const float *in, float *out, const __nv_bfloat16 *W, const float *bias, int B, int cin,
                           int cout, int din, int dout, int stride, int relu, int64_t in_stride, int64_t out_stride) {
  const int64_t per = (int64_t)cout * dout * dout * dout;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * per) return;
  const int b = (int)(i / per);
  int64_t r = i - (int64_t)b * per;
  const int co = (int)(r / ((int64_t)dout * dout * dout));
  r -= (int64_t)co * dout * dout * dout;
  const int z = (int)(r / (dout * dout)), y = (int)((r / dout) % dout), x = (int)(r % dout);
  float acc = bias[co];
  const float *inb = in + (int64_t)b * in_stride;
  for (int ci = 0; ci < cin; ++ci) {
    const float *inc = inb + (int64_t)ci * din * din * din;
    const __nv_bfloat16 *w = W + ((int64_t)co * cin + ci) * 27;
    for (int dz = 0; dz < 3; ++dz) {
      const int zi = z * stride - 1 + dz;
      if (zi < 0 || zi >= din) continue;
      for (int dy = 0; dy < 3; ++dy) {
        const int yi = y * stride - 1 + dy;
        if (yi < 0 || yi >= din) continue;
        for (int dx = 0; dx < 3; ++dx) {
          const int xi = x * stride - 1 + dx;
          if (xi < 0 || xi >= din) continue;
          acc += __bfloat162float(w[dz * 9 + dy * 3 + dx]) * inc[((int64_t)zi * din + yi) * din + xi];
        }
      }
    }
  }
  if (relu && acc < 0.f) acc = 0.f;
  out[(int64_t)b * out_stride + r + (int64_t)co * dout * dout * dout] = acc;
}

// gradient w.r.t. the conv input: din[b][ci][zi][yi][xi] = sum_{co,d} W[co][ci][d] dout[b][co][(zi+1-dz)/s ...]
__global__ void k_conv_bwd_data(const float *dout_, float *din_, const __nv_bfloat16 *W, int B, int cin, int cout, int din,
                                int dout, int stride, int64_t in_stride, int64_t out_stride) {
  const int64_t per = (int64_t)cin * din * din * din;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * per) return;
  const int b = (int)(i / per);
  int64_t r = i - (int64_t)b * per;
  const int ci = (int)(r / ((int64_t)din * din * din));
  r -= (int64_t)ci * din * din * din;
  const int zi = (int)(r / (din * din)), yi = (int)((r / din) % din), xi = (int)(r % din);
  float acc = 0.f;
  const float *gb = dout_ + (int64_t)b * out_stride;
  for (int co = 0; co < cout; ++co) {
    const __nv_bfloat16 *w = W + ((int64_t)co * cin + ci) * 27;
    const float *g = gb + (int64_t)co * dout * dout * dout;
    for (int dz = 0; dz < 3; ++dz) {
      const int zn = zi + 1 - dz;
      if (zn < 0 || zn % stride) continue;
      const int z = zn / stride;
      if (z >= dout) continue;
      for (int dy = 0; dy < 3; ++dy) {
        const int yn = yi + 1 - dy;
        if (yn < 0 || yn % stride) continue;
        const int y = yn / stride;
        if (y >= dout) continue;
        for (int dx = 0; dx < 3; ++dx) {
          const int xn = xi + 1 - dx;
          if (xn < 0 || xn % stride) continue;
          const int x = xn / stride;
          if (x >= dout) continue;
          acc += __bfloat162float(w[dz * 9 + dy * 3 + dx]) * g[((int64_t)z * dout + y) * dout + x];
        }
      }
    }
  }
  din_[(int64_t)b * in_stride + (int64_t)ci * din * din * din + ((int64_t)zi * din + yi) * din + xi] = acc;
}

// weight and bias gradients of a conv layer (one thread per weight, deterministic sums)
__global__ void k_conv_bwd_w(const float *in, const float *dout_, float *gW, float *gb, int B, int cin, int cout, int din,
                             int dout, int stride, int64_t in_stride, int64_t out_stride) {
  const int64_t nw = (int64_t)cout * cin * 27;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nw) {
    const int co = (int)(i / (cin * 27));
    const int ci = (int)((i / 27) % cin);
    const int d = (int)(i % 27), dz = d / 9, dy = (d / 3) % 3, dx = d % 3;
    float acc = 0.f;
    for (int b = 0; b < B; ++b) {
      const float *inc = in + (int64_t)b * in_stride + (int64_t)ci * din * din * din;
      const float *g = dout_ + (int64_t)b * out_stride + (int64_t)co * dout * dout * dout;
      for (int z = 0; z < dout; ++z) {
        const int zi = z * stride - 1 + dz;
        if (zi < 0 || zi >= din) continue;
        for (int y = 0; y < dout; ++y) {
          const int yi = y * stride - 1 + dy;
          if (yi < 0 || yi >= din) continue;
          for (int x = 0; x < dout; ++x) {
            const int xi = x * stride - 1 + dx;
            if (xi < 0 || xi >= din) continue;
            acc += g[((int64_t)z * dout + y) * dout + x] * inc[((int64_t)zi * din + yi) * din + xi];
          }
        }
      }
    }
    gW[i] = acc;
  } else if (i < nw + cout) {
    const int co = (int)(i - nw);
    float acc = 0.f;
    for (int b = 0; b < B; ++b) {
      const float *g = dout_ + (int64_t)b * out_stride + (int64_t)co * dout * dout * dout;
      for (int p = 0; p < dout * dout * dout; ++p) acc += g[p];
    }
    gb[co] = acc;
  }
}

// dense forward: out[b][o] = bias[o] + sum_i W[o][i] in[b][i]
__global__ void k_dense_fwd(const float *in, float *out, const __nv_bfloat16 *W, const float *bias, int B, int nin, int nout,
                            int relu, int64_t in_stride, int64_t out_stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * nout) return;
  const int b = (int)(i / nout), o = (int)(i % nout);
  const float *x = in + (int64_t)b * in_stride;
  const __nv_bfloat16 *w = W + (int64_t)o * nin;
  float acc = bias[o];
  for (int k = 0; k < nin; ++k) acc += __bfloat162float(w[k]) * x[k];
  if (relu && acc < 0.f) acc = 0.f;
  out[(int64_t)b * out_stride + o] = acc;
}

__global__ void k_dense_bwd_data(const float *dout_, float *din_, const __nv_bfloat16 *W, int B, int nin, int nout,
                                 int64_t in_stride, int64_t out_stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * nin) return;
  const int b = (int)(i / nin), k = (int)(i % nin);
  const float *g = dout_ + (int64_t)b * out_stride;
  float acc = 0.f;
  for (int o = 0; o < nout; ++o) acc += __bfloat162float(W[(int64_t)o * nin + k]) * g[o];
  din_[(int64_t)b * in_stride + k] = acc;
}

__global__ void k_dense_bwd_w(const float *in, const float *dout_, float *gW, float *gb, int B, int nin, int nout,
                              int64_t in_stride, int64_t out_stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nw = (int64_t)nin * nout;
  if (i < nw) {
    const int o = (int)(i / nin), k = (int)(i % nin);
    float acc = 0.f;
    for (int b = 0; b < B; ++b) acc += dout_[(int64_t)b * out_stride + o] * in[(int64_t)b * in_stride + k];
    gW[i] = acc;
  } else if (i < nw + nout) {
    const int o = (int)(i - nw);
    float acc = 0.f;
    for (int b = 0; b < B; ++b) acc += dout_[(int64_t)b * out_stride + o];
    gb[o] = acc;
  }
}

// ReLU backward in place on the gradient: g *= (a > 0), a = the layer's post-activation output
__global__ void k_relu_bwd(float *g, const float *a, int B, int64_t n, int64_t stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * n) return;
  const int b = (int)(i / n);
  const int64_t j = (int64_t)b * stride + (i - (int64_t)b * n);
  if (a[j] <= 0.f) g[j] = 0.f;
}

// MSE loss and its gradient: dy = 2 (y - t') / (B D) over masked entries (mask may be null),
// t' = (t - mean) / scale per output when an output transform is set (mean null otherwise)
__global__ void k_mse(const float *y, const float *t, const float *mask, const float *mean, const float *scale, float *dy,
                      float *part, int B, int D, int64_t y_stride) {
  __shared__ float sm[kT];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < (int64_t)B * D) {
    const int b = (int)(i / D), o = (int)(i % D);
    const float mk = mask ? mask[i] : 1.f;
    const float tt = mean ? (t[i] - mean[o]) / scale[o] : t[i];
    const float d = (y[(int64_t)b * y_stride + o] - tt) * mk;
    dy[(int64_t)b * y_stride + o] = 2.f * d / ((float)B * D);
    l = d * d;
  }
  sm[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// y = mean + scale * y per output
__global__ void k_affine(float *y, const float *mean, const float *scale, int B, int D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * D) return;
  const int o = (int)(i % D);
  y[i] = mean[o] + scale[o] * y[i];
}

__global__ void k_sum_parts(const float *part, int n, float *out, float scale) {
  __shared__ float sm[kT];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0] * scale;
}

// Adam on the FP32 masters, then the BF16 copy of the weights (biases stay FP32)
__global__ void k_adam(float *p, const float *g, float *m1, float *m2, __nv_bfloat16 *wbf, const unsigned char *is_w,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  const float mh = a / c1, vh = v / c2;
  p[i] -= lr * mh / (sqrtf(vh) + eps);
  if (is_w[i]) wbf[i] = __float2bfloat16_rn(p[i]);
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *wbf, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wbf[i] = __float2bfloat16_rn(p[i]);
}

// concatenate flattened conv output (8C per sample) and the features into the dense input
__global__ void k_concat(const float *a, int na, const float *f, int nf, float *out, int B, int64_t a_stride,
                         int64_t out_stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * (na + nf)) return;
  const int b = (int)(i / (na + nf)), j = (int)(i % (na + nf));
  out[(int64_t)b * out_stride + j] = j < na ? a[(int64_t)b * a_stride + j] : f[(int64_t)b * nf + (j - na)];
}

__global__ void k_split(const float *g, int na, float *ga, int B, int64_t g_stride, int64_t a_stride, int nf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * na) return;
  const int b = (int)(i / na), j = (int)(i % na);
  ga[(int64_t)b * a_stride + j] = g[(int64_t)b * g_stride + j];
  (void)nf;
}

}  // namespace

}  // namespace mss

struct mss_surrogate {
  int cell = 16, nfeat = 0, nout = 0, C = 32, H = 256, batch_max = 0;
  std::vector<mss::LayerDesc> L;
  int64_t nparam = 0, act_per = 0;   // activation arena elements per sample
  int64_t step = 0;
  mss::DevMem p, g, m1, m2, wbf, isw, act, dact, part, loss;
  mss::DevMem out_mean, out_scale;   // output transform (empty: identity)
};

namespace mss {

static void sur_layout(mss_surrogate &s) {
  s.L.clear();
  int64_t w = 0, a = 0;
  int d = s.cell;
  a = 2LL * d * d * d;   // input arena
  int64_t in_off = 0;
  int cin = 2;
  const int nstride2 = (int)std::lround(std::log2((double)s.cell)) - 1;
  for (int l = 0; l < nstride2 + 1; ++l) {
    LayerDesc ld{};
    ld.conv = 1;
    ld.cin = cin;
    ld.cout = s.C;
    ld.din = d;
    ld.stride = l < nstride2 ? 2 : 1;
    ld.dout = (d + 2 - 3) / ld.stride + 1;
    ld.relu = 1;
    ld.woff = w;
    w += (int64_t)ld.cout * ld.cin * 27;
    ld.boff = w;
    w += ld.cout;
    ld.in_off = in_off;
    ld.out_off = a;
    a += (int64_t)ld.cout * ld.dout * ld.dout * ld.dout;
    in_off = ld.out_off;
    s.L.push_back(ld);
    cin = s.C;
    d = ld.dout;
  }
  // dense input: flattened conv output + features
  const int nflat = s.C * d * d * d;
  const int64_t cat_off = a;
  a += nflat + s.nfeat;
  LayerDesc h{};
  h.conv = 0;
  h.cin = nflat + s.nfeat;
  h.cout = s.H;
  h.din = h.dout = 1;
  h.stride = 1;
  h.relu = 1;
  h.woff = w;
  w += (int64_t)h.cin * h.cout;
  h.boff = w;
  w += h.cout;
  h.in_off = cat_off;
  h.out_off = a;
  a += h.cout;
  s.L.push_back(h);
  LayerDesc o{};
  o.conv = 0;
  o.cin = s.H;
  o.cout = s.nout;
  o.din = o.dout = 1;
  o.stride = 1;
  o.relu = 0;
  o.woff = w;
  w += (int64_t)o.cin * o.cout;
  o.boff = w;
  w += o.cout;
  o.in_off = h.out_off;
  o.out_off = a;
  a += o.cout;
  s.L.push_back(o);
  s.nparam = w;
  s.act_per = a;
}

static void sur_alloc_batch(mss_surrogate &s, int B) {
  if (B <= s.batch_max) return;
  s.act.alloc((size_t)B * s.act_per * 4);
  s.dact.alloc((size_t)B * s.act_per * 4);
  s.part.alloc((size_t)nb((int64_t)B * s.nout) * 4 + 16);
  s.batch_max = B;
}

// forward through all layers; x: [B][2 c^3], f: [B][F]; leaves outputs in the arena
static void sur_forward(mss_surrogate &s, int B, const float *x, const float *f, cudaStream_t st) {
  float *A = s.act.as<float>();
  const int64_t P = s.act_per;
  const int64_t n0 = 2LL * s.cell * s.cell * s.cell;
  MSS_CUDA(cudaMemcpy2DAsync(A, P * 4, x, n0 * 4, n0 * 4, B, cudaMemcpyDeviceToDevice, st));
  const float *prm = s.p.as<float>();
  const __nv_bfloat16 *wb = s.wbf.as<__nv_bfloat16>();
  for (auto &l : s.L) {
    if (l.conv) {
      const int64_t n = (int64_t)B * l.cout * l.dout * l.dout * l.dout;
      k_conv_fwd<<<nb(n), kT, 0, st>>>(A + l.in_off, A + l.out_off, wb + l.woff, prm + l.boff, B, l.cin, l.cout, l.din,
                                       l.dout, l.stride, l.relu, P, P);
    } else {
      if (&l == &s.L[s.L.size() - 2]) {
        const auto &lc = s.L[s.L.size() - 3];
        const int na = lc.cout * lc.dout * lc.dout * lc.dout;
        k_concat<<<nb((int64_t)B * (na + s.nfeat)), kT, 0, st>>>(A + lc.out_off, na, f, s.nfeat, A + l.in_off, B, P, P);
      }
      k_dense_fwd<<<nb((int64_t)B * l.cout), kT, 0, st>>>(A + l.in_off, A + l.out_off, wb + l.woff, prm + l.boff, B, l.cin,
                                                           l.cout, l.relu, P, P);
    }
  }
  MSS_CUDA(cudaGetLastError());
}

// backward from dy (already in the gradient arena at the output offset); gradients into s.g
static void sur_backward(mss_surrogate &s, int B, cudaStream_t st) {
  float *A = s.act.as<float>(), *G = s.dact.as<float>();
  const int64_t P = s.act_per;
  float *gp = s.g.as<float>();
  const __nv_bfloat16 *wb = s.wbf.as<__nv_bfloat16>();
  for (int li = (int)s.L.size() - 1; li >= 0; --li) {
    const auto &l = s.L[li];
    const int64_t nout_el = (int64_t)l.cout * l.dout * l.dout * l.dout;
    if (l.relu) k_relu_bwd<<<nb((int64_t)B * nout_el), kT, 0, st>>>(G + l.out_off, A + l.out_off, B, nout_el, P);
    if (l.conv) {
      const int64_t nw = (int64_t)l.cout * l.cin * 27;
      k_conv_bwd_w<<<nb(nw + l.cout), kT, 0, st>>>(A + l.in_off, G + l.out_off, gp + l.woff, gp + l.boff, B, l.cin, l.cout,
                                                   l.din, l.dout, l.stride, P, P);
      if (li > 0) {
        const int64_t nin = (int64_t)B * l.cin * l.din * l.din * l.din;
        k_conv_bwd_data<<<nb(nin), kT, 0, st>>>(G + l.out_off, G + l.in_off, wb + l.woff, B, l.cin, l.cout, l.din, l.dout,
                                                l.stride, P, P);
      }
    } else {
      const int64_t nw = (int64_t)l.cin * l.cout;
      k_dense_bwd_w<<<nb(nw + l.cout), kT, 0, st>>>(A + l.in_off, G + l.out_off, gp + l.woff, gp + l.boff, B, l.cin, l.cout,
                                                    P, P);
      k_dense_bwd_data<<<nb((int64_t)B * l.cin), kT, 0, st>>>(G + l.out_off, G + l.in_off, wb + l.woff, B, l.cin, l.cout,
                                                              P, P);
      if (li == (int)s.L.size() - 2) {
        // gradient of the concatenation: the conv part goes back to the last conv layer's output
        const auto &lc = s.L[li - 1];
        const int na = lc.cout * lc.dout * lc.dout * lc.dout;
        k_split<<<nb((int64_t)B * na), kT, 0, st>>>(G + l.in_off, na, G + lc.out_off, B, P, P, s.nfeat);
      }
    }
  }
  MSS_CUDA(cudaGetLastError());
}

}  // namespace mss

using namespace mss;

extern "C" {

mss_status mss_surrogate_create(int32_t cell, int32_t n_feat, int32_t n_out, int32_t channels, int32_t hidden,
                                uint64_t seed, mss_surrogate **out) {
  return guard([&] {
    MSS_REQUIRE(out && cell >= 4 && (cell & (cell - 1)) == 0 && cell <= 64 && n_feat >= 0 && n_out >= 1 &&
                    channels >= 1 && hidden >= 1,
                MSS_ERR_INVALID_ARG, "bad surrogate shape (cell a power of two in 4..64)");
    auto s = std::make_unique<mss_surrogate>();
    s->cell = cell;
    s->nfeat = n_feat;
    s->nout = n_out;
    s->C = channels;
    s->H = hidden;
    sur_layout(*s);
    // He-style initialisation from a seeded generator (host), biases zero
    std::vector<float> p(s->nparam, 0.f);
    std::vector<unsigned char> isw(s->nparam, 0);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (auto &l : s->L) {
      const int64_t nw = l.conv ? (int64_t)l.cout * l.cin * 27 : (int64_t)l.cout * l.cin;
      const float fan = l.conv ? (float)l.cin * 27 : (float)l.cin;
      const float sd = std::sqrt((l.relu ? 2.f : 1.f) / fan);
      for (int64_t i = 0; i < nw; ++i) {
        p[l.woff + i] = sd * nd(rng);
        isw[l.woff + i] = 1;
      }
    }
    upload(s->p, p);
    upload(s->isw, isw);
    s->g.alloc(s->nparam * 4);
    s->m1.alloc(s->nparam * 4);
    s->m2.alloc(s->nparam * 4);
    MSS_CUDA(cudaMemset(s->m1.p, 0, s->nparam * 4));
    MSS_CUDA(cudaMemset(s->m2.p, 0, s->nparam * 4));
    s->wbf.alloc(s->nparam * 2);
    k_to_bf16<<<nb(s->nparam), kT>>>(s->p.as<float>(), s->wbf.as<__nv_bfloat16>(), s->nparam);
    s->loss.alloc(16);
    MSS_CUDA(cudaDeviceSynchronize());
    *out = s.release();
  });
}

mss_status mss_surrogate_info(const mss_surrogate *s, int64_t info[4]) {
  return guard([&] {
    MSS_REQUIRE(s && info, MSS_ERR_INVALID_ARG, "null argument");
    info[0] = s->nparam;
    info[1] = 2LL * s->cell * s->cell * s->cell;
    info[2] = s->nfeat;
    info[3] = s->nout;
  });
}

mss_status mss_surrogate_get_params(const mss_surrogate *s, float *host) {
  return guard([&] {
    MSS_REQUIRE(s && host, MSS_ERR_INVALID_ARG, "null argument");
    MSS_CUDA(cudaMemcpy(host, s->p.p, s->nparam * 4, cudaMemcpyDeviceToHost));
  });
}

mss_status mss_surrogate_set_params(mss_surrogate *s, const float *host) {
  return guard([&] {
    MSS_REQUIRE(s && host, MSS_ERR_INVALID_ARG, "null argument");
    MSS_CUDA(cudaMemcpy(s->p.p, host, s->nparam * 4, cudaMemcpyHostToDevice));
    k_to_bf16<<<nb(s->nparam), kT>>>(s->p.as<float>(), s->wbf.as<__nv_bfloat16>(), s->nparam);
    MSS_CUDA(cudaDeviceSynchronize());
    MSS_CUDA(cudaMemset(s->m1.p, 0, s->nparam * 4));
    MSS_CUDA(cudaMemset(s->m2.p, 0, s->nparam * 4));
    s->step = 0;
  });
}

mss_status mss_surrogate_forward(mss_surrogate *s, int32_t batch, const float *x, const float *feat, float *y,
                                 void *stream) {
  return guard([&] {
    MSS_REQUIRE(s && batch >= 1 && x && y && (s->nfeat == 0 || feat), MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sur_alloc_batch(*s, batch);
    sur_forward(*s, batch, x, feat, st);
    const auto &lo = s->L.back();
    MSS_CUDA(cudaMemcpy2DAsync(y, (size_t)s->nout * 4, s->act.as<float>() + lo.out_off, (size_t)s->act_per * 4,
                               (size_t)s->nout * 4, batch, cudaMemcpyDeviceToDevice, st));
  });
}

mss_status mss_surrogate_backward(mss_surrogate *s, int32_t batch, const float *x, const float *feat, const float *dy,
                                  float *grad, void *stream) {
  return guard([&] {
    MSS_REQUIRE(s && batch >= 1 && x && dy && grad && (s->nfeat == 0 || feat), MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sur_alloc_batch(*s, batch);
    sur_forward(*s, batch, x, feat, st);
    const auto &lo = s->L.back();
    MSS_CUDA(cudaMemsetAsync(s->dact.p, 0, (size_t)batch * s->act_per * 4, st));
    MSS_CUDA(cudaMemcpy2DAsync(s->dact.as<float>() + lo.out_off, (size_t)s->act_per * 4, dy, (size_t)s->nout * 4,
                               (size_t)s->nout * 4, batch, cudaMemcpyDeviceToDevice, st));
    sur_backward(*s, batch, st);
    MSS_CUDA(cudaMemcpyAsync(grad, s->g.p, s->nparam * 4, cudaMemcpyDeviceToDevice, st));
  });
}

mss_status mss_surrogate_train_step(mss_surrogate *s, int32_t batch, const float *x, const float *feat,
                                    const float *target, const float *mask, float lr, float *loss, void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_surrogate_train_step");
    MSS_REQUIRE(s && batch >= 1 && x && target && (s->nfeat == 0 || feat) && lr > 0, MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sur_alloc_batch(*s, batch);
    sur_forward(*s, batch, x, feat, st);
    const auto &lo = s->L.back();
    MSS_CUDA(cudaMemsetAsync(s->dact.p, 0, (size_t)batch * s->act_per * 4, st));
    const int64_t n = (int64_t)batch * s->nout;
    const bool aff = s->out_mean.p != nullptr;
    k_mse<<<nb(n), kT, 0, st>>>(s->act.as<float>() + lo.out_off, target, mask, aff ? s->out_mean.as<float>() : nullptr,
                                aff ? s->out_scale.as<float>() : nullptr, s->dact.as<float>() + lo.out_off,
                                s->part.as<float>(), batch, s->nout, s->act_per);
    k_sum_parts<<<1, kT, 0, st>>>(s->part.as<float>(), (int)nb(n), s->loss.as<float>(), 1.f / (float)n);
    sur_backward(*s, batch, st);
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<nb(s->nparam), kT, 0, st>>>(s->p.as<float>(), s->g.as<float>(), s->m1.as<float>(), s->m2.as<float>(),
                                         s->wbf.as<__nv_bfloat16>(), s->isw.as<unsigned char>(), s->nparam, lr, b1, b2,
                                         1e-8f, 1.f - std::pow(b1, (float)s->step), 1.f - std::pow(b2, (float)s->step));
    if (loss) MSS_CUDA(cudaMemcpyAsync(loss, s->loss.p, 4, cudaMemcpyDeviceToDevice, st));
    MSS_CUDA(cudaGetLastError());
  });
}

mss_status mss_surrogate_set_output_transform(mss_surrogate *s, const float *mean, const float *scale) {
  return guard([&] {
    MSS_REQUIRE(s && ((mean == nullptr) == (scale == nullptr)), MSS_ERR_INVALID_ARG, "bad argument");
    if (!mean) {
      s->out_mean.release();
      s->out_scale.release();
      return;
    }
    for (int o = 0; o < s->nout; ++o)
      MSS_REQUIRE(scale[o] > 0 && std::isfinite(scale[o]) && std::isfinite(mean[o]), MSS_ERR_INVALID_ARG,
                  "output scales must be positive and finite");
    upload(s->out_mean, std::vector<float>(mean, mean + s->nout));
    upload(s->out_scale, std::vector<float>(scale, scale + s->nout));
  });
}

mss_status mss_surrogate_fit_output_transform(mss_surrogate *s, int32_t n, const double *targets, const float *mask) {
  return guard([&] {
    MSS_REQUIRE(s && n >= 1 && targets, MSS_ERR_INVALID_ARG, "bad argument");
    const int D = s->nout;
    std::vector<double> sum(D, 0.0), sq(D, 0.0), cnt(D, 0.0);
    for (int i = 0; i < n; ++i)
      for (int o = 0; o < D; ++o) {
        const double w = mask ? (double)mask[(int64_t)i * D + o] : 1.0;
        const double v = targets[(int64_t)i * D + o];
        sum[o] += w * v;
        sq[o] += w * v * v;
        cnt[o] += w;
      }
    std::vector<float> mean(D, 0.f), scale(D, 1.f);
    for (int o = 0; o < D; ++o) {
      if (cnt[o] <= 0) continue;
      const double mu = sum[o] / cnt[o];
      const double var = std::max(0.0, sq[o] / cnt[o] - mu * mu);
      mean[o] = (float)mu;
      scale[o] = (float)std::max(std::sqrt(var), 1e-3 * std::max(1.0, std::fabs(mu)));
    }
    upload(s->out_mean, mean);
    upload(s->out_scale, scale);
  });
}

mss_status mss_surrogate_predict(mss_surrogate *s, int32_t batch, const float *x, const float *feat, float *y,
                                 void *stream) {
  return guard([&] {
    MSS_REQUIRE(s && batch >= 1 && x && y && (s->nfeat == 0 || feat), MSS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sur_alloc_batch(*s, batch);
    sur_forward(*s, batch, x, feat, st);
    const auto &lo = s->L.back();
    MSS_CUDA(cudaMemcpy2DAsync(y, (size_t)s->nout * 4, s->act.as<float>() + lo.out_off, (size_t)s->act_per * 4,
                               (size_t)s->nout * 4, batch, cudaMemcpyDeviceToDevice, st));
    if (s->out_mean.p)
      k_affine<<<nb((int64_t)batch * s->nout), kT, 0, st>>>(y, s->out_mean.as<float>(), s->out_scale.as<float>(), batch,
                                                             s->nout);
    MSS_CUDA(cudaGetLastError());
  });
}

void mss_surrogate_destroy(mss_surrogate *s) { delete s; }

}  // extern "C"
