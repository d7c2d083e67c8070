// Fine-grid leapfrog on the GPU (Section 1, Eq. wave_fll), batched over sources:
//   u^{n+1} = 2 u^n - u^{n-1} + tau^2 B^{-1} (A u^n - g w(t_n)),   trace n = q^T u^n.
// State lives on the full node grid ([node][source], x fastest), removed Dirichlet nodes hold 0,
// so the 5/7-point couplings are constant-stride neighbours.  Per node: diag(A)/b and the
// couplings A(p, p + e_a)/b ... stored as A(p, p + e_a) and 1/b (the lower coupling of p is the
// upper coupling of p - e_a).  HBM-bound: one read of u^n (neighbours from cache), u^{n-1},
// one write, d + 2 coefficients per node.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>

#include "cuda_util.h"

namespace mss {

template <typename T>
struct FineArgs {
  const T *diag, *cp0, *cp1, *cp2, *binv;
  const int64_t *src_node, *rcv_node;
  T *u0, *u1;
  int64_t nodes, s0, s1, s2;
  int d, S, R;
  T tau2;
};

constexpr int kFineThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFineThreads) k_fine(const FineArgs<T> a, const int cur, const double *w, T *traces) {
  const int64_t total = a.nodes * a.S;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const T *u = cur ? a.u1 : a.u0;
  T *uo = cur ? a.u0 : a.u1;
  if (i < total) {
    const int64_t p = i / a.S;
    const int s = (int)(i - p * a.S);
    const T bi = a.binv[p];
    if (bi == T(0)) return;   // removed node: stays zero
    const int S = a.S;
    T lap = a.diag[p] * u[i];
    const T *cp[3] = {a.cp0, a.cp1, a.cp2};
    const int64_t st[3] = {a.s0, a.s1, a.s2};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= a.d) break;
      const int64_t q = p + st[ax], r = p - st[ax];
      if (q < a.nodes) lap += cp[ax][p] * u[q * S + s];
      if (r >= 0) lap += cp[ax][r] * u[r * S + s];
    }
    if (a.src_node[s] == p) lap -= (T)(*w);
    uo[i] = T(2) * u[i] - uo[i] + a.tau2 * bi * lap;
  } else {
    const int64_t j = i - ((total + kFineThreads - 1) / kFineThreads) * kFineThreads;
    if (j < 0 || j >= (int64_t)a.R * a.S) return;
    const int64_t r = j / a.S;
    const int s = (int)(j - r * a.S);
    traces[j] = u[a.rcv_node[r] * a.S + s];
  }
}

// 16-byte vector of T over sources (4 floats or 2 doubles).
template <typename T> struct FineVec;
template <> struct FineVec<float> { using type = float4; static constexpr int n = 4; };
template <> struct FineVec<double> { using type = double2; static constexpr int n = 2; };

// Same step with one thread per (node, vector of VN sources) when S is a multiple of VN: 16-byte
// loads and stores of the state, the node's coefficients read once per vector instead of once per
// source, and 32-bit index arithmetic whenever the thread count allows.  Every element takes the
// same operations in the same order as k_fine.
template <typename T>
__global__ void __launch_bounds__(kFineThreads) k_fine_v(const FineArgs<T> a, const int cur, const double *w,
                                                         T *traces) {
  using V = typename FineVec<T>::type;
  constexpr int VN = FineVec<T>::n;
  const int nv = a.S / VN;
  const int64_t total = a.nodes * nv;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const T *u = cur ? a.u1 : a.u0;
  T *uo = cur ? a.u0 : a.u1;
  if (i < total) {
    int64_t p;
    int v;
    if (total <= 0xffffffffLL) {
      const unsigned ii = (unsigned)i, pp = ii / (unsigned)nv;
      p = pp;
      v = (int)(ii - pp * (unsigned)nv);
    } else {
      p = i / nv;
      v = (int)(i - p * nv);
    }
    const T bi = a.binv[p];
    if (bi == T(0)) return;   // removed node: stays zero
    const int S = a.S;
    const int64_t off = p * S + (int64_t)v * VN;
    const V uc = *reinterpret_cast<const V *>(u + off);
    const T *ue = reinterpret_cast<const T *>(&uc);
    const T dg = a.diag[p];
    T lap[VN];
#pragma unroll
    for (int e = 0; e < VN; ++e) lap[e] = dg * ue[e];
    const T *cp[3] = {a.cp0, a.cp1, a.cp2};
    const int64_t st[3] = {a.s0, a.s1, a.s2};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= a.d) break;
      const int64_t q = p + st[ax], r = p - st[ax];
      if (q < a.nodes) {
        const T c = cp[ax][p];
        const V x = *reinterpret_cast<const V *>(u + off + st[ax] * S);
        const T *xe = reinterpret_cast<const T *>(&x);
#pragma unroll
        for (int e = 0; e < VN; ++e) lap[e] += c * xe[e];
      }
      if (r >= 0) {
        const T c = cp[ax][r];
        const V x = *reinterpret_cast<const V *>(u + off - st[ax] * S);
        const T *xe = reinterpret_cast<const T *>(&x);
#pragma unroll
        for (int e = 0; e < VN; ++e) lap[e] += c * xe[e];
      }
    }
#pragma unroll
    for (int e = 0; e < VN; ++e)
      if (a.src_node[v * VN + e] == p) lap[e] -= (T)(*w);
    V o = *reinterpret_cast<const V *>(uo + off);
    T *oe = reinterpret_cast<T *>(&o);
#pragma unroll
    for (int e = 0; e < VN; ++e) oe[e] = T(2) * ue[e] - oe[e] + a.tau2 * bi * lap[e];
    *reinterpret_cast<V *>(uo + off) = o;
  } else {
    const int64_t j = i - ((total + kFineThreads - 1) / kFineThreads) * kFineThreads;
    if (j < 0 || j >= (int64_t)a.R * a.S) return;
    const int64_t r = j / a.S;
    const int s = (int)(j - r * a.S);
    traces[j] = u[a.rcv_node[r] * a.S + s];
  }
}

// Same leapfrog on the operator's CSR rows, for any operator (the elastic one has 3 unknowns per
// node and a 27-node stencil): state [unknown][source]; thread (row u, source s) forms the row's
// product in column order; the extra threads past N S write the traces.
template <typename T>
struct FineCsrArgs {
  const int64_t *rp, *col;
  const T *val, *binv;
  const int64_t *src, *rcv;   // unknowns
  T *u0, *u1;
  int64_t N;
  int S, R;
  T tau2;
};

template <typename T>
__global__ void __launch_bounds__(kFineThreads) k_fine_csr(const FineCsrArgs<T> a, const int cur, const double *w,
                                                           T *traces) {
  const int64_t total = a.N * a.S;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const T *u = cur ? a.u1 : a.u0;
  T *uo = cur ? a.u0 : a.u1;
  if (i < total) {
    const int64_t r = i / a.S;
    const int s = (int)(i - r * a.S);
    T acc = T(0);
    for (int64_t k = a.rp[r]; k < a.rp[r + 1]; ++k) acc += a.val[k] * u[a.col[k] * a.S + s];
    if (a.src[s] == r) acc -= (T)(*w);
    uo[i] = T(2) * u[i] - uo[i] + a.tau2 * a.binv[r] * acc;
  } else {
    const int64_t j = i - ((total + kFineThreads - 1) / kFineThreads) * kFineThreads;
    if (j < 0 || j >= (int64_t)a.R * a.S) return;
    const int64_t r = j / a.S;
    const int s = (int)(j - r * a.S);
    traces[j] = u[a.rcv[r] * a.S + s];
  }
}

struct FineGraphKey {
  int64_t n;
  const void *w, *t;
  int cur;
  bool operator<(const FineGraphKey &o) const {
    if (n != o.n) return n < o.n;
    if (w != o.w) return w < o.w;
    if (t != o.t) return t < o.t;
    return cur < o.cur;
  }
};

}  // namespace mss

struct mss_fine {
  int prec = MSS_FP64, d = 0, S = 0, R = 0, cur = 0;
  int64_t nodes = 0, str[3] = {0, 0, 0}, steps = 0;
  double tau = 0;
  mss::DevMem diag, cp[3], binv, src, rcv, u[2];
  int csr = 0;                      // 1: the CSR kernel on unknowns (mss_fine_create_unknowns)
  int64_t N = 0;
  mss::DevMem rp, col, val;
  std::map<mss::FineGraphKey, cudaGraphExec_t> graphs;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ~mss_fine() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace mss {

template <typename T>
static FineArgs<T> fine_args(const mss_fine &f) {
  FineArgs<T> a;
  a.diag = f.diag.as<T>();
  a.cp0 = f.cp[0].as<T>();
  a.cp1 = f.cp[1].as<T>();
  a.cp2 = f.cp[2].as<T>();
  a.binv = f.binv.as<T>();
  a.src_node = f.src.as<int64_t>();
  a.rcv_node = f.rcv.as<int64_t>();
  a.u0 = f.u[0].as<T>();
  a.u1 = f.u[1].as<T>();
  a.nodes = f.nodes;
  a.s0 = f.str[0];
  a.s1 = f.str[1];
  a.s2 = f.str[2];
  a.d = f.d;
  a.S = f.S;
  a.R = f.R;
  a.tau2 = (T)(f.tau * f.tau);
  return a;
}

template <typename T>
static void fine_launch(mss_fine &f, int64_t n, const double *w, T *traces, cudaStream_t st) {
  if (f.csr) {
    FineCsrArgs<T> c;
    c.rp = f.rp.as<int64_t>();
    c.col = f.col.as<int64_t>();
    c.val = f.val.as<T>();
    c.binv = f.binv.as<T>();
    c.src = f.src.as<int64_t>();
    c.rcv = f.rcv.as<int64_t>();
    c.u0 = f.u[0].as<T>();
    c.u1 = f.u[1].as<T>();
    c.N = f.N;
    c.S = f.S;
    c.R = f.R;
    c.tau2 = (T)(f.tau * f.tau);
    const int64_t nb = (f.N * f.S + kFineThreads - 1) / kFineThreads + ((int64_t)f.R * f.S + kFineThreads - 1) / kFineThreads;
    int cur = f.cur;
    for (int64_t j = 0; j < n; ++j) {
      k_fine_csr<T><<<(unsigned)nb, kFineThreads, 0, st>>>(c, cur, w + j, traces + j * (int64_t)f.R * f.S);
      cur ^= 1;
    }
    MSS_CUDA(cudaGetLastError());
    return;
  }
  const FineArgs<T> a = fine_args<T>(f);
  constexpr int VN = FineVec<T>::n;
  const bool vec = f.S % VN == 0;
  const int64_t total = f.nodes * (vec ? f.S / VN : f.S);
  const int64_t nb = (total + kFineThreads - 1) / kFineThreads + ((int64_t)f.R * f.S + kFineThreads - 1) / kFineThreads;
  int cur = f.cur;
  for (int64_t j = 0; j < n; ++j) {
    if (vec) k_fine_v<T><<<(unsigned)nb, kFineThreads, 0, st>>>(a, cur, w + j, traces + j * (int64_t)f.R * f.S);
    else k_fine<T><<<(unsigned)nb, kFineThreads, 0, st>>>(a, cur, w + j, traces + j * (int64_t)f.R * f.S);
    cur ^= 1;
  }
  MSS_CUDA(cudaGetLastError());
}

template <typename T>
static void fine_step(mss_fine &f, int64_t n, const double *w, void *traces, int use_graph, cudaStream_t st) {
  if (!use_graph) {
    fine_launch<T>(f, n, w, (T *)traces, st);
  } else {
    MSS_CUDA(cudaEventRecord(f.ev_in, st));
    MSS_CUDA(cudaStreamWaitEvent(f.cap, f.ev_in, 0));
    FineGraphKey key{n, w, traces, f.cur};
    auto it = f.graphs.find(key);
    if (it == f.graphs.end()) {
      cudaGraph_t g = nullptr;
      MSS_CUDA(cudaStreamBeginCapture(f.cap, cudaStreamCaptureModeThreadLocal));
      try {
        fine_launch<T>(f, n, w, (T *)traces, f.cap);
      } catch (...) {
        cudaStreamEndCapture(f.cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      MSS_CUDA(cudaStreamEndCapture(f.cap, &g));
      cudaGraphExec_t ge;
      cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      MSS_CUDA(e);
      it = f.graphs.emplace(key, ge).first;
    }
    MSS_CUDA(cudaGraphLaunch(it->second, f.cap));
    MSS_CUDA(cudaEventRecord(f.ev_out, f.cap));
    MSS_CUDA(cudaStreamWaitEvent(st, f.ev_out, 0));
  }
  f.cur = (int)((f.cur + n) & 1);
  f.steps += n;
}

}  // namespace mss

using namespace mss;

extern "C" {

mss_status mss_fine_create(const mss_operator *op, int32_t precision, double tau, int32_t n_src,
                           const int32_t *src_nodes, int32_t n_rcv, const int32_t *rcv_nodes, mss_fine **out) {
  return guard([&] {
    MSS_REQUIRE(op && out && n_src >= 1 && src_nodes && n_rcv >= 0 && (n_rcv == 0 || rcv_nodes), MSS_ERR_INVALID_ARG,
                "bad argument");
    MSS_REQUIRE(precision == MSS_FP64 || precision == MSS_FP32, MSS_ERR_INVALID_ARG, "precision must be FP64 or FP32");
    MSS_REQUIRE(tau > 0 && std::isfinite(tau), MSS_ERR_CFL, "tau must be positive");
    const Operator &o = op->o;
    MSS_REQUIRE(o.comps == 1, MSS_ERR_INVALID_ARG, "the fine-grid kernels take one unknown per node (acoustic operator)");
    auto f = std::make_unique<mss_fine>();
    MSS_CUDA(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking));
    MSS_CUDA(cudaEventCreateWithFlags(&f->ev_in, cudaEventDisableTiming));
    MSS_CUDA(cudaEventCreateWithFlags(&f->ev_out, cudaEventDisableTiming));
    f->prec = precision;
    f->d = o.g.dim;
    f->S = n_src;
    f->R = n_rcv;
    f->tau = tau;
    f->nodes = o.nodes;
    int64_t ext[3];
    for (int a = 0; a < 3; ++a) ext[a] = a < o.g.dim ? o.g.n[a] + 1 : 1;
    f->str[o.g.dim - 1] = 1;
    for (int a = o.g.dim - 2; a >= 0; --a) f->str[a] = f->str[a + 1] * ext[a + 1];
    std::vector<double> diag(o.nodes, 0.0), binv(o.nodes, 0.0), cp[3];
    for (int a = 0; a < 3; ++a) cp[a].assign(a < o.g.dim ? o.nodes : 1, 0.0);
    for (int64_t u = 0; u < o.N; ++u) {
      const int64_t p = o.node_of[u];
      binv[p] = 1.0 / o.B[u];
      for (int64_t k = o.A.ptr[u]; k < o.A.ptr[u + 1]; ++k) {
        const int64_t q = o.node_of[o.A.col[k]];
        if (q == p) diag[p] = o.A.val[k];
        for (int a = 0; a < o.g.dim; ++a)
          if (q == p + f->str[a]) cp[a][p] = o.A.val[k];
      }
    }
    auto conv = [&](DevMem &m, const std::vector<double> &v) {
      if (precision == MSS_FP64) upload(m, v);
      else upload(m, std::vector<float>(v.begin(), v.end()));
    };
    conv(f->diag, diag);
    conv(f->binv, binv);
    for (int a = 0; a < 3; ++a) conv(f->cp[a], cp[a]);
    auto nodes_of = [&](int32_t n, const int32_t *nd) {
      std::vector<int64_t> out(n);
      for (int32_t j = 0; j < n; ++j) {
        int64_t p = 0;
        for (int a = 0; a < o.g.dim; ++a) {
          const int32_t x = nd[(int64_t)j * o.g.dim + a];
          MSS_REQUIRE(x >= 0 && x <= o.g.n[a], MSS_ERR_INVALID_ARG, "node outside the grid");
          p += x * f->str[a];
        }
        MSS_REQUIRE(o.unknown[p] >= 0, MSS_ERR_INVALID_ARG, "node on a Dirichlet wall");
        out[j] = p;
      }
      return out;
    };
    upload(f->src, nodes_of(n_src, src_nodes));
    upload(f->rcv, nodes_of(n_rcv, rcv_nodes));
    const size_t es = precision == MSS_FP64 ? 8 : 4;
    for (int l = 0; l < 2; ++l) {
      f->u[l].alloc((size_t)o.nodes * n_src * es);
      MSS_CUDA(cudaMemset(f->u[l].p, 0, f->u[l].bytes));
    }
    *out = f.release();
  });
}

mss_status mss_fine_create_unknowns(const mss_operator *op, int32_t precision, double tau, int32_t n_src,
                                    const int64_t *src_unknowns, int32_t n_rcv, const int64_t *rcv_unknowns,
                                    mss_fine **out) {
  return guard([&] {
    MSS_REQUIRE(op && out && n_src >= 1 && src_unknowns && n_rcv >= 0 && (n_rcv == 0 || rcv_unknowns),
                MSS_ERR_INVALID_ARG, "bad argument");
    MSS_REQUIRE(precision == MSS_FP64 || precision == MSS_FP32, MSS_ERR_INVALID_ARG, "precision must be FP64 or FP32");
    MSS_REQUIRE(tau > 0 && std::isfinite(tau), MSS_ERR_CFL, "tau must be positive");
    const Operator &o = op->o;
    for (int32_t j = 0; j < n_src; ++j)
      MSS_REQUIRE(src_unknowns[j] >= 0 && src_unknowns[j] < o.N, MSS_ERR_INVALID_ARG, "source unknown out of range");
    for (int32_t j = 0; j < n_rcv; ++j)
      MSS_REQUIRE(rcv_unknowns[j] >= 0 && rcv_unknowns[j] < o.N, MSS_ERR_INVALID_ARG, "receiver unknown out of range");
    auto f = std::make_unique<mss_fine>();
    MSS_CUDA(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking));
    MSS_CUDA(cudaEventCreateWithFlags(&f->ev_in, cudaEventDisableTiming));
    MSS_CUDA(cudaEventCreateWithFlags(&f->ev_out, cudaEventDisableTiming));
    f->prec = precision;
    f->csr = 1;
    f->N = o.N;
    f->S = n_src;
    f->R = n_rcv;
    f->tau = tau;
    upload(f->rp, o.A.ptr);
    upload(f->col, o.A.col);
    std::vector<double> binv(o.N);
    for (int64_t u = 0; u < o.N; ++u) binv[u] = 1.0 / o.B[u];
    if (precision == MSS_FP64) {
      upload(f->val, o.A.val);
      upload(f->binv, binv);
    } else {
      upload(f->val, std::vector<float>(o.A.val.begin(), o.A.val.end()));
      upload(f->binv, std::vector<float>(binv.begin(), binv.end()));
    }
    upload(f->src, std::vector<int64_t>(src_unknowns, src_unknowns + n_src));
    upload(f->rcv, n_rcv ? std::vector<int64_t>(rcv_unknowns, rcv_unknowns + n_rcv) : std::vector<int64_t>(1, 0));
    const size_t es = precision == MSS_FP64 ? 8 : 4;
    for (int l = 0; l < 2; ++l) {
      f->u[l].alloc((size_t)o.N * n_src * es);
      MSS_CUDA(cudaMemset(f->u[l].p, 0, f->u[l].bytes));
    }
    *out = f.release();
  });
}

mss_status mss_fine_reset(mss_fine *f, void *stream) {
  return guard([&] {
    MSS_REQUIRE(f, MSS_ERR_INVALID_ARG, "null handle");
    for (int l = 0; l < 2; ++l) MSS_CUDA(cudaMemsetAsync(f->u[l].p, 0, f->u[l].bytes, (cudaStream_t)stream));
    f->cur = 0;
    f->steps = 0;
  });
}

mss_status mss_fine_step(mss_fine *f, int64_t n_steps, const double *waveform, void *traces, int32_t use_graph,
                         void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_fine_step");
    MSS_REQUIRE(f && waveform && traces && n_steps >= 0, MSS_ERR_INVALID_ARG, "bad argument");
    if (n_steps == 0) return;
    if (f->prec == MSS_FP64) fine_step<double>(*f, n_steps, waveform, traces, use_graph, (cudaStream_t)stream);
    else fine_step<float>(*f, n_steps, waveform, traces, use_graph, (cudaStream_t)stream);
  });
}

void mss_fine_destroy(mss_fine *f) { delete f; }

}  // extern "C"
