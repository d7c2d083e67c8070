// CUDA helpers shared by the .cu translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.h"

namespace mss {

#define MSS_CUDA(x)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (x);                                                                            \
    if (e_ != cudaSuccess)                                                                           \
      throw ::mss::Error(e_ == cudaErrorMemoryAllocation ? MSS_ERR_OOM : MSS_ERR_CUDA,             \
                         std::string(#x) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

// Owning device allocation (cudaMalloc / cudaFree).
struct DevMem {
  void *p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem &) = delete;
  DevMem &operator=(const DevMem &) = delete;
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    MSS_CUDA(cudaMalloc(&p, n));
    bytes = n;
  }
  template <typename T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

template <typename T>
void upload(DevMem &m, const std::vector<T> &v) {
  m.alloc(v.size() * sizeof(T));
  if (!v.empty()) MSS_CUDA(cudaMemcpy(m.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

}  // namespace mss
