// Empirical stability (CFL) check of an on-line simulation: leapfrog from a seeded random state
// with zero velocity and no source, through the sim's own step kernels, and compare the state
// norm after n steps with the initial one.  Below the CFL limit the leapfrog conserves the
// discrete energy and the norm stays within a factor set by the conditioning of the masses;
// above it the highest mode grows geometrically (amplification |r| > 1 per step), so a growth far
// beyond that factor identifies a step size above the ROM's CFL limit (Section 6; leapfrog
// stability of the three-point scheme, Eq. intrtstep_td).  The sim's state and step counter are
// restored afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "common.h"
#include "cuda_util.h"

using namespace mss;

extern "C" mss_status mss_sim_check_stability(mss_sim *s, int32_t n_steps, uint64_t seed, double max_growth,
                                              double *growth, void *stream) {
  return guard([&] {
    const Range nvtx_range("mss_sim_check_stability");
    MSS_REQUIRE(s && n_steps >= 1 && max_growth > 1.0, MSS_ERR_INVALID_ARG, "bad argument");
    int64_t info[8];
    mss_status e = mss_sim_info(s, info);
    MSS_REQUIRE(e == MSS_OK, e, "sim info");
    const int64_t n_src = info[0], n_rcv = info[1], prec = info[2], n_state = info[4];
    const size_t es = prec == MSS_FP64 ? 8 : 4;
    std::vector<double> now(n_state), old(n_state), u0(n_state), u1(n_state), v1(n_state);
    int64_t taken0 = 0, taken1 = 0;
    e = mss_sim_save_state(s, now.data(), old.data(), &taken0);
    MSS_REQUIRE(e == MSS_OK, e, "save state");
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (auto &x : u0) x = nd(rng);
    e = mss_sim_load_state(s, u0.data(), u0.data(), 0);
    MSS_REQUIRE(e == MSS_OK, e, "load state");
    DevMem w, tr;
    w.alloc((size_t)n_steps * 8);
    MSS_CUDA(cudaMemset(w.p, 0, (size_t)n_steps * 8));
    tr.alloc((size_t)n_steps * std::max<int64_t>(1, n_rcv) * n_src * es);
    mss_status e_step = mss_step(s, n_steps, w.as<double>(), tr.p, 0, stream);
    if (e_step == MSS_OK) {
      const cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
      if (ce != cudaSuccess) e_step = MSS_ERR_CUDA;
    }
    mss_status e_save = e_step == MSS_OK ? mss_sim_save_state(s, u1.data(), v1.data(), &taken1) : MSS_OK;
    const mss_status e_restore = mss_sim_load_state(s, now.data(), old.data(), taken0);
    MSS_REQUIRE(e_step == MSS_OK, e_step, "stepping failed");
    MSS_REQUIRE(e_save == MSS_OK, e_save, "save state");
    MSS_REQUIRE(e_restore == MSS_OK, e_restore, "restore state");
    double n0 = 0, n1 = 0;
    for (int64_t i = 0; i < n_state; ++i) {
      n0 += u0[i] * u0[i];
      n1 += std::isfinite(u1[i]) ? u1[i] * u1[i] : INFINITY;
    }
    const double g = std::sqrt(n1 / std::max(n0, 1e-300));
    if (growth) *growth = g;
    MSS_REQUIRE(g <= max_growth, MSS_ERR_CFL,
                "state grew " + std::to_string(g) + "x in " + std::to_string(n_steps) +
                    " source-free steps: the step size is above the CFL limit");
  });
}
