// Internal declarations shared by the translation units of libmss.
#pragma once

#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mss.h"

namespace mss {

// Scoped NVTX range around an entry point (off-line stages, time blocks, autotuning), so that a
// profiler's timeline shows them by name; a no-op when no tool is attached.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

// An error carrying a status code; caught at the C ABI boundary.
struct Error : std::runtime_error {
  mss_status code;
  Error(mss_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string &m);

#define MSS_REQUIRE(cond, code, msg)                                                  \
  do {                                                                                \
    if (!(cond)) throw ::mss::Error((code), std::string(msg));                        \
  } while (0)

// Run a body, translating exceptions into a status and the thread-local message.
template <typename F>
mss_status guard(F &&f) {
  try {
    f();
    set_last_error("");
    return MSS_OK;
  } catch (const Error &e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return MSS_ERR_OOM;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return MSS_ERR_INVALID_ARG;
  }
}

// ------------------------------------------------------------------ CSR (host)
struct Csr {
  int64_t n = 0;
  std::vector<int64_t> ptr, col;
  std::vector<double> val;
};

// ------------------------------------------------------------------ fine operator
struct Operator {
  mss_grid g{};
  int64_t nodes = 0;               // full node grid size
  int64_t N = 0;                   // unknowns
  std::vector<int64_t> unknown;    // full node -> unknown or -1
  std::vector<int64_t> node_of;    // unknown -> full node
  Csr A;
  std::vector<double> B;
  int64_t nshape[3] = {1, 1, 1};   // node grid extents per array axis
  int comps = 1;                   // unknowns per kept node: 1 (acoustic) or 3 (elastic, node-major)
};

// ------------------------------------------------------------------ partition
struct Face {
  int kind = 0;                    // 0 interior, 1 I/O
  int cells[2] = {-1, -1};
  int axis = -1;
  int shape[2] = {1, 1};           // face node grid (tangential axes, array order)
  std::vector<int64_t> nodes;      // prime ids, face order
  std::vector<int64_t> parents;    // unknowns
};

struct Cell {
  int coords[3] = {0, 0, 0};
  std::vector<int> faces;          // ascending
  bool built = false;
  std::vector<int64_t> nodes;      // prime ids: boundary (face order) then interior ascending
  int64_t K = 0;
  Csr A;
  std::vector<double> B;
};

struct Partition {
  const Operator *op = nullptr;
  std::vector<double> sigma, rho;
  int d = 0;
  int cs[3] = {1, 1, 1};
  int nc[3] = {1, 1, 1};
  int n_cells = 0;
  std::vector<Face> faces;
  int n_int_faces = 0;
  std::vector<Cell> cells;
  // faces holding each unknown (CSR over unknowns, ascending face ids)
  std::vector<int64_t> nf_ptr;
  std::vector<int32_t> nf_face;
  std::vector<int64_t> plain_prime;   // unknown -> prime id, -1 for corner-set nodes
  std::vector<int64_t> hang_first;    // unknown -> first hanging id (faces ascending), -1 otherwise
  std::vector<int64_t> corner_set;    // unknowns with > 1 face
  int64_t Np = 0;
  std::vector<int64_t> prime_parent;
  // face bases set by the caller (mss_partition_set_face_bases): per face K_f x M_f row-major, or
  // empty where the DCT reading applies
  std::vector<std::vector<double>> user_bases;
  std::vector<int> user_M;
  // nodes strictly inside cells whose Galerkin lift (Remark MFEM) the off-line stage computes
  // (mss_partition_set_lift_nodes): unknown, cell, and position in the cell's node list
  std::vector<int64_t> lift_unknown;
  std::vector<int> lift_cell;
  std::vector<int64_t> lift_local;

  int faces_of(int64_t u, const int32_t **list) const {
    *list = nf_face.data() + nf_ptr[u];
    return (int)(nf_ptr[u + 1] - nf_ptr[u]);
  }
  void build_cell(int c);
  double cell_node_mass(int c, int64_t u) const;
  double hanging_mass(int64_t u, int f) const;
};

// ------------------------------------------------------------------ ROM (host, FP64 master copy)
struct Rom {
  int n_cells = 0, n_faces = 0;
  std::vector<int32_t> cell_m, cell_face_ptr, cell_faces, face_M, face_cells;
  std::vector<int32_t> cell_K;
  std::vector<int64_t> coef_off;      // per cell, offset of Gamma^1 (and Gamma-hat^1) blocks
  std::vector<double> gamma, gamma_hat;
  std::vector<int64_t> fmass_off;
  std::vector<double> face_mass;
  // projected I/O
  int n_src = 0, n_rcv = 0;
  bool has_io = false;
  std::vector<int32_t> src_face, src_index, rcv_face, rcv_index;
  std::vector<double> src_vals, rcv_vals;    // concatenated M_f values per entry
  // Appendix D
  std::vector<int32_t> cg_ptr, cg_face;
  std::vector<double> cg_rows, cg_weight;
  // face bases (built ROMs only)
  std::vector<int32_t> face_K;
  std::vector<int64_t> basis_off;
  std::vector<double> bases;
  const Partition *source = nullptr;
  // Galerkin lift of the partition's lift nodes (built ROMs): node l of cell lift_cell[l] reads
  // sum_k w_k . U^k with w = lift_w[lift_off[l] ..] (m_c blocks of K_c values, layer 1 first)
  std::vector<int64_t> lift_unknown, lift_off;
  std::vector<int> lift_cell;
  std::vector<double> lift_w;
  // receivers read off hidden layers (layer 2..m of a cell): receiver, cell, layer (1-based),
  // K_c values each, concatenated
  std::vector<int32_t> rcv_h_index, rcv_h_cell, rcv_h_layer;
  std::vector<double> rcv_h_vals;
  mss_rom_params prm{};            // parameters of the off-line construction (built ROMs)

  void finalize_topology();   // validates and fills cell_K, coef_off, fmass_off
};

// face bases: lowest-wavenumber DCT-II modes of a face grid (rows: face nodes, cols: modes)
void face_basis(const Face &f, int n_modes, std::vector<double> &S, int &M);

}  // namespace mss

struct mss_operator { mss::Operator o; };
struct mss_partition { mss::Partition p; };
struct mss_rom { mss::Rom r; };
