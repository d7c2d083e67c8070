// ROM handle: topology, FP64 coefficient master copy, projected I/O, Appendix D data.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.h"

namespace mss {

static thread_local std::string g_last_error;
void set_last_error(const std::string &m) { g_last_error = m; }

// Lowest-wavenumber DCT-II modes of the face node grid (Section 4.1 reading: Neumann modes of
// a uniform face), orthonormal in the Euclidean inner product.  I/O faces: identity.
void face_basis(const Face &f, int n_modes, std::vector<double> &S, int &M) {
  const int K = (int)f.nodes.size();
  if (f.kind == 1) {
    M = K;
    S.assign((size_t)K * K, 0.0);
    for (int i = 0; i < K; ++i) S[(size_t)i * K + i] = 1.0;
    return;
  }
  const int n1 = f.shape[0], n2 = f.shape[1];
  M = std::min(n_modes, K);
  struct Mode { int64_t key; int a, b; };
  std::vector<Mode> modes;
  modes.reserve((size_t)n1 * n2);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) modes.push_back({(int64_t)a * a * n2 * n2 + (int64_t)b * b * n1 * n1, a, b});
  std::stable_sort(modes.begin(), modes.end(), [](const Mode &x, const Mode &y) {
    if (x.key != y.key) return x.key < y.key;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
  });
  auto dct = [](int n, int a, int j) {
    const double c = a == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    return c * std::cos(M_PI * a * (j + 0.5) / n);
  };
  S.assign((size_t)K * M, 0.0);
  for (int k = 0; k < M; ++k)
    for (int j1 = 0; j1 < n1; ++j1)
      for (int j2 = 0; j2 < n2; ++j2)
        S[(size_t)(j1 * n2 + j2) * M + k] = dct(n1, modes[k].a, j1) * dct(n2, modes[k].b, j2);
}

void Rom::finalize_topology() {
  MSS_REQUIRE(n_cells >= 1 && n_faces >= 1, MSS_ERR_INVALID_ARG, "empty topology");
  MSS_REQUIRE((int)cell_m.size() == n_cells && (int)cell_face_ptr.size() == n_cells + 1 &&
                  (int)face_M.size() == n_faces && (int)face_cells.size() == 2 * n_faces,
              MSS_ERR_INVALID_ARG, "topology arrays have wrong sizes");
  MSS_REQUIRE(cell_face_ptr[0] == 0 && (int64_t)cell_faces.size() == cell_face_ptr[n_cells], MSS_ERR_INVALID_ARG,
              "cell_face_ptr inconsistent");
  for (int f = 0; f < n_faces; ++f) {
    MSS_REQUIRE(face_M[f] >= 1, MSS_ERR_INVALID_ARG, "face with no modes");
    MSS_REQUIRE(face_cells[2 * f] >= 0 && face_cells[2 * f] < n_cells && face_cells[2 * f + 1] < n_cells &&
                    face_cells[2 * f + 1] != face_cells[2 * f],
                MSS_ERR_INVALID_ARG, "face cells out of range");
  }
  cell_K.assign(n_cells, 0);
  coef_off.assign(n_cells + 1, 0);
  std::vector<int> seen(n_faces, 0);
  for (int c = 0; c < n_cells; ++c) {
    MSS_REQUIRE(cell_m[c] >= 1, MSS_ERR_INVALID_ARG, "cell with m < 1");
    MSS_REQUIRE(cell_face_ptr[c + 1] > cell_face_ptr[c], MSS_ERR_INVALID_ARG, "cell without faces");
    int K = 0;
    for (int k = cell_face_ptr[c]; k < cell_face_ptr[c + 1]; ++k) {
      const int f = cell_faces[k];
      MSS_REQUIRE(f >= 0 && f < n_faces, MSS_ERR_INVALID_ARG, "face index out of range");
      MSS_REQUIRE(face_cells[2 * f] == c || face_cells[2 * f + 1] == c, MSS_ERR_INVALID_ARG,
                  "cell lists a face that does not list the cell");
      seen[f]++;
      K += face_M[f];
    }
    cell_K[c] = K;
    coef_off[c + 1] = coef_off[c] + (int64_t)cell_m[c] * K * K;
  }
  for (int f = 0; f < n_faces; ++f)
    MSS_REQUIRE(seen[f] == (face_cells[2 * f + 1] >= 0 ? 2 : 1), MSS_ERR_INVALID_ARG,
                "face not listed by exactly its cells");
  fmass_off.assign(n_faces + 1, 0);
  for (int f = 0; f < n_faces; ++f) fmass_off[f + 1] = fmass_off[f] + (int64_t)face_M[f] * face_M[f];
}

// Cholesky check of a symmetric matrix (row-major n x n).
static bool spd(const double *A, int n) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(s > 0)) return false;
    L[(size_t)j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / L[(size_t)j * n + j];
    }
  }
  return true;
}

}  // namespace mss

using namespace mss;

extern "C" {

const char *mss_last_error(void) { return g_last_error.c_str(); }

const char *mss_version(void) { return "mss 0.1 (sm_103a)"; }

const char *mss_status_string(mss_status s) {
  switch (s) {
    case MSS_OK: return "ok";
    case MSS_ERR_INVALID_ARG: return "invalid argument";
    case MSS_ERR_NOT_SPD: return "operator not definite";
    case MSS_ERR_KRYLOV_DEFLATION: return "Krylov deflation";
    case MSS_ERR_LANCZOS_BREAKDOWN: return "block Lanczos breakdown";
    case MSS_ERR_COEF_NOT_SPD: return "S-fraction coefficient not SPD";
    case MSS_ERR_CFL: return "time step above the stability limit";
    case MSS_ERR_TIMEOUT: return "device wait timed out";
    case MSS_ERR_CUDA: return "CUDA error";
    case MSS_ERR_OOM: return "out of memory";
    case MSS_ERR_NOT_CONVERGED: return "iterative solve did not converge";
    case MSS_ERR_STATE: return "invalid state";
    default: return "unknown status";
  }
}

mss_status mss_rom_import(const mss_rom_desc *d, mss_rom **out) {
  return guard([&] {
    MSS_REQUIRE(d && out && d->cell_m && d->cell_face_ptr && d->cell_faces && d->face_M && d->face_cells &&
                    d->gamma && d->gamma_hat && d->face_mass,
                MSS_ERR_INVALID_ARG, "null argument");
    auto h = std::make_unique<mss_rom>();
    Rom &R = h->r;
    R.n_cells = d->n_cells;
    R.n_faces = d->n_faces;
    MSS_REQUIRE(R.n_cells > 0 && R.n_faces > 0, MSS_ERR_INVALID_ARG, "empty topology");
    R.cell_m.assign(d->cell_m, d->cell_m + R.n_cells);
    R.cell_face_ptr.assign(d->cell_face_ptr, d->cell_face_ptr + R.n_cells + 1);
    MSS_REQUIRE(R.cell_face_ptr[R.n_cells] >= 0, MSS_ERR_INVALID_ARG, "cell_face_ptr inconsistent");
    R.cell_faces.assign(d->cell_faces, d->cell_faces + R.cell_face_ptr[R.n_cells]);
    R.face_M.assign(d->face_M, d->face_M + R.n_faces);
    R.face_cells.assign(d->face_cells, d->face_cells + 2 * R.n_faces);
    R.finalize_topology();
    const int64_t nc = R.coef_off[R.n_cells];
    R.gamma.assign(d->gamma, d->gamma + nc);
    R.gamma_hat.assign(d->gamma_hat, d->gamma_hat + nc);
    R.face_mass.assign(d->face_mass, d->face_mass + R.fmass_off[R.n_faces]);
    for (int c = 0; c < R.n_cells; ++c) {
      const int K = R.cell_K[c];
      for (int k = 0; k < R.cell_m[c]; ++k) {
        const double *Gh = R.gamma_hat.data() + R.coef_off[c] + (int64_t)k * K * K;
        MSS_REQUIRE(spd(Gh, K), MSS_ERR_COEF_NOT_SPD, "Gamma-hat^" + std::to_string(k + 1) + " of cell " +
                                                          std::to_string(c) + " is not SPD");
      }
    }
    for (int f = 0; f < R.n_faces; ++f)
      MSS_REQUIRE(spd(R.face_mass.data() + R.fmass_off[f], R.face_M[f]), MSS_ERR_COEF_NOT_SPD,
                  "face mass " + std::to_string(f) + " is not SPD");
    *out = h.release();
  });
}

mss_status mss_rom_info(const mss_rom *r, int64_t info[8]) {
  return guard([&] {
    MSS_REQUIRE(r && info, MSS_ERR_INVALID_ARG, "null argument");
    const Rom &R = r->r;
    info[0] = R.n_cells;
    info[1] = R.n_faces;
    info[2] = *std::max_element(R.cell_K.begin(), R.cell_K.end());
    info[3] = *std::max_element(R.cell_m.begin(), R.cell_m.end());
    info[4] = R.coef_off[R.n_cells];
    info[5] = R.fmass_off[R.n_faces];
    info[6] = std::accumulate(R.face_M.begin(), R.face_M.end(), (int64_t)0);
    info[7] = R.cg_ptr.empty() ? 0 : (int64_t)R.cg_ptr.size() - 1;
  });
}

mss_status mss_rom_export(const mss_rom *r, int32_t *cell_m, int32_t *cell_face_ptr, int32_t *cell_faces,
                          int32_t *face_M, int32_t *face_cells, double *gamma, double *gamma_hat, double *face_mass) {
  return guard([&] {
    MSS_REQUIRE(r, MSS_ERR_INVALID_ARG, "null rom");
    const Rom &R = r->r;
    if (cell_m) std::copy(R.cell_m.begin(), R.cell_m.end(), cell_m);
    if (cell_face_ptr) std::copy(R.cell_face_ptr.begin(), R.cell_face_ptr.end(), cell_face_ptr);
    if (cell_faces) std::copy(R.cell_faces.begin(), R.cell_faces.end(), cell_faces);
    if (face_M) std::copy(R.face_M.begin(), R.face_M.end(), face_M);
    if (face_cells) std::copy(R.face_cells.begin(), R.face_cells.end(), face_cells);
    if (gamma) std::copy(R.gamma.begin(), R.gamma.end(), gamma);
    if (gamma_hat) std::copy(R.gamma_hat.begin(), R.gamma_hat.end(), gamma_hat);
    if (face_mass) std::copy(R.face_mass.begin(), R.face_mass.end(), face_mass);
  });
}

mss_status mss_rom_face_bases(const mss_rom *r, int64_t *count, double *bases) {
  return guard([&] {
    MSS_REQUIRE(r && count, MSS_ERR_INVALID_ARG, "null argument");
    const Rom &R = r->r;
    MSS_REQUIRE(!R.bases.empty(), MSS_ERR_STATE, "ROM has no face bases (imported)");
    *count = (int64_t)R.bases.size();
    if (bases) std::copy(R.bases.begin(), R.bases.end(), bases);
  });
}

mss_status mss_partition_set_face_bases(mss_partition *p, int32_t n_faces, const int32_t *face_M,
                                        const double *bases) {
  return guard([&] {
    MSS_REQUIRE(p, MSS_ERR_INVALID_ARG, "null argument");
    Partition &P = p->p;
    if (n_faces == 0) {
      P.user_bases.clear();
      P.user_M.clear();
      return;
    }
    const int nf = (int)P.faces.size();
    MSS_REQUIRE(n_faces == nf && face_M && bases, MSS_ERR_INVALID_ARG, "need face_M and bases for every face");
    std::vector<std::vector<double>> ub(nf);
    std::vector<int> um(nf, 0);
    size_t o = 0;
    for (int f = 0; f < nf; ++f) {
      const int K = (int)P.faces[f].nodes.size(), M = face_M[f];
      MSS_REQUIRE(M >= 0 && M <= K, MSS_ERR_INVALID_ARG, "face_M[f] must lie in 0..K_f");
      if (M == 0) continue;
      const double *S = bases + o;
      o += (size_t)K * M;
      for (int a = 0; a < M; ++a)
        for (int b = 0; b <= a; ++b) {
          double g = 0.0;
          for (int r = 0; r < K; ++r) g += S[(size_t)r * M + a] * S[(size_t)r * M + b];
          MSS_REQUIRE(std::abs(g - (a == b ? 1.0 : 0.0)) <= 1e-10, MSS_ERR_INVALID_ARG,
                      "face basis columns are not orthonormal");
        }
      ub[f].assign(S, S + (size_t)K * M);
      um[f] = M;
    }
    P.user_bases.swap(ub);
    P.user_M.swap(um);
  });
}

mss_status mss_partition_set_lift_nodes(mss_partition *p, int32_t n, const int32_t *nodes) {
  return guard([&] {
    MSS_REQUIRE(p && n >= 0 && (n == 0 || nodes), MSS_ERR_INVALID_ARG, "bad argument");
    Partition &P = p->p;
    const Operator &o = *P.op;
    std::vector<int64_t> lu, ll;
    std::vector<int> lc;
    int64_t str[3];
    str[o.g.dim - 1] = 1;
    for (int a = o.g.dim - 2; a >= 0; --a) str[a] = str[a + 1] * (o.g.n[a + 1] + 1);
    for (int32_t j = 0; j < n; ++j) {
      int64_t pn = 0;
      int cc[3] = {0, 0, 0};
      for (int a = 0; a < o.g.dim; ++a) {
        const int32_t x = nodes[(int64_t)j * o.g.dim + a];
        MSS_REQUIRE(x >= 0 && x <= o.g.n[a], MSS_ERR_INVALID_ARG, "lift node outside the grid");
        pn += x * str[a];
        cc[a] = std::min(x / P.cs[a], P.nc[a] - 1);
      }
      const int64_t u = o.unknown[pn];
      MSS_REQUIRE(u >= 0, MSS_ERR_INVALID_ARG, "lift node on a Dirichlet wall");
      const int32_t *lst;
      MSS_REQUIRE(P.faces_of(u, &lst) == 0, MSS_ERR_INVALID_ARG,
                  "lift node on a face (skeleton or I/O node): it is read from the face state");
      int c = 0;
      for (int a = 0; a < o.g.dim; ++a) c = c * P.nc[a] + cc[a];
      P.build_cell(c);
      const Cell &C = P.cells[c];
      const int64_t prime = P.plain_prime[u];
      const auto it = std::find(C.nodes.begin(), C.nodes.end(), prime);
      MSS_REQUIRE(it != C.nodes.end() && (int64_t)(it - C.nodes.begin()) >= C.K, MSS_ERR_INVALID_ARG,
                  "lift node is not inside its cell");
      lu.push_back(u);
      lc.push_back(c);
      ll.push_back((int64_t)(it - C.nodes.begin()));
    }
    P.lift_unknown.swap(lu);
    P.lift_cell.swap(lc);
    P.lift_local.swap(ll);
  });
}

mss_status mss_rom_set_io(mss_rom *r, int32_t n_src, int32_t n_src_entries, const int32_t *src_face,
                          const int32_t *src_index, const double *src_vals, int32_t n_rcv, int32_t n_rcv_entries,
                          const int32_t *rcv_face, const int32_t *rcv_index, const double *rcv_vals) {
  return guard([&] {
    MSS_REQUIRE(r, MSS_ERR_INVALID_ARG, "null rom");
    Rom &R = r->r;
    MSS_REQUIRE(n_src >= 1 && n_rcv >= 0 && n_src_entries >= 0 && n_rcv_entries >= 0, MSS_ERR_INVALID_ARG,
                "bad I/O counts");
    MSS_REQUIRE((n_src_entries == 0 || (src_face && src_index && src_vals)) &&
                    (n_rcv_entries == 0 || (rcv_face && rcv_index && rcv_vals)),
                MSS_ERR_INVALID_ARG, "null I/O array");
    std::vector<int32_t> sf, si, rf, ri;
    std::vector<double> sv, rv;
    int64_t o = 0;
    for (int e = 0; e < n_src_entries; ++e) {
      MSS_REQUIRE(src_face[e] >= 0 && src_face[e] < R.n_faces && src_index[e] >= 0 && src_index[e] < n_src,
                  MSS_ERR_INVALID_ARG, "source entry out of range");
      sf.push_back(src_face[e]);
      si.push_back(src_index[e]);
      sv.insert(sv.end(), src_vals + o, src_vals + o + R.face_M[src_face[e]]);
      o += R.face_M[src_face[e]];
    }
    o = 0;
    for (int e = 0; e < n_rcv_entries; ++e) {
      MSS_REQUIRE(rcv_face[e] >= 0 && rcv_face[e] < R.n_faces && rcv_index[e] >= 0 && rcv_index[e] < n_rcv,
                  MSS_ERR_INVALID_ARG, "receiver entry out of range");
      rf.push_back(rcv_face[e]);
      ri.push_back(rcv_index[e]);
      rv.insert(rv.end(), rcv_vals + o, rcv_vals + o + R.face_M[rcv_face[e]]);
      o += R.face_M[rcv_face[e]];
    }
    R.rcv_h_index.clear();
    R.rcv_h_cell.clear();
    R.rcv_h_layer.clear();
    R.rcv_h_vals.clear();
    R.n_src = n_src;
    R.n_rcv = n_rcv;
    R.src_face.swap(sf);
    R.src_index.swap(si);
    R.src_vals.swap(sv);
    R.rcv_face.swap(rf);
    R.rcv_index.swap(ri);
    R.rcv_vals.swap(rv);
    R.has_io = true;
  });
}

mss_status mss_rom_set_io_nodes(mss_rom *r, const mss_partition *p, int32_t n_src, const int32_t *src_nodes,
                                const double *src_w, int32_t n_rcv, const int32_t *rcv_nodes, const double *rcv_w) {
  return guard([&] {
    MSS_REQUIRE(r && p && n_src >= 1 && src_nodes && n_rcv >= 0 && (n_rcv == 0 || rcv_nodes), MSS_ERR_INVALID_ARG,
                "bad argument");
    Rom &R = r->r;
    const Partition &P = p->p;
    MSS_REQUIRE(R.source == &P && !R.bases.empty(), MSS_ERR_STATE, "ROM was not built from this partition");
    const Operator &o = *P.op;
    int64_t ext[3], str[3];
    for (int a = 0; a < 3; ++a) ext[a] = a < o.g.dim ? o.g.n[a] + 1 : 1;
    str[o.g.dim - 1] = 1;
    for (int a = o.g.dim - 2; a >= 0; --a) str[a] = str[a + 1] * ext[a + 1];
    // entries: for each I/O point and each of its prime copies, S_f^T e_row * weight
    std::vector<int32_t> hi, hc, hl;
    std::vector<double> hv;
    auto project = [&](int32_t n, const int32_t *nodes, const double *w, std::vector<int32_t> &fo,
                       std::vector<int32_t> &io, std::vector<double> &vo, bool lift) {
      for (int32_t j = 0; j < n; ++j) {
        int64_t pn = 0;
        for (int a = 0; a < o.g.dim; ++a) {
          const int32_t x = nodes[(int64_t)j * o.g.dim + a];
          MSS_REQUIRE(x >= 0 && x <= o.g.n[a], MSS_ERR_INVALID_ARG, "I/O node outside the grid");
          pn += x * str[a];
        }
        const int64_t u = o.unknown[pn];
        MSS_REQUIRE(u >= 0, MSS_ERR_INVALID_ARG, "I/O node on a Dirichlet wall");
        const int32_t *lst;
        const int nf = P.faces_of(u, &lst);
        if (nf == 0 && lift) {
          // receiver inside a cell: its Galerkin lift, layer 1 as face entries, layers 2..m hidden
          const auto it = std::find(R.lift_unknown.begin(), R.lift_unknown.end(), u);
          MSS_REQUIRE(it != R.lift_unknown.end(), MSS_ERR_INVALID_ARG,
                      "receiver inside a cell is neither an I/O node nor a lift node of the build");
          const int l = (int)(it - R.lift_unknown.begin()), c = R.lift_cell[l];
          const int K = R.cell_K[c], m = R.cell_m[c];
          const double *wl = R.lift_w.data() + R.lift_off[l];
          const double ww = w ? w[j] : 1.0;
          int o = 0;
          for (int k = R.cell_face_ptr[c]; k < R.cell_face_ptr[c + 1]; ++k) {
            const int f = R.cell_faces[k], M = R.face_M[f];
            fo.push_back(f);
            io.push_back(j);
            for (int q = 0; q < M; ++q) vo.push_back(wl[o + q] * ww);
            o += M;
          }
          for (int k = 2; k <= m; ++k) {
            hi.push_back(j);
            hc.push_back(c);
            hl.push_back(k);
            for (int q = 0; q < K; ++q) hv.push_back(wl[(int64_t)(k - 1) * K + q] * ww);
          }
          continue;
        }
        MSS_REQUIRE(nf >= 1, MSS_ERR_INVALID_ARG,
                    "I/O node inside a cell was not given to mss_partition_create");
        std::vector<double> wt(nf, 1.0);
        if (nf > 1) {
          double tot = 0;
          for (int k = 0; k < nf; ++k) tot += (wt[k] = P.hanging_mass(u, lst[k]));
          for (auto &x : wt) x /= tot;
        }
        const double ww = w ? w[j] : 1.0;
        for (int k = 0; k < nf; ++k) {
          const int f = lst[k];
          const Face &F = P.faces[f];
          const int64_t prime = nf > 1 ? P.hang_first[u] + k : P.plain_prime[u];
          const int row = (int)(std::find(F.nodes.begin(), F.nodes.end(), prime) - F.nodes.begin());
          const int M = R.face_M[f];
          const double *S = R.bases.data() + R.basis_off[f];
          fo.push_back(f);
          io.push_back(j);
          for (int c = 0; c < M; ++c) vo.push_back(S[(int64_t)row * M + c] * wt[k] * ww);
        }
      }
    };
    std::vector<int32_t> sf, si, rf, ri;
    std::vector<double> sv, rv;
    project(n_src, src_nodes, src_w, sf, si, sv, false);
    project(n_rcv, rcv_nodes, rcv_w, rf, ri, rv, true);
    R.rcv_h_index.swap(hi);
    R.rcv_h_cell.swap(hc);
    R.rcv_h_layer.swap(hl);
    R.rcv_h_vals.swap(hv);
    R.n_src = n_src;
    R.n_rcv = n_rcv;
    R.src_face.swap(sf);
    R.src_index.swap(si);
    R.src_vals.swap(sv);
    R.rcv_face.swap(rf);
    R.rcv_index.swap(ri);
    R.rcv_vals.swap(rv);
    R.has_io = true;
  });
}

mss_status mss_rom_set_corners(mss_rom *r, int32_t n_groups, const int32_t *group_ptr, const int32_t *face,
                               const double *rows, const double *weight) {
  return guard([&] {
    MSS_REQUIRE(r && n_groups >= 0, MSS_ERR_INVALID_ARG, "bad argument");
    Rom &R = r->r;
    if (n_groups == 0) {
      R.cg_ptr.clear();
      R.cg_face.clear();
      R.cg_rows.clear();
      R.cg_weight.clear();
      return;
    }
    MSS_REQUIRE(group_ptr && face && rows && weight && group_ptr[0] == 0, MSS_ERR_INVALID_ARG, "null corner array");
    const int32_t ne = group_ptr[n_groups];
    int64_t nr = 0;
    for (int e = 0; e < ne; ++e) {
      MSS_REQUIRE(face[e] >= 0 && face[e] < R.n_faces, MSS_ERR_INVALID_ARG, "corner face out of range");
      nr += R.face_M[face[e]];
    }
    R.cg_ptr.assign(group_ptr, group_ptr + n_groups + 1);
    R.cg_face.assign(face, face + ne);
    R.cg_rows.assign(rows, rows + nr);
    R.cg_weight.assign(weight, weight + ne);
  });
}

mss_status mss_rom_export_io(const mss_rom *r, int64_t counts[9], int32_t *src_face, int32_t *src_index,
                             double *src_vals, int32_t *rcv_face, int32_t *rcv_index, double *rcv_vals,
                             int32_t *group_ptr, int32_t *member_face, double *member_rows, double *member_weight) {
  return guard([&] {
    MSS_REQUIRE(r && counts, MSS_ERR_INVALID_ARG, "null argument");
    const Rom &R = r->r;
    const int64_t ng = R.cg_ptr.empty() ? 0 : (int64_t)R.cg_ptr.size() - 1;
    const int64_t c[9] = {R.n_src, (int64_t)R.src_face.size(), (int64_t)R.src_vals.size(), R.n_rcv,
                          (int64_t)R.rcv_face.size(), (int64_t)R.rcv_vals.size(), ng, (int64_t)R.cg_face.size(),
                          (int64_t)R.cg_rows.size()};
    std::copy(c, c + 9, counts);
    auto put = [](auto *dst, const auto &v) {
      if (dst) std::copy(v.begin(), v.end(), dst);
    };
    put(src_face, R.src_face);
    put(src_index, R.src_index);
    put(src_vals, R.src_vals);
    put(rcv_face, R.rcv_face);
    put(rcv_index, R.rcv_index);
    put(rcv_vals, R.rcv_vals);
    put(group_ptr, R.cg_ptr);
    put(member_face, R.cg_face);
    put(member_rows, R.cg_rows);
    put(member_weight, R.cg_weight);
  });
}

void mss_rom_destroy(mss_rom *r) { delete r; }

}  // extern "C"
