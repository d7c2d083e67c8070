// Fine-grid assembly (Section 1) and box partition with corner-set removal
// (Section 2 Eq. splitN_c, Section 3 Eq. nocorners, Appendix B), host side, FP64.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <unordered_map>

#include "common.h"

namespace mss {

namespace {

// Node-grid strides of a grid (array order, last axis fastest).
void node_strides(const mss_grid &g, int64_t ext[3], int64_t str[3]) {
  for (int a = 0; a < 3; ++a) ext[a] = a < g.dim ? g.n[a] + 1 : 1;
  str[g.dim - 1] = 1;
  for (int a = g.dim - 2; a >= 0; --a) str[a] = str[a + 1] * ext[a + 1];
}

bool wall_removed(const mss_grid &g, int a, int64_t p) {
  return (p == 0 && g.bc[a][0] == MSS_DIRICHLET) || (p == g.n[a] && g.bc[a][1] == MSS_DIRICHLET);
}

}  // namespace

// ------------------------------------------------------------------ assembly
static void assemble(Operator &o, const mss_grid &g, const double *sigma, const double *rho) {
  MSS_REQUIRE(g.dim >= 1 && g.dim <= 3, MSS_ERR_INVALID_ARG, "grid dim must be 1..3");
  MSS_REQUIRE(g.h > 0 && std::isfinite(g.h), MSS_ERR_INVALID_ARG, "grid step must be positive");
  int64_t nvox = 1;
  for (int a = 0; a < g.dim; ++a) {
    MSS_REQUIRE(g.n[a] >= 1, MSS_ERR_INVALID_ARG, "voxel counts must be >= 1");
    for (int s = 0; s < 2; ++s)
      MSS_REQUIRE(g.bc[a][s] == MSS_DIRICHLET || g.bc[a][s] == MSS_NEUMANN, MSS_ERR_INVALID_ARG, "bad wall type");
    nvox *= g.n[a];
  }
  for (int64_t v = 0; v < nvox; ++v)
    MSS_REQUIRE(sigma[v] > 0 && rho[v] > 0 && std::isfinite(sigma[v]) && std::isfinite(rho[v]), MSS_ERR_NOT_SPD,
                "sigma and rho must be positive and finite");
  o.g = g;
  int64_t ext[3], str[3];
  node_strides(g, ext, str);
  for (int a = 0; a < 3; ++a) o.nshape[a] = ext[a];
  o.nodes = ext[0] * ext[1] * ext[2];
  const int d = g.dim;
  // per-node forward edge weights along each axis and lumped masses
  std::vector<double> E[3];
  for (int a = 0; a < d; ++a) E[a].assign(o.nodes, 0.0);
  std::vector<double> mass(o.nodes, 0.0);
  const double wfac = std::pow(g.h, d - 2) / double(1 << (d - 1));
  const double mfac = std::pow(g.h, d) / double(1 << d);
  int64_t vext[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) vext[a] = g.n[a];
  int64_t v = 0;
  for (int64_t i0 = 0; i0 < vext[0]; ++i0)
    for (int64_t i1 = 0; i1 < vext[1]; ++i1)
      for (int64_t i2 = 0; i2 < vext[2]; ++i2, ++v) {
        const int64_t base = i0 * str[0] + (d > 1 ? i1 * str[1] : 0) + (d > 2 ? i2 * str[2] : 0);
        const double w = sigma[v] * wfac, mv = rho[v] * mfac;
        for (int corner = 0; corner < (1 << d); ++corner) {
          int64_t p = base;
          for (int a = 0; a < d; ++a)
            if (corner >> a & 1) p += str[a];
          mass[p] += mv;
          for (int a = 0; a < d; ++a)
            if (!(corner >> a & 1)) E[a][p] += w;   // edge from this corner along +a stays in the voxel
        }
      }
  // unknown numbering
  o.unknown.assign(o.nodes, -1);
  o.node_of.clear();
  for (int64_t p = 0; p < o.nodes; ++p) {
    int64_t rem = p;
    bool keep = true;
    for (int a = 0; a < d; ++a) {
      int64_t c = rem / str[a];
      rem -= c * str[a];
      if (wall_removed(g, a, c)) keep = false;
    }
    if (keep) {
      o.unknown[p] = (int64_t)o.node_of.size();
      o.node_of.push_back(p);
    }
  }
  o.N = (int64_t)o.node_of.size();
  o.B.resize(o.N);
  o.A.n = o.N;
  o.A.ptr.assign(o.N + 1, 0);
  o.A.col.clear();
  o.A.val.clear();
  o.A.col.reserve(o.N * (2 * d + 1));
  o.A.val.reserve(o.N * (2 * d + 1));
  for (int64_t u = 0; u < o.N; ++u) {
    const int64_t p = o.node_of[u];
    o.B[u] = mass[p];
    int64_t coord[3] = {0, 0, 0};
    int64_t rem = p;
    for (int a = 0; a < d; ++a) {
      coord[a] = rem / str[a];
      rem -= coord[a] * str[a];
    }
    double diag = 0.0;
    // lower neighbours (largest stride first), the node, upper neighbours -> ascending columns
    struct Ent { int64_t c; double w; };
    Ent lo[3], hi[3];
    int nlo = 0, nhi = 0;
    for (int a = 0; a < d; ++a) {
      if (coord[a] > 0) {
        const double w = E[a][p - str[a]];
        diag -= w;
        const int64_t q = o.unknown[p - str[a]];
        if (q >= 0) lo[nlo++] = {q, w};
      }
      if (coord[a] < g.n[a]) {
        const double w = E[a][p];
        diag -= w;
        const int64_t q = o.unknown[p + str[a]];
        if (q >= 0) hi[nhi++] = {q, w};
      }
    }
    for (int i = 0; i < nlo; ++i) { o.A.col.push_back(lo[i].c); o.A.val.push_back(lo[i].w); }
    o.A.col.push_back(u);
    o.A.val.push_back(diag);
    for (int i = nhi - 1; i >= 0; --i) { o.A.col.push_back(hi[i].c); o.A.val.push_back(hi[i].w); }
    o.A.ptr[u + 1] = (int64_t)o.A.col.size();
  }
}

// ------------------------------------------------------------------ elastic assembly
// Element stiffness of a voxel of edge h for each unit Voigt entry: Eab[a][b] (24 x 24, dof 3 c + p
// = displacement component p, physical axis, at corner c in C order over the array axes) is
// the integral over the voxel of sum_{q,s} T_pqrs dN_c/dx_q dN_d/dx_s with T the stiffness tensor
// of the Voigt matrix whose only non-zero entry is (a, b).  Trilinear N_c: the 2 x 2 x 2 Gauss rule
// integrates these products (quadratic per axis) exactly.  Array axis a is physical axis 2 - a.
static void elastic_unit_stiffness(double h, std::vector<double> &Eab) {
  static const int vo[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};   // Voigt index of (i, j), physical
  Eab.assign((size_t)36 * 576, 0.0);
  const double g[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  const double w = h * h * h / 8.0;
  for (int gp = 0; gp < 8; ++gp) {
    const double xi[3] = {g[gp >> 2 & 1], g[gp >> 1 & 1], g[gp & 1]};   // array axes 0, 1, 2
    double G[8][3];                                                       // [corner][physical axis]
    for (int c = 0; c < 8; ++c) {
      const int cc[3] = {c >> 2 & 1, c >> 1 & 1, c & 1};
      double f[3];
      for (int a = 0; a < 3; ++a) f[a] = cc[a] ? xi[a] : 1.0 - xi[a];
      for (int a = 0; a < 3; ++a) G[c][2 - a] = (cc[a] ? 1.0 : -1.0) / h * f[(a + 1) % 3] * f[(a + 2) % 3];
    }
    for (int c = 0; c < 8; ++c)
      for (int d = 0; d < 8; ++d)
        for (int pp = 0; pp < 3; ++pp)
          for (int q = 0; q < 3; ++q)
            for (int r = 0; r < 3; ++r)
              for (int t = 0; t < 3; ++t) {
                const int a = vo[pp][q], bb = vo[r][t];
                Eab[((size_t)a * 6 + bb) * 576 + (size_t)(3 * c + pp) * 24 + 3 * d + r] += w * G[c][q] * G[d][t];
              }
  }
}

static void assemble_elastic(Operator &o, const mss_grid &g, const double *Cv, const double *rho) {
  MSS_REQUIRE(g.dim == 3, MSS_ERR_INVALID_ARG, "the elastic operator is 3D");
  MSS_REQUIRE(g.h > 0 && std::isfinite(g.h), MSS_ERR_INVALID_ARG, "grid step must be positive");
  int64_t nvox = 1;
  for (int a = 0; a < 3; ++a) {
    MSS_REQUIRE(g.n[a] >= 1, MSS_ERR_INVALID_ARG, "voxel counts must be >= 1");
    for (int sd = 0; sd < 2; ++sd)
      MSS_REQUIRE(g.bc[a][sd] == MSS_DIRICHLET || g.bc[a][sd] == MSS_NEUMANN, MSS_ERR_INVALID_ARG, "bad wall type");
    nvox *= g.n[a];
  }
  for (int64_t v = 0; v < nvox; ++v) {
    const double *C = Cv + v * 36;
    double L[36] = {0};
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        MSS_REQUIRE(std::isfinite(C[i * 6 + j]), MSS_ERR_NOT_SPD, "stiffness entries must be finite");
        MSS_REQUIRE(std::fabs(C[i * 6 + j] - C[j * 6 + i]) <= 1e-12 * (std::fabs(C[i * 6 + j]) + std::fabs(C[j * 6 + i])),
                    MSS_ERR_INVALID_ARG, "Voigt stiffness must be symmetric");
      }
    // positive definite: Cholesky of the 6 x 6 Voigt matrix
    for (int j = 0; j < 6; ++j) {
      double dj = C[j * 6 + j];
      for (int k = 0; k < j; ++k) dj -= L[j * 6 + k] * L[j * 6 + k];
      MSS_REQUIRE(dj > 0, MSS_ERR_NOT_SPD, "Voigt stiffness must be positive definite");
      L[j * 6 + j] = std::sqrt(dj);
      for (int i = j + 1; i < 6; ++i) {
        double x = C[i * 6 + j];
        for (int k = 0; k < j; ++k) x -= L[i * 6 + k] * L[j * 6 + k];
        L[i * 6 + j] = x / L[j * 6 + j];
      }
    }
    MSS_REQUIRE(rho[v] > 0 && std::isfinite(rho[v]), MSS_ERR_NOT_SPD, "rho must be positive and finite");
  }
  o.g = g;
  int64_t ext[3], str[3];
  node_strides(g, ext, str);
  for (int a = 0; a < 3; ++a) o.nshape[a] = ext[a];
  o.nodes = ext[0] * ext[1] * ext[2];
  o.comps = 3;
  // kept nodes (the scalar rule) and their numbers k; unknown 3 k + p
  std::vector<int64_t> kept(o.nodes, -1), knode;
  for (int64_t p = 0; p < o.nodes; ++p) {
    const int64_t c0 = p / str[0], c1 = (p - c0 * str[0]) / str[1], c2 = p - c0 * str[0] - c1 * str[1];
    if (wall_removed(g, 0, c0) || wall_removed(g, 1, c1) || wall_removed(g, 2, c2)) continue;
    kept[p] = (int64_t)knode.size();
    knode.push_back(p);
  }
  const int64_t nk = (int64_t)knode.size();
  o.N = 3 * nk;
  o.unknown.assign(o.nodes, -1);
  o.node_of.assign(o.N, 0);
  for (int64_t k = 0; k < nk; ++k) {
    o.unknown[knode[k]] = 3 * k;
    for (int p = 0; p < 3; ++p) o.node_of[3 * k + p] = knode[k];
  }
  // CSR structure: row 3k + p holds the three components of every kept node within one step along
  // each axis (ascending node order = ascending columns); slot[27 k + offset] = that node's place
  std::vector<int8_t> slot((size_t)27 * nk, -1);
  o.A.n = o.N;
  o.A.ptr.assign(o.N + 1, 0);
  std::vector<int64_t> nb;
  for (int64_t k = 0; k < nk; ++k) {
    const int64_t p = knode[k];
    const int64_t c[3] = {p / str[0], (p % str[0]) / str[1], p % str[1]};
    int cnt = 0;
    for (int o27 = 0; o27 < 27; ++o27) {
      const int d[3] = {o27 / 9 - 1, (o27 / 3) % 3 - 1, o27 % 3 - 1};
      bool in = true;
      for (int a = 0; a < 3; ++a) in = in && c[a] + d[a] >= 0 && c[a] + d[a] <= g.n[a];
      if (!in) continue;
      const int64_t q = p + d[0] * str[0] + d[1] * str[1] + d[2] * str[2];
      if (kept[q] < 0) continue;
      slot[(size_t)27 * k + o27] = (int8_t)cnt++;
      nb.push_back(kept[q]);
    }
    for (int pp = 0; pp < 3; ++pp) o.A.ptr[3 * k + pp + 1] = 3 * cnt;
  }
  for (int64_t u = 0; u < o.N; ++u) o.A.ptr[u + 1] += o.A.ptr[u];
  o.A.col.assign(o.A.ptr[o.N], 0);
  o.A.val.assign(o.A.ptr[o.N], 0.0);
  {
    int64_t off = 0;
    for (int64_t k = 0; k < nk; ++k) {
      const int cnt = (int)((o.A.ptr[3 * k + 1] - o.A.ptr[3 * k]) / 3);
      for (int pp = 0; pp < 3; ++pp)
        for (int i = 0; i < cnt; ++i)
          for (int r = 0; r < 3; ++r) o.A.col[o.A.ptr[3 * k + pp] + 3 * i + r] = 3 * nb[off + i] + r;
      off += cnt;
    }
  }
  // A = -K voxel by voxel: K_e = sum over the symmetric Voigt pairs of C_ab (E_ab + E_ba) (a < b)
  std::vector<double> Eab;
  elastic_unit_stiffness(g.h, Eab);
  std::vector<double> mass(o.nodes, 0.0), Ke(576);
  const double mfac = g.h * g.h * g.h / 8.0;
  int64_t v = 0;
  for (int64_t i0 = 0; i0 < g.n[0]; ++i0)
    for (int64_t i1 = 0; i1 < g.n[1]; ++i1)
      for (int64_t i2 = 0; i2 < g.n[2]; ++i2, ++v) {
        const double *C = Cv + v * 36;
        std::fill(Ke.begin(), Ke.end(), 0.0);
        for (int a = 0; a < 6; ++a)
          for (int bb = a; bb < 6; ++bb) {
            const double cab = C[a * 6 + bb];
            if (cab == 0.0) continue;
            const double *E1 = Eab.data() + ((size_t)a * 6 + bb) * 576;
            const double *E2 = Eab.data() + ((size_t)bb * 6 + a) * 576;
            if (a == bb)
              for (int i = 0; i < 576; ++i) Ke[i] += cab * E1[i];
            else
              for (int i = 0; i < 576; ++i) Ke[i] += cab * (E1[i] + E2[i]);
          }
        const int64_t base = i0 * str[0] + i1 * str[1] + i2 * str[2];
        int64_t cn[8];
        for (int c = 0; c < 8; ++c) {
          const int64_t q = base + (c >> 2 & 1) * str[0] + (c >> 1 & 1) * str[1] + (c & 1) * str[2];
          mass[q] += rho[v] * mfac;
          cn[c] = kept[q];
        }
        for (int c = 0; c < 8; ++c) {
          if (cn[c] < 0) continue;
          for (int d = 0; d < 8; ++d) {
            if (cn[d] < 0) continue;
            const int o27 = ((d >> 2 & 1) - (c >> 2 & 1) + 1) * 9 + ((d >> 1 & 1) - (c >> 1 & 1) + 1) * 3 +
                            ((d & 1) - (c & 1) + 1);
            const int sl = slot[(size_t)27 * cn[c] + o27];
            for (int pp = 0; pp < 3; ++pp) {
              double *row = o.A.val.data() + o.A.ptr[3 * cn[c] + pp] + 3 * sl;
              for (int r = 0; r < 3; ++r) row[r] -= Ke[(size_t)(3 * c + pp) * 24 + 3 * d + r];
            }
          }
        }
      }
  o.B.assign(o.N, 0.0);
  for (int64_t k = 0; k < nk; ++k)
    for (int pp = 0; pp < 3; ++pp) o.B[3 * k + pp] = mass[knode[k]];
}

static double lambda_max_lanczos(const Operator &o, double tol) {
  // Lanczos on B^{-1/2}(-A)B^{-1/2}; returns the largest Ritz value once it settles.
  const int64_t N = o.N;
  std::vector<double> sb(N), q(N), qo(N, 0.0), w(N);
  for (int64_t i = 0; i < N; ++i) sb[i] = 1.0 / std::sqrt(o.B[i]);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  double nrm = 0;
  for (int64_t i = 0; i < N; ++i) {
    st ^= st << 13; st ^= st >> 7; st ^= st << 17;
    q[i] = double(st >> 11) / double(1ull << 53) - 0.5;
    nrm += q[i] * q[i];
  }
  nrm = std::sqrt(nrm);
  for (auto &x : q) x /= nrm;
  std::vector<double> al, be;
  double prev = 0, beta = 0;
  const int maxit = (int)std::min<int64_t>(N, 400);
  for (int it = 0; it < maxit; ++it) {
    for (int64_t i = 0; i < N; ++i) {
      double s = 0;
      for (int64_t k = o.A.ptr[i]; k < o.A.ptr[i + 1]; ++k) s += o.A.val[k] * sb[o.A.col[k]] * q[o.A.col[k]];
      w[i] = -sb[i] * s;
    }
    double a = 0;
    for (int64_t i = 0; i < N; ++i) a += w[i] * q[i];
    for (int64_t i = 0; i < N; ++i) w[i] -= a * q[i] + beta * qo[i];
    al.push_back(a);
    double b = 0;
    for (int64_t i = 0; i < N; ++i) b += w[i] * w[i];
    b = std::sqrt(b);
    // largest eigenvalue of the tridiagonal (bisection on Sturm counts)
    const int n = (int)al.size();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      double r = (i > 0 ? std::fabs(be[i - 1]) : 0) + (i + 1 < n ? std::fabs(i < (int)be.size() ? be[i] : 0) : 0);
      lo = std::min(lo, al[i] - r - std::fabs(b));
      hi = std::max(hi, al[i] + r + std::fabs(b));
    }
    for (int k = 0; k < 200; ++k) {
      const double mid = 0.5 * (lo + hi);
      int cnt = 0;
      double dd = 1.0;
      for (int i = 0; i < n; ++i) {
        const double bb = i > 0 ? be[i - 1] : 0.0;
        dd = al[i] - mid - (i > 0 ? bb * bb / dd : 0.0);
        if (dd == 0) dd = 1e-300;
        if (dd < 0) ++cnt;
      }
      if (cnt == n) hi = mid; else lo = mid;   // cnt = eigenvalues below mid
    }
    const double lam = 0.5 * (lo + hi);
    if (it > 20 && std::fabs(lam - prev) <= tol * lam) return lam;
    prev = lam;
    if (b < 1e-300) return lam;
    be.push_back(b);
    beta = b;
    qo = q;
    for (int64_t i = 0; i < N; ++i) q[i] = w[i] / b;
  }
  return prev;
}

// ------------------------------------------------------------------ partition
static void partition(Partition &P, const Operator &o, const double *sigma, const double *rho,
                      const int32_t *cell, int32_t n_io, const int32_t *io) {
  const mss_grid &g = o.g;
  const int d = g.dim;
  P.op = &o;
  P.d = d;
  int64_t nvox = 1;
  for (int a = 0; a < d; ++a) nvox *= g.n[a];
  P.sigma.assign(sigma, sigma + nvox);
  P.rho.assign(rho, rho + nvox);
  P.n_cells = 1;
  for (int a = 0; a < 3; ++a) {
    P.cs[a] = a < d ? cell[a] : 1;
    if (a < d) {
      MSS_REQUIRE(cell[a] >= 2 && g.n[a] % cell[a] == 0, MSS_ERR_INVALID_ARG,
                  "cell size must be >= 2 and divide the voxel count");
      P.nc[a] = g.n[a] / cell[a];
    } else {
      P.nc[a] = 1;
    }
    P.n_cells *= P.nc[a];
  }
  int64_t ext[3], str[3];
  node_strides(g, ext, str);
  auto cell_id = [&](const int C[3]) { return (C[0] * P.nc[1] + C[1]) * P.nc[2] + C[2]; };
  P.cells.assign(P.n_cells, Cell());
  for (int c = 0; c < P.n_cells; ++c) {
    P.cells[c].coords[0] = c / (P.nc[1] * P.nc[2]);
    P.cells[c].coords[1] = (c / P.nc[2]) % P.nc[1];
    P.cells[c].coords[2] = c % P.nc[2];
  }
  // interior faces, axis-major, lower cell in C order
  P.faces.clear();
  std::vector<int64_t> cnt(o.N + 1, 0);
  for (int a = 0; a < d; ++a) {
    for (int c = 0; c < P.n_cells; ++c) {
      const int *C = P.cells[c].coords;
      if (C[a] + 1 >= P.nc[a]) continue;
      Face f;
      f.kind = 0;
      f.axis = a;
      int C1[3] = {C[0], C[1], C[2]};
      C1[a] += 1;
      f.cells[0] = c;
      f.cells[1] = cell_id(C1);
      // tangential ranges of kept node coordinates
      std::vector<int64_t> rng[3];
      for (int b = 0; b < d; ++b) {
        if (b == a) {
          rng[b].push_back((int64_t)P.cs[a] * (C[a] + 1));
        } else {
          for (int64_t p = (int64_t)P.cs[b] * C[b]; p <= (int64_t)P.cs[b] * (C[b] + 1); ++p)
            if (!wall_removed(g, b, p)) rng[b].push_back(p);
        }
      }
      for (int b = d; b < 3; ++b) rng[b].push_back(0);
      int t = 0;
      for (int b = 0; b < d; ++b)
        if (b != a) f.shape[t++] = (int)rng[b].size();
      for (int64_t x0 : rng[0])
        for (int64_t x1 : rng[1])
          for (int64_t x2 : rng[2]) {
            const int64_t p = x0 * str[0] + (d > 1 ? x1 * str[1] : 0) + (d > 2 ? x2 * str[2] : 0);
            const int64_t u = o.unknown[p];
            MSS_REQUIRE(u >= 0, MSS_ERR_INVALID_ARG, "internal: removed node on a face");
            f.parents.push_back(u);
            cnt[u + 1]++;
          }
      P.faces.push_back(std::move(f));
    }
  }
  P.n_int_faces = (int)P.faces.size();
  // I/O nodes strictly inside one cell
  std::map<int, std::vector<int64_t>> io_cell;
  for (int32_t k = 0; k < n_io; ++k) {
    int64_t p = 0;
    int C[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      const int32_t x = io[(int64_t)k * d + a];
      MSS_REQUIRE(x >= 0 && x <= g.n[a], MSS_ERR_INVALID_ARG, "I/O node outside the grid");
      p += x * str[a];
      C[a] = std::min(x / P.cs[a], P.nc[a] - 1);
    }
    const int64_t u = o.unknown[p];
    MSS_REQUIRE(u >= 0, MSS_ERR_INVALID_ARG, "I/O node on a Dirichlet wall");
    if (cnt[u + 1] > 0) continue;                         // carried by an interior face
    auto &lst = io_cell[cell_id(C)];
    if (std::find(lst.begin(), lst.end(), u) == lst.end()) lst.push_back(u);
  }
  for (auto &kv : io_cell) {
    Face f;
    f.kind = 1;
    f.cells[0] = kv.first;
    std::sort(kv.second.begin(), kv.second.end());
    f.parents = kv.second;
    f.shape[0] = (int)f.parents.size();
    for (int64_t u : f.parents) cnt[u + 1]++;
    P.faces.push_back(std::move(f));
  }
  for (int fi = 0; fi < (int)P.faces.size(); ++fi)
    for (int s = 0; s < 2; ++s)
      if (P.faces[fi].cells[s] >= 0) P.cells[P.faces[fi].cells[s]].faces.push_back(fi);
  // faces per unknown
  P.nf_ptr.assign(o.N + 1, 0);
  for (int64_t u = 0; u < o.N; ++u) P.nf_ptr[u + 1] = P.nf_ptr[u] + cnt[u + 1];
  P.nf_face.assign(P.nf_ptr[o.N], 0);
  std::vector<int64_t> fill(P.nf_ptr.begin(), P.nf_ptr.end() - 1);
  for (int fi = 0; fi < (int)P.faces.size(); ++fi)
    for (int64_t u : P.faces[fi].parents) P.nf_face[fill[u]++] = fi;   // faces visited ascending
  // prime numbering
  P.plain_prime.assign(o.N, -1);
  P.hang_first.assign(o.N, -1);
  P.corner_set.clear();
  int64_t next = 0;
  for (int64_t u = 0; u < o.N; ++u) {
    if (P.nf_ptr[u + 1] - P.nf_ptr[u] > 1) P.corner_set.push_back(u);
    else P.plain_prime[u] = next++;
  }
  P.prime_parent.assign(next, 0);
  for (int64_t u = 0; u < o.N; ++u)
    if (P.plain_prime[u] >= 0) P.prime_parent[P.plain_prime[u]] = u;
  for (int64_t u : P.corner_set) {
    P.hang_first[u] = next;
    for (int64_t k = P.nf_ptr[u]; k < P.nf_ptr[u + 1]; ++k) P.prime_parent.push_back(u);
    next += P.nf_ptr[u + 1] - P.nf_ptr[u];
  }
  P.Np = next;
  for (int fi = 0; fi < (int)P.faces.size(); ++fi) {
    Face &f = P.faces[fi];
    f.nodes.resize(f.parents.size());
    for (size_t k = 0; k < f.parents.size(); ++k) {
      const int64_t u = f.parents[k];
      if (P.plain_prime[u] >= 0) {
        f.nodes[k] = P.plain_prime[u];
      } else {
        const int32_t *lst;
        const int n = P.faces_of(u, &lst);
        const int pos = (int)(std::find(lst, lst + n, fi) - lst);
        f.nodes[k] = P.hang_first[u] + pos;
      }
    }
  }
}

// Cell share of the mass of unknown u (voxels of cell c touching u).
double Partition::cell_node_mass(int c, int64_t u) const {
  const mss_grid &g = op->g;
  int64_t ext[3], str[3];
  node_strides(g, ext, str);
  int64_t p = op->node_of[u], coord[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    coord[a] = p / str[a];
    p -= coord[a] * str[a];
  }
  const int *C = cells[c].coords;
  double m = 0;
  for (int corner = 0; corner < (1 << d); ++corner) {
    int64_t vi[3] = {0, 0, 0};
    bool in = true;
    for (int a = 0; a < d; ++a) {
      vi[a] = coord[a] - ((corner >> a) & 1);
      if (vi[a] < (int64_t)cs[a] * C[a] || vi[a] >= (int64_t)cs[a] * (C[a] + 1)) in = false;
    }
    if (!in) continue;
    int64_t v = 0;
    for (int a = 0; a < d; ++a) v = v * g.n[a] + vi[a];
    m += rho[v] * std::pow(g.h, d) / double(1 << d);
  }
  return m;
}

// b'_{k_f}: each cell of face f holding u gives its share divided by its faces holding u.
double Partition::hanging_mass(int64_t u, int f) const {
  double m = 0;
  const int32_t *lst;
  const int n = faces_of(u, &lst);
  for (int s = 0; s < 2; ++s) {
    const int c = faces[f].cells[s];
    if (c < 0) continue;
    int held = 0;
    for (int k = 0; k < n; ++k) {
      const Face &ff = faces[lst[k]];
      if (ff.cells[0] == c || ff.cells[1] == c) ++held;
    }
    m += cell_node_mass(c, u) / held;
  }
  return m;
}

void Partition::build_cell(int c) {
  Cell &cl = cells[c];
  if (cl.built) return;
  const mss_grid &g = op->g;
  int64_t ext[3], str[3];
  node_strides(g, ext, str);
  const int *C = cl.coords;
  int64_t lext[3] = {1, 1, 1}, lstr[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) lext[a] = cs[a] + 1;
  for (int a = d - 2; a >= 0; --a) lstr[a] = lstr[a + 1] * lext[a + 1];
  if (d >= 1) lstr[d - 1] = 1;
  const int64_t nloc = lext[0] * lext[1] * lext[2];
  // local node -> unknown
  std::vector<int64_t> loc(nloc, -1);
  for (int64_t l = 0; l < nloc; ++l) {
    int64_t rem = l, p = 0;
    for (int a = 0; a < d; ++a) {
      const int64_t q = rem / lstr[a];
      rem -= q * lstr[a];
      p += ((int64_t)cs[a] * C[a] + q) * str[a];
    }
    loc[l] = op->unknown[p];
  }
  // edge weights and masses contributed by this cell's voxels
  std::vector<double> E[3];
  for (int a = 0; a < d; ++a) E[a].assign(nloc, 0.0);
  std::vector<double> mass(nloc, 0.0);
  const double wfac = std::pow(g.h, d - 2) / double(1 << (d - 1));
  const double mfac = std::pow(g.h, d) / double(1 << d);
  int64_t vext[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) vext[a] = cs[a];
  for (int64_t i0 = 0; i0 < vext[0]; ++i0)
    for (int64_t i1 = 0; i1 < vext[1]; ++i1)
      for (int64_t i2 = 0; i2 < vext[2]; ++i2) {
        const int64_t iv[3] = {i0, i1, i2};
        int64_t v = 0, base = 0;
        for (int a = 0; a < d; ++a) {
          v = v * g.n[a] + (int64_t)cs[a] * C[a] + iv[a];
          base += iv[a] * lstr[a];
        }
        const double w = sigma[v] * wfac, mv = rho[v] * mfac;
        for (int corner = 0; corner < (1 << d); ++corner) {
          int64_t l = base;
          for (int a = 0; a < d; ++a)
            if (corner >> a & 1) l += lstr[a];
          mass[l] += mv;
          for (int a = 0; a < d; ++a)
            if (!(corner >> a & 1)) E[a][l] += w;
        }
      }
  // faces of this cell holding unknown u, as hanging ids (corner nodes) or the plain id
  auto copies = [&](int64_t u, std::vector<int64_t> &out, std::vector<int> *fl) {
    out.clear();
    if (fl) fl->clear();
    if (plain_prime[u] >= 0) {
      out.push_back(plain_prime[u]);
      return;
    }
    const int32_t *lst;
    const int n = faces_of(u, &lst);
    for (int k = 0; k < n; ++k) {
      const Face &ff = faces[lst[k]];
      if (ff.cells[0] == c || ff.cells[1] == c) {
        out.push_back(hang_first[u] + k);
        if (fl) fl->push_back(lst[k]);
      }
    }
  };
  std::map<std::pair<int64_t, int64_t>, double> ent;
  std::map<int64_t, double> bm;
  std::vector<int64_t> cu, cv;
  std::vector<int> fu, fv;
  for (int a = 0; a < d; ++a) {
    for (int64_t l = 0; l < nloc; ++l) {
      // edge from local node l along +a exists iff l is not on the cell's high side along a
      if ((l / lstr[a]) % lext[a] == lext[a] - 1) continue;
      const double w = E[a][l];
      const int64_t u = loc[l], v = loc[l + lstr[a]];
      if (u < 0 && v < 0) continue;
      if (u >= 0 && v >= 0) {
        copies(u, cu, &fu);
        copies(v, cv, &fv);
        const bool ku = plain_prime[u] < 0, kv = plain_prime[v] < 0;
        std::vector<std::pair<int64_t, int64_t>> pairs;
        if (ku && kv) {
          for (size_t i = 0; i < fu.size(); ++i)
            for (size_t j = 0; j < fv.size(); ++j)
              if (fu[i] == fv[j]) pairs.push_back({cu[i], cv[j]});
          MSS_REQUIRE(!pairs.empty(), MSS_ERR_INVALID_ARG, "edge between corner nodes of different faces");
        } else if (ku) {
          for (int64_t x : cu) pairs.push_back({x, cv[0]});
        } else if (kv) {
          for (int64_t x : cv) pairs.push_back({cu[0], x});
        } else {
          pairs.push_back({cu[0], cv[0]});
        }
        const double ws = w / (double)pairs.size();
        for (auto &pr : pairs) {
          ent[{pr.first, pr.second}] += ws;
          ent[{pr.second, pr.first}] += ws;
          ent[{pr.first, pr.first}] -= ws;
          ent[{pr.second, pr.second}] -= ws;
        }
      } else {
        copies(u >= 0 ? u : v, cu, nullptr);
        for (int64_t x : cu) ent[{x, x}] -= w / (double)cu.size();
      }
    }
  }
  for (int64_t l = 0; l < nloc; ++l) {
    if (loc[l] < 0) continue;
    copies(loc[l], cu, nullptr);
    for (int64_t x : cu) bm[x] += mass[l] / (double)cu.size();
  }
  // local order: boundary nodes face by face, then interior ascending
  std::vector<int64_t> order;
  for (int fi : cl.faces)
    for (int64_t x : faces[fi].nodes) order.push_back(x);
  cl.K = (int64_t)order.size();
  std::vector<int64_t> bnd(order);
  std::sort(bnd.begin(), bnd.end());
  for (auto &kv : bm)
    if (!std::binary_search(bnd.begin(), bnd.end(), kv.first)) order.push_back(kv.first);
  MSS_REQUIRE(order.size() == bm.size(), MSS_ERR_INVALID_ARG, "internal: cell node split inconsistent");
  std::unordered_map<int64_t, int64_t> pos;
  for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int64_t)i;
  const int64_t n = (int64_t)order.size();
  std::vector<std::vector<std::pair<int64_t, double>>> rows(n);
  for (auto &kv : ent) rows[pos[kv.first.first]].push_back({pos[kv.first.second], kv.second});
  cl.A.n = n;
  cl.A.ptr.assign(n + 1, 0);
  cl.A.col.clear();
  cl.A.val.clear();
  for (int64_t i = 0; i < n; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    for (auto &e : rows[i]) {
      cl.A.col.push_back(e.first);
      cl.A.val.push_back(e.second);
    }
    cl.A.ptr[i + 1] = (int64_t)cl.A.col.size();
  }
  cl.B.resize(n);
  for (int64_t i = 0; i < n; ++i) cl.B[i] = bm[order[i]];
  cl.nodes = order;
  cl.built = true;
}

}  // namespace mss

using namespace mss;

extern "C" {

mss_status mss_assemble(const mss_grid *g, const double *sigma, const double *rho, mss_operator **out) {
  return guard([&] {
    const Range nvtx_range("mss_assemble");
    MSS_REQUIRE(g && sigma && rho && out, MSS_ERR_INVALID_ARG, "null argument");
    auto h = std::make_unique<mss_operator>();
    assemble(h->o, *g, sigma, rho);
    *out = h.release();
  });
}

mss_status mss_assemble_elastic(const mss_grid *g, const double *C, const double *rho, mss_operator **out) {
  return guard([&] {
    const Range nvtx_range("mss_assemble_elastic");
    MSS_REQUIRE(g && C && rho && out, MSS_ERR_INVALID_ARG, "null argument");
    auto h = std::make_unique<mss_operator>();
    assemble_elastic(h->o, *g, C, rho);
    *out = h.release();
  });
}

mss_status mss_operator_info(const mss_operator *op, int64_t info[2]) {
  return guard([&] {
    MSS_REQUIRE(op && info, MSS_ERR_INVALID_ARG, "null argument");
    info[0] = op->o.N;
    info[1] = (int64_t)op->o.A.col.size();
  });
}

mss_status mss_operator_export(const mss_operator *op, int64_t *rowptr, int64_t *col, double *val, double *bdiag) {
  return guard([&] {
    MSS_REQUIRE(op, MSS_ERR_INVALID_ARG, "null operator");
    const Operator &o = op->o;
    if (rowptr) std::copy(o.A.ptr.begin(), o.A.ptr.end(), rowptr);
    if (col) std::copy(o.A.col.begin(), o.A.col.end(), col);
    if (val) std::copy(o.A.val.begin(), o.A.val.end(), val);
    if (bdiag) std::copy(o.B.begin(), o.B.end(), bdiag);
  });
}

mss_status mss_operator_node(const mss_operator *op, const int32_t *node, int64_t *unknown) {
  return guard([&] {
    MSS_REQUIRE(op && node && unknown, MSS_ERR_INVALID_ARG, "null argument");
    const Operator &o = op->o;
    int64_t ext[3], str[3];
    node_strides(o.g, ext, str);
    int64_t p = 0;
    for (int a = 0; a < o.g.dim; ++a) {
      MSS_REQUIRE(node[a] >= 0 && node[a] <= o.g.n[a], MSS_ERR_INVALID_ARG, "node outside the grid");
      p += node[a] * str[a];
    }
    *unknown = o.unknown[p];
  });
}

mss_status mss_operator_lambda_max(const mss_operator *op, double tol, double *lam) {
  return guard([&] {
    MSS_REQUIRE(op && lam && tol > 0, MSS_ERR_INVALID_ARG, "bad argument");
    *lam = lambda_max_lanczos(op->o, tol);
  });
}

void mss_operator_destroy(mss_operator *op) { delete op; }

mss_status mss_partition_create(const mss_operator *op, const double *sigma, const double *rho, const int32_t *cell,
                                int32_t n_io, const int32_t *io_nodes, mss_partition **out) {
  return guard([&] {
    const Range nvtx_range("mss_partition_create");
    MSS_REQUIRE(op && sigma && rho && cell && out && n_io >= 0 && (n_io == 0 || io_nodes), MSS_ERR_INVALID_ARG,
                "null argument");
    MSS_REQUIRE(op->o.comps == 1, MSS_ERR_INVALID_ARG,
                "the partition takes one unknown per node (vector faces of the elastic operator are not built)");
    auto h = std::make_unique<mss_partition>();
    partition(h->p, op->o, sigma, rho, cell, n_io, io_nodes);
    *out = h.release();
  });
}

mss_status mss_partition_info(const mss_partition *p, int64_t info[8]) {
  return guard([&] {
    MSS_REQUIRE(p && info, MSS_ERR_INVALID_ARG, "null argument");
    const Partition &P = p->p;
    int64_t fn = 0;
    for (auto &f : P.faces) fn += (int64_t)f.nodes.size();
    // cell node counts without building the cells: box nodes + extra hanging copies
    info[0] = P.n_cells;
    info[1] = (int64_t)P.faces.size();
    info[2] = P.n_int_faces;
    info[3] = P.Np;
    info[4] = (int64_t)P.corner_set.size();
    info[5] = fn;
    int64_t tot = 0, mx = 0;
    for (int c = 0; c < P.n_cells; ++c) {
      const_cast<Partition &>(P).build_cell(c);
      tot += (int64_t)P.cells[c].nodes.size();
      mx = std::max<int64_t>(mx, (int64_t)P.cells[c].nodes.size());
    }
    info[6] = tot;
    info[7] = mx;
  });
}

mss_status mss_partition_faces(const mss_partition *p, int32_t *kind, int32_t *cells, int32_t *shape,
                               int64_t *node_ptr, int64_t *nodes, int64_t *parents) {
  return guard([&] {
    MSS_REQUIRE(p, MSS_ERR_INVALID_ARG, "null partition");
    const Partition &P = p->p;
    int64_t o = 0;
    for (size_t f = 0; f < P.faces.size(); ++f) {
      const Face &F = P.faces[f];
      if (kind) kind[f] = F.kind;
      if (cells) { cells[2 * f] = F.cells[0]; cells[2 * f + 1] = F.cells[1]; }
      if (shape) { shape[2 * f] = F.shape[0]; shape[2 * f + 1] = F.shape[1]; }
      if (node_ptr) node_ptr[f] = o;
      for (size_t k = 0; k < F.nodes.size(); ++k) {
        if (nodes) nodes[o + k] = F.nodes[k];
        if (parents) parents[o + k] = F.parents[k];
      }
      o += (int64_t)F.nodes.size();
    }
    if (node_ptr) node_ptr[P.faces.size()] = o;
  });
}

mss_status mss_partition_cell(const mss_partition *p, int32_t c, int64_t counts[4], int32_t *faces, int64_t *nodes,
                              int64_t *rowptr, int64_t *col, double *val, double *bdiag) {
  return guard([&] {
    MSS_REQUIRE(p && counts, MSS_ERR_INVALID_ARG, "null argument");
    Partition &P = const_cast<Partition &>(p->p);
    MSS_REQUIRE(c >= 0 && c < P.n_cells, MSS_ERR_INVALID_ARG, "cell index out of range");
    P.build_cell(c);
    const Cell &C = P.cells[c];
    counts[0] = (int64_t)C.nodes.size();
    counts[1] = (int64_t)C.A.col.size();
    counts[2] = (int64_t)C.faces.size();
    counts[3] = C.K;
    if (faces) std::copy(C.faces.begin(), C.faces.end(), faces);
    if (nodes) std::copy(C.nodes.begin(), C.nodes.end(), nodes);
    if (rowptr) std::copy(C.A.ptr.begin(), C.A.ptr.end(), rowptr);
    if (col) std::copy(C.A.col.begin(), C.A.col.end(), col);
    if (val) std::copy(C.A.val.begin(), C.A.val.end(), val);
    if (bdiag) std::copy(C.B.begin(), C.B.end(), bdiag);
  });
}

void mss_partition_destroy(mss_partition *p) { delete p; }

}  // extern "C"
