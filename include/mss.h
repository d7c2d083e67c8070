/*
 * mss.h -- C ABI of the GB300 implementation of the multiscale S-fraction
 * reduced-order method (Druskin, Mamonov, Zaslavsky, "Multi-scale S-fraction
 * reduced-order models for massive wavefield simulations").
 *
 * The semi-discrete problem is A u - B u_tt = g w(t) (Section 1, Eq. wave_fll).
 * The library covers both stages of Algorithm alg1red:
 *   stage 1 (off-line): assemble A, B (Section 1); partition into coarse cells
 *     and remove the corner set (Sections 2-3, Appendix B); build each cell's
 *     rational Krylov ROM and its matrix S-fraction coefficients (Sections 4-5,
 *     Appendix C); project sources and receivers (Eqs. BEINCr, solatrec);
 *   stage 2 (on-line): leapfrog stepping of the coupled ROM for many sources
 *     at once (Eqs. intrtstep_td, bdrytstep), sampled at receivers.
 * plus the fine-grid leapfrog on the GPU for comparison.
 *
 * Conventions
 *   - Every call returns mss_status; 0 is success.  On failure nothing the
 *     call was asked to create is returned, and mss_last_error() (thread
 *     local) holds a one-line reason.
 *   - Handles (mss_operator, mss_partition, mss_rom, mss_sim, mss_fine) are
 *     opaque and owned by the library; free them with the matching *_destroy.
 *     Device memory they hold is allocated with cudaMalloc on the current
 *     device at creation time and freed by *_destroy.
 *   - Caller buffers are plain pointers.  "host" buffers are read or written
 *     before the call returns.  "device" buffers must stay valid until the
 *     work queued on the given stream has finished; the library never frees
 *     them.  Streams are cudaStream_t passed as void* (NULL = legacy stream).
 *   - Grid arrays are indexed in array order [z][y][x] (3D) or [y][x] (2D),
 *     x fastest.  Node coordinates are given in the same order.
 *   - All off-line arithmetic is FP64.
 */
#ifndef MSS_H
#define MSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mss_status;
enum {
  MSS_OK = 0,
  MSS_ERR_INVALID_ARG = 1,       /* bad size, pointer, index or parameter            */
  MSS_ERR_NOT_SPD = 2,           /* A not <= 0 or B not > 0 (Section 1)              */
  MSS_ERR_KRYLOV_DEFLATION = 3,  /* Krylov blocks linearly dependent (Assumption ass1) */
  MSS_ERR_LANCZOS_BREAKDOWN = 4, /* block Lanczos breakdown (Appendix C)             */
  MSS_ERR_COEF_NOT_SPD = 5,      /* a Gamma^k or Gamma-hat^k not SPD (Eq. S-fraction) */
  MSS_ERR_CFL = 6,               /* time step above the leapfrog stability limit     */
  MSS_ERR_TIMEOUT = 7,           /* a bounded device-side wait gave up               */
  MSS_ERR_CUDA = 8,              /* a CUDA runtime call failed                       */
  MSS_ERR_OOM = 9,               /* device or host allocation failed                 */
  MSS_ERR_NOT_CONVERGED = 10,    /* an iterative off-line solve missed its tolerance  */
  MSS_ERR_STATE = 11             /* call not valid in the handle's current state     */
};

enum { MSS_DIRICHLET = 0, MSS_NEUMANN = 1 };
/* Precisions of the on-line stage.  MSS_FP32_TC: FP32 state, cell products on the tensor cores
 * (tcgen05, BF16 operands split into hi + lo parts, three products, FP32 accumulation);
 * MSS_BF16_TC: the same with one BF16 product; both need K_i <= 128.  MSS_TF32_TC: FP32 state and
 * coefficients, cell products on the tensor cores as TF32 with both operands split hi + lo (three
 * products, FP32-class), the last coefficient applied as its Cholesky factor; K_i <= 384. */
enum { MSS_FP64 = 0, MSS_FP32 = 1, MSS_FP32_TC = 2, MSS_BF16_TC = 3, MSS_TF32_TC = 4 };

const char *mss_status_string(mss_status s);
/* Reason of the last failed call on this thread ("" if none). */
const char *mss_last_error(void);
/* Library version string. */
const char *mss_version(void);

/* ------------------------------------------------------------------------- */
/* Fine grid (Section 1, Eq. wave_fll and the acoustic equation below it).    */
/* ------------------------------------------------------------------------- */

/* Box of voxels: n[a] voxels of edge h along array axis a (a < dim, dim = 1..3);
 * bc[a][0], bc[a][1] = MSS_DIRICHLET (wall nodes removed) or MSS_NEUMANN (kept)
 * for the low / high wall of axis a. */
typedef struct mss_grid {
  int32_t dim;
  int32_t n[3];
  double h;
  int32_t bc[3][2];
} mss_grid;

typedef struct mss_operator mss_operator;

/* Assemble the conservative node-based discretisation of div(sigma grad u) - rho u_tt:
 * voxel v adds -(sigma_v h^(d-2)/2^(d-1)) (e_k - e_l)(e_k - e_l)^T to A for each of its
 * edges (k,l) and rho_v h^d/2^d to the mass of each of its 2^d corner nodes (Section 1).
 * sigma, rho: host, prod(n) doubles, > 0.  Unknowns: kept nodes in node order.
 * Errors: INVALID_ARG (sizes), NOT_SPD (a sigma or rho <= 0 or not finite). */
mss_status mss_assemble(const mss_grid *g, const double *sigma, const double *rho, mss_operator **out);
/* Elastic operator of the paper's anisotropic elastic experiment (Section 7: u_tt = div sigma with
 * sigma_ij = C_ijkl u_k,l), as a symmetric non-positive pencil (Section 1): A = -K, K the stiffness
 * of trilinear finite elements on the voxel grid, exact for a constant stiffness per voxel (2 x 2 x 2
 * Gauss points); B the lumped mass, rho_v h^3/8 from each voxel to each of its corners, per
 * component.  Unknowns: 3 per kept node, node-major: 3k + p is displacement component p (physical
 * axis x, y, z = array axis 2, 1, 0) of the k-th kept node (nodes in node order; Dirichlet walls
 * remove their nodes as in mss_assemble).  C: host, prod(n) x 36 doubles, per voxel (C order) the
 * 6 x 6 Voigt stiffness, row-major, order (xx, yy, zz, yz, xz, xy) in physical axes, symmetric
 * positive definite (a VTI medium from Thomsen's parameters, or any other); rho: host, prod(n)
 * doubles.  dim must be 3.  The operator serves mss_operator_info / export / lambda_max and
 * mss_operator_node (which returns the unknown of component 0); the partition and the fine-grid
 * kernels take one unknown per node and refuse it (vector faces are not built).
 * Errors: INVALID_ARG (dim, sizes, walls, C not symmetric), NOT_SPD (C not positive definite,
 * rho <= 0, a value not finite). */
mss_status mss_assemble_elastic(const mss_grid *g, const double *C, const double *rho, mss_operator **out);
/* info[0] = unknowns N, info[1] = nonzeros of A (CSR, diagonal included). */
mss_status mss_operator_info(const mss_operator *op, int64_t info[2]);
/* Copy A as CSR (rowptr[N+1], col[nnz], val[nnz], columns ascending) and diag(B)[N] to host buffers. */
mss_status mss_operator_export(const mss_operator *op, int64_t *rowptr, int64_t *col, double *val, double *bdiag);
/* Unknown number of a node (array-order coordinates), -1 if removed by a Dirichlet wall. */
mss_status mss_operator_node(const mss_operator *op, const int32_t *node, int64_t *unknown);
/* Largest eigenvalue of -B^{-1} A by Lanczos on the host (FP64; stops when the top Ritz value changes by < tol relative). */
mss_status mss_operator_lambda_max(const mss_operator *op, double tol, double *lambda_max);
void mss_operator_destroy(mss_operator *op);

/* ------------------------------------------------------------------------- */
/* Partition (Section 2 Eq. part / splitN_c; Section 3 Eq. nocorners,        */
/* Example cs_multidom_ex; Appendix B; I/O faces for Eq. gsupport).            */
/* ------------------------------------------------------------------------- */
typedef struct mss_partition mss_partition;

/* Box cells of cell[a] voxels (>= 2, dividing n[a]); cell i receives the terms of its own
 * voxels (voxel ownership).  Interior faces are numbered axis-major, then by the lower
 * cell in C order; a node on more than one face is replaced by one hanging node per face,
 * every cell splitting its share of the node's row (edge weights, Dirichlet losses, mass)
 * equally among its faces holding the node.  io_nodes (host, n_io x dim, may repeat) that
 * fall strictly inside a cell become that cell's one-sided I/O face (nodes in unknown order).
 * sigma, rho: the arrays given to mss_assemble.  Errors: INVALID_ARG. */
mss_status mss_partition_create(const mss_operator *op, const double *sigma, const double *rho,
                                const int32_t *cell, int32_t n_io, const int32_t *io_nodes,
                                mss_partition **out);
/* info: [0] cells, [1] faces, [2] interior faces, [3] prime nodes N', [4] corner-set nodes,
 *       [5] total face nodes, [6] total cell nodes, [7] max cell nodes. */
mss_status mss_partition_info(const mss_partition *p, int64_t info[8]);
/* Faces: kind[f] (0 interior, 1 I/O), cells[2f..2f+1] (-1 if none), shape[2f..2f+1] (face
 * node grid, 1 for missing axes), node_ptr[F+1], nodes[] (prime ids, face order),
 * parents[] (original unknowns).  Host buffers sized from mss_partition_info. */
mss_status mss_partition_faces(const mss_partition *p, int32_t *kind, int32_t *cells, int32_t *shape,
                               int64_t *node_ptr, int64_t *nodes, int64_t *parents);
/* Cell c: face_ptr/faces (ascending), nodes (prime ids: boundary face by face, then interior),
 * K = boundary node count, A_c as CSR in that local order, diag(B_c).  Pass NULL to query
 * counts: counts[0] = nodes, counts[1] = nonzeros, counts[2] = faces, counts[3] = K. */
mss_status mss_partition_cell(const mss_partition *p, int32_t c, int64_t counts[4], int32_t *faces,
                              int64_t *nodes, int64_t *rowptr, int64_t *col, double *val, double *bdiag);
void mss_partition_destroy(mss_partition *p);

/* ------------------------------------------------------------------------- */
/* Cell ROMs and S-fraction coefficients (Sections 4-6, Appendix C).          */
/* ------------------------------------------------------------------------- */
typedef struct mss_rom mss_rom;

/* Off-line parameters.  m: S-fraction layers per cell (cell_m overrides per cell);
 * n_modes: modes kept per interior face (lowest-wavenumber DCT-II modes of the face grid;
 * I/O faces keep all nodes); shift s < 0 of the rational Krylov space (Eq. npks);
 * cg_tol / cg_maxit: relative residual and iteration cap of the shifted solves. */
typedef struct mss_rom_params {
  int32_t m;
  int32_t n_modes;
  double shift;
  double cg_tol;
  int32_t cg_maxit;
  int32_t reserved;
} mss_rom_params;

/* Build every cell's ROM on the current device in FP64 (Algorithm alg1red stage 1):
 * V = B-orthonormal basis of span{B^{-1}C, K B^{-1}C, .., K^{m-1}B^{-1}C}, K = (A+sB)^{-1}B,
 * C = P^Gamma S (Eq. npks, Remark Sinsubspace); A^m = V^T A V, S^m = V^T C (Eq. tfprj);
 * block Lanczos (Eq. NtDtri); Gamma^k, Gamma-hat^k (Eq. GammaTrans, symmetric form);
 * face masses M_f = sum_i (Gamma-hat^1_{i,f})^{-1} (Eq. bdrytstep); Appendix D data.
 * Errors: INVALID_ARG, KRYLOV_DEFLATION, LANCZOS_BREAKDOWN, COEF_NOT_SPD, NOT_CONVERGED,
 * CUDA, OOM.  Synchronises the stream before returning. */
mss_status mss_build_roms(const mss_partition *p, const mss_rom_params *prm, const int32_t *cell_m,
                          void *stream, mss_rom **out);

/* Per-cell number of S-fraction layers by the rule of the dipping-layer workload (the paper fixes
 * m_i per cell, Section 7, without the rule; this one is a reading of it): cell_m[i] = the smallest
 * m in [m_lo, m_hi] whose ROM transfer function F^m(z) = S_m^T (A_m + z I)^{-1} S_m (Eq. tfprj) is
 * within tol of F^{m_hi} at the n_freq damped test points z_j = -w_j^2 + i w_j omega_max / 10,
 * w_j = j omega_max / n_freq (relative Frobenius error, largest over j); err[i] (may be NULL) that
 * error (0 at m_hi).  A_m, S_m are the leading m K_i rows/columns of the m_hi projection built as
 * mss_build_roms builds it (FP64 on the GPU; the block Krylov spaces are nested); the transfer
 * functions are evaluated on the host in FP64 complex arithmetic, one block LDL^T of A + z I by
 * K_i x K_i blocks per point giving every m at once.  cell_m, err: host, one entry per cell of p.
 * Pass cell_m to mss_build_roms.  Errors: as mss_build_roms (m_hi K_i must fit the cell),
 * INVALID_ARG, LANCZOS_BREAKDOWN (a singular pivot block). */
mss_status mss_layer_rule(const mss_partition *p, const mss_rom_params *prm, int32_t m_lo, int32_t m_hi,
                          double omega_max, double tol, int32_t n_freq, int32_t *cell_m, double *err, void *stream);
/* The host part of the rule for one cell, on a projection given by the caller: A (n x n, symmetric)
 * and S (n x K), n = m_hi K, row-major FP64 host buffers, leading m K rows/columns being the m-layer
 * ROM.  errs[m] (host, m_hi + 1 entries) = the rule's error of m for m_lo <= m <= m_hi (0 at m_hi
 * and below m_lo); *m_out = the chosen m.  No device work.  Errors: INVALID_ARG,
 * LANCZOS_BREAKDOWN (a singular pivot block). */
mss_status mss_layer_rule_cell(const double *A, const double *S, int32_t K, int32_t m_lo, int32_t m_hi,
                               double omega_max, double tol, int32_t n_freq, int32_t *m_out, double *errs);

/* Coefficient set given by the caller (host, FP64), for ROMs built elsewhere.
 * cell_m[C], cell_face_ptr[C+1], cell_faces[] (faces of each cell in boundary-vector order),
 * face_M[F], face_cells[2F] (lower cell first, -1 for a one-sided face);
 * gamma: per cell m_i blocks K_i x K_i (Gamma^1..Gamma^m, row-major, concatenated over cells);
 * gamma_hat: per cell m_i blocks (Gamma-hat^1..Gamma-hat^m); face_mass: per face M_f x M_f.
 * K_i = sum of M_f over the cell's faces.  Matrices must be symmetric. */
typedef struct mss_rom_desc {
  int32_t n_cells;
  int32_t n_faces;
  const int32_t *cell_m;
  const int32_t *cell_face_ptr;
  const int32_t *cell_faces;
  const int32_t *face_M;
  const int32_t *face_cells;
  const double *gamma;
  const double *gamma_hat;
  const double *face_mass;
} mss_rom_desc;
/* Errors: INVALID_ARG (inconsistent topology), COEF_NOT_SPD (a Gamma-hat^k or M_f fails Cholesky). */
mss_status mss_rom_import(const mss_rom_desc *d, mss_rom **out);
/* info: [0] cells, [1] faces, [2] max K, [3] max m, [4] coefficient doubles,
 *       [5] face-mass doubles, [6] total face modes, [7] corner groups. */
mss_status mss_rom_info(const mss_rom *r, int64_t info[8]);
/* Copy the coefficients to host in the mss_rom_desc layout (sizes from mss_rom_info):
 * cell_m, cell_face_ptr, cell_faces, face_M, face_cells, gamma, gamma_hat, face_mass. */
mss_status mss_rom_export(const mss_rom *r, int32_t *cell_m, int32_t *cell_face_ptr, int32_t *cell_faces,
                          int32_t *face_M, int32_t *face_cells, double *gamma, double *gamma_hat,
                          double *face_mass);
/* Face bases S_f (K_f x M_f, row-major, concatenated over faces) of a ROM built by
 * mss_build_roms; sizes: sum K_f M_f. */
mss_status mss_rom_face_bases(const mss_rom *r, int64_t *count, double *bases);
/* Caller-supplied face bases S_f in place of the DCT modes, for example the frequency-limited
 * Gramian basis of Eq. trgr (Section 4.1).  They apply to every later mss_build_roms /
 * mss_rom_skeleton / mss_rom_rebuild_cells of p, which ignore n_modes for those faces.
 * face_M[f] = M_f columns of face f (1 <= M_f <= K_f, K_f its node count from
 * mss_partition_faces), or 0 to keep the DCT modes there.  bases holds, face by face, the
 * faces with M_f > 0 as K_f x M_f row-major blocks in the face's node order (host buffer, copied).
 * n_faces must be the partition's face count; n_faces = 0 clears the bases.
 * Errors: INVALID_ARG (count, sizes, or columns not orthonormal to 1e-10). */
mss_status mss_partition_set_face_bases(mss_partition *p, int32_t n_faces, const int32_t *face_M,
                                        const double *bases);

/* Receivers inside cells through the Galerkin lift (Remark MFEM: the ROM is a Galerkin method, the
 * cell's fine state is approximately V x, x its projected state).  nodes (host, n x dim) must lie
 * strictly inside a cell: on no face and not an I/O node of mss_partition_create.  The next
 * mss_build_roms / mss_rom_rebuild_cells of p computes, per node and cell layer k, the weights
 * w_k = G_k^{-T} Q_k^T V^T e_node (Q_k the block Lanczos vectors of Eq. NtDtri, G_k the change of
 * variables of Eq. GammaTrans), and mss_rom_set_io_nodes then reads a receiver at such a node as
 * sum_k w_k . U^k (layer 1 = the cell's face state, layers 2..m its hidden state), so the node
 * needs no I/O face.  n = 0 clears the list.  Errors: INVALID_ARG (a node outside the grid, on a
 * Dirichlet wall, on a face or an I/O node). */
mss_status mss_partition_set_lift_nodes(mss_partition *p, int32_t n, const int32_t *nodes);

/* Projected inputs/outputs (Eq. BEINCr g~_f = S_f^T g|_f, Eq. solatrec q~_f = S_f^T q|_f) from
 * point sources/receivers at fine-grid nodes with weights (NULL = 1); a node of the corner set
 * is spread over its hanging copies with weights b_{k_f}/b_k; a receiver at a lift node of the build
 * (mss_partition_set_lift_nodes) is read through its lift.  Needs a ROM built by mss_build_roms from
 * the same partition.  Replaces any previous I/O of the ROM. */
mss_status mss_rom_set_io_nodes(mss_rom *r, const mss_partition *p, int32_t n_src, const int32_t *src_nodes,
                                const double *src_w, int32_t n_rcv, const int32_t *rcv_nodes,
                                const double *rcv_w);
/* Projected inputs/outputs given directly as entries (face, index, M_f values):
 * src_face[e], src_index[e], src_vals (concatenated M_f values per entry), likewise receivers. */
mss_status mss_rom_set_io(mss_rom *r, int32_t n_src, int32_t n_src_entries, const int32_t *src_face,
                          const int32_t *src_index, const double *src_vals, int32_t n_rcv,
                          int32_t n_rcv_entries, const int32_t *rcv_face, const int32_t *rcv_index,
                          const double *rcv_vals);
/* Appendix D corner correction data: group_ptr[G+1]; per member: face, the S_f row of the
 * hanging node (M_f values, concatenated), weight b_{k_f}/b_k.  Built automatically by
 * mss_build_roms; this call replaces it (n_groups = 0 clears it). */
mss_status mss_rom_set_corners(mss_rom *r, int32_t n_groups, const int32_t *group_ptr, const int32_t *face,
                               const double *rows, const double *weight);
/* Host copies of a ROM's projected I/O (Eq. BEINCr g~_f = S_f^T g|_f, Eq. solatrec q~_f = S_f^T q|_f)
 * and Appendix D data, in the layouts of mss_rom_set_io and mss_rom_set_corners.
 * counts (host, [9]): sources, source entries, source values, receivers, receiver entries,
 * receiver values, corner groups, corner members, corner row values (receiver entries on hidden
 * layers, from lifted receivers, are not part of this export).  Any array may be NULL
 * (counts only); otherwise it must hold its count (group_ptr: groups + 1).  Errors: INVALID_ARG. */
mss_status mss_rom_export_io(const mss_rom *r, int64_t counts[9], int32_t *src_face, int32_t *src_index,
                             double *src_vals, int32_t *rcv_face, int32_t *rcv_index, double *rcv_vals,
                             int32_t *group_ptr, int32_t *member_face, double *member_rows, double *member_weight);
void mss_rom_destroy(mss_rom *r);

/* ------------------------------------------------------------------------- */
/* On-line stage (Algorithm alg1red stage 2; Eqs. intrtstep_td, bdrytstep,    */
/* contred, solatrec).                                                        */
/* ------------------------------------------------------------------------- */
typedef struct mss_sim mss_sim;

/* Per step n (t_n = n tau), for every cell i and source:
 *   F^k_i = Gamma^k_i (U^{k+1}_i - U^k_i), k = 1..m_i, U^1_i = the cell's faces' u~_f, U^{m+1} = 0
 *   U^k_i <- 2 U^k_i - U^k_i,old + tau^2 Gamma-hat^k_i (F^k_i - F^{k-1}_i),          k = 2..m_i
 *   u~_f  <- 2 u~_f - u~_f,old + tau^2 M_f^{-1} (sum_{i on f} F^1_i|_f - g~_f w(t_n))
 *   then (if enabled) the Appendix D correction of the new u~;
 * trace sample n = sum_f q~_f^T u~_f at step n (before it is advanced).
 * precision: MSS_FP64, MSS_FP32 (state, coefficients and arithmetic), MSS_FP32_TC or MSS_BF16_TC
 * (FP32 state, tensor-core cell products with BF16 operands, split hi + lo for FP32_TC; K_i <= 128;
 * traces are float), MSS_TF32_TC (FP32 state and coefficients, cell products on the tensor cores as
 * TF32 with both operands split hi + lo, three products per pair, FP32-class; K_i <= 384 and
 * 2 m_i ceil(K_i / 128) <= 32; the last coefficient always applied as its Cholesky factor, as with
 * MSS_SIM_FACTOR_LAST below; schedule GRAPH; traces are float).
 * flags: MSS_SIM_CORNERS (the Appendix D correction; 1 keeps its old meaning) | MSS_SIM_FACTOR_LAST
 * (MSS_FP32 and MSS_TF32_TC: the last coefficient is applied as F^m = L (L^T D^m), L the lower Cholesky factor
 * of Gamma^m computed in FP64 at creation, pivots at or below 1e-13 of its largest diagonal entry
 * raised to that floor; stored as one K x K matrix W = L + L^T - diag(L), so the coefficient bytes
 * do not change.  Rounding the entries of a nearly singular Gamma^m -- a cell without a Dirichlet
 * node, whose constant mode makes it semidefinite, Eq. intrtstep_td with Lemma lemStil -- to FP32
 * can make it indefinite; a rounded factor keeps L L^T semidefinite.  With MSS_FP32: schedules
 * GRAPH and PERSIST, and GRAPH_STREAM (the wide streamed kernel) when the source tile is 16.
 * COEF_NOT_SPD if a Gamma^m is indefinite beyond -1e-8 of its scale).  Needs I/O set on the ROM
 * (n_src >= 1).
 * The sim copies what it needs from the ROM (the ROM may be destroyed afterwards).
 * Errors: INVALID_ARG (unknown flags), STATE (ROM without I/O), CFL (tau <= 0), COEF_NOT_SPD, CUDA,
 * OOM, TIMEOUT (a tensor-core
 * kernel's bounded wait gave up; reported by the next mss_step / mss_sim_info call). */
#define MSS_SIM_CORNERS 1
#define MSS_SIM_FACTOR_LAST 2
mss_status mss_sim_create(const mss_rom *r, int32_t precision, double tau, int32_t flags, mss_sim **out);
/* info: [0] sources, [1] receivers, [2] precision, [3] steps taken, [4] state values per level,
 *       [5] device bytes held, [6] kernels launched per step, [7] source tile. */
mss_status mss_sim_info(const mss_sim *s, int64_t info[8]);
/* Zero the state (u = u_old = 0) and the step counter. */
mss_status mss_sim_reset(mss_sim *s, void *stream);
/* Advance n_steps.  waveform: device, FP64, w(t_j) for j = steps_taken .. steps_taken+n_steps-1
 * (indexed from the pointer: waveform[j - steps_taken]); traces: device, [n_steps][n_rcv][n_src]
 * of double (FP64) or float (FP32).  use_graph: capture the loop as a CUDA graph (cached per
 * (n_steps, pointers)).  Errors: INVALID_ARG, CUDA. */
mss_status mss_step(mss_sim *s, int64_t n_steps, const double *waveform, void *traces, int32_t use_graph,
                    void *stream);
/* End-to-end call on host buffers: copies waveform (host, n_steps doubles) to the device,
 * resets the state, steps, and copies the traces back into traces_host (same layout as
 * mss_step), all on the stream; returns after the copy has completed. */
mss_status mss_run_host(mss_sim *s, int64_t n_steps, const double *waveform_host, void *traces_host,
                        void *stream);
/* Per-kernel timing of the step loop: runs n_steps eagerly on the stream with CUDA events around
 * every kernel and returns the mean device duration (ms) of each kernel kind:
 * ms[0] cell kernel, ms[1] face+receiver kernel, ms[2] corner kernel (0 when disabled).
 * Same waveform/trace conventions as mss_step; the state advances like mss_step. */
mss_status mss_step_profile(mss_sim *s, int64_t n_steps, const double *waveform, void *traces, double ms[3],
                            void *stream);
/* Two time levels of the state as FP64 on host, faces first (total face modes x n_src) then
 * hidden layers (cell by cell, layer by layer, K_i x n_src); count = mss_sim_info[4] each.
 * save: now[], old[] <- state; load: state <- now[], old[] (and the step counter).
 * Resuming from a saved state continues bit-identically on the same precision. */
mss_status mss_sim_save_state(const mss_sim *s, double *now, double *old, int64_t *steps_taken);

/* Schedules of one step (Algorithm alg1red step 2; all give the same arithmetic, element by
 * element, for the same precision and tile):
 *   GRAPH            cell, face(+receivers) and corner kernels per step, the loop captured as a
 *                    CUDA graph when use_graph is set;
 *   GRAPH_STREAM     as GRAPH with the streamed FP32 cell kernel: each cell's coefficient stream
 *                    staged into shared memory by 1-D TMA bulk copies through a 4-slot ring
 *                    (FP32, 16-source tiles, K_i <= 128; 256 or 512 threads, the autotuner
 *                    picks; 512 by default);
 *   PERSIST          CUDA-core precisions: one cooperative persistent kernel per block of up to
 *                    512 steps, phases separated by a grid barrier with a 1 s time limit;
 *                    tensor-core precisions: the split products on a resident grid that loops
 *                    over (cell, matrix, tile) items with the next matrix's bulk copy in flight;
 *   PERSIST_STREAM   CUDA-core: PERSIST with the streamed cell body; tensor-core precisions: a
 *                    warp-specialised persistent kernel (one CTA per SM, a producer warp
 *                    streaming the matrices through a 4-slot mbarrier ring, compute warps
 *                    issuing the products and epilogues);
 *   GRAPH_SPLIT      as GRAPH with the cell phase split into a flux kernel and an acceleration
 *                    kernel of one small CTA per (cell, matrix), fluxes through a scratch block
 *                    (CUDA-core precisions).
 * The default is GRAPH; mss_sim_autotune times every available schedule and keeps the fastest. */
#define MSS_SCHED_GRAPH 0
#define MSS_SCHED_GRAPH_STREAM 1
#define MSS_SCHED_PERSIST 2
#define MSS_SCHED_PERSIST_STREAM 3
#define MSS_SCHED_GRAPH_SPLIT 4
#define MSS_SCHED_COUNT 5
/* Errors: INVALID_ARG (schedule not available for this sim's precision, tile or cell sizes). */
mss_status mss_sim_set_schedule(mss_sim *s, int32_t sched);
/* Stability (CFL) check of tau for this sim: n_steps source-free steps from a seeded random
 * state with zero velocity through the sim's own kernels; growth = |u_n| / |u_0| (Euclidean,
 * FP64 on the host).  Below the CFL limit the leapfrog conserves the discrete energy and the
 * growth stays bounded; above it grows geometrically.  The sim's state and step counter are
 * restored.  Errors: CFL (growth > max_growth or not finite), INVALID_ARG, CUDA. */
mss_status mss_sim_check_stability(mss_sim *s, int32_t n_steps, uint64_t seed, double max_growth, double *growth,
                                   void *stream);
/* Failure-path hooks for tests (they cannot fault: each only makes a bounded wait run out, after
 * which the kernel records MSS_ERR_TIMEOUT in the sim's error word and returns):
 *   MSS_DEBUG_GRID_EXTRA_ARRIVALS  the persistent CUDA-core kernel's grid barrier waits for
 *                                  `value` CTAs beyond the grid (a missing neighbour);
 *   MSS_DEBUG_TC_EXTRA_TX          the split tensor-core kernels' matrix barrier, the wide
 *                                  streamed cell kernel's chunk barriers and the wide tensor-core
 *                                  (MSS_TF32_TC) kernel's copy barriers expect `value` bytes
 *                                  beyond their copies.
 * value 0 restores normal operation.  mss_sim_clear_error resets the error word (and the grid
 * barrier) after a reported TIMEOUT; the state of the failed steps is undefined (reset or load a
 * saved state).  Errors: INVALID_ARG, CUDA. */
#define MSS_DEBUG_GRID_EXTRA_ARRIVALS 1
#define MSS_DEBUG_TC_EXTRA_TX 2
mss_status mss_sim_debug(mss_sim *s, int32_t knob, int32_t value);
mss_status mss_sim_clear_error(mss_sim *s, void *stream);
/* Tile of the step kernels (values <= 0 leave a field unchanged): CUDA-core source tile (a power
 * of two up to the one chosen at creation; 16 is needed by the streamed schedules, the schedule
 * falls back to GRAPH otherwise), sources per CTA of the split tensor-core kernels (16, 32, 64,
 * 128), thread groups of the streamed FP32 kernel (2 or 4; for a sim whose streamed schedule runs
 * the wide kernel -- K_i > 128 or the factored last coefficient -- its variant 1..8: unroll depth
 * 2 or 4 of the row loops, 4 or 2 rows per thread, 16 or 8 sources per CTA, as 1 = (2, 4, 16),
 * 2 = (4, 4, 16), 3 = (2, 2, 16), 4 = (4, 2, 16), 5..8 the same with 8 sources; every variant
 * gives the same bits; for an MSS_TF32_TC sim, the copy-ring slots of its cell kernel, 2 up to the
 * most that fit shared memory, also bit-identical).  Errors: INVALID_ARG. */
mss_status mss_sim_set_tile(mss_sim *s, int32_t source_tile, int32_t tc_sources, int32_t groups);
/* sched: current schedule; available (may be NULL): [MSS_SCHED_COUNT] 1 where usable; tile (may
 * be NULL): [3] = CUDA-core source tile, sources per CTA of the split tensor-core kernels (0 for
 * CUDA-core precisions), thread groups of the streamed FP32 kernel (the wide kernel's variant; the
 * copy-ring slots for an MSS_TF32_TC sim). */
mss_status mss_sim_get_schedule(const mss_sim *s, int32_t *sched, int32_t *available, int32_t *tile);
/* Time n_steps (rounded up to even) of every available schedule and tile variant (CUDA-core
 * source tile 16 or 8, split tensor-core N of 16..128, streamed-kernel block size) on zero
 * input, after one untimed pass each, restoring the state after each; keep the fastest.  ms
 * (host, may be NULL): [MSS_SCHED_COUNT] best ms per step of each schedule, -1 where unavailable;
 * chosen (may be NULL) receives the schedule.  Synchronises the stream.
 * Errors: INVALID_ARG, TIMEOUT, CUDA. */
mss_status mss_sim_autotune(mss_sim *s, int32_t n_steps, void *stream, double *ms, int32_t *chosen);
mss_status mss_sim_load_state(mss_sim *s, const double *now, const double *old, int64_t steps_taken);
void mss_sim_destroy(mss_sim *s);

/* ------------------------------------------------------------------------- */
/* Fine-grid leapfrog on the GPU (Section 1; the comparison baseline):        */
/* u^{n+1} = 2u^n - u^{n-1} + tau^2 B^{-1}(A u^n - g w(t_n)), sample q^T u^n.  */
/* ------------------------------------------------------------------------- */
typedef struct mss_fine mss_fine;
/* Point sources/receivers at nodes (host, n x dim), unit weights.  Sources batched:
 * state layout [node][source].  precision: MSS_FP64 or MSS_FP32. */
mss_status mss_fine_create(const mss_operator *op, int32_t precision, double tau, int32_t n_src,
                           const int32_t *src_nodes, int32_t n_rcv, const int32_t *rcv_nodes, mss_fine **out);
/* The same leapfrog for any operator, the elastic one included (Section 7's elastic experiment uses
 * it as the reference), on the operator's CSR rows: point sources and receivers at unknowns
 * (host, int64, 0 <= u < N; for the elastic operator unknown 3k + p is component p of kept node k),
 * unit weights; state layout [unknown][source].  One thread per (row, source) forms the row's
 * product in column order.  precision: MSS_FP64 or MSS_FP32.  mss_fine_reset / step / destroy
 * apply unchanged.  Errors: INVALID_ARG (counts, unknowns out of range, precision), CFL (tau <= 0),
 * CUDA, OOM. */
mss_status mss_fine_create_unknowns(const mss_operator *op, int32_t precision, double tau, int32_t n_src,
                                    const int64_t *src_unknowns, int32_t n_rcv, const int64_t *rcv_unknowns,
                                    mss_fine **out);
mss_status mss_fine_reset(mss_fine *f, void *stream);
/* Same waveform/trace conventions as mss_step. */
mss_status mss_fine_step(mss_fine *f, int64_t n_steps, const double *waveform, void *traces, int32_t use_graph,
                         void *stream);
void mss_fine_destroy(mss_fine *f);

/* ------------------------------------------------------------------------- */
/* Learned surrogate of the off-line stage (no counterpart in the paper: it    */
/* replaces the Krylov/Lanczos construction for repeated media; the exact      */
/* construction stays the fallback and decides which cells need it).          */
/* ------------------------------------------------------------------------- */
typedef struct mss_surrogate mss_surrogate;

/* 3D CNN: 3x3x3 convolutions (pad 1) 2 -> C stride 2, stride-2 C -> C convs down to edge 2, one
 * stride-1 C -> C conv, ReLU after each; flattened output ++ n_feat features -> dense H (ReLU) ->
 * dense n_out.  Input x: [batch][2][cell][cell][cell] FP32, features [batch][n_feat], outputs
 * [batch][n_out].  Weights: FP32 masters, BF16 in the forward/backward products, FP32
 * accumulation; seeded normal initialisation.  cell: a power of two in 4..64. */
mss_status mss_surrogate_create(int32_t cell, int32_t n_feat, int32_t n_out, int32_t channels, int32_t hidden,
                                uint64_t seed, mss_surrogate **out);
/* info: [0] parameters, [1] input values per sample, [2] features, [3] outputs. */
mss_status mss_surrogate_info(const mss_surrogate *s, int64_t info[4]);
/* FP32 parameter vector (host): per layer weights then bias, layers in order. set also resets Adam. */
mss_status mss_surrogate_get_params(const mss_surrogate *s, float *host);
mss_status mss_surrogate_set_params(mss_surrogate *s, const float *host);
/* Device buffers; y: [batch][n_out]. */
mss_status mss_surrogate_forward(mss_surrogate *s, int32_t batch, const float *x, const float *feat, float *y,
                                 void *stream);
/* grad (device, n_params) = d sum(dy * forward(x)) / d params (with the BF16-rounded weights). */
mss_status mss_surrogate_backward(mss_surrogate *s, int32_t batch, const float *x, const float *feat, const float *dy,
                                  float *grad, void *stream);
/* One Adam step (beta 0.9 / 0.999) on the mean squared error to target [batch][n_out] (mask of 0/1
 * weights, may be NULL); loss (device float, may be NULL) receives the batch loss. */
mss_status mss_surrogate_train_step(mss_surrogate *s, int32_t batch, const float *x, const float *feat,
                                    const float *target, const float *mask, float lr, float *loss, void *stream);
void mss_surrogate_destroy(mss_surrogate *s);

/* Output transform: predict() returns mean + scale * network, and train_step fits the network
 * to (target - mean) / scale.  set: host arrays [n_out] (both NULL: identity); fit: per-output
 * masked mean and standard deviation (floored at 1e-3 max(1, |mean|)) of targets [n][n_out]. */
mss_status mss_surrogate_set_output_transform(mss_surrogate *s, const float *mean, const float *scale);
mss_status mss_surrogate_fit_output_transform(mss_surrogate *s, int32_t n, const double *targets, const float *mask);
/* Device buffers; y [batch][n_out] = mean + scale * forward. */
mss_status mss_surrogate_predict(mss_surrogate *s, int32_t batch, const float *x, const float *feat, float *y,
                                 void *stream);

/* Surrogate data layout.  A cell's boundary rows go to fixed slots of a padded dimension
 * Kp = 6 slot_modes + io_slots: the face on the low / high side of array axis a fills slot
 * 2a / 2a+1 (its M_f <= slot_modes modes in face order), an I/O face fills the last io_slots
 * rows; absent faces leave their rows empty.  A cell's target vector holds, for Gamma^1..Gamma^m
 * then Gamma-hat^2..Gamma-hat^m (Eq. GammaTrans), the row-major lower triangle (Kp (Kp+1)/2
 * values) of the lower Cholesky factor L (M = L L^T) with log L_ii on the diagonal, so that any
 * prediction unpacks to SPD coefficients; (2m-1) Kp (Kp+1)/2 values per cell.  Slots ascend with
 * the cell's face order, so a cell's rows keep their order and the restriction of a padded
 * factor to them stays lower triangular.  Gamma-hat^1 is not predicted: it is the exact
 * projected inverse mass S^T B^-1 S of the boundary (first Markov parameter, Eq. GammaTrans with
 * G_1 = beta_1^T), which also fixes the face masses (Eq. NtDtri).  Cubic 3D cells only. */

/* Inputs of cells[n] (host): x [n][2][c][c][c] = (log sigma, log rho) of the cell's voxels in
 * array order; feat [n][7] = 1 for each of the 6 face slots present, then (I/O rows)/io_slots.
 * Errors: INVALID_ARG (cells not cubic 3D, a face larger than its slot). */
mss_status mss_surrogate_cell_inputs(const mss_partition *p, int32_t n, const int32_t *cells, int32_t slot_modes,
                                     int32_t io_slots, float *x, float *feat);
/* Targets of cells[n] (all of one m) from a ROM's coefficients: targets [n][(2m-1) Kp(Kp+1)/2]
 * (host doubles), mask (host floats, may be NULL) 1 where the entry belongs to the cell.
 * Errors: COEF_NOT_SPD (a block has no Cholesky factor). */
mss_status mss_surrogate_pack(const mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells,
                              int32_t slot_modes, int32_t io_slots, double *targets, float *mask);
/* Inverse of mss_surrogate_pack: write Gamma^k = L L^T, Gamma-hat^(k>=2) of cells[n] into r
 * (Gamma-hat^1 and the face masses stay). */
mss_status mss_surrogate_unpack(mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells,
                                int32_t slot_modes, int32_t io_slots, const double *packed);
/* Off-line stage without the Krylov/Lanczos part: topology, face bases, exact Gamma-hat^1 of
 * every cell, face masses and Appendix D corner data as mss_build_roms makes them; Gamma^k and
 * Gamma-hat^(k>=2) are zero until mss_surrogate_unpack or mss_rom_rebuild_cells fills them. */
mss_status mss_rom_skeleton(const mss_partition *p, const mss_rom_params *prm, const int32_t *cell_m, mss_rom **out);
/* Exact off-line construction (as mss_build_roms, same parameters) of cells[n] of a ROM built or
 * skeletoned from p, replacing their coefficients.  Errors: STATE (other partition), NOT_CONVERGED. */
mss_status mss_rom_rebuild_cells(mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells, void *stream);
/* Screen of cells[n]: err[n] (host) = ||U^1(s) - F(s)||_F / ||F(s)||_F at the ROM's shift s,
 * U^1 the S-fraction transfer function of the ROM's current coefficients (Eqs. GammaU1st,
 * GammaUrem, tfgamma) and F(s) = C^T (A + sB)^{-1} C of the cell's exact operator (shifted CG
 * on the GPU, FP64).  A singular recursion gives err = 1e300.  Errors: STATE, NOT_CONVERGED. */
mss_status mss_surrogate_screen(const mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells, double *err,
                                void *stream);
/* Surrogate off-line stage for cells[n] (one m) of a ROM from mss_rom_skeleton or mss_build_roms:
 * inputs -> predict (GPU) -> unpack into r -> screen (err[n], host) -> exact rebuild of every cell
 * with err > tol (fallback[n] = 1 for those, host).  The surrogate must have 7 features and
 * (2m-1) Kp(Kp+1)/2 outputs.  Errors: INVALID_ARG, STATE, NOT_CONVERGED, CUDA. */
mss_status mss_surrogate_infer(mss_surrogate *sur, mss_rom *r, const mss_partition *p, int32_t n, const int32_t *cells,
                               int32_t slot_modes, int32_t io_slots, double tol, double *err, int32_t *fallback,
                               void *stream);

/* ------------------------------------------------------------------------- */
/* Stepping without allocation.  The paper has no counterpart: this entry     */
/* point exists for callers that cannot let a library allocate device memory  */
/* -- e.g. a solver embedded in a host application that owns every device     */
/* buffer through its own pool and fixed budget, or a latency-critical loop   */
/* where cudaMalloc/cudaFree would synchronise the device and stall other     */
/* streams.  Such a caller lays out all inputs and outputs itself (same        */
/* layout as an mss_sim, described field by field below) and the library      */
/* only launches kernels.  The one scratch buffer the step needs -- the face   */
/* flux exchange, [face row][side 0/1][source] -- lives in a fixed, file-scope */
/* device array of MSS_NOALLOC_SCRATCH_BYTES that every GPU loading the        */
/* library holds until the process exits.                                     */
/* ------------------------------------------------------------------------- */
#define MSS_NOALLOC_SCRATCH_BYTES (16u << 20)

/* All pointers are device pointers owned by the caller; values are double (MSS_FP64) or float
 * (MSS_FP32).  Sizes: C cells, F faces, S sources, R receivers, Kc = sum of the M_f of cell c's
 * faces, face rows FR = sum_f M_f, hidden rows HR = sum_c (m_c - 1) Kc.
 *   cell_K[C], cell_m[C]            int32  Kc and m_c
 *   cell_coef[C]                     int64  offset (elements) of Gamma^1 of cell c in coef; Gamma^1..m
 *                                           follow, then Gamma-hat^2..m, each Kc x Kc row-major
 *   cell_ghat[C]                     int64  offset of Gamma-hat^2 of cell c (= cell_coef[c] + m_c Kc^2)
 *   cell_state[C]                    int64  first hidden row of cell c (layer 2), layers contiguous
 *   cell_row[C]                      int64  offset of cell c in row_face_row / row_side
 *   row_face_row[sum Kc]             int64  face row of each boundary row of each cell (face order)
 *   row_side[sum Kc]                 int8   0 if the cell is the face's first cell, 1 otherwise
 *   face_M[F], face_two[F]           int32  modes of face f; 1 if the face has two cells
 *   face_row[F], face_minv[F]        int64  first face row of f; offset of M_f^{-1} (M_f x M_f) in minv
 *   fsrc_ptr[F+1], fsrc_index[], fsrc_val[]   sources per face: source index and offset of its
 *                                           M_f projected values in src_val
 *   rcv_ptr[R+1], rcv_face[], rcv_off[]       receivers: faces and offsets of the M_f values in rcv_val
 *   coef, minv, src_val, rcv_val     values as described
 *   face_state[2]  FR x S, cell_state_buf[2]  HR x S: two time levels; level `cur` is "now".
 * max_K, max_m, max_M: maxima of Kc, m_c, M_f.  cur is advanced by the call. */
typedef struct mss_step_buffers {
  int32_t precision, n_cells, n_faces, n_src, n_rcv, max_K, max_m, max_M, cur, reserved;
  int64_t face_rows;
  double tau;
  const int32_t *cell_K, *cell_m;
  const int64_t *cell_coef, *cell_ghat, *cell_state, *cell_row, *row_face_row;
  const int8_t *row_side;
  const int32_t *face_M, *face_two;
  const int64_t *face_row, *face_minv;
  const int32_t *fsrc_ptr, *fsrc_index;
  const int64_t *fsrc_val;
  const int32_t *rcv_ptr, *rcv_face;
  const int64_t *rcv_off;
  const void *coef, *minv, *src_val, *rcv_val;
  void *face_state[2], *cell_state_buf[2];
} mss_step_buffers;

/* n_steps of the same step as mss_step without the corner correction, launched eagerly on
 * `stream` with the flux exchange in the library's fixed scratch array.
 * waveform: device FP64, n_steps samples; traces: device [n_steps][R][S] of the precision.
 * Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).  The first call on a
 * device looks up the scratch array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is cached for the rest
 * of the process: after cudaDeviceReset on a device, do not call this entry point on it again
 * (the cached address would be stale).  Every call on a device shares the
 * one scratch array and leaves its contents behind (the step writes every flux slot before it
 * reads it, so nothing needs clearing); calls that overlap on the GPU (different streams, or
 * different threads) race on it and must be serialised by the caller.
 * The four state buffers must be 16-byte aligned (vector loads).  face_rows must equal FR, the
 * sum of face_M: the kernels index the scratch through face_row and row_face_row, so a smaller
 * face_rows passes the size check below and then writes past the end of the scratch array.
 * Errors: INVALID_ARG (null pointers, counts, precision, alignment), INVALID_ARG if 2 FR S x
 * element size exceeds MSS_NOALLOC_SCRATCH_BYTES, CUDA. */
mss_status mss_step_noalloc(mss_step_buffers *b, int64_t n_steps, const double *waveform, void *traces,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MSS_H */
