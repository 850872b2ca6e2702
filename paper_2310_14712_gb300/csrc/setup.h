// Host-side setup of the immersed Newmark IMEX method (C++17, no CUDA types).
//
// Everything the time-stepping kernels need is computed here once, on the host:
// the 1D spectral basis, cell classification and spacetree quadrature of cut
// cells, the DOF partition, the dense cut-cell element matrices, the implicit
// system S = M^cc + beta dt^2 K^cc and M^cc with their supernodal
// nested-dissection Cholesky factors, and the source vector f_x.
// (Paper: Sec. "Spatial discretization", Sec. "Partitioning", Fig. TrapCDMIMEX
// "Calculation and factorization of system matrix".)
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace imex {

enum CellType : int8_t { CELL_UNCUT = 0, CELL_CUT = 1, CELL_EMPTY = 2 };
enum NodeClass : uint8_t { NODE_INACTIVE = 0, NODE_D = 1, NODE_C = 2 };

constexpr int kMaxCols = 256;   // independent source columns of one context

struct Problem {
  int dim = 2;
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int ncells[3] = {1, 1, 1};
  int p = 1;
  double alpha = 1e-5;
  int depth = 0;
  std::vector<double> holes;   // nholes x (centre[dim], semi_axes[dim])
  double rho = 1.0, c0 = 1.0;
  std::vector<double> cell_c;  // optional per-cell wave speed, flat cell order (x fastest)
  int nsrc = 1;
  std::vector<double> src_pos; // nsrc x dim
  int ncols = 1;               // > 1: independent columns, column k loaded by source k alone
  double f0 = 1.0, sigma = 0.1, amp = 10.0;
  int wavelet = 0;
  double dt = 0.0;             // <= 0: dt_factor * the scheme's cell-wise critical step
  double dt_factor = 0.9;
  int scheme = 0;              // kScheme*
  bool factorize = true;       // false: no dissection and no factorisation (iterative solve only)
  std::vector<int64_t> export_cells;  // cells whose element matrices are kept (HostSetup::export_K/M)
};

// Time integration schemes on the same discretisation (the method and the
// paper's comparison schemes).  The values are the public IMEX_SCHEME_* codes.
constexpr int kSchemeImex = 0;         // Newmark IMEX (Fig. TrapCDMIMEX)
constexpr int kSchemeCdm = 1;          // central differences, consistent cut-cell masses
constexpr int kSchemeCdmHrz = 2;       // central differences, HRZ-lumped cut-cell masses (Eqs. HRZ)
constexpr int kSchemeTrapezoidal = 3;  // trapezoidal Newmark on every DOF
inline bool scheme_is_cdm(int s) { return s == kSchemeCdm || s == kSchemeCdmHrz; }

// One node of the nested-dissection tree of the implicit partition.  Its DOFs
// are the contiguous c-index range [beg, end); `rows` are the ancestor
// c-indices in the column structure of L below the diagonal block.
struct TreeNode {
  int beg = 0, end = 0;
  int parent = -1;
  int level = 0;               // 0 = leaf level; parent level > child level
  int comp = 0;
  std::vector<int> rows;
  int64_t off_diag = 0;        // offset of L_tt^{-1} (column-major, b x b) in the value array
  int64_t off_diagT = 0;       // offset of (L_tt^{-1})^T (column-major, b x b)
  int64_t off_rect = 0;        // offset of L_{rows,t} (column-major, m x b)
  int64_t off_rectT = 0;       // offset of L_{rows,t}^T (column-major, b x m)
  int64_t off_rows = 0;        // offset of `rows` in the index array
  int64_t off_upd = 0;         // offset of this node's update vector in the scratch array
};

struct Factor {
  std::vector<double> vals;    // per tree node: L_tt^{-1}, its transpose, L_{rows,t}, its transpose
  std::vector<double> Ld;      // per tree node: L_tt itself (column-major), host only
  std::vector<int64_t> ld_off; // offset of each node's L_tt in Ld
};

struct HostSetup {
  Problem pb;
  int dim = 2, p = 1, P = 2, Pd = 4;
  double h[3] = {1, 1, 1};
  int nn[3] = {1, 1, 1};       // nodes per axis
  int64_t nnodes = 0;
  int ncell_total = 0;
  std::vector<int8_t> cell_type;
  std::vector<double> fill;
  std::vector<uint8_t> node_class;
  int64_t n_d = 0, n_c = 0, n_cut = 0, n_uncut = 0, n_empty = 0;
  std::vector<int> c_node;     // c-index -> grid node
  std::vector<int> node_c;     // grid node -> c-index or -1
  std::vector<double> fx;      // full grid, canonical order; ncols grids, column after column

  // 1D operators on [-1,1] (exact Gauss-Legendre integrals of the GLL basis).
  std::vector<double> gll_x, gll_w, K1, M1;   // K1, M1 are P x P row-major
  std::vector<double> uncutK;  // Pd x Pd dense uncut-cell stiffness (c = c0), column-major

  // Interface cells: every non-empty cell containing at least one c-node.
  std::vector<int> if_cell;    // flat cell id
  std::vector<int> if_kidx;    // index into cutK (>= 0) or -1 (uncut form)
  std::vector<double> if_c2;   // c^2 multiplier for the uncut form (c_e^2 / c0^2)
  std::vector<double> cutK;    // n_cut x Pd x Pd, column-major per cell
  // Element matrices of Problem::export_cells as assembled (Pd x Pd each,
  // column-major): cut cells by spacetree quadrature, uncut cells the
  // reference form (stiffness scaled by c_e^2 / c0^2, GLL-lumped mass),
  // empty cells zero.
  std::vector<double> export_K, export_M;
  // For each c-index r: list of positions (if_cell * Pd + local node) whose
  // element products add into row r of K^c u.
  std::vector<int> contrib_ptr, contrib_pos;

  // Nested-dissection tree (all components), postorder, c-index ranges.
  std::vector<TreeNode> tree;
  std::vector<int> comp_tree_ptr;   // component k owns tree nodes [ptr[k], ptr[k+1]) (postorder)
  std::vector<int> comp_level_ptr;  // per component: nlevels+1 offsets into level_nodes
  std::vector<int> comp_level_base; // per component: offset into comp_level_ptr
  std::vector<int> level_nodes;     // tree node ids grouped by (component, level)
  std::vector<int> rows_idx;        // concatenated `rows` of all tree nodes
  std::vector<int> fwd_ptr, fwd_pos;// per c-index: scratch positions of descendant updates
  int64_t upd_size = 0;
  int max_block = 0, max_rows = 0, ncomp = 0, max_comp = 0;
  Factor S, Mcc;
  // S itself (c-order, full symmetric pattern, CSR): the operator of the
  // iterative solve and of preconditioner training.
  std::vector<int> S_ptr, S_col;
  std::vector<double> S_val;
  std::vector<double> M_val;   // M^cc on the pattern of S (zeros where M^cc has none)
  int64_t nnz_L = 0;
  double residual_S = 0, residual_M = 0;  // ||A x - b|| / ||b|| of a host replay of the device solve

  double dt = 0, dt_crit_uncut = 0;
  // Smallest cell-wise critical step of the cut cells for the mass the scheme
  // uses (central-difference schemes only; 0 when not computed).
  double dt_crit_cut_min = 0;
  double setup_seconds = 0;
};

// Build everything; returns "" on success or an error message.
std::string build_setup(const Problem& pb, HostSetup& out);

// Host replay of the supernodal tree solve, x = A^{-1} b (x holds b on entry).
void replay_solve(const HostSetup& hs, const Factor& F, std::vector<double>& x);

// Pieces exposed for host-side tests through the C-ABI.
void gll_points(int p, std::vector<double>& x, std::vector<double>& w);
void gauss_points(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace imex
