// Time-stepping kernels of the immersed Newmark IMEX method (sm_103a, FP64).
//
// One IMEX step (Fig. TrapCDMIMEX) is these launches:
//   k_explicit   A1 + A2: K^d u_n over uncut cells by sum factorisation on the
//                tensor grid (exact for every I_d row, whose cells are all
//                uncut), fused with the CDM update on the lumped mass
//                (Eqs. CDMacc, CDMstep); extra blocks do the Newmark
//                prediction on I_c (A3).
//   k_walk / k_top   A4 + A5 + A6: right-hand side f_t(t_{n+1}) f_x^c -
//                K^c u_pred (row by row from the interface cells' matrices, in
//                the first forward launch), forward walk over the lower levels
//                of the supernodal nested-dissection Cholesky factor of S
//                (inverted diagonal blocks), one dense product per component
//                for the upper levels, backward walk, Newmark correction.  One
//                launch per level; kernel boundaries are the level barriers,
//                so every launch can use every SM.
#pragma once
#include <cstdint>

namespace imex {

constexpr double kNewmarkBeta = 0.25;
constexpr double kNewmarkGamma = 0.5;

// Source time function f_t (Sec. Spatial discretization, f(t) = f_t(t) f_x).
__host__ __device__ inline double wavelet_value(int kind, double f0, double t) {
  const double pi = 3.14159265358979323846;
  if (kind == 0) {  // Ricker, centred at 1/f0
    double s = pi * f0 * (t - 1.0 / f0);
    double a = s * s;
    return (1.0 - 2.0 * a) * exp(-a);
  } else if (kind == 1) {  // Eq. ft: derivative of a Gaussian, t0 = 1/f0, sigma_t = 1/(2 pi f0)
    double t0 = 1.0 / f0, sg = 1.0 / (2.0 * pi * f0);
    double d = t - t0;
    return -d / (sqrt(2.0 * pi) * sg * sg * sg) * exp(-d * d / (2.0 * sg * sg));
  } else {  // two-cycle sine burst of the 3D example
    const double nc = 2.0;
    if (t > nc / f0) return 0.0;
    double s = sin(pi * f0 * t / nc);
    return sin(2.0 * pi * f0 * t) * s * s;
  }
}

// 1D operators of the explicit apply (2D):
//   r = sx (M1_y (x) K1_x) u + sy (K1_y (x) M1_x) u
// K1 (stiffness) in even-odd form, rows i <= (P-1)/2:
//   ke[i][j] = (A[i][j] + A[i][P-1-j]) / 2, ko[i][j] = (A[i][j] - A[i][P-1-j]) / 2
//   (j < H = P/2), kc[i] = A[i][H] (P odd);  then for i < H, with e_j, o_j the
//   even and odd parts of v:  (A v)_i = Ev_i + Od_i, (A v)_{P-1-i} = Ev_i - Od_i.
// M1 (mass) = diag(w) + C a a^T; ca = C a.
// The 2D kernels apply dt^2 M^{-1} K with the inverse lumped mass folded in:
// on a uniform grid M^{-1} of an explicit node is (1/W_x)(1/W_y)/(rho |J|)
// with per-axis assembled GLL weights W, which per local node are w_i
// (interior) or 2 w_0 (a vertex shared by two cells; w_0 at the grid's edge,
// where the kernels double the vertex sum exactly).  So with f_i = 1/w_i or
// 1/(2 w_0) and kappa = dt^2 / (rho |J|):
//   x pass  A = f (x) sx K1 (kxe, kxo, kxc),  M1 -> f M1: interior rows
//           v_i + cax_i (a^T v), vertex rows v_i / 2 + cax_i (a^T v),
//   y pass  A = kappa f (x) sy K1 (kye, kyo, kyc),  M1 -> kappa f M1:
//           wy_i v_i + cay_i (a^T v).
// At a vertex the two cells' halves of the nodal term go to one cell (the
// x pass's last node: v; the y pass's last node: wyv = kappa times v).
// (3D builds its Ops3D from the unscaled form: w, ca.)
struct Ops2D {
  double kxe[5][4], kxo[4][4], kxc[5];
  double kye[5][4], kyo[4][4], kyc[5];
  double w[9], ca[9], a[9];
  double cax[9], wy[9], cay[9];
  double wyv;   // kappa: the whole nodal mass share of a vertex in y (split asymmetrically)
};

// 1D operators of the 3D explicit apply:
//   r = sx (M1_z (x) M1_y (x) K1_x) u + sy (M1_z (x) K1_y (x) M1_x) u
//     + sz (K1_z (x) M1_y (x) M1_x) u
// K1 in even-odd form per axis (scaled by sx, sy, sz), M1 = diag(w) + C a a^T.
struct Ops3D {
  double ke[3][5][4], ko[3][4][4], kc[3][5];
  double w[9], ca[9], a[9];
};

struct ExplicitArgs {
  const double* U;        // u_n (full grid)
  const double* W;        // u_{n-1} (step) or v_0 (init), full grid
  double* OUT;            // u_{n+1} on I_d (may alias W); u_pred on I_c
  const uint8_t* cls;     // node class (0 inactive, 1 I_d, 2 I_c)
  const double* fx;       // f_x, full grid
  const double* winv_x;   // 1 / assembled GLL weight along x, per node column
  const double* winv_y;   // idem along y (2D: scaled by dt-independent 1/(rho |J|))
  const double* winv_z;   // 3D: idem along z, scaled by 1/(rho |J|)
  int nx, ny, nz;         // nodes per axis (nz = 1 in 2D)
  int ncx, ncy, ncz;      // cells per axis
  int ntx, nty, ntz;      // tiles per axis
  double cu, cw, ca;      // out = cu u + cw w + ca minv (ft fx - r)
  const double* fxs;      // 2D: dt^2 M^{-1} f_x per node (explicit nodes), full grid
  double kappa2;          // 2D: ca / dt^2 (the kernels form dt^2 M^{-1} (ft fx - r))
  double ft;              // f_t(t_n)
  const double* ft_dev;   // if set: f_t(t_n) = ft_dev[0] (user-supplied samples)
  // Newmark prediction on I_c (blocks after the tiles); n_c = 0 disables it.
  int n_c;
  const int* c_node;
  const double* v_c;
  const double* a_c;
  double dt;
  // independent columns (blockIdx.y): strides of full-grid and I_c fields
  int64_t cs_node, cs_c;
  // 2D tiles: if set, CTA b takes tile tiles[b] (b < ntl; the CTAs after
  // them predict); persistent: a fixed grid loops over the ntl x ncols
  // (tile, column) items of the list instead, without prediction.
  const int* tiles;
  int ntl;
  int persistent;
  int ncols;
};

// One level of the supernodal walk of A5 (forward or backward), all
// components at once.  The level's supernodes are packed into CTAs; each
// CTA's blocks [L_tt^{-1} packed by diagonals | L_{rows,t} (ld m|1)] are
// stored contiguously in `blob`, its index list (layout in imex.cu,
// WalkList) in `ilist`.  The first forward launch also forms the right-hand sides (A4).
struct WalkArgs {
  int cta0;                     // first CTA of this level in the per-CTA arrays
  const double* blob;
  const int64_t* blob_off;      // [cta] (16-byte aligned)
  const int64_t* blob_len;      // [cta] (even)
  int64_t max_blob;             // doubles reserved for the blob in shared memory (even; 0 if not staged)
  const int* ilist;
  const int64_t* ilist_off;     // [cta] (multiple of 4)
  const int64_t* ilist_len;     // [cta] (multiple of 4)
  int max_slots, max_m, max_pairs;  // shared-memory vector sizes (even)
  // right-hand sides f_t f_x^c - K^c u (first forward launch)
  int first;
  int rhs_only;                 // first launch: only form the right-hand sides (into rhs0)
  int rhs_given;                // first launch: every right-hand side is already in rhs0
  const int* skip;              // if set and *skip != 0: the launch does nothing (PCG converged)
  const double* SRC;            // u_pred (step), u_n (mode 3) or u_0 (initial acceleration), full grid
  const double* Kpair;          // per CTA: rows of the cell matrices of its pairs (m-major, scaled)
  const int64_t* kp_off;        // [cta] (16-byte aligned)
  const int64_t* kp_len;        // [cta] (even)
  int64_t max_kp;               // doubles reserved for them in shared memory (even)
  int kp_smem;                  // 1: staged in shared memory; 0: read from global memory
  int P, Pd, dim, nx, ny;
  const double* fxc;
  double ft;                    // f_t(t_{n+1}) (step; t_n in mode 3) or f_t(0) (initial acceleration)
  const double* ft_dev;         // if set: f_t(t_{n+1}) = ft_dev[1] (mode 3: f_t(t_n) = ft_dev[0])
  double* rhs0;                 // right-hand side of every c-row not solved by the first launch
  double* upd;
  double* sol;
  // correction of the rows this launch finalises (backward only)
  int mode;                     // 0: Newmark correction; 1: store the acceleration only;
                                // 2: nothing (solution left in sol); 3: central-difference update
  const int* c_node;
  double* U;                    // holds u_pred (mode 0) or u^c_{n-1} (mode 3) on I_c; receives u^c_{n+1}
  double* v_c;
  double* a_c;
  double dt;
  // independent columns: strides of full-grid, I_c and update fields; a CTA
  // takes the block of cb columns blockIdx.y * cb ... (of ncols)
  int64_t cs_node, cs_c, cs_upd;
  int cb, ncols;
};

// Dense top block of every component: x_Z = A_Z (rhs_Z - updates from the
// walked levels), A_Z = (L_ZZ L_ZZ^T)^{-1}; each CTA owns a chunk of rows.
struct TopArgs {
  const int* cta_comp;          // [cta] component
  const int* cta_r0;            // [cta] first row of the chunk (within the component's Z)
  const int* cta_r1;
  const int* zsize;             // [comp] |Z|
  const int* zbase;             // [comp] offset into zrow
  const int* zrow;              // c-index of each Z row
  const int64_t* zA_off;        // [comp] offset of A_Z (|Z| x |Z|, 16-byte aligned; each CTA's chunk of rows column-major)
  const double* zA;
  int max_zn;                   // even
  int64_t max_arows;            // even: largest (r1 - r0) * |Z| over the CTAs
  const int* skip;              // if set and *skip != 0: the launch does nothing (PCG converged)
  const int* ilist;             // per component: per Z row {update begin, update end}, then positions
  const int64_t* ilist_off;     // [cta]
  const int64_t* ilist_len;     // [cta]
  const double* rhs0;
  const double* upd;
  double* sol;
  int mode;
  const int* c_node;
  double* U;
  const double* Un;             // u_n for the central-difference update (mode 3)
  double* v_c;
  double* a_c;
  double dt;
  int64_t cs_node, cs_c, cs_upd;  // independent columns: strides
  int cb, ncols;                  // a CTA takes the block of cb columns blockIdx.y * cb ... (of ncols)
};

// Large supernodes of the walked levels (more than 256 diagonal or ancestor
// rows), one launch per level and phase, each CTA one chunk of rows of a
// dense block times a gathered vector:
//   kind 0 (forward)   y_t = L_tt^{-1} g_t, g_t = rhs - descendant updates -> sol
//   kind 1 (forward)   upd_t = L_{rows,t} y_t                               -> upd
//   kind 2 (backward)  h_t = y_t - L_{rows,t}^T x_rows                      -> hbuf
//   kind 3 (backward)  x_t = L_tt^{-T} h_t, then the correction of the row -> sol
// Per CTA: desc[8 cta + 0..3] = kind, nr (rows), nv (vector length), index
// list offset; the chunk is nr x nv, column-major (row i, column j at
// j nr + i), at a_off[cta] in A.  Index list: nv input c-indices (kind 0:
// then 2 nv update ranges into the list itself), nr output indices (c-rows;
// kind 1: update positions), then kind 0's update positions.
struct PanelArgs {
  int cta0;
  const int* desc;
  const int64_t* a_off;
  const double* A;
  const int* idx;
  int64_t max_chunk;            // doubles reserved for a chunk in shared memory (even)
  int max_nv;                   // doubles reserved for the vector (even)
  const int* skip;              // if set and *skip != 0: the launch does nothing (PCG converged)
  const double* rhs0;
  double* upd;
  double* sol;
  double* hbuf;
  int mode;                     // correction mode (WalkArgs)
  const int* c_node;
  double* U;
  const double* Un;
  double* v_c;
  double* a_c;
  double dt;
  int64_t cs_node, cs_c, cs_upd;
};

// Preconditioned conjugate gradients for S a = rhs (the iterative alternative
// to A5), one cooperative grid, single column.
struct PcgArgs {
  int n;                          // implicit rows (c-order)
  const int* s_ptr;               // S, CSR, full symmetric pattern
  const int* s_col;
  const double* s_val;
  const int* g_ptr;               // G, CSR, lower triangle of S's pattern
  const int* g_col;
  const double* g_val;
  const int* gt_ptr;              // G^T: per column j the entries (row, index into g_val)
  const int* gt_row;
  const int* gt_idx;
  const double* dinv;             // 1 / S_ii
  int precond;                    // 1: M^{-1} = G G^T; 2: M^{-1} = diag(S)^{-1}
  const double* b;                // right-hand side
  double *x, *r, *z, *p, *q, *w;  // n each: iterate, residual, u = M^{-1} r, direction, S p, G^T r
  double* v;                      // n: S u
  double* part;                   // 10 x gridDim.x block partial sums
  double tol;                     // stop when ||r|| <= tol ||b||
  int maxit;
  int* status;                    // [0] iterations of the last solve, [1] 1: converged, 0: fallback
  long long* counters;            // [0] iterations summed, [1] fallbacks
  double* res;                    // relative residual of the last solve
  // Learned starting guess: x0 = w0 a^c_n + w1 a^c_{n-1} + w2 a^c_{n-2} when
  // guess_w is set (device, 3 weights), else x0 = a^c_n; the two history
  // vectors are shifted every solve (hist1 <- a^c_n, hist2 <- hist1).
  const double* guess_w;
  double* hist1;
  double* hist2;
  // Newmark correction on convergence (as in the direct solve), or always
  // (always_correct: no direct solve to fall back on; misses are counted)
  int always_correct;
  int mode;
  const int* c_node;
  double* U;
  double* v_c;
  double* a_c;
  double dt;
};

// Cell-by-cell form of K used where the tensor-grid apply does not apply
// (per-cell wave speed, the adjoint): every non-empty cell e has its nodal
// block at cell_base[e] (+ the local offsets of a cell), its matrix row-major
// in Kall (cut cells: their stored matrix; uncut cells: the uncut matrix),
// and weight w[e] (c_e^2 / c0^2 for uncut cells, 1 for cut cells, whose
// stored matrices carry c_e^2).  Each node lists its cells (CSR), so a row
// of K x is gathered in a fixed order.
struct HetArgs {
  int ncell;                      // non-empty cells
  const int* cell_base;
  const int* cell_koff;           // matrix index into Kall (Pd x Pd each)
  const double* cell_w;
  const double* cell_c;           // wave speed c_e
  const int* cell_id;             // flat cell id (gradient index)
  const double* Kall;
  const int* nc_ptr;              // node -> its (cell, local node) entries
  const int* nc_cell;
  const int* nc_local;
  int P, Pd, dim, nx, ny;
  int64_t nnodes;
};

}  // namespace imex
