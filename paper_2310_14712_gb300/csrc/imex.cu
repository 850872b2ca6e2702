// libimex: device state, time-stepping kernels and the C-ABI (include/imex.h).
//
// Paper: Faßbender et al., "Implicit-Explicit Time Integration for the Immersed
// Wave Equation", Sec. "Time integration", Fig. TrapCDMIMEX (Newmark IMEX),
// Eqs. CDMstep / CDMacc (diagonal CDM step), Eqs. Newmark1/2 (prediction and
// correction, beta = 1/4, gamma = 1/2), Eqs. Kd / Kc (partitioned stiffness).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>
#include <thread>
#include <mutex>

#include "../../include/imex.h"
#include "kernels.cuh"
#include "setup.h"

using namespace imex;
namespace cg = cooperative_groups;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

constexpr int kThreads = 256;
constexpr int kIoRing = 8;   // slots of the host-I/O rings (imex_step_io)
constexpr int kWarps = kThreads / 32;

#include "step_kernels.cuh"

// ---------------------------------------------------------------------------
// Iterative alternative for A5: preconditioned conjugate gradients (Saad,
// Algorithm 9.1) on S a = rhs with M^{-1} = G G^T (G lower triangular on the
// pattern of S, learned) or diag(S)^{-1}, started from the previous
// acceleration, stopped at ||r|| <= tol ||b||.  One cooperative grid runs all
// iterations; grid-wide barriers separate the phases that read other
// threads' rows.  Every block sums the block partials of a dot product in the
// same order, so all blocks take the same decisions and the result is
// deterministic.  On convergence the kernel applies the Newmark correction;
// otherwise it leaves the state alone and the direct solve that follows runs
// (its launches test status[1]).

// Block partial of a sum into part[slot * gridDim.x + blockIdx.x].
__device__ __forceinline__ void block_partial(double v, double* part, int slot, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red[w];
    part[(size_t)slot * gridDim.x + blockIdx.x] = s;
  }
  __syncthreads();
}

// Sum of the block partials of `slot`, the same bits in every thread.
__device__ __forceinline__ double grid_total(const double* part, int slot) {
  double s = 0.0;
  for (int b = threadIdx.x % 32; b < (int)gridDim.x; b += 32) s += __ldcg(part + (size_t)slot * gridDim.x + b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Values of G in the column order of its transpose lists (gt_val[k] =
// g_val[gt_idx[k]]), refreshed whenever G changes: G^T r then streams them.
struct PcgCols {
  const double* gt_val;
};

template <int LPR>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgs a, PcgCols t2) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[kWarps];
  const int n = a.n;
  const int g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  // Sparse products: a group of LPR lanes per row (32 / LPR rows per warp in
  // flight), lanes striding the row (coalesced column and value loads), a
  // fixed xor tree within the group sums them; every lane of the group gets
  // the value.  Rows go to warps in rounds, the same number for every lane
  // of a warp.
  constexpr int GPW = 32 / LPR;
  const int lane = threadIdx.x & 31, w0 = g0 >> 5, ws = gs >> 5;
  const int sub = lane % LPR, grp = lane / LPR;
  auto group_dot = [&](const int* ptr, const int* col, const double* val, const double* v, int i, bool ok) {
    double t0 = 0.0, t1 = 0.0;
    if (ok) {
      const int end = ptr[i + 1];
      int k = ptr[i] + sub;
      for (; k + LPR < end; k += 2 * LPR) {   // two independent gathers in flight per lane
        const int c0 = col[k], c1 = col[k + LPR];
        const double v0 = val[k], v1 = val[k + LPR];
        t0 = fma(v0, __ldcg(v + c0), t0);
        t1 = fma(v1, __ldcg(v + c1), t1);
      }
      if (k < end) t0 = fma(val[k], __ldcg(v + col[k]), t0);
    }
    double t = t0 + t1;
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
  };
  // z = M^{-1} r
  auto apply_minv = [&]() {
    if (a.precond == 2) {
      for (int i = g0; i < n; i += gs) a.z[i] = a.dinv[i] * a.r[i];
    } else {
      for (int base = w0 * GPW; base < n; base += ws * GPW) {   // w = G^T r, column j of G
        const int j = base + grp;
        const double wj = group_dot(a.gt_ptr, a.gt_row, t2.gt_val, a.r, j, j < n);
        if (sub == 0 && j < n) a.w[j] = wj;
      }
      grid.sync();
      for (int base = w0 * GPW; base < n; base += ws * GPW) {
        const int i = base + grp;
        const double zi = group_dot(a.g_ptr, a.g_col, a.g_val, a.w, i, i < n);
        if (sub == 0 && i < n) a.z[i] = zi;
      }
      grid.sync();   // z is read below by other threads than its writers
    }
  };
  if (a.hist1) {   // learned starting guess (or a^c_n), then shift the history
    const double w0 = a.guess_w ? a.guess_w[0] : 1.0, w1 = a.guess_w ? a.guess_w[1] : 0.0,
                 w2 = a.guess_w ? a.guess_w[2] : 0.0;
    for (int i = g0; i < n; i += gs) {
      const double an = a.a_c[i], h1 = a.hist1[i], h2 = a.hist2[i];
      a.x[i] = a.guess_w ? fma(w0, an, fma(w1, h1, w2 * h2)) : an;
      a.hist2[i] = h1;
      a.hist1[i] = an;
    }
  } else {
    for (int i = g0; i < n; i += gs) a.x[i] = a.a_c[i];
  }
  grid.sync();
  double bb = 0.0, rr = 0.0;
  for (int base = w0 * GPW; base < n; base += ws * GPW) {
    const int i = base + grp;
    const double ri0 = group_dot(a.s_ptr, a.s_col, a.s_val, a.x, i, i < n);
    if (sub == 0 && i < n) {
      const double bi = a.b[i], ri = bi - ri0;
      a.r[i] = ri;
      bb = fma(bi, bi, bb);
      rr = fma(ri, ri, rr);
    }
  }
  block_partial(bb, a.part, 3, red);
  block_partial(rr, a.part, 1, red);
  grid.sync();
  const double nb2 = grid_total(a.part, 3);
  double rr_t = grid_total(a.part, 1);
  const double tol2 = a.tol * a.tol * nb2;
  bool conv = rr_t <= tol2;
  int k = 0;
  if (!conv) {
    // Preconditioned CG in the single-reduction form of Chronopoulos and
    // Gear (Chronopoulos & Gear 1989, J. Comput. Appl. Math. 25): besides p
    // it carries s = S p, so that per iteration the three inner products
    // gamma = (r, u), delta = (S u, u) and (r, r) (u = M^{-1} r) are formed
    // in one reduction: one grid barrier for them, one before S u, and two
    // inside G G^T r (FSAI) or none (Jacobi, applied elementwise).  In exact
    // arithmetic the iterates are those of standard PCG.  Partial sums
    // alternate between two sets of slots by iteration parity, because the
    // next iteration writes them before its next barrier.
    auto reduce3 = [&](double gam, double del, double rr2, int set, double& G, double& D, double& R) {
      block_partial(gam, a.part, 4 + 3 * set, red);
      block_partial(del, a.part, 5 + 3 * set, red);
      block_partial(rr2, a.part, 6 + 3 * set, red);
      grid.sync();
      G = grid_total(a.part, 4 + 3 * set);
      D = grid_total(a.part, 5 + 3 * set);
      R = grid_total(a.part, 6 + 3 * set);
    };
    // w = S u, with the partials of (r, u) and (w, u) of this thread's rows.
    auto apply_S_u = [&](double& gam, double& del) {
      for (int base = w0 * GPW; base < n; base += ws * GPW) {
        const int i = base + grp;
        const double wi = group_dot(a.s_ptr, a.s_col, a.s_val, a.z, i, i < n);
        if (sub == 0 && i < n) {
          const double ui = a.z[i];
          a.v[i] = wi;
          gam = fma(a.r[i], ui, gam);
          del = fma(wi, ui, del);
        }
      }
    };
    apply_minv();
    if (a.precond == 2) grid.sync();   // u complete before S u
    double gam = 0.0, del = 0.0, R = rr_t;
    apply_S_u(gam, del);
    double rr_unused = 0.0;
    reduce3(gam, del, rr_unused, 0, gam, del, rr_unused);
    double alpha = gam / del, beta = 0.0;
    for (k = 1; k <= a.maxit; ++k) {
      double rr2 = 0.0;
      for (int i = g0; i < n; i += gs) {
        // First iteration: p = u, s = S u (p and s hold nothing yet).
        const double pi = k == 1 ? a.z[i] : fma(beta, a.p[i], a.z[i]);
        const double si = k == 1 ? a.v[i] : fma(beta, a.q[i], a.v[i]);
        a.p[i] = pi;
        a.q[i] = si;
        a.x[i] = fma(alpha, pi, a.x[i]);
        const double ri = fma(-alpha, si, a.r[i]);
        a.r[i] = ri;
        rr2 = fma(ri, ri, rr2);
        if (a.precond == 2) a.z[i] = a.dinv[i] * ri;
      }
      if (a.precond == 2) grid.sync();   // u complete before S u
      else {
        grid.sync();                      // r complete before G^T r
        apply_minv();                     // ends with u complete
      }
      double g1 = 0.0, d1 = 0.0;
      apply_S_u(g1, d1);
      reduce3(g1, d1, rr2, k & 1, g1, d1, R);
      rr_t = R;
      if (rr_t <= tol2) {
        conv = true;
        break;
      }
      beta = g1 / gam;
      alpha = g1 / (d1 - beta * g1 / alpha);
      gam = g1;
    }
    if (k > a.maxit) k = a.maxit;
  }
  if (conv || a.always_correct) {
    const Corr cor{a.mode, a.c_node, a.U, a.v_c, a.a_c, a.dt, nullptr};
    for (int i = g0; i < n; i += gs) cor.row(i, a.x[i]);
  }
  if (g0 == 0) {
    a.status[0] = k;
    a.status[1] = conv ? 1 : 0;
    a.counters[0] += k;
    a.counters[1] += conv ? 0 : 1;
    *a.res = nb2 > 0.0 ? sqrt(rr_t / nb2) : 0.0;
  }
}

// Right-hand sides of the implicit rows without a solve plan (one warp per
// row): rhs_r = f_t f^c_r - sum over the row's (interface cell, local row)
// pairs of sc_e (row of the cell matrix) . (the cell's nodal values of src),
// the same pairs and cell matrices as the first walk launch uses (Eq. Kc).
__global__ void __launch_bounds__(kThreads) k_rhs_c(int n_c, const int* pr_ptr, const int* pr_pos,
                                                    const int* if_base, const int* if_koff, const double* if_sc,
                                                    const double* Krows, int P, int Pd, int nx, int ny,
                                                    const double* fxc, double ft, const double* ft_dev,
                                                    const double* src, double* rhs) {
  const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32), lane = threadIdx.x % 32;
  if (r >= n_c) return;
  double acc = 0.0;
  for (int q = pr_ptr[r]; q < pr_ptr[r + 1]; ++q) {
    const int e = pr_pos[q] / Pd, l = pr_pos[q] % Pd;
    const double* row = Krows + ((size_t)if_koff[e] * Pd + l) * Pd;
    const double* u = src + if_base[e];
    double t = 0.0;
    for (int m = lane; m < Pd; m += 32)
      t = fma(row[m], __ldg(u + (m % P) + nx * ((m / P) % P) + nx * ny * (m / (P * P))), t);
    acc = fma(if_sc[e], t, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) rhs[r] = (ft_dev ? ft_dev[1] : ft) * fxc[r] - acc;   // ft_dev[1] = f_t(t_{n+1})
}

// Training of G (Kaporin's functional K(G) = tr(G^T S G) - 2 sum log G_ii on
// the lower pattern; Adam).  sg = (S G) on the pattern of G: for entry
// (i, j), sum over S's row i of S_ik G_kj (G_kj found in G's row k, k >= j).
__global__ void k_kap_sg(int n, const int* s_ptr, const int* s_col, const double* s_val, const int* g_ptr,
                         const int* g_col, const double* g_val, double* sg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = g_ptr[i]; e < g_ptr[i + 1]; ++e) {
    const int j = g_col[e];
    double s = 0.0;
    for (int t = s_ptr[i]; t < s_ptr[i + 1]; ++t) {
      const int kk = s_col[t];
      if (kk < j) continue;
      int lo = g_ptr[kk], hi = g_ptr[kk + 1];
      while (lo < hi) {   // first entry of row kk with column >= j
        const int mid = (lo + hi) / 2;
        if (g_col[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      if (lo < g_ptr[kk + 1] && g_col[lo] == j) s = fma(s_val[t], g_val[lo], s);
    }
    sg[e] = s;
  }
}

// Gradient 2 sg - 2 delta_ij / G_ii and the per-block partials of K.
__global__ void k_kap_grad(int n, const int* g_ptr, const int* g_col, const double* g_val, const double* sg,
                           double* grad, double* part) {
  __shared__ double red[kWarps];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    for (int e = g_ptr[i]; e < g_ptr[i + 1]; ++e) {
      double g = 2.0 * sg[e];
      l = fma(g_val[e], sg[e], l);
      if (g_col[e] == i) {
        g -= 2.0 / g_val[e];
        l -= 2.0 * log(g_val[e]);
      }
      grad[e] = g;
    }
  }
  block_partial(l, part, 0, red);
}

// One Adam step (Kingma and Ba, Algorithm 1) in row-scaled units theta =
// G_ij / scale_ij; the diagonal stays >= floor.  Writes the new G values.
__global__ void k_adam(int64_t nnz, double* theta, const double* grad, const double* scale, const uint8_t* is_diag,
                       double* m, double* v, double b1t, double b2t, double lr, double floor_, double* g_val) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double g = grad[e] * scale[e];
  const double me = b1 * m[e] + (1.0 - b1) * g;
  const double ve = b2 * v[e] + (1.0 - b2) * g * g;
  m[e] = me;
  v[e] = ve;
  double th = theta[e] - lr * (me / (1.0 - b1t)) / (sqrt(ve / (1.0 - b2t)) + eps);
  if (is_diag[e]) th = fmax(th, floor_);
  theta[e] = th;
  g_val[e] = th * scale[e];
}

// Training of the learned starting guess (three weights w, Adam) on the
// method's own solutions A (column t: a^c after t steps, n rows each):
// sample s (2 <= s < T-1) has history (A_s, A_{s-1}, A_{s-2}) and target
// A_{s+1}; E(w) = sum_s wt_s ||e_s||^2, e_s = sum_k w_k A_{s-k} - A_{s+1},
// wt_s = 1 / ||A_{s+1}||^2.  k_guess_grad: per block partials of E and of
// dE/dw_k = sum_s 2 wt_s (e_s . A_{s-k}) into part[(0..3) gridDim.x + b].
__global__ void __launch_bounds__(kThreads) k_guess_grad(int n, int T, const double* A, const double* wt,
                                                         const double* w, double* part) {
  __shared__ double red[kWarps];
  const double w0 = w[0], w1 = w[1], w2 = w[2];
  double l = 0.0, g[3] = {0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int s = 2; s < T - 1; ++s) {
      const double h0 = A[(size_t)s * n + i], h1 = A[(size_t)(s - 1) * n + i], h2 = A[(size_t)(s - 2) * n + i];
      const double e = fma(w0, h0, fma(w1, h1, w2 * h2)) - A[(size_t)(s + 1) * n + i];
      const double we = wt[s] * e;
      l = fma(we, e, l);
      g[0] = fma(2.0 * we, h0, g[0]);
      g[1] = fma(2.0 * we, h1, g[1]);
      g[2] = fma(2.0 * we, h2, g[2]);
    }
  }
  block_partial(l, part, 0, red);
  for (int k = 0; k < 3; ++k) block_partial(g[k], part, 1 + k, red);
}

// Squared norm of column s of A into part[s] (one block per column,
// fixed-order reduction).
__global__ void __launch_bounds__(kThreads) k_col_sqnorm(int n, const double* A, double* out) {
  __shared__ double red[kWarps];
  const double* x = A + (size_t)blockIdx.x * n;
  double l = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) l = fma(x[i], x[i], l);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kWarps; ++q) s += red[q];
    out[blockIdx.x] = s > 0.0 ? 1.0 / s : 0.0;
  }
}

// One Adam step on the three weights (state[0..2] w, [3..5] m, [6..8] v)
// from the summed block partials; loss_out (may be NULL) receives E.
__global__ void k_guess_adam(int nb, const double* part, double* state, double b1t, double b2t, double lr,
                             double* loss_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < 4; ++q)
    for (int b = 0; b < nb; ++b) sum[q] += part[(size_t)q * nb + b];
  if (loss_out) *loss_out = sum[0];
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int k = 0; k < 3; ++k) {
    const double g = sum[1 + k];
    const double m = b1 * state[3 + k] + (1.0 - b1) * g;
    const double v = b2 * state[6 + k] + (1.0 - b2) * g * g;
    state[3 + k] = m;
    state[6 + k] = v;
    state[k] -= lr * (m / (1.0 - b1t)) / (sqrt(v / (1.0 - b2t)) + eps);
  }
}

// Health check: per block max |x| over the entries whose class is nonzero
// (out[b]) and whether any of the n entries (class-masked) is non-finite
// (flag[b] = 1).  Grid-stride, kHealthBlocks blocks.
constexpr int kHealthBlocks = 1024;
__global__ void __launch_bounds__(kThreads) k_health(const double* x, int64_t n, const uint8_t* cls,
                                                     int64_t cs, double* out, int* flag, int accumulate) {
  __shared__ double smax[kThreads];
  __shared__ int sbad[kThreads];
  double m = 0.0;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (cls && cls[i % cs] == 0) continue;
    const double v = x[i];
    if (!isfinite(v)) bad = 1;
    else m = fmax(m, fabs(v));
  }
  smax[threadIdx.x] = m;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
      sbad[threadIdx.x] |= sbad[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[blockIdx.x] = accumulate ? fmax(out[blockIdx.x], smax[0]) : smax[0];
    flag[blockIdx.x] = accumulate ? (flag[blockIdx.x] | sbad[0]) : sbad[0];
  }
}

// gt_val[k] = g_val[gt_idx[k]] (G's values in transpose order).
__global__ void k_gt_vals(int64_t nnz, const double* g_val, const int* gt_idx, double* gt_val) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) gt_val[k] = g_val[gt_idx[k]];
}

// ---------------------------------------------------------------------------
// Cell-by-cell K (HetArgs): the explicit step for per-cell wave speed, and the
// adjoint.  off: grid offsets of the local nodes of a cell.

__device__ __forceinline__ int local_offset(const HetArgs& h, int m) {
  return (m % h.P) + h.nx * ((m / h.P) % h.P) + h.nx * h.ny * (m / (h.P * h.P));
}

// (K x)_i: the cells of node i in list order.
__device__ __forceinline__ double het_row(const HetArgs& h, const double* x, int64_t i) {
  double s = 0.0;
  for (int t = h.nc_ptr[i]; t < h.nc_ptr[i + 1]; ++t) {
    const int e = h.nc_cell[t], l = h.nc_local[t];
    const double* K = h.Kall + ((size_t)h.cell_koff[e] * h.Pd + l) * h.Pd;
    const double* xe = x + h.cell_base[e];
    double d0 = 0.0, d1 = 0.0;
    int m = 0;
    for (; m + 2 <= h.Pd; m += 2) {
      d0 = fma(K[m], xe[local_offset(h, m)], d0);
      d1 = fma(K[m + 1], xe[local_offset(h, m + 1)], d1);
    }
    if (m < h.Pd) d0 = fma(K[m], xe[local_offset(h, m)], d0);
    s = fma(h.cell_w[e], d0 + d1, s);
  }
  return s;
}

// A1 + A2 (+ A3) with cell-by-cell K (any dimension).
__global__ void __launch_bounds__(kThreads) k_explicit_het(ExplicitArgs a, HetArgs h) {
  const int64_t on = (int64_t)blockIdx.y * a.cs_node, oc = (int64_t)blockIdx.y * a.cs_c;
  const double* Uc = a.U + on;
  const double* Wc = a.W + on;
  double* OUTc = a.OUT + on;
  const double* fxc = a.fx + on;
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int nb = (int)((h.nnodes + kThreads - 1) / kThreads);
  if ((int)blockIdx.x >= nb) {
    const double c1 = a.dt, c2 = (0.5 - kNewmarkBeta) * a.dt * a.dt;
    const int stride = (gridDim.x - nb) * blockDim.x;
    for (int r = (blockIdx.x - nb) * blockDim.x + threadIdx.x; r < a.n_c; r += stride) {
      const int node = a.c_node[r];
      OUTc[node] = Uc[node] + c1 * a.v_c[oc + r] + c2 * a.a_c[oc + r];
    }
    return;
  }
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= h.nnodes || a.cls[g] != NODE_D) return;
  const int gx = (int)(g % a.nx), gy = (int)((g / a.nx) % a.ny), gz = (int)(g / ((int64_t)a.nx * a.ny));
  double minv = a.winv_x[gx] * a.winv_y[gy];
  if (h.dim == 3) minv *= a.winv_z[gz];
  const double ft = a.ft_dev ? a.ft_dev[0] : a.ft;
  const double r = het_row(h, Uc, g);
  const double acc = minv * (ft * fxc[g] - r);
  OUTc[g] = a.cu * Uc[g] + a.cw * Wc[g] + a.ca * acc;
}

// out = K x on every active node (0 elsewhere), per column (blockIdx.y).
__global__ void k_applyK(HetArgs h, const uint8_t* cls, const double* x, double* out, int64_t cs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= h.nnodes) return;
  const int64_t o = (int64_t)blockIdx.y * cs;
  out[o + i] = cls[i] ? het_row(h, x + o, i) : 0.0;
}

// grad[cell_id[e]] -= (2 / c_e) sum over columns of (hv_e . K_e un_e + gv_e . K_e un1_e)
// (dK/dc_e = 2 c_e K_e(1) = (2 / c_e) K_e, K_e = w_e times the stored matrix).
// One CTA per cell.  The cell matrix is staged in
// shared memory when it fits (kGradKSmem), the cell's values kGradCols
// columns at a time; threads take (column, row) items in a fixed assignment
// and the block sums in a fixed tree, so results are deterministic.
constexpr int kGradThreads = 128;
constexpr int kGradCols = 16;
constexpr int kGradKSmem = 4096;   // doubles of K_e staged (P^d <= 64)
__global__ void __launch_bounds__(kGradThreads) k_grad_cells(HetArgs h, int ncols, int64_t cs, const double* hv,
                                                             const double* un, const double* gv, const double* un1,
                                                             double* grad) {
  extern __shared__ double sgc[];
  const int e = blockIdx.x;
  const int tid = threadIdx.x, Pd = h.Pd;
  const bool kin = Pd * Pd <= kGradKSmem;
  double* Ks = sgc;                                   // Pd x Pd when it fits
  double* vh = sgc + (kin ? Pd * Pd : 0);             // kGradCols x Pd each
  double* vu = vh + kGradCols * Pd;
  double* vg = vu + kGradCols * Pd;
  double* vu1 = vg + kGradCols * Pd;
  double* red = vu1 + kGradCols * Pd;                 // kGradThreads
  const double* Kg = h.Kall + (size_t)h.cell_koff[e] * Pd * Pd;
  if (kin)
    for (int i = tid; i < Pd * Pd; i += kGradThreads) Ks[i] = Kg[i];
  const double* K = kin ? Ks : Kg;
  const int64_t base = h.cell_base[e];
  double part = 0.0;
  for (int c0 = 0; c0 < ncols; c0 += kGradCols) {
    const int ncl = min(kGradCols, ncols - c0);
    for (int i = tid; i < ncl * Pd; i += kGradThreads) {
      const int64_t b = (int64_t)(c0 + i / Pd) * cs + base + local_offset(h, i % Pd);
      vh[i] = hv[b];
      vu[i] = un[b];
      vg[i] = gv[b];
      vu1[i] = un1[b];
    }
    __syncthreads();
    for (int i = tid; i < ncl * Pd; i += kGradThreads) {
      const double hl = vh[i], gl = vg[i];
      if (hl == 0.0 && gl == 0.0) continue;
      const int l = i % Pd, o = i - l;
      double ku = 0.0, ku1 = 0.0;
      for (int m = 0; m < Pd; ++m) {
        const double k = K[l * Pd + m];
        ku = fma(k, vu[o + m], ku);
        ku1 = fma(k, vu1[o + m], ku1);
      }
      part = fma(hl, ku, fma(gl, ku1, part));
    }
    __syncthreads();
  }
  red[tid] = part;
  __syncthreads();
  for (int w = kGradThreads / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) grad[h.cell_id[e]] -= 2.0 / h.cell_c[e] * (h.cell_w[e] * red[0]);
}

size_t grad_cells_smem(int Pd) {
  return ((Pd * Pd <= kGradKSmem ? (size_t)Pd * Pd : 0) + 4 * (size_t)kGradCols * Pd + kGradThreads) *
         sizeof(double);
}

// Adjoint step, part 1 (c rows): rhs0 = abar + beta dt^2 ubar^c + gamma dt vbar;
// ucp = ubar^c, vcp = vbar.
__global__ void k_adj_pre(int n_c, int64_t cs_node, int64_t cs_c, const int* c_node, const double* ubar,
                          const double* vbar, const double* abar, double* rhs0, double* ucp, double* vcp,
                          double dt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  const int64_t oc = (int64_t)blockIdx.y * cs_c + r;
  const double ub = ubar[(int64_t)blockIdx.y * cs_node + c_node[r]];
  rhs0[oc] = abar[oc] + kNewmarkBeta * dt * dt * ub + kNewmarkGamma * dt * vbar[oc];
  ucp[oc] = ub;
  vcp[oc] = vbar[oc];
}

// z[c_node[r]] = v[r] per column (z zeroed beforehand).
__global__ void k_c_to_grid_set(int n_c, int64_t cs_node, int64_t cs_c, const int* c_node, const double* v,
                                double* z) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  z[(int64_t)blockIdx.y * cs_node + c_node[r]] = v[(int64_t)blockIdx.y * cs_c + r];
}

// Adjoint step, part 2 (all nodes): with wbar = -K[:, I_c] g (kg = K z1):
// I_d: T = ubar + wbar, h = dt^2 M^{-1} T (into z2), I_c: ucp += wbar.
__global__ void k_adj_mid(ExplicitArgs a, int64_t nnodes, const double* ubar, const double* kg, double* T,
                          double* z2, const int* node_c, double* ucp, double dt) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nnodes) return;
  const int64_t o = (int64_t)blockIdx.y * a.cs_node + g;
  z2[o] = 0.0;
  T[o] = 0.0;
  if (a.cls[g] == NODE_D) {
    const int gx = (int)(g % a.nx), gy = (int)((g / a.nx) % a.ny), gz = (int)(g / ((int64_t)a.nx * a.ny));
    double minv = a.winv_x[gx] * a.winv_y[gy];
    if (a.nz > 1) minv *= a.winv_z[gz];
    const double t = ubar[o] - kg[o];
    T[o] = t;
    z2[o] = dt * dt * minv * t;
  } else if (a.cls[g] == NODE_C) {
    ucp[(int64_t)blockIdx.y * a.cs_c + node_c[g]] -= kg[o];
  }
}

// Adjoint step, part 3: ubar_n = -K[:, I_d] h (kh = K z2) + 2 T + ubar_prev (I_d),
// + ucp (I_c); ubar_prev = -T (I_d); vbar, abar of step n (I_c).
__global__ void k_adj_post(ExplicitArgs a, int64_t nnodes, const double* kh, const double* T, double* ubar,
                           double* ubar_prev, const int* node_c, const double* ucp, const double* vcp, double* vbar,
                           double* abar, double dt) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nnodes) return;
  const int64_t o = (int64_t)blockIdx.y * a.cs_node + g;
  double ub = -kh[o];
  if (a.cls[g] == NODE_D) {
    ub += 2.0 * T[o] + ubar_prev[o];
    ubar_prev[o] = -T[o];
  } else if (a.cls[g] == NODE_C) {
    const int64_t r = (int64_t)blockIdx.y * a.cs_c + node_c[g];
    const double uc = ucp[r], vc = vcp[r];
    ub += uc;
    vbar[r] = dt * uc + vc;
    abar[r] = (0.5 - kNewmarkBeta) * dt * dt * uc + (1.0 - kNewmarkGamma) * dt * vc;
    ubar_prev[o] = 0.0;
  } else {
    ub = 0.0;
    ubar_prev[o] = 0.0;
  }
  ubar[o] = ub;
}

// Misfit at the receivers: ubar[rec] += u[rec] - d (per column), and the
// per-column partial 1/2 sum (u[rec] - d)^2 into jpart[col].
__global__ void k_misfit(int nrec, int64_t cs_node, const int64_t* rec, const double* u, const double* data,
                         double* ubar, double* jpart, int add_adjoint) {
  // one block per column, data: (ncols x nrec) for this step
  __shared__ double red[kWarps];
  const int col = blockIdx.x;
  double j = 0.0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    const int64_t o = (int64_t)col * cs_node + rec[k];
    const double e = u[o] - data[(int64_t)col * nrec + k];
    j = fma(0.5 * e, e, j);
    if (add_adjoint) ubar[o] += e;
  }
  for (int o = 16; o > 0; o >>= 1) j += __shfl_xor_sync(0xffffffffu, j, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = j;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    jpart[col] += t;
  }
}

// ---------------------------------------------------------------------------
// Small field kernels (layout conversion only).
__global__ void k_gather_c(double* dst, const double* src, const int* c_node, int n_c) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_c) dst[r] = src[c_node[r]];
}
// Central-difference start on I_c (column blockIdx.y):
// u^c_{-1} = u^c_0 - dt v^c_0 + dt^2/2 a^c_0 into Uo.
__global__ void k_cdm_start_c(double* Uo, const double* U0, const double* v_c, const double* a_c,
                              const int* c_node, int n_c, int64_t cs_node, double dt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_c) return;
  const int64_t on = (int64_t)blockIdx.y * cs_node, oc = (int64_t)blockIdx.y * n_c;
  const int node = c_node[r];
  Uo[on + node] = U0[on + node] - dt * v_c[oc + r] + 0.5 * dt * dt * a_c[oc + r];
}
__global__ void k_scatter_c(double* dst, const double* src, const int* c_node, int n_c) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_c) dst[c_node[r]] = src[r];
}
// dst[g] = (mask(cls[g])) ? src[g] : 0 ; want: 1 -> I_d, 2 -> I_c, 3 -> active, 4 -> 1.0 on I_d, 5 -> 1.0 on I_c
__global__ void k_masked(double* dst, const double* src, const uint8_t* cls, int64_t n, int want) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int c = cls[g];
  double v = 0.0;
  if (want == 1) v = (c == NODE_D) ? src[g] : 0.0;
  else if (want == 2) v = (c == NODE_C) ? src[g] : 0.0;
  else if (want == 3) v = (c != NODE_INACTIVE) ? src[g] : 0.0;
  else if (want == 4) v = (c == NODE_D) ? 1.0 : 0.0;
  else if (want == 5) v = (c == NODE_C) ? 1.0 : 0.0;
  dst[g] = v;
}
// dst[g] = src[g] where cls[g] == want (other entries kept).
__global__ void k_masked_set(double* dst, const double* src, const uint8_t* cls, int64_t n, int want) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < n && cls[g] == want) dst[g] = src[g];
}

// Receiver samples: out[k] = u[nodes[k]].
__global__ void k_gather_nodes(double* out, const double* u, const int64_t* nodes, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = u[nodes[k]];
}

// Explicit-apply variants, the candidates of the setup autotuner (the
// environment variable IMEX_EXPLICIT_TILE = large | small | sweep fixes one):
//   0 tiles of kTileLarge[P] cells per side (less halo work),
//   1 tiles of kTileSmall[P] (finer load balance on small grids),
//   2 (2D) the persistent strip sweep, strips of kSweepCells[P] cells and
//     chunks of as many cell rows, up to kSweepMinBlocks[0][P] CTAs per SM.
constexpr int kTileLarge[10] = {0, 0, 16, 16, 10, 8, 6, 5, 4, 4};
constexpr int kTileSmall[10] = {0, 0, 8, 8, 5, 4, 3, 3, 2, 2};
constexpr int kSweepCells[10] = {0, 0, 32, 16, 10, 8, 6, 5, 4, 4};
//   3 (2D) the same strips in chunks of half as many cell rows, with more
//     resident CTAs per SM (kSweepMinBlocks[1][P]).
constexpr int kSweepMinBlocks[2][10] = {{0, 0, 3, 3, 3, 3, 2, 2, 2, 1}, {0, 0, 4, 4, 4, 4, 3, 3, 3, 2}};
constexpr int kExplicitSweep = 2, kExplicitSweepShort = 3;
// Explicit candidates of the autotuner: the kernel form (tiles, strip sweep)
// and, for tiles, the split launch: the tiles whose nodes the implicit solve
// reads (with the prediction), then the solve, while the other tiles run on
// a second stream with a fixed number of CTAs per SM.  Split candidate s
// (variant 4 + s) uses tile form kSplitTile[s] with kSplitPerSM[s] CTAs.
constexpr int kExplicitSplit = 4, kSplitVariants = 4;
constexpr int kSplitTile[kSplitVariants] = {0, 0, 1, 1};
constexpr int kSplitPerSM[kSplitVariants] = {1, 2, 2, 4};
const char* const kExplicitNames[8] = {"large",        "small",        "sweep",        "sweep_short",
                                       "large_split1", "large_split2", "small_split2", "small_split4"};
template <int P>
constexpr int sweep_chunk(int short_chunks) { return short_chunks ? (kSweepCells[P] + 1) / 2 : kSweepCells[P]; }
// 3D (P <= 5): tiles of TC^3 cells.
constexpr int kTileLarge3[6] = {0, 0, 8, 4, 3, 3};
constexpr int kTileSmall3[6] = {0, 0, 4, 2, 2, 2};

size_t explicit_smem_doubles3(int P, int TC) {
  const size_t p = P - 1, OX = TC * p, R = (TC + 1) * p + 1, NC = TC + 1;
  return R * R * R + 2 * R * R * OX + std::max(4 * R * R * NC, 2 * R * OX * OX + 4 * R * NC * OX);
}

size_t explicit_smem_doubles(int P, int TC) {
  const int p = P - 1, OX = TC * p, OY = OX, RX = (TC + 1) * p + 1, RY = RX, NC = TC + 1;
  size_t scr = std::max<size_t>((size_t)4 * RY * NC, (size_t)OY * OX + 2 * (size_t)NC * OX);
  return (size_t)RY * RX + 2 * (size_t)RY * OX + scr;
}

}  // namespace

// ---------------------------------------------------------------------------
// Context.
struct imex_ctx {
  HostSetup hs;
  imex_alloc hooks{};
  bool has_hooks = false;
  char* base = nullptr;
  size_t bytes = 0;
  int device = 0;
  // full-grid fields
  double *U[2] = {nullptr, nullptr};
  double* tmp = nullptr;    // full grid scratch (initial velocity, exports)
  double* fx = nullptr;
  double* fxs = nullptr;    // 2D: dt^2 M^{-1} f_x (the explicit kernels' source term)
  double *winv_x = nullptr, *winv_y = nullptr, *winv_z = nullptr;
  uint8_t* cls = nullptr;
  // implicit partition
  int* c_node = nullptr;
  double *v_c = nullptr, *a_c = nullptr, *fxc = nullptr;
  // right-hand sides: rows of the interface cell matrices, per-cell scales
  double *Kpair = nullptr, *rhs0 = nullptr;
  int64_t *kp_off = nullptr, *kp_len = nullptr;
  int64_t walk_max_kp = 0;
  int walk_kp_smem = 1;   // cell-matrix rows of the pairs staged in shared memory
  // solve: per-CTA factor blobs (S and M^cc) and index lists, dense tops, scratch
  double *blob_S = nullptr, *blob_M = nullptr;
  int64_t *blob_off = nullptr, *blob_len = nullptr;
  int* ilist = nullptr;
  int64_t *ilist_off = nullptr, *ilist_len = nullptr;
  int64_t walk_max_blob = 0;
  int walk_max_slots = 2, walk_max_m = 2, walk_max_pairs = 2;
  int* tlist = nullptr;
  int64_t *tlist_off = nullptr, *tlist_len = nullptr;
  int top_max_zn = 2;
  int64_t top_max_arows = 0;
  std::vector<int> lev_cta0, lev_ncta, lev_has_nodes;   // per walked level: CTA range
  int walk_smem_mode = 0;
  size_t smem_walk = 0, smem_top = 0;
  // Dynamic shared memory requested per walk launch (>= smem_walk).  A
  // larger request changes which CTAs of the neighbouring launches share an
  // SM with a walk CTA; the setup autotuner times a few requests.
  size_t smem_walk_req = 0;
  // Independent columns per walk / dense-top CTA (autotuned for ncols > 1):
  // the factor blocks are staged once per block of columns.  Shared memory
  // of a walk CTA = blob + cell-matrix rows + cb x walk_vec doubles +
  // walk_ilist ints; of a dense-top CTA = max_arows + cb x (max_zn +
  // kThreads) doubles + top_ilist ints.
  int col_block = 1;
  size_t walk_fixed = 0, walk_vec = 0, top_fixed = 0, top_vec = 0;
  float cb_us[7] = {};   // setup timing with 1, 2, 4, ..., 64 columns per CTA (0: not timed)
  int ntop = 0;
  int *top_comp = nullptr, *top_r0 = nullptr, *top_r1 = nullptr;
  int *zsize = nullptr, *zbase = nullptr, *zrow = nullptr;
  int64_t* zA_off = nullptr;
  double *zA_S = nullptr, *zA_M = nullptr;
  int64_t nzrow = 0;
  double *upd = nullptr, *sol = nullptr;
  // large supernodes of the walked levels (k_panel)
  int *pan_desc = nullptr, *pan_idx = nullptr;
  int64_t* pan_aoff = nullptr;
  double *panS = nullptr, *panM = nullptr, *hbuf = nullptr;
  std::vector<int> pan_cta0, pan_ncta;   // [4 level + phase]
  int64_t pan_max_chunk = 2;
  int pan_max_nv = 2;
  size_t smem_panel = 0;
  int64_t n_large = 0;   // supernodes walked by k_panel
  // host I/O (imex_step_io): rings of kIoRing slots for the source samples
  // (2 doubles each) and the receiver values (io_cap * ncols each), filled and
  // drained on two copy streams, with events guarding slot reuse
  double *ft_buf = nullptr, *rec_buf = nullptr;
  int64_t* rec_nodes = nullptr;
  int io_cap = 4096;
  cudaStream_t io_h2d = nullptr, io_d2h = nullptr;
  cudaEvent_t io_ev[3][kIoRing] = {};   // [h2d done | step and gather done | d2h done][slot]
  // state
  int ncols = 1;            // independent source columns (fields column after column)
  // cell-by-cell K (per-cell wave speed; the adjoint)
  int hetero = 0;
  int het_ncell = 0;
  int *het_base = nullptr, *het_koff = nullptr, *het_id = nullptr, *het_ptr = nullptr, *het_cell = nullptr,
      *het_local = nullptr, *node_c_dev = nullptr;
  double *het_w = nullptr, *het_c = nullptr, *Kall = nullptr;
  // iterative solve (PCG) and its learned preconditioner
  int solver = IMEX_SOLVER_DIRECT;
  double pcg_tol = 1e-10;
  int pcg_maxit = 200;
  int pcg_grid = 0;
  int pcg_lpr = 32;   // lanes per sparse row of the PCG products (from the mean row length of S)
  int64_t g_nnz = 0;
  int *s_ptr = nullptr, *s_col = nullptr;
  double* s_val = nullptr;
  int *g_ptr = nullptr, *g_col = nullptr, *gt_ptr = nullptr, *gt_row = nullptr, *gt_idx = nullptr;
  double *g_val = nullptr, *g_scale = nullptr, *g_theta = nullptr, *g_m = nullptr, *g_v = nullptr;
  double *g_grad = nullptr, *g_sg = nullptr, *dinv = nullptr;
  uint8_t* g_isdiag = nullptr;
  double* gt_val = nullptr;   // G's values in transpose order
  // no factorisation (imex_setup_pcg): M^cc on S's pattern for the initial
  // acceleration, and the (row, interface cell) pairs of K^c u per row
  int factorized = 1;
  double *m_val = nullptr, *dinv_m = nullptr, *if_sc_dev = nullptr;
  int *pr_ptr = nullptr, *pr_pos = nullptr, *if_base_dev = nullptr, *if_koff_dev = nullptr;
  double *pcg_x = nullptr, *pcg_r = nullptr, *pcg_z = nullptr, *pcg_p = nullptr, *pcg_q = nullptr, *pcg_w = nullptr,
         *pcg_v = nullptr;
  double *pcg_part = nullptr, *pcg_res = nullptr;
  // learned starting guess of the PCG solves: history a^c_{n-1}, a^c_{n-2}
  // (pcg_hist, 2 n_c) and the Adam state of the three weights (guess_state:
  // w, m, v); used once two PCG solves have filled the history
  double *pcg_hist = nullptr, *guess_state = nullptr;
  int guess_on = 0;
  int64_t guess_valid = 0, guess_t = 0;
  int* pcg_status = nullptr;
  long long* pcg_counters = nullptr;
  int64_t adam_t = 0;
  int cur = 0;              // U[cur] holds u_n
  int64_t step = 0;
  cudaStream_t stream = nullptr;
  Ops2D ops{};
  int TC = 4, ntx = 1, nty = 1, ntz = 1;
  Ops3D ops3{};
  int xvar = 0;                   // explicit kernel form: 0 large tile, 1 small tile, 2/3 sweep (autotuned)
  int xsplit = 0;                 // split launch in use (variant 4 + split candidate; autotuned)
  int split_per_sm = 1;           // CTAs per SM of the split launch's second half
  float tile_us[8] = {};          // measured time of each candidate (0: not timed)
  // Split explicit launch (2D tiles): per tile size, the tiles owning an I_d
  // node of an interface cell (read by the implicit solve) and the others,
  // which run on the stream `side` beside the solve.
  int split_ok = 0;
  int *tile_near[2] = {nullptr, nullptr}, *tile_far[2] = {nullptr, nullptr};
  int n_near[2] = {0, 0}, n_far[2] = {0, 0};
  cudaStream_t side = nullptr;
  cudaEvent_t ov_fork = nullptr, ov_join = nullptr;
  int explicit_per_sm = 1;    // resident CTAs of the explicit kernel per SM
  int num_sms = 152;
  size_t smem_explicit = 0;
};

namespace {

struct Arena {
  std::vector<std::pair<void**, size_t>> items;
  template <class T>
  void add(T** p, size_t n) { items.emplace_back((void**)p, ((n * sizeof(T) + 255) / 256) * 256 + 256); }
  size_t total() const { size_t s = 0; for (auto& i : items) s += i.second; return s; }
  void assign(char* base) {
    size_t off = 0;
    for (auto& i : items) { *i.first = base + off; off += i.second; }
  }
};

template <class T>
cudaError_t upload(T* dst, const std::vector<T>& src) {
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return IMEX_OK;
}

template <int P>
void launch_explicit(imex_ctx* c, const ExplicitArgs& ea, int grid, cudaStream_t s) {
  const dim3 g(grid, ea.persistent ? 1 : c->ncols);   // a persistent launch loops over the columns
  if (c->xvar == kExplicitSweep)
    k_sweep2d<P, kSweepCells[P], sweep_chunk<P>(0), kSweepMinBlocks[0][P]>
        <<<g, kThreads, c->smem_explicit, s>>>(ea, c->ops);
  else if (c->xvar == kExplicitSweepShort)
    k_sweep2d<P, kSweepCells[P], sweep_chunk<P>(1), kSweepMinBlocks[1][P]>
        <<<g, kThreads, c->smem_explicit, s>>>(ea, c->ops);
  else if (c->xvar == 1)
    k_explicit2d<P, kTileSmall[P]><<<g, kThreads, c->smem_explicit, s>>>(ea, c->ops);
  else
    k_explicit2d<P, kTileLarge[P]><<<g, kThreads, c->smem_explicit, s>>>(ea, c->ops);
}

template <int P>
void launch_explicit3(imex_ctx* c, const ExplicitArgs& ea, int grid, cudaStream_t s) {
  if (c->xvar == 1)
    k_explicit3d<P, kTileSmall3[P]><<<dim3(grid, c->ncols), kThreads, c->smem_explicit, s>>>(ea, c->ops3);
  else
    k_explicit3d<P, kTileLarge3[P]><<<dim3(grid, c->ncols), kThreads, c->smem_explicit, s>>>(ea, c->ops3);
}

int ntiles(const imex_ctx* c) { return c->ntx * c->nty * c->ntz; }

HetArgs het_args(const imex_ctx* c) {
  const HostSetup& hs = c->hs;
  HetArgs h{};
  h.ncell = c->het_ncell;
  h.cell_base = c->het_base;
  h.cell_koff = c->het_koff;
  h.cell_w = c->het_w;
  h.cell_c = c->het_c;
  h.cell_id = c->het_id;
  h.Kall = c->Kall;
  h.nc_ptr = c->het_ptr;
  h.nc_cell = c->het_cell;
  h.nc_local = c->het_local;
  h.P = hs.P;
  h.Pd = hs.Pd;
  h.dim = hs.dim;
  h.nx = hs.nn[0];
  h.ny = hs.nn[1];
  h.nnodes = hs.nnodes;
  return h;
}

void explicit_dispatch(imex_ctx* c, const ExplicitArgs& ea, int grid, cudaStream_t s) {
  if (c->hetero) {   // grid = tiles + prediction blocks; the cell-by-cell kernel takes nodes instead of tiles
    const int nb = (int)((c->hs.nnodes + kThreads - 1) / kThreads);
    k_explicit_het<<<dim3(nb + (grid - ntiles(c)), c->ncols), kThreads, 0, s>>>(ea, het_args(c));
    return;
  }
  if (c->hs.dim == 3) {
    switch (c->hs.P) {
      case 2: launch_explicit3<2>(c, ea, grid, s); break;
      case 3: launch_explicit3<3>(c, ea, grid, s); break;
      case 4: launch_explicit3<4>(c, ea, grid, s); break;
      case 5: launch_explicit3<5>(c, ea, grid, s); break;
    }
    return;
  }
  switch (c->hs.P) {
    case 2: launch_explicit<2>(c, ea, grid, s); break;
    case 3: launch_explicit<3>(c, ea, grid, s); break;
    case 4: launch_explicit<4>(c, ea, grid, s); break;
    case 5: launch_explicit<5>(c, ea, grid, s); break;
    case 6: launch_explicit<6>(c, ea, grid, s); break;
    case 7: launch_explicit<7>(c, ea, grid, s); break;
    case 8: launch_explicit<8>(c, ea, grid, s); break;
    case 9: launch_explicit<9>(c, ea, grid, s); break;
  }
}

// Shared-memory attribute and resident CTAs per SM of the explicit kernel.
template <int P>
cudaError_t explicit_config(int var, size_t bytes, int* per_sm) {
  auto fn = var == kExplicitSweep      ? k_sweep2d<P, kSweepCells[P], sweep_chunk<P>(0), kSweepMinBlocks[0][P]>
            : var == kExplicitSweepShort ? k_sweep2d<P, kSweepCells[P], sweep_chunk<P>(1), kSweepMinBlocks[1][P]>
            : var == 1                   ? k_explicit2d<P, kTileSmall[P]>
                                         : k_explicit2d<P, kTileLarge[P]>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e ? e : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, kThreads, bytes);
}

template <int P>
cudaError_t explicit_config3(int var, size_t bytes, int* per_sm) {
  auto fn = var == 1 ? k_explicit3d<P, kTileSmall3[P]> : k_explicit3d<P, kTileLarge3[P]>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e ? e : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, kThreads, bytes);
}

cudaError_t explicit_config_dispatch(int dim, int P, int small, size_t bytes, int* per_sm) {
  if (dim == 3) {
    switch (P) {
      case 2: return explicit_config3<2>(small, bytes, per_sm);
      case 3: return explicit_config3<3>(small, bytes, per_sm);
      case 4: return explicit_config3<4>(small, bytes, per_sm);
      case 5: return explicit_config3<5>(small, bytes, per_sm);
    }
    return cudaErrorInvalidValue;
  }
  switch (P) {
    case 2: return explicit_config<2>(small, bytes, per_sm);
    case 3: return explicit_config<3>(small, bytes, per_sm);
    case 4: return explicit_config<4>(small, bytes, per_sm);
    case 5: return explicit_config<5>(small, bytes, per_sm);
    case 6: return explicit_config<6>(small, bytes, per_sm);
    case 7: return explicit_config<7>(small, bytes, per_sm);
    case 8: return explicit_config<8>(small, bytes, per_sm);
    case 9: return explicit_config<9>(small, bytes, per_sm);
  }
  return cudaErrorInvalidValue;
}

// Shared memory (doubles) of the sweep kernel of order P (SweepShape).
size_t sweep_smem_doubles(int P, int short_chunks) {
  switch (P) {
#define IMEX_SWEEP_SHAPE(PP)                                                                           \
  case PP:                                                                                             \
    return short_chunks ? SweepShape<PP, kSweepCells[PP], sweep_chunk<PP>(1)>::DOUBLES                 \
                        : SweepShape<PP, kSweepCells[PP], sweep_chunk<PP>(0)>::DOUBLES;
    IMEX_SWEEP_SHAPE(2) IMEX_SWEEP_SHAPE(3) IMEX_SWEEP_SHAPE(4) IMEX_SWEEP_SHAPE(5)
    IMEX_SWEEP_SHAPE(6) IMEX_SWEEP_SHAPE(7) IMEX_SWEEP_SHAPE(8) IMEX_SWEEP_SHAPE(9)
#undef IMEX_SWEEP_SHAPE
  }
  return 0;
}

// Number of explicit variants of a context: tiles (large, small) and, in 2D,
// the sweep.
int explicit_variants(const imex_ctx* c) {
  return c->hs.dim == 3 ? 2 : (c->split_ok ? kExplicitSplit + kSplitVariants : 4);
}

// Select an explicit variant: tile counts (for the sweep: ntx = its CTAs),
// shared memory and occupancy follow it.
cudaError_t use_explicit(imex_ctx* c, int var) {
  const HostSetup& hs = c->hs;
  const bool d3 = hs.dim == 3;
  if (var < 0 || var >= explicit_variants(c)) var = 0;
  c->xsplit = var >= kExplicitSplit ? 1 : 0;
  if (c->xsplit) {
    c->split_per_sm = kSplitPerSM[var - kExplicitSplit];
    var = kSplitTile[var - kExplicitSplit];
  }
  c->xvar = var;
  if (var == kExplicitSweep || var == kExplicitSweepShort) {
    c->TC = kSweepCells[hs.P];
    c->nty = c->ntz = 1;
    c->smem_explicit = sweep_smem_doubles(hs.P, var == kExplicitSweepShort) * sizeof(double);
    int per_sm = 0;
    cudaError_t e = explicit_config_dispatch(hs.dim, hs.P, var, c->smem_explicit, &per_sm);
    c->explicit_per_sm = std::max(1, per_sm);
    // As many sweep CTAs as are resident at once (up to three per SM), never
    // more than work units; IMEX_SWEEP_CTAS = n fixes the number (tests:
    // segments that cross strip boundaries on small grids).
    const int64_t units = (int64_t)((hs.pb.ncells[0] + c->TC - 1) / c->TC) * hs.pb.ncells[1];
    int64_t n = std::min<int64_t>(units, (int64_t)std::max(1, c->num_sms) *
                                             std::min(kSweepMinBlocks[var - kExplicitSweep][hs.P], c->explicit_per_sm));
    if (const char* env = std::getenv("IMEX_SWEEP_CTAS")) n = std::min<int64_t>(units, std::atoll(env));
    c->ntx = (int)std::max<int64_t>(1, n);
    return e;
  } else {
    const bool small = var == 1;
    c->TC = d3 ? (small ? kTileSmall3[hs.P] : kTileLarge3[hs.P]) : (small ? kTileSmall[hs.P] : kTileLarge[hs.P]);
    const int OX = c->TC * hs.p;
    c->ntx = (hs.nn[0] + OX - 1) / OX;
    c->nty = (hs.nn[1] + OX - 1) / OX;
    c->ntz = d3 ? (hs.nn[2] + OX - 1) / OX : 1;
    c->smem_explicit =
        (d3 ? explicit_smem_doubles3(hs.P, c->TC) : explicit_smem_doubles(hs.P, c->TC)) * sizeof(double);
  }
  int per_sm = 0;
  cudaError_t e = explicit_config_dispatch(hs.dim, hs.P, var, c->smem_explicit, &per_sm);
  c->explicit_per_sm = std::max(1, per_sm);
  return e;
}

// Index of the variant named by IMEX_EXPLICIT_TILE, or -1.
int explicit_env_variant(const imex_ctx* c) {
  const char* env = std::getenv("IMEX_EXPLICIT_TILE");
  if (!env) return -1;
  for (int k = 0; k < explicit_variants(c); ++k)
    if (std::string(env) == kExplicitNames[k]) return k;
  return -1;
}

ExplicitArgs explicit_args(imex_ctx* c, const double* U, const double* W, double* OUT, double cu, double cw,
                           double ca, double ft, bool predict) {
  const HostSetup& hs = c->hs;
  ExplicitArgs ea{};
  ea.U = U;
  ea.W = W;
  ea.OUT = OUT;
  ea.cls = c->cls;
  ea.fx = c->fx;
  ea.fxs = c->fxs;
  ea.kappa2 = ca / (hs.dt * hs.dt);
  ea.winv_x = c->winv_x;
  ea.winv_y = c->winv_y;
  ea.winv_z = c->winv_z;
  ea.nx = hs.nn[0];
  ea.ny = hs.nn[1];
  ea.nz = hs.dim == 3 ? hs.nn[2] : 1;
  ea.ncx = hs.pb.ncells[0];
  ea.ncy = hs.pb.ncells[1];
  ea.ncz = hs.dim == 3 ? hs.pb.ncells[2] : 1;
  ea.ntx = c->ntx;
  ea.nty = c->nty;
  ea.ntz = c->ntz;
  ea.cu = cu;
  ea.cw = cw;
  ea.ca = ca;
  ea.ft = ft;
  ea.n_c = predict ? (int)hs.n_c : 0;
  ea.c_node = c->c_node;
  ea.v_c = c->v_c;
  ea.a_c = c->a_c;
  ea.dt = hs.dt;
  ea.cs_node = hs.nnodes;
  ea.cs_c = hs.n_c;
  ea.ncols = c->ncols;
  return ea;
}

// CTAs for the Newmark prediction, appended to the tiles of the explicit
// launch.  The tiles are FP64-bound and the block scheduler hands CTAs to the
// SMs in turn, so the launch is sized to ceil(tiles / SMs) CTAs per SM: the
// prediction fills the last round instead of adding a further CTA to some
// SMs.  At least one, at most one per 256 rows.
int pred_blocks(imex_ctx* c, bool predict) {
  if (!predict || c->hs.n_c == 0) return 0;
  if (c->xvar >= kExplicitSweep) return 0;   // the sweep CTAs predict their share themselves
  const int64_t tiles = (int64_t)ntiles(c);
  const int64_t nsm = std::max(1, c->num_sms);
  const int64_t per_sm = std::min<int64_t>((tiles + nsm - 1) / nsm, std::max(1, c->explicit_per_sm));
  int64_t spare = (per_sm * nsm - tiles % (per_sm * nsm)) % (per_sm * nsm);
  if (spare == 0) spare = 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>(spare, (c->hs.n_c + kThreads - 1) / kThreads));
}

constexpr int kMaxWidth = 256;                 // largest supernode / row set one walk CTA takes
constexpr int64_t kPanelChunk = 12288;         // doubles of a k_panel chunk (96 KB of shared memory)
constexpr size_t kWalkSmemBudget = 200 * 1024;  // shared memory per walk CTA (staged factor)
constexpr size_t kTopSmemBudget = 200 * 1024;   // shared memory per dense-top CTA
constexpr size_t kMaxDynSmem = 220 * 1024;      // dynamic shared memory limit we set (static use < 7 KB)

// The walk kernel for a direction, staging mode and column mode (one column
// per CTA, or a block of columns).
using WalkFn = void (*)(WalkArgs);
WalkFn walk_kernel(bool fwd, bool smem, bool cols) {
  if (fwd) {
    if (smem) return cols ? k_walk<true, true, true> : k_walk<true, true, false>;
    return cols ? k_walk<true, false, true> : k_walk<true, false, false>;
  }
  if (smem) return cols ? k_walk<false, true, true> : k_walk<false, true, false>;
  return cols ? k_walk<false, false, true> : k_walk<false, false, false>;
}

// The launches of the implicit solve: forward walk over the lower levels
// (the first also forms every right-hand side from src), dense tops,
// backward walk with the correction.  use_S selects the factor of S (step)
// or of M^cc (initial acceleration, mode 1).  upd/sol/rhs0 are the solve's
// scratch vectors.
cudaError_t launch_solve_chain(imex_ctx* c, bool use_S, double ft, const double* ft_dev, int mode, double* Ubuf,
                               const double* src, double* upd, double* sol, double* rhs0, double* hbuf,
                               cudaStream_t s, const int* skip = nullptr, bool rhs_only = false,
                               bool rhs_given = false) {
  const HostSetup& hs = c->hs;
  WalkArgs w{};
  w.blob = use_S ? c->blob_S : c->blob_M;
  w.blob_off = c->blob_off;
  w.blob_len = c->blob_len;
  w.max_blob = c->walk_max_blob;
  w.ilist = c->ilist;
  w.ilist_off = c->ilist_off;
  w.ilist_len = c->ilist_len;
  w.max_slots = c->walk_max_slots;
  w.max_m = c->walk_max_m;
  w.max_pairs = c->walk_max_pairs;
  w.SRC = src;
  w.Kpair = c->Kpair;
  w.kp_off = c->kp_off;
  w.kp_len = c->kp_len;
  w.max_kp = c->walk_max_kp;
  w.kp_smem = c->walk_kp_smem;
  w.P = hs.P;
  w.Pd = hs.Pd;
  w.dim = hs.dim;
  w.nx = hs.nn[0];
  w.ny = hs.nn[1];
  w.fxc = c->fxc;
  w.ft = ft;
  w.ft_dev = ft_dev;
  w.rhs0 = rhs0;
  w.upd = upd;
  w.sol = sol;
  w.mode = mode;
  w.c_node = c->c_node;
  w.U = Ubuf;
  w.v_c = c->v_c;
  w.a_c = c->a_c;
  w.dt = hs.dt;
  w.skip = skip;
  w.rhs_given = rhs_given ? 1 : 0;
  w.cs_node = hs.nnodes;
  w.cs_c = hs.n_c;
  w.cs_upd = std::max<int64_t>(hs.upd_size, 1);
  w.cb = c->col_block;
  w.ncols = c->ncols;
  TopArgs z{};
  z.cta_comp = c->top_comp;
  z.cta_r0 = c->top_r0;
  z.cta_r1 = c->top_r1;
  z.zsize = c->zsize;
  z.zbase = c->zbase;
  z.zrow = c->zrow;
  z.zA_off = c->zA_off;
  z.zA = use_S ? c->zA_S : c->zA_M;
  z.max_zn = c->top_max_zn;
  z.max_arows = c->top_max_arows;
  z.ilist = c->tlist;
  z.ilist_off = c->tlist_off;
  z.ilist_len = c->tlist_len;
  z.rhs0 = rhs0;
  z.upd = upd;
  z.sol = sol;
  z.mode = mode;
  z.c_node = c->c_node;
  z.U = Ubuf;
  z.Un = src;
  z.v_c = c->v_c;
  z.a_c = c->a_c;
  z.dt = hs.dt;
  z.skip = skip;
  z.cs_node = w.cs_node;
  z.cs_c = w.cs_c;
  z.cs_upd = w.cs_upd;
  z.cb = w.cb;
  z.ncols = w.ncols;

  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int nlev = (int)c->lev_cta0.size();
  auto walk = [&](int l, bool fwd) {
    w.cta0 = c->lev_cta0[l];
    w.first = (fwd && l == 0) ? 1 : 0;
    cfg.gridDim = dim3(c->lev_ncta[l], (c->ncols + c->col_block - 1) / c->col_block);
    cfg.dynamicSmemBytes = c->smem_walk_req;
    return cudaLaunchKernelEx(&cfg, walk_kernel(fwd, c->walk_smem_mode != 0, c->col_block > 1), w);
  };
  PanelArgs pa{};
  pa.desc = c->pan_desc;
  pa.a_off = c->pan_aoff;
  pa.A = use_S ? c->panS : c->panM;
  pa.idx = c->pan_idx;
  pa.max_chunk = c->pan_max_chunk;
  pa.max_nv = c->pan_max_nv;
  pa.skip = skip;
  pa.rhs0 = rhs0;
  pa.upd = upd;
  pa.sol = sol;
  pa.hbuf = hbuf;
  pa.mode = mode;
  pa.c_node = c->c_node;
  pa.U = Ubuf;
  pa.Un = src;
  pa.v_c = c->v_c;
  pa.a_c = c->a_c;
  pa.dt = hs.dt;
  pa.cs_node = w.cs_node;
  pa.cs_c = w.cs_c;
  pa.cs_upd = w.cs_upd;
  auto panel = [&](int l, int phase) {
    const int n = c->pan_ncta.empty() ? 0 : c->pan_ncta[4 * l + phase];
    if (n == 0) return cudaSuccess;
    pa.cta0 = c->pan_cta0[4 * l + phase];
    cfg.gridDim = dim3(n, c->ncols);
    cfg.dynamicSmemBytes = c->smem_panel;
    return cudaLaunchKernelEx(&cfg, k_panel, pa);
  };
  cudaError_t e = cudaSuccess;
  if (rhs_only) {   // the first forward launch forms every right-hand side into rhs0, nothing else
    w.rhs_only = 1;
    return walk(0, true);
  }
  // Per walked level: the walk of its small supernodes, then the two
  // forward phases of its large ones (k_panel); backwards in reverse.
  for (int l = 0; l < nlev && e == cudaSuccess; ++l) {
    if (l == 0 || c->lev_ncta[l] > 0) e = walk(l, true);
    for (int ph = 0; ph < 2 && e == cudaSuccess; ++ph) e = panel(l, ph);
  }
  if (e == cudaSuccess && c->ntop > 0) {
    cfg.gridDim = dim3(c->ntop, (c->ncols + c->col_block - 1) / c->col_block);
    cfg.dynamicSmemBytes = c->smem_top;
    e = cudaLaunchKernelEx(&cfg, c->col_block > 1 ? k_top<true> : k_top<false>, z);
  }
  for (int l = nlev - 1; l >= 0 && e == cudaSuccess; --l) {
    for (int ph = 2; ph < 4 && e == cudaSuccess; ++ph) e = panel(l, ph);
    if (e == cudaSuccess && c->lev_has_nodes[l]) e = walk(l, false);
  }
  return e;
}

// Columns per walk and dense-top CTA; false (nothing changed) if the
// shared memory would exceed a CTA's limit.
bool set_col_block(imex_ctx* c, int cb) {
  cb = std::max(1, std::min(cb, c->ncols));
  const size_t w = c->walk_fixed + (size_t)cb * c->walk_vec, tp = c->top_fixed + (size_t)cb * c->top_vec;
  if (w > kMaxDynSmem || tp > kMaxDynSmem) return false;
  c->col_block = cb;
  c->smem_walk = w;
  c->smem_walk_req = w;
  c->smem_top = tp;
  return true;
}

// IMEX_COL_BLOCK = n pins the columns per walk / dense-top CTA (else tuned).
int col_block_env() {
  const char* env = std::getenv("IMEX_COL_BLOCK");
  return env ? std::max(1, std::atoi(env)) : 0;
}

// The split candidate in use (index into kSplitTile / kSplitPerSM).
int split_index(const imex_ctx* c) {
  for (int s = 0; s < kSplitVariants; ++s)
    if (kSplitTile[s] == c->xvar && kSplitPerSM[s] == c->split_per_sm) return s;
  return 0;
}

// The split explicit launch is in use (see step_once): direct solve by the
// launch chain, whose launches are not cooperative.
bool split_active(const imex_ctx* c) {
  return c->xsplit && c->split_ok && c->hs.n_d > 0 && c->solver == IMEX_SOLVER_DIRECT;
}

// Kernel launches of one step.
int64_t launches_per_step(const imex_ctx* c) {
  int64_t n = 1;   // explicit apply
  if (split_active(c) && !scheme_is_cdm(c->hs.pb.scheme)) n += 1;   // its far tiles, on the side stream
  if (c->hs.n_c > 0 && !c->factorized) return n + 2;   // right-hand sides, PCG
  if (c->hs.n_c > 0) {
    for (size_t l = 0; l < c->lev_cta0.size(); ++l) n += (l == 0 || c->lev_ncta[l] > 0) ? 1 : 0;
    n += c->ntop > 0 ? 1 : 0;
    for (int h : c->lev_has_nodes) n += h;
    for (int k : c->pan_ncta) n += k > 0 ? 1 : 0;
    if (c->solver != IMEX_SOLVER_DIRECT) n += 2;   // right-hand sides, PCG (the direct launches follow, skipped)
  }
  return n;
}

// The autotuner of the explicit variant: time every candidate on this problem
// (one warm-up and five timed launches each, over all columns, writing into
// the scratch grid) and keep the fastest.  IMEX_EXPLICIT_TILE = large |
// small | sweep in the environment fixes the choice instead.
cudaError_t autotune_tile(imex_ctx* c) {
  const HostSetup& hs = c->hs;
  if (int v = explicit_env_variant(c); v >= 0) return use_explicit(c, v);
  cudaEvent_t ev[2];
  cudaError_t e = cudaEventCreate(&ev[0]);
  e = e ? e : cudaEventCreate(&ev[1]);
  float best = 1e30f;
  int best_var = 0;
  for (int k = 0; k < explicit_variants(c) && e == cudaSuccess; ++k) {
    e = use_explicit(c, k);
    if (e != cudaSuccess) break;
    ExplicitArgs ea = explicit_args(c, c->U[0], c->tmp, c->tmp, 2.0, -1.0, hs.dt * hs.dt, 0.0, false);
    explicit_dispatch(c, ea, ntiles(c), nullptr);
    e = cudaEventRecord(ev[0], nullptr);
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) explicit_dispatch(c, ea, ntiles(c), nullptr);
    e = e ? e : cudaEventRecord(ev[1], nullptr);
    e = e ? e : cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    e = e ? e : cudaEventElapsedTime(&ms, ev[0], ev[1]);
    c->tile_us[k] = 1e3f * ms / 5.f;
    if (e == cudaSuccess && c->tile_us[k] < best) {
      best = c->tile_us[k];
      best_var = k;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return e ? e : use_explicit(c, best_var);
}

// PCG on S (the step; Newmark correction) or, for the initial acceleration
// of a context without a factorisation, on M^cc with Jacobi (mode 1).
// The PCG kernel with `lpr` lanes per sparse row.
const void* pcg_kernel(int lpr) {
  switch (lpr) {
    case 4: return (const void*)k_pcg<4>;
    case 8: return (const void*)k_pcg<8>;
    case 16: return (const void*)k_pcg<16>;
    default: return (const void*)k_pcg<32>;
  }
}

cudaError_t launch_pcg(imex_ctx* c, double* Ubuf, cudaStream_t s, bool on_M = false) {
  const HostSetup& hs = c->hs;
  PcgArgs a{};
  a.n = (int)hs.n_c;
  a.s_ptr = c->s_ptr;
  a.s_col = c->s_col;
  a.s_val = on_M ? c->m_val : c->s_val;
  a.g_ptr = c->g_ptr;
  a.g_col = c->g_col;
  a.g_val = c->g_val;
  a.gt_ptr = c->gt_ptr;
  a.gt_row = c->gt_row;
  a.gt_idx = c->gt_idx;
  a.dinv = on_M ? c->dinv_m : c->dinv;
  a.precond = (on_M || c->solver == IMEX_SOLVER_PCG_JACOBI) ? 2 : 1;
  a.b = c->rhs0;
  a.x = c->pcg_x;
  a.r = c->pcg_r;
  a.z = c->pcg_z;
  a.p = c->pcg_p;
  a.q = c->pcg_q;
  a.w = c->pcg_w;
  a.v = c->pcg_v;
  a.part = c->pcg_part;
  a.tol = on_M ? 1e-12 : c->pcg_tol;
  a.maxit = on_M ? 100000 : c->pcg_maxit;
  a.hist1 = on_M ? nullptr : c->pcg_hist;
  a.hist2 = on_M ? nullptr : c->pcg_hist + hs.n_c;
  a.guess_w = (!on_M && c->guess_on && c->guess_valid >= 2) ? c->guess_state : nullptr;
  a.always_correct = c->factorized ? 0 : 1;   // no direct solve to fall back on
  a.status = c->pcg_status;
  a.counters = c->pcg_counters;
  a.res = c->pcg_res;
  a.mode = on_M ? 1 : 0;
  a.c_node = c->c_node;
  a.U = Ubuf;
  a.v_c = c->v_c;
  a.a_c = c->a_c;
  a.dt = hs.dt;
  PcgCols t2{c->gt_val};
  void* args[] = {&a, &t2};
  return cudaLaunchCooperativeKernel(pcg_kernel(c->pcg_lpr), dim3(c->pcg_grid), dim3(kThreads), args, 0, s);
}

// Right-hand sides rhs0 = f_t f^c - K^c src of a context without a solve plan.
void launch_rhs_c(imex_ctx* c, double ft, const double* src, cudaStream_t s, const double* ft_dev = nullptr) {
  const HostSetup& hs = c->hs;
  const int nc = (int)hs.n_c;
  const int64_t blocks = ((int64_t)nc * 32 + kThreads - 1) / kThreads;
  k_rhs_c<<<(unsigned)blocks, kThreads, 0, s>>>(nc, c->pr_ptr, c->pr_pos, c->if_base_dev, c->if_koff_dev,
                                                c->if_sc_dev, c->Kall, hs.P, hs.Pd, hs.nn[0], hs.nn[1], c->fxc,
                                                ft, ft_dev, src, c->rhs0);
}

double ft_at(const HostSetup& hs, int64_t n) {
  return wavelet_value(hs.pb.wavelet, hs.pb.f0, (double)n * hs.dt);
}

// Derived initial state from U[cur] = u_0 and tmp = v_0 (full grid):
// u^d_{-1} (Taylor start of CDM) into U[1-cur], a^c_0 from M^cc, v^c_0.
int compute_initial(imex_ctx* c, cudaStream_t s) {
  const HostSetup& hs = c->hs;
  double* U0 = c->U[c->cur];
  double* Uo = c->U[1 - c->cur];
  const double dt = hs.dt;
  const double ft0 = wavelet_value(hs.pb.wavelet, hs.pb.f0, 0.0);
  ExplicitArgs ea = explicit_args(c, U0, c->tmp, Uo, 1.0, -dt, 0.5 * dt * dt, ft0, false);
  explicit_dispatch(c, ea, ntiles(c), s);
  if (int rc = check_launch("explicit (initial)")) return rc;
  if (hs.n_c > 0) {
    const int nc = (int)hs.n_c;
    for (int col = 0; col < c->ncols; ++col)
      k_gather_c<<<(nc + 255) / 256, 256, 0, s>>>(c->v_c + (size_t)col * nc, c->tmp + (size_t)col * hs.nnodes,
                                                  c->c_node, nc);
    if (!c->factorized) {   // M^cc a^c_0 = f_t(0) f^c - K^c u_0 by Jacobi-PCG
      launch_rhs_c(c, ft0, U0, s);
      if (cudaError_t e = launch_pcg(c, U0, s, true))
        return fail(IMEX_ERR_CUDA, std::string("PCG (initial): ") + cudaGetErrorString(e));
    } else if (cudaError_t e = launch_solve_chain(c, false, ft0, nullptr, 1, U0, U0, c->upd, c->sol, c->rhs0, c->hbuf, s))
      return fail(IMEX_ERR_CUDA, std::string("solve (initial): ") + cudaGetErrorString(e));
    if (int rc = check_launch("solve (initial)")) return rc;
    if (scheme_is_cdm(hs.pb.scheme)) {   // the central-difference history of I_c as well
      k_cdm_start_c<<<dim3((nc + 255) / 256, c->ncols), 256, 0, s>>>(Uo, U0, c->v_c, c->a_c, c->c_node, nc,
                                                                       hs.nnodes, dt);
      if (int rc = check_launch("central-difference start")) return rc;
    }
  }
  return IMEX_OK;
}

// Static schedule of the implicit solve.
//  * Split level per component: the smallest level L >= 1 such that the nodes
//    at levels >= L hold at most kZmax rows; those rows form the dense top.
//  * Walked levels l = 0 .. max L - 1: the level's nodes of every component are
//    packed into CTAs, largest FP64 work first (level 0: with the right-hand
//    side pairs of their rows) onto the least-loaded CTA that has room in its
//    shared-memory blob (at most kMaxNodesPerCTA nodes; all threads of a CTA
//    share the rows of all its nodes in each phase), aiming at one CTA per SM;
//    supernodes above kMaxWidth rows go to k_panel instead.  A CTA's blob
//    holds its nodes' [L_tt^{-1} packed by diagonals | L_{rows,t} (ld m|1)],
//    16-byte aligned, for S and M^cc.
//  * Dense tops: each component's rows are cut into chunks so that the whole
//    launch has about one CTA per SM.
struct SolvePlan {
  std::vector<int> lev_cta0, lev_ncta, cta_node_ptr, cta_nodes;
  std::vector<int64_t> blob_off, blob_len, node_boff;
  std::vector<double> blobS, blobM;
  int64_t max_blob = 0;
  // Per-CTA index lists of the walk (layout: WalkList).
  std::vector<int> ilist;
  std::vector<int64_t> ilist_off, ilist_len;
  int64_t max_ilist = 0;
  int max_slots = 2, max_m = 2, max_pairs = 2;
  std::vector<int> lev_has_nodes;
  // Rows of the interface cell matrices (row-major) and per-cell scale; per
  // level-0 CTA the rows of its pairs (m-major, scaled).
  std::vector<double> Krows, if_sc, Kpair;
  std::vector<int64_t> kp_off, kp_len;
  int64_t max_kp = 0;
  std::vector<int> top_comp, top_r0, top_r1;
  // Per-component index lists of the dense tops (one entry per top CTA).
  std::vector<int> tlist;
  std::vector<int64_t> tlist_off, tlist_len;
  int64_t max_tlist = 0, max_arows = 0;
  std::vector<int> zsize, zbase, zrow, zfwd_ptr, zfwd_pos;
  std::vector<int64_t> zA_off;
  std::vector<double> zA_S, zA_M;
  int max_zn = 0;
  // Large supernodes of the walked levels (k_panel): per CTA a descriptor
  // (8 ints), the offset of its chunk in panS / panM, and its index list;
  // per level and phase (0..3) the CTA range.
  std::vector<int> pan_desc, pan_idx;
  std::vector<int64_t> pan_aoff;
  std::vector<double> panS, panM;
  std::vector<int> pan_cta0, pan_ncta;   // [4 level + phase]
  int64_t pan_max_chunk = 2;
  int pan_max_nv = 2;
  int64_t n_large = 0;
};

#ifndef IMEX_DENSE_TOP_MAX
#define IMEX_DENSE_TOP_MAX 600
#endif
constexpr int kZmax = IMEX_DENSE_TOP_MAX;   // largest dense top block per component
constexpr int kTargetCTAs = 152;            // one CTA per SM
constexpr int kMaxNodesPerCTA = 32;

// A_Z = (L_ZZ L_ZZ^T)^{-1} (row-major zn x zn) from the factor blocks of the
// component's top nodes; Z rows are the nodes' c-indices in ascending order.
void dense_top(const HostSetup& hs, const Factor& F, const std::vector<int>& znodes,
               const std::vector<int>& zpos, int zn, std::vector<double>& A) {
  std::vector<double> L((size_t)zn * zn, 0.0);   // column-major lower
  for (int t : znodes) {
    const TreeNode& T = hs.tree[t];
    const int b = T.end - T.beg, m = (int)T.rows.size();
    const double* Ld = F.Ld.data() + F.ld_off[t];
    const double* L21 = F.vals.data() + T.off_rect;
    for (int j = 0; j < b; ++j) {
      const int cj = zpos[T.beg + j];
      for (int i = j; i < b; ++i) L[zpos[T.beg + i] + (size_t)zn * cj] = Ld[i + (size_t)b * j];
      for (int i = 0; i < m; ++i) L[zpos[T.rows[i]] + (size_t)zn * cj] = L21[i + (size_t)m * j];
    }
  }
  std::vector<double> Mi((size_t)zn * zn, 0.0);  // L^{-1}, column-major lower
  for (int k = 0; k < zn; ++k)
    for (int i = k; i < zn; ++i) {
      double sum = (i == k) ? 1.0 : 0.0;
      for (int q = k; q < i; ++q) sum -= L[i + (size_t)zn * q] * Mi[q + (size_t)zn * k];
      Mi[i + (size_t)zn * k] = sum / L[i + (size_t)zn * i];
    }
  A.assign((size_t)zn * zn, 0.0);
  for (int i = 0; i < zn; ++i)
    for (int j = 0; j <= i; ++j) {
      double sum = 0.0;
      for (int k = i; k < zn; ++k) sum += Mi[k + (size_t)zn * i] * Mi[k + (size_t)zn * j];
      A[(size_t)i * zn + j] = sum;
      A[(size_t)j * zn + i] = sum;
    }
}

// Rows of the interface-cell matrices (the stored cut-cell matrices, then the
// uncut one at index n_cut; row-major), the scale of each interface cell
// (c_e^2 / c0^2 for the uncut form, 1 for cut cells) and its first grid node.
int interface_rows(const HostSetup& hs, std::vector<double>& Krows, std::vector<double>& if_sc,
                   std::vector<int>& if_base) {
  const int Pd = hs.Pd, n_cut = (int)hs.n_cut, nif = (int)hs.if_cell.size();
  Krows.assign(((size_t)n_cut + 1) * Pd * Pd, 0.0);
  for (int k = 0; k < n_cut; ++k)
    for (int l = 0; l < Pd; ++l)
      for (int m = 0; m < Pd; ++m)
        Krows[((size_t)k * Pd + l) * Pd + m] = hs.cutK[(size_t)k * Pd * Pd + l + (size_t)Pd * m];
  for (int l = 0; l < Pd; ++l)
    for (int m = 0; m < Pd; ++m) Krows[((size_t)n_cut * Pd + l) * Pd + m] = hs.uncutK[l + (size_t)Pd * m];
  if_sc.assign(std::max(nif, 1), 1.0);
  if_base.assign(std::max(nif, 1), 0);
  const int ncx = hs.pb.ncells[0], ncy = hs.pb.ncells[1];
  for (int e = 0; e < nif; ++e) {
    const int cid = hs.if_cell[e];
    const int cx = cid % ncx, cy = (cid / ncx) % ncy, cz = cid / (ncx * ncy);
    const int64_t base = (int64_t)cx * hs.p + (int64_t)hs.nn[0] * cy * hs.p + (int64_t)hs.nn[0] * hs.nn[1] * cz * hs.p;
    if (base > INT32_MAX) return fail(IMEX_ERR_ARG, "grid too large for 32-bit node indices");
    if_base[e] = (int)base;
    if (hs.if_kidx[e] < 0) if_sc[e] = hs.if_c2[e];
  }
  return IMEX_OK;
}

// Row chunks of the large supernodes `big` of walked level l, for both
// factors (S and M^cc), in the four k_panel phases (PanelArgs): forward
// y = L_tt^{-1} g and upd = L_{rows,t} y, backward h = y - L_{rows,t}^T x_rows
// and x = L_tt^{-T} h.  Chunks hold at most kPanelChunk doubles and at most
// kThreads rows; the triangular blocks keep only their nonzero columns.
int plan_panels(const HostSetup& hs, const std::vector<int>& big, int l, SolvePlan& P) {
  auto rows_per = [](int64_t nv) { return (int)std::max<int64_t>(1, std::min<int64_t>(kThreads, kPanelChunk / std::max<int64_t>(nv, 1))); };
  for (int phase = 0; phase < 4; ++phase) {
    P.pan_cta0[4 * l + phase] = (int)P.pan_aoff.size();
    int ncta = 0;
    for (int t : big) {
      const TreeNode& T = hs.tree[t];
      const int b = T.end - T.beg, m = (int)T.rows.size();
      const int nout = phase == 1 ? m : b;
      const int step = rows_per(phase == 2 ? m : b);
      for (int r0 = 0; r0 < nout; r0 += step) {
        const int r1 = std::min(nout, r0 + step), nr = r1 - r0;
        const int nv = phase == 0 ? r1 : phase == 1 ? b : phase == 2 ? m : b - r0;
        // index list
        std::vector<int> il;
        for (int j = 0; j < nv; ++j)
          il.push_back(phase == 0 || phase == 1 ? T.beg + j : phase == 2 ? T.rows[j] : T.beg + r0 + j);
        if (phase == 0) {
          il.resize((size_t)3 * nv + nr, 0);
          for (int j = 0; j < nv; ++j) {
            const int r = T.beg + j;
            il[nv + 2 * j] = (int)il.size();
            for (int k = hs.fwd_ptr[r]; k < hs.fwd_ptr[r + 1]; ++k) il.push_back(hs.fwd_pos[k]);
            il[nv + 2 * j + 1] = (int)il.size();
          }
          for (int i = 0; i < nr; ++i) il[3 * nv + i] = T.beg + r0 + i;
        } else {
          for (int i = 0; i < nr; ++i) il.push_back(phase == 1 ? (int)T.off_upd + r0 + i : T.beg + r0 + i);
        }
        P.pan_desc.insert(P.pan_desc.end(), {phase, nr, nv, (int)P.pan_idx.size(), t, r0, 0, 0});
        P.pan_idx.insert(P.pan_idx.end(), il.begin(), il.end());
        // chunk, column-major: element (i, j) at j nr + i
        for (const Factor* F : {&hs.S, &hs.Mcc}) {
          std::vector<double>& out = (F == &hs.S) ? P.panS : P.panM;
          if (out.size() % 2) out.push_back(0.0);
          if (F == &hs.S) P.pan_aoff.push_back((int64_t)out.size());
          const double* Li = F->vals.data() + T.off_diag;    // L_tt^{-1}[i][j] = Li[i + b j]
          const double* L21 = F->vals.data() + T.off_rect;   // L_{rows,t}[k][j] = L21[k + m j]
          for (int j = 0; j < nv; ++j)
            for (int i = 0; i < nr; ++i) {
              double v;
              if (phase == 0) v = (j <= r0 + i) ? Li[(r0 + i) + (size_t)b * j] : 0.0;
              else if (phase == 1) v = L21[(r0 + i) + (size_t)m * j];
              else if (phase == 2) v = L21[j + (size_t)m * (r0 + i)];
              else v = (r0 + j >= r0 + i) ? Li[(r0 + j) + (size_t)b * (r0 + i)] : 0.0;
              out.push_back(v);
            }
          if (out.size() % 2) out.push_back(0.0);
        }
        const int64_t n = (int64_t)nr * nv;
        P.pan_max_chunk = std::max<int64_t>(P.pan_max_chunk, n + (n & 1));
        P.pan_max_nv = std::max(P.pan_max_nv, nv + (nv & 1));
        ++ncta;
      }
    }
    P.pan_ncta[4 * l + phase] = ncta;
  }
  if (P.panS.size() != P.panM.size()) return fail(IMEX_ERR_ARG, "internal error: panel chunks of S and M differ");
  if (P.pan_idx.size() > (size_t)INT32_MAX) return fail(IMEX_ERR_ARG, "panel index lists too large");
  return IMEX_OK;
}

int plan_solve(imex_ctx* c, SolvePlan& P) {
  const HostSetup& hs = c->hs;
  const int64_t nt = (int64_t)hs.tree.size();
  // FP64 work of a supernode in a walk CTA: its triangular and rectangular
  // products and, at level 0 (which forms the right-hand sides), one P^d dot
  // product per (row, interface cell) pair of its rows, issued in batches
  // of 16 (the kernel's pair_product).
  const int64_t pair_cost = ((int64_t)hs.Pd + 15) / 16 * 16;
  auto node_work = [&](int t) {
    const TreeNode& T = hs.tree[t];
    const int64_t b = T.end - T.beg, m = (int64_t)T.rows.size();
    int64_t w = b * b / 2 + m * b + b;
    if (T.level == 0)
      for (int r = T.beg; r < T.end; ++r) w += pair_cost * (hs.contrib_ptr[r + 1] - hs.contrib_ptr[r]);
    return w;
  };
  // Split level of each component: nodes at level >= lz form the dense top part.
  std::vector<int> lz(hs.ncomp, 1), zsize(hs.ncomp, 0), zbase(hs.ncomp, 0), zrow, zpos(hs.n_c, -1);
  std::vector<int64_t> zA_off(hs.ncomp, 0);
  std::vector<double> zA_S, zA_M;
  int max_zn = 0;
  for (int k = 0; k < hs.ncomp; ++k) {
    int maxlev = 0;
    for (int t = hs.comp_tree_ptr[k]; t < hs.comp_tree_ptr[k + 1]; ++t) maxlev = std::max(maxlev, hs.tree[t].level);
    int L = maxlev + 1;
    for (int cand = 1; cand <= maxlev + 1; ++cand) {
      int z = 0;
      for (int t = hs.comp_tree_ptr[k]; t < hs.comp_tree_ptr[k + 1]; ++t)
        if (hs.tree[t].level >= cand) z += hs.tree[t].end - hs.tree[t].beg;
      if (z <= kZmax) { L = cand; break; }
    }
    lz[k] = L;
    std::vector<int> znodes;
    for (int t = hs.comp_tree_ptr[k]; t < hs.comp_tree_ptr[k + 1]; ++t)
      if (hs.tree[t].level >= L) znodes.push_back(t);
    zbase[k] = (int)zrow.size();
    for (int t : znodes)
      for (int r = hs.tree[t].beg; r < hs.tree[t].end; ++r) zrow.push_back(r);
    std::sort(zrow.begin() + zbase[k], zrow.end());
    zsize[k] = (int)zrow.size() - zbase[k];
    max_zn = std::max(max_zn, zsize[k]);
    for (int i = 0; i < zsize[k]; ++i) zpos[zrow[zbase[k] + i]] = i;
    if (zA_S.size() % 2) { zA_S.push_back(0.0); zA_M.push_back(0.0); }
    zA_off[k] = (int64_t)zA_S.size();
    if (zsize[k] > 0) {
      std::vector<double> A;
      dense_top(hs, hs.S, znodes, zpos, zsize[k], A);
      zA_S.insert(zA_S.end(), A.begin(), A.end());
      dense_top(hs, hs.Mcc, znodes, zpos, zsize[k], A);
      zA_M.insert(zA_M.end(), A.begin(), A.end());
    }
  }
  // Updates into the dense rows from the walked levels only.
  std::vector<int> upd_owner(std::max<int64_t>(hs.upd_size, 1), -1);
  for (size_t t = 0; t < hs.tree.size(); ++t)
    for (size_t i = 0; i < hs.tree[t].rows.size(); ++i) upd_owner[hs.tree[t].off_upd + i] = (int)t;
  auto is_top = [&](int t) { return hs.tree[t].level >= lz[hs.tree[t].comp]; };
  std::vector<int> zfwd_ptr(1, 0), zfwd_pos;
  for (int r : zrow) {
    for (int k = hs.fwd_ptr[r]; k < hs.fwd_ptr[r + 1]; ++k)
      if (!is_top(upd_owner[hs.fwd_pos[k]])) zfwd_pos.push_back(hs.fwd_pos[k]);
    zfwd_ptr.push_back((int)zfwd_pos.size());
  }
  // Check the split algorithm (walked levels + dense top) against the tree solve.
  for (const Factor* F : {&hs.S, &hs.Mcc}) {
    const std::vector<double>& zA = (F == &hs.S) ? zA_S : zA_M;
    std::vector<double> b(hs.n_c), xref, x(hs.n_c, 0.0), upd(std::max<int64_t>(hs.upd_size, 1), 0.0), g, y;
    for (int64_t i = 0; i < hs.n_c; ++i) b[i] = std::cos(0.71 * i + 0.3) + 0.25;
    xref = b;
    replay_solve(hs, *F, xref);
    std::vector<std::vector<int>> byl;
    for (size_t t = 0; t < hs.tree.size(); ++t)
      if (!is_top((int)t)) {
        if ((int)byl.size() <= hs.tree[t].level) byl.resize(hs.tree[t].level + 1);
        byl[hs.tree[t].level].push_back((int)t);
      }
    for (size_t l = 0; l < byl.size(); ++l)
      for (int t : byl[l]) {
        const TreeNode& T = hs.tree[t];
        const int bsz = T.end - T.beg, m = (int)T.rows.size();
        g.assign(bsz, 0.0);
        y.assign(bsz, 0.0);
        for (int i = 0; i < bsz; ++i) {
          const int r = T.beg + i;
          double sum = b[r];
          for (int k = hs.fwd_ptr[r]; k < hs.fwd_ptr[r + 1]; ++k) sum -= upd[hs.fwd_pos[k]];
          g[i] = sum;
        }
        for (int i = 0; i < bsz; ++i) {
          double sum = 0.0;
          for (int j = 0; j <= i; ++j) sum += F->vals[T.off_diag + i + (int64_t)bsz * j] * g[j];
          y[i] = sum;
          x[T.beg + i] = sum;
        }
        for (int k = 0; k < m; ++k) {
          double sum = 0.0;
          for (int j = 0; j < bsz; ++j) sum += F->vals[T.off_rect + k + (int64_t)m * j] * y[j];
          upd[T.off_upd + k] = sum;
        }
      }
    for (int k = 0; k < hs.ncomp; ++k) {
      const int zn = zsize[k], zb = zbase[k];
      std::vector<double> zg(zn);
      for (int i = 0; i < zn; ++i) {
        double sum = b[zrow[zb + i]];
        for (int q = zfwd_ptr[zb + i]; q < zfwd_ptr[zb + i + 1]; ++q) sum -= upd[zfwd_pos[q]];
        zg[i] = sum;
      }
      for (int i = 0; i < zn; ++i) {
        double sum = 0.0;
        for (int j = 0; j < zn; ++j) sum += zA[zA_off[k] + (int64_t)i * zn + j] * zg[j];
        x[zrow[zb + i]] = sum;
      }
    }
    for (int l = (int)byl.size() - 1; l >= 0; --l)
      for (int t : byl[l]) {
        const TreeNode& T = hs.tree[t];
        const int bsz = T.end - T.beg, m = (int)T.rows.size();
        g.assign(bsz, 0.0);
        for (int j = 0; j < bsz; ++j) {
          double sum = x[T.beg + j];
          for (int k = 0; k < m; ++k) sum -= F->vals[T.off_rect + k + (int64_t)m * j] * x[T.rows[k]];
          g[j] = sum;
        }
        for (int i = 0; i < bsz; ++i) {
          double sum = 0.0;
          for (int j = i; j < bsz; ++j) sum += F->vals[T.off_diag + j + (int64_t)bsz * i] * g[j];
          x[T.beg + i] = sum;
        }
      }
    double dn = 0.0, rn = 0.0;
    for (int64_t i = 0; i < hs.n_c; ++i) {
      dn += (x[i] - xref[i]) * (x[i] - xref[i]);
      rn += xref[i] * xref[i];
    }
    if (!(std::sqrt(dn / std::max(rn, 1e-300)) < 1e-9))
      return fail(IMEX_ERR_NOT_SPD, "dense top-level solve disagrees with the tree solve");
  }
  // Interface cells: rows of their matrices and scales, first node of each.
  const int Pd = hs.Pd, n_cut = (int)hs.n_cut;
  std::vector<int> if_base;
  if (int rc = interface_rows(hs, P.Krows, P.if_sc, if_base)) return rc;
  if (hs.upd_size > INT32_MAX) return fail(IMEX_ERR_ARG, "implicit partition too large for 32-bit update offsets");
  auto npairs_of = [&](int r) { return hs.contrib_ptr[r + 1] - hs.contrib_ptr[r]; };

  // Walked levels: pack each level's nodes into CTAs by longest processing
  // time.  Level 0 always has a launch: it forms every right-hand side.
  int nlev = 0;
  for (size_t t = 0; t < hs.tree.size(); ++t)
    if (!is_top((int)t)) nlev = std::max(nlev, hs.tree[t].level + 1);
  const int nlaunch = std::max(nlev, 1);
  std::vector<char> own0(std::max<int64_t>(hs.n_c, 1), 0);
  for (size_t t = 0; t < hs.tree.size(); ++t)
    if (!is_top((int)t) && hs.tree[t].level == 0)
      for (int r = hs.tree[t].beg; r < hs.tree[t].end; ++r) own0[r] = 1;
  std::vector<int> extra_rows;
  for (int64_t r = 0; r < hs.n_c; ++r)
    if (!own0[r]) extra_rows.push_back((int)r);
  const size_t vec_doubles = 0;
  const int64_t blob_cap = (int64_t)(kWalkSmemBudget / sizeof(double));
  P.node_boff.assign(nt, 0);
  P.cta_node_ptr.assign(1, 0);
  // Supernodes with more than kMaxWidth diagonal or ancestor rows are
  // walked by k_panel (row chunks over many CTAs) instead of one walk CTA.
  auto is_big = [&](int t) {
    const TreeNode& T = hs.tree[t];
    return T.end - T.beg > kMaxWidth || (int)T.rows.size() > kMaxWidth;
  };
  P.pan_cta0.assign(4 * (size_t)nlaunch, 0);
  P.pan_ncta.assign(4 * (size_t)nlaunch, 0);
  for (int l = 0; l < nlaunch; ++l) {
    std::vector<int> nodes, big;
    for (size_t t = 0; t < hs.tree.size(); ++t)
      if (!is_top((int)t) && hs.tree[t].level == l) (is_big((int)t) ? big : nodes).push_back((int)t);
    std::sort(nodes.begin(), nodes.end(), [&](int x, int y) { return node_work(x) > node_work(y); });
    if (int rc = plan_panels(hs, big, l, P)) return rc;
    P.n_large += (int64_t)big.size();
    auto bytes_of = [&](int t) {   // shared memory of a node, in doubles
      const TreeNode& T = hs.tree[t];
      const int64_t b = T.end - T.beg, m = (int64_t)T.rows.size();
      int64_t ints = 4 * b + 2 * m + 8;
      int64_t pairs = 0;
      for (int r = T.beg; r < T.end; ++r) {
        ints += hs.fwd_ptr[r + 1] - hs.fwd_ptr[r];
        if (l == 0) pairs += npairs_of(r);
      }
      ints += l == 0 ? 4 * b + 4 * pairs : 0;
      return b * (b + 1) / 2 + (m | 1) * b + 2 * b + m + (Pd + 1) * pairs + (ints + 1) / 2 + 2;
    };
    int target = std::max(1, std::min<int>((int)nodes.size(), kTargetCTAs));
    if (l == 0) {
      int64_t extra_pairs = 0;
      for (int r : extra_rows) extra_pairs += npairs_of(r);
      // at most 32 extra rows and about 48 KB of their cell-matrix rows per CTA
      const int64_t by_pairs = (extra_pairs * (Pd + 1) * (int64_t)sizeof(double) + 49151) / 49152;
      target = std::max(target, (int)std::min<int64_t>(kTargetCTAs, std::max<int64_t>(
                                                                          ((int64_t)extra_rows.size() + 31) / 32, by_pairs)));
    }
    std::vector<std::vector<int>> per(target);
    std::vector<int64_t> work(target, 0), used(target, 0);
    for (int t : nodes) {
      int best = -1;
      for (int r = 0; r < (int)per.size(); ++r) {
        if ((int)per[r].size() >= kMaxNodesPerCTA) continue;
        if (!per[r].empty() && used[r] + bytes_of(t) > blob_cap) continue;
        if (best < 0 || work[r] < work[best]) best = r;
      }
      if (best < 0) {
        per.emplace_back();
        work.push_back(0);
        used.push_back(0);
        best = (int)per.size() - 1;
      }
      per[best].push_back(t);
      work[best] += node_work(t);
      used[best] += bytes_of(t);
    }
    // Level 0: the rows it does not solve get their right-hand side from the
    // least loaded CTA (work of a pair: one P^d dot product).
    std::vector<std::vector<int>> xrows(per.size());
    if (l == 0) {
      std::vector<int> order = extra_rows;
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return npairs_of(x) > npairs_of(y); });
      for (int r : order) {
        int best = 0;
        for (int q = 1; q < (int)per.size(); ++q)
          if (work[q] < work[best]) best = q;
        xrows[best].push_back(r);
        work[best] += pair_cost * npairs_of(r) + 1;
      }
      for (auto& xr : xrows) std::sort(xr.begin(), xr.end());
    }
    P.lev_cta0.push_back((int)P.blob_off.size());
    P.lev_has_nodes.push_back(nodes.empty() ? 0 : 1);
    int ncta = 0;
    for (size_t q0 = 0; q0 < per.size(); ++q0) {
      const std::vector<int>& list = per[q0];
      if (list.empty() && xrows[q0].empty()) continue;
      ++ncta;
      if (P.blobS.size() % 2) { P.blobS.push_back(0.0); P.blobM.push_back(0.0); }
      P.blob_off.push_back((int64_t)P.blobS.size());
      int64_t local = 0;
      int nslot = 0, nm = 0, npair = 0;
      std::vector<int> slot0(list.size()), moff(list.size());
      // Per supernode: L_tt^{-1} packed by diagonals (diagonal d: entries
      // (d + i, i), i < b - d), then L_{rows,t} column-major with an odd
      // leading dimension.
      for (size_t q = 0; q < list.size(); ++q) {
        const TreeNode& T = hs.tree[list[q]];
        const int b = T.end - T.beg, m = (int)T.rows.size();
        const int ldr = m | 1;
        P.node_boff[list[q]] = local;
        slot0[q] = nslot;
        moff[q] = nm;
        nslot += b;
        nm += m;
        for (const Factor* F : {&hs.S, &hs.Mcc}) {
          std::vector<double>& out = (F == &hs.S) ? P.blobS : P.blobM;
          const double* Li = F->vals.data() + T.off_diag;
          const double* L21 = F->vals.data() + T.off_rect;
          for (int d = 0; d < b; ++d)
            for (int i = 0; i + d < b; ++i) out.push_back(Li[(i + d) + (size_t)b * i]);
          for (int j = 0; j < b; ++j)
            for (int i = 0; i < ldr; ++i) out.push_back(i < m ? L21[i + (size_t)m * j] : 0.0);
        }
        local += (int64_t)b * (b + 1) / 2 + (int64_t)ldr * b;
        P.cta_nodes.push_back(list[q]);
      }
      if (local % 2) { P.blobS.push_back(0.0); P.blobM.push_back(0.0); ++local; }
      if (local > INT32_MAX) return fail(IMEX_ERR_ARG, "solve CTA blob too large");
      P.blob_len.push_back(local);
      P.max_blob = std::max(P.max_blob, local);
      P.cta_node_ptr.push_back((int)P.cta_nodes.size());
      // Right-hand-side rows (level 0): own rows in slot order, then the extra rows.
      std::vector<int> rrows, rslot;
      if (l == 0) {
        for (size_t q = 0; q < list.size(); ++q)
          for (int r = hs.tree[list[q]].beg; r < hs.tree[list[q]].end; ++r) {
            rrows.push_back(r);
            rslot.push_back(slot0[q] + r - hs.tree[list[q]].beg);
          }
        for (int r : xrows[q0]) {
          rrows.push_back(r);
          rslot.push_back(-1);
        }
        for (int r : rrows) npair += npairs_of(r);
      }
      const int nrhs = (int)rrows.size();
      const int o_node = 8, o_slot = o_node + 8 * (int)list.size(), o_anc = o_slot + 4 * nslot;
      const int o_rhs = o_anc + ((2 * nm + 3) & ~3), o_pair = o_rhs + 4 * nrhs, o_pos = o_pair + 4 * npair;
      std::vector<int> Lst(o_pos, 0);
      Lst[0] = (int)list.size();
      Lst[1] = nslot;
      Lst[2] = nm;
      Lst[3] = nrhs;
      Lst[4] = npair;
      for (size_t q = 0; q < list.size(); ++q) {
        const TreeNode& T = hs.tree[list[q]];
        const int b = T.end - T.beg, m = (int)T.rows.size();
        int* nd = &Lst[o_node + 8 * q];
        nd[0] = list[q];
        nd[1] = T.beg;
        nd[2] = b;
        nd[3] = m;
        nd[4] = slot0[q];
        nd[5] = moff[q];
        nd[6] = (int)P.node_boff[list[q]];
        nd[7] = (int)T.off_upd;
        for (int i = 0; i < b; ++i) {
          // Indices, not pointers: the appends below may reallocate Lst.
          const int r = T.beg + i;
          const size_t st = (size_t)o_slot + 4 * (size_t)(slot0[q] + i);
          Lst[st] = (int)q;
          Lst[st + 1] = (int)Lst.size();
          for (int k = hs.fwd_ptr[r]; k < hs.fwd_ptr[r + 1]; ++k) Lst.push_back(hs.fwd_pos[k]);
          Lst[st + 2] = (int)Lst.size();
        }
        for (int k = 0; k < m; ++k) {
          Lst[o_anc + 2 * (moff[q] + k)] = (int)q;
          Lst[o_anc + 2 * (moff[q] + k) + 1] = T.rows[k];
        }
      }
      int pq = 0;
      for (int k = 0; k < nrhs; ++k) {
        const int r = rrows[k];
        int* rr = &Lst[o_rhs + 4 * k];
        rr[0] = r;
        rr[1] = pq;
        for (int q = hs.contrib_ptr[r]; q < hs.contrib_ptr[r + 1]; ++q, ++pq) {
          const int e = hs.contrib_pos[q] / Pd, lnode = hs.contrib_pos[q] % Pd;
          int* pr = &Lst[o_pair + 4 * pq];
          pr[0] = if_base[e];
          pr[1] = (hs.if_kidx[e] >= 0 ? hs.if_kidx[e] : n_cut) * Pd + lnode;
          pr[2] = e;
        }
        rr[2] = pq;
        rr[3] = rslot[k];
      }
      Lst[5] = npair + (npair & 1);
      // Rows of the cell matrices of the pairs, m-major, scales folded in.
      if (P.Kpair.size() % 2) P.Kpair.push_back(0.0);
      P.kp_off.push_back((int64_t)P.Kpair.size());
      {
        const int np = npair + (npair & 1);
        std::vector<double> blk((size_t)Pd * np, 0.0);
        for (int k = 0; k < npair; ++k) {
          const int* pr = &Lst[o_pair + 4 * k];
          const double* row = P.Krows.data() + (size_t)pr[1] * Pd;
          const double sc = P.if_sc[pr[2]];
          for (int m = 0; m < Pd; ++m) blk[(size_t)m * np + k] = sc * row[m];
        }
        P.Kpair.insert(P.Kpair.end(), blk.begin(), blk.end());
        P.kp_len.push_back((int64_t)blk.size());
        P.max_kp = std::max<int64_t>(P.max_kp, (int64_t)blk.size());
      }
      while (Lst.size() % 4) Lst.push_back(0);
      P.ilist_off.push_back((int64_t)P.ilist.size());
      P.ilist_len.push_back((int64_t)Lst.size());
      P.ilist.insert(P.ilist.end(), Lst.begin(), Lst.end());
      P.max_ilist = std::max<int64_t>(P.max_ilist, (int64_t)Lst.size());
      P.max_slots = std::max(P.max_slots, nslot + (nslot & 1));
      P.max_m = std::max(P.max_m, nm + (nm & 1));
      P.max_pairs = std::max(P.max_pairs, npair + (npair & 1));
    }
    P.lev_ncta.push_back(ncta);
  }
  (void)vec_doubles;
  // Dense tops: row chunks, about one CTA per SM over the whole launch.
  std::vector<std::vector<int>> tl(hs.ncomp);
  for (int k = 0; k < hs.ncomp; ++k) {
    const int zn = zsize[k], zb = zbase[k];
    std::vector<int>& L = tl[k];
    L.assign(2 * (size_t)zn, 0);
    for (int i = 0; i < zn; ++i) {
      L[2 * i] = (int)L.size();
      for (int q = zfwd_ptr[zb + i]; q < zfwd_ptr[zb + i + 1]; ++q) L.push_back(zfwd_pos[q]);
      L[2 * i + 1] = (int)L.size();
    }
    while (L.size() % 4) L.push_back(0);
    P.max_tlist = std::max<int64_t>(P.max_tlist, (int64_t)L.size());
  }
  const int64_t max_zn_even = std::max(2, max_zn + (max_zn & 1));
  // Rows per CTA from the FP64 work |Z|^2 spread over at most one CTA per SM
  // (even, so that every chunk of A_Z starts on a 16-byte boundary; at most
  // one row per thread).
  int64_t zwork = 0;
  for (int k = 0; k < hs.ncomp; ++k) zwork += (int64_t)zsize[k] * zsize[k];
  std::vector<int> chunk_of(hs.ncomp, 2);
  auto top_smem = [&](int64_t rows, int) {
    return (size_t)(max_zn_even + rows + (rows & 1) + kThreads) * sizeof(double) + (size_t)P.max_tlist * sizeof(int);
  };
  for (int64_t wcta = std::max<int64_t>(1, zwork / kTargetCTAs);; wcta += wcta / 8 + 1) {
    int64_t nctas = 0;
    for (int k = 0; k < hs.ncomp; ++k) {
      const int zn = std::max(1, zsize[k]);
      int ch = (int)std::max<int64_t>(2, std::min<int64_t>({(int64_t)zn, wcta / zn, (int64_t)kThreads}));
      ch += ch & 1;
      while (ch > 2 && top_smem((int64_t)ch * zn, ch) > kTopSmemBudget) ch -= 2;
      if (top_smem((int64_t)ch * zn, ch) > kTopSmemBudget)
        return fail(IMEX_ERR_ARG, "dense top block too large for shared memory (lower IMEX_DENSE_TOP_MAX)");
      chunk_of[k] = ch;
      if (zsize[k] > 0) nctas += (zsize[k] + ch - 1) / ch;
    }
    if (nctas <= kTargetCTAs || wcta > zwork) break;
  }
  std::vector<int64_t> comp_off(hs.ncomp, 0);
  for (int k = 0; k < hs.ncomp; ++k) {
    comp_off[k] = (int64_t)P.tlist.size();
    P.tlist.insert(P.tlist.end(), tl[k].begin(), tl[k].end());
  }
  for (int k = 0; k < hs.ncomp; ++k)
    for (int r0 = 0; r0 < zsize[k]; r0 += chunk_of[k]) {
      const int r1 = std::min(zsize[k], r0 + chunk_of[k]);
      P.top_comp.push_back(k);
      P.top_r0.push_back(r0);
      P.top_r1.push_back(r1);
      P.tlist_off.push_back(comp_off[k]);
      P.tlist_len.push_back((int64_t)tl[k].size());
      const int64_t rows = (int64_t)(r1 - r0) * zsize[k];
      P.max_arows = std::max<int64_t>(P.max_arows, rows + (rows & 1));
    }
  P.zsize = zsize;
  P.zbase = zbase;
  P.zrow = zrow;
  P.zfwd_ptr = zfwd_ptr;
  P.zfwd_pos = zfwd_pos;
  P.zA_off = zA_off;
  // Each CTA's chunk of rows [r0, r1) of A_Z column-major in place (the
  // kernel's column slices read consecutive words); the check above used the
  // row-major form.
  for (size_t q = 0; q < P.top_comp.size(); ++q) {
    const int k = P.top_comp[q], zn = zsize[k], r0 = P.top_r0[q], nr = P.top_r1[q] - r0;
    const int64_t off = zA_off[k] + (int64_t)r0 * zn;
    for (std::vector<double>* A : {&zA_S, &zA_M}) {
      std::vector<double> blk(A->begin() + off, A->begin() + off + (int64_t)nr * zn);
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < zn; ++j) (*A)[off + (int64_t)j * nr + i] = blk[(size_t)i * zn + j];
    }
  }
  for (int k = 0; k < 2; ++k) { zA_S.push_back(0.0); zA_M.push_back(0.0); }   // tail of the last 16-byte copy
  P.zA_S = std::move(zA_S);
  P.zA_M = std::move(zA_M);
  P.max_zn = max_zn;
  return IMEX_OK;
}

// Data of the iterative solve: S (CSR), the lower pattern of G with its
// transpose map, the per-entry row scale 1/sqrt(S_ii), and the start
// G = diag(S)^{-1/2} (theta = G / scale: 1 on the diagonal, 0 elsewhere).
struct PcgPlan {
  std::vector<int> g_ptr, g_col, gt_ptr, gt_row, gt_idx;
  std::vector<double> g_val, g_scale, g_theta, dinv;
  std::vector<uint8_t> g_isdiag;
};

int plan_pcg(const HostSetup& hs, PcgPlan& q) {
  const int n = (int)hs.n_c;
  q.g_ptr.assign(1, 0);
  q.dinv.assign(std::max(n, 1), 0.0);
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int k = hs.S_ptr[i]; k < hs.S_ptr[i + 1]; ++k)
      if (hs.S_col[k] == i) d = hs.S_val[k];
    if (!(d > 0.0)) return fail(IMEX_ERR_NOT_SPD, "S has a nonpositive diagonal entry");
    q.dinv[i] = 1.0 / d;
    const double sc = 1.0 / std::sqrt(d);
    for (int k = hs.S_ptr[i]; k < hs.S_ptr[i + 1]; ++k) {
      const int j = hs.S_col[k];
      if (j > i) continue;
      q.g_col.push_back(j);
      q.g_scale.push_back(sc);
      q.g_isdiag.push_back(j == i ? 1 : 0);
      q.g_theta.push_back(j == i ? 1.0 : 0.0);
      q.g_val.push_back(j == i ? sc : 0.0);
    }
    q.g_ptr.push_back((int)q.g_col.size());
  }
  // Transpose map: entries of each column j in row order.
  q.gt_ptr.assign(n + 1, 0);
  for (int j : q.g_col) q.gt_ptr[j + 1]++;
  for (int j = 0; j < n; ++j) q.gt_ptr[j + 1] += q.gt_ptr[j];
  q.gt_row.assign(q.g_col.size(), 0);
  q.gt_idx.assign(q.g_col.size(), 0);
  std::vector<int> fill(q.gt_ptr.begin(), q.gt_ptr.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int e = q.g_ptr[i]; e < q.g_ptr[i + 1]; ++e) {
      const int j = q.g_col[e];
      q.gt_row[fill[j]] = i;
      q.gt_idx[fill[j]++] = e;
    }
  return IMEX_OK;
}

// Even-odd and rank-one forms of the 1D operators of the explicit apply, each
// checked against the plain matrices it replaces.
int explicit_ops(const HostSetup& hs, double sx, double sy, Ops2D& ops) {
  const int P = hs.P, p = hs.p, H = P / 2;
  const bool odd = (P % 2) == 1;
  double kmax = 0.0, mmax = 0.0, asym = 0.0;
  for (int i = 0; i < P * P; ++i) {
    kmax = std::max(kmax, std::fabs(hs.K1[i]));
    mmax = std::max(mmax, std::fabs(hs.M1[i]));
  }
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j)
      asym = std::max(asym, std::fabs(hs.K1[i * P + j] - hs.K1[(P - 1 - i) * P + (P - 1 - j)]));
  if (asym > 1e-11 * kmax) return fail(IMEX_ERR_ARG, "1D stiffness is not centrosymmetric");
  ops = Ops2D{};
  for (int q = 0; q < 2; ++q) {
    const double sc = q == 0 ? sx : sy;
    double(&ke)[5][4] = q == 0 ? ops.kxe : ops.kye;
    double(&ko)[4][4] = q == 0 ? ops.kxo : ops.kyo;
    double(&kc)[5] = q == 0 ? ops.kxc : ops.kyc;
    for (int i = 0; i <= (odd ? H : H - 1); ++i) {
      for (int j = 0; j < H; ++j) {
        ke[i][j] = 0.5 * sc * (hs.K1[i * P + j] + hs.K1[i * P + (P - 1 - j)]);
        if (i < H) ko[i][j] = 0.5 * sc * (hs.K1[i * P + j] - hs.K1[i * P + (P - 1 - j)]);
      }
      if (odd) kc[i] = sc * hs.K1[i * P + H];
    }
  }
  // M1 = diag(w) + C a a^T, C = int x^{2p} - sum_k w_k x_k^{2p}.
  double C = 2.0 / (2.0 * p + 1.0);
  for (int k = 0; k < P; ++k) C -= hs.gll_w[k] * std::pow(hs.gll_x[k], 2 * p);
  for (int i = 0; i < P; ++i) {
    double d = 1.0;
    for (int k = 0; k < P; ++k)
      if (k != i) d *= hs.gll_x[i] - hs.gll_x[k];
    ops.a[i] = 1.0 / d;
    ops.w[i] = hs.gll_w[i];
    ops.ca[i] = C * ops.a[i];
  }
  double err = 0.0;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j)
      err = std::max(err, std::fabs(hs.M1[i * P + j] - ((i == j ? ops.w[i] : 0.0) + C * ops.a[i] * ops.a[j])));
  if (err > 1e-11 * mmax) return fail(IMEX_ERR_ARG, "1D mass does not split into GLL weights plus rank one");
  for (int i = 0; i < P; ++i) {
    const double s = (p % 2 == 0) ? 1.0 : -1.0;   // a_{P-1-i} = (-1)^p a_i
    if (std::fabs(ops.a[P - 1 - i] - s * ops.a[i]) > 1e-10 * std::fabs(ops.a[i]))
      return fail(IMEX_ERR_ARG, "GLL leading coefficients are not symmetric");
  }
  return IMEX_OK;
}

// 3D: even-odd stiffness per axis (scales s3) and the rank-one mass, from
// the 2D routine (whose checks apply to the same 1D matrices).
// Fold dt^2 M^{-1} into the 2D operators (Ops2D): x rows scaled by f_i, y
// rows by kappa f_i, f_i = 1 / (assembled GLL weight of local node i for an
// interior vertex: w_i, or w_0 + w_p at a vertex), kappa = dt^2 / (rho |J|).
void mass_scaled_ops(const HostSetup& hs, double kappa, Ops2D& ops) {
  const int P = hs.P, p = hs.p, H = P / 2;
  const bool odd = (P % 2) == 1;
  double f[9];
  for (int i = 0; i < P; ++i) f[i] = (i == 0 || i == p) ? 1.0 / (hs.gll_w[0] + hs.gll_w[p]) : 1.0 / hs.gll_w[i];
  for (int i = 0; i <= (odd ? H : H - 1); ++i) {   // row i (and P-1-i, f symmetric)
    for (int j = 0; j < H; ++j) {
      ops.kxe[i][j] *= f[i];
      ops.kye[i][j] *= kappa * f[i];
      if (i < H) {
        ops.kxo[i][j] *= f[i];
        ops.kyo[i][j] *= kappa * f[i];
      }
    }
    if (odd) {
      ops.kxc[i] *= f[i];
      ops.kyc[i] *= kappa * f[i];
    }
  }
  for (int i = 0; i < P; ++i) {
    ops.cax[i] = f[i] * ops.ca[i];
    ops.wy[i] = kappa * f[i] * ops.w[i];
    ops.cay[i] = kappa * f[i] * ops.ca[i];
  }
  ops.wyv = kappa;
}

int explicit_ops3(const HostSetup& hs, const double* s3, Ops3D& ops) {
  Ops2D a{}, b{};
  if (int rc = explicit_ops(hs, s3[0], s3[1], a)) return rc;
  if (int rc = explicit_ops(hs, s3[2], s3[2], b)) return rc;
  ops = Ops3D{};
  std::memcpy(ops.ke[0], a.kxe, sizeof(a.kxe));
  std::memcpy(ops.ko[0], a.kxo, sizeof(a.kxo));
  std::memcpy(ops.kc[0], a.kxc, sizeof(a.kxc));
  std::memcpy(ops.ke[1], a.kye, sizeof(a.kye));
  std::memcpy(ops.ko[1], a.kyo, sizeof(a.kyo));
  std::memcpy(ops.kc[1], a.kyc, sizeof(a.kyc));
  std::memcpy(ops.ke[2], b.kxe, sizeof(b.kxe));
  std::memcpy(ops.ko[2], b.kxo, sizeof(b.kxo));
  std::memcpy(ops.kc[2], b.kxc, sizeof(b.kxc));
  std::memcpy(ops.w, a.w, sizeof(a.w));
  std::memcpy(ops.ca, a.ca, sizeof(a.ca));
  std::memcpy(ops.a, a.a, sizeof(a.a));
  return IMEX_OK;
}

int build_context(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src,
                  Problem& pb) {
  if (!mesh || !src) return fail(IMEX_ERR_ARG, "mesh and source must not be NULL");
  pb.dim = mesh->dim;
  if (pb.dim != 2 && pb.dim != 3) return fail(IMEX_ERR_ARG, "dim must be 2 or 3");
  for (int d = 0; d < 3; ++d) {
    pb.lo[d] = mesh->lo[d];
    pb.hi[d] = mesh->hi[d];
    pb.ncells[d] = d < pb.dim ? mesh->ncells[d] : 1;
  }
  pb.p = p;
  pb.alpha = alpha;
  pb.depth = mesh->tree_depth;
  if (mesh->nholes < 0 || (mesh->nholes > 0 && !mesh->holes)) return fail(IMEX_ERR_ARG, "bad holes");
  pb.holes.assign(mesh->holes, mesh->holes + (size_t)mesh->nholes * 2 * pb.dim);
  pb.rho = mesh->rho;
  pb.c0 = mesh->c0;
  if (mesh->cell_c) {
    int64_t n = 1;
    for (int d = 0; d < pb.dim; ++d) n *= mesh->ncells[d];
    if (n <= 0) return fail(IMEX_ERR_ARG, "bad ncells");
    pb.cell_c.assign(mesh->cell_c, mesh->cell_c + n);
  }
  if (src->nsrc < 1 || !src->pos) return fail(IMEX_ERR_ARG, "source needs nsrc >= 1 positions");
  pb.nsrc = src->nsrc;
  pb.src_pos.assign(src->pos, src->pos + (size_t)src->nsrc * pb.dim);
  pb.f0 = src->f0;
  pb.sigma = src->sigma;
  pb.amp = src->amp;
  pb.wavelet = src->wavelet;
  if (pb.wavelet < 0 || pb.wavelet > 2) return fail(IMEX_ERR_ARG, "unknown wavelet");
  if (!(pb.f0 > 0.0)) return fail(IMEX_ERR_ARG, "f0 must be positive");
  pb.dt = dt;
  return IMEX_OK;
}

int setup_error_code(const std::string& e) {
  if (e.find("positive definite") != std::string::npos) return IMEX_ERR_NOT_SPD;
  if (e.find("degenerate") != std::string::npos) return IMEX_ERR_GEOM;
  return IMEX_ERR_ARG;
}

int setup_impl(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src, int ncols, int scheme,
               bool factorize, const imex_alloc* alloc, imex_ctx** out);

}  // namespace

extern "C" {

const char* imex_last_error(void) { return g_last_error.c_str(); }

int imex_gll_points(int p, double* x, double* w) {
  if (p < 1 || p > 32 || !x || !w) return fail(IMEX_ERR_ARG, "bad arguments");
  std::vector<double> xv, wv;
  gll_points(p, xv, wv);
  std::copy(xv.begin(), xv.end(), x);
  std::copy(wv.begin(), wv.end(), w);
  return IMEX_OK;
}

int imex_gauss_points(int n, double* x, double* w) {
  if (n < 1 || n > 64 || !x || !w) return fail(IMEX_ERR_ARG, "bad arguments");
  std::vector<double> xv, wv;
  gauss_points(n, xv, wv);
  std::copy(xv.begin(), xv.end(), x);
  std::copy(wv.begin(), wv.end(), w);
  return IMEX_OK;
}

// IMEX_LOG=1 in the environment: one JSON line of setup statistics on stderr.
static void log_setup(const HostSetup& hs, const char* where) {
  const char* v = std::getenv("IMEX_LOG");
  if (!v || std::strcmp(v, "1") != 0) return;
  std::fprintf(stderr,
               "{\"imex_setup\": \"%s\", \"dim\": %d, \"p\": %d, \"n_nodes\": %lld, \"n_d\": %lld, "
               "\"n_c\": %lld, \"n_uncut\": %lld, \"n_cut\": %lld, \"n_empty\": %lld, \"components\": %d, "
               "\"nnz_L\": %lld, \"max_block\": %d, \"dt\": %.17g, \"dt_crit_uncut\": %.17g, "
               "\"dt_crit_cut_min\": %.17g, \"scheme\": %d, \"factorized\": %d, \"setup_seconds\": %.6f}\n",
               where, hs.dim, hs.p, (long long)hs.nnodes, (long long)hs.n_d, (long long)hs.n_c,
               (long long)hs.n_uncut, (long long)hs.n_cut, (long long)hs.n_empty, hs.ncomp, (long long)hs.nnz_L,
               hs.max_block, hs.dt, hs.dt_crit_uncut, hs.dt_crit_cut_min, hs.pb.scheme, hs.pb.factorize ? 1 : 0,
               hs.setup_seconds);
}

void fill_stats(const HostSetup& hs, imex_stats* st) {
  std::memset(st, 0, sizeof(*st));
  st->n_nodes = hs.nnodes;
  st->n_d = hs.n_d;
  st->n_c = hs.n_c;
  st->n_cut = hs.n_cut;
  st->n_uncut = hs.n_uncut;
  st->n_empty = hs.n_empty;
  st->n_iface = (int64_t)hs.if_cell.size();
  st->nnz_L = hs.nnz_L;
  st->n_components = hs.ncomp;
  st->n_tree = (int64_t)hs.tree.size();
  st->max_block = hs.max_block;
  st->dt = hs.dt;
  st->dt_crit_uncut = hs.dt_crit_uncut;
  st->setup_seconds = hs.setup_seconds;
  st->residual_S = hs.residual_S;
  st->residual_M = hs.residual_M;
  st->scheme = hs.pb.scheme;
  st->dt_crit_cut_min = hs.dt_crit_cut_min;
}

int imex_host_implicit_system(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src,
                              int64_t* n_c, int64_t* nnz, int64_t* c_node, int64_t* s_ptr, int32_t* s_col,
                              double* s_val, double* m_val) {
  if (!n_c || !nnz) return fail(IMEX_ERR_ARG, "bad arguments");
  try {
    Problem pb;
    if (int rc = build_context(mesh, p, alpha, dt, src, pb)) return rc;
    HostSetup hs;
    std::string err = build_setup(pb, hs);
    if (!err.empty()) return fail(setup_error_code(err), err);
    const int64_t nc = hs.n_c, nz = (int64_t)hs.S_col.size();
    if (s_col) {   // the second call: arrays of the sizes the first one returned
      if (*n_c != nc || *nnz != nz) return fail(IMEX_ERR_ARG, "array sizes differ from the system's");
      if (!c_node || !s_ptr || !s_val || !m_val) return fail(IMEX_ERR_ARG, "bad arguments");
      for (int64_t r = 0; r < nc; ++r) c_node[r] = hs.c_node[r];
      for (int64_t r = 0; r <= nc; ++r) s_ptr[r] = hs.S_ptr[r];
      std::memcpy(s_col, hs.S_col.data(), (size_t)nz * sizeof(int32_t));
      std::memcpy(s_val, hs.S_val.data(), (size_t)nz * sizeof(double));
      std::memcpy(m_val, hs.M_val.data(), (size_t)nz * sizeof(double));
    }
    *n_c = nc;
    *nnz = nz;
    return IMEX_OK;
  } catch (const std::exception& ex) {
    return fail(IMEX_ERR_ALLOC, std::string("host setup failed: ") + ex.what());
  }
}

int imex_host_element_matrices(const imex_mesh* mesh, int p, double alpha, const imex_source* src, int ncell,
                               const int64_t* cells, double* K, double* M, int8_t* cell_type) {
  if (ncell < 0 || (ncell > 0 && (!cells || !K || !M))) return fail(IMEX_ERR_ARG, "bad arguments");
  try {
    Problem pb;
    if (int rc = build_context(mesh, p, alpha, 0.0, src, pb)) return rc;
    pb.factorize = false;
    pb.export_cells.assign(cells, cells + ncell);
    HostSetup hs;
    std::string err = build_setup(pb, hs);
    if (!err.empty()) return fail(setup_error_code(err), err);
    std::memcpy(K, hs.export_K.data(), hs.export_K.size() * sizeof(double));
    std::memcpy(M, hs.export_M.data(), hs.export_M.size() * sizeof(double));
    if (cell_type)
      for (int q = 0; q < ncell; ++q) cell_type[q] = hs.cell_type[cells[q]];
    return IMEX_OK;
  } catch (const std::exception& ex) {
    return fail(IMEX_ERR_ALLOC, std::string("host setup failed: ") + ex.what());
  }
}

int imex_host_setup_export(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src,
                           uint8_t* node_class, double* fx, imex_stats* stats) {
  try {
    Problem pb;
    if (int rc = build_context(mesh, p, alpha, dt, src, pb)) return rc;
    HostSetup hs;
    std::string err = build_setup(pb, hs);
    if (!err.empty()) return fail(setup_error_code(err), err);
    if (node_class) std::memcpy(node_class, hs.node_class.data(), hs.node_class.size());
    if (fx) std::memcpy(fx, hs.fx.data(), hs.fx.size() * sizeof(double));
    if (stats) fill_stats(hs, stats);
    log_setup(hs, "host");
    return IMEX_OK;
  } catch (const std::exception& ex) {
    return fail(IMEX_ERR_ALLOC, std::string("host setup failed: ") + ex.what());
  }
}

int imex_setup(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src,
               const imex_alloc* alloc, imex_ctx** out) {
  return imex_setup_batch(mesh, p, alpha, dt, src, 1, alloc, out);
}

int imex_setup_batch(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src, int ncols,
                     const imex_alloc* alloc, imex_ctx** out) {
  return imex_setup_scheme(mesh, p, alpha, dt, src, ncols, IMEX_SCHEME_IMEX, alloc, out);
}

static_assert(IMEX_SCHEME_IMEX == kSchemeImex && IMEX_SCHEME_CDM == kSchemeCdm &&
                  IMEX_SCHEME_CDM_HRZ == kSchemeCdmHrz && IMEX_SCHEME_TRAPEZOIDAL == kSchemeTrapezoidal,
              "scheme codes");

static int autotune_tile_steps(imex_ctx* c);

int imex_setup_scheme(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src, int ncols,
                      int scheme, const imex_alloc* alloc, imex_ctx** out) {
  int rc = setup_impl(mesh, p, alpha, dt, src, ncols, scheme, true, alloc, out);
  if (rc == IMEX_OK && (rc = autotune_tile_steps(*out)) != IMEX_OK) {
    imex_destroy(*out);
    *out = nullptr;
  }
  return rc;
}

int imex_setup_pcg(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src, int scheme,
                   const imex_alloc* alloc, imex_ctx** out) {
  if (scheme != IMEX_SCHEME_IMEX && scheme != IMEX_SCHEME_TRAPEZOIDAL)
    return fail(IMEX_ERR_ARG, "without a factorisation the scheme must be IMEX or trapezoidal");
  return setup_impl(mesh, p, alpha, dt, src, 1, scheme, false, alloc, out);
}

}  // extern "C"

namespace {

int setup_impl(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src, int ncols, int scheme,
               bool factorize, const imex_alloc* alloc, imex_ctx** out) {
  if (!out) return fail(IMEX_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  imex_ctx* c = nullptr;
  try {
    Problem pb;
    if (int rc = build_context(mesh, p, alpha, dt, src, pb)) return rc;
    if (ncols < 1 || ncols > kMaxCols) return fail(IMEX_ERR_ARG, "ncols must be in [1, 256]");
    if (ncols > 1 && ncols != pb.nsrc) return fail(IMEX_ERR_ARG, "ncols > 1 needs one source per column");
    if (scheme < IMEX_SCHEME_IMEX || scheme > IMEX_SCHEME_TRAPEZOIDAL) return fail(IMEX_ERR_ARG, "unknown scheme");
    pb.ncols = ncols;
    pb.scheme = scheme;
    pb.factorize = factorize;
    if (pb.dim == 3 && pb.p > 4) return fail(IMEX_ERR_ARG, "the 3D GPU time stepper supports p <= 4");
    c = new imex_ctx();
    c->ncols = ncols;
    std::string err = build_setup(pb, c->hs);
    if (!err.empty()) {
      delete c;
      return fail(setup_error_code(err), err);
    }
    HostSetup& hs = c->hs;
    if (hs.Pd > kMaxPd) {
      delete c;
      return fail(IMEX_ERR_ARG, "cell too large for the device right-hand side (P^d > 128)");
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
      delete c;
      return fail(IMEX_ERR_CUDA, "no CUDA device");
    }
    const int P = hs.P;
    c->TC = kTileLarge[P];
    const int OX = c->TC * hs.p;
    c->ntx = (hs.nn[0] + OX - 1) / OX;
    c->nty = (hs.nn[1] + OX - 1) / OX;
    c->smem_explicit = explicit_smem_doubles(P, c->TC) * sizeof(double);

    // Operators of the explicit apply: in 2D sx = rho c^2 h_y / h_x,
    // sy = rho c^2 h_x / h_y (|J| (2/h_d)^2 with |J| = h_x h_y / 4); in 3D
    // sx = rho c^2 h_y h_z / (2 h_x) and cyclic (|J| = h_x h_y h_z / 8).
    const double rc2 = pb.rho * pb.c0 * pb.c0;
    if (hs.dim == 2) {
      if (int rc = explicit_ops(hs, rc2 * hs.h[1] / hs.h[0], rc2 * hs.h[0] / hs.h[1], c->ops)) {
        delete c;
        return rc;
      }
      mass_scaled_ops(hs, hs.dt * hs.dt / (pb.rho * 0.25 * hs.h[0] * hs.h[1]), c->ops);
    } else {
      const double s3[3] = {0.5 * rc2 * hs.h[1] * hs.h[2] / hs.h[0], 0.5 * rc2 * hs.h[0] * hs.h[2] / hs.h[1],
                            0.5 * rc2 * hs.h[0] * hs.h[1] / hs.h[2]};
      if (int rc = explicit_ops3(hs, s3, c->ops3)) {
        delete c;
        return rc;
      }
    }
    c->hetero = pb.cell_c.empty() ? 0 : 1;   // per-cell speed: cell-by-cell explicit apply
    // Assembled GLL weights per node column/row; lumped mass = rho |J| W_x W_y.
    std::vector<double> wx(hs.nn[0]), wy(hs.nn[1]), wz(hs.dim == 3 ? hs.nn[2] : 1, 1.0);
    auto assembled = [&](int i, int n) {
      const int loc = i % hs.p;
      if (loc != 0) return hs.gll_w[loc];
      double w = 0.0;
      if (i > 0) w += hs.gll_w[hs.p];
      if (i < n - 1) w += hs.gll_w[0];
      return w;
    };
    if (hs.dim == 2) {
      const double jac = 0.25 * hs.h[0] * hs.h[1];
      for (int i = 0; i < hs.nn[0]; ++i) wx[i] = 1.0 / assembled(i, hs.nn[0]);
      for (int i = 0; i < hs.nn[1]; ++i) wy[i] = 1.0 / (assembled(i, hs.nn[1]) * pb.rho * jac);
    } else {
      const double jac = 0.125 * hs.h[0] * hs.h[1] * hs.h[2];
      for (int i = 0; i < hs.nn[0]; ++i) wx[i] = 1.0 / assembled(i, hs.nn[0]);
      for (int i = 0; i < hs.nn[1]; ++i) wy[i] = 1.0 / assembled(i, hs.nn[1]);
      for (int i = 0; i < hs.nn[2]; ++i) wz[i] = 1.0 / (assembled(i, hs.nn[2]) * pb.rho * jac);
    }

    // Compact per-c arrays and tree metadata.
    const int64_t nn = hs.nnodes, nc = hs.n_c, nt = (int64_t)hs.tree.size();
    const int ncols = c->ncols;
    std::vector<double> fxc((size_t)nc * ncols);
    for (int col = 0; col < ncols; ++col)
      for (int64_t r = 0; r < nc; ++r) fxc[(size_t)col * nc + r] = hs.fx[(size_t)col * nn + hs.c_node[r]];
    (void)nt;
    SolvePlan plan;
    std::vector<int> if_base_h, if_koff_h;
    if (factorize) {
      if (int rc = plan_solve(c, plan)) {
        delete c;
        return rc;
      }
    } else {   // no solve plan: the rows of the cell matrices and the pairs only
      if (int rc = interface_rows(hs, plan.Krows, plan.if_sc, if_base_h)) {
        delete c;
        return rc;
      }
      for (size_t e = 0; e < hs.if_cell.size(); ++e)
        if_koff_h.push_back(hs.if_kidx[e] >= 0 ? hs.if_kidx[e] : (int)hs.n_cut);
      if (if_koff_h.empty()) if_koff_h.push_back(0);
    }
    c->factorized = factorize ? 1 : 0;
    PcgPlan pp;
    if (int rc = plan_pcg(hs, pp)) {
      delete c;
      return rc;
    }
    c->g_nnz = (int64_t)pp.g_col.size();
    // Cell-by-cell K: every non-empty cell, and each node's cells.
    std::vector<int> hb, hk, hid, hptr, hcell, hloc;
    std::vector<double> hw, hc;
    {
      std::vector<int> cut_k(hs.ncell_total, -1);
      for (size_t e = 0; e < hs.if_cell.size(); ++e)
        if (hs.if_kidx[e] >= 0) cut_k[hs.if_cell[e]] = hs.if_kidx[e];
      const int ncx = pb.ncells[0], ncy = pb.ncells[1];
      std::vector<int> cnt(hs.nnodes + 1, 0);
      for (int cid = 0; cid < hs.ncell_total; ++cid) {
        if (hs.cell_type[cid] == CELL_EMPTY) continue;
        const int cx = cid % ncx, cy = (cid / ncx) % ncy, cz = cid / (ncx * ncy);
        hb.push_back(cx * hs.p + hs.nn[0] * cy * hs.p + hs.nn[0] * hs.nn[1] * cz * hs.p);
        const double ce = pb.cell_c.empty() ? pb.c0 : pb.cell_c[cid];
        if (hs.cell_type[cid] == CELL_CUT) {
          hk.push_back(cut_k[cid]);
          hw.push_back(1.0);
        } else {
          hk.push_back((int)hs.n_cut);
          hw.push_back((ce / pb.c0) * (ce / pb.c0));
        }
        hc.push_back(ce);
        hid.push_back(cid);
      }
      auto loc = [&](int m) {
        return (m % hs.P) + hs.nn[0] * ((m / hs.P) % hs.P) + hs.nn[0] * hs.nn[1] * (m / (hs.P * hs.P));
      };
      for (size_t e = 0; e < hb.size(); ++e)
        for (int l = 0; l < hs.Pd; ++l) cnt[hb[e] + loc(l) + 1]++;
      for (int64_t i = 0; i < hs.nnodes; ++i) cnt[i + 1] += cnt[i];
      hptr = cnt;
      hcell.assign(cnt[hs.nnodes], 0);
      hloc.assign(cnt[hs.nnodes], 0);
      std::vector<int> fill(cnt.begin(), cnt.end() - 1);
      for (size_t e = 0; e < hb.size(); ++e)
        for (int l = 0; l < hs.Pd; ++l) {
          const int node = hb[e] + loc(l);
          hcell[fill[node]] = (int)e;
          hloc[fill[node]++] = l;
        }
      for (int k : hk)
        if (k < 0) {
          delete c;
          return fail(IMEX_ERR_GEOM, "a cut cell without a stored matrix");
        }
      c->het_ncell = (int)hb.size();
    }
    {
      c->walk_max_slots = plan.max_slots;
      c->walk_max_m = plan.max_m;
      c->walk_max_pairs = plan.max_pairs;
      // Shared memory of a walk CTA: vectors and index lists always; the
      // cell-matrix rows of the pairs and the factor blocks when they fit
      // (otherwise they are read from global memory).
      const size_t kp = (size_t)(plan.max_kp + (plan.max_kp & 1)) * sizeof(double);
      const size_t blob = (size_t)plan.max_blob * sizeof(double);
      c->walk_vec = (size_t)(2 * plan.max_slots + plan.max_m + plan.max_pairs) * sizeof(double);
      const size_t base = c->walk_vec + (size_t)plan.max_ilist * sizeof(int);
      c->walk_kp_smem = base + kp <= kMaxDynSmem ? 1 : 0;
      c->walk_max_kp = c->walk_kp_smem ? (plan.max_kp + (plan.max_kp & 1)) : 0;
      const size_t used = base + (c->walk_kp_smem ? kp : 0);
      c->walk_smem_mode = used + blob <= kMaxDynSmem ? 1 : 0;
      c->walk_max_blob = c->walk_smem_mode ? plan.max_blob : 0;
      c->smem_walk = used + (c->walk_smem_mode ? blob : 0);
      c->smem_walk_req = c->smem_walk;
      c->walk_fixed = c->smem_walk - c->walk_vec;
      c->lev_has_nodes = plan.lev_has_nodes;
      c->top_max_zn = std::max(2, plan.max_zn + (plan.max_zn & 1));
      c->top_max_arows = plan.max_arows;
      c->smem_top = (size_t)(c->top_max_zn + plan.max_arows + kThreads) * sizeof(double) +
                    (size_t)plan.max_tlist * sizeof(int);
      c->top_vec = (size_t)(c->top_max_zn + kThreads) * sizeof(double);
      c->top_fixed = c->smem_top - c->top_vec;
      if (c->smem_walk > kMaxDynSmem || c->smem_top > kMaxDynSmem) {
        delete c;
        return fail(IMEX_ERR_ARG, "solve schedule exceeds the shared memory of a CTA");
      }
      c->n_large = plan.n_large;
      c->pan_cta0 = plan.pan_cta0;
      c->pan_ncta = plan.pan_ncta;
      c->pan_max_chunk = plan.pan_max_chunk;
      c->pan_max_nv = plan.pan_max_nv;
      c->smem_panel = (size_t)(plan.pan_max_chunk + plan.pan_max_nv + kThreads) * sizeof(double);
      if (c->smem_panel > kMaxDynSmem) {
        delete c;
        return fail(IMEX_ERR_ARG, "large-supernode chunk exceeds the shared memory of a CTA");
      }
      c->lev_cta0 = plan.lev_cta0;
      c->lev_ncta = plan.lev_ncta;
      c->ntop = (int)plan.top_comp.size();
      c->nzrow = (int64_t)plan.zrow.size();
    }
    const int64_t nif = (int64_t)hs.if_cell.size();
    const size_t nblobcta = std::max<size_t>(plan.blob_off.size(), 1);
    // Split explicit launch (2D tiles): per tile size, the tiles owning an
    // I_d node of an interface cell (the solve reads its u_pred) and the others.
    std::vector<int> tile_lists[2][2];   // [tile size][near, far]
    bool split_tiles = false;
    if (hs.dim == 2 && factorize && !c->hetero && hs.n_c > 0 && hs.n_d > 0) {
      std::vector<uint8_t> need(hs.nnodes, 0);
      const int ncx = hs.pb.ncells[0], nx = hs.nn[0], ny = hs.nn[1], p = hs.p;
      for (int cid : hs.if_cell) {
        const int cx = cid % ncx, cy = cid / ncx;
        for (int j = 0; j <= p; ++j)
          for (int i = 0; i <= p; ++i) {
            const int64_t g = (int64_t)(cy * p + j) * nx + cx * p + i;
            if (hs.node_class[g] == NODE_D) need[g] = 1;
          }
      }
      for (int v = 0; v < 2; ++v) {
        const int OX = (v ? kTileSmall[hs.P] : kTileLarge[hs.P]) * p;
        const int ntx = (nx + OX - 1) / OX, nty = (ny + OX - 1) / OX;
        for (int ty = 0; ty < nty; ++ty)
          for (int tx = 0; tx < ntx; ++tx) {
            bool near = false;
            for (int y = ty * OX; y < std::min(ny, ty * OX + OX) && !near; ++y)
              for (int x = tx * OX; x < std::min(nx, tx * OX + OX) && !near; ++x) near = need[(int64_t)y * nx + x];
            tile_lists[v][near ? 0 : 1].push_back(ty * ntx + tx);
          }
        c->n_near[v] = (int)tile_lists[v][0].size();
        c->n_far[v] = (int)tile_lists[v][1].size();
      }
      split_tiles = c->n_far[0] > 0 && c->n_far[1] > 0;
    }

    Arena ar;
    ar.add(&c->U[0], nn * ncols);
    ar.add(&c->U[1], nn * ncols);
    ar.add(&c->tmp, nn * ncols);
    ar.add(&c->fx, nn * ncols);
    ar.add(&c->fxs, hs.dim == 2 ? nn * ncols : 1);
    ar.add(&c->winv_x, hs.nn[0]);
    ar.add(&c->winv_y, hs.nn[1]);
    ar.add(&c->winv_z, wz.size());
    ar.add(&c->cls, nn);
    ar.add(&c->c_node, std::max<int64_t>(nc, 1));
    ar.add(&c->v_c, std::max<int64_t>(nc, 1) * ncols);
    ar.add(&c->a_c, std::max<int64_t>(nc, 1) * ncols);
    ar.add(&c->fxc, std::max<int64_t>(nc, 1) * ncols);
    ar.add(&c->sol, std::max<int64_t>(nc, 1) * ncols);
    ar.add(&c->rhs0, std::max<int64_t>(nc, 1) * ncols);
    ar.add(&c->upd, std::max<int64_t>(hs.upd_size, 1) * ncols);
    ar.add(&c->hbuf, std::max<int64_t>(nc, 1) * ncols);
    ar.add(&c->pan_desc, std::max<size_t>(plan.pan_desc.size(), 8));
    ar.add(&c->pan_idx, std::max<size_t>(plan.pan_idx.size(), 4));
    ar.add(&c->pan_aoff, std::max<size_t>(plan.pan_aoff.size(), 1));
    ar.add(&c->panS, std::max<size_t>(plan.panS.size(), 2));
    ar.add(&c->panM, std::max<size_t>(plan.panM.size(), 2));
    ar.add(&c->Kpair, std::max<size_t>(plan.Kpair.size(), 2));
    ar.add(&c->kp_off, nblobcta);
    ar.add(&c->kp_len, nblobcta);
    ar.add(&c->blob_S, std::max<size_t>(plan.blobS.size(), 2));
    ar.add(&c->blob_M, std::max<size_t>(plan.blobM.size(), 2));
    ar.add(&c->blob_off, nblobcta);
    ar.add(&c->blob_len, nblobcta);
    ar.add(&c->ilist, std::max<size_t>(plan.ilist.size(), 4));
    ar.add(&c->ilist_off, nblobcta);
    ar.add(&c->ilist_len, nblobcta);
    ar.add(&c->tlist, std::max<size_t>(plan.tlist.size(), 4));
    ar.add(&c->tlist_off, std::max<size_t>(plan.tlist_off.size(), 1));
    ar.add(&c->tlist_len, std::max<size_t>(plan.tlist_len.size(), 1));
    ar.add(&c->top_comp, std::max<size_t>(plan.top_comp.size(), 1));
    ar.add(&c->top_r0, std::max<size_t>(plan.top_r0.size(), 1));
    ar.add(&c->top_r1, std::max<size_t>(plan.top_r1.size(), 1));
    ar.add(&c->zsize, std::max<size_t>(plan.zsize.size(), 1));
    ar.add(&c->zbase, std::max<size_t>(plan.zbase.size(), 1));
    ar.add(&c->zrow, std::max<size_t>(plan.zrow.size(), 1));
    ar.add(&c->zA_off, std::max<size_t>(plan.zA_off.size(), 1));
    ar.add(&c->zA_S, std::max<size_t>(plan.zA_S.size(), 1));
    ar.add(&c->zA_M, std::max<size_t>(plan.zA_M.size(), 1));
    for (int v = 0; v < 2; ++v) {
      ar.add(&c->tile_near[v], std::max<size_t>(tile_lists[v][0].size(), 1));
      ar.add(&c->tile_far[v], std::max<size_t>(tile_lists[v][1].size(), 1));
    }
    {
      const int64_t ncm = std::max<int64_t>(nc, 1), gnz = std::max<int64_t>(c->g_nnz, 1);
      ar.add(&c->s_ptr, hs.S_ptr.size());
      ar.add(&c->s_col, std::max<size_t>(hs.S_col.size(), 1));
      ar.add(&c->s_val, std::max<size_t>(hs.S_val.size(), 1));
      ar.add(&c->g_ptr, pp.g_ptr.size());
      ar.add(&c->g_col, gnz);
      ar.add(&c->gt_ptr, ncm + 1);
      ar.add(&c->gt_row, gnz);
      ar.add(&c->gt_idx, gnz);
      ar.add(&c->g_val, gnz);
      ar.add(&c->gt_val, gnz);
      ar.add(&c->g_scale, gnz);
      ar.add(&c->g_theta, gnz);
      ar.add(&c->g_m, gnz);
      ar.add(&c->g_v, gnz);
      ar.add(&c->g_grad, gnz);
      ar.add(&c->g_sg, gnz);
      ar.add(&c->g_isdiag, gnz);
      ar.add(&c->dinv, ncm);
      for (double** v : {&c->pcg_x, &c->pcg_r, &c->pcg_z, &c->pcg_p, &c->pcg_q, &c->pcg_w, &c->pcg_v}) ar.add(v, ncm);
      ar.add(&c->pcg_part, 10 * std::max<int64_t>(1024, (ncm + kThreads - 1) / kThreads));
      ar.add(&c->pcg_hist, 2 * ncm);
      ar.add(&c->guess_state, 16);
      ar.add(&c->pcg_res, 2);
      ar.add(&c->pcg_status, 4);
      ar.add(&c->pcg_counters, 2);
    }
    ar.add(&c->het_base, std::max<size_t>(hb.size(), 1));
    ar.add(&c->het_koff, std::max<size_t>(hk.size(), 1));
    ar.add(&c->het_id, std::max<size_t>(hid.size(), 1));
    ar.add(&c->het_w, std::max<size_t>(hw.size(), 1));
    ar.add(&c->het_c, std::max<size_t>(hc.size(), 1));
    ar.add(&c->het_ptr, hptr.size());
    ar.add(&c->het_cell, std::max<size_t>(hcell.size(), 1));
    ar.add(&c->het_local, std::max<size_t>(hloc.size(), 1));
    ar.add(&c->Kall, std::max<size_t>(plan.Krows.size(), 1));
    ar.add(&c->node_c_dev, std::max<int64_t>(nn, 1));
    {
      const bool nf = !factorize;
      ar.add(&c->m_val, nf ? std::max<size_t>(hs.M_val.size(), 1) : 1);
      ar.add(&c->dinv_m, nf ? std::max<int64_t>(nc, 1) : 1);
      ar.add(&c->pr_ptr, nf ? hs.contrib_ptr.size() : 1);
      ar.add(&c->pr_pos, nf ? std::max<size_t>(hs.contrib_pos.size(), 1) : 1);
      ar.add(&c->if_base_dev, nf ? if_base_h.size() : 1);
      ar.add(&c->if_koff_dev, nf ? if_koff_h.size() : 1);
      ar.add(&c->if_sc_dev, nf ? plan.if_sc.size() : 1);
    }
    ar.add(&c->ft_buf, 2 * kIoRing);
    ar.add(&c->rec_buf, (size_t)kIoRing * c->io_cap * ncols);
    ar.add(&c->rec_nodes, c->io_cap);
    c->bytes = ar.total();
    void* basep = nullptr;
    if (alloc && alloc->alloc) {
      c->hooks = *alloc;
      c->has_hooks = true;
      basep = alloc->alloc(c->bytes, alloc->user);
      if (!basep) {
        delete c;
        return fail(IMEX_ERR_ALLOC, "allocator hook returned NULL");
      }
    } else if (cudaMalloc(&basep, c->bytes) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return fail(IMEX_ERR_ALLOC, "cudaMalloc of the device state failed");
    }
    c->base = (char*)basep;
    ar.assign(c->base);

    cudaError_t e = cudaMemset(c->base, 0, c->bytes);
    e = e ? e : upload(c->fx, hs.fx);
    if (hs.dim == 2) {   // dt^2 M^{-1} f_x with the per-axis inverse lumped weights
      std::vector<double> fxs(hs.fx.size());
      const double dt2 = hs.dt * hs.dt;
      for (size_t g = 0; g < fxs.size(); ++g) {
        const int64_t gl = (int64_t)(g % (size_t)nn);
        const int gx = (int)(gl % hs.nn[0]), gy = (int)(gl / hs.nn[0]);
        fxs[g] = dt2 * (wx[gx] * wy[gy]) * hs.fx[g];
      }
      e = e ? e : upload(c->fxs, fxs);
    }
    e = e ? e : upload(c->winv_x, wx);
    e = e ? e : upload(c->winv_y, wy);
    e = e ? e : upload(c->winv_z, wz);
    e = e ? e : upload(c->cls, hs.node_class);
    e = e ? e : upload(c->c_node, hs.c_node);
    e = e ? e : upload(c->fxc, fxc);
    e = e ? e : upload(c->s_ptr, hs.S_ptr);
    e = e ? e : upload(c->s_col, hs.S_col);
    e = e ? e : upload(c->s_val, hs.S_val);
    e = e ? e : upload(c->g_ptr, pp.g_ptr);
    e = e ? e : upload(c->g_col, pp.g_col);
    e = e ? e : upload(c->gt_ptr, pp.gt_ptr);
    e = e ? e : upload(c->gt_row, pp.gt_row);
    e = e ? e : upload(c->gt_idx, pp.gt_idx);
    e = e ? e : upload(c->g_val, pp.g_val);
    {
      std::vector<double> gtv(pp.gt_idx.size());
      for (size_t k = 0; k < gtv.size(); ++k) gtv[k] = pp.g_val[pp.gt_idx[k]];
      e = e ? e : upload(c->gt_val, gtv);
    }
    e = e ? e : upload(c->g_scale, pp.g_scale);
    e = e ? e : upload(c->g_theta, pp.g_theta);
    e = e ? e : upload(c->g_isdiag, pp.g_isdiag);
    e = e ? e : upload(c->dinv, pp.dinv);
    if (e == cudaSuccess) {
      // Lanes per sparse row: about six entries of a mean row of S per lane
      // (4 .. 32, a power of two).  Grid: small partitions one CTA per SM
      // (the grid barriers grow with the CTAs: on the 256x128 plate, 8 lanes
      // per row and one CTA per SM took 58 us per FSAI iteration, four CTAs
      // per SM 78 us, 32 lanes 101 us); large ones (3D) every co-resident
      // CTA; never more CTAs than the rows fill.
      const double avg = hs.n_c > 0 ? (double)hs.S_ptr[hs.n_c] / (double)hs.n_c : 1.0;
      c->pcg_lpr = 4;
      while (c->pcg_lpr < 32 && c->pcg_lpr * 6 < avg) c->pcg_lpr *= 2;
      int occ = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_kernel(c->pcg_lpr), kThreads, 0);
      int nsm = 0;
      e = e ? e : cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
      const int64_t rows_per_cta = (int64_t)kWarps * (32 / c->pcg_lpr);
      const int64_t rows_ctas = std::max<int64_t>(1, (hs.n_c + rows_per_cta - 1) / rows_per_cta);
      const int64_t cap = hs.n_c >= 65536 ? (int64_t)nsm * occ : nsm;
      c->pcg_grid = (int)std::max<int64_t>(1, std::min<int64_t>({cap, (int64_t)nsm * occ, 1024, rows_ctas}));
    }
    e = e ? e : upload(c->het_base, hb);
    e = e ? e : upload(c->het_koff, hk);
    e = e ? e : upload(c->het_id, hid);
    e = e ? e : upload(c->het_w, hw);
    e = e ? e : upload(c->het_c, hc);
    e = e ? e : upload(c->het_ptr, hptr);
    e = e ? e : upload(c->het_cell, hcell);
    e = e ? e : upload(c->het_local, hloc);
    e = e ? e : upload(c->Kall, plan.Krows);
    e = e ? e : upload(c->node_c_dev, hs.node_c);
    if (!factorize && e == cudaSuccess) {
      std::vector<double> dm(std::max<int64_t>(nc, 1), 0.0);
      for (int64_t r = 0; r < nc; ++r)
        for (int k = hs.S_ptr[r]; k < hs.S_ptr[r + 1]; ++k)
          if (hs.S_col[k] == r) dm[r] = 1.0 / hs.M_val[k];
      e = upload(c->m_val, hs.M_val);
      e = e ? e : upload(c->dinv_m, dm);
      e = e ? e : upload(c->pr_ptr, hs.contrib_ptr);
      e = e ? e : upload(c->pr_pos, hs.contrib_pos);
      e = e ? e : upload(c->if_base_dev, if_base_h);
      e = e ? e : upload(c->if_koff_dev, if_koff_h);
      e = e ? e : upload(c->if_sc_dev, plan.if_sc);
      c->solver = IMEX_SOLVER_PCG_JACOBI;
      c->pcg_maxit = 5000;
    }
    e = e ? e : upload(c->Kpair, plan.Kpair);
    e = e ? e : upload(c->kp_off, plan.kp_off);
    e = e ? e : upload(c->kp_len, plan.kp_len);
    e = e ? e : upload(c->blob_S, plan.blobS);
    e = e ? e : upload(c->blob_M, plan.blobM);
    e = e ? e : upload(c->blob_off, plan.blob_off);
    e = e ? e : upload(c->blob_len, plan.blob_len);
    e = e ? e : upload(c->ilist, plan.ilist);
    e = e ? e : upload(c->ilist_off, plan.ilist_off);
    e = e ? e : upload(c->ilist_len, plan.ilist_len);
    e = e ? e : upload(c->tlist, plan.tlist);
    e = e ? e : upload(c->tlist_off, plan.tlist_off);
    e = e ? e : upload(c->tlist_len, plan.tlist_len);
    e = e ? e : upload(c->top_comp, plan.top_comp);
    e = e ? e : upload(c->top_r0, plan.top_r0);
    e = e ? e : upload(c->top_r1, plan.top_r1);
    e = e ? e : upload(c->zsize, plan.zsize);
    e = e ? e : upload(c->zbase, plan.zbase);
    e = e ? e : upload(c->zrow, plan.zrow);
    e = e ? e : upload(c->zA_off, plan.zA_off);
    e = e ? e : upload(c->zA_S, plan.zA_S);
    e = e ? e : upload(c->zA_M, plan.zA_M);
    e = e ? e : upload(c->pan_desc, plan.pan_desc);
    e = e ? e : upload(c->pan_idx, plan.pan_idx);
    e = e ? e : upload(c->pan_aoff, plan.pan_aoff);
    e = e ? e : upload(c->panS, plan.panS);
    e = e ? e : upload(c->panM, plan.panM);
    for (int v = 0; v < 2; ++v) {
      e = e ? e : upload(c->tile_near[v], tile_lists[v][0]);
      e = e ? e : upload(c->tile_far[v], tile_lists[v][1]);
    }
    for (int k = 0; k < 8 && e == cudaSuccess; ++k)
      e = cudaFuncSetAttribute(walk_kernel(k & 1, k & 2, k & 4), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kMaxDynSmem);
    for (auto fn : {k_top<true>, k_top<false>})
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    if (e == cudaSuccess) {
      int nsm = 0;
      e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
      c->num_sms = std::max(1, nsm);
    }
    // The side stream and events of the split explicit launch.
    if (e == cudaSuccess && split_tiles) {
      int lo = 0, hi = 0;
      e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
      e = e ? e : cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, lo);
      e = e ? e : cudaEventCreateWithFlags(&c->ov_fork, cudaEventDisableTiming);
      e = e ? e : cudaEventCreateWithFlags(&c->ov_join, cudaEventDisableTiming);
      c->split_ok = e == cudaSuccess ? 1 : 0;
    }
    e = e ? e : (c->hetero ? use_explicit(c, 0) : autotune_tile(c));
    if (e != cudaSuccess) {
      std::string msg = std::string("upload failed: ") + cudaGetErrorString(e);
      imex_destroy(c);
      return fail(IMEX_ERR_CUDA, msg);
    }
    c->cur = 0;
    c->step = 0;
    // u_0 = 0, v_0 = 0 (tmp is zero after the memset).
    if (int rc = compute_initial(c, nullptr)) {
      imex_destroy(c);
      return rc;
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      std::string msg = std::string("initial state: ") + cudaGetErrorString(e);
      imex_destroy(c);
      return fail(IMEX_ERR_CUDA, msg);
    }
    log_setup(c->hs, "device");
    *out = c;
    return IMEX_OK;
  } catch (const std::exception& ex) {
    delete c;
    return fail(IMEX_ERR_ALLOC, std::string("setup failed: ") + ex.what());
  }
}

}  // namespace

extern "C" {

// CTAs of an explicit launch that only predicts (no explicit DOFs).
int pred_only_blocks(const imex_ctx* c) {
  const int64_t nb = (c->hs.n_c + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(nb, 4LL * std::max(1, c->num_sms)));
}

// One step n -> n+1 on stream s; events (may be NULL) are recorded before
// the explicit kernel, after it, and after the implicit chain.  Scratch
// (upd, sol, rhs0) of the factorised solve defaults to the context's own
// (imex_step_noalloc passes its fixed array and accepts direct-solver
// contexts only).
//   IMEX / trapezoidal: diagonal CDM step on I_d with the prediction of I_c,
//     then S a^c_{n+1} = f_t(t_{n+1}) f^c - K^c u_pred and the correction.
//   Central differences (consistent or HRZ mass): the same explicit kernel
//     without prediction, then M^cc a^c_n = f_t(t_n) f^c - K^c u_n and
//     u^c_{n+1} = 2 u^c_n - u^c_{n-1} + dt^2 a^c_n (Eqs. CDMstep, CDMacc).
static int step_once(imex_ctx* c, cudaStream_t s, cudaEvent_t* ev, const double* ft_dev = nullptr,
                     double* upd = nullptr, double* sol = nullptr, double* rhs0 = nullptr, double* hbuf = nullptr) {
  const HostSetup& hs = c->hs;
  const bool own = upd == nullptr;
  if (own) {
    upd = c->upd;
    sol = c->sol;
    rhs0 = c->rhs0;
    hbuf = c->hbuf;
  }
  const double dt = hs.dt;
  double* Ucur = c->U[c->cur];
  double* Unext = c->U[1 - c->cur];
  const int64_t step = c->step;
  const bool cdm = scheme_is_cdm(hs.pb.scheme);
  if (ev) cudaEventRecord(ev[0], s);
  ExplicitArgs ea = explicit_args(c, Ucur, Unext, Unext, 2.0, -1.0, dt * dt, ft_at(hs, step), !cdm);
  ea.ft_dev = ft_dev;
  int grid = ntiles(c) + pred_blocks(c, !cdm);
  if (hs.n_d == 0 && !c->hetero) {   // no explicit DOFs: prediction CTAs only
    ea.ntx = ea.nty = ea.ntz = 0;
    grid = pred_only_blocks(c);
  }
  // Split launch (2D tiles, IMEX scheme, direct solve, not in a per-phase
  // timing): the tiles owning I_d nodes of interface cells, and the
  // prediction, on s; the other tiles on the side stream, beside the solve.
  // Neither half reads what the other writes (owned nodes are disjoint; both
  // read u_n, which nothing writes during the step); the solve reads only the
  // first half's nodes (u_pred of the interface cells) and writes only I_c
  // rows, which the second half neither reads nor writes; the step ends on s
  // once both streams have.
  const bool split = split_active(c) && !cdm && !ev;
  if (split) {
    const int v = c->xvar;
    cudaEventRecord(c->ov_fork, s);
    ExplicitArgs en = ea;
    en.tiles = c->tile_near[v];
    en.ntl = c->n_near[v];
    const int npred = (int)std::max<int64_t>(1, std::min<int64_t>((hs.n_c + kThreads - 1) / kThreads, c->num_sms));
    explicit_dispatch(c, en, en.ntl + npred, s);
    cudaStreamWaitEvent(c->side, c->ov_fork, 0);
    ExplicitArgs ef = ea;
    ef.tiles = c->tile_far[v];
    ef.ntl = c->n_far[v];
    ef.persistent = 1;
    ef.n_c = 0;
    explicit_dispatch(c, ef, (int)std::min<int64_t>((int64_t)ef.ntl * c->ncols, (int64_t)c->num_sms * c->split_per_sm),
                      c->side);
    cudaEventRecord(c->ov_join, c->side);
  } else {
    explicit_dispatch(c, ea, grid, s);
  }
  if (ev) cudaEventRecord(ev[1], s);
  if (hs.n_c > 0) {
    if (!c->factorized) {   // right-hand sides, then PCG with the correction
      launch_rhs_c(c, ft_at(hs, step + 1), Unext, s, ft_dev);
      if (cudaError_t e = launch_pcg(c, Unext, s))
        return fail(IMEX_ERR_CUDA, std::string("imex_step: PCG launch: ") + cudaGetErrorString(e));
      ++c->guess_valid;
    } else if (cdm) {
      launch_solve_chain(c, false, ft_at(hs, step), ft_dev, 3, Unext, Ucur, upd, sol, rhs0, hbuf, s);
    } else if (c->solver == IMEX_SOLVER_DIRECT) {
      launch_solve_chain(c, true, ft_at(hs, step + 1), ft_dev, 0, Unext, Unext, upd, sol, rhs0, hbuf, s);
      c->guess_valid = 0;   // the PCG history is not advanced by the direct solve
    } else {
      // Right-hand sides, PCG (correction included on convergence), then the
      // direct solve, whose launches return at once unless PCG fell short.
      launch_solve_chain(c, true, ft_at(hs, step + 1), ft_dev, 0, Unext, Unext, upd, sol, rhs0, hbuf, s,
                         nullptr, true);
      if (cudaError_t e = launch_pcg(c, Unext, s))
        return fail(IMEX_ERR_CUDA, std::string("imex_step: PCG launch: ") + cudaGetErrorString(e));
      launch_solve_chain(c, true, ft_at(hs, step + 1), ft_dev, 0, Unext, Unext, upd, sol, rhs0, hbuf, s,
                         c->pcg_status + 1);
      ++c->guess_valid;
    }
  }
  if (split) cudaStreamWaitEvent(s, c->ov_join, 0);
  if (ev) cudaEventRecord(ev[2], s);
  if (int rc = check_launch("imex_step")) return rc;
  c->cur = 1 - c->cur;
  c->step = step + 1;
  return IMEX_OK;
}

// Tile choice of a factorised context with implicit DOFs, by whole steps: the
// solve chain's first launch stages its constants while the tail of the
// explicit kernel runs, so the tile that makes the explicit kernel fastest
// alone is not the one that makes the step fastest (on the 256x128 plate,
// p = 4: 8-cell tiles 80.8 us per step, 4-cell tiles 89.6, although the
// 4-cell kernel alone can time faster).  Four steps with each tile after one
// warm-up step; the state (both field buffers, v^c, a^c, the step counter) is
// saved before and restored after.  IMEX_EXPLICIT_TILE = large | small keeps
// the forced tile.
static int autotune_tile_steps(imex_ctx* c) {
  const HostSetup& hs = c->hs;
  if (c->hetero || !c->factorized || hs.n_c == 0) return IMEX_OK;
  const bool pinned = explicit_env_variant(c) >= 0;
  const size_t nn = (size_t)hs.nnodes * c->ncols, ncv = (size_t)hs.n_c * c->ncols;
  double* save = nullptr;
  if (cudaMalloc(&save, (2 * nn + 2 * ncv) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(IMEX_ERR_ALLOC, "tile tuning: device buffer");
  }
  double* const dst[4] = {save, save + nn, save + 2 * nn, save + 2 * nn + ncv};
  double* const src[4] = {c->U[0], c->U[1], c->v_c, c->a_c};
  const size_t len[4] = {nn, nn, ncv, ncv};
  const int cur0 = c->cur;
  const int64_t step0 = c->step;
  auto copy_state = [&](bool to_save) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
      e = to_save ? cudaMemcpy(dst[k], src[k], len[k] * sizeof(double), cudaMemcpyDeviceToDevice)
                  : cudaMemcpy(src[k], dst[k], len[k] * sizeof(double), cudaMemcpyDeviceToDevice);
    c->cur = cur0;
    c->step = step0;
    return e;
  };
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = copy_state(true);
  e = e ? e : cudaEventCreate(&ev[0]);
  e = e ? e : cudaEventCreate(&ev[1]);
  // One untimed and four timed whole steps from the saved state.
  auto time_steps = [&](float* us) {
    e = copy_state(false);
    if (e != cudaSuccess) return IMEX_OK;
    int r = step_once(c, nullptr, nullptr);
    e = cudaEventRecord(ev[0], nullptr);
    for (int k = 0; k < 4 && r == IMEX_OK && e == cudaSuccess; ++k) r = step_once(c, nullptr, nullptr);
    e = e ? e : cudaEventRecord(ev[1], nullptr);
    e = e ? e : cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    e = e ? e : cudaEventElapsedTime(&ms, ev[0], ev[1]);
    *us = 1e3f * ms / 4.f;
    return r;
  };
  int rc = IMEX_OK;
  // Independent columns per walk / dense-top CTA (1, 2, 4, ..., 64), with the
  // explicit variant chosen so far.
  if (c->ncols > 1 && e == cudaSuccess) {
    if (int pin = col_block_env()) {
      set_col_block(c, pin);
    } else {
      float bbest = 1e30f;
      int bcb = 1;
      for (int k = 0; k < 7 && e == cudaSuccess && rc == IMEX_OK; ++k) {
        const int cb = 1 << k;
        if (cb > c->ncols || !set_col_block(c, cb)) continue;
        rc = time_steps(&c->cb_us[k]);
        if (e == cudaSuccess && rc == IMEX_OK && c->cb_us[k] < bbest) {
          bbest = c->cb_us[k];
          bcb = cb;
        }
      }
      set_col_block(c, bcb);
    }
  }
  // Candidates: every explicit variant (or the pinned one) with each shared
  // memory request of the walk launches: what the walk needs, or enough that
  // fewer CTAs of other launches share its SM (140 and 184 KB).  A larger
  // request changes which CTAs of neighbouring launches (the explicit
  // tiles, the dense tops, the split launch's second half) can be resident
  // beside a walk CTA.  One untimed and four timed whole steps each, from
  // the saved state; the fastest pair is kept.
  const size_t wreq[3] = {c->smem_walk, std::max<size_t>(c->smem_walk, 140 * 1024),
                          std::max<size_t>(c->smem_walk, 184 * 1024)};
  float best = 1e30f;
  int best_var = c->xvar + (c->xsplit ? kExplicitSplit + split_index(c) : 0);
  size_t best_req = c->smem_walk;
  for (int k = 0; k < explicit_variants(c) && e == cudaSuccess && rc == IMEX_OK; ++k) {
    if (pinned && k != explicit_env_variant(c)) continue;
    e = use_explicit(c, k);
    if (e != cudaSuccess) break;
    float kbest = 1e30f;
    for (int w = 0; w < 3 && e == cudaSuccess && rc == IMEX_OK; ++w) {
      if (wreq[w] > kMaxDynSmem || (w > 0 && wreq[w] == wreq[w - 1])) continue;
      c->smem_walk_req = wreq[w];
      float us = 0.f;
      rc = time_steps(&us);
      if (e != cudaSuccess) break;
      kbest = std::min(kbest, us);
      if (us < best) {
        best = us;
        best_var = k;
        best_req = wreq[w];
      }
    }
    c->tile_us[k] = kbest < 1e30f ? kbest : 0.f;
  }
  e = e ? e : use_explicit(c, best_var);
  c->smem_walk_req = best_req;
  // The column block was tuned with the explicit variant chosen before; with
  // the final variant and walk request, the neighbouring block sizes are
  // timed once more and the fastest kept.
  if (c->ncols > 1 && !col_block_env() && e == cudaSuccess && rc == IMEX_OK) {
    const int cb0 = c->col_block;
    float bbest = best;
    int bcb = cb0;
    for (int cb : {cb0 / 2, cb0 * 2}) {
      if (cb < 1 || cb > c->ncols || !set_col_block(c, cb)) continue;
      c->smem_walk_req = std::max(c->smem_walk, best_req);
      float us = 0.f;
      rc = time_steps(&us);
      if (e != cudaSuccess || rc != IMEX_OK) break;
      for (int k = 0; k < 7; ++k)
        if ((1 << k) == cb) c->cb_us[k] = us;
      if (us < bbest) {
        bbest = us;
        bcb = cb;
      }
    }
    set_col_block(c, bcb);
    c->smem_walk_req = std::max(c->smem_walk, best_req);
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  e = e ? e : copy_state(false);
  e = e ? e : cudaDeviceSynchronize();
  cudaFree(save);
  if (rc != IMEX_OK) return rc;
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("tile tuning: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_step(imex_ctx* c, int64_t n, void* stream) {
  if (!c || n < 0) return fail(IMEX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->stream = s;
  for (int64_t k = 0; k < n; ++k)
    if (int rc = step_once(c, s, nullptr)) return rc;
  return IMEX_OK;
}

int imex_step_profile(imex_ctx* c, int64_t n, void* stream, double* phase_ms) {
  if (!c || n < 0 || !phase_ms) return fail(IMEX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->stream = s;
  cudaEvent_t ev[3];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(IMEX_ERR_CUDA, "cudaEventCreate failed");
  // explicit apply, implicit chain, whole step
  const int from[IMEX_PROFILE_PHASES] = {0, 1, 0}, to[IMEX_PROFILE_PHASES] = {1, 2, 2};
  double acc[IMEX_PROFILE_PHASES] = {0, 0, 0};
  int rc = IMEX_OK;
  for (int64_t k = 0; k < n && rc == IMEX_OK; ++k) {
    rc = step_once(c, s, ev);
    if (rc) break;
    if (cudaEventSynchronize(ev[2]) != cudaSuccess) {
      rc = fail(IMEX_ERR_CUDA, "imex_step_profile: synchronisation failed");
      break;
    }
    for (int ph = 0; ph < IMEX_PROFILE_PHASES; ++ph) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[from[ph]], ev[to[ph]]);
      acc[ph] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (int ph = 0; ph < IMEX_PROFILE_PHASES; ++ph) phase_ms[ph] = acc[ph];
  return rc;
}

int imex_step_io(imex_ctx* c, int64_t n, const double* ft_samples, const int64_t* rec_nodes, int nrec,
                 double* traces, void* stream) {
  if (!c || n < 0 || nrec < 0 || (nrec > 0 && (!rec_nodes || !traces)))
    return fail(IMEX_ERR_ARG, "bad arguments");
  if (nrec > c->io_cap) return fail(IMEX_ERR_ARG, "too many receivers (max 4096)");
  for (int k = 0; k < nrec; ++k)
    if (rec_nodes[k] < 0 || rec_nodes[k] >= c->hs.nnodes) return fail(IMEX_ERR_ARG, "receiver node out of range");
  cudaStream_t s = (cudaStream_t)stream;
  c->stream = s;
  cudaError_t e = cudaSuccess;
  // Copies run on two streams of their own so that the step kernels do not
  // wait for them: the source samples of step k go into ring slot k % kIoRing
  // ahead of the step (the slot is reused once step k - kIoRing has run), the
  // receiver values of step k are gathered into a ring slot on the compute
  // stream and copied out behind an event (the slot is reused once that copy
  // is done).  Every step still copies its own inputs in and results out.
  if (!c->io_h2d) {
    e = cudaStreamCreateWithFlags(&c->io_h2d, cudaStreamNonBlocking);
    e = e ? e : cudaStreamCreateWithFlags(&c->io_d2h, cudaStreamNonBlocking);
    for (auto& row : c->io_ev)
      for (cudaEvent_t& ev : row)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_step_io: ") + cudaGetErrorString(e));
  }
  if (nrec > 0) e = cudaMemcpyAsync(c->rec_nodes, rec_nodes, nrec * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  const size_t slot_len = (size_t)c->io_cap * c->ncols, rec_len = (size_t)nrec * c->ncols;
  for (int64_t k = 0; k < n && e == cudaSuccess; ++k) {
    const int j = (int)(k % kIoRing);
    const double* ftd = nullptr;
    if (ft_samples) {
      if (k >= kIoRing) e = cudaStreamWaitEvent(c->io_h2d, c->io_ev[1][j], 0);
      e = e ? e : cudaMemcpyAsync(c->ft_buf + 2 * j, ft_samples + k, 2 * sizeof(double), cudaMemcpyHostToDevice,
                                  c->io_h2d);
      e = e ? e : cudaEventRecord(c->io_ev[0][j], c->io_h2d);
      e = e ? e : cudaStreamWaitEvent(s, c->io_ev[0][j], 0);
      if (e != cudaSuccess) break;
      ftd = c->ft_buf + 2 * j;
    }
    if (int rc = step_once(c, s, nullptr, ftd)) return rc;
    double* slot = c->rec_buf + (size_t)j * slot_len;
    if (nrec > 0) {
      if (k >= kIoRing) e = cudaStreamWaitEvent(s, c->io_ev[2][j], 0);
      for (int col = 0; col < c->ncols; ++col)
        k_gather_nodes<<<(nrec + 255) / 256, 256, 0, s>>>(slot + (size_t)col * nrec,
                                                          c->U[c->cur] + (size_t)col * c->hs.nnodes, c->rec_nodes, nrec);
    }
    e = e ? e : cudaEventRecord(c->io_ev[1][j], s);
    if (nrec > 0) {
      e = e ? e : cudaStreamWaitEvent(c->io_d2h, c->io_ev[1][j], 0);
      e = e ? e : cudaMemcpyAsync(traces + k * rec_len, slot, rec_len * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->io_d2h);
      e = e ? e : cudaEventRecord(c->io_ev[2][j], c->io_d2h);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->io_h2d);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->io_d2h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_step_io: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

static int field_io_check(imex_ctx* c, int64_t len) {
  if (!c) return fail(IMEX_ERR_ARG, "NULL context");
  if (len != c->hs.nnodes * c->ncols) return fail(IMEX_ERR_ARG, "len must equal ncols * n_nodes");
  return IMEX_OK;
}

int imex_fields(imex_ctx* c, int which, double* dst, int64_t len, int dst_on_device) {
  if (int rc = field_io_check(c, len)) return rc;
  if (!dst) return fail(IMEX_ERR_ARG, "NULL destination");
  cudaStream_t s = c->stream;
  const int64_t n = c->hs.nnodes;
  const int nb = (int)((n + 255) / 256);
  const int nc = (int)c->hs.n_c;
  for (int col = 0; col < c->ncols; ++col) {
    const int64_t on = (int64_t)col * n, oc = (int64_t)col * nc;
    double* out = c->tmp + on;
    switch (which) {
      case IMEX_FIELD_U: k_masked<<<nb, 256, 0, s>>>(out, c->U[c->cur] + on, c->cls, n, 3); break;
      case IMEX_FIELD_U_PREV_D:   // u_{n-1} on I_d; on every active DOF for central differences
        k_masked<<<nb, 256, 0, s>>>(out, c->U[1 - c->cur] + on, c->cls, n, scheme_is_cdm(c->hs.pb.scheme) ? 3 : 1);
        break;
      case IMEX_FIELD_V_C:
      case IMEX_FIELD_A_C:
        cudaMemsetAsync(out, 0, n * sizeof(double), s);
        if (nc > 0)
          k_scatter_c<<<(nc + 255) / 256, 256, 0, s>>>(out, (which == IMEX_FIELD_V_C ? c->v_c : c->a_c) + oc,
                                                       c->c_node, nc);
        break;
      case IMEX_FIELD_FX: k_masked<<<nb, 256, 0, s>>>(out, c->fx + on, c->cls, n, 3); break;
      case IMEX_FIELD_MASK_D: k_masked<<<nb, 256, 0, s>>>(out, c->fx, c->cls, n, 4); break;
      case IMEX_FIELD_MASK_C: k_masked<<<nb, 256, 0, s>>>(out, c->fx, c->cls, n, 5); break;
      default: return fail(IMEX_ERR_ARG, "unknown field");
    }
  }
  if (int rc = check_launch("imex_fields")) return rc;
  cudaError_t e = cudaMemcpyAsync(dst, c->tmp, len * sizeof(double),
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_fields: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_set_fields(imex_ctx* c, int which, const double* src, int64_t len, int src_on_device) {
  if (int rc = field_io_check(c, len)) return rc;
  if (!src) return fail(IMEX_ERR_ARG, "NULL source");
  c->guess_valid = 0;
  cudaStream_t s = c->stream;
  const int64_t n = c->hs.nnodes;
  const int nb = (int)((n + 255) / 256);
  const int nc = (int)c->hs.n_c;
  cudaError_t e = cudaMemcpyAsync(c->tmp, src, len * sizeof(double),
                                  src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_fields: ") + cudaGetErrorString(e));
  for (int col = 0; col < c->ncols; ++col) {
    const int64_t on = (int64_t)col * n, oc = (int64_t)col * nc;
    const double* in = c->tmp + on;
    switch (which) {
      case IMEX_FIELD_U:
        k_masked_set<<<nb, 256, 0, s>>>(c->U[c->cur] + on, in, c->cls, n, NODE_D);
        k_masked_set<<<nb, 256, 0, s>>>(c->U[c->cur] + on, in, c->cls, n, NODE_C);
        break;
      case IMEX_FIELD_U_PREV_D:
        k_masked_set<<<nb, 256, 0, s>>>(c->U[1 - c->cur] + on, in, c->cls, n, NODE_D);
        if (scheme_is_cdm(c->hs.pb.scheme)) k_masked_set<<<nb, 256, 0, s>>>(c->U[1 - c->cur] + on, in, c->cls, n, NODE_C);
        break;
      case IMEX_FIELD_V_C:
      case IMEX_FIELD_A_C:
        if (nc > 0)
          k_gather_c<<<(nc + 255) / 256, 256, 0, s>>>((which == IMEX_FIELD_V_C ? c->v_c : c->a_c) + oc, in,
                                                      c->c_node, nc);
        break;
      default: return fail(IMEX_ERR_ARG, "field is not settable");
    }
  }
  if (int rc = check_launch("imex_set_fields")) return rc;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_fields: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_set_step(imex_ctx* c, int64_t n) {
  if (!c || n < 0) return fail(IMEX_ERR_ARG, "bad arguments");
  c->step = n;
  c->guess_valid = 0;
  return IMEX_OK;
}

int imex_set_initial(imex_ctx* c, const double* u0, const double* v0, int64_t len, int on_device) {
  if (int rc = field_io_check(c, len)) return rc;
  if (!u0) return fail(IMEX_ERR_ARG, "NULL u0");
  c->guess_valid = 0;
  cudaStream_t s = c->stream;
  const int64_t n = c->hs.nnodes;
  const int nb = (int)((n + 255) / 256);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(c->tmp, u0, len * sizeof(double), kind, s);
  if (e == cudaSuccess) {
    c->cur = 0;
    for (int col = 0; col < c->ncols; ++col)
      k_masked<<<nb, 256, 0, s>>>(c->U[0] + (size_t)col * n, c->tmp + (size_t)col * n, c->cls, n, 3);
    e = v0 ? cudaMemcpyAsync(c->tmp, v0, len * sizeof(double), kind, s)
           : cudaMemsetAsync(c->tmp, 0, len * sizeof(double), s);
  }
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_initial: ") + cudaGetErrorString(e));
  c->step = 0;
  if (int rc = compute_initial(c, s)) return rc;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_initial: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_set_solver(imex_ctx* c, int solver, double tol, int maxit) {
  if (!c) return fail(IMEX_ERR_ARG, "NULL context");
  if (solver != IMEX_SOLVER_DIRECT && solver != IMEX_SOLVER_PCG_FSAI && solver != IMEX_SOLVER_PCG_JACOBI)
    return fail(IMEX_ERR_ARG, "unknown solver");
  if (!(tol > 0.0) || maxit < 1 || maxit > 100000) return fail(IMEX_ERR_ARG, "need tol > 0 and 1 <= maxit <= 100000");
  if (solver != IMEX_SOLVER_DIRECT && c->ncols > 1)
    return fail(IMEX_ERR_ARG, "the iterative solve serves single-column contexts");
  if (solver == IMEX_SOLVER_DIRECT && !c->factorized)
    return fail(IMEX_ERR_ARG, "the context has no factorisation (imex_setup_pcg)");
  if (solver != IMEX_SOLVER_DIRECT && scheme_is_cdm(c->hs.pb.scheme))
    return fail(IMEX_ERR_ARG, "the iterative solve is of S; central differences solve with M^cc");
  c->solver = solver;
  c->pcg_tol = tol;
  c->pcg_maxit = maxit;
  return IMEX_OK;
}

int imex_pcg_train(imex_ctx* c, int epochs, double lr, double* loss_hist) {
  if (!c || epochs < 0 || !(lr > 0.0)) return fail(IMEX_ERR_ARG, "bad arguments");
  const int n = (int)c->hs.n_c;
  if (n == 0) return IMEX_OK;
  const int nb = (n + kThreads - 1) / kThreads;
  const int nbe = (int)((c->g_nnz + kThreads - 1) / kThreads);
  std::vector<double> part(nb);
  cudaStream_t s = c->stream;
  for (int ep = 0; ep < epochs; ++ep) {
    k_kap_sg<<<nb, kThreads, 0, s>>>(n, c->s_ptr, c->s_col, c->s_val, c->g_ptr, c->g_col, c->g_val, c->g_sg);
    k_kap_grad<<<nb, kThreads, 0, s>>>(n, c->g_ptr, c->g_col, c->g_val, c->g_sg, c->g_grad, c->pcg_part);
    if (loss_hist) {
      cudaError_t e = cudaMemcpyAsync(part.data(), c->pcg_part, nb * sizeof(double), cudaMemcpyDeviceToHost, s);
      e = e ? e : cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_pcg_train: ") + cudaGetErrorString(e));
      double l = 0.0;
      for (double v : part) l += v;
      loss_hist[ep] = l;
    }
    const int64_t t = ++c->adam_t;
    k_adam<<<nbe, kThreads, 0, s>>>(c->g_nnz, c->g_theta, c->g_grad, c->g_scale, c->g_isdiag, c->g_m, c->g_v,
                                    std::pow(0.9, (double)t), std::pow(0.999, (double)t), lr, 1e-3, c->g_val);
    if (int rc = check_launch("imex_pcg_train")) return rc;
  }
  if (epochs > 0 && c->g_nnz > 0)
    k_gt_vals<<<(unsigned)((c->g_nnz + kThreads - 1) / kThreads), kThreads, 0, s>>>(c->g_nnz, c->g_val, c->gt_idx,
                                                                                      c->gt_val);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_pcg_train: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_pcg_train_guess(imex_ctx* c, int nsteps, int epochs, double lr, double* loss_hist, double* w_out) {
  if (!c || nsteps < 4 || epochs < 0 || !(lr > 0.0)) return fail(IMEX_ERR_ARG, "need nsteps >= 4, epochs >= 0, lr > 0");
  if (c->ncols > 1 || !c->pcg_hist) return fail(IMEX_ERR_ARG, "the learned guess serves single-column PCG contexts");
  const int n = (int)c->hs.n_c;
  if (n == 0) return fail(IMEX_ERR_ARG, "no implicit DOFs");
  cudaStream_t s = c->stream;
  const int T = nsteps + 1;
  double* A = nullptr;
  if (cudaMalloc(&A, ((size_t)T * n + T + 4 * 1024 + (size_t)std::max(epochs, 1)) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(IMEX_ERR_ALLOC, "imex_pcg_train_guess: device buffer");
  }
  double* inv = A + (size_t)T * n;           // 1 / ||A_t||^2
  double* part = inv + T;                    // 4 x nb block partials
  double* lhist = part + 4 * 1024;           // loss per epoch
  cudaError_t e = cudaMemcpyAsync(A, c->a_c, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  int rc = IMEX_OK;
  for (int t = 1; t < T && e == cudaSuccess && rc == IMEX_OK; ++t) {
    rc = step_once(c, s, nullptr);
    if (rc == IMEX_OK)
      e = cudaMemcpyAsync(A + (size_t)t * n, c->a_c, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  const int nb = (int)std::min<int64_t>(1024, ((int64_t)n + kThreads - 1) / kThreads);
  if (e == cudaSuccess && rc == IMEX_OK) {
    k_col_sqnorm<<<T, kThreads, 0, s>>>(n, A, inv);
    const double w0[9] = {1.0, 0.0, 0.0, 0, 0, 0, 0, 0, 0};   // start from a^c_n alone
    e = cudaMemcpyAsync(c->guess_state, w0, sizeof(w0), cudaMemcpyHostToDevice, s);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
      k_guess_grad<<<nb, kThreads, 0, s>>>(n, T, A, inv + 1, c->guess_state, part);
      const int64_t t = ep + 1;
      k_guess_adam<<<1, 1, 0, s>>>(nb, part, c->guess_state, std::pow(0.9, (double)t), std::pow(0.999, (double)t),
                                   lr, lhist + ep);
      e = cudaGetLastError();
    }
    // The history of the next PCG solve: a^c after the last two steps.
    e = e ? e : cudaMemcpyAsync(c->pcg_hist, A + (size_t)(T - 2) * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    e = e ? e : cudaMemcpyAsync(c->pcg_hist + n, A + (size_t)(T - 3) * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    double w[3] = {1.0, 0.0, 0.0};
    e = e ? e : cudaMemcpyAsync(w, c->guess_state, sizeof(w), cudaMemcpyDeviceToHost, s);
    if (loss_hist && epochs > 0) e = e ? e : cudaMemcpyAsync(loss_hist, lhist, epochs * sizeof(double), cudaMemcpyDeviceToHost, s);
    e = e ? e : cudaStreamSynchronize(s);
    if (e == cudaSuccess && w_out) std::copy(w, w + 3, w_out);
  }
  cudaFree(A);
  if (rc != IMEX_OK) return rc;
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_pcg_train_guess: ") + cudaGetErrorString(e));
  c->guess_on = 1;
  c->guess_valid = 2;
  return IMEX_OK;
}

int imex_pcg_fsai_closed_form(imex_ctx* c) {
  if (!c || !c->g_val) return fail(IMEX_ERR_ARG, "the context has no PCG solver");
  const HostSetup& hs = c->hs;
  const int n = (int)hs.n_c;
  if (n == 0) return IMEX_OK;
  // G's pattern as the setup built it: row i holds the columns j <= i of S's
  // row i, in S's order.
  std::vector<int> g_ptr(1, 0), g_col;
  for (int i = 0; i < n; ++i) {
    for (int k = hs.S_ptr[i]; k < hs.S_ptr[i + 1]; ++k)
      if (hs.S_col[k] <= i) g_col.push_back(hs.S_col[k]);
    g_ptr.push_back((int)g_col.size());
  }
  if ((int64_t)g_col.size() != c->g_nnz) return fail(IMEX_ERR_ARG, "internal error: G pattern mismatch");
  // Column j: rows Q (i >= j with G_ij on the pattern) and their positions.
  std::vector<int> ct_ptr(n + 1, 0), ct_row(g_col.size()), ct_pos(g_col.size());
  for (int j : g_col) ct_ptr[j + 1]++;
  for (int j = 0; j < n; ++j) ct_ptr[j + 1] += ct_ptr[j];
  {
    std::vector<int> fill(ct_ptr.begin(), ct_ptr.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int e = g_ptr[i]; e < g_ptr[i + 1]; ++e) {
        ct_row[fill[g_col[e]]] = i;
        ct_pos[fill[g_col[e]]++] = e;
      }
  }
  auto s_at = [&](int a, int b) {   // S_ab (0 off the pattern)
    const int* lo = hs.S_col.data() + hs.S_ptr[a];
    const int* hi = hs.S_col.data() + hs.S_ptr[a + 1];
    for (const int* q = lo; q < hi; ++q)
      if (*q == b) return hs.S_val[q - hs.S_col.data()];
    return 0.0;
  };
  std::vector<double> val(g_col.size(), 0.0);
  std::string err;
  std::mutex mu;
  auto work = [&](int j0, int j1) {
    std::vector<double> A, y;
    for (int j = j0; j < j1; ++j) {
      const int q0 = ct_ptr[j], m = ct_ptr[j + 1] - q0;
      const int* Q = ct_row.data() + q0;   // ascending; Q[0] = j
      A.assign((size_t)m * m, 0.0);
      for (int a = 0; a < m; ++a)
        for (int b = 0; b <= a; ++b) A[(size_t)a * m + b] = s_at(Q[a], Q[b]);
      // Cholesky of S_QQ (lower, in place), then S_QQ y = e_0.
      bool ok = true;
      for (int k = 0; k < m && ok; ++k) {
        double d = A[(size_t)k * m + k];
        for (int q = 0; q < k; ++q) d -= A[(size_t)k * m + q] * A[(size_t)k * m + q];
        if (!(d > 0.0)) { ok = false; break; }
        const double l = std::sqrt(d);
        A[(size_t)k * m + k] = l;
        for (int i = k + 1; i < m; ++i) {
          double t = A[(size_t)i * m + k];
          for (int q = 0; q < k; ++q) t -= A[(size_t)i * m + q] * A[(size_t)k * m + q];
          A[(size_t)i * m + k] = t / l;
        }
      }
      if (!ok) {
        std::lock_guard<std::mutex> lk(mu);
        err = "S_QQ not positive definite";
        return;
      }
      y.assign(m, 0.0);
      for (int i = 0; i < m; ++i) {   // L z = e_0
        double t = i == 0 ? 1.0 : 0.0;
        for (int q = 0; q < i; ++q) t -= A[(size_t)i * m + q] * y[q];
        y[i] = t / A[(size_t)i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {   // L^T y = z
        double t = y[i];
        for (int q = i + 1; q < m; ++q) t -= A[(size_t)q * m + i] * y[q];
        y[i] = t / A[(size_t)i * m + i];
      }
      const double sc = 1.0 / std::sqrt(y[0]);
      for (int a = 0; a < m; ++a) val[ct_pos[q0 + a]] = y[a] * sc;
    }
  };
  const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) th.emplace_back(work, (int)((int64_t)n * t / nth), (int)((int64_t)n * (t + 1) / nth));
  for (auto& t : th) t.join();
  if (!err.empty()) return fail(IMEX_ERR_NOT_SPD, "imex_pcg_fsai_closed_form: " + err);
  // Values, their row-scaled parameters for further training, the
  // transposed copy; the Adam state starts afresh.
  std::vector<double> scale(g_col.size()), theta(g_col.size());
  cudaError_t e = cudaMemcpy(scale.data(), c->g_scale, scale.size() * sizeof(double), cudaMemcpyDeviceToHost);
  for (size_t k = 0; k < val.size(); ++k) theta[k] = val[k] / scale[k];
  e = e ? e : cudaMemcpy(c->g_val, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice);
  e = e ? e : cudaMemcpy(c->g_theta, theta.data(), theta.size() * sizeof(double), cudaMemcpyHostToDevice);
  e = e ? e : cudaMemset(c->g_m, 0, val.size() * sizeof(double));
  e = e ? e : cudaMemset(c->g_v, 0, val.size() * sizeof(double));
  if (e == cudaSuccess) {
    k_gt_vals<<<(unsigned)((c->g_nnz + kThreads - 1) / kThreads), kThreads>>>(c->g_nnz, c->g_val, c->gt_idx, c->gt_val);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_pcg_fsai_closed_form: ") + cudaGetErrorString(e));
  c->adam_t = 0;
  return IMEX_OK;
}

int imex_pcg_set_guess(imex_ctx* c, int enable, const double* w) {
  if (!c) return fail(IMEX_ERR_ARG, "NULL context");
  if (!c->pcg_hist) return fail(IMEX_ERR_ARG, "the context has no PCG solver");
  if (enable && w) {
    const double st[9] = {w[0], w[1], w[2], 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(c->guess_state, st, sizeof(st), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_pcg_set_guess: ") + cudaGetErrorString(e));
  }
  c->guess_on = enable ? 1 : 0;
  return IMEX_OK;
}

int imex_pcg_status(imex_ctx* c, int64_t* iters_last, double* res_last, int64_t* iters_total, int64_t* fallbacks) {
  if (!c) return fail(IMEX_ERR_ARG, "NULL context");
  int st[2] = {0, 0};
  long long cnt[2] = {0, 0};
  double res = 0.0;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  e = e ? e : cudaMemcpy(st, c->pcg_status, sizeof(st), cudaMemcpyDeviceToHost);
  e = e ? e : cudaMemcpy(cnt, c->pcg_counters, sizeof(cnt), cudaMemcpyDeviceToHost);
  e = e ? e : cudaMemcpy(&res, c->pcg_res, sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_pcg_status: ") + cudaGetErrorString(e));
  if (iters_last) *iters_last = st[0];
  if (res_last) *res_last = res;
  if (iters_total) *iters_total = cnt[0];
  if (fallbacks) *fallbacks = cnt[1];
  return IMEX_OK;
}

int imex_fsai_kaporin(int n, const int* s_ptr, const int* s_col, const double* s_val, const int* g_ptr,
                      const int* g_col, const double* g_val, double* grad, double* loss, void* stream) {
  if (n < 1 || !s_ptr || !s_col || !s_val || !g_ptr || !g_col || !g_val || !grad || !loss)
    return fail(IMEX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int nnz = 0;
  cudaError_t e = cudaMemcpyAsync(&nnz, g_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = e ? e : cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_fsai_kaporin: ") + cudaGetErrorString(e));
  const int nb = (n + kThreads - 1) / kThreads;
  double *sg = nullptr, *part = nullptr;
  e = cudaMalloc(&sg, std::max(nnz, 1) * sizeof(double));
  e = e ? e : cudaMalloc(&part, nb * sizeof(double));
  if (e == cudaSuccess) {
    k_kap_sg<<<nb, kThreads, 0, s>>>(n, s_ptr, s_col, s_val, g_ptr, g_col, g_val, sg);
    k_kap_grad<<<nb, kThreads, 0, s>>>(n, g_ptr, g_col, g_val, sg, grad, part);
    e = cudaGetLastError();
  }
  std::vector<double> hp(nb);
  e = e ? e : cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, s);
  e = e ? e : cudaStreamSynchronize(s);
  cudaFree(sg);
  cudaFree(part);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_fsai_kaporin: ") + cudaGetErrorString(e));
  double l = 0.0;
  for (double v : hp) l += v;
  *loss = l;
  return IMEX_OK;
}

int imex_adjoint(imex_ctx* c, int64_t nsteps, const int64_t* rec_nodes, int nrec, const double* data,
                 int checkpoint_every, double* grad, double* misfit) {
  if (!c || nsteps < 1 || nrec < 1 || !rec_nodes || !data || !grad || !misfit || checkpoint_every < 1)
    return fail(IMEX_ERR_ARG, "bad arguments");
  const HostSetup& hs = c->hs;
  if (hs.pb.scheme != kSchemeImex) return fail(IMEX_ERR_ARG, "the adjoint is of the Newmark IMEX scheme");
  if (!c->factorized) return fail(IMEX_ERR_ARG, "the adjoint needs a factorised context");
  for (int k = 0; k < nrec; ++k)
    if (rec_nodes[k] < 0 || rec_nodes[k] >= hs.nnodes) return fail(IMEX_ERR_ARG, "receiver node out of range");
  cudaStream_t s = c->stream;
  const int ncols = c->ncols;
  const int64_t nn = hs.nnodes, nc = std::max<int64_t>(hs.n_c, 1), N = nsteps, Kc = checkpoint_every;
  const int64_t nseg = (N + Kc - 1) / Kc;
  const int64_t ck_len = (int64_t)ncols * (2 * nn + 2 * nc);
  std::vector<void*> bufs;
  auto dalloc = [&](size_t bytes) -> double* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return static_cast<double*>(p);
  };
  auto cleanup = [&]() {
    for (void* p : bufs) cudaFree(p);
  };
  double* ck = dalloc((size_t)(nseg + 1) * ck_len * sizeof(double));
  double* fin = dalloc((size_t)ck_len * sizeof(double));
  double* seg = dalloc((size_t)(Kc + 1) * ncols * nn * sizeof(double));
  double* ubar = dalloc((size_t)ncols * nn * sizeof(double));
  double* ubar_prev = dalloc((size_t)ncols * nn * sizeof(double));
  double* T = dalloc((size_t)ncols * nn * sizeof(double));
  double* z1 = dalloc((size_t)ncols * nn * sizeof(double));
  double* z2 = dalloc((size_t)ncols * nn * sizeof(double));
  double* kg = dalloc((size_t)ncols * nn * sizeof(double));
  double* kh = dalloc((size_t)ncols * nn * sizeof(double));
  double* vbar = dalloc((size_t)ncols * nc * sizeof(double));
  double* abar = dalloc((size_t)ncols * nc * sizeof(double));
  double* ucp = dalloc((size_t)ncols * nc * sizeof(double));
  double* vcp = dalloc((size_t)ncols * nc * sizeof(double));
  double* dgrad = dalloc((size_t)hs.ncell_total * sizeof(double));
  double* jpart = dalloc((size_t)ncols * 2 * sizeof(double));
  double* ddata = dalloc((size_t)N * ncols * nrec * sizeof(double));
  int64_t* drec = reinterpret_cast<int64_t*>(dalloc((size_t)nrec * sizeof(int64_t)));
  for (void* p : bufs)
    if (!p) {
      cleanup();
      return fail(IMEX_ERR_ALLOC, "imex_adjoint: device buffers");
    }
  if (std::count(bufs.begin(), bufs.end(), nullptr) || bufs.size() != 18) {
    cleanup();
    return fail(IMEX_ERR_ALLOC, "imex_adjoint: device buffers");
  }
  cudaError_t e = cudaMemcpyAsync(ddata, data, (size_t)N * ncols * nrec * sizeof(double), cudaMemcpyHostToDevice, s);
  e = e ? e : cudaMemcpyAsync(drec, rec_nodes, nrec * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  e = e ? e : cudaMemsetAsync(jpart, 0, ncols * 2 * sizeof(double), s);
  e = e ? e : cudaMemsetAsync(dgrad, 0, hs.ncell_total * sizeof(double), s);
  // State copies: U[cur], U[1-cur], v_c, a_c of every column.
  auto save = [&](double* dst) {
    cudaError_t r = cudaMemcpyAsync(dst, c->U[c->cur], ncols * nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    r = r ? r : cudaMemcpyAsync(dst + ncols * nn, c->U[1 - c->cur], ncols * nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    r = r ? r : cudaMemcpyAsync(dst + 2 * ncols * nn, c->v_c, ncols * nc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    r = r ? r : cudaMemcpyAsync(dst + 2 * ncols * nn + ncols * nc, c->a_c, ncols * nc * sizeof(double),
                                cudaMemcpyDeviceToDevice, s);
    return r;
  };
  auto restore = [&](const double* src) {
    cudaError_t r = cudaMemcpyAsync(c->U[c->cur], src, ncols * nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    r = r ? r : cudaMemcpyAsync(c->U[1 - c->cur], src + ncols * nn, ncols * nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    r = r ? r : cudaMemcpyAsync(c->v_c, src + 2 * ncols * nn, ncols * nc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    r = r ? r : cudaMemcpyAsync(c->a_c, src + 2 * ncols * nn + ncols * nc, ncols * nc * sizeof(double),
                                cudaMemcpyDeviceToDevice, s);
    return r;
  };
  const int64_t n0 = c->step;
  const int nbn = (int)((nn + kThreads - 1) / kThreads), nbc = (int)((nc + kThreads - 1) / kThreads);
  const dim3 gn(nbn, ncols), gc(nbc, ncols);
  const HetArgs ha = het_args(c);
  // Forward with checkpoints and the misfit.
  e = e ? e : save(ck);
  for (int64_t n = 0; n < N && e == cudaSuccess; ++n) {
    if (int rc = step_once(c, s, nullptr)) {
      cleanup();
      return rc;
    }
    k_misfit<<<ncols, kThreads, 0, s>>>(nrec, nn, drec, c->U[c->cur], ddata + n * ncols * nrec, nullptr, jpart, 0);
    if ((n + 1) % Kc == 0) e = save(ck + ((n + 1) / Kc) * ck_len);
  }
  e = e ? e : save(fin);
  // Reverse over the segments, each recomputed from its checkpoint.
  e = e ? e : cudaMemsetAsync(ubar, 0, ncols * nn * sizeof(double), s);
  e = e ? e : cudaMemsetAsync(ubar_prev, 0, ncols * nn * sizeof(double), s);
  e = e ? e : cudaMemsetAsync(vbar, 0, ncols * nc * sizeof(double), s);
  e = e ? e : cudaMemsetAsync(abar, 0, ncols * nc * sizeof(double), s);
  const double dt = hs.dt;
  ExplicitArgs ea = explicit_args(c, c->U[0], c->U[0], c->U[0], 0.0, 0.0, 0.0, 0.0, false);
  e = e ? e : cudaFuncSetAttribute(k_grad_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)grad_cells_smem(hs.Pd));
  for (int64_t sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg) {
    const int64_t nb = sg * Kc, ne = std::min(N, nb + Kc);
    e = restore(ck + sg * ck_len);
    c->step = n0 + nb;
    e = e ? e : cudaMemcpyAsync(seg, c->U[c->cur], ncols * nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    for (int64_t n = nb; n < ne && e == cudaSuccess; ++n) {
      if (int rc = step_once(c, s, nullptr)) {
        cleanup();
        return rc;
      }
      e = cudaMemcpyAsync(seg + (n - nb + 1) * ncols * nn, c->U[c->cur], ncols * nn * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    }
    for (int64_t n = ne - 1; n >= nb && e == cudaSuccess; --n) {
      const double* un = seg + (n - nb) * ncols * nn;
      const double* un1 = seg + (n - nb + 1) * ncols * nn;
      k_misfit<<<ncols, kThreads, 0, s>>>(nrec, nn, drec, un1, ddata + n * ncols * nrec, ubar, jpart + ncols, 1);
      if (hs.n_c > 0) {
        k_adj_pre<<<gc, kThreads, 0, s>>>((int)hs.n_c, nn, nc, c->c_node, ubar, vbar, abar, c->rhs0, ucp, vcp, dt);
        e = launch_solve_chain(c, true, 0.0, nullptr, 2, c->U[c->cur], c->U[c->cur], c->upd, c->sol, c->rhs0, c->hbuf, s,
                               nullptr, false, true);
      }
      e = e ? e : cudaMemsetAsync(z1, 0, ncols * nn * sizeof(double), s);
      if (hs.n_c > 0) k_c_to_grid_set<<<gc, kThreads, 0, s>>>((int)hs.n_c, nn, nc, c->c_node, c->sol, z1);
      k_applyK<<<gn, kThreads, 0, s>>>(ha, c->cls, z1, kg, nn);
      k_adj_mid<<<gn, kThreads, 0, s>>>(ea, nn, ubar, kg, T, z2, c->node_c_dev, ucp, dt);
      k_applyK<<<gn, kThreads, 0, s>>>(ha, c->cls, z2, kh, nn);
      k_grad_cells<<<ha.ncell, kGradThreads, grad_cells_smem(hs.Pd), s>>>(ha, ncols, nn, z2, un, z1, un1, dgrad);
      k_adj_post<<<gn, kThreads, 0, s>>>(ea, nn, kh, T, ubar, ubar_prev, c->node_c_dev, ucp, vcp, vbar, abar, dt);
      if (int rc = check_launch("imex_adjoint")) {
        cleanup();
        return rc;
      }
    }
  }
  // Leave the context at the end of the forward run.
  e = e ? e : restore(fin);
  c->step = n0 + N;
  std::vector<double> jp(ncols * 2);
  e = e ? e : cudaMemcpyAsync(grad, dgrad, hs.ncell_total * sizeof(double), cudaMemcpyDeviceToHost, s);
  e = e ? e : cudaMemcpyAsync(jp.data(), jpart, ncols * 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  e = e ? e : cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_adjoint: ") + cudaGetErrorString(e));
  double J = 0.0;
  for (int col = 0; col < ncols; ++col) J += jp[col];
  *misfit = J;
  return IMEX_OK;
}

int imex_info(imex_ctx* c, imex_stats* st) {
  if (!c || !st) return fail(IMEX_ERR_ARG, "bad arguments");
  fill_stats(c->hs, st);
  st->step = c->step;
  st->solve_levels = (int64_t)c->lev_cta0.size();
  int64_t widest = c->ntop;
  for (int n : c->lev_ncta) widest = std::max<int64_t>(widest, n);
  st->solve_ctas = widest;
  st->solve_smem_bytes = (int64_t)c->smem_walk_req;
  st->solve_smem_needed = (int64_t)c->smem_walk;
  st->solve_col_block = c->col_block;
  for (int k = 0; k < 7; ++k) st->solve_col_block_us[k] = c->cb_us[k];
  st->launches_per_step = launches_per_step(c);
  st->rhs_pairs = (int64_t)c->hs.contrib_pos.size();
  st->ncols = c->ncols;
  st->explicit_tile_cells = c->TC;
  st->explicit_tile_us_large = c->tile_us[0];
  st->explicit_tile_us_small = c->tile_us[1];
  st->explicit_variant = c->xsplit ? kExplicitSplit + split_index(c) : c->xvar;
  for (int s = 0; s < kSplitVariants; ++s) st->explicit_split_us[s] = c->tile_us[kExplicitSplit + s];
  st->explicit_sweep_us = c->tile_us[2];
  st->explicit_sweep_short_us = c->tile_us[3];
  st->large_supernodes = c->n_large;
  st->max_rows = c->hs.max_rows;
  st->device_bytes = (int64_t)c->bytes;
  st->factorized = c->factorized;
  return IMEX_OK;
}

int imex_check_finite(imex_ctx* c, double* max_abs_u) {
  if (!c) return fail(IMEX_ERR_ARG, "NULL context");
  const HostSetup& hs = c->hs;
  cudaStream_t s = c->stream;
  const int64_t nn = hs.nnodes * c->ncols, nc = hs.n_c * c->ncols;
  double* out = c->pcg_part;                          // kHealthBlocks maxima
  int* flag = reinterpret_cast<int*>(c->pcg_part + kHealthBlocks);
  k_health<<<kHealthBlocks, kThreads, 0, s>>>(c->U[c->cur], nn, c->cls, hs.nnodes, out, flag, 0);
  k_health<<<kHealthBlocks, kThreads, 0, s>>>(c->U[1 - c->cur], nn, c->cls, hs.nnodes, c->pcg_part + 2 * kHealthBlocks,
                                              flag, 1);
  if (nc > 0) {
    k_health<<<kHealthBlocks, kThreads, 0, s>>>(c->v_c, nc, nullptr, 1, c->pcg_part + 2 * kHealthBlocks, flag, 1);
    k_health<<<kHealthBlocks, kThreads, 0, s>>>(c->a_c, nc, nullptr, 1, c->pcg_part + 2 * kHealthBlocks, flag, 1);
  }
  std::vector<double> m(kHealthBlocks);
  std::vector<int> f(kHealthBlocks);
  cudaError_t e = cudaMemcpyAsync(m.data(), out, kHealthBlocks * sizeof(double), cudaMemcpyDeviceToHost, s);
  e = e ? e : cudaMemcpyAsync(f.data(), flag, kHealthBlocks * sizeof(int), cudaMemcpyDeviceToHost, s);
  e = e ? e : cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_check_finite: ") + cudaGetErrorString(e));
  double mx = 0.0;
  int bad = 0;
  for (int b = 0; b < kHealthBlocks; ++b) {
    mx = std::max(mx, m[b]);
    bad |= f[b];
  }
  if (max_abs_u) *max_abs_u = mx;
  if (bad) return fail(IMEX_ERR_DIVERGED, "non-finite values in the state");
  return IMEX_OK;
}

void imex_destroy(imex_ctx* c) {
  if (!c) return;
  if (c->base) {
    cudaDeviceSynchronize();
    for (auto& row : c->io_ev)
      for (cudaEvent_t& ev : row)
        if (ev) cudaEventDestroy(ev);
    if (c->io_h2d) cudaStreamDestroy(c->io_h2d);
    if (c->io_d2h) cudaStreamDestroy(c->io_d2h);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ov_fork) cudaEventDestroy(c->ov_fork);
    if (c->ov_join) cudaEventDestroy(c->ov_join);
    if (c->has_hooks) {
      if (c->hooks.release) c->hooks.release(c->base, c->hooks.user);
    } else {
      cudaFree(c->base);
    }
  }
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// imex_step_noalloc: imex_step with the implicit solve's scratch (descendant
// update vectors, solution vector, right-hand sides) in a fixed array
// compiled into the library instead of context memory.
#include <mutex>

namespace {
constexpr int64_t kStaticScratchDoubles = 262144;  // 2 MiB
constexpr int kMaxDevices = 64;
std::mutex g_static_scratch_mu;
double* g_static_scratch_addr[kMaxDevices] = {nullptr};
}  // namespace

static __device__ __align__(256) double g_static_solve_scratch[kStaticScratchDoubles];

extern "C" int imex_step_noalloc(imex_ctx* c, int64_t n, void* stream) {
  if (!c || n < 0) return fail(IMEX_ERR_ARG, "bad arguments");
  if (!c->factorized) return fail(IMEX_ERR_ARG, "imex_step_noalloc needs a factorised context");
  // The PCG solvers keep their right-hand side and iterates in context
  // memory; only the factorised solve runs on the fixed array.
  if (c->solver != IMEX_SOLVER_DIRECT)
    return fail(IMEX_ERR_ARG, "imex_step_noalloc runs the factorised direct solve only (imex_set_solver: direct)");
  const HostSetup& hs = c->hs;
  auto even = [](int64_t v) { return v + (v & 1); };
  const int64_t n_upd = even(std::max<int64_t>(hs.upd_size, 1)) * c->ncols;
  const int64_t n_sol = even(std::max<int64_t>(hs.n_c, 1)) * c->ncols;
  // A third vector for the backward products of supernodes above 256 rows.
  bool panels = false;
  for (int k : c->pan_ncta) panels = panels || k > 0;
  const int64_t need = n_upd + (panels ? 3 : 2) * n_sol;
  if (need > kStaticScratchDoubles)
    return fail(IMEX_ERR_ARG, "imex_step_noalloc: the implicit solve needs " + std::to_string(need) +
                                  " doubles of scratch; the static scratch holds " +
                                  std::to_string(kStaticScratchDoubles) + " (use imex_step)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(IMEX_ERR_CUDA, "imex_step_noalloc: no current CUDA device");
  if (dev != c->device) return fail(IMEX_ERR_ARG, "imex_step_noalloc: the context lives on another device");
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_scratch_mu);
    if (!g_static_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_solve_scratch);
      if (e != cudaSuccess)
        return fail(IMEX_ERR_CUDA, std::string("imex_step_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_static_scratch_addr[dev] = static_cast<double*>(p);
    }
    base = g_static_scratch_addr[dev];
  }
  double* upd = base;
  double* sol = upd + n_upd;
  double* rhs0 = sol + n_sol;
  double* hbuf = panels ? rhs0 + n_sol : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  c->stream = s;
  for (int64_t k = 0; k < n; ++k)
    if (int rc = step_once(c, s, nullptr, nullptr, upd, sol, rhs0, hbuf)) return rc;
  return IMEX_OK;
}

