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
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/imex.h"
#include "kernels.cuh"
#include "setup.h"

using namespace imex;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------------------
// A1 + A2 (+ A3): explicit apply on the tensor grid, CDM update, prediction.
//
// A tile owns OX x OY nodes (TC x TC cells).  With u staged in shared memory
// together with one halo cell on the low side, the stiffness rows of the
// owned nodes are formed by sum factorisation:
//   x pass: T1 = (sx K1)_x u, T2 = (M1)_x u, cell by cell (the two cell
//           contributions at a vertex are added in a fix-up pass),
//   y pass: r = (M1)_y T1 + (sy K1)_y T2, again cell by cell plus fix-up.
// For an I_d node every surrounding cell is uncut, so this equals its row of
// K^d u_n (Eq. Kd).  Nodes of I_c and inactive nodes are computed but not
// written.  Cells outside the grid contribute nothing.
template <int P, int TC>
__global__ void __launch_bounds__(kThreads) k_explicit2d(ExplicitArgs a, Ops2D ops) {
  constexpr int p = P - 1;
  constexpr int OX = TC * p, OY = TC * p;
  constexpr int RX = (TC + 1) * p + 1, RY = RX;
  constexpr int NC = TC + 1;
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int ntiles = a.ntx * a.nty;

  if ((int)blockIdx.x >= ntiles) {
    // Newmark prediction on I_c (Fig. TrapCDMIMEX, "Prediction").
    const double c1 = a.dt, c2 = (0.5 - kNewmarkBeta) * a.dt * a.dt;
    const int stride = (gridDim.x - ntiles) * blockDim.x;
    for (int r = (blockIdx.x - ntiles) * blockDim.x + tid; r < a.n_c; r += stride) {
      const int node = a.c_node[r];
      a.OUT[node] = a.U[node] + c1 * a.v_c[r] + c2 * a.a_c[r];
    }
    return;
  }

  double* su = sm;                 // RY x RX
  double* t1 = su + RY * RX;       // RY x OX
  double* t2 = t1 + RY * OX;       // RY x OX
  double* scr = t2 + RY * OX;
  double* tl1 = scr;               // RY x NC vertex partials (x pass)
  double* tr1 = tl1 + RY * NC;
  double* tl2 = tr1 + RY * NC;
  double* tr2 = tl2 + RY * NC;
  double* rr = scr;                // OY x OX (aliases the x-pass partials)
  double* rb = rr + OY * OX;       // NC x OX vertex partials (y pass)
  double* rt = rb + NC * OX;

  const int tx = blockIdx.x % a.ntx, ty = blockIdx.x / a.ntx;
  const int X0 = tx * OX, Y0 = ty * OY;
  const int cx0 = X0 / p - 1, cy0 = Y0 / p - 1;

  for (int idx = tid; idx < RY * RX; idx += kThreads) {
    const int yy = idx / RX, xx = idx - yy * RX;
    const int gx = X0 - p + xx, gy = Y0 - p + yy;
    su[idx] = (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) ? a.U[(size_t)gy * a.nx + gx] : 0.0;
  }
  __syncthreads();

  // x pass: item = (row yy, cell cc), rows fastest.
  for (int it = tid; it < RY * NC; it += kThreads) {
    const int cc = it / RY, yy = it - cc * RY;
    const int cx = cx0 + cc;
    double v[P], o1[P], o2[P];
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = su[yy * RX + cc * p + j];
    const bool valid = (cx >= 0 && cx < a.ncx);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      double s1 = 0.0, s2 = 0.0;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        s1 = fma(ops.kx[i * P + j], v[j], s1);
        s2 = fma(ops.mx[i * P + j], v[j], s2);
      }
      o1[i] = valid ? s1 : 0.0;
      o2[i] = valid ? s2 : 0.0;
    }
    if (cc >= 1) {
#pragma unroll
      for (int i = 1; i < p; ++i) {
        t1[yy * OX + (cc - 1) * p + i] = o1[i];
        t2[yy * OX + (cc - 1) * p + i] = o2[i];
      }
    }
    tl1[yy * NC + cc] = o1[0];
    tr1[yy * NC + cc] = o1[p];
    tl2[yy * NC + cc] = o2[0];
    tr2[yy * NC + cc] = o2[p];
  }
  __syncthreads();
  for (int it = tid; it < RY * TC; it += kThreads) {
    const int k = it / RY, yy = it - k * RY;
    t1[yy * OX + k * p] = tr1[yy * NC + k] + tl1[yy * NC + k + 1];
    t2[yy * OX + k * p] = tr2[yy * NC + k] + tl2[yy * NC + k + 1];
  }
  __syncthreads();

  // y pass: item = (column xo, cell row cr), columns fastest.
  for (int it = tid; it < OX * NC; it += kThreads) {
    const int cr = it / OX, xo = it - cr * OX;
    const int cy = cy0 + cr;
    double va[P], vb[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      va[j] = t1[(cr * p + j) * OX + xo];
      vb[j] = t2[(cr * p + j) * OX + xo];
    }
    const bool valid = (cy >= 0 && cy < a.ncy);
    double o[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        s = fma(ops.my[i * P + j], va[j], s);
        s = fma(ops.ky[i * P + j], vb[j], s);
      }
      o[i] = valid ? s : 0.0;
    }
    if (cr >= 1) {
#pragma unroll
      for (int i = 1; i < p; ++i) rr[((cr - 1) * p + i) * OX + xo] = o[i];
    }
    rb[cr * OX + xo] = o[0];
    rt[cr * OX + xo] = o[p];
  }
  __syncthreads();
  for (int it = tid; it < TC * OX; it += kThreads) {
    const int k = it / OX, xo = it - k * OX;
    rr[(k * p) * OX + xo] = rt[k * OX + xo] + rb[(k + 1) * OX + xo];
  }
  __syncthreads();

  // CDM update of the owned I_d nodes (Eqs. CDMacc, CDMstep).
  for (int it = tid; it < OY * OX; it += kThreads) {
    const int yo = it / OX, xo = it - yo * OX;
    const int gx = X0 + xo, gy = Y0 + yo;
    if (gx >= a.nx || gy >= a.ny) continue;
    const size_t g = (size_t)gy * a.nx + gx;
    if (a.cls[g] != NODE_D) continue;
    const double r = rr[yo * OX + xo];
    const double u = su[(yo + p) * RX + xo + p];
    const double minv = a.winv_x[gx] * a.winv_y[gy];
    const double ft = a.ft_dev ? a.ft_dev[0] : a.ft;
    const double acc = minv * (ft * a.fx[g] - r);
    a.OUT[g] = a.cu * u + a.cw * a.W[g] + a.ca * acc;
  }
}

// ---------------------------------------------------------------------------
// A4: element products y_e = K_e u_pred,e for every cell touching I_c.  One
// warp per cell; the cell's nodal block is staged in shared memory.
__global__ void __launch_bounds__(kThreads) k_iface(IfaceArgs a) {
  __shared__ double ue[kWarps][128];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int e = blockIdx.x * kWarps + warp;
  if (e >= a.n_iface) return;
  const int cid = a.cell[e];
  const int cx = cid % a.ncx;
  const int cy = (cid / a.ncx) % a.ncy;
  const int cz = cid / (a.ncx * a.ncy);
  const size_t base = (size_t)cx * a.p + (size_t)a.nx * ((size_t)cy * a.p) +
                      (size_t)a.nx * a.ny * ((size_t)cz * a.p);
  for (int l = lane; l < a.Pd; l += 32) {
    const int i = l % a.P, j = (l / a.P) % a.P, k = l / (a.P * a.P);
    ue[warp][l] = a.SRC[base + i + (size_t)a.nx * j + (size_t)a.nx * a.ny * k];
  }
  __syncwarp();
  const int ki = a.kidx[e];
  const double* K = ki >= 0 ? a.cutK + (size_t)ki * a.Pd * a.Pd : a.uncutK;
  const double sc = ki >= 0 ? 1.0 : a.c2[e];
  for (int l = lane; l < a.Pd; l += 32) {
    double s = 0.0;
    for (int m = 0; m < a.Pd; ++m) s = fma(K[l + (size_t)a.Pd * m], ue[warp][m], s);
    a.Y[(size_t)e * a.Pd + l] = sc * s;
  }
}

// ---------------------------------------------------------------------------
// A4 gather + A5 + A6.  One thread-block cluster per group of connected
// components of I_c (components are bin-packed into groups by factor size).
// The nested-dissection tree is walked level by level:
//   forward   y_t = L_tt^{-1} (rhs_t - sum of descendant updates),  upd_t = L_{rows,t} y_t
//   backward  x_t = L_tt^{-T} (y_t - L_{rows,t}^T x_rows)
// Each supernode is handled by one CTA with all its warps: every dense
// product is split along its inner dimension across the warps (lanes own the
// output rows), and the warp partials are summed in shared memory in a fixed
// order, so the result is deterministic.  The nodes of a level go to the
// cluster's CTAs round-robin, largest first; a cluster barrier (release /
// acquire at cluster scope) separates levels, and values written by another
// CTA are read with L1-bypassing loads.
constexpr int kMaxWidth = 256;       // largest supernode / row set the solve handles
constexpr int kSolveSmemBudget = 200 * 1024;

// Partial products of a warp over the inner range [j0, j1):
// part[i] = sum_j M[i si + j sj] v[j] for rows i = lane + 32 r < nrows (R row
// groups), restricted to j <= i (tri > 0, lower) or j >= i (tri < 0, upper).
// (si, sj) = (1, ld) reads a column-major block, (ld, 1) its transpose; with
// an odd ld both are free of shared-memory bank conflicts.
template <int R>
__device__ __forceinline__ void warp_partial_r(const double* M, int si, int sj, int nrows,
                                               const double* v, int j0, int j1, int tri, double* part,
                                               int lane) {
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  for (int j = j0; j < j1; ++j) {
    const double vj = v[j];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      const bool ok = i < nrows && (tri == 0 || (tri > 0 ? j <= i : j >= i));
      if (ok) acc[r] = fma(M[(size_t)i * si + (size_t)j * sj], vj, acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < nrows) part[i] = acc[r];
  }
}

__device__ __forceinline__ void warp_partial(const double* M, int si, int sj, int nrows,
                                             const double* v, int j0, int j1, int tri, double* part,
                                             int lane) {
  switch ((nrows + 31) / 32) {
    case 0: break;
    case 1: warp_partial_r<1>(M, si, sj, nrows, v, j0, j1, tri, part, lane); break;
    case 2: warp_partial_r<2>(M, si, sj, nrows, v, j0, j1, tri, part, lane); break;
    case 3: warp_partial_r<3>(M, si, sj, nrows, v, j0, j1, tri, part, lane); break;
    case 4: warp_partial_r<4>(M, si, sj, nrows, v, j0, j1, tri, part, lane); break;
    default: warp_partial_r<8>(M, si, sj, nrows, v, j0, j1, tri, part, lane); break;
  }
}

// Start an asynchronous copy of n 16-byte chunks global -> shared with all
// threads (cp.async, no register staging); completed by async_copy_wait().
__device__ __forceinline__ void async_copy_16(void* dst, const void* src, int64_t nchunks) {
  const char* s8 = reinterpret_cast<const char*>(src);
  char* d8 = reinterpret_cast<char*>(dst);
  for (int64_t k = threadIdx.x; k < nchunks; k += blockDim.x) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(d8 + 16 * k);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(s8 + 16 * k) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void async_copy_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

template <bool kSmem>
__global__ void __launch_bounds__(kThreads) k_solve(SolveArgs a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) double smg[];
  const int CL = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int grp = blockIdx.x / CL;
  const int cta = grp * CL + crank;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, tid = threadIdx.x;
  const int W = a.max_width;                  // >= max(max_block, max_rows)
  double* g = smg;                            // W: gathered rhs / y / h
  double* y = g + W;                          // W
  double* xr = y + W;                         // W: ancestor values
  double* part = xr + W;                      // kWarps x W warp partials
  double* rhs = part + kWarps * W + a.max_zn;  // this CTA's rows: f_t f_x^c - (K^c u_pred) part
  double* blob = rhs + a.max_cta_rows;        // this CTA's factor blocks (max_cta_rows is even)
  const int64_t boff = a.blob_off[cta], blen = a.blob_len[cta];
  const double* Bf = kSmem ? blob : a.vals + boff;
  // This CTA's index lists: row pointers and positions of descendant updates,
  // then the ancestor rows of its nodes (16-byte padded in global memory).
  int* ilist = reinterpret_cast<int*>(blob + (kSmem ? a.max_blob : 0));
  const int64_t ioff = a.ilist_off[cta], ilen = a.ilist_len[cta];
  if (kSmem) async_copy_16(blob, a.vals + boff, blen / 2);
  async_copy_16(ilist, a.ilist + ioff, ilen / 4);
  const int lb = a.grp_level_base[grp];
  const int nlev = a.grp_level_base[grp + 1] - lb - 1;
  const double ft = a.ft_dev ? a.ft_dev[1] : a.ft;

  // Right-hand-side part that does not depend on the tree walk:
  // f_t(t_{n+1}) f_x^c - K^c u_pred, for every row this CTA owns.
  for (int l = 0; l < nlev; ++l) {
    const int qb = a.grp_level_ptr[lb + l], qe = a.grp_level_ptr[lb + l + 1];
    for (int q = qb + crank; q < qe; q += CL) {
      const int t = a.grp_level_nodes[q];
      const int beg = a.t_beg[t], b = a.t_end[t] - beg, slot = a.t_slot[t];
      for (int i = tid; i < b; i += kThreads) {
        const int r = beg + i;
        double s = ft * a.fxc[r];
        const int c0 = a.contrib_ptr[r], c1 = a.contrib_ptr[r + 1];
#pragma unroll 4
        for (int k = c0; k < c1; ++k) s -= a.Y[a.contrib_pos[k]];
        rhs[slot + i] = s;
      }
    }
  }
  async_copy_wait();
  const int* rptr = ilist;                      // row slot -> first position

  for (int l = 0; l < nlev; ++l) {
    const int qb = a.grp_level_ptr[lb + l], qe = a.grp_level_ptr[lb + l + 1];
    for (int q = qb + crank; q < qe; q += CL) {
      const int t = a.grp_level_nodes[q];
      const int beg = a.t_beg[t], b = a.t_end[t] - beg, m = a.t_nrows[t];
      const int ldi = b | 1, ldr = m | 1;            // odd leading dimensions
      const double* Li = Bf + a.t_foff[t];          // L_tt^{-1}: b x b, column-major, ld ldi
      const double* L21 = Li + (size_t)ldi * b;      // L_{rows,t}: m x b, column-major, ld ldr
      if (tid < b) {
        const int sl = a.t_slot[t] + tid;
        double s = rhs[sl];
        const int f0 = rptr[sl], f1 = rptr[sl + 1];
#pragma unroll 4
        for (int k = f0; k < f1; ++k) s -= __ldcg(a.upd + ilist[k]);
        g[tid] = s;
      }
      __syncthreads();
      {  // y = L_tt^{-1} g  (lower triangular)
        const int ch = (b + kWarps - 1) / kWarps;
        const int j0 = min(b, warp * ch), j1 = min(b, j0 + ch);
        warp_partial(Li, 1, ldi, b, g, j0, j1, 1, part + warp * W, lane);
      }
      __syncthreads();
      if (tid < b) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += part[w * W + tid];
        y[tid] = s;
        a.sol[beg + tid] = s;
      }
      __syncthreads();
      if (m > 0) {  // upd = L_{rows,t} y
        const int ch = (b + kWarps - 1) / kWarps;
        const int j0 = min(b, warp * ch), j1 = min(b, j0 + ch);
        warp_partial(L21, 1, ldr, m, y, j0, j1, 0, part + warp * W, lane);
        __syncthreads();
        if (tid < m) {
          double s = 0.0;
#pragma unroll
          for (int w = 0; w < kWarps; ++w) s += part[w * W + tid];
          a.upd[a.t_off_upd[t] + tid] = s;
        }
      }
      __syncthreads();
    }
    cluster.sync();
  }

  // Dense top of each component (the tree levels above the ones walked):
  // x_Z = A_Z (rhs_Z - updates from below), A_Z = (L_ZZ L_ZZ^T)^{-1}.
  {
    const int cb = a.grp_comp_ptr[grp], ce = a.grp_comp_ptr[grp + 1];
    for (int ci = cb; ci < ce; ++ci) {
      const int comp = a.grp_comps[ci], zn = a.zsize[comp], zb = a.zbase[comp];
      const int ch = (zn + CL - 1) / CL, i0 = min(zn, crank * ch), i1 = min(zn, i0 + ch);
      for (int i = i0 + tid; i < i1; i += kThreads) {
        const int r = a.zrow[zb + i];
        double s = ft * a.fxc[r];
        for (int k = a.contrib_ptr[r]; k < a.contrib_ptr[r + 1]; ++k) s -= a.Y[a.contrib_pos[k]];
        for (int k = a.zfwd_ptr[zb + i]; k < a.zfwd_ptr[zb + i + 1]; ++k) s -= __ldcg(a.upd + a.zfwd_pos[k]);
        a.zg[zb + i] = s;
      }
    }
    cluster.sync();
    double* zs = part + kWarps * W;   // max_zn doubles
    for (int ci = cb; ci < ce; ++ci) {
      const int comp = a.grp_comps[ci], zn = a.zsize[comp], zb = a.zbase[comp];
      if (zn == 0) continue;
      for (int j = tid; j < zn; j += kThreads) zs[j] = __ldcg(a.zg + zb + j);
      __syncthreads();
      const int ch = (zn + CL - 1) / CL, i0 = min(zn, crank * ch), i1 = min(zn, i0 + ch);
      const double* A = a.zA + a.zA_off[comp];
      for (int i = i0 + warp; i < i1; i += kWarps) {
        const double* Ar = A + (size_t)i * zn;
        double s0 = 0.0, s1 = 0.0;
        int j = lane;
        for (; j + 32 < zn; j += 64) {
          s0 = fma(__ldg(Ar + j), zs[j], s0);
          s1 = fma(__ldg(Ar + j + 32), zs[j + 32], s1);
        }
        if (j < zn) s0 = fma(__ldg(Ar + j), zs[j], s0);
        double v = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) a.sol[a.zrow[zb + i]] = v;
      }
      __syncthreads();
    }
    cluster.sync();
  }

  for (int l = nlev - 1; l >= 0; --l) {
    const int qb = a.grp_level_ptr[lb + l], qe = a.grp_level_ptr[lb + l + 1];
    for (int q = qb + crank; q < qe; q += CL) {
      const int t = a.grp_level_nodes[q];
      const int beg = a.t_beg[t], b = a.t_end[t] - beg, m = a.t_nrows[t];
      const int ldi = b | 1, ldr = m | 1;
      const double* Li = Bf + a.t_foff[t];           // read transposed below
      const double* L21 = Li + (size_t)ldi * b;
      const int* rows = ilist + a.t_roff[t];
      if (tid < m) xr[tid] = __ldcg(a.sol + rows[tid]);
      if (tid < b) y[tid] = __ldcg(a.sol + beg + tid);
      __syncthreads();
      if (m > 0) {  // h = y - L_{rows,t}^T x_rows
        const int ch = (m + kWarps - 1) / kWarps;
        const int k0 = min(m, warp * ch), k1 = min(m, k0 + ch);
        warp_partial(L21, ldr, 1, b, xr, k0, k1, 0, part + warp * W, lane);
        __syncthreads();
        if (tid < b) {
          double s = y[tid];
#pragma unroll
          for (int w = 0; w < kWarps; ++w) s -= part[w * W + tid];
          g[tid] = s;
        }
      } else if (tid < b) {
        g[tid] = y[tid];
      }
      __syncthreads();
      {  // x = L_tt^{-T} h  (upper triangular)
        const int ch = (b + kWarps - 1) / kWarps;
        const int j0 = min(b, warp * ch), j1 = min(b, j0 + ch);
        warp_partial(Li, ldi, 1, b, g, j0, j1, -1, part + warp * W, lane);
      }
      __syncthreads();
      if (tid < b) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += part[w * W + tid];
        a.sol[beg + tid] = s;
      }
      __syncthreads();
    }
    cluster.sync();
  }

  // Correction (Fig. TrapCDMIMEX) or the initial acceleration.
  const double bdt2 = kNewmarkBeta * a.dt * a.dt, gdt = kNewmarkGamma * a.dt,
               g1dt = (1.0 - kNewmarkGamma) * a.dt;
  for (int ci = a.grp_comp_ptr[grp]; ci < a.grp_comp_ptr[grp + 1]; ++ci) {
    const int comp = a.grp_comps[ci];
    for (int r = a.comp_cbeg[comp] + crank * kThreads + threadIdx.x; r < a.comp_cend[comp];
         r += CL * kThreads) {
      const double acc = __ldcg(a.sol + r);
      if (a.mode == 0) {
        const int node = a.c_node[r];
        const double vpred = a.v_c[r] + g1dt * a.a_c[r];
        a.U[node] = a.U[node] + bdt2 * acc;
        a.v_c[r] = vpred + gdt * acc;
      }
      a.a_c[r] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Small field kernels (layout conversion only).
__global__ void k_gather_c(double* dst, const double* src, const int* c_node, int n_c) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_c) dst[r] = src[c_node[r]];
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

int tile_cells(int P) {
  switch (P) {
    case 2: return 16;
    case 3: return 16;
    case 4: return 10;
    case 5: return 8;
    case 6: return 6;
    case 7: return 5;
    default: return 4;
  }
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
  double *winv_x = nullptr, *winv_y = nullptr;
  uint8_t* cls = nullptr;
  // implicit partition
  int* c_node = nullptr;
  double *v_c = nullptr, *a_c = nullptr, *fxc = nullptr;
  int *if_cell = nullptr, *if_kidx = nullptr;
  double *if_c2 = nullptr, *cutK = nullptr, *uncutK = nullptr, *Y = nullptr;
  int *t_beg = nullptr, *t_end = nullptr, *t_nrows = nullptr;
  int64_t *t_off_diag = nullptr, *t_off_diagT = nullptr, *t_off_rect = nullptr, *t_off_rows = nullptr,
          *t_off_upd = nullptr;
  int *rows_idx = nullptr, *grp_level_nodes = nullptr, *grp_level_ptr = nullptr, *grp_level_base = nullptr;
  int *grp_comp_ptr = nullptr, *grp_comps = nullptr;
  int64_t* t_off_rectT = nullptr;
  int ngroups = 0;
  int cluster = 8;
  int solve_width = 1;
  int solve_smem_mode = 0;
  int max_cta_rows = 1;
  double *S_blob = nullptr, *M_blob = nullptr;
  int64_t *blob_off = nullptr, *blob_len = nullptr, *t_foff = nullptr;
  int64_t *ilist_off = nullptr, *ilist_len = nullptr, *t_roff = nullptr;
  int* ilist = nullptr;
  int64_t max_blob = 0;
  int *zsize = nullptr, *zbase = nullptr, *zrow = nullptr, *zfwd_ptr = nullptr, *zfwd_pos = nullptr;
  int64_t* zA_off = nullptr;
  double *zA_S = nullptr, *zA_M = nullptr, *zg = nullptr;
  int max_zn = 0;
  int64_t nzrow = 0;
  int* t_slot = nullptr;
  int *comp_cbeg = nullptr, *comp_cend = nullptr;
  int *contrib_ptr = nullptr, *contrib_pos = nullptr, *fwd_ptr = nullptr, *fwd_pos = nullptr;
  double *upd = nullptr, *sol = nullptr;
  double *ft_buf = nullptr, *rec_buf = nullptr;
  int64_t* rec_nodes = nullptr;
  int io_cap = 4096;
  int cur = 0;              // U[cur] holds u_n
  int64_t step = 0;
  cudaStream_t stream = nullptr;
  Ops2D ops{};
  int TC = 4, ntx = 1, nty = 1;
  size_t smem_explicit = 0, smem_solve = 0;
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
  constexpr int TCs[10] = {0, 0, 16, 16, 10, 8, 6, 5, 4, 4};
  constexpr int TC = TCs[P];
  k_explicit2d<P, TC><<<grid, kThreads, c->smem_explicit, s>>>(ea, c->ops);
}

void explicit_dispatch(imex_ctx* c, const ExplicitArgs& ea, int grid, cudaStream_t s) {
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

template <int P>
cudaError_t set_explicit_smem(size_t bytes) {
  constexpr int TCs[10] = {0, 0, 16, 16, 10, 8, 6, 5, 4, 4};
  return cudaFuncSetAttribute(k_explicit2d<P, TCs[P]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

cudaError_t set_explicit_smem_dispatch(int P, size_t bytes) {
  switch (P) {
    case 2: return set_explicit_smem<2>(bytes);
    case 3: return set_explicit_smem<3>(bytes);
    case 4: return set_explicit_smem<4>(bytes);
    case 5: return set_explicit_smem<5>(bytes);
    case 6: return set_explicit_smem<6>(bytes);
    case 7: return set_explicit_smem<7>(bytes);
    case 8: return set_explicit_smem<8>(bytes);
    case 9: return set_explicit_smem<9>(bytes);
  }
  return cudaErrorInvalidValue;
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
  ea.winv_x = c->winv_x;
  ea.winv_y = c->winv_y;
  ea.nx = hs.nn[0];
  ea.ny = hs.nn[1];
  ea.ncx = hs.pb.ncells[0];
  ea.ncy = hs.pb.ncells[1];
  ea.ntx = c->ntx;
  ea.nty = c->nty;
  ea.cu = cu;
  ea.cw = cw;
  ea.ca = ca;
  ea.ft = ft;
  ea.n_c = predict ? (int)hs.n_c : 0;
  ea.c_node = c->c_node;
  ea.v_c = c->v_c;
  ea.a_c = c->a_c;
  ea.dt = hs.dt;
  return ea;
}

int pred_blocks(imex_ctx* c, bool predict) {
  if (!predict || c->hs.n_c == 0) return 0;
  return (int)std::min<int64_t>(152, (c->hs.n_c + kThreads - 1) / kThreads);
}

IfaceArgs iface_args(imex_ctx* c, const double* src) {
  const HostSetup& hs = c->hs;
  IfaceArgs ia{};
  ia.SRC = src;
  ia.cell = c->if_cell;
  ia.kidx = c->if_kidx;
  ia.c2 = c->if_c2;
  ia.cutK = c->cutK;
  ia.uncutK = c->uncutK;
  ia.Y = c->Y;
  ia.n_iface = (int)hs.if_cell.size();
  ia.dim = hs.dim;
  ia.p = hs.p;
  ia.P = hs.P;
  ia.Pd = hs.Pd;
  ia.ncx = hs.pb.ncells[0];
  ia.ncy = hs.pb.ncells[1];
  ia.nx = hs.nn[0];
  ia.ny = hs.nn[1];
  return ia;
}

SolveArgs solve_args(imex_ctx* c, bool use_S, double ft, int mode, double* Ubuf) {
  SolveArgs sa{};
  sa.vals = use_S ? c->S_blob : c->M_blob;
  sa.blob_off = c->blob_off;
  sa.blob_len = c->blob_len;
  sa.t_foff = c->t_foff;
  sa.t_roff = c->t_roff;
  sa.ilist = c->ilist;
  sa.ilist_off = c->ilist_off;
  sa.ilist_len = c->ilist_len;
  sa.max_blob = c->max_blob;
  sa.zsize = c->zsize;
  sa.zbase = c->zbase;
  sa.zrow = c->zrow;
  sa.zA = use_S ? c->zA_S : c->zA_M;
  sa.zA_off = c->zA_off;
  sa.zfwd_ptr = c->zfwd_ptr;
  sa.zfwd_pos = c->zfwd_pos;
  sa.zg = c->zg;
  sa.max_zn = c->max_zn;
  sa.t_slot = c->t_slot;
  sa.max_cta_rows = c->max_cta_rows;
  sa.t_beg = c->t_beg;
  sa.t_end = c->t_end;
  sa.t_nrows = c->t_nrows;
  sa.t_off_diag = c->t_off_diag;
  sa.t_off_diagT = c->t_off_diagT;
  sa.t_off_rect = c->t_off_rect;
  sa.t_off_rows = c->t_off_rows;
  sa.t_off_upd = c->t_off_upd;
  sa.t_off_rectT = c->t_off_rectT;
  sa.rows_idx = c->rows_idx;
  sa.grp_level_nodes = c->grp_level_nodes;
  sa.grp_level_ptr = c->grp_level_ptr;
  sa.grp_level_base = c->grp_level_base;
  sa.grp_comp_ptr = c->grp_comp_ptr;
  sa.grp_comps = c->grp_comps;
  sa.comp_cbeg = c->comp_cbeg;
  sa.comp_cend = c->comp_cend;
  sa.contrib_ptr = c->contrib_ptr;
  sa.contrib_pos = c->contrib_pos;
  sa.Y = c->Y;
  sa.fwd_ptr = c->fwd_ptr;
  sa.fwd_pos = c->fwd_pos;
  sa.upd = c->upd;
  sa.sol = c->sol;
  sa.fxc = c->fxc;
  sa.ft = ft;
  sa.mode = mode;
  sa.c_node = c->c_node;
  sa.U = Ubuf;
  sa.v_c = c->v_c;
  sa.a_c = c->a_c;
  sa.dt = c->hs.dt;
  sa.max_width = c->solve_width;
  return sa;
}

cudaError_t launch_solve(imex_ctx* c, const SolveArgs& sa, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->ngroups * c->cluster);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = c->smem_solve;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c->cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return c->solve_smem_mode ? cudaLaunchKernelEx(&cfg, k_solve<true>, sa)
                            : cudaLaunchKernelEx(&cfg, k_solve<false>, sa);
}

// How many clusters of `cl` CTAs with `smem` bytes each the device co-schedules.
int max_clusters(int cl, size_t smem) {
  for (auto fn : {k_solve<true>, k_solve<false>}) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmemBudget) != cudaSuccess)
      return 0;
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  cudaGetLastError();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_solve<true>, &cfg) != cudaSuccess) n = 0;
  cudaGetLastError();
  return n;
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
  explicit_dispatch(c, ea, c->ntx * c->nty, s);
  if (int rc = check_launch("explicit (initial)")) return rc;
  if (hs.n_c > 0) {
    const int nc = (int)hs.n_c;
    k_gather_c<<<(nc + 255) / 256, 256, 0, s>>>(c->v_c, c->tmp, c->c_node, nc);
    const int nif = (int)hs.if_cell.size();
    IfaceArgs ia = iface_args(c, U0);
    k_iface<<<(nif + kWarps - 1) / kWarps, kThreads, 0, s>>>(ia);
    if (int rc = check_launch("iface (initial)")) return rc;
    SolveArgs sa = solve_args(c, false, ft0, 1, U0);
    if (cudaError_t e = launch_solve(c, sa, s)) return fail(IMEX_ERR_CUDA, std::string("solve (initial): ") + cudaGetErrorString(e));
    if (int rc = check_launch("solve (initial)")) return rc;
  }
  return IMEX_OK;
}

// Static schedule of the implicit solve.  Components are bin-packed into
// groups (one cluster each), largest factor first onto the lightest group;
// each level's nodes are sorted by decreasing work and dealt to the cluster's
// CTAs round-robin.  Every CTA gets one blob holding, in the order it visits
// them, each of its nodes' [L_tt^{-1} (ld b|1) | L_{rows,t} (ld m|1)],
// 16-byte aligned, for both S and M^cc.  The plan tries shared-memory budgets
// from small (more co-resident clusters) to large and keeps the first whose
// largest blob fits; otherwise the blobs are read from global memory.
struct SolvePlan {
  std::vector<int> gl_nodes, gl_ptr, gl_base, gc_ptr, gc_list, slot, ilist;
  std::vector<int64_t> b_off, b_len, foff, i_off, i_len, roff;
  std::vector<double> blobS, blobM;
  int64_t max_blob = 0;
  // dense top part per component
  std::vector<int> lz, zsize, zbase, zrow, zfwd_ptr, zfwd_pos;
  std::vector<int64_t> zA_off;
  std::vector<double> zA_S, zA_M;
  int max_zn = 0;
};

constexpr int kZmax = 400;   // largest dense top block per component

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

int plan_solve(imex_ctx* c, SolvePlan& best) {
  const HostSetup& hs = c->hs;
  const int64_t nt = (int64_t)hs.tree.size();
  auto node_work = [&](int t) {
    const TreeNode& T = hs.tree[t];
    const int64_t b = T.end - T.beg, m = (int64_t)T.rows.size();
    return b * b + m * b;
  };
  std::vector<int64_t> cw(hs.ncomp, 0);
  for (int k = 0; k < hs.ncomp; ++k)
    for (int t = hs.comp_tree_ptr[k]; t < hs.comp_tree_ptr[k + 1]; ++t) cw[k] += node_work(t);
  // Split level of each component: nodes at level >= lz form the dense top part.
  std::vector<int> lz(hs.ncomp, 1), zsize(hs.ncomp, 0), zbase(hs.ncomp, 0), zrow, zpos(hs.n_c, -1);
  std::vector<int64_t> zA_off(hs.ncomp, 0);
  std::vector<double> zA_S, zA_M;
  int max_zn = 0;
  {
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
      zA_off[k] = (int64_t)zA_S.size();
      if (zsize[k] > 0) {
        std::vector<double> A;
        dense_top(hs, hs.S, znodes, zpos, zsize[k], A);
        zA_S.insert(zA_S.end(), A.begin(), A.end());
        dense_top(hs, hs.Mcc, znodes, zpos, zsize[k], A);
        zA_M.insert(zA_M.end(), A.begin(), A.end());
      }
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
  const size_t vec_doubles = (size_t)(3 + kWarps) * c->solve_width + (size_t)((max_zn + 1) / 2) * 2;
  bool have = false;
  for (int cl : {16, 8}) {
    for (int budget_kb : {64, 96, 128, 160, 200}) {
      const size_t budget = (size_t)budget_kb * 1024;
      const int nclu = max_clusters(cl, budget);
      if (nclu <= 0) continue;
      SolvePlan P;
      const int ngroups = std::max(1, std::min(hs.ncomp, nclu));
      std::vector<int> order(hs.ncomp);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](int x, int y) { return cw[x] > cw[y]; });
      std::vector<std::vector<int>> members(ngroups);
      std::vector<int64_t> load(ngroups, 0);
      for (int k : order) {
        int gsel = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        members[gsel].push_back(k);
        load[gsel] += cw[k];
      }
      P.gc_ptr.push_back(0);
      for (int gi = 0; gi < ngroups; ++gi) {
        int nl = 0;
        for (int k : members[gi]) {
          P.gc_list.push_back(k);
          for (int t = hs.comp_tree_ptr[k]; t < hs.comp_tree_ptr[k + 1]; ++t) nl = std::max(nl, hs.tree[t].level + 1);
        }
        P.gc_ptr.push_back((int)P.gc_list.size());
        std::vector<std::vector<int>> byl(nl);
        for (int k : members[gi])
          for (int t = hs.comp_tree_ptr[k]; t < hs.comp_tree_ptr[k + 1]; ++t)
            if (!is_top(t)) byl[hs.tree[t].level].push_back(t);
        while (!byl.empty() && byl.back().empty()) byl.pop_back();
        nl = (int)byl.size();
        P.gl_base.push_back((int)P.gl_ptr.size());
        P.gl_ptr.push_back((int)P.gl_nodes.size());
        for (int l = 0; l < nl; ++l) {
          std::sort(byl[l].begin(), byl[l].end(), [&](int x, int y) { return node_work(x) > node_work(y); });
          P.gl_nodes.insert(P.gl_nodes.end(), byl[l].begin(), byl[l].end());
          P.gl_ptr.push_back((int)P.gl_nodes.size());
        }
      }
      P.gl_base.push_back((int)P.gl_ptr.size());
      P.b_off.assign((size_t)ngroups * cl, 0);
      P.b_len.assign((size_t)ngroups * cl, 0);
      P.foff.assign(nt, 0);
      P.slot.assign(nt, 0);
      P.roff.assign(nt, 0);
      P.i_off.assign((size_t)ngroups * cl, 0);
      P.i_len.assign((size_t)ngroups * cl, 0);
      int max_rows = 2;
      int64_t max_blob = 0, max_ilist = 0;
      for (int gi = 0; gi < ngroups; ++gi) {
        const int nlv = P.gl_base[gi + 1] - P.gl_base[gi] - 1;
        for (int rk = 0; rk < cl; ++rk) {
          const int cta = gi * cl + rk;
          int rows_here = 0;
          if (P.blobS.size() % 2) { P.blobS.push_back(0.0); P.blobM.push_back(0.0); }
          P.b_off[cta] = (int64_t)P.blobS.size();
          int64_t local = 0;
          for (int l = 0; l < nlv; ++l) {
            const int qb = P.gl_ptr[P.gl_base[gi] + l], qe = P.gl_ptr[P.gl_base[gi] + l + 1];
            for (int q = qb + rk; q < qe; q += cl) {
              const int t = P.gl_nodes[q];
              const TreeNode& T = hs.tree[t];
              const int b = T.end - T.beg, m = (int)T.rows.size();
              const int ldi = b | 1, ldr = m | 1;
              P.slot[t] = rows_here;
              rows_here += b;
              P.foff[t] = local;
              for (const Factor* F : {&hs.S, &hs.Mcc}) {
                std::vector<double>& out = (F == &hs.S) ? P.blobS : P.blobM;
                const double* Li = F->vals.data() + T.off_diag;
                const double* L21 = F->vals.data() + T.off_rect;
                for (int j = 0; j < b; ++j)
                  for (int i = 0; i < ldi; ++i) out.push_back(i < b ? Li[i + (size_t)b * j] : 0.0);
                for (int j = 0; j < b; ++j)
                  for (int i = 0; i < ldr; ++i) out.push_back(i < m ? L21[i + (size_t)m * j] : 0.0);
              }
              local += (int64_t)ldi * b + (int64_t)ldr * b;
            }
          }
          if (local % 2) { P.blobS.push_back(0.0); P.blobM.push_back(0.0); ++local; }
          P.b_len[cta] = local;
          max_blob = std::max(max_blob, local);
          max_rows = std::max(max_rows, rows_here + (rows_here & 1));
          // Index lists of this CTA: [row ptr (rows_here + 1) | positions | ancestor rows].
          std::vector<int> mine;
          for (int l = 0; l < nlv; ++l) {
            const int qb = P.gl_ptr[P.gl_base[gi] + l], qe = P.gl_ptr[P.gl_base[gi] + l + 1];
            for (int q = qb + rk; q < qe; q += cl) mine.push_back(P.gl_nodes[q]);
          }
          std::vector<int> rp(1, 0), pos, anc;
          for (int t : mine)
            for (int r = hs.tree[t].beg; r < hs.tree[t].end; ++r) {
              for (int k = hs.fwd_ptr[r]; k < hs.fwd_ptr[r + 1]; ++k) pos.push_back(hs.fwd_pos[k]);
              rp.push_back((int)pos.size());
            }
          const int npos_base = (int)rp.size();
          for (int& v : rp) v += npos_base;            // positions follow the row pointers
          std::vector<int> lst = rp;
          lst.insert(lst.end(), pos.begin(), pos.end());
          for (int t : mine) {
            P.roff[t] = (int64_t)lst.size();
            lst.insert(lst.end(), hs.tree[t].rows.begin(), hs.tree[t].rows.end());
          }
          while (lst.size() % 4) lst.push_back(0);
          while (P.ilist.size() % 4) P.ilist.push_back(0);
          P.i_off[cta] = (int64_t)P.ilist.size();
          P.i_len[cta] = (int64_t)lst.size();
          P.ilist.insert(P.ilist.end(), lst.begin(), lst.end());
          max_ilist = std::max(max_ilist, (int64_t)lst.size());
        }
      }
      const size_t ibytes = (size_t)max_ilist * sizeof(int);
      const size_t need = (vec_doubles + (size_t)max_rows + (size_t)max_blob) * sizeof(double) + ibytes;
      const bool fits = need <= budget;
      P.max_blob = max_blob;
      P.lz = lz;
      P.zsize = zsize;
      P.zbase = zbase;
      P.zrow = zrow;
      P.zfwd_ptr = zfwd_ptr;
      P.zfwd_pos = zfwd_pos;
      P.zA_off = zA_off;
      P.max_zn = max_zn;
      if (fits || (!have && budget_kb == 200 && cl == 8)) {
        c->max_zn = ((max_zn + 1) / 2) * 2;
        c->cluster = cl;
        c->ngroups = ngroups;
        c->max_cta_rows = max_rows;
        c->solve_smem_mode = fits ? 1 : 0;
        c->smem_solve = fits ? need : (vec_doubles + (size_t)max_rows) * sizeof(double) + ibytes;
        c->max_blob = fits ? max_blob : 0;
        P.zA_S = zA_S;
        P.zA_M = zA_M;
        best = std::move(P);
        have = true;
        if (fits) return IMEX_OK;
      }
    }
    if (have && c->solve_smem_mode) break;
  }
  if (!have) return fail(IMEX_ERR_CUDA, "no thread-block cluster configuration fits the solve kernel");
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

static void fill_stats(const HostSetup& hs, imex_stats* st) {
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
    return IMEX_OK;
  } catch (const std::exception& ex) {
    return fail(IMEX_ERR_ALLOC, std::string("host setup failed: ") + ex.what());
  }
}

int imex_setup(const imex_mesh* mesh, int p, double alpha, double dt, const imex_source* src,
               const imex_alloc* alloc, imex_ctx** out) {
  if (!out) return fail(IMEX_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  imex_ctx* c = nullptr;
  try {
    Problem pb;
    if (int rc = build_context(mesh, p, alpha, dt, src, pb)) return rc;
    if (pb.dim != 2) return fail(IMEX_ERR_ARG, "the GPU time stepper supports dim = 2");
    c = new imex_ctx();
    std::string err = build_setup(pb, c->hs);
    if (!err.empty()) {
      delete c;
      return fail(setup_error_code(err), err);
    }
    HostSetup& hs = c->hs;
    if (hs.max_block > kMaxWidth || hs.max_rows > kMaxWidth) {
      delete c;
      return fail(IMEX_ERR_ARG, "supernode too large for the device solve (max 256)");
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
      delete c;
      return fail(IMEX_ERR_CUDA, "no CUDA device");
    }
    const int P = hs.P;
    c->TC = tile_cells(P);
    const int OX = c->TC * hs.p;
    c->ntx = (hs.nn[0] + OX - 1) / OX;
    c->nty = (hs.nn[1] + OX - 1) / OX;
    c->smem_explicit = explicit_smem_doubles(P, c->TC) * sizeof(double);
    c->solve_width = std::max(1, std::max(hs.max_block, hs.max_rows));
    c->solve_width += c->solve_width % 2;

    // Operators of the explicit apply: sx = rho c^2 h_y / h_x, sy = rho c^2 h_x / h_y.
    const double sx = pb.rho * pb.c0 * pb.c0 * hs.h[1] / hs.h[0];
    const double sy = pb.rho * pb.c0 * pb.c0 * hs.h[0] / hs.h[1];
    for (int i = 0; i < P * P; ++i) {
      c->ops.kx[i] = sx * hs.K1[i];
      c->ops.mx[i] = hs.M1[i];
      c->ops.my[i] = hs.M1[i];
      c->ops.ky[i] = sy * hs.K1[i];
    }
    if (!pb.cell_c.empty()) {
      delete c;
      return fail(IMEX_ERR_ARG, "per-cell wave speed is not supported by the 2D explicit kernel");
    }
    // Assembled GLL weights per node column/row; lumped mass = rho |J| W_x W_y.
    std::vector<double> wx(hs.nn[0]), wy(hs.nn[1]);
    auto assembled = [&](int i, int n) {
      const int loc = i % hs.p;
      if (loc != 0) return hs.gll_w[loc];
      double w = 0.0;
      if (i > 0) w += hs.gll_w[hs.p];
      if (i < n - 1) w += hs.gll_w[0];
      return w;
    };
    const double jac = 0.25 * hs.h[0] * hs.h[1];
    for (int i = 0; i < hs.nn[0]; ++i) wx[i] = 1.0 / assembled(i, hs.nn[0]);
    for (int i = 0; i < hs.nn[1]; ++i) wy[i] = 1.0 / (assembled(i, hs.nn[1]) * pb.rho * jac);

    // Compact per-c arrays and tree metadata.
    const int64_t nn = hs.nnodes, nc = hs.n_c, nt = (int64_t)hs.tree.size();
    std::vector<double> fxc(nc);
    for (int64_t r = 0; r < nc; ++r) fxc[r] = hs.fx[hs.c_node[r]];
    std::vector<int> tb(nt), te(nt), tn(nt);
    std::vector<int64_t> od(nt), odT(nt), orc(nt), orw(nt), ou(nt);
    for (int64_t t = 0; t < nt; ++t) {
      const TreeNode& T = hs.tree[t];
      tb[t] = T.beg;
      te[t] = T.end;
      tn[t] = (int)T.rows.size();
      od[t] = T.off_diag;
      odT[t] = T.off_diagT;
      orc[t] = T.off_rect;
      orw[t] = T.off_rows;
      ou[t] = T.off_upd;
    }
    std::vector<int> ccb(hs.ncomp), cce(hs.ncomp);
    for (int k = 0; k < hs.ncomp; ++k) {
      ccb[k] = hs.tree[hs.comp_tree_ptr[k]].beg;
      cce[k] = hs.tree[hs.comp_tree_ptr[k + 1] - 1].end;
    }
    std::vector<int64_t> off_rT(nt);
    for (int64_t t = 0; t < nt; ++t) off_rT[t] = hs.tree[t].off_rectT;
    SolvePlan plan;
    if (int rc = plan_solve(c, plan)) {
      imex_destroy(c);
      return rc;
    }
    const int64_t nif = (int64_t)hs.if_cell.size();

    Arena ar;
    ar.add(&c->U[0], nn);
    ar.add(&c->U[1], nn);
    ar.add(&c->tmp, nn);
    ar.add(&c->fx, nn);
    ar.add(&c->winv_x, hs.nn[0]);
    ar.add(&c->winv_y, hs.nn[1]);
    ar.add(&c->cls, nn);
    ar.add(&c->c_node, std::max<int64_t>(nc, 1));
    ar.add(&c->v_c, std::max<int64_t>(nc, 1));
    ar.add(&c->a_c, std::max<int64_t>(nc, 1));
    ar.add(&c->fxc, std::max<int64_t>(nc, 1));
    ar.add(&c->sol, std::max<int64_t>(nc, 1));
    ar.add(&c->if_cell, std::max<int64_t>(nif, 1));
    ar.add(&c->if_kidx, std::max<int64_t>(nif, 1));
    ar.add(&c->if_c2, std::max<int64_t>(nif, 1));
    ar.add(&c->cutK, std::max<size_t>(hs.cutK.size(), 1));
    ar.add(&c->uncutK, hs.uncutK.size());
    ar.add(&c->Y, std::max<int64_t>(nif * hs.Pd, 1));
    ar.add(&c->S_blob, std::max<size_t>(plan.blobS.size(), 2));
    ar.add(&c->M_blob, std::max<size_t>(plan.blobM.size(), 2));
    ar.add(&c->blob_off, std::max<size_t>(plan.b_off.size(), 1));
    ar.add(&c->blob_len, std::max<size_t>(plan.b_len.size(), 1));
    ar.add(&c->t_foff, std::max<int64_t>(nt, 1));
    ar.add(&c->t_slot, std::max<int64_t>(nt, 1));
    ar.add(&c->t_roff, std::max<int64_t>(nt, 1));
    ar.add(&c->ilist, std::max<size_t>(plan.ilist.size(), 4));
    ar.add(&c->ilist_off, std::max<size_t>(plan.i_off.size(), 1));
    ar.add(&c->ilist_len, std::max<size_t>(plan.i_len.size(), 1));
    ar.add(&c->zsize, std::max<size_t>(plan.zsize.size(), 1));
    ar.add(&c->zbase, std::max<size_t>(plan.zbase.size(), 1));
    ar.add(&c->zrow, std::max<size_t>(plan.zrow.size(), 1));
    ar.add(&c->zfwd_ptr, std::max<size_t>(plan.zfwd_ptr.size(), 1));
    ar.add(&c->zfwd_pos, std::max<size_t>(plan.zfwd_pos.size(), 1));
    ar.add(&c->zA_off, std::max<size_t>(plan.zA_off.size(), 1));
    ar.add(&c->zA_S, std::max<size_t>(plan.zA_S.size(), 1));
    ar.add(&c->zA_M, std::max<size_t>(plan.zA_M.size(), 1));
    ar.add(&c->zg, std::max<size_t>(plan.zrow.size(), 1));
    ar.add(&c->t_beg, std::max<int64_t>(nt, 1));
    ar.add(&c->t_end, std::max<int64_t>(nt, 1));
    ar.add(&c->t_nrows, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_diag, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_diagT, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_rect, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_rows, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_upd, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_rectT, std::max<int64_t>(nt, 1));
    ar.add(&c->rows_idx, std::max<size_t>(hs.rows_idx.size(), 1));
    ar.add(&c->grp_level_nodes, std::max<size_t>(plan.gl_nodes.size(), 1));
    ar.add(&c->grp_level_ptr, std::max<size_t>(plan.gl_ptr.size(), 1));
    ar.add(&c->grp_level_base, std::max<size_t>(plan.gl_base.size(), 1));
    ar.add(&c->grp_comp_ptr, std::max<size_t>(plan.gc_ptr.size(), 1));
    ar.add(&c->grp_comps, std::max<size_t>(plan.gc_list.size(), 1));
    ar.add(&c->comp_cbeg, std::max(hs.ncomp, 1));
    ar.add(&c->comp_cend, std::max(hs.ncomp, 1));
    ar.add(&c->contrib_ptr, hs.contrib_ptr.size());
    ar.add(&c->contrib_pos, std::max<size_t>(hs.contrib_pos.size(), 1));
    ar.add(&c->fwd_ptr, hs.fwd_ptr.size());
    ar.add(&c->fwd_pos, std::max<size_t>(hs.fwd_pos.size(), 1));
    ar.add(&c->upd, std::max<int64_t>(hs.upd_size, 1));
    ar.add(&c->ft_buf, 2);
    ar.add(&c->rec_buf, c->io_cap);
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
    e = e ? e : upload(c->winv_x, wx);
    e = e ? e : upload(c->winv_y, wy);
    e = e ? e : upload(c->cls, hs.node_class);
    e = e ? e : upload(c->c_node, hs.c_node);
    e = e ? e : upload(c->fxc, fxc);
    e = e ? e : upload(c->if_cell, hs.if_cell);
    e = e ? e : upload(c->if_kidx, hs.if_kidx);
    e = e ? e : upload(c->if_c2, hs.if_c2);
    e = e ? e : upload(c->cutK, hs.cutK);
    e = e ? e : upload(c->uncutK, hs.uncutK);
    e = e ? e : upload(c->S_blob, plan.blobS);
    e = e ? e : upload(c->M_blob, plan.blobM);
    e = e ? e : upload(c->blob_off, plan.b_off);
    e = e ? e : upload(c->blob_len, plan.b_len);
    e = e ? e : upload(c->t_foff, plan.foff);
    e = e ? e : upload(c->t_slot, plan.slot);
    e = e ? e : upload(c->t_roff, plan.roff);
    e = e ? e : upload(c->ilist, plan.ilist);
    e = e ? e : upload(c->ilist_off, plan.i_off);
    e = e ? e : upload(c->ilist_len, plan.i_len);
    e = e ? e : upload(c->zsize, plan.zsize);
    e = e ? e : upload(c->zbase, plan.zbase);
    e = e ? e : upload(c->zrow, plan.zrow);
    e = e ? e : upload(c->zfwd_ptr, plan.zfwd_ptr);
    e = e ? e : upload(c->zfwd_pos, plan.zfwd_pos);
    e = e ? e : upload(c->zA_off, plan.zA_off);
    e = e ? e : upload(c->zA_S, plan.zA_S);
    e = e ? e : upload(c->zA_M, plan.zA_M);
    c->nzrow = (int64_t)plan.zrow.size();
    e = e ? e : upload(c->t_beg, tb);
    e = e ? e : upload(c->t_end, te);
    e = e ? e : upload(c->t_nrows, tn);
    e = e ? e : upload(c->t_off_diag, od);
    e = e ? e : upload(c->t_off_diagT, odT);
    e = e ? e : upload(c->t_off_rect, orc);
    e = e ? e : upload(c->t_off_rows, orw);
    e = e ? e : upload(c->t_off_upd, ou);
    e = e ? e : upload(c->t_off_rectT, off_rT);
    e = e ? e : upload(c->rows_idx, hs.rows_idx);
    e = e ? e : upload(c->grp_level_nodes, plan.gl_nodes);
    e = e ? e : upload(c->grp_level_ptr, plan.gl_ptr);
    e = e ? e : upload(c->grp_level_base, plan.gl_base);
    e = e ? e : upload(c->grp_comp_ptr, plan.gc_ptr);
    e = e ? e : upload(c->grp_comps, plan.gc_list);
    e = e ? e : upload(c->comp_cbeg, ccb);
    e = e ? e : upload(c->comp_cend, cce);
    e = e ? e : upload(c->contrib_ptr, hs.contrib_ptr);
    e = e ? e : upload(c->contrib_pos, hs.contrib_pos);
    e = e ? e : upload(c->fwd_ptr, hs.fwd_ptr);
    e = e ? e : upload(c->fwd_pos, hs.fwd_pos);
    e = e ? e : set_explicit_smem_dispatch(P, c->smem_explicit);
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
    *out = c;
    return IMEX_OK;
  } catch (const std::exception& ex) {
    delete c;
    return fail(IMEX_ERR_ALLOC, std::string("setup failed: ") + ex.what());
  }
}

// One IMEX step n -> n+1 on stream s; events (may be NULL) are recorded before
// the explicit kernel and after each of the three kernels.
static int step_once(imex_ctx* c, cudaStream_t s, cudaEvent_t* ev, const double* ft_dev = nullptr) {
  const HostSetup& hs = c->hs;
  const double dt = hs.dt;
  double* Ucur = c->U[c->cur];
  double* Unext = c->U[1 - c->cur];
  const int64_t step = c->step;
  const int nif = (int)hs.if_cell.size();
  if (ev) cudaEventRecord(ev[0], s);
  ExplicitArgs ea = explicit_args(c, Ucur, Unext, Unext, 2.0, -1.0, dt * dt, ft_at(hs, step), true);
  ea.ft_dev = ft_dev;
  explicit_dispatch(c, ea, c->ntx * c->nty + pred_blocks(c, true), s);
  if (ev) cudaEventRecord(ev[1], s);
  if (hs.n_c > 0) {
    IfaceArgs ia = iface_args(c, Unext);
    k_iface<<<(nif + kWarps - 1) / kWarps, kThreads, 0, s>>>(ia);
    if (ev) cudaEventRecord(ev[2], s);
    SolveArgs sa = solve_args(c, true, ft_at(hs, step + 1), 0, Unext);
    sa.ft_dev = ft_dev;
    launch_solve(c, sa, s);
  } else if (ev) {
    cudaEventRecord(ev[2], s);
  }
  if (ev) cudaEventRecord(ev[3], s);
  if (int rc = check_launch("imex_step")) return rc;
  c->cur = 1 - c->cur;
  c->step = step + 1;
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
  cudaEvent_t ev[4];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(IMEX_ERR_CUDA, "cudaEventCreate failed");
  double acc[3] = {0, 0, 0};
  int rc = IMEX_OK;
  for (int64_t k = 0; k < n && rc == IMEX_OK; ++k) {
    rc = step_once(c, s, ev);
    if (rc) break;
    if (cudaEventSynchronize(ev[3]) != cudaSuccess) {
      rc = fail(IMEX_ERR_CUDA, "imex_step_profile: synchronisation failed");
      break;
    }
    for (int ph = 0; ph < 3; ++ph) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]);
      acc[ph] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (int ph = 0; ph < 3; ++ph) phase_ms[ph] = acc[ph];
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
  if (nrec > 0) e = cudaMemcpyAsync(c->rec_nodes, rec_nodes, nrec * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  for (int64_t k = 0; k < n && e == cudaSuccess; ++k) {
    const double* ftd = nullptr;
    if (ft_samples) {
      e = cudaMemcpyAsync(c->ft_buf, ft_samples + k, 2 * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) break;
      ftd = c->ft_buf;
    }
    if (int rc = step_once(c, s, nullptr, ftd)) return rc;
    if (nrec > 0) {
      k_gather_nodes<<<(nrec + 255) / 256, 256, 0, s>>>(c->rec_buf, c->U[c->cur], c->rec_nodes, nrec);
      e = cudaMemcpyAsync(traces + k * nrec, c->rec_buf, nrec * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    // ft_buf is rewritten by the next step's copy, which the stream orders
    // after this step's kernels.
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_step_io: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

static int field_io_check(imex_ctx* c, int64_t len) {
  if (!c) return fail(IMEX_ERR_ARG, "NULL context");
  if (len != c->hs.nnodes) return fail(IMEX_ERR_ARG, "len must equal n_nodes");
  return IMEX_OK;
}

int imex_fields(imex_ctx* c, int which, double* dst, int64_t len, int dst_on_device) {
  if (int rc = field_io_check(c, len)) return rc;
  if (!dst) return fail(IMEX_ERR_ARG, "NULL destination");
  cudaStream_t s = c->stream;
  const int64_t n = c->hs.nnodes;
  const int nb = (int)((n + 255) / 256);
  const int nc = (int)c->hs.n_c;
  double* out = c->tmp;
  switch (which) {
    case IMEX_FIELD_U: k_masked<<<nb, 256, 0, s>>>(out, c->U[c->cur], c->cls, n, 3); break;
    case IMEX_FIELD_U_PREV_D: k_masked<<<nb, 256, 0, s>>>(out, c->U[1 - c->cur], c->cls, n, 1); break;
    case IMEX_FIELD_V_C:
    case IMEX_FIELD_A_C:
      cudaMemsetAsync(out, 0, n * sizeof(double), s);
      if (nc > 0)
        k_scatter_c<<<(nc + 255) / 256, 256, 0, s>>>(out, which == IMEX_FIELD_V_C ? c->v_c : c->a_c,
                                                     c->c_node, nc);
      break;
    case IMEX_FIELD_FX: k_masked<<<nb, 256, 0, s>>>(out, c->fx, c->cls, n, 3); break;
    case IMEX_FIELD_MASK_D: k_masked<<<nb, 256, 0, s>>>(out, c->fx, c->cls, n, 4); break;
    case IMEX_FIELD_MASK_C: k_masked<<<nb, 256, 0, s>>>(out, c->fx, c->cls, n, 5); break;
    default: return fail(IMEX_ERR_ARG, "unknown field");
  }
  if (int rc = check_launch("imex_fields")) return rc;
  cudaError_t e = cudaMemcpyAsync(dst, out, n * sizeof(double),
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_fields: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_set_fields(imex_ctx* c, int which, const double* src, int64_t len, int src_on_device) {
  if (int rc = field_io_check(c, len)) return rc;
  if (!src) return fail(IMEX_ERR_ARG, "NULL source");
  cudaStream_t s = c->stream;
  const int64_t n = c->hs.nnodes;
  const int nb = (int)((n + 255) / 256);
  const int nc = (int)c->hs.n_c;
  cudaError_t e = cudaMemcpyAsync(c->tmp, src, n * sizeof(double),
                                  src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_fields: ") + cudaGetErrorString(e));
  switch (which) {
    case IMEX_FIELD_U:
      k_masked_set<<<nb, 256, 0, s>>>(c->U[c->cur], c->tmp, c->cls, n, NODE_D);
      k_masked_set<<<nb, 256, 0, s>>>(c->U[c->cur], c->tmp, c->cls, n, NODE_C);
      break;
    case IMEX_FIELD_U_PREV_D: k_masked_set<<<nb, 256, 0, s>>>(c->U[1 - c->cur], c->tmp, c->cls, n, NODE_D); break;
    case IMEX_FIELD_V_C:
    case IMEX_FIELD_A_C:
      if (nc > 0)
        k_gather_c<<<(nc + 255) / 256, 256, 0, s>>>(which == IMEX_FIELD_V_C ? c->v_c : c->a_c, c->tmp,
                                                    c->c_node, nc);
      break;
    default: return fail(IMEX_ERR_ARG, "field is not settable");
  }
  if (int rc = check_launch("imex_set_fields")) return rc;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_fields: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_set_step(imex_ctx* c, int64_t n) {
  if (!c || n < 0) return fail(IMEX_ERR_ARG, "bad arguments");
  c->step = n;
  return IMEX_OK;
}

int imex_set_initial(imex_ctx* c, const double* u0, const double* v0, int64_t len, int on_device) {
  if (int rc = field_io_check(c, len)) return rc;
  if (!u0) return fail(IMEX_ERR_ARG, "NULL u0");
  cudaStream_t s = c->stream;
  const int64_t n = c->hs.nnodes;
  const int nb = (int)((n + 255) / 256);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(c->tmp, u0, n * sizeof(double), kind, s);
  if (e == cudaSuccess) {
    c->cur = 0;
    k_masked<<<nb, 256, 0, s>>>(c->U[0], c->tmp, c->cls, n, 3);
    e = v0 ? cudaMemcpyAsync(c->tmp, v0, n * sizeof(double), kind, s)
           : cudaMemsetAsync(c->tmp, 0, n * sizeof(double), s);
  }
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_initial: ") + cudaGetErrorString(e));
  c->step = 0;
  if (int rc = compute_initial(c, s)) return rc;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(IMEX_ERR_CUDA, std::string("imex_set_initial: ") + cudaGetErrorString(e));
  return IMEX_OK;
}

int imex_info(imex_ctx* c, imex_stats* st) {
  if (!c || !st) return fail(IMEX_ERR_ARG, "bad arguments");
  fill_stats(c->hs, st);
  st->step = c->step;
  st->solve_cluster = c->cluster;
  st->solve_groups = c->ngroups;
  st->solve_smem_bytes = (int64_t)c->smem_solve;
  st->device_bytes = (int64_t)c->bytes;
  return IMEX_OK;
}

void imex_destroy(imex_ctx* c) {
  if (!c) return;
  if (c->base) {
    cudaDeviceSynchronize();
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
// update vectors, right-hand sides of the dense top blocks, solution vector)
// in a fixed array compiled into the library instead of context memory.
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
  const HostSetup& hs = c->hs;
  auto even = [](int64_t v) { return v + (v & 1); };
  const int64_t n_upd = even(std::max<int64_t>(hs.upd_size, 1));
  const int64_t n_zg = even(std::max<int64_t>(c->nzrow, 1));
  const int64_t n_sol = even(std::max<int64_t>(hs.n_c, 1));
  if (n_upd + n_zg + n_sol > kStaticScratchDoubles)
    return fail(IMEX_ERR_ARG, "imex_step_noalloc: the implicit solve needs " + std::to_string(n_upd + n_zg + n_sol) +
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
  double* zg = upd + n_upd;
  double* sol = zg + n_zg;
  cudaStream_t s = (cudaStream_t)stream;
  c->stream = s;
  const double dt = hs.dt;
  const int nif = (int)hs.if_cell.size();
  for (int64_t k = 0; k < n; ++k) {
    double* Ucur = c->U[c->cur];
    double* Unext = c->U[1 - c->cur];
    const int64_t step = c->step;
    ExplicitArgs ea = explicit_args(c, Ucur, Unext, Unext, 2.0, -1.0, dt * dt, ft_at(hs, step), true);
    explicit_dispatch(c, ea, c->ntx * c->nty + pred_blocks(c, true), s);
    if (hs.n_c > 0) {
      IfaceArgs ia = iface_args(c, Unext);
      k_iface<<<(nif + kWarps - 1) / kWarps, kThreads, 0, s>>>(ia);
      SolveArgs sa = solve_args(c, true, ft_at(hs, step + 1), 0, Unext);
      sa.upd = upd;
      sa.zg = zg;
      sa.sol = sol;
      launch_solve(c, sa, s);
    }
    if (int rc = check_launch("imex_step_noalloc")) return rc;
    c->cur = 1 - c->cur;
    c->step = step + 1;
  }
  return IMEX_OK;
}

