// libimex: device state, time-stepping kernels and the C-ABI (include/imex.h).
//
// Paper: Faßbender et al., "Implicit-Explicit Time Integration for the Immersed
// Wave Equation", Sec. "Time integration", Fig. TrapCDMIMEX (Newmark IMEX),
// Eqs. CDMstep / CDMacc (diagonal CDM step), Eqs. Newmark1/2 (prediction and
// correction, beta = 1/4, gamma = 1/2), Eqs. Kd / Kc (partitioned stiffness).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
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
    const double acc = minv * (a.ft * a.fx[g] - r);
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
// A4 gather + A5 + A6: one CTA per connected component of I_c.  Tree levels
// are processed bottom-up (forward L y = rhs) and top-down (backward
// L^T x = y); the nodes of one level are independent and go to different
// warps.  All sums run in a fixed order, so the result is deterministic.
__global__ void __launch_bounds__(kThreads) k_solve(SolveArgs a) {
  extern __shared__ double smg[];
  const int comp = blockIdx.x;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double* g = smg + warp * a.max_block;
  const int lb = a.comp_level_base[comp];
  const int nlev = a.comp_level_base[comp + 1] - lb - 1;

  for (int l = 0; l < nlev; ++l) {
    const int qb = a.comp_level_ptr[lb + l], qe = a.comp_level_ptr[lb + l + 1];
    for (int q = qb + warp; q < qe; q += kWarps) {
      const int t = a.level_nodes[q];
      const int beg = a.t_beg[t], b = a.t_end[t] - beg, m = a.t_nrows[t];
      const double* Ld = a.vals + a.t_off_diag[t];
      const double* Lr = a.vals + a.t_off_rect[t];
      for (int i = lane; i < b; i += 32) {
        const int r = beg + i;
        double s = a.ft * a.fxc[r];
        for (int k = a.contrib_ptr[r]; k < a.contrib_ptr[r + 1]; ++k) s -= a.Y[a.contrib_pos[k]];
        for (int k = a.fwd_ptr[r]; k < a.fwd_ptr[r + 1]; ++k) s -= a.upd[a.fwd_pos[k]];
        g[i] = s;
      }
      __syncwarp();
      for (int j = 0; j < b; ++j) {
        const double yj = g[j] * a.invdiag[beg + j];
        __syncwarp();
        if (lane == 0) g[j] = yj;
        for (int i = j + 1 + lane; i < b; i += 32) g[i] = fma(-Ld[i + (size_t)b * j], yj, g[i]);
        __syncwarp();
      }
      for (int i = lane; i < b; i += 32) a.sol[beg + i] = g[i];
      double* up = a.upd + a.t_off_upd[t];
      for (int k = lane; k < m; k += 32) {
        double s = 0.0;
        for (int j = 0; j < b; ++j) s = fma(Lr[k + (size_t)m * j], g[j], s);
        up[k] = s;
      }
      __syncwarp();
    }
    __syncthreads();
  }

  for (int l = nlev - 1; l >= 0; --l) {
    const int qb = a.comp_level_ptr[lb + l], qe = a.comp_level_ptr[lb + l + 1];
    for (int q = qb + warp; q < qe; q += kWarps) {
      const int t = a.level_nodes[q];
      const int beg = a.t_beg[t], b = a.t_end[t] - beg, m = a.t_nrows[t];
      const double* LdT = a.vals + a.t_off_diagT[t];
      const double* Lr = a.vals + a.t_off_rect[t];
      const int* rows = a.rows_idx + a.t_off_rows[t];
      for (int j = lane; j < b; j += 32) {
        double s = a.sol[beg + j];
        for (int k = 0; k < m; ++k) s = fma(-Lr[k + (size_t)m * j], a.sol[rows[k]], s);
        g[j] = s;
      }
      __syncwarp();
      for (int j = b - 1; j >= 0; --j) {
        const double xj = g[j] * a.invdiag[beg + j];
        __syncwarp();
        if (lane == 0) g[j] = xj;
        for (int i = lane; i < j; i += 32) g[i] = fma(-LdT[i + (size_t)b * j], xj, g[i]);
        __syncwarp();
      }
      for (int i = lane; i < b; i += 32) a.sol[beg + i] = g[i];
      __syncwarp();
    }
    __syncthreads();
  }

  // Correction (Fig. TrapCDMIMEX) or the initial acceleration.
  const double bdt2 = kNewmarkBeta * a.dt * a.dt, gdt = kNewmarkGamma * a.dt,
               g1dt = (1.0 - kNewmarkGamma) * a.dt;
  for (int r = a.comp_cbeg[comp] + threadIdx.x; r < a.comp_cend[comp]; r += blockDim.x) {
    const double acc = a.sol[r];
    if (a.mode == 0) {
      const int node = a.c_node[r];
      const double vpred = a.v_c[r] + g1dt * a.a_c[r];
      a.U[node] = a.U[node] + bdt2 * acc;
      a.v_c[r] = vpred + gdt * acc;
    }
    a.a_c[r] = acc;
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
  double *S_vals = nullptr, *S_inv = nullptr, *M_vals = nullptr, *M_inv = nullptr;
  int *t_beg = nullptr, *t_end = nullptr, *t_nrows = nullptr;
  int64_t *t_off_diag = nullptr, *t_off_diagT = nullptr, *t_off_rect = nullptr, *t_off_rows = nullptr,
          *t_off_upd = nullptr;
  int *rows_idx = nullptr, *level_nodes = nullptr, *comp_level_ptr = nullptr, *comp_level_base = nullptr;
  int *comp_cbeg = nullptr, *comp_cend = nullptr;
  int *contrib_ptr = nullptr, *contrib_pos = nullptr, *fwd_ptr = nullptr, *fwd_pos = nullptr;
  double *upd = nullptr, *sol = nullptr;
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
  sa.vals = use_S ? c->S_vals : c->M_vals;
  sa.invdiag = use_S ? c->S_inv : c->M_inv;
  sa.t_beg = c->t_beg;
  sa.t_end = c->t_end;
  sa.t_nrows = c->t_nrows;
  sa.t_off_diag = c->t_off_diag;
  sa.t_off_diagT = c->t_off_diagT;
  sa.t_off_rect = c->t_off_rect;
  sa.t_off_rows = c->t_off_rows;
  sa.t_off_upd = c->t_off_upd;
  sa.rows_idx = c->rows_idx;
  sa.level_nodes = c->level_nodes;
  sa.comp_level_ptr = c->comp_level_ptr;
  sa.comp_level_base = c->comp_level_base;
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
  sa.max_block = c->hs.max_block;
  return sa;
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
    k_solve<<<hs.ncomp, kThreads, c->smem_solve, s>>>(sa);
    if (int rc = check_launch("solve (initial)")) return rc;
  }
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
    if (hs.max_block > 1024) {
      delete c;
      return fail(IMEX_ERR_ARG, "supernode too large for the device solve");
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
    c->smem_solve = (size_t)kWarps * std::max(1, hs.max_block) * sizeof(double);

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
    ar.add(&c->S_vals, std::max<size_t>(hs.S.vals.size(), 1));
    ar.add(&c->S_inv, std::max<int64_t>(nc, 1));
    ar.add(&c->M_vals, std::max<size_t>(hs.Mcc.vals.size(), 1));
    ar.add(&c->M_inv, std::max<int64_t>(nc, 1));
    ar.add(&c->t_beg, std::max<int64_t>(nt, 1));
    ar.add(&c->t_end, std::max<int64_t>(nt, 1));
    ar.add(&c->t_nrows, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_diag, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_diagT, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_rect, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_rows, std::max<int64_t>(nt, 1));
    ar.add(&c->t_off_upd, std::max<int64_t>(nt, 1));
    ar.add(&c->rows_idx, std::max<size_t>(hs.rows_idx.size(), 1));
    ar.add(&c->level_nodes, std::max<size_t>(hs.level_nodes.size(), 1));
    ar.add(&c->comp_level_ptr, std::max<size_t>(hs.comp_level_ptr.size(), 1));
    ar.add(&c->comp_level_base, std::max<size_t>(hs.comp_level_base.size(), 1));
    ar.add(&c->comp_cbeg, std::max(hs.ncomp, 1));
    ar.add(&c->comp_cend, std::max(hs.ncomp, 1));
    ar.add(&c->contrib_ptr, hs.contrib_ptr.size());
    ar.add(&c->contrib_pos, std::max<size_t>(hs.contrib_pos.size(), 1));
    ar.add(&c->fwd_ptr, hs.fwd_ptr.size());
    ar.add(&c->fwd_pos, std::max<size_t>(hs.fwd_pos.size(), 1));
    ar.add(&c->upd, std::max<int64_t>(hs.upd_size, 1));
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
    e = e ? e : upload(c->S_vals, hs.S.vals);
    e = e ? e : upload(c->S_inv, hs.S.invdiag);
    e = e ? e : upload(c->M_vals, hs.Mcc.vals);
    e = e ? e : upload(c->M_inv, hs.Mcc.invdiag);
    e = e ? e : upload(c->t_beg, tb);
    e = e ? e : upload(c->t_end, te);
    e = e ? e : upload(c->t_nrows, tn);
    e = e ? e : upload(c->t_off_diag, od);
    e = e ? e : upload(c->t_off_diagT, odT);
    e = e ? e : upload(c->t_off_rect, orc);
    e = e ? e : upload(c->t_off_rows, orw);
    e = e ? e : upload(c->t_off_upd, ou);
    e = e ? e : upload(c->rows_idx, hs.rows_idx);
    e = e ? e : upload(c->level_nodes, hs.level_nodes);
    e = e ? e : upload(c->comp_level_ptr, hs.comp_level_ptr);
    e = e ? e : upload(c->comp_level_base, hs.comp_level_base);
    e = e ? e : upload(c->comp_cbeg, ccb);
    e = e ? e : upload(c->comp_cend, cce);
    e = e ? e : upload(c->contrib_ptr, hs.contrib_ptr);
    e = e ? e : upload(c->contrib_pos, hs.contrib_pos);
    e = e ? e : upload(c->fwd_ptr, hs.fwd_ptr);
    e = e ? e : upload(c->fwd_pos, hs.fwd_pos);
    e = e ? e : set_explicit_smem_dispatch(P, c->smem_explicit);
    if (e == cudaSuccess && c->smem_solve > 48 * 1024)
      e = cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_solve);
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

int imex_step(imex_ctx* c, int64_t n, void* stream) {
  if (!c || n < 0) return fail(IMEX_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  c->stream = s;
  const HostSetup& hs = c->hs;
  const double dt = hs.dt;
  const int grid_tiles = c->ntx * c->nty;
  const int npb = pred_blocks(c, true);
  const int nif = (int)hs.if_cell.size();
  for (int64_t k = 0; k < n; ++k) {
    double* Ucur = c->U[c->cur];
    double* Unext = c->U[1 - c->cur];
    const int64_t step = c->step;
    ExplicitArgs ea = explicit_args(c, Ucur, Unext, Unext, 2.0, -1.0, dt * dt, ft_at(hs, step), true);
    explicit_dispatch(c, ea, grid_tiles + npb, s);
    if (hs.n_c > 0) {
      IfaceArgs ia = iface_args(c, Unext);
      k_iface<<<(nif + kWarps - 1) / kWarps, kThreads, 0, s>>>(ia);
      SolveArgs sa = solve_args(c, true, ft_at(hs, step + 1), 0, Unext);
      k_solve<<<hs.ncomp, kThreads, c->smem_solve, s>>>(sa);
    }
    if (int rc = check_launch("imex_step")) return rc;
    c->cur = 1 - c->cur;
    c->step = step + 1;
  }
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
