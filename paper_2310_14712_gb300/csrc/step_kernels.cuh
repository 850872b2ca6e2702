// Time-stepping kernels of one IMEX step: the explicit apply with the CDM
// update and the prediction (2D and 3D), and the implicit solve with the
// correction (walked levels and dense tops).  Textually included by imex.cu
// inside its internal namespace (constants and argument structs come from
// there and from kernels.cuh); not a standalone header.
#pragma once

// ---------------------------------------------------------------------------
// A1 + A2 (+ A3): explicit apply on the tensor grid, CDM update, prediction.

// CDM update of one explicit node (Eqs. CDMacc, CDMstep):
//   out = cu u + cw w + ca M_ii^{-1} (f_t f_x - (K u)_i)
//       = cu u + cw w + kappa2 (f_t g - r),
// with g = dt^2 M_ii^{-1} f_x (stored), r = dt^2 M_ii^{-1} (K u)_i (the
// mass-scaled apply) and kappa2 = ca / dt^2.  The step (cu = 2, cw = -1,
// kappa2 = 1) costs three FP64 operations.  Every 2D explicit kernel uses
// this helper, so they agree bit for bit.
__device__ __forceinline__ double cdm_node(double u, double w, double r, double g, double ft, double cu,
                                           double cw, double kappa2) {
  const double t = fma(ft, g, -r);
  if (cw == -1.0 && kappa2 == 1.0) return fma(cu, u, -w) + t;
  return fma(kappa2, t, fma(cu, u, cw * w));
}
//
// A tile owns OX x OY nodes (TC x TC cells).  With u staged in shared memory
// together with one halo cell on the low side, the stiffness rows of the
// owned nodes are formed by sum factorisation:
//   x pass: T1 = (sx K1)_x u, T2 = (M1)_x u, cell by cell (the two cell
//           contributions at a vertex are added in a fix-up pass),
//   y pass: r = (M1)_y T1 + (sy K1)_y T2, again cell by cell plus fix-up.
// Each 1D product uses the symmetry of the GLL nodes: K1 commutes with the
// reflection x -> -x, so it maps the even and odd parts of a vector
// separately (P^2 -> about P^2/2 FMAs), and the exact mass is the GLL-lumped
// mass plus a rank-one term, M1 = diag(w) + C a a^T (GLL quadrature is exact
// to degree 2p-1; the product of two basis functions differs from a
// polynomial it integrates exactly by a_i a_j x^{2p}, a_i the leading
// coefficient of the i-th basis function), so M1 v costs about 3P.
// For an I_d node every surrounding cell is uncut, so this equals its row of
// K^d u_n (Eq. Kd).  Nodes of I_c and inactive nodes are computed but not
// written.  Cells outside the grid contribute nothing.
// The 1D products of the 2D explicit apply, on the P nodal values of one
// cell along one grid line.  Each uses the symmetry of the GLL nodes: K1
// commutes with the reflection x -> -x, so it maps the even and odd parts of
// a vector separately (P^2 -> about P^2/2 FMAs), and the exact mass is the
// GLL-lumped mass plus a rank-one term, M1 = diag(w) + C a a^T (GLL
// quadrature is exact to degree 2p-1; the product of two basis functions
// differs from a polynomial it integrates exactly by a_i a_j x^{2p}, a_i the
// leading coefficient of the i-th basis function), so M1 v costs about 3P.
// The coefficients carry the inverse lumped mass and dt^2 (Ops2D), so r is
// dt^2 M^{-1} K u at explicit nodes.  The diagonal (nodal) mass term of a
// vertex shared by two cells is split asymmetrically: the cell on the low
// side adds all of it (its last node: v, or kappa va in y), the cell on the
// high side none (its first node: only the rank-one term), so each vertex
// output costs one FP64 operation less; at the grid's edge, where one cell
// holds the vertex, the fix-ups restore twice the half share exactly
// (2 sum + v at the low edge, 2 sum - v at the high edge).  Every 2D
// explicit kernel calls these, so their results agree bit for bit.

// x pass: o1 = (sx K1) v, o2 = M1 v.
template <int P>
__device__ __forceinline__ void x_item(const Ops2D& ops, const double (&v)[P], double (&o1)[P], double (&o2)[P]) {
  constexpr int H = P / 2;
  constexpr bool kOdd = (P % 2) == 1;
  double e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j] + v[P - 1 - j];
    o[j] = v[j] - v[P - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double ev = kOdd ? ops.kxc[i] * v[H] : 0.0, od = 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      ev = fma(ops.kxe[i][j], e[j], ev);
      od = fma(ops.kxo[i][j], o[j], od);
    }
    o1[i] = ev + od;
    o1[P - 1 - i] = ev - od;
  }
  if (kOdd) {
    double ev = ops.kxc[H] * v[H];
#pragma unroll
    for (int j = 0; j < H; ++j) ev = fma(ops.kxe[H][j], e[j], ev);
    o1[H] = ev;
  }
  double sa = kOdd ? ops.a[H] * v[H] : 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) sa = fma(ops.a[j], kOdd ? e[j] : o[j], sa);
#pragma unroll
  for (int i = 0; i < P; ++i)
    o2[i] = i == 0 ? ops.cax[0] * sa : fma(ops.cax[i], sa, v[i]);   // vertex mass split, see below
}

// The same, last node only (o1[P-1], o2[P-1]): the right vertex of a cell
// whose other outputs are not needed.  Same operations as x_item for them.
template <int P>
__device__ __forceinline__ void x_item_last(const Ops2D& ops, const double (&v)[P], double& o1p, double& o2p) {
  constexpr int H = P / 2;
  constexpr bool kOdd = (P % 2) == 1;
  double e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j] + v[P - 1 - j];
    o[j] = v[j] - v[P - 1 - j];
  }
  double ev = kOdd ? ops.kxc[0] * v[H] : 0.0, od = 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    ev = fma(ops.kxe[0][j], e[j], ev);
    od = fma(ops.kxo[0][j], o[j], od);
  }
  o1p = ev - od;
  double sa = kOdd ? ops.a[H] * v[H] : 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) sa = fma(ops.a[j], kOdd ? e[j] : o[j], sa);
  o2p = fma(ops.cax[P - 1], sa, v[P - 1]);
}

// y pass: o = M1 va + (sy K1) vb.
template <int P>
__device__ __forceinline__ void y_item(const Ops2D& ops, const double (&va)[P], const double (&vb)[P], double (&o)[P]) {
  constexpr int H = P / 2;
  constexpr bool kOdd = (P % 2) == 1;
  double sa = kOdd ? ops.a[H] * va[H] : 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) sa = fma(ops.a[j], kOdd ? va[j] + va[P - 1 - j] : va[j] - va[P - 1 - j], sa);
  double e[H], od_[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = vb[j] + vb[P - 1 - j];
    od_[j] = vb[j] - vb[P - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double ev = kOdd ? ops.kyc[i] * vb[H] : 0.0, od = 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      ev = fma(ops.kye[i][j], e[j], ev);
      od = fma(ops.kyo[i][j], od_[j], od);
    }
    // The rank-one mass term of the pair: cay_{P-1-i} = cay_i (p even) or
    // -cay_i (p odd), so it joins the even or the odd accumulator.
    if (kOdd) ev = fma(ops.cay[i], sa, ev);
    else od = fma(ops.cay[i], sa, od);
    const int k = P - 1 - i;
    if (i == 0) {   // vertex mass split, see below
      o[0] = ev + od;
      o[k] = fma(ops.wyv, va[k], ev - od);
    } else {
      o[i] = fma(ops.wy[i], va[i], ev + od);
      o[k] = fma(ops.wy[k], va[k], ev - od);
    }
  }
  if (kOdd) {
    double ev = ops.kyc[H] * vb[H];
#pragma unroll
    for (int j = 0; j < H; ++j) ev = fma(ops.kye[H][j], e[j], ev);
    o[H] = fma(ops.wy[H], va[H], fma(ops.cay[H], sa, ev));
  }
}

// The same, last node only (o[P-1]).
template <int P>
__device__ __forceinline__ double y_item_last(const Ops2D& ops, const double (&va)[P], const double (&vb)[P]) {
  constexpr int H = P / 2;
  constexpr bool kOdd = (P % 2) == 1;
  double sa = kOdd ? ops.a[H] * va[H] : 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) sa = fma(ops.a[j], kOdd ? va[j] + va[P - 1 - j] : va[j] - va[P - 1 - j], sa);
  double e[H], od_[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = vb[j] + vb[P - 1 - j];
    od_[j] = vb[j] - vb[P - 1 - j];
  }
  double ev = kOdd ? ops.kyc[0] * vb[H] : 0.0, od = 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    ev = fma(ops.kye[0][j], e[j], ev);
    od = fma(ops.kyo[0][j], od_[j], od);
  }
  if (kOdd) ev = fma(ops.cay[0], sa, ev);
  else od = fma(ops.cay[0], sa, od);
  return fma(ops.wyv, va[P - 1], ev - od);
}

// One tile of the 2D explicit apply (owned nodes of tile `tile`, column col).
template <int P, int TC>
__device__ __forceinline__ void explicit_tile(const ExplicitArgs& a, const Ops2D& ops, int tile, int col,
                                              double* sm) {
  constexpr int p = P - 1;
  constexpr int OX = TC * p, OY = TC * p;
  constexpr int RX = (TC + 1) * p + 1, RY = RX;
  constexpr int NC = TC + 1;
  const int tid = threadIdx.x;
  const int64_t on = (int64_t)col * a.cs_node;
  const double* Uc = a.U + on;
  const double* Wc = a.W + on;     // may alias OUTc
  double* OUTc = a.OUT + on;

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

  const int tx = tile % a.ntx, ty = tile / a.ntx;
  const int X0 = tx * OX, Y0 = ty * OY;
  const int cx0 = X0 / p - 1, cy0 = Y0 / p - 1;

  for (int idx = tid; idx < RY * RX; idx += kThreads) {
    const int yy = idx / RX, xx = idx - yy * RX;
    const int gx = X0 - p + xx, gy = Y0 - p + yy;
    su[idx] = (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) ? Uc[(size_t)gy * a.nx + gx] : 0.0;
  }
  __syncthreads();

  // x pass: item = (row yy, cell cc), rows fastest.  Rows outside the grid
  // (a tile past the last node row) feed no cell inside it: skipped.
  for (int it = tid; it < RY * NC; it += kThreads) {
    const int cc = it / RY, yy = it - cc * RY;
    const int gyr = Y0 - p + yy;
    if (gyr < 0 || gyr >= a.ny) continue;
    const int cx = cx0 + cc;
    if (cx < 0 || cx >= a.ncx) {   // a cell outside the grid contributes nothing
      if (cc >= 1) {
#pragma unroll
        for (int i = 1; i < p; ++i) {
          t1[yy * OX + (cc - 1) * p + i] = 0.0;
          t2[yy * OX + (cc - 1) * p + i] = 0.0;
        }
      }
      tl1[yy * NC + cc] = 0.0;
      tr1[yy * NC + cc] = 0.0;
      tl2[yy * NC + cc] = 0.0;
      tr2[yy * NC + cc] = 0.0;
      continue;
    }
    double v[P], o1[P], o2[P];
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = su[yy * RX + cc * p + j];
    x_item<P>(ops, v, o1, o2);
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
    const int gx = X0 + k * p;
    double v1 = tr1[yy * NC + k] + tl1[yy * NC + k + 1];
    double v2 = tr2[yy * NC + k] + tl2[yy * NC + k + 1];
    if (gx == 0 || gx == a.nx - 1) {   // one cell at the grid's edge: its weight is w_0, not 2 w_0
      const double u = su[yy * RX + k * p + p];
      v1 *= 2.0;
      v2 = gx == 0 ? fma(2.0, v2, u) : fma(2.0, v2, -u);
    }
    t1[yy * OX + k * p] = v1;
    t2[yy * OX + k * p] = v2;
  }
  __syncthreads();

  // y pass: item = (column xo, cell row cr), columns fastest.  Columns
  // past the last node column own no node: skipped.
  for (int it = tid; it < OX * NC; it += kThreads) {
    const int cr = it / OX, xo = it - cr * OX;
    if (X0 + xo >= a.nx) continue;
    const int cy = cy0 + cr;
    if (cy < 0 || cy >= a.ncy) {   // a cell outside the grid contributes nothing
      if (cr >= 1) {
#pragma unroll
        for (int i = 1; i < p; ++i) rr[((cr - 1) * p + i) * OX + xo] = 0.0;
      }
      rb[cr * OX + xo] = 0.0;
      rt[cr * OX + xo] = 0.0;
      continue;
    }
    double va[P], vb[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      va[j] = t1[(cr * p + j) * OX + xo];
      vb[j] = t2[(cr * p + j) * OX + xo];
    }
    double o[P];
    y_item<P>(ops, va, vb, o);
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
    const int gy = Y0 + k * p;
    double v = rt[k * OX + xo] + rb[(k + 1) * OX + xo];
    if (gy == 0 || gy == a.ny - 1) {   // one cell at the grid's edge
      const double ka = ops.wyv * t1[((k + 1) * p) * OX + xo];
      v = gy == 0 ? fma(2.0, v, ka) : fma(2.0, v, -ka);
    }
    rr[(k * p) * OX + xo] = v;
  }
  __syncthreads();

  // CDM update of the owned I_d nodes (Eqs. CDMacc, CDMstep).
  const double ft = a.ft_dev ? a.ft_dev[0] : a.ft;
  const double* gxs = a.fxs + on;
  for (int it = tid; it < OY * OX; it += kThreads) {
    const int yo = it / OX, xo = it - yo * OX;
    const int gx = X0 + xo, gy = Y0 + yo;
    if (gx >= a.nx || gy >= a.ny) continue;
    const size_t g = (size_t)gy * a.nx + gx;
    if (a.cls[g] != NODE_D) continue;
    const double r = rr[yo * OX + xo];
    const double u = su[(yo + p) * RX + xo + p];
    OUTc[g] = cdm_node(u, Wc[g], r, gxs[g], ft, a.cu, a.cw, a.kappa2);
  }
}

// The 2D explicit apply: one CTA per tile (of the list a.tiles, if given),
// then the prediction CTAs; or (a.persistent) a fixed grid looping over the
// listed tiles of every column, without prediction.
template <int P, int TC>
__global__ void __launch_bounds__(kThreads) k_explicit2d(ExplicitArgs a, Ops2D ops) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int ntl = a.tiles ? a.ntl : a.ntx * a.nty;
  // The first solve launch may start staging its constant factor blocks now;
  // it waits for this grid (griddepcontrol.wait) before it reads u.
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  if (a.persistent) {
    const int nitem = ntl * a.ncols;
    for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
      const int col = it / ntl;
      explicit_tile<P, TC>(a, ops, a.tiles[it - col * ntl], col, sm);
      __syncthreads();
    }
    return;
  }
  if ((int)blockIdx.x >= ntl) {
    // Newmark prediction on I_c (Fig. TrapCDMIMEX, "Prediction").
    const int64_t on = (int64_t)blockIdx.y * a.cs_node, oc = (int64_t)blockIdx.y * a.cs_c;
    const double* Uc = a.U + on;
    double* OUTc = a.OUT + on;
    const double c1 = a.dt, c2 = (0.5 - kNewmarkBeta) * a.dt * a.dt;
    const int stride = (gridDim.x - ntl) * blockDim.x;
    for (int r = (blockIdx.x - ntl) * blockDim.x + tid; r < a.n_c; r += stride) {
      const int node = a.c_node[r];
      OUTc[node] = Uc[node] + c1 * a.v_c[oc + r] + c2 * a.a_c[oc + r];
    }
    return;
  }
  explicit_tile<P, TC>(a, ops, a.tiles ? a.tiles[blockIdx.x] : (int)blockIdx.x, blockIdx.y, sm);
}

// ---------------------------------------------------------------------------
// A1 + A2 (+ A3) in 2D, persistent sweep form.  The grid is cut into strips
// of TCX cells (OX = TCX p owned node columns); the work units are (strip,
// cell row) pairs, strip-major, and CTA b of the nsweep = a.ntx sweep CTAs
// takes the contiguous units [b U / nsweep, (b+1) U / nsweep), so every CTA has the same
// number of cell rows within one.  A CTA walks each of its strip segments
// upwards in chunks of CH cell rows.  Between chunks it keeps the top node
// row of the chunk: its staged u, its x-pass products (T1 = (sx K1)_x u,
// T2 = (M1)_x u) and its partial stiffness row from the cell row below, so
// no row of the strip is staged or contracted twice except the cell row
// below a segment's start (its top output only).  The left halo cell of the
// strip contributes only its right vertex column (x_item_last).  The next
// chunk's rows of u are copied into the other of two buffers (cp.async)
// while the current chunk is contracted.  Same products and sums as
// k_explicit2d, in the same order: the two kernels agree bit for bit.
// Shared memory (doubles): u 2 x SR x RX, T1 and T2 SR x OXP each, x-pass
// vertex partials or y-pass rows (aliased), the carried partial row.
template <int P, int TCX, int CH>
struct SweepShape {
  static constexpr int p = P - 1;
  static constexpr int OX = TCX * p;        // owned node columns of a full strip
  static constexpr int OXP = OX + 1;        // + the grid's last column in the last strip
  static constexpr int RX = OX + p + 1;     // staged columns: halo cell, strip cells
  static constexpr int NC = TCX + 1;        // staged cells per row (halo first)
  static constexpr int NR = CH * p;         // new node rows per chunk
  static constexpr int SR = NR + 1;         // staged rows (carried row first)
  static constexpr int XR = NR > P ? NR : P;  // rows of x-pass partials
  static constexpr int SCR = (4 * XR * NC > SR * OXP + 2 * CH * OXP) ? 4 * XR * NC : SR * OXP + 2 * CH * OXP;
  static constexpr int KF = (SR * OXP + kThreads - 1) / kThreads;  // CDM nodes per thread per chunk
  // u (2 buffers), T1, T2, scratch, carried row (2 buffers)
  static constexpr int DOUBLES = 2 * SR * RX + 2 * SR * OXP + SCR + 2 * OXP;
};

// Stage rows [gy0, gy0 + nrows) of u (columns X0 - p ... X0 + OX) into su
// rows [r0, r0 + nrows): cp.async of 8 bytes per node inside the grid,
// zeros outside.
template <int RX>
__device__ __forceinline__ void sweep_stage(double* su, int r0, const double* Uc, int gy0, int nrows, int X0, int p,
                                            int nx) {
  for (int idx = threadIdx.x; idx < nrows * RX; idx += blockDim.x) {
    const int yy = idx / RX, xx = idx - yy * RX;
    const int gx = X0 - p + xx;
    double* d = su + (r0 + yy) * RX + xx;
    if (gx >= 0 && gx < nx) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(d);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa),
                   "l"(Uc + (size_t)(gy0 + yy) * nx + gx)
                   : "memory");
    } else {
      *d = 0.0;
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int P, int TCX, int CH, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_sweep2d(ExplicitArgs a, Ops2D ops) {
  using S = SweepShape<P, TCX, CH>;
  constexpr int p = S::p, OX = S::OX, OXP = S::OXP, RX = S::RX, NC = S::NC, NR = S::NR, SR = S::SR;
  constexpr int XR = S::XR, KF = S::KF;
  extern __shared__ __align__(16) double sm[];
  const int tid = threadIdx.x;
  const int64_t on = (int64_t)blockIdx.y * a.cs_node, oc = (int64_t)blockIdx.y * a.cs_c;
  const double* Uc = a.U + on;
  const double* Wc = a.W + on;     // may alias OUTc
  double* OUTc = a.OUT + on;
  const double* gxs = a.fxs + on;   // dt^2 M^{-1} f_x
  // The first solve launch may start staging its constant factor blocks now;
  // it waits for this grid (griddepcontrol.wait) before it reads u.
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

  const int nsweep = a.ntx;        // sweep CTAs; the rest of the grid (if any) predicts
  const double c1p = a.dt, c2p = (0.5 - kNewmarkBeta) * a.dt * a.dt;
  if ((int)blockIdx.x >= nsweep) {
    // Newmark prediction on I_c (Fig. TrapCDMIMEX, "Prediction").
    const int stride = (gridDim.x - nsweep) * blockDim.x;
    for (int r = (blockIdx.x - nsweep) * blockDim.x + tid; r < a.n_c; r += stride) {
      const int node = a.c_node[r];
      OUTc[node] = Uc[node] + c1p * a.v_c[oc + r] + c2p * a.a_c[oc + r];
    }
    return;
  }
  // No prediction CTAs (gridDim.x == nsweep): each sweep CTA predicts its
  // share of I_c while its first rows arrive (a CTA launched after the
  // sweep CTAs would only start once one of them has finished).
  bool predict = (int)gridDim.x == nsweep && a.n_c > 0;
  auto predict_share = [&]() {
    const int r0 = (int)((int64_t)a.n_c * blockIdx.x / nsweep);
    const int r1 = (int)((int64_t)a.n_c * (blockIdx.x + 1) / nsweep);
    for (int r = r0 + tid; r < r1; r += kThreads) {
      const int node = a.c_node[r];
      OUTc[node] = Uc[node] + c1p * a.v_c[oc + r] + c2p * a.a_c[oc + r];
    }
    predict = false;
  };

  double* const ub0 = sm;                    // u, two buffers of SR x RX
  double* const ub1 = sm + SR * RX;
  double* t1 = sm + 2 * SR * RX;             // SR x OXP
  double* t2 = t1 + SR * OXP;
  double* scr = t2 + SR * OXP;
  double* tl1 = scr;                         // XR x NC vertex partials (x pass)
  double* tr1 = tl1 + XR * NC;
  double* tl2 = tr1 + XR * NC;
  double* tr2 = tl2 + XR * NC;
  double* rr = scr;                          // SR x OXP rows of K^d u (aliases the x partials)
  double* rb = rr + SR * OXP;                // CH x OXP bottom-vertex partials (y pass)
  double* rt = rb + CH * OXP;                // CH x OXP top-vertex partials
  double* const carry0 = scr + S::SCR;       // OXP: partial row from the cell row below,
  double* const carry1 = carry0 + OXP;       //   two buffers (read, then written, in one phase)

  const int ncy = a.ncy;
  const int nstrip = (a.ncx + TCX - 1) / TCX;
  const int64_t units = (int64_t)nstrip * ncy;
  int64_t u0 = units * blockIdx.x / nsweep;
  const int64_t u1 = units * (blockIdx.x + 1) / nsweep;
  const double ft = a.ft_dev ? a.ft_dev[0] : a.ft;

  // x pass over staged rows [r_lo, r_lo + nrows) of su into T1/T2 rows
  // [r_lo, ...): cell by cell, then the vertex columns.
  auto xpass = [&](const double* su, int r_lo, int nrows, int cx0) {
    for (int it = tid; it < nrows * NC; it += kThreads) {
      const int cc = it / nrows, yl = it - cc * nrows, yy = r_lo + yl;
      const int cx = cx0 + cc;
      double* T1 = t1 + yy * OXP + (cc - 1) * p;
      double* T2 = t2 + yy * OXP + (cc - 1) * p;
      if (cx < 0 || cx >= a.ncx) {   // a cell outside the grid contributes nothing
        if (cc >= 1) {
#pragma unroll
          for (int i = 1; i < p; ++i) {
            T1[i] = 0.0;
            T2[i] = 0.0;
          }
        }
        tl1[yl * NC + cc] = 0.0;
        tr1[yl * NC + cc] = 0.0;
        tl2[yl * NC + cc] = 0.0;
        tr2[yl * NC + cc] = 0.0;
        continue;
      }
      double v[P];
#pragma unroll
      for (int j = 0; j < P; ++j) v[j] = su[yy * RX + cc * p + j];
      if (cc == 0) {   // halo cell: its right vertex only
        double o1p, o2p;
        x_item_last<P>(ops, v, o1p, o2p);
        tr1[yl * NC] = o1p;
        tr2[yl * NC] = o2p;
        continue;
      }
      double o1[P], o2[P];
      x_item<P>(ops, v, o1, o2);
#pragma unroll
      for (int i = 1; i < p; ++i) {
        T1[i] = o1[i];
        T2[i] = o2[i];
      }
      tl1[yl * NC + cc] = o1[0];
      tr1[yl * NC + cc] = o1[p];
      tl2[yl * NC + cc] = o2[0];
      tr2[yl * NC + cc] = o2[p];
    }
    __syncthreads();
    for (int it = tid; it < nrows * NC; it += kThreads) {   // vertex columns k p, k = 0..TCX
      const int k = it / nrows, yl = it - k * nrows, yy = r_lo + yl;
      const double r1 = k < TCX ? tl1[yl * NC + k + 1] : 0.0;
      const double r2 = k < TCX ? tl2[yl * NC + k + 1] : 0.0;
      const int gx = cx0 * p + p + k * p;
      double v1 = tr1[yl * NC + k] + r1;
      double v2 = tr2[yl * NC + k] + r2;
      if (gx == 0 || gx == a.nx - 1) {   // one cell at the grid's edge: its weight is w_0, not 2 w_0
        const double u = su[yy * RX + k * p + p];
        v1 *= 2.0;
        v2 = gx == 0 ? fma(2.0, v2, u) : fma(2.0, v2, -u);
      }
      t1[yy * OXP + k * p] = v1;
      t2[yy * OXP + k * p] = v2;
    }
    __syncthreads();
  };

  while (u0 < u1) {
    // One segment: strip sx, cell rows [ra, rb).
    const int sx = (int)(u0 / ncy);
    const int ra = (int)(u0 - (int64_t)sx * ncy);
    const int64_t rlim = ra + (u1 - u0);
    const int rb_ = rlim < ncy ? (int)rlim : ncy;
    u0 += rb_ - ra;
    const int X0 = sx * OX;
    const int cx0 = sx * TCX - 1;                 // the halo cell
    const int oxe = min(OXP, a.nx - X0);          // owned columns (the last strip also owns column nx - 1)
    const int ocols = (sx == nstrip - 1) ? oxe : min(OX, oxe);
    int cur = 0;
    int c0 = ra;
    int ch = min(CH, rb_ - c0);
    // Everything the segment's start needs, in one round trip: u of the
    // first chunk's rows and, below a segment that does not start at the
    // grid's bottom, the P rows of the cell row below (buffer 1).
    if (ra == 0) sweep_stage<RX>(ub0, 0, Uc, 0, ch * p + 1, X0, p, a.nx);
    else {
      sweep_stage<RX>(ub1, 0, Uc, (ra - 1) * p, P, X0, p, a.nx);
      sweep_stage<RX>(ub0, 1, Uc, c0 * p + 1, ch * p, X0, p, a.nx);
    }
    if (predict) predict_share();
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // Prologue: node row ra p (staged u, T1, T2 in row 0 of buffer 0) and
    // the partial of that row from the cell row below.
    if (ra == 0) {
      xpass(ub0, 0, 1, cx0);
      for (int xo = tid; xo < OXP; xo += kThreads) carry0[xo] = 0.0;
    } else {
      // x pass on the P rows of the cell row below, its top output; then row
      // ra p moves to row 0 of buffer 0.
      xpass(ub1, 0, P, cx0);
      for (int xo = tid; xo < ocols; xo += kThreads) {
        double va[P], vb[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          va[j] = t1[j * OXP + xo];
          vb[j] = t2[j * OXP + xo];
        }
        carry0[xo] = y_item_last<P>(ops, va, vb);
      }
      __syncthreads();
      for (int xx = tid; xx < RX; xx += kThreads) ub0[xx] = ub1[p * RX + xx];
      for (int xo = tid; xo < OXP; xo += kThreads) {
        t1[xo] = t1[p * OXP + xo];
        t2[xo] = t2[p * OXP + xo];
      }
      __syncthreads();
    }
    while (ch > 0) {
      double* const su = cur ? ub1 : ub0;
      double* const sn = cur ? ub0 : ub1;
      const double* const carry = cur ? carry1 : carry0;
      double* const carry_next = cur ? carry0 : carry1;
      const int c1 = c0 + ch;
      const int chn = min(CH, rb_ - c1);         // next chunk's cell rows
      const bool top = c1 == ncy;                 // the grid's top row is final too
      const int nfin = ch * p + (top ? 1 : 0);
      // The CDM update's inputs of this thread's nodes (u_{n-1}, scaled f_x, class),
      // loaded now so that they arrive while the passes run.
      double pw[KF], pf[KF];
      int pcl[KF];
#pragma unroll
      for (int q = 0; q < KF; ++q) {
        const int it = tid + q * kThreads;
        pcl[q] = NODE_INACTIVE;
        pw[q] = pf[q] = 0.0;
        if (it < ocols * nfin) {
          const int yl = it / ocols, xo = it - yl * ocols;
          const size_t g = (size_t)(c0 * p + yl) * a.nx + X0 + xo;
          pcl[q] = a.cls[g];
          pw[q] = Wc[g];
          pf[q] = gxs[g];
        }
      }
      if (chn > 0) sweep_stage<RX>(sn, 1, Uc, c1 * p + 1, chn * p, X0, p, a.nx);
      xpass(su, 1, ch * p, cx0);
      // y pass: item = (column xo, cell row k), columns fastest.
      for (int it = tid; it < ocols * ch; it += kThreads) {
        const int k = it / ocols, xo = it - k * ocols;
        double va[P], vb[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          va[j] = t1[(k * p + j) * OXP + xo];
          vb[j] = t2[(k * p + j) * OXP + xo];
        }
        double o[P];
        y_item<P>(ops, va, vb, o);
#pragma unroll
        for (int i = 1; i < p; ++i) rr[(k * p + i) * OXP + xo] = o[i];
        rb[k * OXP + xo] = o[0];
        rt[k * OXP + xo] = o[p];
      }
      __syncthreads();
      // CDM update of the finished rows (Eqs. CDMacc, CDMstep).  A vertex
      // row k p adds the contributions of the cell rows below and above it
      // here (rows are warp-uniform for full strips).
#pragma unroll
      for (int q = 0; q < KF; ++q) {
        const int it = tid + q * kThreads;
        if (pcl[q] != NODE_D) continue;   // also every it >= ocols * nfin
        const int yl = it / ocols, xo = it - yl * ocols;
        const size_t g = (size_t)(c0 * p + yl) * a.nx + X0 + xo;
        const int k = yl / p;
        double r;
        if (yl != k * p) {
          r = rr[yl * OXP + xo];
        } else if (k < ch) {
          const double below = k == 0 ? carry[xo] : rt[(k - 1) * OXP + xo];
          r = below + rb[k * OXP + xo];
          if (c0 == 0 && k == 0) r = fma(2.0, r, ops.wyv * t1[xo]);   // one cell at the grid's bottom edge
        } else {   // the grid's top row: nothing above (one cell)
          r = fma(2.0, rt[(k - 1) * OXP + xo], -(ops.wyv * t1[(k * p) * OXP + xo]));
        }
        const double u = su[yl * RX + xo + p];
        OUTc[g] = cdm_node(u, pw[q], r, pf[q], ft, a.cu, a.cw, a.kappa2);
      }
      if (!top)
        for (int xo = tid; xo < ocols; xo += kThreads) carry_next[xo] = rt[(ch - 1) * OXP + xo];
      // Carry the top row (u, T1, T2) to row 0 of the next buffer.
      if (chn > 0) {
        for (int xx = tid; xx < RX; xx += kThreads) sn[xx] = su[(ch * p) * RX + xx];
        for (int xo = tid; xo < OXP; xo += kThreads) {
          t1[xo] = t1[(ch * p) * OXP + xo];
          t2[xo] = t2[(ch * p) * OXP + xo];
        }
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      cur = 1 - cur;
      c0 = c1;
      ch = chn;
    }
  }
}

// ---------------------------------------------------------------------------
// A1 + A2 (+ A3) in 3D: the same tensor-grid scheme with three passes.  A
// tile owns OX^3 nodes (TC^3 cells); u is staged with one halo cell on the
// low side of each axis.
//   x pass: TK = (sx K1)_x u, TM = (M1)_x u          (every staged (z, y) row)
//   y pass: AB = (M1)_y TK + (sy K1)_y TM, C = (M1)_y TM   (staged z, owned x)
//   z pass: r = (M1)_z AB + (sz K1)_z C              (owned y, x)
// each pass cell by cell, the two cell contributions at a vertex plane added
// in a fix-up pass.  For an I_d node every surrounding cell is uncut, so r is
// its row of K^d u_n (Eq. Kd).  The 1D products use the even-odd form of K1
// and the rank-one form of M1, as in 2D.

// o = (s K1) v on axis ax (even-odd form).
template <int P>
__device__ __forceinline__ void k1d3(const Ops3D& ops, int ax, const double (&v)[P], double (&o)[P]) {
  constexpr int H = P / 2;
  constexpr bool kOdd = (P % 2) == 1;
  double e[H], od[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j] + v[P - 1 - j];
    od[j] = v[j] - v[P - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double ev = kOdd ? ops.kc[ax][i] * v[H] : 0.0, odd = 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      ev = fma(ops.ke[ax][i][j], e[j], ev);
      odd = fma(ops.ko[ax][i][j], od[j], odd);
    }
    o[i] = ev + odd;
    o[P - 1 - i] = ev - odd;
  }
  if (kOdd) {
    double ev = ops.kc[ax][H] * v[H];
#pragma unroll
    for (int j = 0; j < H; ++j) ev = fma(ops.ke[ax][H][j], e[j], ev);
    o[H] = ev;
  }
}

// a^T v for the rank-one part of M1.
template <int P>
__device__ __forceinline__ double m1d3_sa(const Ops3D& ops, const double (&v)[P]) {
  constexpr int H = P / 2;
  constexpr bool kOdd = (P % 2) == 1;
  double sa = kOdd ? ops.a[H] * v[H] : 0.0;
#pragma unroll
  for (int j = 0; j < H; ++j) sa = fma(ops.a[j], kOdd ? v[j] + v[P - 1 - j] : v[j] - v[P - 1 - j], sa);
  return sa;
}

template <int P, int TC>
__global__ void __launch_bounds__(kThreads) k_explicit3d(ExplicitArgs a, Ops3D ops) {
  constexpr int p = P - 1;
  constexpr int OX = TC * p;
  constexpr int R = (TC + 1) * p + 1;   // staged nodes per axis
  constexpr int NC = TC + 1;            // staged cells per axis
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const int ntiles = a.ntx * a.nty * a.ntz;
  const int64_t on = (int64_t)blockIdx.y * a.cs_node, oc = (int64_t)blockIdx.y * a.cs_c;
  const double* Uc = a.U + on;
  const double* Wc = a.W + on;     // may alias OUTc
  double* OUTc = a.OUT + on;
  const double* fxc = a.fx + on;
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");

  if ((int)blockIdx.x >= ntiles) {
    // Newmark prediction on I_c (Fig. TrapCDMIMEX, "Prediction").
    const double c1 = a.dt, c2 = (0.5 - kNewmarkBeta) * a.dt * a.dt;
    const int stride = (gridDim.x - ntiles) * blockDim.x;
    for (int r = (blockIdx.x - ntiles) * blockDim.x + tid; r < a.n_c; r += stride) {
      const int node = a.c_node[r];
      OUTc[node] = Uc[node] + c1 * a.v_c[oc + r] + c2 * a.a_c[oc + r];
    }
    return;
  }

  double* su = sm;                          // R^3
  double* TK = su + R * R * R;              // R x R x OX
  double* TM = TK + R * R * OX;
  double* reg = TM + R * R * OX;            // x-pass partials, then y-pass arrays
  double* xlk = reg;                        // R*R x NC each
  double* xrk = xlk + R * R * NC;
  double* xlm = xrk + R * R * NC;
  double* xrm = xlm + R * R * NC;
  double* AB = reg;                         // R x OX(y) x OX(x)
  double* CC = AB + R * OX * OX;
  double* ylab = CC + R * OX * OX;          // R x NC x OX each
  double* yrab = ylab + R * NC * OX;
  double* ylc = yrab + R * NC * OX;
  double* yrc = ylc + R * NC * OX;
  double* rr = TK;                          // OX^3 (aliases TK/TM after the y pass)
  double* zl = rr + OX * OX * OX;           // NC x OX x OX each
  double* zr = zl + NC * OX * OX;

  const int tile = blockIdx.x;
  const int tx = tile % a.ntx, ty = (tile / a.ntx) % a.nty, tz = tile / (a.ntx * a.nty);
  const int X0 = tx * OX, Y0 = ty * OX, Z0 = tz * OX;
  const int cx0 = X0 / p - 1, cy0 = Y0 / p - 1, cz0 = Z0 / p - 1;
  const int64_t nxy = (int64_t)a.nx * a.ny;

  for (int idx = tid; idx < R * R * R; idx += kThreads) {
    const int zz = idx / (R * R), yy = (idx / R) % R, xx = idx % R;
    const int gx = X0 - p + xx, gy = Y0 - p + yy, gz = Z0 - p + zz;
    su[idx] = (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz)
                  ? Uc[(int64_t)gz * nxy + (int64_t)gy * a.nx + gx]
                  : 0.0;
  }
  __syncthreads();

  // x pass: item = (row zy, cell cc), rows fastest.
  for (int it = tid; it < R * R * NC; it += kThreads) {
    const int cc = it / (R * R), zy = it - cc * (R * R);
    const int cx = cx0 + cc;
    double ok[P], om[P];
    if (cx < 0 || cx >= a.ncx) {
#pragma unroll
      for (int i = 0; i < P; ++i) ok[i] = om[i] = 0.0;
    } else {
      double v[P];
#pragma unroll
      for (int j = 0; j < P; ++j) v[j] = su[zy * R + cc * p + j];
      k1d3<P>(ops, 0, v, ok);
      const double sa = m1d3_sa<P>(ops, v);
#pragma unroll
      for (int i = 0; i < P; ++i) om[i] = fma(ops.w[i], v[i], ops.ca[i] * sa);
    }
    if (cc >= 1) {
#pragma unroll
      for (int i = 1; i < p; ++i) {
        TK[zy * OX + (cc - 1) * p + i] = ok[i];
        TM[zy * OX + (cc - 1) * p + i] = om[i];
      }
    }
    xlk[zy * NC + cc] = ok[0];
    xrk[zy * NC + cc] = ok[p];
    xlm[zy * NC + cc] = om[0];
    xrm[zy * NC + cc] = om[p];
  }
  __syncthreads();
  for (int it = tid; it < R * R * TC; it += kThreads) {
    const int k = it / (R * R), zy = it - k * (R * R);
    TK[zy * OX + k * p] = xrk[zy * NC + k] + xlk[zy * NC + k + 1];
    TM[zy * OX + k * p] = xrm[zy * NC + k] + xlm[zy * NC + k + 1];
  }
  __syncthreads();

  // y pass: item = (z, x, cell row cr), x fastest.
  for (int it = tid; it < R * OX * NC; it += kThreads) {
    const int cr = it / (R * OX), rem = it - cr * (R * OX);
    const int z = rem / OX, x = rem - z * OX;
    const int cy = cy0 + cr;
    double ab[P], cm[P];
    if (cy < 0 || cy >= a.ncy) {
#pragma unroll
      for (int i = 0; i < P; ++i) ab[i] = cm[i] = 0.0;
    } else {
      double va[P], vb[P];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        va[j] = TK[(z * R + cr * p + j) * OX + x];
        vb[j] = TM[(z * R + cr * p + j) * OX + x];
      }
      double kb[P];
      k1d3<P>(ops, 1, vb, kb);
      const double sa = m1d3_sa<P>(ops, va), sb = m1d3_sa<P>(ops, vb);
#pragma unroll
      for (int i = 0; i < P; ++i) {
        ab[i] = fma(ops.w[i], va[i], fma(ops.ca[i], sa, kb[i]));
        cm[i] = fma(ops.w[i], vb[i], ops.ca[i] * sb);
      }
    }
    if (cr >= 1) {
#pragma unroll
      for (int i = 1; i < p; ++i) {
        AB[(z * OX + (cr - 1) * p + i) * OX + x] = ab[i];
        CC[(z * OX + (cr - 1) * p + i) * OX + x] = cm[i];
      }
    }
    ylab[(z * NC + cr) * OX + x] = ab[0];
    yrab[(z * NC + cr) * OX + x] = ab[p];
    ylc[(z * NC + cr) * OX + x] = cm[0];
    yrc[(z * NC + cr) * OX + x] = cm[p];
  }
  __syncthreads();
  for (int it = tid; it < R * TC * OX; it += kThreads) {
    const int k = it / (R * OX), rem = it - k * (R * OX);
    const int z = rem / OX, x = rem - z * OX;
    AB[(z * OX + k * p) * OX + x] = yrab[(z * NC + k) * OX + x] + ylab[(z * NC + k + 1) * OX + x];
    CC[(z * OX + k * p) * OX + x] = yrc[(z * NC + k) * OX + x] + ylc[(z * NC + k + 1) * OX + x];
  }
  __syncthreads();

  // z pass: item = (y, x, cell layer cl), x fastest.
  for (int it = tid; it < OX * OX * NC; it += kThreads) {
    const int cl = it / (OX * OX), yx = it - cl * (OX * OX);
    const int cz = cz0 + cl;
    double o[P];
    if (cz < 0 || cz >= a.ncz) {
#pragma unroll
      for (int i = 0; i < P; ++i) o[i] = 0.0;
    } else {
      double va[P], vb[P];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        va[j] = AB[(cl * p + j) * OX * OX + yx];
        vb[j] = CC[(cl * p + j) * OX * OX + yx];
      }
      double kb[P];
      k1d3<P>(ops, 2, vb, kb);
      const double sa = m1d3_sa<P>(ops, va);
#pragma unroll
      for (int i = 0; i < P; ++i) o[i] = fma(ops.w[i], va[i], fma(ops.ca[i], sa, kb[i]));
    }
    if (cl >= 1) {
#pragma unroll
      for (int i = 1; i < p; ++i) rr[((cl - 1) * p + i) * OX * OX + yx] = o[i];
    }
    zl[cl * OX * OX + yx] = o[0];
    zr[cl * OX * OX + yx] = o[p];
  }
  __syncthreads();
  for (int it = tid; it < TC * OX * OX; it += kThreads) {
    const int k = it / (OX * OX), yx = it - k * (OX * OX);
    rr[(k * p) * OX * OX + yx] = zr[k * OX * OX + yx] + zl[(k + 1) * OX * OX + yx];
  }
  __syncthreads();

  // CDM update of the owned I_d nodes (Eqs. CDMacc, CDMstep).
  const double ft = a.ft_dev ? a.ft_dev[0] : a.ft;
  for (int it = tid; it < OX * OX * OX; it += kThreads) {
    const int zo = it / (OX * OX), yo = (it / OX) % OX, xo = it % OX;
    const int gx = X0 + xo, gy = Y0 + yo, gz = Z0 + zo;
    if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
    const int64_t g = (int64_t)gz * nxy + (int64_t)gy * a.nx + gx;
    if (a.cls[g] != NODE_D) continue;
    const double r = rr[it];
    const double u = su[((zo + p) * R + yo + p) * R + xo + p];
    const double minv = a.winv_x[gx] * a.winv_y[gy] * a.winv_z[gz];
    const double acc = minv * (ft * fxc[g] - r);
    OUTc[g] = a.cu * u + a.cw * Wc[g] + a.ca * acc;
  }
}

// ---------------------------------------------------------------------------
// A4 + A5 + A6: the implicit solve S a = f_t(t_{n+1}) f_x^c - K^c u_pred with
// the supernodal nested-dissection Cholesky factor of S, and the Newmark
// correction.  Per component, the lower levels of the dissection tree are
// walked level by level (forward: y_t = L_tt^{-1}(rhs_t - descendant updates),
// upd_t = L_{rows,t} y_t; backward: x_t = L_tt^{-T}(y_t - L_{rows,t}^T x_rows)),
// and the upper levels are one dense product x_Z = A_Z (rhs_Z - updates from
// below), A_Z = (L_ZZ L_ZZ^T)^{-1} (no lower node is an ancestor of an upper
// one, so L_BZ = 0).  Every level is one launch over all components: kernel
// boundaries are the barriers, so each launch spreads its FP64 work over every
// SM.  Within a CTA all threads share the rows of all its supernodes in each
// phase.  The first forward launch also forms the right-hand side of every
// implicit row: K^c u_pred row by row, one dot product of a row of K_e with the
// cell's nodal values per (row, interface cell) pair.  Launches are chained
// with programmatic dependent launch: a kernel stages its constant factor
// blocks and index lists (cp.async) while its predecessor runs and waits
// (griddepcontrol.wait, a hardware wait) before it reads its results.  All
// sums run in a fixed order, so results are deterministic.

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

// Newmark correction of one implicit row (Fig. TrapCDMIMEX "Correction"), or
// the initial acceleration only (mode 1), on one column's fields.
struct Corr {
  int mode;
  const int* c_node;
  double* U;      // holds u_pred on I_c (mode 0) or u^c_{n-1} (mode 3); receives u^c_{n+1}
  double* v_c;
  double* a_c;
  double dt;
  const double* Un;  // u_n (mode 3)
  __device__ void row(int r, double acc) const {
    if (mode == 2) return;   // solve only: the solution stays in sol
    if (mode == 3) {         // central differences on I_c (Eq. CDMstep): acc = a^c_n
      const int node = c_node[r];
      U[node] = 2.0 * Un[node] - U[node] + dt * dt * acc;
    } else if (mode == 0) {
      const int node = c_node[r];
      const double vpred = v_c[r] + (1.0 - kNewmarkGamma) * dt * a_c[r];
      U[node] = U[node] + kNewmarkBeta * dt * dt * acc;
      v_c[r] = vpred + kNewmarkGamma * dt * acc;
    }
    a_c[r] = acc;
  }
  // The same with c_node[r], v_c[r] and a_c[r] loaded beforehand (they are not
  // written by the kernels of the step that run before the correction).
  __device__ void row_pre(int r, double acc, int node, double v_old, double a_old) const {
    if (mode == 2) return;
    if (mode == 3) {
      U[node] = 2.0 * Un[node] - U[node] + dt * dt * acc;
    } else if (mode == 0) {
      const double vpred = v_old + (1.0 - kNewmarkGamma) * dt * a_old;
      U[node] = U[node] + kNewmarkBeta * dt * dt * acc;
      v_c[r] = vpred + kNewmarkGamma * dt * acc;
    }
    a_c[r] = acc;
  }
  // The same with U[node] (u_in) and, in mode 3, Un[node] (un_in) loaded too.
  __device__ void row_in(int r, double acc, double v_old, double a_old, int node, double u_in,
                         double un_in) const {
    if (mode == 2) return;
    if (mode == 3) {
      U[node] = 2.0 * un_in - u_in + dt * dt * acc;
    } else if (mode == 0) {
      const double vpred = v_old + (1.0 - kNewmarkGamma) * dt * a_old;
      U[node] = u_in + kNewmarkBeta * dt * dt * acc;
      v_c[r] = vpred + kNewmarkGamma * dt * acc;
    }
    a_c[r] = acc;
  }
};

// Per-CTA index list of a walk launch (ints, offsets relative to its start):
//   [0] nq nodes, [1] nslot rows (sum of b), [2] nm ancestor rows (sum of m),
//   [3] nrhs, [4] npair, [5] np = npair rounded up to even (first launch
//   only; the cell-matrix rows of the pairs are staged separately), [6..7] 0
//   node table at 8:          nq x {t, beg, b, m, slot0, moff, boff, updoff}
//   slot table:               nslot x {q, update begin, update end, 0}
//   ancestor table:           nm x {q, c-row}
//   right-hand-side rows:     nrhs x {c-row, pair begin, pair end, slot or -1}
//   pairs:                    npair x {first node of the cell, 0, 0, 0}
//   update positions (into upd).
struct WalkList {
  const int* h;
  const int* node;
  const int* slot;
  const int* anc;
  const int* rhs;
  const int* pair;
  __device__ explicit WalkList(const int* il) : h(il) {
    node = il + 8;
    slot = node + 8 * il[0];
    anc = slot + 4 * il[1];
    rhs = anc + ((2 * il[2] + 3) & ~3);
    pair = rhs + 4 * il[3];
  }
};

// Right-hand side of one (row, cell) pair k: row l of the cell matrix (scaled
// by the cell's c_e^2 / c0^2 where the uncut form is used), staged m-major in
// shared memory (kp[m * np + k]), times the cell's nodal values (off[m] is the
// grid offset of local node m from the cell's first node).  Loads are issued
// in batches of 16 before the products.
constexpr int kMaxPd = 128;
__device__ __forceinline__ double pair_product(const WalkArgs& a, const double* src, const double* kp, int np,
                                               int k, int base, const int* off) {
  const double* u = src + base;
  double s0 = 0.0, s1 = 0.0;
  for (int m0 = 0; m0 < a.Pd; m0 += 16) {
    double kv[16], uv[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const bool ok = m0 + t < a.Pd;
      kv[t] = ok ? kp[(size_t)(m0 + t) * np + k] : 0.0;
      uv[t] = ok ? __ldg(u + off[ok ? m0 + t : 0]) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 16; t += 2) {
      s0 = fma(kv[t], uv[t], s0);
      s1 = fma(kv[t + 1], uv[t + 1], s1);
    }
  }
  return s0 + s1;
}

// Diagonal blocks L_tt^{-1} (b x b, lower triangular) are stored packed by
// diagonals: diagonal d (entries (d + i, i), i < b - d) starts at
// d b - d (d - 1) / 2, and L_{rows,t} follows at tri_size(b).  Row i of the
// forward product reads entry (i, i - d) and column i of the backward
// product entry (i + d, i) at step d: in both, the lanes of a warp
// (consecutive i of one block) read consecutive words, and only the
// triangle is stored, staged and read.
__device__ __forceinline__ int tri_size(int b) { return b * (b + 1) / 2; }

template <bool kForward, bool kSmem, bool kCols>
__global__ void __launch_bounds__(kThreads, 1) k_walk(WalkArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int cta = a.cta0 + blockIdx.x;
  const int tid = threadIdx.x;
  // Block of independent columns (blockIdx.y): col0 .. col0 + ncb - 1.  Every
  // vector below holds one slice per column; the factor blocks are staged
  // once for all of them, and each loop runs over (item, column) pairs with
  // the item fastest.  kCols = false: one column per CTA (no column index
  // arithmetic).
  const int col0 = kCols ? blockIdx.y * a.cb : blockIdx.y, ncb = kCols ? min(a.cb, a.ncols - col0) : 1;
  const int MS = a.max_slots, MM = a.max_m, MP = a.max_pairs;
  auto on = [&](int c) { return (int64_t)(col0 + c) * a.cs_node; };
  auto oc = [&](int c) { return (int64_t)(col0 + c) * a.cs_c; };
  auto updc = [&](int c) { return a.upd + (int64_t)(col0 + c) * a.cs_upd; };
  auto corr = [&](int c) {
    return Corr{a.mode, a.c_node, a.U + on(c), a.v_c + oc(c), a.a_c + oc(c), a.dt, a.SRC + on(c)};
  };
  double* blob = sm;                                   // max_blob (smem mode)
  double* kp = blob + a.max_blob;                      // max_kp: rows of the cell matrices (first launch)
  double* vg = kp + a.max_kp;                          // cb x max_slots: g (fwd) / y (bwd)
  double* vy = vg + (size_t)a.cb * MS;                 // cb x max_slots: y (fwd) / h (bwd)
  double* vm = vy + (size_t)a.cb * MS;                 // cb x max_m: x of the ancestor rows (bwd)
  double* pc = vm + (size_t)a.cb * MM;                 // cb x max_pairs: pair products (first launch)
  int* il = reinterpret_cast<int*>(pc + (size_t)a.cb * MP);
  __shared__ int s_off[kForward ? kMaxPd : 1];         // grid offset of each local node of a cell
  if (kForward && a.first)
    for (int m = tid; m < a.Pd; m += kThreads)
      s_off[m] = (m % a.P) + a.nx * ((m / a.P) % a.P) + a.nx * a.ny * (m / (a.P * a.P));
  const int64_t boff = a.blob_off[cta];
  if (kSmem) async_copy_16(blob, a.blob + boff, a.blob_len[cta] / 2);
  async_copy_16(il, a.ilist + a.ilist_off[cta], a.ilist_len[cta] / 4);
  if (kForward && a.first && a.kp_smem) async_copy_16(kp, a.Kpair + a.kp_off[cta], a.kp_len[cta] / 2);
  const double* KP = (kForward && a.first && !a.kp_smem) ? a.Kpair + a.kp_off[cta] : kp;
  const double* B = kSmem ? blob : a.blob + boff;
  // Let the next launch stage its constants.
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  async_copy_wait();
  const WalkList L(il);
  const int nslot = il[1], nm = il[2];
  const int nsi = nslot * ncb;   // (slot, column) items
  // Backward: the correction state of this thread's first two items.
  int pre_node[2] = {0, 0};
  double pre_v[2] = {0.0, 0.0}, pre_a[2] = {0.0, 0.0};
  if (!kForward) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int it = tid + q * kThreads;
      if (it < nsi) {
        const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
        const int* nd = L.node + 8 * L.slot[4 * sl];
        const int r = nd[1] + (sl - nd[4]);
        pre_node[q] = a.c_node[r];
        pre_v[q] = a.v_c[oc(c) + r];
        pre_a[q] = a.a_c[oc(c) + r];
      }
    }
  }
  // Wait for the previous launch's results.
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  if (a.skip && *a.skip) return;   // the iterative solve converged: nothing to do
  if (kForward) {
    if (a.first && a.rhs_given) {
      for (int it = tid; it < nsi; it += kThreads) {
        const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
        const int* st = L.slot + 4 * sl;
        const int* nd = L.node + 8 * st[0];
        const double* upd = updc(c);
        double v = a.rhs0[oc(c) + nd[1] + (sl - nd[4])];
        for (int k = st[1]; k < st[2]; ++k) v -= __ldcg(upd + il[k]);
        vg[c * MS + sl] = v;
      }
    } else if (a.first) {
      const int npair = il[4], nrhs = il[3];
      // f_t at t_{n+1}, or at t_n for the central-difference form (mode 3).
      const double ft = a.ft_dev ? a.ft_dev[a.mode == 3 ? 0 : 1] : a.ft;
      const int np = il[5];
      for (int it = tid; it < npair * ncb; it += kThreads) {
        const int c = kCols ? it / npair : 0, k = kCols ? it - c * npair : it;
        pc[c * MP + k] = pair_product(a, a.SRC + on(c), KP, np, k, L.pair[4 * k], s_off);
      }
      __syncthreads();
      for (int it = tid; it < nrhs * ncb; it += kThreads) {
        const int c = kCols ? it / nrhs : 0, k = kCols ? it - c * nrhs : it;
        const int* rr = L.rhs + 4 * k;
        double v = ft * a.fxc[oc(c) + rr[0]];
        for (int q = rr[1]; q < rr[2]; ++q) v -= pc[c * MP + q];
        if (rr[3] >= 0 && !a.rhs_only) vg[c * MS + rr[3]] = v;
        else a.rhs0[oc(c) + rr[0]] = v;
      }
      if (a.rhs_only) return;   // every row's right-hand side is in rhs0
      __syncthreads();
      for (int it = tid; it < nsi; it += kThreads) {
        const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
        const int* st = L.slot + 4 * sl;
        const double* upd = updc(c);
        double v = vg[c * MS + sl];
        for (int k = st[1]; k < st[2]; ++k) v -= __ldcg(upd + il[k]);
        vg[c * MS + sl] = v;
      }
    } else {
      for (int it = tid; it < nsi; it += kThreads) {
        const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
        const int* st = L.slot + 4 * sl;
        const int* nd = L.node + 8 * st[0];
        const double* upd = updc(c);
        double v = __ldcg(a.rhs0 + oc(c) + nd[1] + (sl - nd[4]));
#pragma unroll 4
        for (int k = st[1]; k < st[2]; ++k) v -= __ldcg(upd + il[k]);
        vg[c * MS + sl] = v;
      }
    }
    __syncthreads();
    // y = L_tt^{-1} g, every row of every supernode of this CTA; row i
    // reads entry (i, i - d) at d = 0, 1, ..., i (see tri_size).
    for (int it = tid; it < nsi; it += kThreads) {
      const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
      const int* nd = L.node + 8 * L.slot[4 * sl];
      const int b = nd[2], s0 = nd[4], i = sl - s0;
      const double* Lp = B + nd[6];
      const double* g = vg + c * MS + s0 + i;   // g[-d] = g_{i-d}
      double y0 = 0.0, y1 = 0.0;
      int d = 0, q = i;
      for (; d + 2 <= i + 1; d += 2) {
        y0 = fma(Lp[q], g[-d], y0);
        q += b - d - 1;
        y1 = fma(Lp[q], g[-d - 1], y1);
        q += b - d - 2;
      }
      if (d <= i) y0 = fma(Lp[q], g[-d], y0);
      const double y = y0 + y1;
      vy[c * MS + sl] = y;
      a.sol[oc(c) + nd[1] + i] = y;
    }
    __syncthreads();
    // upd_t = L_{rows,t} y_t.
    for (int it = tid; it < nm * ncb; it += kThreads) {
      const int c = kCols ? it / nm : 0, k = kCols ? it - c * nm : it;
      const int* nd = L.node + 8 * L.anc[2 * k];
      const int b = nd[2], m = nd[3], s0 = nd[4], kk = k - nd[5], ldr = m | 1;
      const double* L21 = B + nd[6] + tri_size(b);
      const double* y = vy + c * MS + s0;
      double u0 = 0.0, u1 = 0.0;
      int j = 0;
      for (; j + 2 <= b; j += 2) {
        u0 = fma(L21[kk + ldr * j], y[j], u0);
        u1 = fma(L21[kk + ldr * (j + 1)], y[j + 1], u1);
      }
      if (j < b) u0 = fma(L21[kk + ldr * j], y[j], u0);
      updc(c)[nd[7] + kk] = u0 + u1;
    }
  } else {
    for (int it = tid; it < nm * ncb; it += kThreads) {
      const int c = kCols ? it / nm : 0, k = kCols ? it - c * nm : it;
      vm[c * MM + k] = __ldcg(a.sol + oc(c) + L.anc[2 * k + 1]);
    }
    for (int it = tid; it < nsi; it += kThreads) {
      const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
      const int* nd = L.node + 8 * L.slot[4 * sl];
      vg[c * MS + sl] = __ldcg(a.sol + oc(c) + nd[1] + (sl - nd[4]));
    }
    __syncthreads();
    // h = y_t - L_{rows,t}^T x_rows.
    for (int it = tid; it < nsi; it += kThreads) {
      const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
      const int* nd = L.node + 8 * L.slot[4 * sl];
      const int b = nd[2], m = nd[3], i = sl - nd[4], mo = nd[5], ldr = m | 1;
      const double* L21 = B + nd[6] + tri_size(b) + (size_t)ldr * i;
      const double* x = vm + c * MM + mo;
      double h0 = 0.0, h1 = 0.0;
      int k = 0;
      for (; k + 2 <= m; k += 2) {
        h0 = fma(L21[k], x[k], h0);
        h1 = fma(L21[k + 1], x[k + 1], h1);
      }
      if (k < m) h0 = fma(L21[k], x[k], h0);
      vy[c * MS + sl] = vg[c * MS + sl] - (h0 + h1);
    }
    __syncthreads();
    // x_t = L_tt^{-T} h, then the correction of the row; column i reads
    // entry (i + d, i) at d = 0, 1, ..., b - 1 - i.
    for (int it = tid; it < nsi; it += kThreads) {
      const int c = kCols ? it / nslot : 0, sl = kCols ? it - c * nslot : it;
      const int* nd = L.node + 8 * L.slot[4 * sl];
      const int b = nd[2], s0 = nd[4], i = sl - s0, n = b - i;
      const double* Lp = B + nd[6];
      const double* h = vy + c * MS + s0 + i;   // h[d] = h_{i+d}
      double x0 = 0.0, x1 = 0.0;
      int d = 0, q = i;
      for (; d + 2 <= n; d += 2) {
        x0 = fma(Lp[q], h[d], x0);
        q += b - d;
        x1 = fma(Lp[q], h[d + 1], x1);
        q += b - d - 1;
      }
      if (d < n) x0 = fma(Lp[q], h[d], x0);
      const double x = x0 + x1;
      a.sol[oc(c) + nd[1] + i] = x;
      const Corr cor = corr(c);
      if (it < tid + kThreads) cor.row_pre(nd[1] + i, x, pre_node[0], pre_v[0], pre_a[0]);
      else if (it < tid + 2 * kThreads) cor.row_pre(nd[1] + i, x, pre_node[1], pre_v[1], pre_a[1]);
      else cor.row(nd[1] + i, x);
    }
  }
}

template <bool kCols>
__global__ void __launch_bounds__(kThreads) k_top(TopArgs a) {
  extern __shared__ __align__(16) double tsm[];
  const int cta = blockIdx.x, tid = threadIdx.x;
  // Block of independent columns (blockIdx.y): col0 .. col0 + ncb - 1; the
  // chunk of A_Z is staged once and each of its entries is loaded once for
  // up to four columns.  kCols = false: one column per CTA.
  const int col0 = kCols ? blockIdx.y * a.cb : blockIdx.y, ncb = kCols ? min(a.cb, a.ncols - col0) : 1;
  auto on = [&](int c) { return (int64_t)(col0 + c) * a.cs_node; };
  auto oc = [&](int c) { return (int64_t)(col0 + c) * a.cs_c; };
  auto corr = [&](int c) {
    return Corr{a.mode, a.c_node, a.U + on(c), a.v_c + oc(c), a.a_c + oc(c), a.dt, a.Un ? a.Un + on(c) : nullptr};
  };
  const int comp = a.cta_comp[cta], r0 = a.cta_r0[cta], r1 = a.cta_r1[cta];
  const int zn = a.zsize[comp], zb = a.zbase[comp], nr = r1 - r0, MZ = a.max_zn;
  double* zs = tsm;                               // cb x max_zn (even): right-hand sides of the block
  double* Ac = zs + (size_t)a.cb * MZ;            // max_arows: this CTA's rows of A_Z
  double* xs = Ac + a.max_arows;                  // cb x kThreads: partial dot products
  int* il = reinterpret_cast<int*>(xs + (size_t)a.cb * kThreads);  // per row {update begin, end}, positions
  async_copy_16(Ac, a.zA + a.zA_off[comp] + (size_t)r0 * zn, ((int64_t)nr * zn + 1) / 2);
  async_copy_16(il, a.ilist + a.ilist_off[cta], a.ilist_len[cta] / 4);
  // c-index of this thread's first kZr rows of the block (registers: the
  // shared memory of this kernel is kept small enough to share an SM with
  // the walk launches that run before it).
  constexpr int kZr = 3;
  int zr[kZr];
#pragma unroll
  for (int q = 0; q < kZr; ++q) zr[q] = tid + q * kThreads < zn ? a.zrow[zb + tid + q * kThreads] : 0;
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  // The correction state of this thread's row in the first column (nr <=
  // blockDim.x); not written by the launches of the step that run before
  // this one.
  const Corr cor0 = corr(0);
  int row = 0, node = 0;
  double v_old = 0.0, a_old = 0.0;
  if (tid < nr) {
    row = a.zrow[zb + r0 + tid];
    node = cor0.c_node[row];
    v_old = cor0.v_c[row];
    a_old = cor0.a_c[row];
  }
  async_copy_wait();
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  if (a.skip && *a.skip) return;   // the iterative solve converged: nothing to do
  // Inputs of the correction written by the earlier launches of the step,
  // loaded now so that their latency overlaps the gather.
  double u_in = 0.0, un_in = 0.0;
  if (tid < nr && cor0.mode != 2) {
    u_in = __ldcg(cor0.U + node);
    if (cor0.mode == 3) un_in = __ldcg(cor0.Un + node);
  }
  // The whole right-hand side of this component's top block, every column
  // (redundant per CTA).
  auto gather = [&](int c, int i, int zri) {
    const int fb = il[2 * i], fe = il[2 * i + 1];
    const double* upd = a.upd + (int64_t)(col0 + c) * a.cs_upd;
    double v = __ldcg(a.rhs0 + oc(c) + zri);
#pragma unroll 4
    for (int k = fb; k < fe; ++k) v -= __ldcg(upd + il[k]);
    zs[(size_t)c * MZ + i] = v;
  };
#pragma unroll
  for (int q = 0; q < kZr; ++q)
    if (tid + q * kThreads < zn) gather(0, tid + q * kThreads, zr[q]);
  for (int i = tid + kZr * kThreads; i < zn; i += kThreads) gather(0, i, a.zrow[zb + i]);
  if (kCols)
    for (int it = tid; it < zn * (ncb - 1); it += kThreads) {
      const int c = 1 + it / zn, i = it - (c - 1) * zn;
      gather(c, i, a.zrow[zb + i]);
    }
  __syncthreads();
  // Rows of A_Z times z.  The chunk is stored column-major (row i, column
  // j at j * nr + i); thread (s, i) takes row i over the s-th of S column
  // slices, so a warp reads consecutive words, and the slices are summed
  // pairwise (S - 1 additions per row, spread over the threads).  Per column
  // the sums run in the same order whatever the column block.
  const int nslice = min(kThreads / max(nr, 1), max(zn / 2, 1));
  if (tid < nslice * nr) {
    const int s = tid / nr, i = tid - s * nr;
    const int j0 = zn * s / nslice, j1 = zn * (s + 1) / nslice;
    const double* Ai = Ac + i;
    int c = 0;
    for (; kCols && c + 4 <= ncb; c += 4) {
      const double* z = zs + (size_t)c * MZ;
      double s0[4] = {0.0, 0.0, 0.0, 0.0}, s1[4] = {0.0, 0.0, 0.0, 0.0};
      int j = j0;
      for (; j + 2 <= j1; j += 2) {
        const double e0 = Ai[(size_t)j * nr], e1 = Ai[(size_t)(j + 1) * nr];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          s0[q] = fma(e0, z[q * MZ + j], s0[q]);
          s1[q] = fma(e1, z[q * MZ + j + 1], s1[q]);
        }
      }
      if (j < j1) {
        const double e0 = Ai[(size_t)j * nr];
#pragma unroll
        for (int q = 0; q < 4; ++q) s0[q] = fma(e0, z[q * MZ + j], s0[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) xs[(size_t)(c + q) * kThreads + tid] = s0[q] + s1[q];
    }
    for (; c < ncb; ++c) {
      const double* z = zs + (size_t)c * MZ;
      double s0 = 0.0, s1 = 0.0;
      int j = j0;
      for (; j + 2 <= j1; j += 2) {
        s0 = fma(Ai[(size_t)j * nr], z[j], s0);
        s1 = fma(Ai[(size_t)(j + 1) * nr], z[j + 1], s1);
      }
      if (j < j1) s0 = fma(Ai[(size_t)j * nr], z[j], s0);
      xs[(size_t)c * kThreads + tid] = s0 + s1;
    }
  }
  __syncthreads();
  for (int h = nslice; h > 1;) {
    const int h2 = (h + 1) / 2;   // slice s < h - h2 takes in slice s + h2
    if (tid < (h - h2) * nr)
      for (int c = 0; c < (kCols ? ncb : 1); ++c) xs[(size_t)c * kThreads + tid] += xs[(size_t)c * kThreads + tid + h2 * nr];
    h = h2;
    __syncthreads();
  }
  if (tid < nr) {
    const double x = xs[tid];
    a.sol[oc(0) + row] = x;
    cor0.row_in(row, x, v_old, a_old, node, u_in, un_in);
    for (int c = 1; kCols && c < ncb; ++c) {
      const double xc = xs[(size_t)c * kThreads + tid];
      a.sol[oc(c) + row] = xc;
      corr(c).row(row, xc);
    }
  }
}


// ---------------------------------------------------------------------------
// Large supernodes of the walked levels (PanelArgs): each CTA multiplies one
// chunk of rows of a dense block (the inverted diagonal block, its
// transpose, the block below it or its transpose) by a gathered vector.  The
// chunk is staged (cp.async) before the grid-dependency wait; threads (s, i)
// take row i over the s-th column slice and the slices are summed pairwise,
// as in k_top.  Fixed-order sums: results do not depend on timing.
__global__ void __launch_bounds__(kThreads) k_panel(PanelArgs a) {
  extern __shared__ __align__(16) double psm[];
  const int cta = a.cta0 + blockIdx.x, tid = threadIdx.x;
  const int64_t on = (int64_t)blockIdx.y * a.cs_node, oc = (int64_t)blockIdx.y * a.cs_c;
  const double* rhs0 = a.rhs0 + oc;
  double* sol = a.sol + oc;
  double* hbuf = a.hbuf + oc;
  double* upd = a.upd + (int64_t)blockIdx.y * a.cs_upd;
  const Corr cor{a.mode, a.c_node, a.U + on, a.v_c + oc, a.a_c + oc, a.dt, a.Un ? a.Un + on : nullptr};
  const int* d = a.desc + 8 * cta;
  const int kind = d[0], nr = d[1], nv = d[2];
  const int* il = a.idx + d[3];
  const int* vin = il;                                  // nv input indices
  const int* vrng = il + nv;                            // kind 0: 2 nv update ranges
  const int* vout = il + (kind == 0 ? 3 * nv : nv);     // nr output indices
  double* Ac = psm;                                     // max_chunk: the chunk, column-major
  double* vs = Ac + a.max_chunk;                        // max_nv: the gathered vector
  double* xs = vs + a.max_nv;                           // kThreads: partial sums
  const int64_t n = (int64_t)nr * nv;
  async_copy_16(Ac, a.A + a.a_off[cta], (n + 1) / 2);
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  async_copy_wait();
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  if (a.skip && *a.skip) return;   // the iterative solve converged: nothing to do
  for (int j = tid; j < nv; j += kThreads) {
    const int c = vin[j];
    double v;
    if (kind == 0) {
      v = __ldcg(rhs0 + c);
      for (int q = vrng[2 * j]; q < vrng[2 * j + 1]; ++q) v -= __ldcg(upd + il[q]);
    } else if (kind == 3) {
      v = __ldcg(hbuf + c);
    } else {
      v = __ldcg(sol + c);
    }
    vs[j] = v;
  }
  __syncthreads();
  const int nslice = min(kThreads / max(nr, 1), max(nv / 2, 1));
  if (tid < nslice * nr) {
    const int s = tid / nr, i = tid - s * nr;
    const int j0 = (int)((int64_t)nv * s / nslice), j1 = (int)((int64_t)nv * (s + 1) / nslice);
    const double* Ai = Ac + i;
    double s0 = 0.0, s1 = 0.0;
    int j = j0;
    for (; j + 2 <= j1; j += 2) {
      s0 = fma(Ai[(size_t)j * nr], vs[j], s0);
      s1 = fma(Ai[(size_t)(j + 1) * nr], vs[j + 1], s1);
    }
    if (j < j1) s0 = fma(Ai[(size_t)j * nr], vs[j], s0);
    xs[tid] = s0 + s1;
  }
  __syncthreads();
  for (int h = nslice; h > 1;) {
    const int h2 = (h + 1) / 2;   // slice s < h - h2 takes in slice s + h2
    if (tid < (h - h2) * nr) xs[tid] += xs[tid + h2 * nr];
    h = h2;
    __syncthreads();
  }
  if (tid < nr) {
    const double acc = xs[tid];
    const int c = vout[tid];
    if (kind == 0) {
      sol[c] = acc;
    } else if (kind == 1) {
      upd[c] = acc;
    } else if (kind == 2) {
      hbuf[c] = __ldcg(sol + c) - acc;
    } else {
      sol[c] = acc;
      cor.row(c, acc);
    }
  }
}
