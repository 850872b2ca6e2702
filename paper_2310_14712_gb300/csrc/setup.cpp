// Host setup of the immersed Newmark IMEX method.  See setup.h.
//
// Paper passages followed:
//   * Sec. "Spatial discretization": GLL Lagrange basis (Eq. Lagrange and the
//     GLL point definition), alpha-scaled M, K, f (Eqs. Mglobal, K, f),
//     quadrature choice (GLL mass / GL stiffness and load on uncut cells,
//     spacetree GL on cut cells), empty cells discarded (fill ratio < 1e-10).
//   * Sec. "Partitioning": I_c = DOFs of cut cells, I_d = the rest (Eq. MStructure).
//   * Fig. TrapCDMIMEX: "Calculation and factorization of system matrix"
//     S = M^cc + beta dt^2 K^cc, factorised once.
// The factorisation is a supernodal Cholesky L L^T on a geometric nested
// dissection of each connected component of I_c (separators are grid lines or
// planes through cell vertices, which no cell crosses); the paper only says
// "factorization", this ordering is chosen for a short dependency chain on the GPU.
#include "setup.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <exception>
#include <functional>
#include <limits>
#include <mutex>
#include <numeric>
#include <thread>

namespace imex {

namespace {

constexpr double kBeta = 0.25;
constexpr double kEmptyFill = 1e-10;
constexpr int kLeafSize = 64;

// ---------------------------------------------------------------- 1D basis

// Legendre P_n(x) by the three-term recurrence; also returns P_{n-1}(x).
void legendre_pair(int n, double x, double& pn, double& pnm1) {
  double a = 1.0, b = x;
  if (n == 0) { pn = 1.0; pnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  pn = b;
  pnm1 = a;
}

}  // namespace

void gauss_points(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre_pair(n, z, pn, pm);
      double dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double pn, pm;
    legendre_pair(n, z, pn, pm);
    double dp = n * (z * pn - pm) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void gll_points(int p, std::vector<double>& x, std::vector<double>& w) {
  // Endpoints and the p-1 roots of P_p' (Newton on P_p' with P_p'' from the
  // Legendre equation), weights 2 / (p (p+1) P_p(x)^2).
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double z = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre_pair(p, z, pn, pm);
      double d1 = p * (z * pn - pm) / (z * z - 1.0);
      double d2 = (2.0 * z * d1 - p * (p + 1.0) * pn) / (1.0 - z * z);
      double dz = d1 / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[j] = z;
  }
  for (int j = 0; j <= p; ++j) {
    double pn, pm;
    legendre_pair(p, x[j], pn, pm);
    w[j] = 2.0 / (p * (p + 1.0) * pn * pn);
  }
}

namespace {

struct Lagrange1D {
  std::vector<double> nodes, lam;  // lam_i = 1 / prod_{k != i} (x_i - x_k)
  explicit Lagrange1D(const std::vector<double>& xn) : nodes(xn), lam(xn.size()) {
    const int n = (int)xn.size();
    for (int i = 0; i < n; ++i) {
      double d = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != i) d *= (xn[i] - xn[k]);
      lam[i] = 1.0 / d;
    }
  }
  // N_i(x) = lam_i prod_{k != i} (x - x_k);  N_i'(x) = lam_i sum_{k != i} prod_{j != i,k} (x - x_j)
  void eval(double x, double* val, double* der) const {
    const int n = (int)nodes.size();
    for (int i = 0; i < n; ++i) {
      double pv = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != i) pv *= (x - nodes[k]);
      val[i] = lam[i] * pv;
      double s = 0.0;
      for (int k = 0; k < n; ++k) {
        if (k == i) continue;
        double t = 1.0;
        for (int j = 0; j < n; ++j)
          if (j != i && j != k) t *= (x - nodes[j]);
        s += t;
      }
      der[i] = lam[i] * s;
    }
  }
};

// ---------------------------------------------------------------- geometry

struct Geometry {
  int dim;
  int nh;
  std::vector<double> c, a;  // nh x dim
  explicit Geometry(const Problem& pb) : dim(pb.dim) {
    nh = (int)(pb.holes.size() / (2 * dim));
    c.resize(nh * dim);
    a.resize(nh * dim);
    for (int k = 0; k < nh; ++k)
      for (int d = 0; d < dim; ++d) {
        c[k * dim + d] = pb.holes[k * 2 * dim + d];
        a[k * dim + d] = pb.holes[k * 2 * dim + dim + d];
      }
  }
  // Physical iff strictly outside every hole.
  bool physical(const double* x) const {
    for (int k = 0; k < nh; ++k) {
      double s = 0.0;
      for (int d = 0; d < dim; ++d) {
        double t = (x[d] - c[k * dim + d]) / a[k * dim + d];
        s += t * t;
      }
      if (s <= 1.0) return false;
    }
    return true;
  }
  // Exact box classification against axis-aligned ellipsoids.
  int classify(const double* lo, const double* hi) const {
    bool cut = false;
    for (int k = 0; k < nh; ++k) {
      double dmin = 0.0, dmax = 0.0;
      for (int d = 0; d < dim; ++d) {
        double l = (lo[d] - c[k * dim + d]) / a[k * dim + d];
        double u = (hi[d] - c[k * dim + d]) / a[k * dim + d];
        double nearest = (l > 0.0) ? l : ((u < 0.0) ? u : 0.0);
        double far = std::max(std::fabs(l), std::fabs(u));
        dmin += nearest * nearest;
        dmax += far * far;
      }
      if (dmax <= 1.0) return CELL_EMPTY;
      if (dmin < 1.0) cut = true;
    }
    return cut ? CELL_CUT : CELL_UNCUT;
  }
};

// ---------------------------------------------------------------- helpers

struct Grid {
  int dim, p, P, Pd;
  int nc[3], nn[3];
  double lo[3], h[3];
  int64_t cell_id(const int* ci) const {
    int64_t id = 0, s = 1;
    for (int d = 0; d < dim; ++d) { id += ci[d] * s; s *= nc[d]; }
    return id;
  }
  void cell_coords(int64_t id, int* ci) const {
    for (int d = 0; d < dim; ++d) { ci[d] = (int)(id % nc[d]); id /= nc[d]; }
  }
  int64_t node_id(const int* ni) const {
    int64_t id = 0, s = 1;
    for (int d = 0; d < dim; ++d) { id += ni[d] * s; s *= nn[d]; }
    return id;
  }
  void node_coords(int64_t id, int* ni) const {
    for (int d = 0; d < dim; ++d) { ni[d] = (int)(id % nn[d]); id /= nn[d]; }
  }
  // Global node ids of a cell, local order x fastest.
  void cell_nodes(int64_t cid, int* out) const {
    int ci[3] = {0, 0, 0};
    cell_coords(cid, ci);
    for (int l = 0; l < Pd; ++l) {
      int r = l, ni[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) { ni[d] = ci[d] * p + r % P; r /= P; }
      out[l] = (int)node_id(ni);
    }
  }
};

// Per-point tensor-basis values and physical gradients.
void tensor_basis(const Grid& g, const Lagrange1D& L, const double* xr, double* N, double* G) {
  double v[3][16], dv[3][16];
  for (int d = 0; d < g.dim; ++d) L.eval(xr[d], v[d], dv[d]);
  for (int l = 0; l < g.Pd; ++l) {
    int idx[3] = {0, 0, 0}, r = l;
    for (int d = 0; d < g.dim; ++d) { idx[d] = r % g.P; r /= g.P; }
    double n = 1.0;
    for (int d = 0; d < g.dim; ++d) n *= v[d][idx[d]];
    N[l] = n;
    for (int gd = 0; gd < g.dim; ++gd) {
      double t = 2.0 / g.h[gd];
      for (int d = 0; d < g.dim; ++d) t *= (d == gd) ? dv[d][idx[d]] : v[d][idx[d]];
      G[gd * g.Pd + l] = t;
    }
  }
}

struct QPoint { double xr[3]; double w; bool phys; };

// Quadrature points of one cut cell are taken in batches of kPointBatch; the
// entries of K_e and M_e are updated kEntryBlock rows at a time.
constexpr int kPointBatch = 64;
constexpr int kEntryBlock = 8;

// K_e += sum_j kw_j G_j G_j^T and M_e += sum_j mw_j N_j N_j^T over a batch of
// nq points (G_j: DIM x Pd physical gradients, N_j: Pd values; column-major
// Pd x Pd).  Each entry is loaded once per batch and takes the points in
// order, every term formed as in a point-by-point loop
// (s = sum_d G_j[d][a] (G_j[d][b] kw_j);  K_ab += s;  M_ab += N_j[a] (N_j[b] mw_j)),
// so the sums are the same, term by term.
template <int DIM>
void accumulate_points(int nq, int Pd, const double* __restrict GB, const double* __restrict NB,
                       const double* __restrict kw, const double* __restrict mw, double* __restrict gb,
                       double* __restrict nb, double* __restrict Ke, double* __restrict Me) {
  const size_t gs = (size_t)3 * Pd;            // stride of one point's gradients
  for (int b = 0; b < Pd; ++b) {
    for (int j = 0; j < nq; ++j) {
      for (int d = 0; d < DIM; ++d) gb[j * DIM + d] = GB[j * gs + (size_t)d * Pd + b] * kw[j];
      nb[j] = NB[(size_t)j * Pd + b] * mw[j];
    }
    double* __restrict kc = Ke + (size_t)Pd * b;
    double* __restrict mc = Me + (size_t)Pd * b;
    int a0 = 0;
    for (; a0 + kEntryBlock <= Pd; a0 += kEntryBlock) {
      double ka[kEntryBlock], ma[kEntryBlock];
      for (int i = 0; i < kEntryBlock; ++i) { ka[i] = kc[a0 + i]; ma[i] = mc[a0 + i]; }
      for (int j = 0; j < nq; ++j) {
        const double* Gj = GB + j * gs + a0;
        const double* Nj = NB + (size_t)j * Pd + a0;
        const double* g = gb + j * DIM;
        const double n = nb[j];
        for (int i = 0; i < kEntryBlock; ++i) {
          double sum = 0.0;
          for (int d = 0; d < DIM; ++d) sum += Gj[(size_t)d * Pd + i] * g[d];
          ka[i] += sum;
          ma[i] += Nj[i] * n;
        }
      }
      for (int i = 0; i < kEntryBlock; ++i) { kc[a0 + i] = ka[i]; mc[a0 + i] = ma[i]; }
    }
    for (int a = a0; a < Pd; ++a) {
      double ka = kc[a], ma = mc[a];
      for (int j = 0; j < nq; ++j) {
        double sum = 0.0;
        for (int d = 0; d < DIM; ++d) sum += GB[j * gs + (size_t)d * Pd + a] * gb[j * DIM + d];
        ka += sum;
        ma += NB[(size_t)j * Pd + a] * nb[j];
      }
      kc[a] = ka;
      mc[a] = ma;
    }
  }
}

// Spacetree quadrature of one cut cell: bisect a (sub)cell in every axis while
// the boundary meets its interior and level < depth; every leaf gets the
// (p+1)^dim tensor Gauss-Legendre rule.  Coordinates are in the reference cell.
void spacetree(const Grid& g, const Geometry& geo, const double* clo, int depth,
               const std::vector<double>& gx, const std::vector<double>& gw,
               std::vector<QPoint>& pts) {
  const int dim = g.dim, n1 = (int)gx.size();
  std::function<void(const double*, const double*, int)> visit =
      [&](const double* rlo, const double* rhi, int level) {
        double plo[3], phi[3];
        for (int d = 0; d < dim; ++d) {
          plo[d] = clo[d] + (rlo[d] + 1.0) * 0.5 * g.h[d];
          phi[d] = clo[d] + (rhi[d] + 1.0) * 0.5 * g.h[d];
        }
        if (level < depth && geo.classify(plo, phi) == CELL_CUT) {
          double mid[3];
          for (int d = 0; d < dim; ++d) mid[d] = 0.5 * (rlo[d] + rhi[d]);
          for (int ch = 0; ch < (1 << dim); ++ch) {
            double a[3], b[3];
            for (int d = 0; d < dim; ++d) {
              bool upper = (ch >> d) & 1;
              a[d] = upper ? mid[d] : rlo[d];
              b[d] = upper ? rhi[d] : mid[d];
            }
            visit(a, b, level + 1);
          }
          return;
        }
        int total = 1;
        for (int d = 0; d < dim; ++d) total *= n1;
        double half[3], vol = 1.0;
        for (int d = 0; d < dim; ++d) { half[d] = 0.5 * (rhi[d] - rlo[d]); vol *= half[d]; }
        for (int q = 0; q < total; ++q) {
          QPoint pt;
          int r = q;
          double w = vol;
          for (int d = 0; d < dim; ++d) {
            int i = r % n1;
            r /= n1;
            pt.xr[d] = rlo[d] + (gx[i] + 1.0) * half[d];
            w *= gw[i];
          }
          pt.w = w;
          double xp[3];
          for (int d = 0; d < dim; ++d) xp[d] = clo[d] + (pt.xr[d] + 1.0) * 0.5 * g.h[d];
          pt.phys = geo.physical(xp);
          pts.push_back(pt);
        }
      };
  double rlo[3] = {-1, -1, -1}, rhi[3] = {1, 1, 1};
  visit(rlo, rhi, 0);
}

// f_x at x: the sum of all bells, or (independent columns) bell `col` alone.
double source_value(const Problem& pb, const double* x, int col) {
  double s = 0.0;
  const int k0 = pb.ncols > 1 ? col : 0, k1 = pb.ncols > 1 ? col + 1 : pb.nsrc;
  for (int k = k0; k < k1; ++k) {
    double r2 = 0.0;
    for (int d = 0; d < pb.dim; ++d) {
      double t = x[d] - pb.src_pos[k * pb.dim + d];
      r2 += t * t;
    }
    s += pb.amp * std::exp(-r2 / (2.0 * pb.sigma * pb.sigma));
  }
  return s;
}

// Largest eigenvalue of a symmetric matrix (cyclic Jacobi rotations).
double sym_max_eig(std::vector<double> A, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = cs * akp - sn * akq;
          A[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = cs * apk - sn * aqk;
          A[q * n + k] = sn * apk + cs * aqk;
        }
      }
  }
  double m = -1e300;
  for (int i = 0; i < n; ++i) m = std::max(m, A[i * n + i]);
  return m;
}

// Largest eigenvalue of the symmetric-definite pencil (K, M), both n x n
// symmetric with M positive definite: lambda_max(L^{-1} K L^{-T}) with
// M = L L^T.  Cyclic Jacobi rotations until the off-diagonal mass is below
// (1e-15)^2 of the diagonal's.  Returns NaN when M is not positive definite.
double gen_max_eig(const double* K, const double* M, int n) {
  std::vector<double> L((size_t)n * n, 0.0), A((size_t)n * n), y(n);
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) return std::numeric_limits<double>::quiet_NaN();
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  auto lsolve = [&](double* v) {   // v <- L^{-1} v
    for (int i = 0; i < n; ++i) {
      double t = v[i];
      for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * v[k];
      v[i] = t / L[(size_t)i * n + i];
    }
  };
  std::vector<double> Y((size_t)n * n);   // Y = L^{-1} K, column j at Y[j*n ..]
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) y[i] = K[(size_t)j * n + i];
    lsolve(y.data());
    for (int i = 0; i < n; ++i) Y[(size_t)j * n + i] = y[i];
  }
  // A = L^{-1} Y^T: column j of Y^T is row j of Y.
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) y[i] = Y[(size_t)i * n + j];
    lsolve(y.data());
    for (int i = 0; i < n; ++i) A[(size_t)i * n + j] = y[i];
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = v;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < n; ++i) {
      dia += A[(size_t)i * n + i] * A[(size_t)i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    }
    if (off <= 1e-30 * dia) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = cs * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = cs * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + cs * aqk;
        }
      }
  }
  double m = -1e300;
  for (int i = 0; i < n; ++i) m = std::max(m, A[(size_t)i * n + i]);
  return m;
}

// The first exception thrown on any of several threads, rethrown by the
// thread that joins them (an exception must not leave a std::thread).
struct FirstError {
  std::mutex mu;
  std::exception_ptr first;
  template <class F>
  void run(F&& f) {
    try {
      f();
    } catch (...) {
      std::lock_guard<std::mutex> lock(mu);
      if (!first) first = std::current_exception();
    }
  }
  bool failed() {
    std::lock_guard<std::mutex> lock(mu);
    return (bool)first;
  }
  void rethrow() {
    if (first) std::rethrow_exception(first);
  }
};

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  nt = (unsigned)std::min<int64_t>(nt, std::max<int64_t>(1, n / 16));
  if (nt <= 1) { fn(0, n); return; }
  std::vector<std::thread> th;
  FirstError err;
  int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min<int64_t>(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([&fn, &err, b, e] { err.run([&] { fn(b, e); }); });
  }
  for (auto& t : th) t.join();
  err.rethrow();
}

// Sparse symmetric matrix on the implicit partition, rows sorted (full pattern).
struct CsrMat {
  int n = 0;
  std::vector<int> ptr, col;
  std::vector<double> val;
};

CsrMat coo_to_csr(int n, std::vector<std::pair<int64_t, double>>& e) {
  std::sort(e.begin(), e.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  CsrMat m;
  m.n = n;
  m.ptr.assign(n + 1, 0);
  for (size_t k = 0; k < e.size();) {
    int64_t key = e[k].first;
    double s = 0.0;
    while (k < e.size() && e[k].first == key) s += e[k++].second;
    int r = (int)(key / n), c = (int)(key % n);
    m.col.push_back(c);
    m.val.push_back(s);
    m.ptr[r + 1]++;
  }
  for (int i = 0; i < n; ++i) m.ptr[i + 1] += m.ptr[i];
  return m;
}

}  // namespace

// ------------------------------------------------------------------ build

namespace {

// fn(b, e) over [0, n) on the host's threads when the loop carries enough
// work (about `work` operations in all); serially otherwise.  Every index is
// computed by the same operations either way.
// parallel_for with dynamic scheduling: threads take blocks of `grain`
// indices from a shared counter, for loops whose iterations differ in cost.
// fn must write only what belongs to its own indices.
void parallel_for_dynamic(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& fn) {
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  nt = (unsigned)std::min<int64_t>(nt, (n + grain - 1) / grain);
  if (nt <= 1) { fn(0, n); return; }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> th;
  FirstError err;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&] {
      err.run([&] {
        for (int64_t b; !err.failed() && (b = next.fetch_add(grain)) < n;) fn(b, std::min(n, b + grain));
      });
    });
  for (auto& t : th) t.join();
  err.rethrow();
}

void parallel_if(int64_t n, double work, const std::function<void(int64_t, int64_t)>& fn) {
  if (work < 2e6) fn(0, n);
  else parallel_for(n, fn);
}

// Multifrontal supernodal Cholesky over the nested-dissection tree.  The
// large fronts (the separators near the root) run their independent rows and
// columns on the host's threads; results do not depend on the thread count.
// Columns of a front are factorised in panels of kPanel.
constexpr int kPanel = 64;

// Partial Cholesky of the first b columns of a front (fm x fm, row-major,
// lower part valid): on return columns 0..b-1 hold L and the trailing block
// holds F22 - L21 L21^T.  Each entry (i, j) is reduced by the products
// L_iq L_jq one at a time in increasing q, starting from the assembled value,
// and column j is then divided by L_jj: the column-by-column (dot-product)
// form, with the same arithmetic per entry.  The order of work differs:
// within a panel the columns are finished one by one using the panel's own
// earlier columns, and then every entry to the right of the panel subtracts
// the panel's products (in increasing q), so each panel is read from cache
// rather than the whole front for every column.
std::string partial_cholesky(double* Fr, int fm, int b) {
  for (int j0 = 0; j0 < b; j0 += kPanel) {
    const int j1 = std::min(b, j0 + kPanel);
    for (int j = j0; j < j1; ++j) {
      double* Rj = Fr + (size_t)j * fm;
      double d = Rj[j];
      for (int q = j0; q < j; ++q) d -= Rj[q] * Rj[q];
      if (!(d > 0.0)) return "implicit system is not positive definite";
      const double l = std::sqrt(d);
      Rj[j] = l;
      for (int i = j + 1; i < fm; ++i) {
        double* Ri = Fr + (size_t)i * fm;
        double s = Ri[j];
        for (int q = j0; q < j; ++q) s -= Ri[q] * Rj[q];
        Ri[j] = s / l;
      }
    }
    const int ntr = fm - j1;
    if (ntr <= 0) continue;
    // Entries right of the panel, row by row, four columns at a time (four
    // independent sums over the panel's q, each in increasing q).
    auto rows = [&](int64_t r0, int64_t r1) {
      for (int i = j1 + (int)r0; i < j1 + (int)r1; ++i) {
        double* Ri = Fr + (size_t)i * fm;
        int jj = j1;
        for (; jj + 4 <= i + 1; jj += 4) {
          const double* C0 = Fr + (size_t)jj * fm;
          const double* C1 = C0 + fm;
          const double* C2 = C1 + fm;
          const double* C3 = C2 + fm;
          double s0 = Ri[jj], s1 = Ri[jj + 1], s2 = Ri[jj + 2], s3 = Ri[jj + 3];
          for (int q = j0; q < j1; ++q) {
            const double x = Ri[q];
            s0 -= x * C0[q];
            s1 -= x * C1[q];
            s2 -= x * C2[q];
            s3 -= x * C3[q];
          }
          Ri[jj] = s0;
          Ri[jj + 1] = s1;
          Ri[jj + 2] = s2;
          Ri[jj + 3] = s3;
        }
        for (; jj <= i; ++jj) {
          const double* C = Fr + (size_t)jj * fm;
          double s = Ri[jj];
          for (int q = j0; q < j1; ++q) s -= Ri[q] * C[q];
          Ri[jj] = s;
        }
      }
    };
    if (0.5 * ntr * (double)ntr * (j1 - j0) < 2e6) rows(0, ntr);
    else parallel_for_dynamic(ntr, 16, rows);
  }
  return "";
}

std::string factorize(const CsrMat& A, HostSetup& hs, Factor& F) {
  const int n = (int)hs.n_c;
  const int nnode = (int)hs.tree.size();
  // Offsets of every node's blocks, in node order (the layout does not depend
  // on the order in which the fronts are computed).
  int64_t total = 0, ld_total = 0;
  F.ld_off.assign(nnode, 0);
  for (int k = 0; k < nnode; ++k) {
    const TreeNode& t = hs.tree[k];
    const int b = t.end - t.beg, m = (int)t.rows.size();
    total += 2LL * b * b + 2LL * m * b;
    F.ld_off[k] = ld_total;
    ld_total += (int64_t)b * b;
  }
  F.vals.assign(total, 0.0);
  F.Ld.assign(ld_total, 0.0);
  std::vector<std::vector<double>> upd(nnode);
  std::vector<std::vector<int>> children(nnode);
  for (int k = 0; k < nnode; ++k)
    if (hs.tree[k].parent >= 0) children[hs.tree[k].parent].push_back(k);

  // One front: assemble it from A and the children's update matrices (in the
  // children's order), factorise its b pivot columns, leave its own update
  // matrix in upd[k] and store its blocks.  pos (n entries, all -1 on entry
  // and on return) maps c-indices to front positions.
  auto front = [&](int k, std::vector<int>& pos) -> std::string {
    const TreeNode& t = hs.tree[k];
    const int b = t.end - t.beg, m = (int)t.rows.size(), fm = b + m;
    struct Reset {   // clears the front's entries of pos on every return
      std::vector<int>& pos;
      const TreeNode& t;
      ~Reset() {
        for (int i = t.beg; i < t.end; ++i) pos[i] = -1;
        for (int r : t.rows) pos[r] = -1;
      }
    } reset{pos, t};
    std::vector<double> Fr((size_t)fm * fm, 0.0);  // row-major frontal matrix (lower part)
    for (int i = 0; i < b; ++i) pos[t.beg + i] = i;
    for (int i = 0; i < m; ++i) pos[t.rows[i]] = b + i;
    for (int j = t.beg; j < t.end; ++j) {
      for (int q = A.ptr[j]; q < A.ptr[j + 1]; ++q) {
        int i = A.col[q];
        if (i < t.beg) continue;
        int pi = pos[i];
        if (pi < 0) return "symbolic structure misses an entry of the implicit system";
        Fr[(size_t)pi * fm + (j - t.beg)] += A.val[q];
      }
    }
    for (int c : children[k]) {
      const TreeNode& tc = hs.tree[c];
      const int mc = (int)tc.rows.size();
      const std::vector<double>& U = upd[c];
      for (int a = 0; a < mc; ++a) {
        int pa = pos[tc.rows[a]];
        for (int bb = 0; bb <= a; ++bb) {
          int pb = pos[tc.rows[bb]];
          if (pa < 0 || pb < 0) return "child update outside the parent front";
          int r = std::max(pa, pb), cc = std::min(pa, pb);
          Fr[(size_t)r * fm + cc] += U[(size_t)a * mc + bb];
        }
      }
      std::vector<double>().swap(upd[c]);
    }
    // Dense partial Cholesky of columns 0..b-1; the trailing block becomes
    // the update matrix for the parent, F22 - L21 L21^T (lower part, m x m row-major).
    {
      std::string err = partial_cholesky(Fr.data(), fm, b);
      if (!err.empty()) return err;
    }
    std::vector<double> U((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a)
      for (int bb = 0; bb <= a; ++bb) U[(size_t)a * m + bb] = Fr[(size_t)(b + a) * fm + b + bb];
    upd[k] = std::move(U);
    // Store, per supernode, the inverse of its diagonal block and the block
    // below it, each in both layouts so that the forward (row-owner) and the
    // backward (column-owner) products read them coalesced:
    //   Linv  = L_tt^{-1}  (b x b, column-major, lower),  LinvT = Linv^T,
    //   L21   = L_{rows,t} (m x b, column-major),         L21T  = L21^T.
    std::vector<double> Li((size_t)b * b, 0.0);
    parallel_if(b, (double)b * b * b / 6.0, [&](int64_t k0, int64_t k1) {
      for (int kc = (int)k0; kc < (int)k1; ++kc) {   // column kc of L_tt^{-1}: L x = e_kc
        for (int i = kc; i < b; ++i) {
          double sum = (i == kc) ? 1.0 : 0.0;
          for (int q = kc; q < i; ++q) sum -= Fr[(size_t)i * fm + q] * Li[q + (size_t)b * kc];
          Li[i + (size_t)b * kc] = sum / Fr[(size_t)i * fm + i];
        }
      }
    });
    // Dense L_tt (column-major), kept on the host for the dense top-level solve.
    double* Ld = F.Ld.data() + F.ld_off[k];
    for (int j = 0; j < b; ++j)
      for (int i = j; i < b; ++i) Ld[i + (size_t)b * j] = Fr[(size_t)i * fm + j];
    double* Linv = F.vals.data() + t.off_diag;
    double* LinvT = F.vals.data() + t.off_diagT;
    double* L21 = F.vals.data() + t.off_rect;
    double* L21T = F.vals.data() + t.off_rectT;
    for (int j = 0; j < b; ++j)
      for (int i = 0; i < b; ++i) {
        Linv[i + (size_t)b * j] = Li[i + (size_t)b * j];
        LinvT[j + (size_t)b * i] = Li[i + (size_t)b * j];
      }
    for (int j = 0; j < b; ++j) {
      for (int i = 0; i < m; ++i) {
        L21[i + (size_t)m * j] = Fr[(size_t)(b + i) * fm + j];
        L21T[j + (size_t)b * i] = Fr[(size_t)(b + i) * fm + j];
      }
    }
    return "";
  };

  // Fronts of different subtrees are independent: worker threads take any
  // front whose children are done (a front's arithmetic does not depend on
  // when it runs, so the factor is the same as in postorder).  After an
  // error no new front starts; the error of the lowest node reported wins.
  std::vector<int> pending(nnode), ready;
  ready.reserve(nnode);   // pushes under the lock never allocate
  for (int k = 0; k < nnode; ++k) {
    pending[k] = (int)children[k].size();
    if (pending[k] == 0) ready.push_back(k);
  }
  std::mutex mu;
  std::condition_variable cv;
  int done = 0, err_node = nnode;
  bool stop = false;
  std::string err_msg;
  FirstError thrown;
  auto worker = [&] {
    std::vector<int> pos(n, -1);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv.wait(lk, [&] { return stop || done == nnode || !ready.empty(); });
      if (stop || done == nnode) return;
      const int k = ready.back();
      ready.pop_back();
      lk.unlock();
      std::string e;
      thrown.run([&] { e = front(k, pos); });
      if (e.empty() && thrown.failed()) e = "exception";
      lk.lock();
      ++done;
      if (!e.empty()) {
        stop = true;
        if (k < err_node) { err_node = k; err_msg = e; }
      } else if (hs.tree[k].parent >= 0 && --pending[hs.tree[k].parent] == 0) {
        ready.push_back(hs.tree[k].parent);
      }
      cv.notify_all();
    }
  };
  const unsigned nt = (unsigned)std::max(1, std::min<int>(nnode, (int)std::max(1u, std::thread::hardware_concurrency())));
  std::vector<std::thread> th;
  for (unsigned i = 1; i < nt; ++i) th.emplace_back([&] { thrown.run(worker); });
  thrown.run(worker);
  for (auto& x : th) x.join();
  thrown.rethrow();
  return err_msg;
}

}  // namespace

// Host replay of the supernodal tree solve with the stored factor blocks:
// x = A^{-1} b.  Used at setup to check the factor and the device schedule.
void replay_solve(const HostSetup& hs, const Factor& F, std::vector<double>& x) {
  std::vector<double> rhs = x, upd(std::max<int64_t>(hs.upd_size, 1), 0.0), g, y;
  for (int k = 0; k < hs.ncomp; ++k) {
    const int lb = hs.comp_level_base[k], nlev = hs.comp_level_base[k + 1] - lb - 1;
    for (int l = 0; l < nlev; ++l)
      for (int q = hs.comp_level_ptr[lb + l]; q < hs.comp_level_ptr[lb + l + 1]; ++q) {
        const TreeNode& t = hs.tree.at(hs.level_nodes.at(q));
        const int b = t.end - t.beg, m = (int)t.rows.size();
        g.assign(b, 0.0);
        y.assign(b, 0.0);
        for (int i = 0; i < b; ++i) {
          const int r = t.beg + i;
          double s = rhs.at(r);
          for (int kk = hs.fwd_ptr.at(r); kk < hs.fwd_ptr.at(r + 1); ++kk) s -= upd.at(hs.fwd_pos.at(kk));
          g[i] = s;
        }
        for (int i = 0; i < b; ++i) {
          double s = 0.0;
          for (int j = 0; j < b; ++j) s += F.vals.at(t.off_diag + i + (int64_t)b * j) * g[j];
          y[i] = s;
          x.at(t.beg + i) = s;
        }
        for (int kk = 0; kk < m; ++kk) {
          double s = 0.0;
          for (int j = 0; j < b; ++j) s += F.vals.at(t.off_rect + kk + (int64_t)m * j) * y[j];
          upd.at(t.off_upd + kk) = s;
        }
      }
    for (int l = nlev - 1; l >= 0; --l)
      for (int q = hs.comp_level_ptr[lb + l]; q < hs.comp_level_ptr[lb + l + 1]; ++q) {
        const TreeNode& t = hs.tree.at(hs.level_nodes.at(q));
        const int b = t.end - t.beg, m = (int)t.rows.size();
        g.assign(b, 0.0);
        for (int j = 0; j < b; ++j) {
          double s = x.at(t.beg + j);
          for (int kk = 0; kk < m; ++kk)
            s -= F.vals.at(t.off_rectT + j + (int64_t)b * kk) * x.at(hs.rows_idx.at(t.off_rows + kk));
          g[j] = s;
        }
        for (int i = 0; i < b; ++i) {
          double s = 0.0;
          for (int j = 0; j < b; ++j) s += F.vals.at(t.off_diagT + i + (int64_t)b * j) * g[j];
          x.at(t.beg + i) = s;
        }
      }
  }
}

namespace {

// Relative residual ||A x - b|| / ||b|| of the replayed solve for a fixed b.
double factor_residual(const HostSetup& hs, const CsrMat& A, const Factor& F) {
  const int n = (int)hs.n_c;
  if (n == 0) return 0.0;
  std::vector<double> b(n), x;
  for (int i = 0; i < n; ++i) b[i] = std::sin(0.37 * i + 0.1) + 0.5;
  x = b;
  replay_solve(hs, F, x);
  double rn = 0.0, bn = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += A.val[q] * x[A.col[q]];
    rn += (s - b[i]) * (s - b[i]);
    bn += b[i] * b[i];
  }
  return std::sqrt(rn / bn);
}

}  // namespace

std::string build_setup(const Problem& pbin, HostSetup& hs) {
  auto t0 = std::chrono::steady_clock::now();
  hs = HostSetup();
  hs.pb = pbin;
  const Problem& pb = hs.pb;
  if (pb.dim != 2 && pb.dim != 3) return "dim must be 2 or 3";
  if (pb.p < 1 || pb.p > 8) return "p must be in [1, 8]";
  if (pb.depth < 0 || pb.depth > 16) return "tree depth must be in [0, 16]";
  if (!(pb.alpha > 0.0) || pb.alpha > 1.0) return "alpha must be in (0, 1]";
  if (!(pb.rho > 0.0) || !(pb.c0 > 0.0)) return "rho and c0 must be positive";
  if (pb.nsrc < 1 || (int)pb.src_pos.size() != pb.nsrc * pb.dim) return "bad source positions";
  if (pb.ncols < 1 || pb.ncols > kMaxCols || (pb.ncols > 1 && pb.ncols != pb.nsrc))
    return "independent columns need one source per column (1 <= columns <= 256)";
  const int ncols = pb.ncols;
  if (!(pb.sigma > 0.0)) return "source width must be positive";
  if (pb.holes.size() % (2 * pb.dim) != 0) return "holes array must be nholes x 2*dim";
  for (size_t k = 0; k < pb.holes.size() / (2 * pb.dim); ++k)
    for (int d = 0; d < pb.dim; ++d)
      if (!(pb.holes[k * 2 * pb.dim + pb.dim + d] > 0.0)) return "hole semi-axes must be positive";

  Grid g;
  g.dim = pb.dim;
  g.p = pb.p;
  g.P = pb.p + 1;
  g.Pd = 1;
  int64_t ncell = 1, nnode = 1;
  for (int d = 0; d < 3; ++d) { g.nc[d] = 1; g.nn[d] = 1; g.lo[d] = 0; g.h[d] = 1; }
  for (int d = 0; d < g.dim; ++d) {
    if (pb.ncells[d] < 1) return "ncells must be >= 1";
    if (!(pb.hi[d] > pb.lo[d])) return "box must have positive extent";
    g.Pd *= g.P;
    g.nc[d] = pb.ncells[d];
    g.nn[d] = pb.ncells[d] * pb.p + 1;
    g.lo[d] = pb.lo[d];
    g.h[d] = (pb.hi[d] - pb.lo[d]) / pb.ncells[d];
    ncell *= g.nc[d];
    nnode *= g.nn[d];
  }
  if (nnode > (int64_t)2000000000) return "grid too large (node ids must fit in int32)";
  if (!pb.cell_c.empty() && (int64_t)pb.cell_c.size() != ncell) return "cell_c must have one entry per cell";
  hs.dim = g.dim; hs.p = g.p; hs.P = g.P; hs.Pd = g.Pd;
  for (int d = 0; d < 3; ++d) { hs.h[d] = g.h[d]; hs.nn[d] = g.nn[d]; }
  hs.nnodes = nnode;
  hs.ncell_total = (int)ncell;
  const int P = g.P, Pd = g.Pd, dim = g.dim;

  // 1D basis and exact 1D operators (GL with P points integrates degree 2p exactly).
  std::vector<double> gx, gw;
  gll_points(g.p, hs.gll_x, hs.gll_w);
  gauss_points(P, gx, gw);
  Lagrange1D L1(hs.gll_x);
  hs.K1.assign(P * P, 0.0);
  hs.M1.assign(P * P, 0.0);
  for (int q = 0; q < P; ++q) {
    double v[16], dv[16];
    L1.eval(gx[q], v, dv);
    for (int i = 0; i < P; ++i)
      for (int k = 0; k < P; ++k) {
        hs.K1[i * P + k] += gw[q] * dv[i] * dv[k];
        hs.M1[i * P + k] += gw[q] * v[i] * v[k];
      }
  }
  const double jac = [&] { double j = 1; for (int d = 0; d < dim; ++d) j *= 0.5 * g.h[d]; return j; }();

  // Uncut-cell dense stiffness for c = c0 (column-major; symmetric).
  hs.uncutK.assign((size_t)Pd * Pd, 0.0);
  for (int a = 0; a < Pd; ++a)
    for (int b = 0; b < Pd; ++b) {
      int ia[3], ib[3], ra = a, rb = b;
      for (int d = 0; d < dim; ++d) { ia[d] = ra % P; ra /= P; ib[d] = rb % P; rb /= P; }
      double s = 0.0;
      for (int gd = 0; gd < dim; ++gd) {
        double t = jac * (2.0 / g.h[gd]) * (2.0 / g.h[gd]);
        for (int d = 0; d < dim; ++d)
          t *= (d == gd) ? hs.K1[ia[d] * P + ib[d]] : hs.M1[ia[d] * P + ib[d]];
        s += t;
      }
      hs.uncutK[a + (size_t)Pd * b] = pb.rho * pb.c0 * pb.c0 * s;
    }
  // Lumped uncut mass per local node: rho |J| prod w.
  std::vector<double> uncutM(Pd);
  for (int a = 0; a < Pd; ++a) {
    int r = a;
    double m = pb.rho * jac;
    for (int d = 0; d < dim; ++d) { m *= hs.gll_w[r % P]; r /= P; }
    uncutM[a] = m;
  }

  // Cell classification (exact box test), then spacetree quadrature of cut cells.
  Geometry geo(pb);
  hs.cell_type.assign(ncell, CELL_EMPTY);
  hs.fill.assign(ncell, 0.0);
  std::vector<int64_t> cut_cells;
  for (int64_t cid = 0; cid < ncell; ++cid) {
    int ci[3] = {0, 0, 0};
    g.cell_coords(cid, ci);
    double lo[3], hi[3];
    for (int d = 0; d < dim; ++d) { lo[d] = g.lo[d] + ci[d] * g.h[d]; hi[d] = lo[d] + g.h[d]; }
    int t = geo.classify(lo, hi);
    hs.cell_type[cid] = (int8_t)t;
    if (t == CELL_UNCUT) hs.fill[cid] = 1.0;
    if (t == CELL_CUT) cut_cells.push_back(cid);
  }
  auto cell_speed = [&](int64_t cid) { return pb.cell_c.empty() ? pb.c0 : pb.cell_c[cid]; };

  // Cut-cell element matrices by spacetree quadrature (threads over cells).
  const int64_t ncut0 = (int64_t)cut_cells.size();
  std::vector<double> cutK_all((size_t)ncut0 * Pd * Pd), cutM_all((size_t)ncut0 * Pd * Pd),
      cutF_all((size_t)ncut0 * Pd * ncols);
  std::vector<double> cut_fill(ncut0), cut_lam(ncut0, 0.0);
  if (pb.scheme < kSchemeImex || pb.scheme > kSchemeTrapezoidal) return "unknown time integration scheme";
  parallel_for_dynamic(ncut0, 8, [&](int64_t b, int64_t e) {
    std::vector<QPoint> pts;
    std::vector<double> NB((size_t)kPointBatch * Pd), GB((size_t)kPointBatch * 3 * Pd);
    std::vector<double> kwB(kPointBatch), mwB(kPointBatch), gbB(kPointBatch * 3), nbB(kPointBatch);
    for (int64_t k = b; k < e; ++k) {
      int64_t cid = cut_cells[k];
      int ci[3] = {0, 0, 0};
      g.cell_coords(cid, ci);
      double clo[3];
      for (int d = 0; d < dim; ++d) clo[d] = g.lo[d] + ci[d] * g.h[d];
      pts.clear();
      spacetree(g, geo, clo, pb.depth, gx, gw, pts);
      double wphys = 0.0, wall = 0.0;
      double* Ke = cutK_all.data() + (size_t)k * Pd * Pd;
      double* Me = cutM_all.data() + (size_t)k * Pd * Pd;
      double* fe = cutF_all.data() + (size_t)k * Pd * ncols;
      const double c = cell_speed(cid);
      for (size_t q0 = 0; q0 < pts.size(); q0 += kPointBatch) {
        const int nq = (int)std::min<size_t>(kPointBatch, pts.size() - q0);
        for (int j = 0; j < nq; ++j) {
          const QPoint& q = pts[q0 + j];
          wall += q.w;
          if (q.phys) wphys += q.w;
          const double al = q.phys ? 1.0 : pb.alpha;
          const double wq = q.w * jac * al;
          double* N = NB.data() + (size_t)j * Pd;
          tensor_basis(g, L1, q.xr, N, GB.data() + (size_t)j * 3 * Pd);
          double xp[3];
          for (int d = 0; d < dim; ++d) xp[d] = clo[d] + (q.xr[d] + 1.0) * 0.5 * g.h[d];
          double fv[kMaxCols];
          for (int col = 0; col < ncols; ++col) fv[col] = source_value(pb, xp, col);
          kwB[j] = wq * pb.rho * c * c;
          mwB[j] = wq * pb.rho;
          for (int bcol = 0; bcol < Pd; ++bcol)
            for (int col = 0; col < ncols; ++col) fe[(size_t)col * Pd + bcol] += wq * fv[col] * N[bcol];
        }
        if (dim == 2)
          accumulate_points<2>(nq, Pd, GB.data(), NB.data(), kwB.data(), mwB.data(), gbB.data(), nbB.data(), Ke, Me);
        else
          accumulate_points<3>(nq, Pd, GB.data(), NB.data(), kwB.data(), mwB.data(), gbB.data(), nbB.data(), Ke, Me);
      }
      cut_fill[k] = wphys / wall;
      if (pb.scheme == kSchemeCdmHrz) {
        // HRZ: the diagonal scaled to the element mass, off-diagonals dropped (Eqs. HRZ).
        double tot = 0.0, dsum = 0.0;
        for (size_t q = 0; q < (size_t)Pd * Pd; ++q) tot += Me[q];
        for (int a = 0; a < Pd; ++a) dsum += Me[a + (size_t)Pd * a];
        for (int a = 0; a < Pd; ++a)
          for (int b2 = 0; b2 < Pd; ++b2)
            if (a != b2) Me[a + (size_t)Pd * b2] = 0.0;
        for (int a = 0; a < Pd; ++a) Me[a + (size_t)Pd * a] *= tot / dsum;
      }
      if (scheme_is_cdm(pb.scheme)) cut_lam[k] = gen_max_eig(Ke, Me, Pd);
    }
  });
  // Fill-ratio test: cells with eta < 1e-10 are empty.
  std::vector<int> cut_slot(ncell, -1);
  std::vector<int64_t> kept;
  for (int64_t k = 0; k < ncut0; ++k) {
    int64_t cid = cut_cells[k];
    hs.fill[cid] = cut_fill[k];
    if (cut_fill[k] < kEmptyFill) {
      hs.cell_type[cid] = CELL_EMPTY;
    } else {
      cut_slot[cid] = (int)k;
      kept.push_back(k);
    }
  }
  for (int64_t cid = 0; cid < ncell; ++cid) {
    if (hs.cell_type[cid] == CELL_UNCUT) hs.n_uncut++;
    else if (hs.cell_type[cid] == CELL_CUT) hs.n_cut++;
    else hs.n_empty++;
  }

  // Node classes (Sec. Partitioning).
  hs.node_class.assign(nnode, NODE_INACTIVE);
  std::vector<int> cn(Pd);
  for (int64_t cid = 0; cid < ncell; ++cid) {
    if (hs.cell_type[cid] == CELL_EMPTY) continue;
    g.cell_nodes(cid, cn.data());
    for (int l = 0; l < Pd; ++l) {
      uint8_t& nc = hs.node_class[cn[l]];
      if (hs.cell_type[cid] == CELL_CUT || pb.scheme == kSchemeTrapezoidal) nc = NODE_C;
      else if (nc == NODE_INACTIVE) nc = NODE_D;
    }
  }
  // The matrix-free explicit apply uses the uncut stencil on every cell around
  // an I_d node; check that none of those cells is empty (only a hole boundary
  // passing exactly through a grid vertex could cause that).
  for (int64_t cid = 0; cid < ncell; ++cid) {
    if (hs.cell_type[cid] != CELL_EMPTY) continue;
    g.cell_nodes(cid, cn.data());
    for (int l = 0; l < Pd; ++l)
      if (hs.node_class[cn[l]] == NODE_D)
        return "degenerate geometry: an explicit DOF touches an empty cell";
  }
  std::vector<int> cnodes;
  for (int64_t i = 0; i < nnode; ++i) {
    if (hs.node_class[i] == NODE_D) hs.n_d++;
    if (hs.node_class[i] == NODE_C) cnodes.push_back((int)i);
  }
  hs.n_c = (int64_t)cnodes.size();

  // Time step: dt_factor times the critical step of one free uncut cell,
  // 2 / sqrt(lambda_max(K_e, M_e)), for the largest wave speed among uncut cells.
  {
    double cmax = 0.0;
    for (int64_t cid = 0; cid < ncell; ++cid)
      if (hs.cell_type[cid] == CELL_UNCUT) cmax = std::max(cmax, cell_speed(cid));
    if (cmax <= 0.0) cmax = pb.c0;
    std::vector<double> A((size_t)Pd * Pd);
    for (int a = 0; a < Pd; ++a)
      for (int b = 0; b < Pd; ++b)
        A[a * Pd + b] = hs.uncutK[a + (size_t)Pd * b] * (cmax * cmax) / (pb.c0 * pb.c0) /
                        std::sqrt(uncutM[a] * uncutM[b]);
    double lam = sym_max_eig(A, Pd);
    hs.dt_crit_uncut = 2.0 / std::sqrt(lam);
    double dt_stable = hs.dt_crit_uncut;
    if (scheme_is_cdm(pb.scheme)) {
      // Central differences on the cut cells too: the smallest cell-wise step
      // (the assembled lambda_max is bounded by the largest cell-wise one).
      double lam_c = 0.0;
      for (int64_t k : kept) {
        if (!(cut_lam[k] > 0.0)) return "cut-cell mass matrix is not positive definite";
        lam_c = std::max(lam_c, cut_lam[k]);
      }
      if (lam_c > 0.0) {
        hs.dt_crit_cut_min = 2.0 / std::sqrt(lam_c);
        dt_stable = std::min(dt_stable, hs.dt_crit_cut_min);
      }
    }
    hs.dt = (pb.dt > 0.0) ? pb.dt : pb.dt_factor * dt_stable;
  }

  // Source vector f_x on the full grid: uncut cells by tensor GL, cut cells by spacetree.
  hs.fx.assign((size_t)nnode * ncols, 0.0);
  {
    std::vector<double> fe_uncut((size_t)ncell * Pd * ncols, 0.0);
    std::vector<double> Nt((size_t)Pd * Pd, 0.0), Wt(Pd, 0.0);
    std::vector<double> Xr((size_t)Pd * 3, 0.0);
    for (int q = 0; q < Pd; ++q) {
      int r = q;
      double w = 1.0;
      for (int d = 0; d < dim; ++d) { Xr[q * 3 + d] = gx[r % P]; w *= gw[r % P]; r /= P; }
      Wt[q] = w;
      std::vector<double> G(3 * Pd);
      tensor_basis(g, L1, &Xr[q * 3], &Nt[(size_t)q * Pd], G.data());
    }
    parallel_for(ncell, [&](int64_t b, int64_t e) {
      for (int64_t cid = b; cid < e; ++cid) {
        if (hs.cell_type[cid] != CELL_UNCUT) continue;
        int ci[3] = {0, 0, 0};
        g.cell_coords(cid, ci);
        for (int q = 0; q < Pd; ++q) {
          double xp[3];
          for (int d = 0; d < dim; ++d) xp[d] = g.lo[d] + ci[d] * g.h[d] + (Xr[q * 3 + d] + 1.0) * 0.5 * g.h[d];
          for (int col = 0; col < ncols; ++col) {
            double fv = source_value(pb, xp, col) * Wt[q] * jac;
            double* fe = fe_uncut.data() + ((size_t)cid * ncols + col) * Pd;
            for (int a = 0; a < Pd; ++a) fe[a] += fv * Nt[(size_t)q * Pd + a];
          }
        }
      }
    });
    for (int64_t cid = 0; cid < ncell; ++cid) {
      if (hs.cell_type[cid] == CELL_EMPTY) continue;
      g.cell_nodes(cid, cn.data());
      for (int col = 0; col < ncols; ++col) {
        const double* fe = (hs.cell_type[cid] == CELL_CUT)
                               ? cutF_all.data() + ((size_t)cut_slot[cid] * ncols + col) * Pd
                               : fe_uncut.data() + ((size_t)cid * ncols + col) * Pd;
        for (int l = 0; l < Pd; ++l) hs.fx[(size_t)col * nnode + cn[l]] += fe[l];
      }
    }
  }

  // ---------------------------------------------------------------- ordering
  // Nested dissection of the implicit DOFs on the node lattice.
  std::vector<int> stamp(nnode, 0);
  int stamp_id = 0;
  std::vector<int> tree_of_node(nnode, -1);
  auto cells_of_node = [&](int node, std::vector<int64_t>& out) {
    out.clear();
    int ni[3] = {0, 0, 0};
    g.node_coords(node, ni);
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) { lo[d] = 0; hi[d] = 0; }
    for (int d = 0; d < dim; ++d) {
      int c = ni[d] / g.p;
      if (ni[d] % g.p == 0) { lo[d] = c - 1; hi[d] = c; } else { lo[d] = c; hi[d] = c; }
      lo[d] = std::max(lo[d], 0);
      hi[d] = std::min(hi[d], g.nc[d] - 1);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          int ci[3] = {x, y, z};
          int64_t cid = g.cell_id(ci);
          if (hs.cell_type[cid] != CELL_EMPTY) out.push_back(cid);
        }
  };
  // Connected pieces of a node set (adjacency: sharing a non-empty cell).
  auto pieces = [&](const std::vector<int>& verts) {
    std::vector<std::vector<int>> out;
    ++stamp_id;
    const int in_set = stamp_id;
    for (int v : verts) stamp[v] = in_set;
    ++stamp_id;
    const int seen = stamp_id;
    std::vector<int64_t> cells;
    std::vector<int> nodes(Pd), queue;
    for (int v0 : verts) {
      if (stamp[v0] != in_set) continue;
      std::vector<int> comp;
      queue.assign(1, v0);
      stamp[v0] = seen;
      while (!queue.empty()) {
        int v = queue.back();
        queue.pop_back();
        comp.push_back(v);
        cells_of_node(v, cells);
        for (int64_t cid : cells) {
          g.cell_nodes(cid, nodes.data());
          for (int w : nodes)
            if (stamp[w] == in_set) { stamp[w] = seen; queue.push_back(w); }
        }
      }
      std::sort(comp.begin(), comp.end());
      out.push_back(std::move(comp));
    }
    return out;
  };
  hs.tree.clear();
  std::vector<std::vector<int>> children;
  int next_c = 0;
  hs.c_node.assign(hs.n_c, -1);
  hs.node_c.assign(nnode, -1);
  auto new_node = [&](const std::vector<int>& verts, int comp) {
    TreeNode t;
    t.beg = next_c;
    for (int v : verts) { hs.c_node[next_c] = v; hs.node_c[v] = next_c; ++next_c; }
    t.end = next_c;
    t.comp = comp;
    hs.tree.push_back(t);
    children.emplace_back();
    return (int)hs.tree.size() - 1;
  };
  std::function<std::vector<int>(const std::vector<int>&, int)> dissect =
      [&](const std::vector<int>& verts, int comp) -> std::vector<int> {
    std::vector<int> roots;
    for (auto& piece : pieces(verts)) {
      int best_ax = -1, best_line = 0;
      if ((int)piece.size() > kLeafSize) {
        // Axes by decreasing extent; separator plane through cell vertices nearest the median.
        int mn[3], mx[3];
        for (int d = 0; d < 3; ++d) { mn[d] = 1 << 30; mx[d] = -1; }
        std::vector<std::vector<int>> coords(dim);
        for (int v : piece) {
          int ni[3] = {0, 0, 0};
          g.node_coords(v, ni);
          for (int d = 0; d < dim; ++d) {
            mn[d] = std::min(mn[d], ni[d]);
            mx[d] = std::max(mx[d], ni[d]);
            coords[d].push_back(ni[d]);
          }
        }
        // Axes by decreasing extent; equal extents keep the axis order (a
        // stable insertion sort of at most three entries).
        int order[3] = {0, 1, 2};
        for (int a = 1; a < dim; ++a)
          for (int q = a; q > 0 && (mx[order[q]] - mn[order[q]]) > (mx[order[q - 1]] - mn[order[q - 1]]); --q)
            std::swap(order[q], order[q - 1]);
        for (int oi = 0; oi < dim && best_ax < 0; ++oi) {
          int ax = order[oi];
          std::vector<int>& cs = coords[ax];
          std::nth_element(cs.begin(), cs.begin() + cs.size() / 2, cs.end());
          double med = cs[cs.size() / 2];
          int bestd = 1 << 30;
          for (int line = ((mn[ax] / g.p) + 1) * g.p; line < mx[ax]; line += g.p) {
            int dd = (int)std::fabs(line - med);
            if (dd < bestd) { bestd = dd; best_line = line; best_ax = ax; }
          }
        }
      }
      if (best_ax < 0) {
        roots.push_back(new_node(piece, comp));
        continue;
      }
      std::vector<int> sep, left, right;
      for (int v : piece) {
        int ni[3] = {0, 0, 0};
        g.node_coords(v, ni);
        if (ni[best_ax] < best_line) left.push_back(v);
        else if (ni[best_ax] > best_line) right.push_back(v);
        else sep.push_back(v);
      }
      std::vector<int> kids;
      if (!left.empty()) { auto r = dissect(left, comp); kids.insert(kids.end(), r.begin(), r.end()); }
      if (!right.empty()) { auto r = dissect(right, comp); kids.insert(kids.end(), r.begin(), r.end()); }
      int id = new_node(sep, comp);
      for (int k : kids) { hs.tree[k].parent = id; children[id].push_back(k); }
      roots.push_back(id);
    }
    return roots;
  };
  if (pb.factorize) {
    auto comps = pieces(cnodes);
    hs.ncomp = (int)comps.size();
    hs.comp_tree_ptr.assign(1, 0);
    for (int k = 0; k < hs.ncomp; ++k) {
      hs.max_comp = std::max(hs.max_comp, (int)comps[k].size());
      dissect(comps[k], k);
      hs.comp_tree_ptr.push_back((int)hs.tree.size());
    }
  } else {
    // Iterative solve only: the implicit DOFs in grid order, no tree.
    auto comps = pieces(cnodes);
    hs.ncomp = (int)comps.size();
    for (auto& cp : comps) hs.max_comp = std::max(hs.max_comp, (int)cp.size());
    hs.comp_tree_ptr.assign(1, 0);
    for (int v : cnodes) {
      hs.c_node[next_c] = v;
      hs.node_c[v] = next_c++;
    }
  }
  if (next_c != hs.n_c) return "internal error: nested dissection lost DOFs";
  // Levels: leaves 0, parent above all children.
  for (size_t k = 0; k < hs.tree.size(); ++k) {
    int lv = 0;
    for (int c : children[k]) lv = std::max(lv, hs.tree[c].level + 1);
    hs.tree[k].level = lv;
  }

  // ---------------------------------------------------------------- interface cells
  // Every non-empty cell with a c-node contributes to K^c u (Eq. Kc).
  std::vector<int> if_of_cell(ncell, -1);
  for (int64_t cid = 0; cid < ncell; ++cid) {
    if (hs.cell_type[cid] == CELL_EMPTY) continue;
    g.cell_nodes(cid, cn.data());
    bool has_c = false;
    for (int l = 0; l < Pd; ++l) has_c |= (hs.node_class[cn[l]] == NODE_C);
    if (!has_c) continue;
    if_of_cell[cid] = (int)hs.if_cell.size();
    hs.if_cell.push_back((int)cid);
    double c = cell_speed(cid);
    hs.if_c2.push_back((c * c) / (pb.c0 * pb.c0));
    hs.if_kidx.push_back(hs.cell_type[cid] == CELL_CUT ? -2 : -1);
  }
  // Element matrices of the requested cells, as the assembly uses them.
  hs.export_K.assign(pb.export_cells.size() * Pd * Pd, 0.0);
  hs.export_M.assign(pb.export_cells.size() * Pd * Pd, 0.0);
  for (size_t q = 0; q < pb.export_cells.size(); ++q) {
    const int64_t cid = pb.export_cells[q];
    if (cid < 0 || cid >= ncell) return "export cell out of range";
    double* K = hs.export_K.data() + q * Pd * Pd;
    double* M = hs.export_M.data() + q * Pd * Pd;
    if (hs.cell_type[cid] == CELL_CUT) {
      std::copy(cutK_all.begin() + (size_t)cut_slot[cid] * Pd * Pd,
                cutK_all.begin() + (size_t)(cut_slot[cid] + 1) * Pd * Pd, K);
      std::copy(cutM_all.begin() + (size_t)cut_slot[cid] * Pd * Pd,
                cutM_all.begin() + (size_t)(cut_slot[cid] + 1) * Pd * Pd, M);
    } else if (hs.cell_type[cid] == CELL_UNCUT) {
      const double c = cell_speed(cid), s = (c * c) / (pb.c0 * pb.c0);
      for (size_t k = 0; k < (size_t)Pd * Pd; ++k) K[k] = s * hs.uncutK[k];
      for (int a = 0; a < Pd; ++a) M[a + (size_t)Pd * a] = uncutM[a];
    }
  }
  // Pack cut-cell stiffness in interface order.
  hs.cutK.clear();
  {
    int nk = 0;
    for (size_t e = 0; e < hs.if_cell.size(); ++e) {
      if (hs.if_kidx[e] != -2) continue;
      int slot = cut_slot[hs.if_cell[e]];
      hs.cutK.insert(hs.cutK.end(), cutK_all.begin() + (size_t)slot * Pd * Pd,
                     cutK_all.begin() + (size_t)(slot + 1) * Pd * Pd);
      hs.if_kidx[e] = nk++;
    }
  }
  // Contribution lists per c-index, in (interface cell, local) order.
  {
    std::vector<std::vector<int>> lists(hs.n_c);
    for (size_t e = 0; e < hs.if_cell.size(); ++e) {
      g.cell_nodes(hs.if_cell[e], cn.data());
      for (int l = 0; l < Pd; ++l) {
        int ci = hs.node_c[cn[l]];
        if (ci >= 0) lists[ci].push_back((int)e * Pd + l);
      }
    }
    hs.contrib_ptr.assign(1, 0);
    for (auto& L : lists) {
      hs.contrib_pos.insert(hs.contrib_pos.end(), L.begin(), L.end());
      hs.contrib_ptr.push_back((int)hs.contrib_pos.size());
    }
  }

  // ---------------------------------------------------------------- implicit matrices
  CsrMat Smat, Mmat;
  if (!pb.factorize) {
    // Row by row (threads over rows): row r of S = M^cc + beta dt^2 K^cc and
    // of M^cc from its (interface cell, local node) contributions, entries of
    // equal column summed in contribution order.
    const int nc = (int)hs.n_c;
    const double bdt2 = kBeta * hs.dt * hs.dt;
    const int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>(nc, 4096));
    std::vector<std::vector<int>> ccol(nchunk), ccnt(nchunk);
    std::vector<std::vector<double>> cs(nchunk), cm(nchunk);
    parallel_for(nchunk, [&](int64_t b0, int64_t e0) {
      std::vector<int> cn2(Pd);
      std::vector<std::pair<int, std::pair<double, double>>> ent;
      for (int64_t ch = b0; ch < e0; ++ch) {
        const int64_t r0 = ch * nc / nchunk, r1 = (ch + 1) * nc / nchunk;
        for (int64_t r = r0; r < r1; ++r) {
          ent.clear();
          for (int q = hs.contrib_ptr[r]; q < hs.contrib_ptr[r + 1]; ++q) {
            const int e = hs.contrib_pos[q] / Pd, la = hs.contrib_pos[q] % Pd;
            const int64_t cid = hs.if_cell[e];
            g.cell_nodes(cid, cn2.data());
            const bool is_cut = hs.cell_type[cid] == CELL_CUT;
            const double* Ke = is_cut ? hs.cutK.data() + (size_t)hs.if_kidx[e] * Pd * Pd : hs.uncutK.data();
            const double ks = is_cut ? 1.0 : hs.if_c2[e];
            const double* Me = is_cut ? cutM_all.data() + (size_t)cut_slot[cid] * Pd * Pd : nullptr;
            for (int lb = 0; lb < Pd; ++lb) {
              const int j = hs.node_c[cn2[lb]];
              if (j < 0) continue;
              const double kv = ks * Ke[la + (size_t)Pd * lb];
              const double mv = is_cut ? Me[la + (size_t)Pd * lb] : (la == lb ? uncutM[la] : 0.0);
              ent.push_back({j, {mv + bdt2 * kv, mv}});
            }
          }
          std::stable_sort(ent.begin(), ent.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
          int cnt = 0;
          for (size_t k = 0; k < ent.size();) {
            const int j = ent[k].first;
            double sv = 0.0, mv = 0.0;
            while (k < ent.size() && ent[k].first == j) {
              sv += ent[k].second.first;
              mv += ent[k].second.second;
              ++k;
            }
            ccol[ch].push_back(j);
            cs[ch].push_back(sv);
            cm[ch].push_back(mv);
            ++cnt;
          }
          ccnt[ch].push_back(cnt);
        }
      }
    });
    hs.S_ptr.assign(1, 0);
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      for (int k : ccnt[ch]) hs.S_ptr.push_back(hs.S_ptr.back() + k);
      hs.S_col.insert(hs.S_col.end(), ccol[ch].begin(), ccol[ch].end());
      hs.S_val.insert(hs.S_val.end(), cs[ch].begin(), cs[ch].end());
      hs.M_val.insert(hs.M_val.end(), cm[ch].begin(), cm[ch].end());
      std::vector<int>().swap(ccol[ch]);
      std::vector<double>().swap(cs[ch]);
      std::vector<double>().swap(cm[ch]);
    }
    if ((int64_t)hs.S_ptr.size() != nc + 1) return "internal error: row assembly lost rows";
  } else {
    const int nc = (int)hs.n_c;
    std::vector<std::pair<int64_t, double>> es, em;
    const double bdt2 = kBeta * hs.dt * hs.dt;
    std::vector<int> cl(Pd), cidx(Pd);
    for (size_t e = 0; e < hs.if_cell.size(); ++e) {
      int64_t cid = hs.if_cell[e];
      g.cell_nodes(cid, cn.data());
      int nl = 0;
      for (int l = 0; l < Pd; ++l)
        if (hs.node_c[cn[l]] >= 0) { cl[nl] = l; cidx[nl] = hs.node_c[cn[l]]; ++nl; }
      const bool is_cut = hs.cell_type[cid] == CELL_CUT;
      const double* Ke = is_cut ? hs.cutK.data() + (size_t)hs.if_kidx[e] * Pd * Pd : hs.uncutK.data();
      const double ks = is_cut ? 1.0 : hs.if_c2[e];
      const double* Me = is_cut ? cutM_all.data() + (size_t)cut_slot[cid] * Pd * Pd : nullptr;
      for (int a = 0; a < nl; ++a)
        for (int b = 0; b < nl; ++b) {
          double kv = ks * Ke[cl[a] + (size_t)Pd * cl[b]];
          double mv = is_cut ? Me[cl[a] + (size_t)Pd * cl[b]] : (a == b ? uncutM[cl[a]] : 0.0);
          int64_t key = (int64_t)cidx[a] * nc + cidx[b];
          es.emplace_back(key, mv + bdt2 * kv);
          if (mv != 0.0) em.emplace_back(key, mv);
        }
    }
    // The two conversions are independent: one thread each.
    FirstError err;
    std::thread tmm([&] { err.run([&] { Mmat = coo_to_csr(nc, em); }); });
    err.run([&] { Smat = coo_to_csr(nc, es); });
    tmm.join();
    err.rethrow();
    hs.S_ptr = Smat.ptr;
    hs.S_col = Smat.col;
    hs.S_val = Smat.val;
    // M^cc on the pattern of S (a subset of it).
    hs.M_val.assign(hs.S_val.size(), 0.0);
    for (int i = 0; i < nc; ++i) {
      int q = Mmat.ptr[i];
      for (int k = Smat.ptr[i]; k < Smat.ptr[i + 1] && q < Mmat.ptr[i + 1]; ++k)
        if (Smat.col[k] == Mmat.col[q]) hs.M_val[k] = Mmat.val[q++];
    }
  }
  if (!pb.factorize) {
    hs.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return "";
  }

  // ---------------------------------------------------------------- symbolic
  {
    std::vector<int> mark(hs.n_c, -1);
    int64_t off = 0, offr = 0, offu = 0;
    for (size_t k = 0; k < hs.tree.size(); ++k) {
      TreeNode& t = hs.tree[k];
      std::vector<int> rows;
      for (int j = t.beg; j < t.end; ++j)
        for (int q = Smat.ptr[j]; q < Smat.ptr[j + 1]; ++q) {
          int i = Smat.col[q];
          if (i >= t.end && mark[i] != (int)k) { mark[i] = (int)k; rows.push_back(i); }
        }
      for (int c : children[k])
        for (int i : hs.tree[c].rows)
          if (i >= t.end && mark[i] != (int)k) { mark[i] = (int)k; rows.push_back(i); }
      std::sort(rows.begin(), rows.end());
      t.rows = std::move(rows);
      const int b = t.end - t.beg, m = (int)t.rows.size();
      t.off_diag = off;
      t.off_diagT = off + (int64_t)b * b;
      t.off_rect = off + 2LL * b * b;
      t.off_rectT = off + 2LL * b * b + (int64_t)m * b;
      off += 2LL * b * b + 2LL * m * b;
      t.off_rows = offr;
      offr += m;
      t.off_upd = offu;
      offu += m;
      hs.max_block = std::max(hs.max_block, b);
      hs.max_rows = std::max(hs.max_rows, m);
      hs.nnz_L += (int64_t)b * (b + 1) / 2 + (int64_t)m * b;
      hs.rows_idx.insert(hs.rows_idx.end(), t.rows.begin(), t.rows.end());
    }
    hs.upd_size = offu;
    // Forward-gather lists: scratch positions of descendant updates per row.
    std::vector<std::vector<int>> fl(hs.n_c);
    for (size_t k = 0; k < hs.tree.size(); ++k) {
      const TreeNode& t = hs.tree[k];
      for (size_t i = 0; i < t.rows.size(); ++i) fl[t.rows[i]].push_back((int)(t.off_upd + i));
    }
    hs.fwd_ptr.assign(1, 0);
    for (auto& L : fl) {
      std::sort(L.begin(), L.end());
      hs.fwd_pos.insert(hs.fwd_pos.end(), L.begin(), L.end());
      hs.fwd_ptr.push_back((int)hs.fwd_pos.size());
    }
    // Level lists per component.
    hs.comp_level_base.clear();
    hs.comp_level_ptr.clear();
    hs.level_nodes.clear();
    for (int k = 0; k < hs.ncomp; ++k) {
      int tb = hs.comp_tree_ptr[k], te = hs.comp_tree_ptr[k + 1];
      int nl = 0;
      for (int t = tb; t < te; ++t) nl = std::max(nl, hs.tree[t].level + 1);
      hs.comp_level_base.push_back((int)hs.comp_level_ptr.size());
      std::vector<std::vector<int>> byl(nl);
      for (int t = tb; t < te; ++t) byl[hs.tree[t].level].push_back(t);
      hs.comp_level_ptr.push_back((int)hs.level_nodes.size());
      for (int l = 0; l < nl; ++l) {
        hs.level_nodes.insert(hs.level_nodes.end(), byl[l].begin(), byl[l].end());
        hs.comp_level_ptr.push_back((int)hs.level_nodes.size());
      }
    }
    hs.comp_level_base.push_back((int)hs.comp_level_ptr.size());
  }

  // ---------------------------------------------------------------- numeric
  {
    // The factors of S and M^cc are independent: one thread each.
    std::string err, errM;
    FirstError thrown;
    std::thread tm([&] { thrown.run([&] { errM = factorize(Mmat, hs, hs.Mcc); }); });
    thrown.run([&] { err = factorize(Smat, hs, hs.S); });
    tm.join();
    thrown.rethrow();
    if (!err.empty()) return err;
    if (!errM.empty()) return "M^cc: " + errM;
    try {
      hs.residual_S = factor_residual(hs, Smat, hs.S);
      hs.residual_M = factor_residual(hs, Mmat, hs.Mcc);
    } catch (const std::exception& ex) {
      return std::string("factor check: index out of range (") + ex.what() + ")";
    }
    if (!(hs.residual_S < 1e-8) || !(hs.residual_M < 1e-8))
      return "factor check: solve residual too large";
  }
  hs.setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return "";
}

}  // namespace imex
