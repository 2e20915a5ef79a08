// multigrid.cu -- inner solver for the compact approximate Jacobian.
//
// The preconditioner of the Newton-Krylov solver is the compact-stencil
// approximate Jacobian P (Sec. 4.1): on every displacement component the
// same scalar operator B = D - O, a graph Laplacian of the cell adjacency
// with face weights Gamma_f / |d . n| and the displacement faces on the
// diagonal.  The paper leaves the solution of P z = v to its linear-algebra
// library.  Here it is approximated by one symmetric V-cycle of
// smoothed-aggregation algebraic multigrid in FP32 (inner_iters = 1), or by
// FP32 conjugate gradients preconditioned by that V-cycle (inner_iters > 1):
//
//   * aggregation (three greedy passes over the strong connections),
//     tentative piecewise-constant prolongator, smoothed by one damped
//     Jacobi step, P = (I - omega D^-1 B) P_tent, omega = 4 / (3 rho) with
//     rho the Gershgorin bound of D^-1 B;
//   * Galerkin coarse operators B_c = P^T B P, down to a few hundred cells,
//     where the operator is inverted densely;
//   * one damped Jacobi sweep before and after the coarse correction (same
//     weights, so the V-cycle is a symmetric operator and CG may use it).
//
// The hierarchy is built on first use on the host from B (stored with
// Kbar = 1, so it depends on the geometry only, plus the mass diagonal when
// the inertia term is on; it is rebuilt when that changes) and lives on the
// device in CSR form: one thread per row for short rows, one warp per row
// for long ones.  Every kernel handles all displacement components at once, so the
// matrices are read once per application.  Reductions are
// deterministic (fixed-order partial sums, last-block finalisation).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "hofv_internal.cuh"
#include "reduce.cuh"

namespace hofv {

namespace {

constexpr int kThreads = 256;
constexpr int64_t kCoarsest = 600;   // stop coarsening at or below this many cells
constexpr int64_t kDenseMax = 1500;  // largest coarsest level inverted densely; a larger
                                     // one (coarsening stalled) gets Jacobi sweeps
constexpr int kCoarseSweeps = 8;
constexpr int64_t kWarpRowNnz = 12;  // mean entries per row above which one warp takes a row
constexpr int kRedBlocks = 304;      // blocks of the CG reductions (2 per SM)
constexpr int kMaxLevels = 16;
constexpr double kTheta0 = 0.08;     // strength threshold on the finest level
constexpr double kThetaC = 0.02;     // on coarser levels, whose stencils spread each
                                     // weight over ~9 (2-D) or ~27 (3-D) neighbours

// ------------------------------------------------------------------ host
struct HostCsr {
  int64_t n = 0;
  std::vector<int64_t> rp;   // [n + 1]
  std::vector<int32_t> ci;   // off-diagonal columns
  std::vector<double> va;    // off-diagonal values
  std::vector<double> dg;    // diagonal
};

// strong(i, k): |b_ij| >= theta sqrt(b_ii b_jj)
inline bool strong(const HostCsr& A, double theta, int64_t i, int64_t k) {
  const double v = A.va[k];
  const int32_t j = A.ci[k];
  return v != 0.0 && fabs(v) >= theta * sqrt(fabs(A.dg[i] * A.dg[j]));
}

// Greedy aggregation: (1) a cell whose strong neighbours are all free roots
// a new aggregate with them; (2) a free cell joins the aggregate of its
// strongest already aggregated neighbour; (3) the cells left form
// aggregates with their free strong neighbours.
int64_t aggregate(const HostCsr& A, double theta, std::vector<int32_t>& agg) {
  const int64_t n = A.n;
  agg.assign(n, -1);
  int64_t na = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool ok = true, any = false;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      if (!strong(A, theta, i, k)) continue;
      any = true;
      if (agg[A.ci[k]] >= 0) {
        ok = false;
        break;
      }
    }
    if (!ok || !any) continue;
    agg[i] = (int32_t)na;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (strong(A, theta, i, k)) agg[A.ci[k]] = (int32_t)na;
    ++na;
  }
  const std::vector<int32_t> first = agg;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    double best = -1.0;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      if (strong(A, theta, i, k) && first[j] >= 0 && fabs(A.va[k]) > best) {
        best = fabs(A.va[k]);
        agg[i] = first[j];
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = (int32_t)na;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (strong(A, theta, i, k) && agg[A.ci[k]] < 0) agg[A.ci[k]] = (int32_t)na;
    ++na;
  }
  return na;
}

// Sparse rows with a dense marker over the columns (Gustavson).
struct RowAcc {
  std::vector<int64_t> pos;
  std::vector<int32_t> cols;
  std::vector<double> vals;
  explicit RowAcc(int64_t ncol) : pos(ncol, -1) {}
  void add(int32_t c, double v) {
    if (pos[c] < 0) {
      pos[c] = (int64_t)cols.size();
      cols.push_back(c);
      vals.push_back(v);
    } else {
      vals[pos[c]] += v;
    }
  }
  template <typename F>
  void flush(F&& emit) {
    std::vector<int> order(cols.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cols[a] < cols[b]; });
    for (int k : order) emit(cols[k], vals[k]);
    for (int32_t c : cols) pos[c] = -1;
    cols.clear();
    vals.clear();
  }
};

struct HostMat {  // general CSR (all entries)
  int64_t nr = 0, nc = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va;
};

// P = (I - omega D^-1 B) P_tent
HostMat smoothed_prolongator(const HostCsr& A, const std::vector<int32_t>& agg, int64_t na) {
  double rho = 0.0;
  for (int64_t i = 0; i < A.n; ++i) {
    double s = fabs(A.dg[i]);
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += fabs(A.va[k]);
    rho = std::max(rho, s / A.dg[i]);
  }
  const double omega = 4.0 / (3.0 * rho);
  HostMat P;
  P.nr = A.n;
  P.nc = na;
  P.rp.assign(A.n + 1, 0);
  RowAcc acc(na);
  for (int64_t i = 0; i < A.n; ++i) {
    const double w = omega / A.dg[i];
    acc.add(agg[i], 1.0 - omega);
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) acc.add(agg[A.ci[k]], -w * A.va[k]);
    acc.flush([&](int32_t c, double v) {
      if (v != 0.0) {
        P.ci.push_back(c);
        P.va.push_back(v);
      }
    });
    P.rp[i + 1] = (int64_t)P.ci.size();
  }
  return P;
}

HostMat transpose(const HostMat& M) {
  HostMat T;
  T.nr = M.nc;
  T.nc = M.nr;
  T.rp.assign(M.nc + 1, 0);
  for (int32_t c : M.ci) T.rp[c + 1]++;
  for (int64_t r = 0; r < M.nc; ++r) T.rp[r + 1] += T.rp[r];
  T.ci.resize(M.ci.size());
  T.va.resize(M.va.size());
  std::vector<int64_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int64_t r = 0; r < M.nr; ++r)
    for (int64_t k = M.rp[r]; k < M.rp[r + 1]; ++k) {
      const int64_t d = fill[M.ci[k]]++;
      T.ci[d] = (int32_t)r;
      T.va[d] = M.va[k];
    }
  return T;
}

// B_c = P^T B P, returned with its diagonal split off
HostCsr galerkin(const HostCsr& A, const HostMat& P, const HostMat& R) {
  // BP = B P
  HostMat BP;
  BP.nr = A.n;
  BP.nc = P.nc;
  BP.rp.assign(A.n + 1, 0);
  RowAcc acc(P.nc);
  for (int64_t i = 0; i < A.n; ++i) {
    for (int64_t q = P.rp[i]; q < P.rp[i + 1]; ++q) acc.add(P.ci[q], A.dg[i] * P.va[q]);
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      for (int64_t q = P.rp[j]; q < P.rp[j + 1]; ++q) acc.add(P.ci[q], A.va[k] * P.va[q]);
    }
    acc.flush([&](int32_t c, double v) {
      BP.ci.push_back(c);
      BP.va.push_back(v);
    });
    BP.rp[i + 1] = (int64_t)BP.ci.size();
  }
  HostCsr C;
  C.n = P.nc;
  C.rp.assign(C.n + 1, 0);
  C.dg.assign(C.n, 0.0);
  for (int64_t I = 0; I < C.n; ++I) {
    for (int64_t q = R.rp[I]; q < R.rp[I + 1]; ++q) {
      const int32_t i = R.ci[q];
      const double p = R.va[q];
      for (int64_t k = BP.rp[i]; k < BP.rp[i + 1]; ++k) acc.add(BP.ci[k], p * BP.va[k]);
    }
    acc.flush([&](int32_t c, double v) {
      if (c == I) {
        C.dg[I] = v;
      } else if (v != 0.0) {
        C.ci.push_back(c);
        C.va.push_back(v);
      }
    });
    C.rp[I + 1] = (int64_t)C.ci.size();
  }
  return C;
}

// Inverse of the (small, SPD) coarsest operator by Cholesky, row-major.
bool dense_inverse(const HostCsr& A, std::vector<float>& inv) {
  const int64_t m = A.n;
  std::vector<double> L(m * m, 0.0), Ad(m * m, 0.0);
  double dmax = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    Ad[i * m + i] = A.dg[i];
    dmax = std::max(dmax, fabs(A.dg[i]));
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) Ad[i * m + A.ci[k]] = A.va[k];
  }
  double shift = 0.0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    bool ok = true;
    for (int64_t j = 0; j < m && ok; ++j) {
      double s = Ad[j * m + j] + shift;
      for (int64_t k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
      if (!(s > 1e-14 * dmax)) {
        ok = false;
        break;
      }
      const double ljj = sqrt(s);
      L[j * m + j] = ljj;
      for (int64_t i = j + 1; i < m; ++i) {
        double t = Ad[i * m + j];
        for (int64_t k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
        L[i * m + j] = t / ljj;
      }
    }
    if (ok) break;
    if (attempt == 3) return false;
    shift = shift == 0.0 ? 1e-10 * dmax : shift * 100.0;  // singular (no Dirichlet face)
    std::fill(L.begin(), L.end(), 0.0);
  }
  inv.assign(m * m, 0.0f);
  std::vector<double> y(m);
  for (int64_t c = 0; c < m; ++c) {  // column c of the inverse
    for (int64_t i = 0; i < m; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int64_t k = 0; k < i; ++k) s -= L[i * m + k] * y[k];
      y[i] = s / L[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t k = i + 1; k < m; ++k) s -= L[k * m + i] * y[k];
      y[i] = s / L[i * m + i];
    }
    for (int64_t i = 0; i < m; ++i) inv[i * m + c] = (float)y[i];
  }
  return true;
}

// ---------------------------------------------------------------- device
struct Level {
  int64_t n = 0;
  int32_t *rp = nullptr, *ci = nullptr;  // off-diagonal part of B, CSR (int32 offsets)
  float *va = nullptr, *dg = nullptr, *dinv = nullptr;
  // prolongation from the next level (rows: this level) and its transpose
  int32_t *prp = nullptr, *pci = nullptr, *rrp = nullptr, *rci = nullptr;
  float *pva = nullptr, *rva = nullptr;
  int64_t nnz = 0, pnnz = 0, rnnz = 0;
  // long rows (coarse operators, restrictions) go one warp per row, so that
  // levels with few rows still spread over the whole GPU
  bool a_warp = false, p_warp = false, r_warp = false;
  float *x = nullptr, *r = nullptr, *b = nullptr, *y = nullptr;  // [dim][n] work
};

struct Mg {
  std::vector<Level> L;
  int64_t m = 0;              // coarsest size
  float* inv = nullptr;       // [m][m]
  // CG vectors on level 0, [dim][n0] each
  float *x = nullptr, *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
  double* part = nullptr;     // [2 dim][blocks]
  unsigned int* cnt = nullptr;
  double* sc = nullptr;       // gamma[dim], alpha[dim], beta[dim]
  int blocks = 0;
  double setup_s = 0.0;
  int64_t nnz_total = 0;
  std::vector<void*> mem;     // device allocations of the hierarchy
};

Mg* get(hofv_ctx* c) { return static_cast<Mg*>(c->mg); }

#define MG_TRY(x)              \
  do {                         \
    const int rc_ = (x);       \
    if (rc_ != 0) return rc_;  \
  } while (0)

template <typename T>
int upload(hofv_ctx* c, T** d, const std::vector<T>& h) {
  if (dev_alloc(c, d, std::max<size_t>(h.size(), 1))) return HOFV_ENOMEM;
  if (!h.empty())
    HOFV_CUDA(c, cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return 0;
}

std::vector<int32_t> to32(const std::vector<int64_t>& v) {
  return std::vector<int32_t>(v.begin(), v.end());
}
std::vector<float> tof(const std::vector<double>& v) {
  return std::vector<float>(v.begin(), v.end());
}

unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 8192));
}

// ---- V-cycle kernels (all components per thread, component stride n) ----

// b as stored (float), or as the caller's FP64 right-hand side times a scale
template <typename TB>
__device__ __forceinline__ float ldb(const TB* b, int64_t k, double bs) {
  if constexpr (sizeof(TB) == 8)
    return (float)(b[k] * bs);
  else
    return b[k];
}

// x = W b (W = omega D^-1), r = b - B x
template <int DIM, typename TB = float>
__global__ void k_pre(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                      const float* __restrict__ va, const float* __restrict__ dg,
                      const float* __restrict__ dinv, const TB* __restrict__ b, double bs,
                      float* x, float* r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float wi = dinv[i], di = dg[i];
    float bi[DIM], s[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      bi[j] = ldb(b, j * n + i, bs);
      s[j] = di * wi * bi[j];
    }
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t c = ci[k];
      const float a = va[k] * dinv[c];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s[j] += a * ldb(b, j * n + c, bs);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      x[j * n + i] = wi * bi[j];
      r[j * n + i] = bi[j] - s[j];
    }
  }
}

// out[I] = sum_k M_Ik in[col_k]  (restriction with R = P^T, or prolongation add)
template <int DIM, bool ADD>
__global__ void k_csr_apply(int64_t nrow, int64_t nin, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const float* __restrict__ va,
                            const float* __restrict__ in, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrow;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] = ADD ? out[j * nrow + i] : 0.0f;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t c = ci[k];
      const float a = va[k];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s[j] += a * in[j * nin + c];
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) out[j * nrow + i] = s[j];
  }
}

// y = x + W (b - B x)
template <int DIM, typename TB = float, typename TY = float>
__global__ void k_post(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const float* __restrict__ va, const float* __restrict__ dg,
                       const float* __restrict__ dinv, const TB* __restrict__ b, double bs,
                       const float* __restrict__ x, TY* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float wi = dinv[i], di = dg[i];
    float xi[DIM], s[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      xi[j] = x[j * n + i];
      s[j] = ldb(b, j * n + i, bs) - di * xi[j];
    }
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t c = ci[k];
      const float a = va[k];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s[j] -= a * x[j * n + c];
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) y[j * n + i] = (TY)(xi[j] + wi * s[j]);
  }
}

// y = inv b on the coarsest level, one warp per row
template <int DIM>
__global__ void k_dense(int64_t m, const float* __restrict__ inv, const float* __restrict__ b,
                        float* y) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= m) return;
  float s[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) s[j] = 0.0f;
  for (int64_t k = lane; k < m; k += 32) {
    const float a = inv[row * m + k];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] += a * b[j * m + k];
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    float v = s[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) y[j * m + row] = v;
  }
}

// ---- the same operations with one warp per row ----
template <int DIM>
__device__ __forceinline__ void warp_reduce(float (&s)[DIM]) {
#pragma unroll
  for (int j = 0; j < DIM; ++j)
    for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
}

// x = W b, r = b - B x
template <int DIM>
__global__ void k_pre_w(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const float* __restrict__ va, const float* __restrict__ dg,
                        const float* __restrict__ dinv, const float* __restrict__ b, float* x,
                        float* r) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    float s[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] = 0.0f;
    for (int32_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const int32_t c = ci[k];
      const float a = va[k] * dinv[c];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s[j] += a * b[j * n + c];
    }
    warp_reduce<DIM>(s);
    if (lane == 0) {
      const float wi = dinv[i], di = dg[i];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const float bi = b[j * n + i];
        x[j * n + i] = wi * bi;
        r[j * n + i] = bi - (di * wi * bi + s[j]);
      }
    }
  }
}

// out = M in, or out += M in
template <int DIM, bool ADD>
__global__ void k_csr_apply_w(int64_t nrow, int64_t nin, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, const float* __restrict__ va,
                              const float* __restrict__ in, float* out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nrow; i += nw) {
    float s[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] = 0.0f;
    for (int32_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const int32_t c = ci[k];
      const float a = va[k];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s[j] += a * in[j * nin + c];
    }
    warp_reduce<DIM>(s);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < DIM; ++j) out[j * nrow + i] = ADD ? out[j * nrow + i] + s[j] : s[j];
    }
  }
}

// y = x + W (b - B x)
template <int DIM>
__global__ void k_post_w(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const float* __restrict__ va, const float* __restrict__ dg,
                         const float* __restrict__ dinv, const float* __restrict__ b,
                         const float* __restrict__ x, float* y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    float s[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] = 0.0f;
    for (int32_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const int32_t c = ci[k];
      const float a = va[k];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s[j] += a * x[j * n + c];
    }
    warp_reduce<DIM>(s);
    if (lane == 0) {
      const float wi = dinv[i], di = dg[i];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const float xi = x[j * n + i];
        y[j * n + i] = xi + wi * (b[j * n + i] - di * xi - s[j]);
      }
    }
  }
}

unsigned grid_warps(int64_t rows) {
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((rows * 32 + kThreads - 1) / kThreads, 8192));
}

template <int DIM>
void pre(const Level& L, const float* b, float* x, float* r, cudaStream_t st) {
  if (L.a_warp)
    k_pre_w<DIM><<<grid_warps(L.n), kThreads, 0, st>>>(L.n, L.rp, L.ci, L.va, L.dg, L.dinv, b, x, r);
  else
    k_pre<DIM><<<grid_for(L.n), kThreads, 0, st>>>(L.n, L.rp, L.ci, L.va, L.dg, L.dinv, b, 1.0, x,
                                                   r);
}

template <int DIM>
void post(const Level& L, const float* b, const float* x, float* y, cudaStream_t st) {
  if (L.a_warp)
    k_post_w<DIM><<<grid_warps(L.n), kThreads, 0, st>>>(L.n, L.rp, L.ci, L.va, L.dg, L.dinv, b, x,
                                                        y);
  else
    k_post<DIM><<<grid_for(L.n), kThreads, 0, st>>>(L.n, L.rp, L.ci, L.va, L.dg, L.dinv, b, 1.0, x,
                                                    y);
}

template <int DIM, bool ADD>
void apply(bool warp, int64_t nrow, int64_t nin, const int32_t* rp, const int32_t* ci,
           const float* va, const float* in, float* out, cudaStream_t st) {
  if (warp)
    k_csr_apply_w<DIM, ADD><<<grid_warps(nrow), kThreads, 0, st>>>(nrow, nin, rp, ci, va, in, out);
  else
    k_csr_apply<DIM, ADD><<<grid_for(nrow), kThreads, 0, st>>>(nrow, nin, rp, ci, va, in, out);
}

template <int DIM>
void vcycle(const Mg& g, int l, const float* b, float* out, cudaStream_t st) {
  const Level& L = g.L[l];
  if (l + 1 == (int)g.L.size()) {
    if (g.inv) {
      k_dense<DIM><<<grid_warps(L.n), kThreads, 0, st>>>(L.n, g.inv, b, out);
      return;
    }
    // damped Jacobi sweeps from zero (a symmetric operator)
    pre<DIM>(L, b, L.x, L.r, st);
    float* src = L.x;
    for (int s = 1; s < kCoarseSweeps; ++s) {
      float* dst = s + 1 == kCoarseSweeps ? out : (src == L.x ? L.r : L.x);
      post<DIM>(L, b, src, dst, st);
      src = dst;
    }
    return;
  }
  const Level& C = g.L[l + 1];
  pre<DIM>(L, b, L.x, L.r, st);
  apply<DIM, false>(L.r_warp, C.n, L.n, L.rrp, L.rci, L.rva, L.r, C.b, st);
  vcycle<DIM>(g, l + 1, C.b, C.y, st);
  apply<DIM, true>(L.p_warp, L.n, C.n, L.prp, L.pci, L.pva, C.y, L.x, st);
  post<DIM>(L, b, L.x, out, st);
}

// ---- conjugate-gradient kernels on level 0 ----

// r = -v / Kbar (FP32), x = 0
template <int DIM>
__global__ void k_cg_start(int64_t n, const double* __restrict__ v, double inv_kbar, float* r,
                           float* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < DIM * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = (float)(-v[i] * inv_kbar);
    x[i] = 0.0f;
  }
}

// gamma_j = r_j . z_j; beta_j = gamma_j / gamma_prev_j (0 on the first pass)
template <int DIM>
__global__ void k_cg_rz(int64_t n, const float* __restrict__ r, const float* __restrict__ z,
                        double* part, unsigned int* cnt, double* sc, int first) {
  __shared__ double sh[32];
  float s[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) s[j] = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] += r[j * n + i] * z[j * n + i];
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double t = block_sum_t(s[j], sh);
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = t;
  }
  if (last_block(cnt, gridDim.x)) {
    __threadfence();
    for (int j = 0; j < DIM; ++j) {
      const double gm = warp0_sum(part + j * gridDim.x, gridDim.x);
      if (threadIdx.x == 0) {
        const double gp = sc[j];
        sc[2 * DIM + j] = (first || gp == 0.0) ? 0.0 : gm / gp;
        sc[j] = gm;
      }
    }
    if (threadIdx.x == 0) *cnt = 0;
  }
}

// p_new = z + beta p_old; q = B p_new; alpha_j = gamma_j / (p_new . q)_j
template <int DIM>
__global__ void k_cg_spmv(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const float* __restrict__ va, const float* __restrict__ dg,
                          const float* __restrict__ z, const float* pold, float* pnew,
                          float* q, double* part, unsigned int* cnt, double* sc, int first) {
  __shared__ double sh[32];
  float beta[DIM], s[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    beta[j] = (float)sc[2 * DIM + j];
    s[j] = 0.0f;
  }
  if (first) pold = z;  // p = z: the old direction is never read

  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float di = dg[i];
    float pi[DIM], qi[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      pi[j] = z[j * n + i] + beta[j] * pold[j * n + i];
      qi[j] = di * pi[j];
    }
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t c = ci[k];
      const float a = va[k];
#pragma unroll
      for (int j = 0; j < DIM; ++j) qi[j] += a * (z[j * n + c] + beta[j] * pold[j * n + c]);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      pnew[j * n + i] = pi[j];
      q[j * n + i] = qi[j];
      s[j] += pi[j] * qi[j];
    }
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double t = block_sum_t(s[j], sh);
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = t;
  }
  if (last_block(cnt, gridDim.x)) {
    __threadfence();
    for (int j = 0; j < DIM; ++j) {
      const double pq = warp0_sum(part + j * gridDim.x, gridDim.x);
      if (threadIdx.x == 0) sc[DIM + j] = pq != 0.0 ? sc[j] / pq : 0.0;
    }
    if (threadIdx.x == 0) *cnt = 0;
  }
}

// x += alpha p; r -= alpha q
template <int DIM>
__global__ void k_cg_update(int64_t n, const float* __restrict__ p, const float* __restrict__ q,
                            float* x, float* r, const double* __restrict__ sc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const float a = (float)sc[DIM + j];
      x[j * n + i] += a * p[j * n + i];
      r[j * n + i] -= a * q[j * n + i];
    }
  }
}

// zout = x + alpha p  (FP64 output)
template <int DIM>
__global__ void k_cg_out(int64_t n, const float* __restrict__ p, const float* __restrict__ x,
                         const double* __restrict__ sc, double* zout) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < DIM; ++j)
      zout[j * n + i] = (double)(x[j * n + i] + (float)sc[DIM + j] * p[j * n + i]);
  }
}

// ---------------------------------------------------------------- build
// the finest level stays one thread per row: the CG kernels read it directly
int upload_level(hofv_ctx* c, Level& L, const HostCsr& A, int dim, bool finest) {
  L.n = A.n;
  L.nnz = (int64_t)A.ci.size();
  L.a_warp = !finest && L.nnz > kWarpRowNnz * A.n;
  if (A.ci.size() >= (size_t)INT32_MAX) return fail(c, HOFV_EINVAL, "multigrid level too large");
  double rho = 0.0;
  for (int64_t i = 0; i < A.n; ++i) {
    double s = fabs(A.dg[i]);
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += fabs(A.va[k]);
    rho = std::max(rho, s / A.dg[i]);
  }
  const double omega = 4.0 / (3.0 * rho);
  std::vector<float> dinv(A.n);
  for (int64_t i = 0; i < A.n; ++i) dinv[i] = (float)(omega / A.dg[i]);
  if (upload(c, &L.rp, to32(A.rp)) || upload(c, &L.ci, A.ci) || upload(c, &L.va, tof(A.va)) ||
      upload(c, &L.dg, tof(A.dg)) || upload(c, &L.dinv, dinv))
    return HOFV_ENOMEM;
  const size_t nv = (size_t)dim * A.n;
  if (dev_alloc(c, &L.x, nv) || dev_alloc(c, &L.r, nv) || dev_alloc(c, &L.b, nv) ||
      dev_alloc(c, &L.y, nv))
    return HOFV_ENOMEM;
  return 0;
}

int build_levels(hofv_ctx* c, Mg* g, HostCsr A, int dim, int64_t n);

int build(hofv_ctx* c) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = c->nc;
  const int nlf = c->nlf, dim = c->dim;
  std::vector<double> diag(n), off((size_t)n * nlf);
  std::vector<int32_t> col((size_t)n * nlf);
  HOFV_CUDA(c, cudaMemcpy(diag.data(), c->d_aj_diag, sizeof(double) * n, cudaMemcpyDeviceToHost));
  HOFV_CUDA(c, cudaMemcpy(off.data(), c->d_aj_off, sizeof(double) * n * nlf, cudaMemcpyDeviceToHost));
  HOFV_CUDA(c, cudaMemcpy(col.data(), c->d_aj_col, sizeof(int32_t) * n * nlf,
                          cudaMemcpyDeviceToHost));
  // B = -A1: positive diagonal, non-positive couplings
  HostCsr A;
  A.n = n;
  A.rp.assign(n + 1, 0);
  A.dg.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    A.dg[i] = -diag[i];
    for (int lf = 0; lf < nlf; ++lf) {
      const int32_t j = col[i * nlf + lf];
      if (j < 0) continue;
      A.ci.push_back(j);
      A.va.push_back(-off[i * nlf + lf]);
    }
    A.rp[i + 1] = (int64_t)A.ci.size();
  }
  Mg* g = new Mg();
  const size_t mark = c->allocs.size();
  const int rc = build_levels(c, g, std::move(A), dim, n);
  g->mem.assign(c->allocs.begin() + mark, c->allocs.end());
  if (rc) {
    for (void* p : g->mem) dev_free(c, p);
    delete g;
    return rc;
  }
  g->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->mg = g;
  return 0;
}

int build_levels(hofv_ctx* c, Mg* g, HostCsr A, int dim, int64_t n) {
  g->L.reserve(kMaxLevels);
  for (int l = 0; l < kMaxLevels; ++l) {
    g->L.emplace_back();
    Level& L = g->L.back();
    MG_TRY(upload_level(c, L, A, dim, l == 0));
    g->nnz_total += (int64_t)A.ci.size() + A.n;
    if (A.n <= kCoarsest || l + 1 == kMaxLevels) break;
    std::vector<int32_t> agg;
    const int64_t na = aggregate(A, l == 0 ? kTheta0 : kThetaC, agg);
    if (3 * na > 2 * A.n) break;  // aggregation stalled
    const HostMat P = smoothed_prolongator(A, agg, na);
    const HostMat R = transpose(P);
    HostCsr Ac = galerkin(A, P, R);
    if ((int64_t)Ac.ci.size() > 400 * Ac.n) break;  // coarse operator too dense
    L.pnnz = (int64_t)P.ci.size();
    L.rnnz = (int64_t)R.ci.size();
    L.p_warp = L.pnnz > kWarpRowNnz * P.nr;
    L.r_warp = L.rnnz > kWarpRowNnz * R.nr;
    if (upload(c, &L.prp, to32(P.rp)) || upload(c, &L.pci, P.ci) || upload(c, &L.pva, tof(P.va)) ||
        upload(c, &L.rrp, to32(R.rp)) || upload(c, &L.rci, R.ci) || upload(c, &L.rva, tof(R.va)))
      return HOFV_ENOMEM;
    A = std::move(Ac);
  }
  // the last level uploaded is the coarsest
  g->m = A.n;
  if (A.n <= kDenseMax) {
    std::vector<float> inv;
    if (!dense_inverse(A, inv)) return fail(c, HOFV_EILLCOND, "coarsest multigrid operator is singular");
    MG_TRY(upload(c, &g->inv, inv));
  }
  const size_t nv = (size_t)dim * n;
  // few blocks for the CG reductions: the last block adds one partial per block
  g->blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, kRedBlocks);
  if (dev_alloc(c, &g->x, nv) || dev_alloc(c, &g->r, nv) || dev_alloc(c, &g->z, nv) ||
      dev_alloc(c, &g->p0, nv) || dev_alloc(c, &g->p1, nv) || dev_alloc(c, &g->q, nv) ||
      dev_alloc(c, &g->part, (size_t)2 * dim * g->blocks) || dev_alloc(c, &g->cnt, 4) ||
      dev_alloc(c, &g->sc, 3 * 3))
    return HOFV_ENOMEM;
  HOFV_CUDA(c, cudaMemset(g->cnt, 0, 4 * sizeof(unsigned int)));
  HOFV_CUDA(c, cudaMemset(g->sc, 0, 9 * sizeof(double)));
  return 0;
}

template <int DIM>
void run(hofv_ctx* c, Mg& g, int iters, const double* v, double* zout) {
  cudaStream_t st = c->stream;
  const int64_t n = c->nc;
  const Level& L = g.L[0];
  const unsigned gb = (unsigned)g.blocks;
  if (iters == 1 && g.L.size() > 1) {
    // one V-cycle applied to b = -v / Kbar, read and written in FP64 by the
    // finest level's smoothers (the flexible outer solver absorbs the
    // missing CG step length: it only scales z)
    const Level& C = g.L[1];
    const double bs = -1.0 / c->mat.kbar;
    k_pre<DIM, double><<<grid_for(n), kThreads, 0, st>>>(n, L.rp, L.ci, L.va, L.dg, L.dinv, v, bs,
                                                         L.x, L.r);
    apply<DIM, false>(L.r_warp, C.n, n, L.rrp, L.rci, L.rva, L.r, C.b, st);
    vcycle<DIM>(g, 1, C.b, C.y, st);
    apply<DIM, true>(L.p_warp, n, C.n, L.prp, L.pci, L.pva, C.y, L.x, st);
    k_post<DIM, double, double><<<grid_for(n), kThreads, 0, st>>>(n, L.rp, L.ci, L.va, L.dg,
                                                                  L.dinv, v, bs, L.x, zout);
    return;
  }
  k_cg_start<DIM><<<grid_for(DIM * n), kThreads, 0, st>>>(n, v, 1.0 / c->mat.kbar, g.r, g.x);
  float* p[2] = {g.p0, g.p1};
  for (int it = 0; it < iters; ++it) {
    vcycle<DIM>(g, 0, g.r, g.z, st);
    k_cg_rz<DIM><<<gb, kThreads, 0, st>>>(n, g.r, g.z, g.part, g.cnt, g.sc, it == 0);
    float* pold = p[(it + 1) & 1];
    float* pnew = p[it & 1];
    k_cg_spmv<DIM><<<gb, kThreads, 0, st>>>(n, L.rp, L.ci, L.va, L.dg, g.z, pold, pnew, g.q, g.part,
                                            g.cnt + 1, g.sc, it == 0);
    if (it + 1 == iters) {
      k_cg_out<DIM><<<grid_for(n), kThreads, 0, st>>>(n, pnew, g.x, g.sc, zout);
    } else {
      k_cg_update<DIM><<<grid_for(n), kThreads, 0, st>>>(n, pnew, g.q, g.x, g.r, g.sc);
    }
  }
}

}  // namespace

int mg_ensure(hofv_ctx* c) { return c->mg ? 0 : build(c); }

int mg_precondition(hofv_ctx* c, int iters, const double* v, double* z) {
  if (!c->mg) {
    const int rc = build(c);
    if (rc) return rc;
  }
  Mg& g = *get(c);
  if (iters < 1) iters = 1;
  if (c->dim == 2)
    run<2>(c, g, iters, v, z);
  else
    run<3>(c, g, iters, v, z);
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

int mg_info(hofv_ctx* c, int32_t* levels, int64_t* sizes, int max_sizes, int64_t* nnz,
            double* setup_s) {
  if (!c->mg) {
    const int rc = build(c);
    if (rc) return rc;
  }
  const Mg& g = *get(c);
  *levels = (int32_t)g.L.size();
  for (int l = 0; l < (int)g.L.size() && l < max_sizes; ++l) sizes[l] = g.L[l].n;
  *nnz = g.nnz_total;
  *setup_s = g.setup_s;
  return 0;
}

// device memory of the hierarchy is owned by the context's allocation list
void mg_release(hofv_ctx* c) {
  delete get(c);
  c->mg = nullptr;
}

void mg_drop(hofv_ctx* c) {
  Mg* g = get(c);
  if (!g) return;
  for (void* p : g->mem) dev_free(c, p);
  delete g;
  c->mg = nullptr;
}

}  // namespace hofv
