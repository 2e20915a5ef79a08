// krylov.cu -- vector kernels of the flexible GMRES outer solver and the
// compact-stencil approximate-Jacobian preconditioner (arXiv 2601.18417,
// Sec. 4.1).
//
// Reductions are deterministic: each block writes a partial sum, and the
// last block to finish (an atomic ticket, no waiting) adds the partials in
// block order and publishes the result to device memory, where the next
// kernel on the stream reads it.  No host round trip is needed inside Jv or
// inside the preconditioner.
#include <stdlib.h>

#include "hofv_internal.cuh"
#include "reduce.cuh"

namespace hofv {

constexpr int kRedThreads = 256;

// out[k] = x_k . y for k = blockIdx.y; x_k = X + k * ldx
__global__ void k_mdot(const double* __restrict__ X, int64_t ldx, const double* __restrict__ y,
                       int64_t n, double* red, unsigned int* count, double* out, int mode) {
  __shared__ double sh[32];
  const int k = blockIdx.y;
  const double* x = X + k * ldx;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) red[k * gridDim.x + blockIdx.x] = s;
  if (last_block(count + k, gridDim.x)) {
    __threadfence();
    const double t = warp0_sum(red + k * gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      out[k] = mode == 1 ? sqrt(t) : t;
      count[k] = 0;
    }
  }
}

void launch_dots(const double* X, int64_t ldx, const double* y, int nvec, int64_t n, double* red,
                 unsigned int* count, double* out, int blocks, cudaStream_t st, int mode) {
  // few blocks per vector: every block ends in FP64 warp reductions
  blocks = (int)std::min<int64_t>(std::max(blocks / 4, 1), (n + kRedThreads - 1) / kRedThreads);
  dim3 grid((unsigned)blocks, (unsigned)nvec);
  k_mdot<<<grid, kRedThreads, 0, st>>>(X, ldx, y, n, red, count, out, mode);
}

void launch_norm2(const double* x, int64_t n, double* red, unsigned int* count, double* out,
                  int blocks, cudaStream_t st) {
  launch_dots(x, 0, x, 1, n, red, count, out, blocks, st, 1);
}

// eps = sqrt(2^-52) (1 + ||u||) / ||v||  (0 if v = 0)
__global__ void k_jv_eps(const double* un, const double* vn, double* eps) {
  const double v = vn[0];
  eps[0] = v > 0.0 ? 1.4901161193847656e-08 * (1.0 + un[0]) / v : 1.0;
}
void launch_jv_eps(const double* u_norm, const double* v_norm, double* eps, cudaStream_t st) {
  k_jv_eps<<<1, 1, 0, st>>>(u_norm, v_norm, eps);
}

// y = x + sign * alpha[0] * v   (alpha read on the device)
__global__ void k_axpy_dev(double* __restrict__ y, const double* __restrict__ x,
                           const double* __restrict__ v, const double* alpha, double sign,
                           int64_t n) {
  const double a = sign * alpha[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, v[i], x[i]);
}
void launch_waxpy_dev(double* y, const double* x, const double* v, const double* alpha,
                      double sign, int64_t n, cudaStream_t st) {
  k_axpy_dev<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(y, x, v, alpha,
                                                                              sign, n);
}

// y = x * s[0] (invert: x / s[0])
__global__ void k_scale_copy(double* __restrict__ y, const double* __restrict__ x,
                             const double* s, int invert, int64_t n) {
  const double f = invert ? 1.0 / s[0] : s[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}
void launch_scale_copy(double* y, const double* x, const double* s, int invert, int64_t n,
                       cudaStream_t st) {
  k_scale_copy<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(y, x, s,
                                                                                invert, n);
}

// w -= sum_k coef[k] V_k  (coef on the device)
__global__ void k_multi_axpy(double* __restrict__ w, const double* __restrict__ V,
                             const double* __restrict__ coef, int k, int64_t n, int64_t ld) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int j = 0; j < k; ++j) s = fma(-coef[j], V[j * ld + i], s);
    w[i] = s;
  }
}
void launch_multi_axpy(double* w, const double* V, const double* coef, int k, int64_t n,
                       int64_t ld, cudaStream_t st) {
  k_multi_axpy<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(w, V, coef, k,
                                                                                 n, ld);
}

// x += sum_k y[k] Z_k  (y on the device)
__global__ void k_combine(double* __restrict__ x, const double* __restrict__ Z,
                          const double* __restrict__ y, int k, int64_t n, int64_t ld) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int j = 0; j < k; ++j) s = fma(y[j], Z[j * ld + i], s);
    x[i] = s;
  }
}
void launch_combine(double* x, const double* Z, const double* y, int k, int64_t n, int64_t ld,
                    cudaStream_t st) {
  k_combine<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(x, Z, y, k, n, ld);
}

// y = a x + b y
__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b,
                        int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}
void launch_axpby(double* y, double a, const double* x, double b, int64_t n, cudaStream_t st) {
  k_axpby<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(y, a, x, b, n);
}

// ---------------------------------------------------------------------
// approximate Jacobian A = Kbar * A1 (Sec. 4.1), A1 negative definite with
// Kbar = 1.  z = A^{-1} v solves B z = -v / Kbar with B = -A1 (SPD), by a
// fixed number of Jacobi-preconditioned conjugate-gradient iterations on
// all `dim` right-hand sides at once, in the single-reduction form of
// Chronopoulos & Gear (J. Comput. Appl. Math. 25, 1989): per iteration one
// product w = B u (u = D^{-1} r) and the two inner products (r,u), (w,u),
// with s = B p carried by recurrence.  One kernel per iteration: the vector
// updates of iteration i-1 are recomputed on the fly for the neighbours
// that the product of iteration i reads (r, w and s are double-buffered),
// so no grid-wide synchronisation is needed.  T = float or double.
// Scalars (double): sc[0..d) gamma_prev, sc[d..2d) alpha, sc[2d..3d) beta.
// ---------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ void cg_finalize(const double* red, unsigned int nb, double* sh,
                                            double* sc, bool first) {
  for (int j = 0; j < DIM; ++j) {
    const double gamma = warp0_sum<T>(red + (2 * j) * nb, nb);
    const double delta = warp0_sum<T>(red + (2 * j + 1) * nb, nb);
    if (threadIdx.x == 0) {
      double alpha, beta;
      if (first) {
        beta = 0.0;
        alpha = delta != 0.0 ? gamma / delta : 0.0;
      } else {
        const double gp = sc[j], ap = sc[DIM + j];
        beta = gp != 0.0 ? gamma / gp : 0.0;
        const double den = ap != 0.0 ? delta - beta * gamma / ap : 0.0;
        alpha = den != 0.0 ? gamma / den : 0.0;
      }
      sc[j] = gamma;
      sc[DIM + j] = alpha;
      sc[2 * DIM + j] = beta;
    }
  }
}

// r0 = b = -v/Kbar, w0 = B D^{-1} r0; x = p = 0, s_{-1} = 0; alpha0 = gamma0/delta0
template <typename T, int DIM, int NLF>
__global__ void k_cg_init(int64_t nc, const double* __restrict__ v, double inv_kbar,
                          const T* __restrict__ diag, const T* __restrict__ invd,
                          const int32_t* __restrict__ col,
                          const T* __restrict__ off, T* __restrict__ r0, T* __restrict__ w0,
                          T* __restrict__ sm1, T* __restrict__ x, T* __restrict__ p, double* red,
                          unsigned int* count, double* sc) {
  __shared__ double sh[32];
  T pg[DIM], pd[DIM];  // per-thread partials in the vector precision
#pragma unroll
  for (int j = 0; j < DIM; ++j) pg[j] = pd[j] = (T)0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const T D = -diag[c], iD = invd[c];
    T u[DIM], w[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const T b = (T)(-v[j * nc + c] * inv_kbar);
      r0[j * nc + c] = b;
      u[j] = b * iD;
      w[j] = D * u[j];
      x[j * nc + c] = (T)0;
      p[j * nc + c] = (T)0;
      sm1[j * nc + c] = (T)0;
      pg[j] += b * u[j];
    }
#pragma unroll
    for (int lf = 0; lf < NLF; ++lf) {
      const int32_t nb = col[c * NLF + lf];
      if (nb < 0) continue;
      const T o = off[c * NLF + lf] * invd[nb];
#pragma unroll
      for (int j = 0; j < DIM; ++j) w[j] -= o * (T)(-v[j * nc + nb] * inv_kbar);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      w0[j * nc + c] = w[j];
      pd[j] += w[j] * u[j];
    }
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double a = block_sum_t(pg[j], sh);
    const double b = block_sum_t(pd[j], sh);
    if (threadIdx.x == 0) {
      red[(2 * j) * gridDim.x + blockIdx.x] = a;
      red[(2 * j + 1) * gridDim.x + blockIdx.x] = b;
    }
  }
  if (last_block(count, gridDim.x)) {
    __threadfence();
    cg_finalize<T, DIM>(red, gridDim.x, sh, sc, true);
    if (threadIdx.x == 0) count[0] = 0;
  }
}

// iteration i: from r_{i-1}, w_{i-1}, s_{i-2} and alpha_{i-1}, beta_{i-1}:
//   s_{i-1} = w_{i-1} + beta s_{i-2};  r_i = r_{i-1} - alpha s_{i-1}
//   p_{i-1} = u_{i-1} + beta p_{i-2};  x += alpha p_{i-1}
//   w_i = B u_i, u_i = D^{-1} r_i;  partial (r_i, u_i), (w_i, u_i)
template <typename T, int DIM, int NLF>
__global__ void k_cg_iter(int64_t nc, const T* __restrict__ diag, const T* __restrict__ invd,
                          const int32_t* __restrict__ col,
                          const T* __restrict__ off, const T* __restrict__ r_old,
                          const T* __restrict__ w_old, const T* __restrict__ s_oldold,
                          T* __restrict__ r_new, T* __restrict__ w_new, T* __restrict__ s_new,
                          T* __restrict__ x, T* __restrict__ p, double* red, unsigned int* count,
                          double* sc) {
  __shared__ double sh[32];
  T alpha[DIM], beta[DIM];
  T pg[DIM], pd[DIM];  // per-thread partials in the vector precision
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    alpha[j] = (T)sc[DIM + j];
    beta[j] = (T)sc[2 * DIM + j];
    pg[j] = pd[j] = 0.0;
  }
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const T D = -diag[c], iD = invd[c];
    T un[DIM], w[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const int64_t i = j * nc + c;
      const T ro = r_old[i];
      const T s1 = w_old[i] + beta[j] * s_oldold[i];
      const T rn = ro - alpha[j] * s1;
      const T pp = ro * iD + beta[j] * p[i];
      p[i] = pp;
      x[i] += alpha[j] * pp;
      s_new[i] = s1;
      r_new[i] = rn;
      un[j] = rn * iD;
      w[j] = D * un[j];
      pg[j] += rn * un[j];
    }
#pragma unroll
    for (int lf = 0; lf < NLF; ++lf) {
      const int32_t nb = col[c * NLF + lf];
      if (nb < 0) continue;
      const T o = off[c * NLF + lf] * invd[nb];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const int64_t i = j * nc + nb;
        const T rn = r_old[i] - alpha[j] * (w_old[i] + beta[j] * s_oldold[i]);
        w[j] -= o * rn;
      }
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      w_new[j * nc + c] = w[j];
      pd[j] += w[j] * un[j];
    }
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double a = block_sum_t(pg[j], sh);
    const double b = block_sum_t(pd[j], sh);
    if (threadIdx.x == 0) {
      red[(2 * j) * gridDim.x + blockIdx.x] = a;
      red[(2 * j + 1) * gridDim.x + blockIdx.x] = b;
    }
  }
  if (last_block(count, gridDim.x)) {
    __threadfence();
    cg_finalize<T, DIM>(red, gridDim.x, sh, sc, false);
    if (threadIdx.x == 0) count[0] = 0;
  }
}

// z = x + alpha (u + beta p), u = D^{-1} r (the last step's update), in FP64
template <typename T, int DIM>
__global__ void k_cg_finish(int64_t nc, const T* __restrict__ invd, const T* __restrict__ r,
                            const T* __restrict__ x, const T* __restrict__ p,
                            const double* __restrict__ sc, double* __restrict__ z) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const T iD = invd[c];
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const int64_t i = j * nc + c;
    const T alpha = (T)sc[DIM + j], beta = (T)sc[2 * DIM + j];
    z[i] = (double)(x[i] + alpha * (r[i] * iD + beta * p[i]));
  }
}

// ---------------------------------------------------------------------
// The same iteration in one persistent cooperative launch: the blocks are
// co-resident (cudaLaunchCooperativeKernel) and meet at one grid barrier
// per iteration, after which every block forms the scalars from the
// per-block partial sums in the same fixed order.  The barrier's spin is
// bounded: on time-out the kernel sets an error flag and returns, and the
// host reports the error at its next synchronisation.
// ---------------------------------------------------------------------
constexpr unsigned int kBarrierSpinLimit = 1u << 24;  // x ~64 ns sleeps: ~1 s

struct GridBarrier {
  unsigned int* count;
  unsigned int* gen;
  int* err;
};

__device__ __forceinline__ bool grid_barrier(const GridBarrier& gb, unsigned int nblocks,
                                             unsigned int spin_limit = kBarrierSpinLimit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = gb.gen;
    volatile int* verr = gb.err;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(gb.count, 1u) == nblocks - 1) {
      atomicExch(gb.count, 0u);
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      unsigned int spins = 0;
      while (*vgen == g) {
        if (++spins > spin_limit || *verr) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (!ok) atomicExch(gb.err, 1);
    __threadfence();
    s_ok = ok && !*verr;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int kPersistThreads = 1024;

template <typename T, int DIM, int NLF>
__global__ void __launch_bounds__(kPersistThreads)
    k_cg_persist(int64_t nc, int iters, const double* __restrict__ v, double inv_kbar,
                 const T* __restrict__ diag, const T* __restrict__ invd,
                 const int32_t* __restrict__ col, const T* __restrict__ off, T* x, T* p, T* r0,
                 T* r1, T* w0, T* w1, T* s0, T* s1, double* part, GridBarrier gb,
                 double* __restrict__ zout) {
  __shared__ double sh[32];
  __shared__ double s_sc[3 * DIM];  // gamma_prev, alpha, beta
  __shared__ T s_ab[2 * DIM];       // alpha, beta in the vector precision
  const unsigned int nb = gridDim.x;
  T* r[2] = {r0, r1};
  T* w[2] = {w0, w1};
  T* s[2] = {s0, s1};
  T pg[DIM], pd[DIM];  // per-thread partials in the vector precision
  // ---- iteration 0: r0 = b, w0 = B D^-1 r0, x = p = 0, s_{-1} = 0
#pragma unroll
  for (int j = 0; j < DIM; ++j) pg[j] = pd[j] = (T)0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const T D = -diag[c], iD = invd[c];
    T u[DIM], ww[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const T b = (T)(-v[j * nc + c] * inv_kbar);
      r[0][j * nc + c] = b;
      u[j] = b * iD;
      ww[j] = D * u[j];
      x[j * nc + c] = (T)0;
      p[j * nc + c] = (T)0;
      s[1][j * nc + c] = (T)0;
      pg[j] += b * u[j];
    }
#pragma unroll
    for (int lf = 0; lf < NLF; ++lf) {
      const int32_t n2 = col[c * NLF + lf];
      if (n2 < 0) continue;
      const T o = off[c * NLF + lf] * invd[n2];
#pragma unroll
      for (int j = 0; j < DIM; ++j) ww[j] -= o * (T)(-v[j * nc + n2] * inv_kbar);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      w[0][j * nc + c] = ww[j];
      pd[j] += ww[j] * u[j];
    }
  }
  for (int it = 0; it < iters; ++it) {
    // partial sums of this block -> part[parity][2j(+1)][block]
    double* pp = part + (int64_t)(it & 1) * 2 * DIM * nb;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const double a = block_sum_t(pg[j], sh);
      const double b = block_sum_t(pd[j], sh);
      if (threadIdx.x == 0) {
        pp[(2 * j) * nb + blockIdx.x] = a;
        pp[(2 * j + 1) * nb + blockIdx.x] = b;
      }
    }
    if (!grid_barrier(gb, nb)) return;
    // every block forms the same scalars in the same order
    for (int j = 0; j < DIM; ++j) {
      const double gamma = warp0_sum<T>(pp + (2 * j) * nb, nb);
      const double delta = warp0_sum<T>(pp + (2 * j + 1) * nb, nb);
      if (threadIdx.x == 0) {
        double alpha, beta;
        if (it == 0) {
          beta = 0.0;
          alpha = delta != 0.0 ? gamma / delta : 0.0;
        } else {
          const double gp = s_sc[j], ap = s_sc[DIM + j];
          beta = gp != 0.0 ? gamma / gp : 0.0;
          const double den = ap != 0.0 ? delta - beta * gamma / ap : 0.0;
          alpha = den != 0.0 ? gamma / den : 0.0;
        }
        s_sc[j] = gamma;
        s_sc[DIM + j] = alpha;
        s_sc[2 * DIM + j] = beta;
        s_ab[j] = (T)alpha;
        s_ab[DIM + j] = (T)beta;
      }
    }
    __syncthreads();
    T alpha[DIM], beta[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      alpha[j] = s_ab[j];
      beta[j] = s_ab[DIM + j];
    }
    const int i = it + 1;  // the iteration this pass computes
    const T* ro_ = r[(i - 1) & 1];
    const T* wo_ = w[(i - 1) & 1];
    const T* so_ = s[i & 1];
    if (i == iters) {
      // last step: z = x + alpha (u + beta p), u = D^-1 r
      for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
           c += (int64_t)gridDim.x * blockDim.x) {
        const T iD = invd[c];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          const int64_t k = j * nc + c;
          zout[k] = (double)(x[k] + alpha[j] * (ro_[k] * iD + beta[j] * p[k]));
        }
      }
      return;
    }
    T* rn_ = r[i & 1];
    T* wn_ = w[i & 1];
    T* sn_ = s[(i - 1) & 1];
#pragma unroll
    for (int j = 0; j < DIM; ++j) pg[j] = pd[j] = (T)0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * blockDim.x) {
      const T D = -diag[c], iD = invd[c];
      T un[DIM], ww[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const int64_t k = j * nc + c;
        const T ro = ro_[k];
        const T s1 = wo_[k] + beta[j] * so_[k];
        const T rn = ro - alpha[j] * s1;
        const T pv = ro * iD + beta[j] * p[k];
        p[k] = pv;
        x[k] += alpha[j] * pv;
        sn_[k] = s1;
        rn_[k] = rn;
        un[j] = rn * iD;
        ww[j] = D * un[j];
        pg[j] += rn * un[j];
      }
#pragma unroll
      for (int lf = 0; lf < NLF; ++lf) {
        const int32_t n2 = col[c * NLF + lf];
        if (n2 < 0) continue;
        const T o = off[c * NLF + lf] * invd[n2];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          const int64_t k = j * nc + n2;
          ww[j] -= o * (ro_[k] - alpha[j] * (wo_[k] + beta[j] * so_[k]));
        }
      }
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        wn_[j * nc + c] = ww[j];
        pd[j] += ww[j] * un[j];
      }
    }
  }
}

template <typename T, int DIM, int NLF>
static bool cg_persist_run(hofv_ctx* c, const T* diag, const T* invd, const T* off, T* work,
                           int iters, const double* v, double* zout) {
  static int mb = -1;  // co-resident blocks of this instantiation, found once
  if (mb < 0) {
    int per_sm = 0, dev = 0, nsm = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persist<T, DIM, NLF>,
                                                      kPersistThreads, 0) != cudaSuccess)
      per_sm = 0;
    mb = std::min(per_sm, 1) * nsm;
    const char* env = getenv("HOFV_CG_PERSISTENT");
    if (env && env[0] == '0') mb = 0;
  }
  if (mb <= 0 || !c->d_bar) return false;
  const int64_t nc = c->nc, n = DIM * nc;
  T* x = work;
  T* p = work + n;
  int64_t nc_ = nc;
  int iters_ = std::max(iters, 1);
  double inv_kbar = 1.0 / c->mat.kbar;
  T *r0 = work + 2 * n, *r1 = work + 3 * n, *w0 = work + 4 * n, *w1 = work + 5 * n;
  T *s0 = work + 6 * n, *s1 = work + 7 * n;
  double* part = c->d_red;
  GridBarrier gb{c->d_bar, c->d_bar + 1, reinterpret_cast<int*>(c->d_bar + 2)};
  void* args[] = {&nc_, &iters_, (void*)&v, &inv_kbar, (void*)&diag, (void*)&invd,
                  (void*)&c->d_aj_col, (void*)&off, &x, &p, &r0, &r1, &w0, &w1, &s0, &s1, &part,
                  &gb, &zout};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_cg_persist<T, DIM, NLF>, dim3(mb),
                                                    dim3(kPersistThreads), args, 0, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <typename T, int DIM, int NLF>
static void cg_run(hofv_ctx* c, const T* diag, const T* invd, const T* off, T* work, int iters,
                   const double* v, double* zout) {
  const int64_t nc = c->nc, n = DIM * nc;
  T* x = work;
  T* p = work + n;
  T* r[2] = {work + 2 * n, work + 3 * n};
  T* w[2] = {work + 4 * n, work + 5 * n};
  T* s[2] = {work + 6 * n, work + 7 * n};
  const int blocks = c->red_blocks;
  double* red = c->d_red;
  unsigned int* cnt = c->d_count;
  double* sc = c->d_scal + 32;  // slots 32..40
  cudaStream_t st = c->stream;
  if (iters < 1) iters = 1;
  k_cg_init<T, DIM, NLF><<<blocks, kRedThreads, 0, st>>>(nc, v, 1.0 / c->mat.kbar, diag, invd, c->d_aj_col,
                                                   off, r[0], w[0], s[1], x, p, red, cnt, sc);
  for (int i = 1; i < iters; ++i)
    k_cg_iter<T, DIM, NLF><<<blocks, kRedThreads, 0, st>>>(nc, diag, invd, c->d_aj_col, off, r[(i - 1) & 1],
                                                     w[(i - 1) & 1], s[i & 1], r[i & 1], w[i & 1],
                                                     s[(i - 1) & 1], x, p, red, cnt, sc);
  k_cg_finish<T, DIM><<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(nc, invd, r[(iters - 1) & 1], x,
                                                                     p, sc, zout);
}

// Two co-resident blocks wait at a barrier that expects one more arrival
// than exists: the wait must run out and latch the error flag.
__global__ void k_barrier_probe(GridBarrier gb, unsigned int spin_limit) {
  grid_barrier(gb, gridDim.x + 1, spin_limit);
}

int barrier_selftest(hofv_ctx* c, int* timed_out) {
  *timed_out = 0;
  if (!c->d_bar) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  GridBarrier gb{c->d_bar, c->d_bar + 1, reinterpret_cast<int*>(c->d_bar + 2)};
  unsigned int limit = 1u << 14;
  void* args[] = {&gb, &limit};
  HOFV_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(2), dim3(32), args,
                                           0, c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  int err = 0;
  HOFV_CUDA(c, cudaMemcpy(&err, c->d_bar + 2, sizeof(int), cudaMemcpyDeviceToHost));
  *timed_out = err != 0;
  HOFV_CUDA(c, cudaMemset(c->d_bar, 0, 4 * sizeof(unsigned int)));
  return 0;
}

// the persistent cooperative solve when it fits on the device, else one
// launch per iteration; NLF = faces per cell (4 / 6 for quads / hexes,
// 3 / 4 for triangles / tetrahedra, 8 slots for polygons, 16 for polyhedra)
template <typename T, int DIM, int NLF>
static void aj_run(hofv_ctx* c, const T* diag, const T* invd, const T* off, T* work, int iters,
                   const double* v, double* z) {
  if (!cg_persist_run<T, DIM, NLF>(c, diag, invd, off, work, iters, v, z))
    cg_run<T, DIM, NLF>(c, diag, invd, off, work, iters, v, z);
}

template <typename T>
static void aj_dispatch(hofv_ctx* c, const T* diag, const T* invd, const T* off, T* work, int iters,
                        const double* v, double* z) {
  const bool simplex = c->nlf == c->dim + 1;
  if (c->dim == 2) {
    if (simplex) aj_run<T, 2, 3>(c, diag, invd, off, work, iters, v, z);
    else if (c->poly) aj_run<T, 2, kPolyMaxSides>(c, diag, invd, off, work, iters, v, z);
    else aj_run<T, 2, 4>(c, diag, invd, off, work, iters, v, z);
  } else {
    if (simplex) aj_run<T, 3, 4>(c, diag, invd, off, work, iters, v, z);
    else if (c->polyh) aj_run<T, 3, kPolyhedronMaxFaces>(c, diag, invd, off, work, iters, v, z);
    else aj_run<T, 3, 6>(c, diag, invd, off, work, iters, v, z);
  }
}

int aj_precondition(hofv_ctx* c, int kind, int iters, const double* v, double* z) {
  if (c->nlf != 2 * c->dim && c->nlf != c->dim + 1 && !(c->poly && c->nlf == kPolyMaxSides) &&
      !(c->polyh && c->nlf == kPolyhedronMaxFaces))
    return fail(c, HOFV_ENOTSUP, "cell shape without an approximate-Jacobian kernel");
  if (kind == HOFV_PC_AJ64)
    aj_dispatch<double>(c, c->d_aj_diag, c->d_aj_invd, c->d_aj_off, c->d_cg64, iters, v, z);
  else
    aj_dispatch<float>(c, c->d_aj_diag32, c->d_aj_invd32, c->d_aj_off32, c->d_cg32, iters, v, z);
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

}  // namespace hofv
