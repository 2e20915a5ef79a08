// krylov.cu -- vector kernels of the flexible GMRES outer solver and the
// compact-stencil approximate-Jacobian preconditioner (arXiv 2601.18417,
// Sec. 4.1).
//
// Reductions are deterministic: each block writes a partial sum, and the
// last block to finish (an atomic ticket, no waiting) adds the partials in
// block order and publishes the result to device memory, where the next
// kernel on the stream reads it.  No host round trip is needed inside Jv or
// inside the preconditioner.
#include "hofv_internal.cuh"

namespace hofv {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// Returns true in thread 0 of the block that finished last.
__device__ __forceinline__ bool last_block(unsigned int* count, unsigned int nblocks) {
  __shared__ bool is_last;
  __threadfence();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(count, 1u);
    is_last = (t == nblocks - 1);
  }
  __syncthreads();
  return is_last;
}

// Sum of partials red[0..nb) by the whole (last) block: thread t adds
// partials t, t + blockDim, ... in order, then a fixed-shape tree.  The
// result (valid in thread 0) does not depend on which block finished last.
__device__ __forceinline__ double final_sum(const double* red, unsigned int nb, double* sh) {
  double s = 0.0;
  for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(red + b);
  return block_sum(s, sh);
}

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
    const double t = final_sum(red + k * gridDim.x, gridDim.x, sh);
    if (threadIdx.x == 0) {
      out[k] = mode == 1 ? sqrt(t) : t;
      count[k] = 0;
    }
  }
}

void launch_dots(const double* X, int64_t ldx, const double* y, int nvec, int64_t n, double* red,
                 unsigned int* count, double* out, int blocks, cudaStream_t st, int mode) {
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
// Kbar = 1.  z = A^{-1} v solves B z = -v / Kbar with B = -A1 (SPD),
// by a fixed number of Jacobi-preconditioned CG iterations on all `dim`
// right-hand sides at once.  T = float (FP32 storage and arithmetic) or
// double.  Scalars: sc[0..d) rz, sc[d..2d) alpha, sc[2d..3d) beta.
// ---------------------------------------------------------------------
template <typename T, int DIM>
__global__ void k_cg_init(int64_t nc, const double* __restrict__ v, double inv_kbar,
                          const T* __restrict__ diag, T* __restrict__ x, T* __restrict__ r,
                          T* __restrict__ z, T* __restrict__ p, double* red,
                          unsigned int* count, double* sc) {
  __shared__ double sh[32];
  double part[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) part[j] = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const T dg = -diag[c];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const int64_t i = j * nc + c;
      const T rr = (T)(-v[i] * inv_kbar);
      const T zz = rr / dg;
      r[i] = rr;
      z[i] = zz;
      x[i] = (T)0;
      p[i] = (T)0;
      part[j] += (double)rr * (double)zz;
    }
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double s = block_sum(part[j], sh);
    if (threadIdx.x == 0) red[j * gridDim.x + blockIdx.x] = s;
  }
  if (last_block(count, gridDim.x)) {
    __threadfence();
    for (int j = 0; j < DIM; ++j) {
      const double t = final_sum(red + j * gridDim.x, gridDim.x, sh);
      if (threadIdx.x == 0) {
        sc[j] = t;
        sc[2 * DIM + j] = 0.0;
      }
    }
    if (threadIdx.x == 0) count[0] = 0;
  }
}

// p_new = z + beta p_old (own and neighbours, on the fly); q = B p_new;
// partial p.q -> alpha = rz / pq
template <typename T, int DIM>
__global__ void k_cg_spmv(int64_t nc, const T* __restrict__ diag, const int32_t* __restrict__ col,
                          const T* __restrict__ off, const T* __restrict__ z,
                          const T* __restrict__ p_old, T* __restrict__ p_new, T* __restrict__ q,
                          double* red, unsigned int* count, double* sc) {
  constexpr int NLF = 2 * DIM;
  __shared__ double sh[32];
  double part[DIM];
  T beta[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    part[j] = 0.0;
    beta[j] = (T)sc[2 * DIM + j];
  }
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const T dg = -diag[c];
    T pc[DIM], qc[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      pc[j] = z[j * nc + c] + beta[j] * p_old[j * nc + c];
      qc[j] = dg * pc[j];
    }
#pragma unroll
    for (int lf = 0; lf < NLF; ++lf) {
      const int32_t nb = col[c * NLF + lf];
      if (nb < 0) continue;
      const T o = off[c * NLF + lf];
#pragma unroll
      for (int j = 0; j < DIM; ++j) qc[j] -= o * (z[j * nc + nb] + beta[j] * p_old[j * nc + nb]);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      p_new[j * nc + c] = pc[j];
      q[j * nc + c] = qc[j];
      part[j] += (double)pc[j] * (double)qc[j];
    }
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double s = block_sum(part[j], sh);
    if (threadIdx.x == 0) red[j * gridDim.x + blockIdx.x] = s;
  }
  if (last_block(count, gridDim.x)) {
    __threadfence();
    for (int j = 0; j < DIM; ++j) {
      const double t = final_sum(red + j * gridDim.x, gridDim.x, sh);
      if (threadIdx.x == 0) sc[DIM + j] = t != 0.0 ? sc[j] / t : 0.0;
    }
    if (threadIdx.x == 0) count[0] = 0;
  }
}

// x += alpha p; r -= alpha q; z = r / D; partial r.z -> beta, rz
template <typename T, int DIM>
__global__ void k_cg_update(int64_t nc, const T* __restrict__ diag, const T* __restrict__ p,
                            const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                            T* __restrict__ z, double* red, unsigned int* count, double* sc) {
  __shared__ double sh[32];
  double part[DIM];
  T alpha[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    part[j] = 0.0;
    alpha[j] = (T)sc[DIM + j];
  }
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const T dg = -diag[c];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const int64_t i = j * nc + c;
      x[i] += alpha[j] * p[i];
      const T rr = r[i] - alpha[j] * q[i];
      const T zz = rr / dg;
      r[i] = rr;
      z[i] = zz;
      part[j] += (double)rr * (double)zz;
    }
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const double s = block_sum(part[j], sh);
    if (threadIdx.x == 0) red[j * gridDim.x + blockIdx.x] = s;
  }
  if (last_block(count, gridDim.x)) {
    __threadfence();
    for (int j = 0; j < DIM; ++j) {
      const double t = final_sum(red + j * gridDim.x, gridDim.x, sh);
      if (threadIdx.x == 0) {
        sc[2 * DIM + j] = sc[j] != 0.0 ? t / sc[j] : 0.0;
        sc[j] = t;
      }
    }
    if (threadIdx.x == 0) count[0] = 0;
  }
}

template <typename T>
__global__ void k_to_double(int64_t n, const T* __restrict__ x, double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = (double)x[i];
}

template <typename T, int DIM>
static void cg_run(hofv_ctx* c, const T* diag, const T* off, T* work, int iters, const double* v,
                   double* zout) {
  const int64_t nc = c->nc, n = DIM * nc;
  T* x = work;
  T* r = work + n;
  T* z = work + 2 * n;
  T* p0 = work + 3 * n;
  T* p1 = work + 4 * n;
  T* q = work + 5 * n;
  const int blocks = c->red_blocks;
  double* red = c->d_red;
  unsigned int* cnt = c->d_count;
  double* sc = c->d_scal + 32;  // slots 32..40: CG rz, alpha, beta per component
  cudaStream_t st = c->stream;
  k_cg_init<T, DIM><<<blocks, kRedThreads, 0, st>>>(nc, v, 1.0 / c->mat.kbar, diag, x, r, z, p0,
                                                   red, cnt, sc);
  for (int it = 0; it < iters; ++it) {
    T* po = (it & 1) ? p1 : p0;
    T* pn = (it & 1) ? p0 : p1;
    k_cg_spmv<T, DIM><<<blocks, kRedThreads, 0, st>>>(nc, diag, c->d_aj_col, off, z, po, pn, q, red,
                                                     cnt, sc);
    k_cg_update<T, DIM><<<blocks, kRedThreads, 0, st>>>(nc, diag, pn, q, x, r, z, red, cnt, sc);
  }
  k_to_double<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(n, x, zout);
}

int aj_precondition(hofv_ctx* c, int kind, int iters, const double* v, double* z) {
  if (kind == HOFV_PC_AJ64) {
    if (c->dim == 2)
      cg_run<double, 2>(c, c->d_aj_diag, c->d_aj_off, c->d_cg64, iters, v, z);
    else
      cg_run<double, 3>(c, c->d_aj_diag, c->d_aj_off, c->d_cg64, iters, v, z);
  } else {
    if (c->dim == 2)
      cg_run<float, 2>(c, c->d_aj_diag32, c->d_aj_off32, c->d_cg32, iters, v, z);
    else
      cg_run<float, 3>(c, c->d_aj_diag32, c->d_aj_off32, c->d_cg32, iters, v, z);
  }
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

}  // namespace hofv
