// setup.cu -- mesh-only set-up on the device: nearest-neighbour stencils, least-squares reconstruction coefficients by
// Householder QR, stabilisation extrapolation weights and the per-face
// auxiliary data of the residual and of the approximate Jacobian.
//
// Method: arXiv 2601.18417, Sec. 3.5.1 (least-squares Taylor reconstruction, eqs. te-lsA, weightFunc),
// Sec. 3.5.2 (stencils), Sec. 3.5.3 (displacement-boundary ghost node),
// Sec. 3.4 and App. B (alpha stabilisation extrapolation), Sec. 4.1 (AJ).
#include <math.h>

#include "hofv_internal.cuh"

namespace hofv {

// ---------------------------------------------------------------------
// stencils: the S nearest cell centroids of each reference point, ordered
// by the key floor(d^2 * 2^(24 - 2 e) + 1/2) (e: exponent of the reference
// cell size) and then by cell id.  One thread per query; the candidates
// come from a uniform bucket grid, grown until every cell outside the
// searched block is provably farther than the S-th member.
// ---------------------------------------------------------------------
struct Buckets {
  const int32_t* start;  // [nbuckets + 1]
  const int32_t* items;  // [nc]
  int nb[3];
  double lo[3], bs;
};

__device__ __forceinline__ long long dist_key(int dim, const double* __restrict__ xc, int32_t cell,
                                              const double* xr, double scale) {
  const double dx = __dsub_rn(xc[3 * (int64_t)cell], xr[0]);
  const double dy = __dsub_rn(xc[3 * (int64_t)cell + 1], xr[1]);
  double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (dim == 3) {
    const double dz = __dsub_rn(xc[3 * (int64_t)cell + 2], xr[2]);
    d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
  }
  return (long long)floor(__dadd_rn(__dmul_rn(d2, scale), 0.5));
}

__global__ void k_stencils(int dim, int S_full, int64_t nq_face, int64_t nq_cell, int64_t nfid,
                           int64_t nsym0, int64_t nc, const double* __restrict__ xf,
                           const double* __restrict__ xc, Buckets B, double scale, int32_t* fst,
                           int32_t* cst, int* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nq_face + nq_cell) return;
  double xr[3];
  const bool is_face = t < nq_face;
  const int64_t id = is_face ? t : t - nq_face;
  // a symmetry face searches ceil(S/2) cells; mirrors fill the other slots
  const bool sym = is_face && id >= nsym0;
  const int S = sym ? (S_full + 1) / 2 : S_full;
  for (int a = 0; a < 3; ++a) xr[a] = is_face ? xf[3 * id + a] : xc[3 * id + a];
  long long key[kMaxS];
  int32_t idx[kMaxS];
  int cnt = 0;
  int ib[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    int i = (int)floor((xr[a] - B.lo[a]) / B.bs);
    ib[a] = min(max(i, 0), B.nb[a] - 1);
  }
  const int maxr = B.nb[0] + B.nb[1] + B.nb[2];
  int prev_lo[3] = {1, 1, 1}, prev_hi[3] = {0, 0, 0};  // empty block
  bool done = false;
  for (int r = 1; r <= maxr && !done; ++r) {
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = a < dim ? max(ib[a] - r, 0) : 0;
      hi[a] = a < dim ? min(ib[a] + r, B.nb[a] - 1) : 0;
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          // skip buckets already visited at the previous radius
          if (i >= prev_lo[0] && i <= prev_hi[0] && j >= prev_lo[1] && j <= prev_hi[1] &&
              k >= prev_lo[2] && k <= prev_hi[2])
            continue;
          const int64_t b = ((int64_t)k * B.nb[1] + j) * B.nb[0] + i;
          for (int32_t s = B.start[b]; s < B.start[b + 1]; ++s) {
            const int32_t cell = B.items[s];
            const long long kk = dist_key(dim, xc, cell, xr, scale);
            if (cnt == S && (kk > key[S - 1] || (kk == key[S - 1] && cell > idx[S - 1]))) continue;
            int pos = cnt < S ? cnt : S - 1;
            while (pos > 0 && (key[pos - 1] > kk || (key[pos - 1] == kk && idx[pos - 1] > cell))) {
              key[pos] = key[pos - 1];
              idx[pos] = idx[pos - 1];
              --pos;
            }
            key[pos] = kk;
            idx[pos] = cell;
            if (cnt < S) ++cnt;
          }
        }
    for (int a = 0; a < 3; ++a) {
      prev_lo[a] = lo[a];
      prev_hi[a] = hi[a];
    }
    if (cnt < S) continue;
    bool whole = true;
    double reach = 1e300;
    for (int a = 0; a < dim; ++a) {
      if (lo[a] > 0) {
        whole = false;
        reach = fmin(reach, xr[a] - (B.lo[a] + lo[a] * B.bs));
      }
      if (hi[a] < B.nb[a] - 1) {
        whole = false;
        reach = fmin(reach, (B.lo[a] + (hi[a] + 1) * B.bs) - xr[a]);
      }
    }
    const double reach_key = __dmul_rn(__dmul_rn(reach, reach), scale);
    if (whole || (double)key[S - 1] + 2.0 < reach_key) done = true;
  }
  if (!done) {
    atomicExch(status, 1);
    return;
  }
  const int64_t tile = id / kTile, li = id % kTile;
  int32_t* out = is_face ? fst : cst;
  for (int n = 0; n < S; ++n) out[(tile * S_full + n) * kTile + li] = idx[n];
  if (sym) {
    const int half2 = S_full / 2;
    for (int k = 0; k < half2; ++k)
      out[(tile * S_full + S + k) * kTile + li] = (int32_t)(nc + (id - nsym0) * half2 + k);
  }
}

// ghosts of the symmetry faces: ghost g = b * floor(S/2) + k mirrors the k-th
// nearest cell of symmetry face b in that face's plane
__global__ void k_ghosts(int64_t ng, int half2, int S, int64_t nc, int64_t nsym0,
                         const int32_t* __restrict__ fst, const double* __restrict__ xf,
                         const double* __restrict__ nrm, const double* __restrict__ xc,
                         int32_t* gsrc, int32_t* gface, double* xce) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const int64_t f = nsym0 + g / half2;
  const int k = (int)(g % half2);
  const int32_t src = fst[((f / kTile) * S + k) * kTile + f % kTile];
  gsrc[g] = src;
  gface[g] = (int32_t)f;
  double dn = 0.0;
  for (int a = 0; a < 3; ++a) dn += (xc[3 * (int64_t)src + a] - xf[3 * f + a]) * nrm[3 * f + a];
  for (int a = 0; a < 3; ++a) xce[3 * (nc + g) + a] = xc[3 * (int64_t)src + a] - 2.0 * dn * nrm[3 * f + a];
}

int run_ghosts(hofv_ctx* c) {
  const int half2 = c->S / 2;
  c->ng = c->nfy * half2;
  if (c->ng == 0) return 0;
  if (dev_alloc(c, &c->d_gsrc, c->ng) || dev_alloc(c, &c->d_gface, c->ng) ||
      dev_alloc(c, &c->d_xce, (c->nc + c->ng) * 3))
    return HOFV_ENOMEM;
  HOFV_CUDA(c, cudaMemcpyAsync(c->d_xce, c->d_xc, sizeof(double) * c->nc * 3,
                               cudaMemcpyDeviceToDevice, c->stream));
  k_ghosts<<<(unsigned)((c->ng + 127) / 128), 128, 0, c->stream>>>(
      c->ng, half2, c->S, c->nc, c->nfi + c->nfd, c->d_fst, c->d_xf, c->d_nrm, c->d_xc, c->d_gsrc,
      c->d_gface, c->d_xce);
  HOFV_CUDA(c, cudaGetLastError());
  c->gsrc_host.resize(c->ng);
  HOFV_CUDA(c, cudaMemcpyAsync(c->gsrc_host.data(), c->d_gsrc, sizeof(int32_t) * c->ng,
                               cudaMemcpyDeviceToHost, c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

int run_stencils(hofv_ctx* c, const std::vector<int64_t>& bstart,
                 const std::vector<int32_t>& bitems, const int nb[3], const double lo[3],
                 double bs) {
  std::vector<int32_t> st32(bstart.size());
  for (size_t i = 0; i < bstart.size(); ++i) st32[i] = (int32_t)bstart[i];
  int32_t *d_start = nullptr, *d_items = nullptr;
  int* d_status = nullptr;
  HOFV_CUDA(c, cudaMalloc(&d_start, st32.size() * sizeof(int32_t)));
  HOFV_CUDA(c, cudaMalloc(&d_items, bitems.size() * sizeof(int32_t) + 4));
  HOFV_CUDA(c, cudaMalloc(&d_status, sizeof(int)));
  HOFV_CUDA(c, cudaMemcpyAsync(d_start, st32.data(), st32.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
  HOFV_CUDA(c, cudaMemcpyAsync(d_items, bitems.data(), bitems.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
  HOFV_CUDA(c, cudaMemsetAsync(d_status, 0, sizeof(int), c->stream));
  Buckets B;
  B.start = d_start;
  B.items = d_items;
  for (int a = 0; a < 3; ++a) {
    B.nb[a] = nb[a];
    B.lo[a] = lo[a];
  }
  B.bs = bs;
  const double scale = ldexp(1.0, 24 - 2 * c->href_exp);
  const int64_t nq = c->nfid + c->nc;
  const int T = 64;
  k_stencils<<<(unsigned)((nq + T - 1) / T), T, 0, c->stream>>>(
      c->dim, c->S, c->nfid, c->nc, c->nfid, c->nfi + c->nfd, c->nc, c->d_xf, c->d_xc, B, scale,
      c->d_fst, c->d_cst, d_status);
  HOFV_CUDA(c, cudaGetLastError());
  int status = 0;
  HOFV_CUDA(c, cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  cudaFree(d_start);
  cudaFree(d_items);
  cudaFree(d_status);
  if (status) return fail(c, HOFV_EINVAL, "stencil search did not converge");
  return 0;
}

// ---------------------------------------------------------------------
// least-squares reconstruction, one warp per system.  A = W^1/2 Q^T
// (rows: stencil nodes [+ ghost], columns: scaled Taylor terms) is
// factorised A = Qh R by Householder reflections in shared memory; a
// linear functional g of the fitted Taylor coefficients then has node
// weights e = W^1/2 Qh R^{-T} g, i.e. e^T = g^T Abar with
// Abar = M^{-1} Q W (eqs. maQw, lsA).
// ---------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// scaled Taylor basis q(X), graded order, 1/(a! b! c!) factors (eq. qAnda, App. B)
__device__ void taylor_basis(int dim, int p, const double* X, double* q) {
  const double fact[4] = {1.0, 1.0, 2.0, 6.0};
  double px[4], py[4], pz[4];
  px[0] = py[0] = pz[0] = 1.0;
  for (int k = 1; k <= 3; ++k) {
    px[k] = px[k - 1] * X[0];
    py[k] = py[k - 1] * X[1];
    pz[k] = pz[k - 1] * X[2];
  }
  int t = 0;
  for (int deg = 0; deg <= p; ++deg) {
    if (dim == 2) {
      for (int a = deg; a >= 0; --a) {
        const int b = deg - a;
        q[t++] = px[a] * py[b] / (fact[a] * fact[b]);
      }
    } else {
      for (int a = deg; a >= 0; --a)
        for (int b = deg - a; b >= 0; --b) {
          const int e = deg - a - b;
          q[t++] = px[a] * py[b] * pz[e] / (fact[a] * fact[b] * fact[e]);
        }
    }
  }
}

struct LsqParams {
  int dim, p, S, Nt, NR, nlf, Q, R;
  double k2, ek;
  int64_t nfid, nfi, nc;
  int64_t nfde;        // displacement faces end (ghost node for f in [nfi, nfde))
  const double* xq;    // [nf][Q][3]
  const double* xf;    // [nf][3]
  const double* xc;    // [nc][3]
  const int32_t* fst;  // tiled
  const int32_t* cst;  // tiled
  const int64_t* cf;   // [nc][nlf] (device copy)
  double* fco;
  double* gco;
  double* cex;
  unsigned long long* cond_bits;
  int* status;
  // cell averages over the cell Gauss points (inertia term)
  int QC;
  const double* cqx;   // [nc][QC][3]
  const double* cqw;   // [nc][QC]
  const double* vol;   // [nc]
  double* cmass;       // tiled like cst
};

// Factorise the system of one reference point.  Each lane owns rows
// lane, lane+32, ... of A (column-major in smem: A[col * NR + row]).
// Returns h = 2 r_s.  sw[row] keeps sqrt(w) of owned rows.
__device__ double lsq_factor(const LsqParams& P, const double* xt, const int32_t* nodes,
                             int nrow, double* A, double* v0, double* beta, double* sw,
                             int lane) {
  const int dim = P.dim;
  // stencil radius measured from the reference point
  double r2 = 0.0;
  for (int r = lane; r < P.S; r += 32) {
    double s = 0;
    for (int a = 0; a < dim; ++a) {
      const double e = P.xc[3 * (int64_t)nodes[r] + a] - xt[a];
      s += e * e;
    }
    r2 = fmax(r2, s);
  }
  const double h = 2.0 * sqrt(warp_max(r2));
  for (int r = lane; r < P.NR; r += 32) {
    double q[kMaxNt];
    double w = 0.0;
    if (r < P.S) {
      double X[3] = {0, 0, 0}, dd = 0;
      for (int a = 0; a < dim; ++a) {
        X[a] = (P.xc[3 * (int64_t)nodes[r] + a] - xt[a]) / h;
        dd += X[a] * X[a];
      }
      w = (exp(-dd * P.k2) - P.ek) / (1.0 - P.ek);
      taylor_basis(dim, P.p, X, q);
    } else if (r < nrow) {  // ghost node at the reference point (Sec. 3.5.3)
      w = 1.0;
      for (int t = 0; t < P.Nt; ++t) q[t] = t == 0 ? 1.0 : 0.0;
    } else {
      for (int t = 0; t < P.Nt; ++t) q[t] = 0.0;
    }
    const double s = sqrt(w);
    sw[r / 32] = s;
    for (int t = 0; t < P.Nt; ++t) A[t * P.NR + r] = s * q[t];
  }
  __syncwarp();
  for (int k = 0; k < P.Nt; ++k) {
    double ss = 0.0;
    for (int r = k + lane; r < nrow; r += 32) {
      const double a = A[k * P.NR + r];
      ss += a * a;
    }
    ss = warp_sum(ss);
    const double x0 = A[k * P.NR + k];
    const double nrm = sqrt(ss);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double vk = x0 - alpha;
    const double vtv = ss - x0 * x0 + vk * vk;
    const double bk = vtv > 0.0 ? 2.0 / vtv : 0.0;
    __syncwarp();
    for (int j = k + 1; j < P.Nt; ++j) {
      double s = 0.0;
      for (int r = k + 1 + lane; r < nrow; r += 32) s += A[k * P.NR + r] * A[j * P.NR + r];
      s = warp_sum(s) + vk * A[j * P.NR + k];
      const double f = bk * s;
      __syncwarp();
      for (int r = k + 1 + lane; r < nrow; r += 32) A[j * P.NR + r] -= f * A[k * P.NR + r];
      if (lane == 0) A[j * P.NR + k] -= f * vk;
      __syncwarp();
    }
    if (lane == 0) {
      A[k * P.NR + k] = alpha;  // R_kk
      v0[k] = vk;
      beta[k] = bk;
    }
    __syncwarp();
  }
  return h;
}

// weights e (owned rows, registers z[]) of the functional g
__device__ void lsq_functional(const LsqParams& P, int nrow, const double* A, const double* v0,
                               const double* beta, const double* sw, const double* g, double* z,
                               int lane) {
  double y[kMaxNt];
  for (int k = 0; k < P.Nt; ++k) {  // R^T y = g (R_ik = A[k*NR + i], i < k)
    double s = g[k];
    for (int i = 0; i < k; ++i) s -= A[k * P.NR + i] * y[i];
    y[k] = s / A[k * P.NR + k];
  }
  const int nown = (P.NR + 31) / 32;
  for (int o = 0; o < nown; ++o) {
    const int r = lane + 32 * o;
    z[o] = r < P.Nt ? y[r] : 0.0;
  }
  for (int k = P.Nt - 1; k >= 0; --k) {
    double s = 0.0;
    for (int o = 0; o < nown; ++o) {
      const int r = lane + 32 * o;
      if (r > k && r < nrow) s += A[k * P.NR + r] * z[o];
    }
    s = warp_sum(s);
    // v_k has first entry v0[k] at row k
    const int ok = k / 32;
    const double zk = __shfl_sync(0xffffffffu, z[ok], k % 32);
    s += v0[k] * zk;
    const double f = beta[k] * s;
    for (int o = 0; o < nown; ++o) {
      const int r = lane + 32 * o;
      if (r > k && r < nrow) z[o] -= f * A[k * P.NR + r];
      if (r == k) z[o] -= f * v0[k];
    }
  }
  for (int o = 0; o < nown; ++o) z[o] *= sw[o];
}

__device__ void record_cond(const LsqParams& P, const double* A, int lane) {
  if (lane != 0) return;
  double mx = 0.0, mn = 1e300;
  for (int k = 0; k < P.Nt; ++k) {
    const double r = fabs(A[k * P.NR + k]);
    mx = fmax(mx, r);
    mn = fmin(mn, r);
  }
  const double est = mn > 0.0 ? (mx / mn) * (mx / mn) : 1e300;
  // rank-deficient stencil (e.g. collinear centroids): cond(M) above ~1e24
  if (!(mn > 1e-12 * mx)) atomicExch(P.status, 2);
  atomicMax(P.cond_bits, (unsigned long long)__double_as_longlong(est));
}

__global__ void k_lsq_faces(LsqParams P) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int per = P.Nt * P.NR + 2 * kMaxNt;
  double* A = sm + wib * per;
  double* v0 = A + P.Nt * P.NR;
  double* beta = v0 + kMaxNt;
  const int64_t sys = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (sys >= P.nfid * P.Q) return;
  const int64_t f = sys / P.Q;
  const int q = (int)(sys % P.Q);
  const int64_t tile = f / kTile, fi = f % kTile;
  int32_t nodes[kMaxS];
  for (int n = 0; n < P.S; ++n) nodes[n] = P.fst[(tile * P.S + n) * kTile + fi];
  const bool ghost = f >= P.nfi && f < P.nfde;
  const int nrow = P.S + (ghost ? 1 : 0);
  double xt[3];
  for (int a = 0; a < 3; ++a) xt[a] = P.xq[(f * P.Q + q) * 3 + a];
  double sw[4];
  const double h = lsq_factor(P, xt, nodes, nrow, A, v0, beta, sw, lane);
  record_cond(P, A, lane);
  const int nown = (P.NR + 31) / 32;
  for (int i = 0; i < P.dim; ++i) {
    double g[kMaxNt];
    for (int t = 0; t < P.Nt; ++t) g[t] = t == 1 + i ? 1.0 / h : 0.0;
    double z[4];
    lsq_functional(P, nrow, A, v0, beta, sw, g, z, lane);
    for (int o = 0; o < nown; ++o) {
      const int r = lane + 32 * o;
      if (r < P.S)
        P.fco[((tile * P.S + r) * kTile + fi) * P.R + q * P.dim + i] = z[o];
      else if (ghost && r == P.S)
        P.gco[(f - P.nfi) * P.R + q * P.dim + i] = z[o];
    }
  }
}

__global__ void k_lsq_cells(LsqParams P) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int per = P.Nt * P.NR + 2 * kMaxNt;
  double* A = sm + wib * per;
  double* v0 = A + P.Nt * P.NR;
  double* beta = v0 + kMaxNt;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (c >= P.nc) return;
  const int64_t tile = c / kTile, ci = c % kTile;
  int32_t nodes[kMaxS];
  for (int n = 0; n < P.S; ++n) nodes[n] = P.cst[(tile * P.S + n) * kTile + ci];
  double xt[3];
  for (int a = 0; a < 3; ++a) xt[a] = P.xc[3 * c + a];
  double sw[4];
  const double h = lsq_factor(P, xt, nodes, P.S, A, v0, beta, sw, lane);
  record_cond(P, A, lane);
  const int nown = (P.NR + 31) / 32;
  for (int lf = 0; lf < P.nlf; ++lf) {
    const int64_t f = P.cf[c * P.nlf + lf];
    if (f < 0) continue;  // polygon slot without a face: its weights stay zero
    double X[3] = {0, 0, 0}, g[kMaxNt];
    for (int a = 0; a < P.dim; ++a) X[a] = (P.xf[3 * f + a] - xt[a]) / h;
    taylor_basis(P.dim, P.p, X, g);
    g[0] = 0.0;  // u_P itself enters eq. (alphaJump) directly
    double z[4];
    lsq_functional(P, P.S, A, v0, beta, sw, g, z, lane);
    for (int o = 0; o < nown; ++o) {
      const int r = lane + 32 * o;
      if (r < P.S) P.cex[((tile * P.S + r) * kTile + ci) * P.nlf + lf] = z[o];
    }
  }
}


// Cell-average weights of the cell fit: the Taylor extrapolation of
// eq. (alphaJump) from the centroid to every cell Gauss point, averaged with
// the Gauss weights, ubar_P = u_P + sum_N cmass_N u_N (eq. inertiaTerm).
__global__ void k_lsq_cell_mass(LsqParams P) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int per = P.Nt * P.NR + 2 * kMaxNt;
  double* A = sm + wib * per;
  double* v0 = A + P.Nt * P.NR;
  double* beta = v0 + kMaxNt;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (c >= P.nc) return;
  const int64_t tile = c / kTile, ci = c % kTile;
  int32_t nodes[kMaxS];
  for (int n = 0; n < P.S; ++n) nodes[n] = P.cst[(tile * P.S + n) * kTile + ci];
  double xt[3];
  for (int a = 0; a < 3; ++a) xt[a] = P.xc[3 * c + a];
  double sw[4];
  const double h = lsq_factor(P, xt, nodes, P.S, A, v0, beta, sw, lane);
  double g[kMaxNt];
  for (int t = 0; t < P.Nt; ++t) g[t] = 0.0;
  const double iv = 1.0 / P.vol[c];
  for (int q = 0; q < P.QC; ++q) {
    double X[3] = {0, 0, 0}, b[kMaxNt];
    for (int a = 0; a < P.dim; ++a) X[a] = (P.cqx[(c * P.QC + q) * 3 + a] - xt[a]) / h;
    taylor_basis(P.dim, P.p, X, b);
    const double wq = P.cqw[c * P.QC + q] * iv;
    for (int t = 1; t < P.Nt; ++t) g[t] = fma(wq, b[t], g[t]);  // u_P enters directly
  }
  double z[4];
  lsq_functional(P, P.S, A, v0, beta, sw, g, z, lane);
  const int nown = (P.NR + 31) / 32;
  for (int o = 0; o < nown; ++o) {
    const int r = lane + 32 * o;
    if (r < P.S) P.cmass[(tile * P.S + r) * kTile + ci] = z[o];
  }
}

static LsqParams lsq_params(hofv_ctx* c) {
  LsqParams P;
  P.dim = c->dim;
  P.p = c->p;
  P.S = c->S;
  P.Nt = c->Nt;
  P.NR = ((c->S + 1 + 31) / 32) * 32;
  P.nlf = c->nlf;
  P.Q = c->Q;
  P.R = c->Q * c->dim;
  P.k2 = c->kw * c->kw;
  P.ek = exp(-P.k2);
  P.nfid = c->nfid;
  P.nfi = c->nfi;
  P.nfde = c->nfi + c->nfd;
  P.nc = c->nc;
  P.xq = c->d_xq;
  P.xf = c->d_xf;
  P.xc = c->ng > 0 ? c->d_xce : c->d_xc;  // with the mirrored positions of the ghosts
  P.fst = c->d_fst;
  P.cst = c->d_cst;
  P.fco = c->d_fco;
  P.gco = c->d_gco;
  P.cex = c->d_cex;
  P.cf = c->d_cf;
  P.QC = c->QC;
  P.cqx = c->d_cqx;
  P.cqw = c->d_cqw;
  P.vol = c->d_vol;
  P.cmass = c->d_cmass;
  P.cond_bits = nullptr;
  P.status = nullptr;
  return P;
}

int run_lsq(hofv_ctx* c) {
  LsqParams P = lsq_params(c);
  unsigned long long* d_cond = nullptr;
  int* d_status = nullptr;
  HOFV_CUDA(c, cudaMalloc(&d_cond, sizeof(unsigned long long)));
  HOFV_CUDA(c, cudaMalloc(&d_status, sizeof(int)));
  HOFV_CUDA(c, cudaMemsetAsync(d_cond, 0, sizeof(unsigned long long), c->stream));
  HOFV_CUDA(c, cudaMemsetAsync(d_status, 0, sizeof(int), c->stream));
  P.cond_bits = d_cond;
  P.status = d_status;
  const int warps = 4;
  const size_t smem = sizeof(double) * warps * (P.Nt * P.NR + 2 * kMaxNt);
  HOFV_CUDA(c, cudaFuncSetAttribute(k_lsq_faces, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  HOFV_CUDA(c, cudaFuncSetAttribute(k_lsq_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  const int64_t nsys = c->nfid * c->Q;
  if (nsys > 0) {
    k_lsq_faces<<<(unsigned)((nsys + warps - 1) / warps), 32 * warps, smem, c->stream>>>(P);
    HOFV_CUDA(c, cudaGetLastError());
  }
  k_lsq_cells<<<(unsigned)((c->nc + warps - 1) / warps), 32 * warps, smem, c->stream>>>(P);
  HOFV_CUDA(c, cudaGetLastError());
  unsigned long long bits = 0;
  int status = 0;
  HOFV_CUDA(c, cudaMemcpyAsync(&bits, d_cond, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  HOFV_CUDA(c, cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  cudaFree(d_cond);
  cudaFree(d_status);
  double cond;
  memcpy(&cond, &bits, sizeof(double));
  c->max_cond = cond;
  if (status)
    return fail(c, HOFV_EILLCOND,
                "singular least-squares reconstruction (degenerate stencil); a larger n_plus "
                "(the paper suggests 20 instead of 10 in 2-D) may help");
  return 0;
}

// ---------------------------------------------------------------------
// per-face data of the residual and the compact approximate Jacobian
// (Kbar = 1): fstar (u* slots of both sides), fstab = Gamma / |d . n|,
// and per cell the ELL row of the AJ.
// ---------------------------------------------------------------------
__global__ void k_face_aux(int dim, int nlf, int64_t nfid, int64_t nfi,
                           const int32_t* __restrict__ fown, const int32_t* __restrict__ fnei,
                           const int32_t* __restrict__ cface, const double* __restrict__ xc,
                           const double* __restrict__ xf, const double* __restrict__ nrm,
                           const double* __restrict__ gam, int32_t* fstar, double* fstab) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nfid) return;
  const int32_t P = fown[f];
  int lfP = -1, lfN = -1;
  for (int lf = 0; lf < nlf; ++lf)
    if (cface[(int64_t)P * nlf + lf] == (int32_t)(f + 1)) lfP = lf;
  double dv[3] = {0, 0, 0};
  if (f < nfi) {
    const int32_t N = fnei[f];
    for (int lf = 0; lf < nlf; ++lf)
      if (cface[(int64_t)N * nlf + lf] == -(int32_t)(f + 1)) lfN = lf;
    for (int a = 0; a < dim; ++a) dv[a] = xc[3 * (int64_t)N + a] - xc[3 * (int64_t)P + a];
    fstar[2 * f + 1] = N * nlf + lfN;
  } else {
    for (int a = 0; a < dim; ++a) dv[a] = xf[3 * f + a] - xc[3 * (int64_t)P + a];
    fstar[2 * f + 1] = -1;
  }
  fstar[2 * f] = P * nlf + lfP;
  double dn = 0.0;
  for (int a = 0; a < dim; ++a) dn += dv[a] * nrm[3 * f + a];
  fstab[f] = gam[f] / fabs(dn);
}

__global__ void k_aj_rows(int nlf, int64_t nc, const int32_t* __restrict__ cface,
                          const int32_t* __restrict__ fown, const int32_t* __restrict__ fnei,
                          int64_t nfi, const double* __restrict__ fstab, double* diag,
                          int32_t* col, double* off, float* diag32, float* off32, double* invd,
                          float* invd32) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double dg = 0.0;
  for (int lf = 0; lf < nlf; ++lf) {
    const int32_t code = cface[c * nlf + lf];
    int32_t cc = -1;
    double o = 0.0;
    if (code != 0) {
      const int64_t f = (code > 0 ? code : -code) - 1;
      const double a = fstab[f];
      dg -= a;
      if (f < nfi) {
        cc = code > 0 ? fnei[f] : fown[f];
        o = a;
      }
    }
    col[c * nlf + lf] = cc;
    off[c * nlf + lf] = o;
    off32[c * nlf + lf] = (float)o;
  }
  diag[c] = dg;
  diag32[c] = (float)dg;
  invd[c] = -1.0 / dg;
  invd32[c] = (float)(-1.0 / dg);
}

int run_cell_mass(hofv_ctx* c) {
  LsqParams P = lsq_params(c);
  const int warps = 4;
  const size_t smem = sizeof(double) * warps * (P.Nt * P.NR + 2 * kMaxNt);
  HOFV_CUDA(c, cudaFuncSetAttribute(k_lsq_cell_mass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  k_lsq_cell_mass<<<(unsigned)((c->nc + warps - 1) / warps), 32 * warps, smem, c->stream>>>(P);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

// inertia on the approximate Jacobian's diagonal: -rho Omega c2 / Kbar
// (the operator is stored with Kbar = 1)
__global__ void k_aj_mass(int64_t nc, const double* __restrict__ mscale, double inv_kbar,
                          double* diag, float* diag32, double* invd, float* invd32) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double dg = diag[c] + mscale[c] * inv_kbar;
  diag[c] = dg;
  diag32[c] = (float)dg;
  invd[c] = -1.0 / dg;
  invd32[c] = (float)(-1.0 / dg);
}

int run_face_aux(hofv_ctx* c) {
  const int T = 128;
  if (c->nfid > 0) {
    k_face_aux<<<(unsigned)((c->nfid + T - 1) / T), T, 0, c->stream>>>(
        c->dim, c->nlf, c->nfid, c->nfi, c->d_fown, c->d_fnei, c->d_cface, c->d_xc, c->d_xf,
        c->d_nrm, c->d_gam, c->d_fstar, c->d_fstab);
    HOFV_CUDA(c, cudaGetLastError());
  }
  return run_aj_rows(c);
}

int run_aj_rows(hofv_ctx* c) {
  const int T = 128;
  k_aj_rows<<<(unsigned)((c->nc + T - 1) / T), T, 0, c->stream>>>(
      c->nlf, c->nc, c->d_cface, c->d_fown, c->d_fnei, c->nfi, c->d_fstab, c->d_aj_diag,
      c->d_aj_col, c->d_aj_off, c->d_aj_diag32, c->d_aj_off32, c->d_aj_invd, c->d_aj_invd32);
  HOFV_CUDA(c, cudaGetLastError());
  if (c->inertia && c->have_mat) {
    k_aj_mass<<<(unsigned)((c->nc + T - 1) / T), T, 0, c->stream>>>(
        c->nc, c->d_mscale, 1.0 / c->mat.kbar, c->d_aj_diag, c->d_aj_diag32, c->d_aj_invd,
        c->d_aj_invd32);
    HOFV_CUDA(c, cudaGetLastError());
  }
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

}  // namespace hofv
