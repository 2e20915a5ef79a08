// nej.cu -- the near-exact Jacobian preconditioner (App. "Preconditioner
// Based on Near-exact Jacobian"), linear-elastic law only.
//
// The near-exact Jacobian (NEJ) is the Jacobian of the face fluxes without
// the stabilisation term.  With Hooke's law the flux of a face is linear in
// its stencil values, flux_f = sum_N T_{f,N} u_N + ghost terms, where T are
// the contracted d x d matrices of the linear form (one per face and stencil
// cell); the ghost-node contributions of displacement faces are constants
// and go to the right-hand side, traction faces contribute nothing.  Row P
// of the NEJ is therefore sum over P's faces of +-T_{f,N}, a block row whose
// columns are the union of the face stencils of P.
//
// Storage: block CSR with d x d FP32 blocks (assembled in FP64 in a fixed
// face order, one warp per row: deterministic), columns sorted per row.  The
// preconditioner applies NEJ^-1 approximately by `inner` iterations of GMRES
// right-preconditioned by one multigrid V-cycle of the compact approximate
// Jacobian; the outer flexible GMRES absorbs the inexactness.
#include <math.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "hofv_internal.cuh"

namespace hofv {

namespace {

struct Nej {
  uint64_t gen = 0;            // context generation the values belong to
  int64_t nnzb = 0;
  int32_t* rp = nullptr;       // [nc + 1]
  int32_t* col = nullptr;      // [nnzb]
  float* val = nullptr;        // [nnzb][d][d]
  // inner GMRES storage
  int kmax = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *h = nullptr, *y = nullptr;
  std::vector<void*> mem;
};

Nej* get(hofv_ctx* c) { return static_cast<Nej*>(c->nej); }

template <typename T>
int nalloc(hofv_ctx* c, Nej* g, T** p, size_t count) {
  if (dev_alloc(c, p, std::max<size_t>(count, 1))) return HOFV_ENOMEM;
  g->mem.push_back(*p);
  return 0;
}

#define NEJ_TRY(x)             \
  do {                         \
    const int rc_ = (x);       \
    if (rc_ != 0) return rc_;  \
  } while (0)

// Row P accumulates sign * T_{f,N} of each of its faces, faces in local
// order; within a face the stencil cells are distinct, so the lanes of the
// warp never add into the same block at once.
template <int DIM>
__global__ void k_nej_assemble(int64_t nc, int nlf, int S, const int32_t* __restrict__ cface,
                               int64_t nfid, const int32_t* __restrict__ fst,
                               const double* __restrict__ tco, const int32_t* __restrict__ rp,
                               const int32_t* __restrict__ col, double* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t P = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (P >= nc) return;
  const int32_t r0 = rp[P], r1 = rp[P + 1];
  for (int lf = 0; lf < nlf; ++lf) {
    const int32_t code = cface[P * nlf + lf];
    if (code == 0) continue;
    const int64_t f = (code > 0 ? code : -code) - 1;
    if (f >= nfid) continue;
    const double sgn = code > 0 ? 1.0 : -1.0;
    const int64_t tile = f / kTile, fi = f % kTile;
    for (int n = lane; n < S; n += 32) {
      const int64_t e = (tile * S + n) * kTile + fi;
      const int32_t N = fst[e];
      int32_t lo = r0, hi = r1 - 1;
      while (lo < hi) {  // the column is present: built from the same stencils
        const int32_t mid = (lo + hi) >> 1;
        if (col[mid] < N) lo = mid + 1; else hi = mid;
      }
      const double* T = tco + e * DIM * DIM;
      double* B = val + (int64_t)lo * DIM * DIM;
#pragma unroll
      for (int q = 0; q < DIM * DIM; ++q) B[q] += sgn * T[q];
    }
    __syncwarp();
  }
}

__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// y = NEJ x, one warp per block row, FP32 blocks, FP64 vectors
template <int DIM>
__global__ void k_nej_spmv(int64_t nc, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const float* __restrict__ val,
                           const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t P = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; P < nc; P += nw) {
    float s[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) s[i] = 0.0f;
    for (int32_t k = rp[P] + lane; k < rp[P + 1]; k += 32) {
      const int32_t N = col[k];
      float xn[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) xn[j] = (float)x[j * nc + N];
      const float* B = val + (int64_t)k * DIM * DIM;
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) s[i] = fmaf(B[i * DIM + j], xn[j], s[i]);
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i)
      for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < DIM; ++i) y[i * nc + P] = (double)s[i];
    }
  }
}

unsigned warps_grid(int64_t rows) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, 16384));
}

// column structure: the union of the face stencils of every cell, sorted
int build_structure(hofv_ctx* c, Nej* g) {
  const int64_t nc = c->nc, nfid = c->nfid;
  const int S = c->S, nlf = c->nlf;
  std::vector<int32_t> fst((size_t)c->nftile * S * kTile);
  HOFV_CUDA(c, cudaMemcpy(fst.data(), c->d_fst, sizeof(int32_t) * fst.size(),
                          cudaMemcpyDeviceToHost));
  auto stencil = [&](int64_t f, int n) {
    return fst[((f / kTile) * S + n) * kTile + f % kTile];
  };
  const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::vector<int32_t>> cols(nth);
  std::vector<std::vector<int32_t>> len(nth);
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) {
    pool.emplace_back([&, t]() {
      const int64_t a = nc * t / nth, b = nc * (t + 1) / nth;
      std::vector<int32_t> row;
      for (int64_t P = a; P < b; ++P) {
        row.clear();
        for (int lf = 0; lf < nlf; ++lf) {
          const int64_t f = c->cf[P * nlf + lf];
          if (f < 0 || f >= nfid) continue;
          for (int n = 0; n < S; ++n) row.push_back(stencil(f, n));
        }
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        len[t].push_back((int32_t)row.size());
        cols[t].insert(cols[t].end(), row.begin(), row.end());
      }
    });
  }
  for (auto& th : pool) th.join();
  std::vector<int32_t> rp(nc + 1, 0), col;
  int64_t k = 0, total = 0;
  for (int t = 0; t < nth; ++t) total += (int64_t)cols[t].size();
  if (total >= INT32_MAX) return fail(c, HOFV_EINVAL, "near-exact Jacobian too large");
  col.reserve(total);
  for (int t = 0; t < nth; ++t) {
    for (int32_t l : len[t]) {
      rp[k + 1] = rp[k] + l;
      ++k;
    }
    col.insert(col.end(), cols[t].begin(), cols[t].end());
  }
  g->nnzb = total;
  NEJ_TRY(nalloc(c, g, &g->rp, rp.size()));
  NEJ_TRY(nalloc(c, g, &g->col, col.size()));
  HOFV_CUDA(c, cudaMemcpy(g->rp, rp.data(), sizeof(int32_t) * rp.size(), cudaMemcpyHostToDevice));
  HOFV_CUDA(c, cudaMemcpy(g->col, col.data(), sizeof(int32_t) * col.size(),
                          cudaMemcpyHostToDevice));
  NEJ_TRY(nalloc(c, g, &g->val, (size_t)total * c->dim * c->dim));
  return 0;
}

int assemble(hofv_ctx* c, Nej* g) {
  const int d = c->dim;
  const size_t nv = (size_t)g->nnzb * d * d;
  double* v64 = nullptr;
  NEJ_TRY(dev_alloc(c, &v64, nv));
  HOFV_CUDA(c, cudaMemsetAsync(v64, 0, sizeof(double) * nv, c->stream));
  const unsigned grid = (unsigned)((c->nc * 32 + 255) / 256);
  if (d == 2)
    k_nej_assemble<2><<<grid, 256, 0, c->stream>>>(c->nc, c->nlf, c->S, c->d_cface, c->nfid,
                                                   c->d_fst, c->d_tco, g->rp, g->col, v64);
  else
    k_nej_assemble<3><<<grid, 256, 0, c->stream>>>(c->nc, c->nlf, c->S, c->d_cface, c->nfid,
                                                   c->d_fst, c->d_tco, g->rp, g->col, v64);
  k_to_float<<<(unsigned)std::min<size_t>((nv + 255) / 256, 65535), 256, 0, c->stream>>>(
      (int64_t)nv, v64, g->val);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  dev_free(c, v64);
  g->gen = c->gen;
  return 0;
}

int ensure_inner(hofv_ctx* c, Nej* g, int k) {
  if (g->kmax >= k) return 0;
  const int64_t n = c->nc * c->dim;
  for (void* p : {(void*)g->V, (void*)g->Z, (void*)g->w, (void*)g->h, (void*)g->y}) {
    if (!p) continue;
    g->mem.erase(std::remove(g->mem.begin(), g->mem.end(), p), g->mem.end());
    dev_free(c, p);
  }
  NEJ_TRY(nalloc(c, g, &g->V, (size_t)(k + 1) * n));
  NEJ_TRY(nalloc(c, g, &g->Z, (size_t)k * n));
  NEJ_TRY(nalloc(c, g, &g->w, (size_t)n));
  NEJ_TRY(nalloc(c, g, &g->h, (size_t)2 * (k + 2) + 8));
  NEJ_TRY(nalloc(c, g, &g->y, (size_t)k + 1));
  g->kmax = k;
  return 0;
}

}  // namespace

int nej_ensure(hofv_ctx* c) {
  if (c->mat.law != HOFV_LAW_LINEAR)
    return fail(c, HOFV_ENOTSUP, "the near-exact Jacobian is built for the linear-elastic law");
  if (c->nfy > 0)
    return fail(c, HOFV_ENOTSUP, "the near-exact Jacobian does not take symmetry faces");
  NEJ_TRY(ensure_tco(c));
  Nej* g = get(c);
  if (!g) {
    g = new Nej();
    const int rc = build_structure(c, g);
    if (rc) {
      for (void* p : g->mem) dev_free(c, p);
      delete g;
      return rc;
    }
    c->nej = g;
    g->gen = 0;
  }
  if (g->gen != c->gen) NEJ_TRY(assemble(c, g));
  return 0;
}

int nej_apply(hofv_ctx* c, const double* x, double* y) {
  NEJ_TRY(nej_ensure(c));
  Nej* g = get(c);
  if (c->dim == 2)
    k_nej_spmv<2><<<warps_grid(c->nc), 256, 0, c->stream>>>(c->nc, g->rp, g->col, g->val, x, y);
  else
    k_nej_spmv<3><<<warps_grid(c->nc), 256, 0, c->stream>>>(c->nc, g->rp, g->col, g->val, x, y);
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

// z ~= NEJ^-1 v: `iters` GMRES iterations from z = 0, right-preconditioned
// by one multigrid V-cycle of the approximate Jacobian, classical
// Gram-Schmidt twice, Givens rotations on the host.
int nej_prepare(hofv_ctx* c, int iters) {
  NEJ_TRY(nej_ensure(c));
  return ensure_inner(c, get(c), std::max(1, std::min(iters, 30)));
}

int nej_precondition(hofv_ctx* c, int iters, const double* v, double* z) {
  NEJ_TRY(nej_ensure(c));
  NEJ_TRY(mg_ensure(c));
  Nej* g = get(c);
  const int k = std::max(1, std::min(iters, 30));
  NEJ_TRY(ensure_inner(c, g, k));
  const int64_t n = c->nc * c->dim;
  cudaStream_t st = c->stream;
  double* h = g->h;                 // [0, k+2): dots, [k+2, 2k+4): second pass, then norms
  double* nrm = g->h + 2 * (k + 2);
  launch_norm2(v, n, c->d_red, c->d_count, nrm, c->red_blocks, st);
  double beta = 0.0;
  HOFV_CUDA(c, cudaMemcpyAsync(&beta, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
  HOFV_CUDA(c, cudaStreamSynchronize(st));
  HOFV_CUDA(c, cudaMemsetAsync(z, 0, sizeof(double) * n, st));
  if (!(beta > 0.0)) return std::isfinite(beta) ? 0 : fail(c, HOFV_ENAN, "non-finite vector");
  launch_scale_copy(g->V, v, nrm, 1, n, st);
  std::vector<double> H((size_t)(k + 1) * k, 0.0), cs(k), sn(k), gv(k + 1, 0.0), hb(2 * (k + 2) + 2);
  gv[0] = beta;
  int j = 0;
  for (; j < k; ++j) {
    double* Vj = g->V + (int64_t)j * n;
    double* Zj = g->Z + (int64_t)j * n;
    NEJ_TRY(mg_precondition(c, 1, Vj, Zj));
    NEJ_TRY(nej_apply(c, Zj, g->w));
    launch_dots(g->V, n, g->w, j + 1, n, c->d_red, c->d_count, h, c->red_blocks, st, 0);
    launch_multi_axpy(g->w, g->V, h, j + 1, n, n, st);
    launch_dots(g->V, n, g->w, j + 1, n, c->d_red, c->d_count, h + (k + 2), c->red_blocks, st, 0);
    launch_multi_axpy(g->w, g->V, h + (k + 2), j + 1, n, n, st);
    launch_norm2(g->w, n, c->d_red, c->d_count, nrm + 1, c->red_blocks, st);
    HOFV_CUDA(c, cudaMemcpyAsync(hb.data(), h, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, st));
    HOFV_CUDA(c, cudaStreamSynchronize(st));
    const double hn = hb[2 * (k + 2) + 1];
    if (!std::isfinite(hn)) return fail(c, HOFV_ENAN, "non-finite value in the near-exact solve");
    double* Hc = H.data() + (size_t)j * (k + 1);
    for (int i = 0; i <= j; ++i) Hc[i] = hb[i] + hb[(k + 2) + i];
    Hc[j + 1] = hn;
    if (hn > 0.0 && j + 1 < k) launch_scale_copy(g->V + (int64_t)(j + 1) * n, g->w, nrm + 1, 1, n, st);
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * Hc[i] + sn[i] * Hc[i + 1];
      Hc[i + 1] = -sn[i] * Hc[i] + cs[i] * Hc[i + 1];
      Hc[i] = t;
    }
    const double den = hypot(Hc[j], Hc[j + 1]);
    cs[j] = den > 0 ? Hc[j] / den : 1.0;
    sn[j] = den > 0 ? Hc[j + 1] / den : 0.0;
    Hc[j] = den;
    Hc[j + 1] = 0.0;
    gv[j + 1] = -sn[j] * gv[j];
    gv[j] = cs[j] * gv[j];
    if (hn == 0.0) {
      ++j;
      break;
    }
  }
  // back substitution, z = Z y
  std::vector<double> y(j, 0.0);
  for (int i = j - 1; i >= 0; --i) {
    double s = gv[i];
    for (int l = i + 1; l < j; ++l) s -= H[(size_t)l * (k + 1) + i] * y[l];
    const double d = H[(size_t)i * (k + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
  HOFV_CUDA(c, cudaMemcpyAsync(g->y, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
  launch_combine(z, g->Z, g->y, j, n, n, st);
  HOFV_CUDA(c, cudaStreamSynchronize(st));  // y lives on the host stack
  return 0;
}

void nej_release(hofv_ctx* c) {
  delete get(c);
  c->nej = nullptr;
}

}  // namespace hofv
