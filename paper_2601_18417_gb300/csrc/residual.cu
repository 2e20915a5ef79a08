// residual.cu -- the matrix-free residual R(u) of the high-order
// cell-centred finite-volume scheme (arXiv 2601.18417):
//
//   k_ustar : cell-ordered; extrapolated face values of the alpha
//             stabilisation, u*_{f,P} = u_P + sum_N e_N u_N (eq. alphaJump,
//             App. B, with the Taylor terms folded into e at set-up)
//   k_flux  : face-ordered, 32 faces per tile; (1) displacement gradient at
//             every Gauss point, grad u = sum_N c_N (x) u_N (+ ghost node,
//             eq. faceQuadGrad), (2) the law (App. A) and traction T a_q,
//             (3) Gauss quadrature over the face plus the stabilisation
//             traction alpha Kbar / |d.n| (u*_N - u*_P) Gamma (eq. alpha)
//   k_cell  : cell-ordered, fixed face order (no atomics):
//             R_P = sum_f +-flux_f + source_P (eq. divStressDiscret +
//             eq. bodyTerm); optional epilogue (R - R0) / eps for Jv.
//   k_tflux : the linear law in contracted form, flux_f = sum_N T_N u_N
//             (replaces k_flux when enabled)
//   k_extend, k_sym_other : symmetry faces (reflected ghost values, mirrored
//             stabilisation value), only when the mesh has symmetry faces
//   k_cell_avg : inertia term of the BDF2 dynamics, only when enabled
//
// All arithmetic is FP64.  Every FP64 instruction of the gradient phase runs
// with all 32 lanes busy: a tile's (face, row) pairs are laid out so that
// consecutive threads own consecutive coefficient rows.
#include <algorithm>
#include <type_traits>

#include "hofv_internal.cuh"

namespace hofv {

// ---------------------------------------------------------------------
// stabilisation extrapolation: one thread per (cell, local face)
// ---------------------------------------------------------------------
// NLF = faces per cell: 4 / 6 for quads / hexes, 3 / 4 for triangles / tetrahedra
template <int DIM, int NLF>
__global__ void __launch_bounds__(32 * NLF)
    k_ustar(DevMesh m, const double* __restrict__ w, double* __restrict__ ustar) {
  const int64_t tile = blockIdx.x;
  const int it = threadIdx.x;            // ci * NLF + lf
  const int ci = it / NLF;
  const int64_t cell = tile * kTile + ci;
  const int32_t* __restrict__ st = m.cst + tile * m.S * kTile + ci;
  const double* __restrict__ ex = m.cex + tile * (int64_t)m.S * kTile * NLF + it;
  double acc[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) acc[j] = 0.0;
  const int64_t ws = m.wst;  // stride of the state read
#pragma unroll 4
  for (int n = 0; n < m.S; ++n) {
    const int32_t id = __ldg(st + n * kTile);
    const double e = __ldg(ex + (int64_t)n * kTile * NLF);
#pragma unroll
    for (int j = 0; j < DIM; ++j) acc[j] = fma(e, __ldg(w + j * ws + id), acc[j]);
  }
  if (cell < m.nc) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) ustar[(cell * NLF + (it % NLF)) * DIM + j] = w[j * ws + cell] + acc[j];
  }
}

// ---------------------------------------------------------------------
// inertia: cell average of the cell fit over the cell's Gauss points,
// ubar_P = u_P + sum_N cmass_N u_N (eq. inertiaTerm with the Taylor
// extrapolation of eq. alphaJump; u_P alone for one point per cell), and,
// scaled, the u-dependent part -rho Omega_P c2 ubar_P of the BDF2 term
// ---------------------------------------------------------------------
template <int DIM, bool SCALE>
__global__ void k_cell_avg(DevMesh m, const double* __restrict__ w, int64_t ws,
                           double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int64_t nc = m.nc;
  double acc[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) acc[j] = w[j * ws + c];
  if (m.cmass) {
    const int64_t tile = c / kTile, ci = c % kTile;
    const int32_t* __restrict__ st = m.cst + tile * m.S * kTile + ci;
    const double* __restrict__ e = m.cmass + tile * m.S * kTile + ci;
    for (int n = 0; n < m.S; ++n) {
      const int32_t id = __ldg(st + n * kTile);
      const double en = __ldg(e + n * kTile);
#pragma unroll
      for (int j = 0; j < DIM; ++j) acc[j] = fma(en, __ldg(w + j * ws + id), acc[j]);
    }
  }
  const double sc = SCALE ? m.mscale[c] : 1.0;
#pragma unroll
  for (int j = 0; j < DIM; ++j) out[j * nc + c] = SCALE ? sc * acc[j] : acc[j];
}

void launch_cell_average(const DevMesh& m, const double* u, double* ubar, cudaStream_t st) {
  const unsigned g = (unsigned)((m.nc + 127) / 128);
  if (m.dim == 2)
    k_cell_avg<2, false><<<g, 128, 0, st>>>(m, u, m.nc, ubar);
  else
    k_cell_avg<3, false><<<g, 128, 0, st>>>(m, u, m.nc, ubar);
}

__global__ void k_combine4(int64_t n, double a, const double* __restrict__ x, double b,
                           const double* __restrict__ y, double g, const double* __restrict__ z,
                           double e, const double* __restrict__ w, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (x) s += a * x[i];
    if (y) s += b * y[i];
    if (z) s += g * z[i];
    if (w) s += e * w[i];
    out[i] = s;
  }
}

void launch_combine4(int64_t n, double a, const double* x, double b, const double* y, double g,
                     const double* z, double e, const double* w, double* out, cudaStream_t st) {
  k_combine4<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(n, a, x, b, y, g,
                                                                                 z, e, w, out);
}

__global__ void k_scale_rows(int dim, int64_t nc, const double* __restrict__ s, double* out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int j = 0; j < dim; ++j) out[j * nc + c] *= s[c];
}

void launch_scale_rows(int dim, int64_t nc, const double* s, double* out, cudaStream_t st) {
  k_scale_rows<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(dim, nc, s, out);
}

// ---------------------------------------------------------------------
// laws: traction t = T a from G[i][j] = du_j/dx_i
// ---------------------------------------------------------------------
template <int DIM, int LAW>
__device__ __forceinline__ void traction(const double (&G)[3][3], const double* a, const Material& mt,
                                         double* t) {
  if (LAW == HOFV_LAW_LINEAR) {
    // sigma = mu (G + G^T) + lambda tr(G) I, eq. (linearElastic)
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) tr += G[i][i];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      double s = mt.lam * tr * a[i];
#pragma unroll
      for (int j = 0; j < DIM; ++j) s = fma(mt.mu * (G[i][j] + G[j][i]), a[j], s);
      t[i] = s;
    }
  } else {
    // neo-Hookean, eq. (neoHook), first Piola-Kirchhoff P = J sigma F^{-T}
    // (eq. nanson).  With B = F F^T, w = cof(F) a and r = J^{-1/3}:
    //   J sigma = mu J^{-2/3} (B - tr(B)/3 I) + kappa/2 (J^2 - 1) I,
    //   t = P a = J sigma w / J = alpha B w + beta w,
    //   alpha = mu r^5,  beta = kappa/2 (J^2 - 1) r^3 - alpha tr(B) / 3,
    // and since F^T cof(F) = J I, B w = F (F^T w) = J F a.
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = (i == j ? 1.0 : 0.0) + G[j][i];
    double C[3][3];  // cofactor matrix
    C[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    C[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    C[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    C[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    C[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    C[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    C[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    C[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    C[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    const double J = F[0][0] * C[0][0] + F[0][1] * C[0][1] + F[0][2] * C[0][2];
    // J^{-1/3}; not defined for J <= 0 (an inverted element): NaN, so the
    // caller's finiteness checks reject the state
    const double r = inv_cbrt(J);
    const double r3 = r * r * r;
    const double alpha = mt.mu * (r * r) * r3;
    double trB = 0.0;  // tr(F F^T): the squares of F's entries
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) trB = fma(F[i][j], F[i][j], trB);
    const double beta = 0.5 * mt.kappa * fma(J, J, -1.0) * r3 - alpha * trB * (1.0 / 3.0);
    const double aJ = alpha * J;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      double wi = 0.0, fa = 0.0;
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        wi = fma(C[i][l], a[l], wi);
        fa = fma(F[i][l], a[l], fa);
      }
      t[i] = fma(aJ, fa, beta * wi);
    }
  }
}

// ---------------------------------------------------------------------
// face fluxes, one tile of 32 faces per block, blockDim = 32 * R
// ---------------------------------------------------------------------
template <int DIM, int LAW>
__global__ void __launch_bounds__(DIM == 3 ? 864 : 256)
    k_flux(DevMesh m, Material mt, const double* __restrict__ w, const double* __restrict__ ustar,
           const double* __restrict__ ubq, const double* __restrict__ ubf,
           double* __restrict__ flux) {
  extern __shared__ double sm[];
  const int R = m.R, Q = m.Q, S = m.S;
  double* Gs = sm;                        // [32][R][DIM]
  double* Ts = sm + kTile * R * DIM;      // [32][Q][DIM]
  const int64_t tile = blockIdx.x;
  const int it = threadIdx.x;
  const int64_t nc = m.wst;  // stride of the state read
  // (1) gradient rows: thread (fi, r) accumulates sum_N c_{r,N} u_N
  {
    const int fi = it / R, r = it % R;
    const int64_t f = tile * kTile + fi;
    const int32_t* __restrict__ st = m.fst + tile * S * kTile + fi;
    const double* __restrict__ co = m.fco + tile * (int64_t)S * kTile * R + it;
    double acc[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) acc[j] = 0.0;
    // rows of points without area (polyhedral fan slots past a face's last
    // corner) are neither read nor formed
    const bool live = m.fql == nullptr || r < __ldg(m.fql + f) * DIM;
#pragma unroll 4
    for (int n = 0; n < (live ? S : 0); ++n) {
      const int32_t id = __ldg(st + n * kTile);
      const double c = __ldg(co + (int64_t)n * kTile * R);
#pragma unroll
      for (int j = 0; j < DIM; ++j) acc[j] = fma(c, __ldg(w + j * nc + id), acc[j]);
    }
    if (live && f >= m.nfi && f < m.nfid) {  // ghost node of a displacement face
      const int64_t fd = f - m.nfi;
      const double cg = m.gco[fd * R + r];
      const int q = r / DIM;
#pragma unroll
      for (int j = 0; j < DIM; ++j) acc[j] = fma(cg, ubq[(fd * Q + q) * DIM + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) Gs[(fi * R + r) * DIM + j] = acc[j];
  }
  __syncthreads();
  // (2) law and traction at each Gauss point
  if (it < kTile * Q) {
    const int fi = it / Q, q = it % Q;
    const int64_t f = tile * kTile + fi;
    double t[DIM];
    if (f < m.nfid) {
      double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) G[i][j] = Gs[(fi * R + q * DIM + i) * DIM + j];
      double a[3];
#pragma unroll
      for (int k = 0; k < DIM; ++k) a[k] = m.aq[(f * Q + q) * 3 + k];
      traction<DIM, LAW>(G, a, mt, t);
    } else {
#pragma unroll
      for (int i = 0; i < DIM; ++i) t[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) Ts[(fi * Q + q) * DIM + i] = t[i];
  }
  __syncthreads();
  // (3) quadrature over the face + alpha stabilisation
  if (it < kTile * DIM) {
    const int fi = it / DIM, i = it % DIM;
    const int64_t f = tile * kTile + fi;
    if (f < m.nfid) {
      double s = 0.0;
      for (int q = 0; q < Q; ++q) s += Ts[(fi * Q + q) * DIM + i];
      const int32_t sp = m.fstar[2 * f], sn = m.fstar[2 * f + 1];
      const double other = sn >= 0 ? ustar[(int64_t)sn * DIM + i] : ubf[(f - m.nfi) * DIM + i];
      const double coef = mt.alpha * mt.kbar * m.fstab[f];
      flux[f * DIM + i] = fma(coef, other - ustar[(int64_t)sp * DIM + i], s);
    }
  }
}

// ---------------------------------------------------------------------
// the same three phases for faces with more points than one thread per
// (face, row) of a 32-face tile allows (polyhedral faces: up to 8 fan
// triangles of q^2 points, R up to 96): kWideThreads threads walk the rows
// and points of the tile in strides
// ---------------------------------------------------------------------
constexpr int kWideThreads = 512;

template <int DIM, int LAW>
__global__ void __launch_bounds__(kWideThreads)
    k_flux_wide(DevMesh m, Material mt, const double* __restrict__ w,
                const double* __restrict__ ustar, const double* __restrict__ ubq,
                const double* __restrict__ ubf, double* __restrict__ flux) {
  extern __shared__ double sm[];
  const int R = m.R, Q = m.Q, S = m.S;
  double* Gs = sm;                        // [32][R][DIM]
  double* Ts = sm + kTile * R * DIM;      // [32][Q][DIM]
  const int64_t tile = blockIdx.x;
  const int64_t nc = m.wst;
  for (int it = threadIdx.x; it < kTile * R; it += blockDim.x) {
    const int fi = it / R, r = it % R;
    const int64_t f = tile * kTile + fi;
    const int32_t* __restrict__ st = m.fst + tile * S * kTile + fi;
    const double* __restrict__ co = m.fco + tile * (int64_t)S * kTile * R + it;
    double acc[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) acc[j] = 0.0;
    // rows of points without area (polyhedral fan slots past a face's last
    // corner) are neither read nor formed
    const bool live = m.fql == nullptr || r < __ldg(m.fql + f) * DIM;
#pragma unroll 4
    for (int n = 0; n < (live ? S : 0); ++n) {
      const int32_t id = __ldg(st + n * kTile);
      const double c = __ldg(co + (int64_t)n * kTile * R);
#pragma unroll
      for (int j = 0; j < DIM; ++j) acc[j] = fma(c, __ldg(w + j * nc + id), acc[j]);
    }
    if (live && f >= m.nfi && f < m.nfid) {
      const int64_t fd = f - m.nfi;
      const double cg = m.gco[fd * R + r];
      const int q = r / DIM;
#pragma unroll
      for (int j = 0; j < DIM; ++j) acc[j] = fma(cg, ubq[(fd * Q + q) * DIM + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) Gs[(fi * R + r) * DIM + j] = acc[j];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < kTile * Q; it += blockDim.x) {
    const int fi = it / Q, q = it % Q;
    const int64_t f = tile * kTile + fi;
    double t[DIM];
    if (f < m.nfid) {
      double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) G[i][j] = Gs[(fi * R + q * DIM + i) * DIM + j];
      double a[3];
#pragma unroll
      for (int k = 0; k < DIM; ++k) a[k] = m.aq[(f * Q + q) * 3 + k];
      traction<DIM, LAW>(G, a, mt, t);
    } else {
#pragma unroll
      for (int i = 0; i < DIM; ++i) t[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) Ts[(fi * Q + q) * DIM + i] = t[i];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < kTile * DIM; it += blockDim.x) {
    const int fi = it / DIM, i = it % DIM;
    const int64_t f = tile * kTile + fi;
    if (f < m.nfid) {
      double s = 0.0;
      for (int q = 0; q < Q; ++q) s += Ts[(fi * Q + q) * DIM + i];
      const int32_t sp = m.fstar[2 * f], sn = m.fstar[2 * f + 1];
      const double other = sn >= 0 ? ustar[(int64_t)sn * DIM + i] : ubf[(f - m.nfi) * DIM + i];
      const double coef = mt.alpha * mt.kbar * m.fstab[f];
      flux[f * DIM + i] = fma(coef, other - ustar[(int64_t)sp * DIM + i], s);
    }
  }
}

// dynamic shared memory of k_flux_wide beyond the default 48 KB, raised to
// what the largest polyhedral face (8 fan slots of 2 x 2 points) needs, so
// that contexts of different point counts never lower it for one another;
// set for both laws before the first launch or capture
int flux_wide_prepare() {
  constexpr int kMaxWideQ = kPolyFaceMaxCorners * 4;
  const int smem = (int)(sizeof(double) * kTile * (kMaxWideQ * 3 * 3 + kMaxWideQ * 3));
  if (cudaFuncSetAttribute(k_flux_wide<3, HOFV_LAW_LINEAR>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_flux_wide<3, HOFV_LAW_NEOHOOKEAN>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return -1;
  return 0;
}

// ---------------------------------------------------------------------
// cell assembly; out = R, or (R - R0) * inv_eps when R0 != nullptr
// ---------------------------------------------------------------------
template <int DIM, int NLF>
__global__ void k_cell(DevMesh m, const double* __restrict__ flux, const double* __restrict__ src,
                       const double* __restrict__ R0, const double* __restrict__ d_eps,
                       double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  double r[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) r[j] = src ? src[j * m.nc + c] : 0.0;
#pragma unroll
  for (int lf = 0; lf < NLF; ++lf) {
    const int32_t code = m.cface[c * NLF + lf];
    if (code == 0) continue;
    const int64_t f = (code > 0 ? code : -code) - 1;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const double v = flux[f * DIM + j];
      r[j] = code > 0 ? r[j] + v : r[j] - v;
    }
  }
  if (m.mscale) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) r[j] += m.inert[j * m.nc + c];
  }
  if (R0) {
    const double ie = 1.0 / d_eps[0];
#pragma unroll
    for (int j = 0; j < DIM; ++j) out[j * m.nc + c] = (r[j] - R0[j * m.nc + c]) * ie;
  } else {
#pragma unroll
    for (int j = 0; j < DIM; ++j) out[j * m.nc + c] = r[j];
  }
}

template <int DIM>
__global__ void __launch_bounds__(32 * DIM)
    k_tflux(DevMesh m, const double* __restrict__ tco, double alpha_kbar,
            const double* __restrict__ w, const double* __restrict__ ustar,
            const double* __restrict__ ubf, double* __restrict__ flux);

// ---------------------------------------------------------------------
// symmetry faces (Sec. 3.5.3): the state extended by the ghosts' reflected
// values R u_src = u - 2 n (n . u), and, after the stabilisation
// extrapolation, the mirror R u*_P of each symmetry face's own value as the
// value beyond the face (its jump then penalises the normal component only)
// ---------------------------------------------------------------------
template <int DIM>
__global__ void k_extend(DevMesh m, const double* __restrict__ w, double* __restrict__ wext) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = m.nc, ws = m.wst;
  if (i < nc) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) wext[j * ws + i] = w[j * nc + i];
  } else if (i < ws) {
    const int64_t g = i - nc;
    const int32_t src = m.gsrc[g];
    const double* n = m.nrm + 3 * (int64_t)m.gface[g];
    double u[DIM], un = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      u[j] = w[j * nc + src];
      un += n[j] * u[j];
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) wext[j * ws + i] = u[j] - 2.0 * un * n[j];
  }
}

template <int DIM>
__global__ void k_sym_other(DevMesh m, const double* __restrict__ ustar) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= m.nfy) return;
  const int64_t f = m.nfi + m.nfd + b;
  const double* us = ustar + (int64_t)m.fstar[2 * f] * DIM;
  const double* n = m.nrm + 3 * f;
  double un = 0.0;
#pragma unroll
  for (int j = 0; j < DIM; ++j) un += n[j] * us[j];
#pragma unroll
  for (int j = 0; j < DIM; ++j) m.ubfw[(f - m.nfi) * DIM + j] = us[j] - 2.0 * un * n[j];
}

// faces per cell as a compile-time constant: d + 1 (triangles /
// tetrahedra), 2 d (quads / hexes), kPolyMaxSides slots (2-D polygons),
// kPolyhedronMaxFaces slots (3-D polyhedra)
template <int DIM, typename F>
static void by_faces_per_cell(const DevMesh& m, F&& launch) {
  if (m.nlf == DIM + 1)
    launch(std::integral_constant<int, DIM + 1>{});
  else if (m.nlf == 2 * DIM)
    launch(std::integral_constant<int, 2 * DIM>{});
  else if constexpr (DIM == 2)
    launch(std::integral_constant<int, kPolyMaxSides>{});
  else
    launch(std::integral_constant<int, kPolyhedronMaxFaces>{});
}

template <int DIM, int LAW>
static void residual_impl(const DevMesh& m, const Material& mat, const double* w,
                          const double* d_eps, const double* R0, double* out, double* ustar,
                          double* flux, const double* ubq, const double* ubf, const double* src,
                          cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  if (m.ng > 0) {
    k_extend<DIM><<<(unsigned)((m.wst + 255) / 256), 256, 0, st>>>(m, w, m.wext);
    w = m.wext;
  }
  by_faces_per_cell<DIM>(m, [&](auto nlf) {
    constexpr int NLF = decltype(nlf)::value;
    k_ustar<DIM, NLF><<<(unsigned)m.nctile, 32 * NLF, 0, st>>>(m, w, ustar);
  });
  if (m.nfy > 0) k_sym_other<DIM><<<(unsigned)((m.nfy + 127) / 128), 128, 0, st>>>(m, ustar);
  if (ev) cudaEventRecord(ev[1], st);
  if (m.nftile > 0) {
    if (LAW == HOFV_LAW_LINEAR && m.tco) {
      k_tflux<DIM><<<(unsigned)m.nftile, 32 * DIM, 0, st>>>(m, m.tco, mat.alpha * mat.kbar, w,
                                                            ustar, ubf, flux);
    } else {
      const size_t smem = sizeof(double) * kTile * (m.R * DIM + m.Q * DIM);
      if (kTile * m.R <= (DIM == 3 ? 864 : 256)) {
        k_flux<DIM, LAW><<<(unsigned)m.nftile, kTile * m.R, smem, st>>>(m, mat, w, ustar, ubq,
                                                                        ubf, flux);
      } else if constexpr (DIM == 3) {  // set-up admits no wider 2-D face
        k_flux_wide<DIM, LAW><<<(unsigned)m.nftile, kWideThreads, smem, st>>>(m, mat, w, ustar,
                                                                              ubq, ubf, flux);
      }
    }
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (m.mscale)
    k_cell_avg<DIM, true><<<(unsigned)((m.nc + 127) / 128), 128, 0, st>>>(m, w, m.wst, m.inert);
  const unsigned cgrid = (unsigned)((m.nc + 255) / 256);
  by_faces_per_cell<DIM>(m, [&](auto nlf) {
    constexpr int NLF = decltype(nlf)::value;
    k_cell<DIM, NLF><<<cgrid, 256, 0, st>>>(m, flux, src, R0, d_eps, out);
  });
  if (ev) cudaEventRecord(ev[3], st);
}

void launch_residual_df(const DevMesh& m, const Material& mat, const double* w,
                        const double* d_eps, const double* R0, double* out, double* ustar,
                        double* flux, const double* ubq, const double* ubf, const double* src,
                        cudaStream_t st, cudaEvent_t* ev);

void launch_residual(const DevMesh& m, const Material& mat, const double* w, const double* /*v*/,
                     const double* d_eps, const double* R0, double* out, double* ustar,
                     double* flux, const double* ubq, const double* ubf, const double* src,
                     cudaStream_t st, cudaEvent_t* ev) {
  if (m.prec == HOFV_PREC_DF64) {
    launch_residual_df(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
    return;
  }
  if (m.dim == 2) {
    if (mat.law == HOFV_LAW_LINEAR)
      residual_impl<2, 0>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
    else
      residual_impl<2, 1>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
  } else {
    if (mat.law == HOFV_LAW_LINEAR)
      residual_impl<3, 0>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
    else
      residual_impl<3, 1>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
  }
}

// ---------------------------------------------------------------------
// constant source per cell: integrated body force + traction-face fluxes
// sum_q |a_q| T_{b,q} (eq. divStressDiscret, traction term)
// ---------------------------------------------------------------------
__global__ void k_source(int dim, int nlf, int Q, int64_t nc, int64_t nfi, int64_t nfd,
                         const int64_t* __restrict__ cf, const int32_t* __restrict__ ftag,
                         const double* __restrict__ aq, const double* __restrict__ tbq,
                         const double* __restrict__ body, const double* __restrict__ gflux,
                         double* __restrict__ src) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int j = 0; j < dim; ++j) {
    double s = body ? body[j * nc + c] : 0.0;
    if (gflux)
      for (int lf = 0; lf < nlf; ++lf) {
        const int64_t f = cf[c * nlf + lf];  // -1: polygon slot without a face
        if (f >= 0 && ftag[f] == 0) s += gflux[(f - nfi) * dim + j];
      }
    if (tbq) {
      for (int lf = 0; lf < nlf; ++lf) {
        const int64_t f = cf[c * nlf + lf];
        if (f < 0 || ftag[f] != 1) continue;
        const int64_t b = f - nfi - nfd;
        for (int q = 0; q < Q; ++q) {
          const double* a = aq + (f * Q + q) * 3;
          const double mag = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
          s += mag * tbq[(b * Q + q) * dim + j];
        }
      }
    }
    src[j * nc + c] = s;
  }
}

void launch_source(const hofv_ctx* c, cudaStream_t st) {
  k_source<<<(unsigned)((c->nc + 127) / 128), 128, 0, st>>>(
      c->dim, c->nlf, c->Q, c->nc, c->nfi, c->nfd + c->nfy, c->d_cf, c->d_ftag, c->d_aq,
      c->nft > 0 ? c->d_tbq : nullptr, c->d_body,
      (c->contract && c->tco_valid && c->mat.law == HOFV_LAW_LINEAR && c->nfd > 0) ? c->d_gflux
                                                                                  : nullptr,
      c->d_src);
}

}  // namespace hofv

namespace hofv {
// per-cell sum of |flux_f| over the cell's internal and displacement faces
// (the force scale F_s = max over cells), from the last residual's fluxes
template <int DIM, int NLF>
__global__ void k_flux_scale(DevMesh m, const double* __restrict__ flux, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  double s = 0.0;
#pragma unroll
  for (int lf = 0; lf < NLF; ++lf) {
    const int32_t code = m.cface[c * NLF + lf];
    if (code == 0) continue;
    const int64_t f = (code > 0 ? code : -code) - 1;
    double q = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) q += flux[f * DIM + j] * flux[f * DIM + j];
    s += sqrt(q);
  }
  out[c] = s;
}

void launch_flux_scale(const DevMesh& m, const double* flux, double* out, cudaStream_t st) {
  const unsigned grid = (unsigned)((m.nc + 255) / 256);
  if (m.dim == 2 && m.nlf == 3)
    k_flux_scale<2, 3><<<grid, 256, 0, st>>>(m, flux, out);
  else if (m.dim == 2 && m.nlf == kPolyMaxSides)
    k_flux_scale<2, kPolyMaxSides><<<grid, 256, 0, st>>>(m, flux, out);
  else if (m.dim == 2)
    k_flux_scale<2, 4><<<grid, 256, 0, st>>>(m, flux, out);
  else if (m.nlf == 4)
    k_flux_scale<3, 4><<<grid, 256, 0, st>>>(m, flux, out);
  else if (m.nlf == kPolyhedronMaxFaces)
    k_flux_scale<3, kPolyhedronMaxFaces><<<grid, 256, 0, st>>>(m, flux, out);
  else
    k_flux_scale<3, 6><<<grid, 256, 0, st>>>(m, flux, out);
}
}  // namespace hofv

// ---------------------------------------------------------------------
// Linear elasticity with the law and the face quadrature folded into the
// coefficients (an exact re-association of eq. divStressDiscret for Hooke's
// law): with sigma = mu (G + G^T) + lambda tr(G) I and G = sum_N c_N (x) u_N,
//   flux_i = sum_N sum_k T_N[i][k] u_N[k],
//   T_N[i][k] = sum_q mu c_qN,i a_q,k + mu (c_qN . a_q) delta_ik + lambda a_q,i c_qN,k.
// One d x d matrix per face and stencil cell replaces Q d coefficients and
// the per-point law: d^2 FMAs per cell instead of Q d^2.  The ghost node of
// a displacement face only multiplies prescribed data, so its part is a
// constant folded into the cell source.
// ---------------------------------------------------------------------
namespace hofv {

// tco[tile][N][fi][i][k] from fco[tile][N][fi][q*d + i] and aq
template <int DIM>
__global__ void k_build_tco(DevMesh m, double mu, double lam, double* __restrict__ tco) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (tile, N, fi)
  const int64_t total = m.nftile * m.S * kTile;
  if (e >= total) return;
  const int fi = (int)(e % kTile);
  const int64_t tile = e / ((int64_t)m.S * kTile);
  const int64_t f = tile * kTile + fi;
  double T[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int k = 0; k < DIM; ++k) T[i][k] = 0.0;
  if (f < m.nfid) {
    const double* co = m.fco + e * m.R;
    for (int q = 0; q < m.Q; ++q) {
      double c[DIM], a[DIM], ca = 0.0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        if (m.prec == HOFV_PREC_DF64) {  // stored as a double-float pair
          const float2 p = reinterpret_cast<const float2*>(co)[q * DIM + i];
          c[i] = (double)p.x + (double)p.y;
        } else {
          c[i] = co[q * DIM + i];
        }
        a[i] = m.aq[(f * m.Q + q) * 3 + i];
        ca += c[i] * a[i];
      }
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          T[i][k] += mu * c[i] * a[k] + lam * a[i] * c[k] + (i == k ? mu * ca : 0.0);
    }
  }
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int k = 0; k < DIM; ++k) tco[(e * DIM + i) * DIM + k] = T[i][k];
}

// ghost-node flux of each displacement face: sum_q Tg_q u_bq (constant data)
template <int DIM>
__global__ void k_ghost_flux(DevMesh m, double mu, double lam, const double* __restrict__ ubq,
                             double* __restrict__ gflux) {
  const int64_t fd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (fd >= m.nfd) return;
  const int64_t f = m.nfi + fd;
  double out[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) out[i] = 0.0;
  for (int q = 0; q < m.Q; ++q) {
    double c[DIM], a[DIM], u[DIM], ca = 0.0, cu = 0.0, au = 0.0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      c[i] = m.gco[fd * m.R + q * DIM + i];
      a[i] = m.aq[(f * m.Q + q) * 3 + i];
      u[i] = ubq[(fd * m.Q + q) * DIM + i];
      ca += c[i] * a[i];
      cu += c[i] * u[i];
      au += a[i] * u[i];
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) out[i] += mu * c[i] * au + mu * ca * u[i] + lam * a[i] * cu;
  }
#pragma unroll
  for (int i = 0; i < DIM; ++i) gflux[fd * DIM + i] = out[i];
}

// face fluxes from the contracted matrices: thread (face, row i), 32 faces
// per block; every FP64 instruction runs with full warps (32 d threads)
template <int DIM>
__global__ void __launch_bounds__(32 * DIM)
    k_tflux(DevMesh m, const double* __restrict__ tco, double alpha_kbar,
            const double* __restrict__ w, const double* __restrict__ ustar,
            const double* __restrict__ ubf, double* __restrict__ flux) {
  const int64_t tile = blockIdx.x;
  const int it = threadIdx.x;  // fi * DIM + i
  const int fi = it / DIM, i = it % DIM;
  const int64_t f = tile * kTile + fi;
  const int S = m.S;
  const int64_t nc = m.wst;  // stride of the state read
  const int32_t* __restrict__ st = m.fst + tile * S * kTile + fi;
  const double* __restrict__ tc = tco + tile * (int64_t)S * kTile * DIM * DIM + it * DIM;
  double acc = 0.0;
#pragma unroll 4
  for (int n = 0; n < S; ++n) {
    const int32_t id = __ldg(st + n * kTile);
    const double* t = tc + (int64_t)n * kTile * DIM * DIM;
#pragma unroll
    for (int k = 0; k < DIM; ++k) acc = fma(__ldg(t + k), __ldg(w + k * nc + id), acc);
  }
  if (f < m.nfid) {
    const int32_t sp = m.fstar[2 * f], sn = m.fstar[2 * f + 1];
    const double other = sn >= 0 ? ustar[(int64_t)sn * DIM + i] : ubf[(f - m.nfi) * DIM + i];
    flux[f * DIM + i] = fma(alpha_kbar * m.fstab[f], other - ustar[(int64_t)sp * DIM + i], acc);
  }
}

void launch_build_tco(const DevMesh& m, double mu, double lam, double* tco, cudaStream_t st) {
  const int64_t total = m.nftile * m.S * kTile;
  if (total == 0) return;
  if (m.dim == 2)
    k_build_tco<2><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(m, mu, lam, tco);
  else
    k_build_tco<3><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(m, mu, lam, tco);
}

void launch_ghost_flux(const DevMesh& m, double mu, double lam, const double* ubq, double* gflux,
                       cudaStream_t st) {
  if (m.nfd == 0) return;
  if (m.dim == 2)
    k_ghost_flux<2><<<(unsigned)((m.nfd + 127) / 128), 128, 0, st>>>(m, mu, lam, ubq, gflux);
  else
    k_ghost_flux<3><<<(unsigned)((m.nfd + 127) / 128), 128, 0, st>>>(m, mu, lam, ubq, gflux);
}

void launch_tflux(const DevMesh& m, const double* tco, double alpha_kbar, const double* w,
                  const double* ustar, const double* ubf, double* flux, cudaStream_t st) {
  if (m.nftile == 0) return;
  if (m.dim == 2)
    k_tflux<2><<<(unsigned)m.nftile, 32 * 2, 0, st>>>(m, tco, alpha_kbar, w, ustar, ubf, flux);
  else
    k_tflux<3><<<(unsigned)m.nftile, 32 * 3, 0, st>>>(m, tco, alpha_kbar, w, ustar, ubf, flux);
}

}  // namespace hofv


// =====================================================================
// Gradient contraction in double-float arithmetic (HOFV_PREC_DF64).
//
// GB300 issues FP64 at 2 FMAs per clock per SM and FP32 at 128, while the
// per-point face kernel does d FP64 FMAs per 8-byte coefficient: it is bound
// by the FP64 pipe at 20-35 % of HBM.  Here every coefficient is stored as a
// pair of floats (hi, lo) in the same 8 bytes and the state is split the
// same way once per call; each product c u is formed as hi*hi exactly
// (TwoProduct by FMA, Dekker 1971) plus the cross terms, and accumulated by
// TwoSum with a compensation float (Dot2, Ogita, Rump & Oishi 2005): twelve
// FP32 instructions per product.  The sum is converted to FP64 for the law,
// the quadrature, the stabilisation jump and the assembly, which stay FP64.
//
// Jv must not difference two residuals contracted separately: each carries
// an independent rounding of 2^-48 relative, which the division by eps
// (~1e-8) would amplify.  For the linear law the residual is affine and the
// difference quotient is evaluated exactly as the homogeneous residual of v
// (no boundary data or sources).  For the neo-Hookean law the kernels
// contract v alone and difference the tractions of grad u + eps grad v and
// grad u in FP64, with grad u and its tractions taken from a cache filled
// once per linearisation point, so the rounding of grad u cancels exactly.
//
// The face kernel keeps several coefficient loads in flight per thread (a
// register ring) and, in 3-D, runs half a tile per block so that two blocks
// share an SM and the FP32 contraction of one overlaps the FP64 law of the
// other.
// =====================================================================
namespace hofv {

// modes of the double-float face kernel
constexpr int kDfResidual = 0;  // flux of u (split a, extrapolated values ua)
constexpr int kDfHomog = 1;     // linear law: flux of v without ghost data or prescribed values
constexpr int kDfFill = 2;      // neo-Hookean: gradient rows and tractions of u into the cache
constexpr int kDfJv = 3;        // neo-Hookean: flux(u + eps v) - flux(u) from the cache

__device__ __forceinline__ void ff_mac(float ch, float cl, float uh, float ul, float& s, float& e) {
  const float p = __fmul_rn(ch, uh);
  float r = __fmaf_rn(ch, uh, -p);  // exact rounding error of ch * uh
  r = __fmaf_rn(ch, ul, r);
  r = __fmaf_rn(cl, uh, r);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // TwoSum error
  s = t;
  e = __fadd_rn(e, __fadd_rn(q, r));
}

__device__ __forceinline__ double ff_value(float s, float e) { return (double)s + (double)e; }

// split state of cell `id` as double-float pairs (hi, mid): 48 bits
template <int DIM>
__device__ __forceinline__ void ld_split(const float4* __restrict__ p, int32_t id, float (&h)[DIM],
                                         float (&l)[DIM]) {
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    const float4 a = __ldg(p + (int64_t)id * DIM + j);
    h[j] = a.x;
    l[j] = a.y;
  }
}

__device__ __forceinline__ void split_value(double a, float& h, float& l) {
  h = __double2float_rn(a);
  l = __double2float_rn(a - (double)h);  // a - h is exact in FP64
}

// a double as hi + mid + lo, three floats, exactly (24 + 24 bits, then the
// at most 5 remaining significant bits)
__device__ __forceinline__ float4 split3(double a) {
  const float h = __double2float_rn(a);
  const double r = a - (double)h;  // exact
  const float m = __double2float_rn(r);
  return make_float4(h, m, __double2float_rn(r - (double)m), 0.f);
}

// n cells of a state read with stride ws -> three-float splits
template <int DIM>
__global__ void k_split(int64_t n, int64_t ws, const double* __restrict__ u, float4* __restrict__ su) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int j = 0; j < DIM; ++j) su[i * DIM + j] = split3(u[j * ws + i]);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// x - r from their three-float splits as a double-float pair: the high and
// middle differences exactly (TwoSum), the low parts' difference rounded
// once (2^-72 of the values), renormalised
__device__ __forceinline__ float2 diff3(const float4 x, const float4 r) {
  float s1, e1, s2, e2, h, e3;
  two_sum(x.x, -r.x, s1, e1);
  two_sum(x.y, -r.y, s2, e2);
  two_sum(s1, s2, h, e3);
  const float l = __fadd_rn(e3, __fadd_rn(e1, __fadd_rn(e2, __fsub_rn(x.z, r.z))));
  const float dh = __fadd_rn(h, l);
  return make_float2(dh, __fsub_rn(l, __fsub_rn(dh, h)));
}

__global__ void k_coef_format(double* __restrict__ a, int64_t n, int to_df) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (to_df) {
      float h, l;
      split_value(a[i], h, l);
      const unsigned long long bits =
          ((unsigned long long)__float_as_uint(l) << 32) | (unsigned long long)__float_as_uint(h);
      a[i] = __longlong_as_double((long long)bits);
    } else {
      const float2 p = reinterpret_cast<const float2*>(a)[i];
      a[i] = ff_value(p.x, p.y);
    }
  }
}

// fcsum[f][r] = sum_n of the stored pair of face f, row r, slot n
__global__ void k_row_sums(DevMesh m, double* __restrict__ fcsum) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (face, row)
  const int R = m.R;
  if (e >= m.nftile * kTile * R) return;
  const int64_t tile = e / (kTile * R);
  const int k = (int)(e % (kTile * R));  // fi * R + r within the tile
  const float2* co = reinterpret_cast<const float2*>(m.fco) + tile * (int64_t)m.S * kTile * R + k;
  double sum = 0.0;
  for (int n = 0; n < m.S; ++n) {
    const float2 p = co[(int64_t)n * kTile * R];
    sum += ff_value(p.x, p.y);
  }
  fcsum[e] = sum;
}

void launch_row_sums(const DevMesh& m, double* fcsum, cudaStream_t st) {
  const int64_t n = m.nftile * kTile * m.R;
  if (n > 0) k_row_sums<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, fcsum);
}

void launch_coef_format(double* a, int64_t n, int to_df, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, int64_t{1} << 16);  // grid-stride
  k_coef_format<<<g, 256, 0, st>>>(a, n, to_df);
}

// stabilisation extrapolation of the state w (split sw), one thread per
// (cell, local face): out[(cell * NLF + lf) * DIM + j] = w_P + sum_N e_N w_N
template <int DIM, int NLF>
__global__ void __launch_bounds__(32 * NLF)
    k_ustar_df(DevMesh m, const float4* __restrict__ sw, const double* __restrict__ w,
               double* __restrict__ out) {
  const int64_t tile = blockIdx.x;
  const int it = threadIdx.x;  // ci * NLF + lf
  const int ci = it / NLF;
  const int64_t cell = tile * kTile + ci;
  const int32_t* __restrict__ st = m.cst + tile * m.S * kTile + ci;
  const float2* __restrict__ ex =
      reinterpret_cast<const float2*>(m.cex) + tile * (int64_t)m.S * kTile * NLF + it;
  float s[DIM], e[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) s[j] = e[j] = 0.f;
#pragma unroll 4
  for (int n = 0; n < m.S; ++n) {
    const int32_t id = __ldg(st + n * kTile);
    const float2 c = __ldg(ex + (int64_t)n * kTile * NLF);
    float h[DIM], l[DIM];
    ld_split<DIM>(sw, id, h, l);
#pragma unroll
    for (int j = 0; j < DIM; ++j) ff_mac(c.x, c.y, h[j], l[j], s[j], e[j]);
  }
  if (cell < m.nc) {
    const int64_t ws = m.wst;
    const int64_t o = (cell * NLF + (it % NLF)) * DIM;
#pragma unroll
    for (int j = 0; j < DIM; ++j) out[o + j] = w[j * ws + cell] + ff_value(s[j], e[j]);
  }
}

// component i of the mirror (I - 2 n n) x of the extrapolated value x of a
// symmetry face (the value beyond the face, as k_sym_other)
template <int DIM>
__device__ __forceinline__ double mirror_i(const double* x, const double* n, int i) {
  double un = 0.0;
#pragma unroll
  for (int j = 0; j < DIM; ++j) un += n[j] * x[j];
  return x[i] - 2.0 * un * n[i];
}

// 16-byte asynchronous copy global -> shared (sm_80 and later), for gathers
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
// n doubles (n even, both ends 16-byte aligned) global -> shared, by the
// block's nthreads threads
__device__ __forceinline__ void stage16(double* dst, const double* src, int n, int it, int nthreads) {
  for (int c = it; c < n / 2; c += nthreads) cp_async16(dst + 2 * c, src + 2 * c);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Face fluxes, double-float gradient rows.  QD Gauss points per face
// (R = QD * DIM rows), FPB faces per block (BPT = 32 / FPB blocks per tile),
// blockDim = FPB * R; sw is the three-float split of the state contracted
// (u, or v in the Jv modes), wd the same state in FP64 and ws its
// extrapolated values.
//
// Each gradient is contracted against the differences to a reference cell,
// the face's nearest stencil cell N0:
//   sum_N c_N w_N = sum_N c_N (w_N - w_N0) + w_N0 sum_N c_N,
// an exact identity; the differences are small where the field is smooth,
// so the rounding of the products and sums of the contraction scales with
// them and not with |w| (on fine meshes |w| exceeds h |grad w| by orders of
// magnitude), and the last term is one FP64 product with the FP64 row sum
// of the stored coefficients.  The stored pairs differ from the FP64
// coefficients by up to 2^-48 of each; through the row sum that difference
// still meets w_N0 itself (the sum of the pairs, not of the originals).  The block first gathers its faces' stencil
// cells' splits into shared memory (16-byte asynchronous copies, [S][FPB]
// entries) and turns each into the double-float difference to its face's
// reference (exact differences of the splits); the contraction then reads
// them from shared memory (the R threads of a face share each entry) and
// skips the reference itself, whose difference is zero: its coefficient
// enters only through the row sum and is never read.  Each
// thread streams its coefficient row through a ring of RING registers: the
// coefficient of slot n + RING is requested when slot n is consumed, keeping
// RING coalesced 8-byte loads in flight per thread; with R a compile-time
// constant every ring offset is an immediate.  Faces come in groups of part
// of a tile, one thread per (face, row): in 3-D a quarter tile of 216
// threads for 3 x 3 points, five blocks an SM (measured on the 128^3
// neo-Hookean block: quarter tiles 7 % faster than half tiles two an SM,
// 10 % faster than eighth tiles), half tiles otherwise, and for faces with
// many points (polyhedral fans, R = 48 or 96) quarter or eighth tiles of 384
// threads.  For 3 x 3 points the operands read after the contraction (row
// sums, reference values, area vectors, the Jv cache) are copied into shared
// memory while it runs.
// A block contracts GPB groups one after the other (the gradients stay in
// shared memory) and then evaluates the law at all their Gauss points at
// once: R = Q d rows a face, so d groups have exactly as many points as the
// block has threads and the FP64 law runs on full warps.
// Rows of points without area (polyhedral fan slots past a face's last
// corner) load nothing.
template <int DIM, int QD>
struct DfShape {
  static constexpr int FPB = DIM == 2  ? 32
                             : QD == 9  ? 8
                             : QD == 16 ? 8
                             : QD == 32 ? 4
                                        : 16;  // faces per group
  // coefficient loads in flight per thread (4 in 2-D: 6 % slower; 3 x 3
  // points: 6, with five blocks an SM, 5 % faster than 8 with four)
  static constexpr int RING = (DIM == 3 && QD == 9) ? 6 : 8;
  static constexpr int THREADS = FPB * QD * DIM;
  // face groups per block: with GPB = d, GPB FPB Q = THREADS and each thread
  // evaluates one law (a face's Gauss point) after the block's contractions
  // (measured: 9 % faster on the 48-layer prisms, 5 % on 512^2 quads); 3 x 3
  // points keep one group a block (5 % slower with three on the 128^3 block)
  static constexpr int GPB = (DIM == 3 && QD == 9) ? 1 : DIM;
  static constexpr int MIN_BLOCKS = DIM == 2 ? 6 : (THREADS <= 256 ? 5 : 2);  // per SM
  // 3 x 3 points: the epilogue's and the law's operands (row sums, reference
  // values, area vectors and, in Jv mode, the cached gradients and
  // tractions) are copied into shared memory while the contraction runs (a
  // second group of asynchronous copies, waited for after it), instead of
  // being loaded after it with their latency exposed (measured: 5 % faster
  // on the 128^3 block; 27 % slower with 2 x 2 points, three groups a block)
  static constexpr bool STAGE = DIM == 3 && QD == 9;
};

// dynamic shared memory: the gathered cell values and the faces' references
// (one group at a time), then the gradients and tractions of all groups
template <int DIM, int QD>
static size_t df_smem_bytes(int S) {
  using SH = DfShape<DIM, QD>;
  constexpr int R = QD * DIM;
  const size_t gath = (size_t)S * SH::FPB * DIM * 16;
  const size_t law = (size_t)SH::GPB * SH::FPB * (R * DIM + QD * DIM) * sizeof(double);
  const size_t staged = SH::STAGE ? (size_t)SH::GPB * SH::FPB * (QD * 3 + R + DIM) * sizeof(double) : 0;
  return gath + law + staged;
}

template <int DIM, int LAW, int MODE, int QD>
__global__ void __launch_bounds__(DfShape<DIM, QD>::THREADS, DfShape<DIM, QD>::MIN_BLOCKS)
    k_flux_df(DevMesh m, Material mt, const float4* __restrict__ sw, const double* __restrict__ wd,
              const double* __restrict__ ws, const double* __restrict__ ubq,
              const double* __restrict__ ubf, const double* __restrict__ d_eps,
              double* __restrict__ flux) {
  using SH = DfShape<DIM, QD>;
  constexpr int FPB = SH::FPB, BPT = kTile / FPB, GPB = SH::GPB, Q = QD, R = QD * DIM;
  constexpr int kRing = SH::RING;
  constexpr int CS = kTile * R;  // coefficient stride between stencil slots
  extern __shared__ __align__(16) double sm[];
  const int S = m.S;
  // [S][FPB][DIM] gathered values of one group; slots 1.. then hold the
  // differences to slot 0, the faces' reference cells (zero difference)
  float4* us = reinterpret_cast<float4*>(sm);
  double* Gs = reinterpret_cast<double*>(us + (size_t)S * FPB * DIM);  // [GPB][FPB][R][DIM]
  double* Ts = Gs + GPB * FPB * R * DIM;                               // [GPB][FPB][Q][DIM]
  constexpr bool STG = SH::STAGE;
  double* As = Ts + GPB * FPB * Q * DIM;  // [GPB][FPB][Q][3] staged area vectors
  double* Cs = As + GPB * FPB * Q * 3;    // [GPB][FPB][R] staged row sums
  double* Ws = Cs + GPB * FPB * R;        // [GPB][FPB][DIM] staged reference values
  const int64_t ldw = m.wst;
  const int64_t ngroups = m.nftile * BPT;
  const int64_t g0 = (int64_t)blockIdx.x * GPB;
  const int ng = (int)(ngroups - g0 < GPB ? ngroups - g0 : GPB);  // the same for every thread
  const int it = threadIdx.x;
  const double eps = MODE == kDfJv ? __ldg(d_eps) : 0.0;
  const int fi = it / R, r = it % R;
  float2 cq[kRing];
  for (int gi = 0; gi < ng; ++gi) {
    const int64_t grp = g0 + gi;
    const int64_t tile = grp / BPT;
    const int fb = (int)(grp % BPT) * FPB;  // first face of the group within its tile
    const int64_t f0 = tile * kTile + fb;
    const int64_t f = f0 + fi;
    const int32_t* __restrict__ st = m.fst + tile * (int64_t)S * kTile + fb;
    const float2* __restrict__ co =
        reinterpret_cast<const float2*>(m.fco) + tile * (int64_t)S * CS + fb * R + it;
    // rows of points without area (polyhedral fan slots past a face's last
    // corner) read no coefficient and keep a zero gradient
    const bool live = m.fql == nullptr || r < __ldg(m.fql + f) * DIM;
    // stencil slots this thread contracts: 1 .. S-1 (slot 0, the reference,
    // enters only through the row sums)
    const int SL = live ? S - 1 : 0;
    co += CS;  // coefficients of slot 1
    // the first coefficients of the ring, then the gather of the cell values
#pragma unroll
    for (int d = 0; d < kRing; ++d) cq[d] = d < SL ? __ldg(co + d * CS) : make_float2(0.f, 0.f);
    for (int t = it; t < S * FPB; t += SH::THREADS) {
      const int n = t / FPB, fj = t % FPB;
      const int32_t id = __ldg(st + n * kTile + fj);
#pragma unroll
      for (int h = 0; h < DIM; ++h) cp_async16(us + t * DIM + h, sw + (int64_t)id * DIM + h);
      if (STG && n == 0) {  // the reference cell's FP64 value
#pragma unroll
        for (int j = 0; j < DIM; ++j) cp_async8(Ws + (gi * FPB + fj) * DIM + j, wd + j * ldw + id);
      }
    }
    cp_async_commit();
    if (STG) {
      // second group, waited for only after the contraction: each thread's
      // own row sum and (Jv) cached gradient row, and the group's area
      // vectors and (Jv) cached tractions for the law
      cp_async8(Cs + gi * FPB * R + it, m.fcsum + f * R + r);
      if (MODE == kDfJv) {
#pragma unroll
        for (int j = 0; j < DIM; ++j)
          cp_async8(Gs + (gi * FPB * R + it) * DIM + j, m.gcache + (f * R + r) * DIM + j);
        stage16(Ts + gi * FPB * Q * DIM, m.tcache + f0 * Q * DIM, FPB * Q * DIM, it, SH::THREADS);
      }
      // area vectors: faces up to the last one stored
      const int na = (int)(m.nf - f0 < FPB ? (m.nf - f0 > 0 ? m.nf - f0 : 0) : FPB) * Q * 3;
      for (int c = it; c < na; c += SH::THREADS) cp_async8(As + gi * FPB * Q * 3 + c, m.aq + f0 * Q * 3 + c);
      cp_async_commit();
      cp_async_wait_group<1>();  // the gather
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();
    for (int t = FPB * DIM + it; t < S * FPB * DIM; t += SH::THREADS) {
      const float2 dv = diff3(us[t], us[t % (FPB * DIM)]);
      us[t] = make_float4(dv.x, dv.y, 0.f, 0.f);
    }
    __syncthreads();
    // (1) gradient rows: thread (fi, r) accumulates sum_N c_{r,N} (w_N - w_N0)
    float s[DIM], e[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] = e[j] = 0.f;
    const float4* __restrict__ uf = us + FPB * DIM + fi * DIM;  // slot 1 of the thread's face
    auto mac_slot = [&](int n, float2 c) {
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const float4 a = uf[n * FPB * DIM + j];
        ff_mac(c.x, c.y, a.x, a.y, s[j], e[j]);
      }
    };
    int n0 = 0;
    // steady part: every request in range
    for (; n0 + 2 * kRing <= SL; n0 += kRing) {
      const float2* cn = co + (n0 + kRing) * CS;
#pragma unroll
      for (int d = 0; d < kRing; ++d) {
        const float2 c = cq[d];
        cq[d] = __ldg(cn + d * CS);
        mac_slot(n0 + d, c);
      }
    }
    // the last kRing .. 2 kRing - 1 slots (fewer if S < kRing)
#pragma unroll
    for (int d = 0; d < 2 * kRing; ++d) {
      const int n = n0 + d;
      if (n < SL) {
        const float2 c = cq[d % kRing];
        if (n + kRing < SL) cq[d % kRing] = __ldg(co + (n + kRing) * CS);
        mac_slot(n, c);
      }
    }
    if (STG) cp_async_wait_group<0>();  // this thread's staged operands
    {
      // + w_N0 sum_N c_N, in FP64
      const double cs = live ? (STG ? Cs[gi * FPB * R + it] : m.fcsum[f * R + r]) : 0.0;
      double g[DIM];
      if (STG) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) g[j] = fma(cs, Ws[(gi * FPB + fi) * DIM + j], ff_value(s[j], e[j]));
      } else {
        const int32_t id0 = __ldg(st + fi);
#pragma unroll
        for (int j = 0; j < DIM; ++j) g[j] = fma(cs, __ldg(wd + j * ldw + id0), ff_value(s[j], e[j]));
      }
      if (MODE == kDfResidual || MODE == kDfFill) {
        if (live && f >= m.nfi && f < m.nfid) {  // ghost node of a displacement face (prescribed data)
          const int64_t fd = f - m.nfi;
          const double cg = m.gco[fd * R + r];
          const int q = r / DIM;
#pragma unroll
          for (int j = 0; j < DIM; ++j) g[j] = fma(cg, ubq[(fd * Q + q) * DIM + j], g[j]);
        }
      }
      const int64_t row = (f0 * R + it) * DIM;  // == (f * R + r) * DIM
      if (MODE == kDfFill) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) m.gcache[row + j] = g[j];
      }
      if (MODE == kDfJv) {  // grad (u + eps v) = grad u + eps grad v
        double* gr = Gs + (gi * FPB * R + it) * DIM;  // staged: this row of the cache
#pragma unroll
        for (int j = 0; j < DIM; ++j) g[j] = fma(eps, g[j], STG ? gr[j] : m.gcache[row + j]);
      }
#pragma unroll
      for (int j = 0; j < DIM; ++j) Gs[(gi * FPB * R + it) * DIM + j] = g[j];
    }
    __syncthreads();  // the next group's gather overwrites the differences
  }
  // (2) law and traction at each Gauss point of the block's groups, one a thread
  {
    const int gi = it / (FPB * Q), rem = it % (FPB * Q), fj = rem / Q, q = rem % Q;
    if (gi < ng) {
      const int64_t grp = g0 + gi;
      const int64_t fq = (grp / BPT) * kTile + (grp % BPT) * FPB + fj;
      double t[DIM];
      if (fq < m.nfid) {
        double a[3];
        const double* aq = STG ? As + ((gi * FPB + fj) * Q + q) * 3 : m.aq + (fq * Q + q) * 3;
#pragma unroll
        for (int k = 0; k < DIM; ++k) a[k] = aq[k];
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const double* gq = Gs + ((gi * FPB + fj) * R + q * DIM) * DIM;
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int j = 0; j < DIM; ++j) G[i][j] = gq[i * DIM + j];
        traction<DIM, LAW>(G, a, mt, t);
      } else {
#pragma unroll
        for (int i = 0; i < DIM; ++i) t[i] = 0.0;
      }
      const int64_t o = (fq * Q + q) * DIM;
      if (MODE == kDfFill) {
#pragma unroll
        for (int i = 0; i < DIM; ++i) m.tcache[o + i] = t[i];
      }
      if (MODE == kDfJv) {
        const double* tc = STG ? Ts + ((gi * FPB + fj) * Q + q) * DIM : m.tcache + o;  // staged: this point
#pragma unroll
        for (int i = 0; i < DIM; ++i) t[i] -= tc[i];
      }
#pragma unroll
      for (int i = 0; i < DIM; ++i) Ts[((gi * FPB + fj) * Q + q) * DIM + i] = t[i];
    }
  }
  if (MODE == kDfFill) return;
  __syncthreads();
  // (3) quadrature over the face + alpha stabilisation
  for (int t3 = it; t3 < ng * FPB * DIM; t3 += SH::THREADS) {
    const int gi = t3 / (FPB * DIM), fj = (t3 / DIM) % FPB, i = t3 % DIM;
    const int64_t grp = g0 + gi;
    const int64_t ff = (grp / BPT) * kTile + (grp % BPT) * FPB + fj;
    if (ff < m.nfid) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc += Ts[((gi * FPB + fj) * Q + q) * DIM + i];
      const int32_t sp = m.fstar[2 * ff], sn = m.fstar[2 * ff + 1];
      const bool sym = sn < 0 && ff >= m.nfi + m.nfd;
      const double up = ws[(int64_t)sp * DIM + i];
      // beyond a displacement face: the prescribed value (the homogeneous and
      // Jv modes differentiate it away)
      const double other = sn >= 0 ? ws[(int64_t)sn * DIM + i]
                           : sym   ? mirror_i<DIM>(ws + (int64_t)sp * DIM, m.nrm + 3 * ff, i)
                           : MODE == kDfResidual ? ubf[(ff - m.nfi) * DIM + i]
                                                 : 0.0;
      // the stabilisation is linear: its difference at u + eps v and u is
      // eps times its value at v
      const double coef = mt.alpha * mt.kbar * m.fstab[ff] * (MODE == kDfJv ? eps : 1.0);
      flux[ff * DIM + i] = fma(coef, other - up, acc);
    }
  }
}

// Packed variant for polyhedral faces of 8 fan slots (Q = 32 points, 96
// rows a face).  The rows of the slots past a face's last corner carry no
// area; rather than one thread for each row of FPB whole faces, a group here
// is a run of consecutive faces of one tile whose rows with area fill the
// block's kPackThreads threads (at most kPackMaxFaces faces; the host builds
// the runs, DevMesh::pgrp).  Thread it of a group takes the group's it-th
// row with area, and the gradients, tractions and staged operands are
// indexed by packed row and packed point.  Everything else is k_flux_df's:
// reference differences, register ring, staged operands, GPB groups one
// after the other and then the law at all their points (at most
// kPackThreads / 3 a group, one a thread), Gauss sums over the points with
// area in the same order, stabilisation.  The fluxes equal k_flux_df's bit
// for bit (the padded points add exact zeros there).
template <int LAW, int MODE>
__global__ void __launch_bounds__(kPackThreads, 2)
    k_flux_df_pk(DevMesh m, Material mt, const float4* __restrict__ sw, const double* __restrict__ wd,
                 const double* __restrict__ ws, const double* __restrict__ ubq,
                 const double* __restrict__ ubf, const double* __restrict__ d_eps,
                 double* __restrict__ flux) {
  constexpr int DIM = 3, Q = 32, R = Q * DIM, PM = kPackMaxFaces, T = kPackThreads, GPB = 3;
  constexpr int PTS = T / DIM;  // points with area of a group, at most
  constexpr int kRing = 8;
  constexpr int CS = kTile * R;  // coefficient stride between stencil slots
  extern __shared__ __align__(16) double sm[];
  const int S = m.S;
  float4* us = reinterpret_cast<float4*>(sm);                         // [S][PM][DIM]
  double* Gs = reinterpret_cast<double*>(us + (size_t)S * PM * DIM);  // [GPB][T][DIM]
  double* Ts = Gs + GPB * T * DIM;                                    // [GPB][PTS][DIM]
  double* As = Ts + GPB * PTS * DIM;                                  // [GPB][PTS][3]
  double* Cs = As + GPB * PTS * 3;                                    // [T] row sums
  double* Ws = Cs + T;                                                // [PM][DIM] reference values
  int* rowp = reinterpret_cast<int*>(Ws + PM * DIM);                  // [GPB][PM + 1] row offsets
  int* gf = rowp + GPB * (PM + 1);                                    // [GPB][2] first face, faces
  const int64_t ldw = m.wst;
  const int64_t g0 = (int64_t)blockIdx.x * GPB;
  const int ng = (int)(m.npg - g0 < GPB ? m.npg - g0 : GPB);
  const int it = threadIdx.x;
  const double eps = MODE == kDfJv ? __ldg(d_eps) : 0.0;
  if (it < GPB) {  // the block's groups and the prefix sums of their rows with area
    int fa = 0, na = 0;
    if (it < ng) {
      fa = m.pgrp[2 * (g0 + it)];
      na = m.pgrp[2 * (g0 + it) + 1];
    }
    gf[2 * it] = fa;
    gf[2 * it + 1] = na;
    int acc = 0;
    rowp[it * (PM + 1)] = 0;
    for (int k = 0; k < PM; ++k) {
      if (k < na) acc += m.fql[fa + k] * DIM;
      rowp[it * (PM + 1) + k + 1] = acc;
    }
  }
  __syncthreads();
  float2 cq[kRing];
  for (int gi = 0; gi < ng; ++gi) {
    const int f0 = gf[2 * gi], nf = gf[2 * gi + 1];
    const int* rp = rowp + gi * (PM + 1);
    const int64_t tile = f0 / kTile;
    const int fb = f0 % kTile;
    const int nrows = rp[nf];
    int fi = 0;  // this thread's face in the group and its row there
    while (fi + 1 < nf && rp[fi + 1] <= it) ++fi;
    const bool live = it < nrows;
    const int r = live ? it - rp[fi] : 0;
    const int64_t f = f0 + fi;
    const int32_t* __restrict__ st = m.fst + tile * (int64_t)S * kTile + fb;
    const float2* __restrict__ co =
        reinterpret_cast<const float2*>(m.fco) + tile * (int64_t)S * CS + (fb + fi) * R + r + CS;
    const int SL = live ? S - 1 : 0;
#pragma unroll
    for (int d = 0; d < kRing; ++d) cq[d] = d < SL ? __ldg(co + d * CS) : make_float2(0.f, 0.f);
    for (int t = it; t < S * nf; t += T) {
      const int n = t / nf, fj = t % nf;
      const int32_t id = __ldg(st + n * kTile + fj);
#pragma unroll
      for (int h = 0; h < DIM; ++h) cp_async16(us + (n * PM + fj) * DIM + h, sw + (int64_t)id * DIM + h);
      if (n == 0) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) cp_async8(Ws + fj * DIM + j, wd + j * ldw + id);
      }
    }
    cp_async_commit();
    // second group: this thread's row sum and (Jv) cached gradient row, the
    // group's area vectors and (Jv) cached tractions by packed point
    if (live) {
      cp_async8(Cs + it, m.fcsum + f * R + r);
      if (MODE == kDfJv) {
#pragma unroll
        for (int j = 0; j < DIM; ++j)
          cp_async8(Gs + (gi * T + it) * DIM + j, m.gcache + (f * R + r) * DIM + j);
      }
    }
    if (it < nrows / DIM) {
      const int p = it;
      int fj = 0;
      while (rp[fj + 1] <= p * DIM) ++fj;
      const int q = p - rp[fj] / DIM;
      const int64_t o = ((int64_t)(f0 + fj) * Q + q) * 3;
#pragma unroll
      for (int k = 0; k < 3; ++k) cp_async8(As + (gi * PTS + p) * 3 + k, m.aq + o + k);
      if (MODE == kDfJv) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) cp_async8(Ts + (gi * PTS + p) * DIM + k, m.tcache + o + k);
      }
    }
    cp_async_commit();
    cp_async_wait_group<1>();  // the gather
    __syncthreads();
    for (int t = it; t < (S - 1) * nf * DIM; t += T) {
      const int n = 1 + t / (nf * DIM), k = t % (nf * DIM);
      const int e = n * PM * DIM + k;  // k = fj * DIM + h
      const float2 dv = diff3(us[e], us[k]);
      us[e] = make_float4(dv.x, dv.y, 0.f, 0.f);
    }
    __syncthreads();
    float s[DIM], e[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s[j] = e[j] = 0.f;
    const float4* __restrict__ uf = us + PM * DIM + fi * DIM;  // slot 1 of the thread's face
    auto mac_slot = [&](int n, float2 c) {
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const float4 a = uf[n * PM * DIM + j];
        ff_mac(c.x, c.y, a.x, a.y, s[j], e[j]);
      }
    };
    int n0 = 0;
    for (; n0 + 2 * kRing <= SL; n0 += kRing) {
      const float2* cn = co + (n0 + kRing) * CS;
#pragma unroll
      for (int d = 0; d < kRing; ++d) {
        const float2 c = cq[d];
        cq[d] = __ldg(cn + d * CS);
        mac_slot(n0 + d, c);
      }
    }
#pragma unroll
    for (int d = 0; d < 2 * kRing; ++d) {
      const int n = n0 + d;
      if (n < SL) {
        const float2 c = cq[d % kRing];
        if (n + kRing < SL) cq[d % kRing] = __ldg(co + (n + kRing) * CS);
        mac_slot(n, c);
      }
    }
    cp_async_wait_group<0>();
    {
      const double cs = live ? Cs[it] : 0.0;
      double g[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) g[j] = fma(cs, Ws[fi * DIM + j], ff_value(s[j], e[j]));
      if (MODE == kDfResidual || MODE == kDfFill) {
        if (live && f >= m.nfi && f < m.nfid) {  // ghost node of a displacement face
          const int64_t fd = f - m.nfi;
          const double cg = m.gco[fd * R + r];
          const int q = r / DIM;
#pragma unroll
          for (int j = 0; j < DIM; ++j) g[j] = fma(cg, ubq[(fd * Q + q) * DIM + j], g[j]);
        }
      }
      double* gr = Gs + (gi * T + it) * DIM;
      if (MODE == kDfFill && live) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) m.gcache[(f * R + r) * DIM + j] = g[j];
      }
      if (MODE == kDfJv) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) g[j] = fma(eps, g[j], live ? gr[j] : 0.0);
      }
#pragma unroll
      for (int j = 0; j < DIM; ++j) gr[j] = g[j];
    }
    __syncthreads();  // the next group's gather overwrites the differences
  }
  // law at each point with area of the block's groups, one a thread
  {
    const int gi = it / PTS, p = it % PTS;
    if (gi < ng) {
      const int* rp = rowp + gi * (PM + 1);
      const int nf = gf[2 * gi + 1];
      if (p < rp[nf] / DIM) {
        int fj = 0;
        while (rp[fj + 1] <= p * DIM) ++fj;
        const int q = p - rp[fj] / DIM;
        const int64_t fq = gf[2 * gi] + fj;
        double t[DIM];
        if (fq < m.nfid) {
          double a[3];
#pragma unroll
          for (int k = 0; k < DIM; ++k) a[k] = As[(gi * PTS + p) * 3 + k];
          double G[3][3];
          const double* gq = Gs + (gi * T + rp[fj] + q * DIM) * DIM;
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) G[i][j] = gq[i * DIM + j];
          traction<DIM, LAW>(G, a, mt, t);
        } else {
#pragma unroll
          for (int i = 0; i < DIM; ++i) t[i] = 0.0;
        }
        double* tp = Ts + (gi * PTS + p) * DIM;
        if (MODE == kDfFill) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) m.tcache[(fq * Q + q) * DIM + i] = t[i];
        }
        if (MODE == kDfJv) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) t[i] -= tp[i];
        }
#pragma unroll
        for (int i = 0; i < DIM; ++i) tp[i] = t[i];
      }
    }
  }
  if (MODE == kDfFill) return;
  __syncthreads();
  // Gauss sums over each face's points with area + alpha stabilisation
  for (int t3 = it; t3 < ng * PM * DIM; t3 += T) {
    const int gi = t3 / (PM * DIM), fj = (t3 / DIM) % PM, i = t3 % DIM;
    const int* rp = rowp + gi * (PM + 1);
    if (fj >= gf[2 * gi + 1]) continue;
    const int64_t ff = gf[2 * gi] + fj;
    if (ff >= m.nfid) continue;
    double acc = 0.0;
    for (int p = rp[fj] / DIM; p < rp[fj + 1] / DIM; ++p) acc += Ts[(gi * PTS + p) * DIM + i];
    const int32_t sp = m.fstar[2 * ff], sn = m.fstar[2 * ff + 1];
    const bool sym = sn < 0 && ff >= m.nfi + m.nfd;
    const double up = ws[(int64_t)sp * DIM + i];
    const double other = sn >= 0 ? ws[(int64_t)sn * DIM + i]
                         : sym   ? mirror_i<DIM>(ws + (int64_t)sp * DIM, m.nrm + 3 * ff, i)
                         : MODE == kDfResidual ? ubf[(ff - m.nfi) * DIM + i]
                                               : 0.0;
    const double coef = mt.alpha * mt.kbar * m.fstab[ff] * (MODE == kDfJv ? eps : 1.0);
    flux[ff * DIM + i] = fma(coef, other - up, acc);
  }
}

static size_t df_pk_smem_bytes(int S) {
  constexpr int PM = kPackMaxFaces, T = kPackThreads, GPB = 3, PTS = T / 3;
  return (size_t)S * PM * 3 * 16 + sizeof(double) * (GPB * T * 3 + GPB * PTS * 3 * 2 + T + PM * 3) +
         sizeof(int) * (GPB * (PM + 1) + GPB * 2);
}

template <int LAW, int MODE>
static void launch_flux_df_pk(const DevMesh& m, const Material& mat, const float4* sw,
                              const double* wd, const double* ws, const double* ubq,
                              const double* ubf, const double* d_eps, double* flux, cudaStream_t st) {
  if (m.npg == 0) return;
  k_flux_df_pk<LAW, MODE><<<(unsigned)((m.npg + 2) / 3), kPackThreads, df_pk_smem_bytes(m.S), st>>>(
      m, mat, sw, wd, ws, ubq, ubf, d_eps, flux);
}

// contracted linear form, homogeneous part at v: sum_N T_N v_N plus the
// stabilisation of v with zero prescribed values (symmetry faces mirror)
template <int DIM>
__global__ void __launch_bounds__(32 * DIM)
    k_tflux_hom(DevMesh m, const double* __restrict__ tco, double alpha_kbar,
                const double* __restrict__ v, const double* __restrict__ vstar,
                double* __restrict__ flux) {
  const int64_t tile = blockIdx.x;
  const int it = threadIdx.x;  // fi * DIM + i
  const int fi = it / DIM, i = it % DIM;
  const int64_t f = tile * kTile + fi;
  const int S = m.S;
  const int64_t ws = m.wst;
  const int32_t* __restrict__ st = m.fst + tile * S * kTile + fi;
  const double* __restrict__ tc = tco + tile * (int64_t)S * kTile * DIM * DIM + it * DIM;
  double acc = 0.0;
#pragma unroll 4
  for (int n = 0; n < S; ++n) {
    const int32_t id = __ldg(st + n * kTile);
    const double* t = tc + (int64_t)n * kTile * DIM * DIM;
#pragma unroll
    for (int k = 0; k < DIM; ++k) acc = fma(__ldg(t + k), __ldg(v + k * ws + id), acc);
  }
  if (f < m.nfid) {
    const int32_t sp = m.fstar[2 * f], sn = m.fstar[2 * f + 1];
    const bool sym = sn < 0 && f >= m.nfi + m.nfd;
    const double up = vstar[(int64_t)sp * DIM + i];
    const double other = sn >= 0 ? vstar[(int64_t)sn * DIM + i]
                         : sym   ? mirror_i<DIM>(vstar + (int64_t)sp * DIM, m.nrm + 3 * f, i)
                                 : 0.0;
    flux[f * DIM + i] = fma(alpha_kbar * m.fstab[f], other - up, acc);
  }
}

// Jv assembly from face-flux differences: out = sum_f +-dflux_f / eps, plus
// the inertia term of v (linear, so its difference quotient is exact)
template <int DIM, int NLF>
__global__ void k_cell_diff(DevMesh m, const double* __restrict__ flux,
                            const double* __restrict__ d_eps, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  double r[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) r[j] = 0.0;
#pragma unroll
  for (int lf = 0; lf < NLF; ++lf) {
    const int32_t code = m.cface[c * NLF + lf];
    if (code == 0) continue;
    const int64_t f = (code > 0 ? code : -code) - 1;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const double v = flux[f * DIM + j];
      r[j] = code > 0 ? r[j] + v : r[j] - v;
    }
  }
  const double ie = 1.0 / d_eps[0];
#pragma unroll
  for (int j = 0; j < DIM; ++j)
    out[j * m.nc + c] = m.mscale ? fma(r[j], ie, m.inert[j * m.nc + c]) : r[j] * ie;
}

template <int DIM>
static void launch_ustar_df(const DevMesh& m, const float4* sw, const double* w, double* out,
                            cudaStream_t st) {
  by_faces_per_cell<DIM>(m, [&](auto nlf) {
    constexpr int NLF = decltype(nlf)::value;
    k_ustar_df<DIM, NLF><<<(unsigned)m.nctile, 32 * NLF, 0, st>>>(m, sw, w, out);
  });
}

template <int DIM, int LAW, int MODE, int QD>
static void launch_flux_df_q(const DevMesh& m, const Material& mat, const float4* sw,
                             const double* wd, const double* ws, const double* ubq,
                             const double* ubf, const double* d_eps, double* flux,
                             cudaStream_t st) {
  using SH = DfShape<DIM, QD>;
  const size_t smem = df_smem_bytes<DIM, QD>(m.S);
  const int64_t groups = m.nftile * (kTile / SH::FPB);
  k_flux_df<DIM, LAW, MODE, QD><<<(unsigned)((groups + SH::GPB - 1) / SH::GPB), SH::THREADS, smem,
                                  st>>>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux);
}

// Gauss points per face: q^(d-1) for q = 1..4 in 2-D, 1..3 in 3-D; on
// polyhedra 4 or 8 fan slots of q^2 points for q = 1, 2
template <int DIM, int LAW, int MODE>
static void launch_flux_df(const DevMesh& m, const Material& mat, const float4* sw,
                           const double* wd, const double* ws, const double* ubq,
                           const double* ubf, const double* d_eps, double* flux, cudaStream_t st) {
  if constexpr (DIM == 2) {
    switch (m.Q) {
      case 1: return launch_flux_df_q<2, LAW, MODE, 1>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      case 2: return launch_flux_df_q<2, LAW, MODE, 2>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      case 3: return launch_flux_df_q<2, LAW, MODE, 3>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      default: return launch_flux_df_q<2, LAW, MODE, 4>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
    }
  } else {
    switch (m.Q) {
      case 1: return launch_flux_df_q<3, LAW, MODE, 1>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      case 4: return launch_flux_df_q<3, LAW, MODE, 4>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      case 8: return launch_flux_df_q<3, LAW, MODE, 8>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      case 16: return launch_flux_df_q<3, LAW, MODE, 16>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      case 32:
        if (m.pgrp) return launch_flux_df_pk<LAW, MODE>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
        return launch_flux_df_q<3, LAW, MODE, 32>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
      default: return launch_flux_df_q<3, LAW, MODE, 9>(m, mat, sw, wd, ws, ubq, ubf, d_eps, flux, st);
    }
  }
}

// the state (extended by the mirror nodes when the mesh has symmetry faces)
// split into double-float pairs; returns the FP64 state the kernels read
template <int DIM>
static const double* split_state(const DevMesh& m, const double* u, double* ext, float4* su,
                                 cudaStream_t st) {
  const unsigned g = (unsigned)((m.wst + 255) / 256);
  if (m.ng > 0) {
    k_extend<DIM><<<g, 256, 0, st>>>(m, u, ext);
    u = ext;
  }
  k_split<DIM><<<g, 256, 0, st>>>(m.wst, m.wst, u, su);
  return u;
}

template <int DIM, int LAW>
static void residual_impl_df(const DevMesh& m, const Material& mat, const double* w,
                             const double* d_eps, const double* R0, double* out, double* ustar,
                             double* flux, const double* ubq, const double* ubf, const double* src,
                             cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  w = split_state<DIM>(m, w, m.wext, m.su, st);
  launch_ustar_df<DIM>(m, m.su, w, ustar, st);
  if (ev) cudaEventRecord(ev[1], st);
  if (m.nftile > 0) {
    if (LAW == HOFV_LAW_LINEAR && m.tco) {
      if (m.nfy > 0) k_sym_other<DIM><<<(unsigned)((m.nfy + 127) / 128), 128, 0, st>>>(m, ustar);
      k_tflux<DIM><<<(unsigned)m.nftile, 32 * DIM, 0, st>>>(m, m.tco, mat.alpha * mat.kbar, w,
                                                            ustar, ubf, flux);
    } else {
      launch_flux_df<DIM, LAW, kDfResidual>(m, mat, m.su, w, ustar, ubq, ubf, nullptr, flux, st);
    }
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (m.mscale)
    k_cell_avg<DIM, true><<<(unsigned)((m.nc + 127) / 128), 128, 0, st>>>(m, w, m.wst, m.inert);
  const unsigned cgrid = (unsigned)((m.nc + 255) / 256);
  by_faces_per_cell<DIM>(m, [&](auto nlf) {
    constexpr int NLF = decltype(nlf)::value;
    k_cell<DIM, NLF><<<cgrid, 256, 0, st>>>(m, flux, src, R0, d_eps, out);
  });
  if (ev) cudaEventRecord(ev[3], st);
}

template <int DIM, int LAW>
static void jv_impl_df(const DevMesh& m, const Material& mat, const double* v,
                       const double* d_eps, double* out, double* flux, cudaStream_t st,
                       cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  v = split_state<DIM>(m, v, m.vext, m.sv, st);
  launch_ustar_df<DIM>(m, m.sv, v, m.ustar_v, st);
  if (ev) cudaEventRecord(ev[1], st);
  if (m.nftile > 0) {
    if (LAW == HOFV_LAW_LINEAR && m.tco)
      k_tflux_hom<DIM><<<(unsigned)m.nftile, 32 * DIM, 0, st>>>(m, m.tco, mat.alpha * mat.kbar, v,
                                                                m.ustar_v, flux);
    else if (LAW == HOFV_LAW_LINEAR)
      launch_flux_df<DIM, LAW, kDfHomog>(m, mat, m.sv, v, m.ustar_v, nullptr, nullptr, nullptr,
                                         flux, st);
    else
      launch_flux_df<DIM, LAW, kDfJv>(m, mat, m.sv, v, m.ustar_v, nullptr, nullptr, d_eps, flux,
                                      st);
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (m.mscale)
    k_cell_avg<DIM, true><<<(unsigned)((m.nc + 127) / 128), 128, 0, st>>>(m, v, m.wst, m.inert);
  const unsigned cgrid = (unsigned)((m.nc + 255) / 256);
  by_faces_per_cell<DIM>(m, [&](auto nlf) {
    constexpr int NLF = decltype(nlf)::value;
    if (LAW == HOFV_LAW_LINEAR)  // the homogeneous residual: J v itself
      k_cell<DIM, NLF><<<cgrid, 256, 0, st>>>(m, flux, nullptr, nullptr, nullptr, out);
    else
      k_cell_diff<DIM, NLF><<<cgrid, 256, 0, st>>>(m, flux, d_eps, out);
  });
  if (ev) cudaEventRecord(ev[3], st);
}

void launch_residual_df(const DevMesh& m, const Material& mat, const double* w,
                        const double* d_eps, const double* R0, double* out, double* ustar,
                        double* flux, const double* ubq, const double* ubf, const double* src,
                        cudaStream_t st, cudaEvent_t* ev) {
  if (m.dim == 2) {
    if (mat.law == HOFV_LAW_LINEAR)
      residual_impl_df<2, 0>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
    else
      residual_impl_df<2, 1>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
  } else {
    if (mat.law == HOFV_LAW_LINEAR)
      residual_impl_df<3, 0>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
    else
      residual_impl_df<3, 1>(m, mat, w, d_eps, R0, out, ustar, flux, ubq, ubf, src, st, ev);
  }
}

void launch_jv_df(const DevMesh& m, const Material& mat, const double* v, const double* d_eps,
                  double* out, double* flux, cudaStream_t st, cudaEvent_t* ev) {
  if (m.dim == 2) {
    if (mat.law == HOFV_LAW_LINEAR)
      jv_impl_df<2, 0>(m, mat, v, d_eps, out, flux, st, ev);
    else
      jv_impl_df<2, 1>(m, mat, v, d_eps, out, flux, st, ev);
  } else {
    if (mat.law == HOFV_LAW_LINEAR)
      jv_impl_df<3, 0>(m, mat, v, d_eps, out, flux, st, ev);
    else
      jv_impl_df<3, 1>(m, mat, v, d_eps, out, flux, st, ev);
  }
}

// the face kernels' gathers exceed the default 48 KB of dynamic shared
// memory for large stencils: raise the limit of every instantiation to what
// kMaxS stencil cells need, once per process (set-up calls only, never
// during stream capture)
template <int DIM, int LAW, int MODE, int QD>
static void raise_smem(cudaError_t& e) {
  const cudaError_t r =
      cudaFuncSetAttribute((const void*)k_flux_df<DIM, LAW, MODE, QD>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)df_smem_bytes<DIM, QD>(kMaxS));
  if (r != cudaSuccess) e = r;
}
template <int LAW, int MODE>
static void raise_smem_pk(cudaError_t& e) {
  const cudaError_t r = cudaFuncSetAttribute((const void*)k_flux_df_pk<LAW, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)df_pk_smem_bytes(kMaxS));
  if (r != cudaSuccess) e = r;
}
template <int DIM, int QD>
static void raise_smem_all(cudaError_t& e) {
  raise_smem<DIM, 0, kDfResidual, QD>(e);
  raise_smem<DIM, 1, kDfResidual, QD>(e);
  raise_smem<DIM, 0, kDfHomog, QD>(e);
  raise_smem<DIM, 1, kDfFill, QD>(e);
  raise_smem<DIM, 1, kDfJv, QD>(e);
}
int setup_df_kernels() {
  static int rc = -1;
  if (rc >= 0) return rc;
  cudaError_t e = cudaSuccess;
  raise_smem_all<2, 1>(e);
  raise_smem_all<2, 2>(e);
  raise_smem_all<2, 3>(e);
  raise_smem_all<2, 4>(e);
  raise_smem_all<3, 1>(e);
  raise_smem_all<3, 4>(e);
  raise_smem_all<3, 9>(e);
  raise_smem_all<3, 8>(e);
  raise_smem_all<3, 16>(e);
  raise_smem_all<3, 32>(e);
  raise_smem_pk<0, kDfResidual>(e);
  raise_smem_pk<1, kDfResidual>(e);
  raise_smem_pk<0, kDfHomog>(e);
  raise_smem_pk<1, kDfFill>(e);
  raise_smem_pk<1, kDfJv>(e);
  rc = e == cudaSuccess ? 0 : (int)e;
  return rc;
}

void launch_jv_cache_fill(const DevMesh& m, const Material& mat, const double* u,
                          const double* ubq, cudaStream_t st) {
  if (m.nftile == 0) return;
  if (m.dim == 2) {
    const double* w = split_state<2>(m, u, m.wext, m.su, st);
    launch_flux_df<2, 1, kDfFill>(m, mat, m.su, w, nullptr, ubq, nullptr, nullptr, nullptr, st);
  } else {
    const double* w = split_state<3>(m, u, m.wext, m.su, st);
    launch_flux_df<3, 1, kDfFill>(m, mat, m.su, w, nullptr, ubq, nullptr, nullptr, nullptr, st);
  }
}

}  // namespace hofv
