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
    // (eq. nanson).  With tau = J sigma = mu dev(bbar) + kappa/2 (J^2-1) I
    // and F^{-T} = cof(F) / J:  P = tau cof(F) / J.
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
    // J^{-2/3}; not defined for J <= 0 (an inverted element): NaN, so the
    // caller's finiteness checks reject the state
    const double jm23 = J > 0.0 ? rcbrt(J * J) : __longlong_as_double(0x7ff8000000000000LL);
    double b[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const double s = F[i][0] * F[j][0] + F[i][1] * F[j][1] + F[i][2] * F[j][2];
        b[i][j] = b[j][i] = jm23 * s;
      }
    const double tb = (b[0][0] + b[1][1] + b[2][2]) * (1.0 / 3.0);
    const double pvol = 0.5 * mt.kappa * (J * J - 1.0);
    double tau[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tau[i][j] = mt.mu * (b[i][j] - (i == j ? tb : 0.0)) + (i == j ? pvol : 0.0);
    // t = P a = tau (cof(F) a) / J
    double ca[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < DIM; ++l) s = fma(C[k][l], a[l], s);
      ca[k] = s;
    }
    const double iJ = 1.0 / J;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) s = fma(tau[i][k], ca[k], s);
      t[i] = s * iJ;
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
#pragma unroll 4
    for (int n = 0; n < S; ++n) {
      const int32_t id = __ldg(st + n * kTile);
      const double c = __ldg(co + (int64_t)n * kTile * R);
#pragma unroll
      for (int j = 0; j < DIM; ++j) acc[j] = fma(c, __ldg(w + j * nc + id), acc[j]);
    }
    if (f >= m.nfi && f < m.nfid) {  // ghost node of a displacement face
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
  // faces per cell: d + 1 (triangles / tetrahedra), 2 d (quads / hexes),
  // kPolyMaxSides slots (2-D polygons)
  if (m.nlf == DIM + 1) {
    k_ustar<DIM, DIM + 1><<<(unsigned)m.nctile, 32 * (DIM + 1), 0, st>>>(m, w, ustar);
  } else if (m.nlf == 2 * DIM) {
    k_ustar<DIM, 2 * DIM><<<(unsigned)m.nctile, 32 * 2 * DIM, 0, st>>>(m, w, ustar);
  } else {
    if constexpr (DIM == 2)
      k_ustar<2, kPolyMaxSides><<<(unsigned)m.nctile, 32 * kPolyMaxSides, 0, st>>>(m, w, ustar);
  }
  if (m.nfy > 0) k_sym_other<DIM><<<(unsigned)((m.nfy + 127) / 128), 128, 0, st>>>(m, ustar);
  if (ev) cudaEventRecord(ev[1], st);
  if (m.nftile > 0) {
    if (LAW == HOFV_LAW_LINEAR && m.tco) {
      k_tflux<DIM><<<(unsigned)m.nftile, 32 * DIM, 0, st>>>(m, m.tco, mat.alpha * mat.kbar, w,
                                                            ustar, ubf, flux);
    } else {
      const size_t smem = sizeof(double) * kTile * (m.R * DIM + m.Q * DIM);
      k_flux<DIM, LAW><<<(unsigned)m.nftile, kTile * m.R, smem, st>>>(m, mat, w, ustar, ubq, ubf,
                                                                      flux);
    }
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (m.mscale)
    k_cell_avg<DIM, true><<<(unsigned)((m.nc + 127) / 128), 128, 0, st>>>(m, w, m.wst, m.inert);
  const unsigned cgrid = (unsigned)((m.nc + 255) / 256);
  if (m.nlf == DIM + 1) {
    k_cell<DIM, DIM + 1><<<cgrid, 256, 0, st>>>(m, flux, src, R0, d_eps, out);
  } else if (m.nlf == 2 * DIM) {
    k_cell<DIM, 2 * DIM><<<cgrid, 256, 0, st>>>(m, flux, src, R0, d_eps, out);
  } else {
    if constexpr (DIM == 2) k_cell<2, kPolyMaxSides><<<cgrid, 256, 0, st>>>(m, flux, src, R0, d_eps, out);
  }
  if (ev) cudaEventRecord(ev[3], st);
}

void launch_residual(const DevMesh& m, const Material& mat, const double* w, const double* /*v*/,
                     const double* d_eps, const double* R0, double* out, double* ustar,
                     double* flux, const double* ubq, const double* ubf, const double* src,
                     cudaStream_t st, cudaEvent_t* ev) {
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
        c[i] = co[q * DIM + i];
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
