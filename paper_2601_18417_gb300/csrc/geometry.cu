// geometry.cu -- face and cell geometry and Gaussian quadrature
// (arXiv 2601.18417, Sec. 3.1-3.3): Gauss points and vector-area elements of
// straight edges (2-D) and bilinear faces (3-D), face areas, normals and
// centres, cell volumes and centroids by the divergence theorem, and cell
// Gauss points of the bilinear / trilinear map.  Triangles and tetrahedra
// use the same tensor rules on the collapsed square / cube (Duffy's
// transformation): a triangular face is the bilinear patch (a, b, c, a), a
// triangle cell the bilinear map of (0, 1, 2, 0) and a tetrahedron the
// trilinear map of (0, 1, 2, 0, 0, 1, 3, 0).  A polygon's cell rule is the
// fan of such collapsed triangles from its corners' average.
//
// This unit is compiled without FMA contraction and evaluates every
// expression in a fixed order, so that face centres and centroids -- which
// decide the nearest-neighbour stencils and their tie order -- are the
// correctly rounded results of the written formulas.
#include <math.h>

#include "hofv_internal.cuh"

namespace hofv {

struct Gauss {
  double x[4], w[4];
  int n;
};

__constant__ int c_quad_lf[4][2] = {{3, 0}, {1, 2}, {0, 1}, {2, 3}};
__constant__ int c_hex_lf[6][4] = {{0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4},
                                   {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};
__constant__ int c_tri_lf[3][2] = {{0, 1}, {1, 2}, {2, 0}};
__constant__ int c_tet_lf[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
// cell node of each corner of the collapsed reference square / cube
__constant__ int c_tri_map[4] = {0, 1, 2, 0};
__constant__ int c_tet_map[8] = {0, 1, 2, 0, 0, 1, 3, 0};

__device__ __forceinline__ int local_face_node(int dim, bool simplex, int lf, int k) {
  if (simplex) return dim == 2 ? c_tri_lf[lf][k] : c_tet_lf[lf][k];
  return dim == 2 ? c_quad_lf[lf][k] : c_hex_lf[lf][k];
}

// Gauss points and vector-area elements of one face.  corner: [nfv][3] in
// outward order; faces are straight edges (2-D) or bilinear patches (3-D).
__device__ void face_points(int dim, const Gauss& g, const double* corner, double* xq,
                            double* aq) {
  const int n = g.n;
  if (dim == 2) {
    const double tx = corner[3] - corner[0], ty = corner[4] - corner[1];
    for (int a = 0; a < n; ++a) {
      const double s = g.x[a];
      for (int k = 0; k < 3; ++k) xq[3 * a + k] = (1.0 - s) * corner[k] + s * corner[3 + k];
      aq[3 * a + 0] = g.w[a] * ty;
      aq[3 * a + 1] = -g.w[a] * tx;
      aq[3 * a + 2] = 0.0;
    }
    return;
  }
  const double *c0 = corner, *c1 = corner + 3, *c2 = corner + 6, *c3 = corner + 9;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const double xi = g.x[a], eta = g.x[b];
      const int q = a * n + b;
      double xs[3], xe[3];
      for (int k = 0; k < 3; ++k) {
        xq[3 * q + k] = (1 - xi) * (1 - eta) * c0[k] + xi * (1 - eta) * c1[k] + xi * eta * c2[k] +
                        (1 - xi) * eta * c3[k];
        xs[k] = (1 - eta) * (c1[k] - c0[k]) + eta * (c2[k] - c3[k]);
        xe[k] = (1 - xi) * (c3[k] - c0[k]) + xi * (c2[k] - c1[k]);
      }
      const double w = g.w[a] * g.w[b];
      aq[3 * q + 0] = w * (xs[1] * xe[2] - xs[2] * xe[1]);
      aq[3 * q + 1] = w * (xs[2] * xe[0] - xs[0] * xe[2]);
      aq[3 * q + 2] = w * (xs[0] * xe[1] - xs[1] * xe[0]);
    }
}

__global__ void k_face_geometry(int dim, int nfv, int Q, int64_t nf, Gauss g,
                                const double* __restrict__ x, const int32_t* __restrict__ fnodes,
                                double* xq, double* aq, double* xf, double* nrm, double* gam) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double corner[12];
  for (int k = 0; k < nfv; ++k)
    for (int a = 0; a < 3; ++a) corner[3 * k + a] = x[3 * (int64_t)fnodes[f * nfv + k] + a];
  if (dim == 3 && nfv == 3)
    for (int a = 0; a < 3; ++a) corner[9 + a] = corner[a];
  double pq[3 * kMaxQ], pa[3 * kMaxQ];
  face_points(dim, g, corner, pq, pa);
  double G = 0, A[3] = {0, 0, 0}, X[3] = {0, 0, 0};
  for (int q = 0; q < Q; ++q) {
    const double m = sqrt(pa[3 * q] * pa[3 * q] + pa[3 * q + 1] * pa[3 * q + 1] +
                          pa[3 * q + 2] * pa[3 * q + 2]);
    G += m;
    for (int k = 0; k < 3; ++k) {
      A[k] += pa[3 * q + k];
      X[k] += m * pq[3 * q + k];
      xq[(f * Q + q) * 3 + k] = pq[3 * q + k];
      aq[(f * Q + q) * 3 + k] = pa[3 * q + k];
    }
  }
  const double An = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
  gam[f] = G;
  for (int k = 0; k < 3; ++k) {
    xf[3 * f + k] = X[k] / G;
    nrm[3 * f + k] = A[k] / An;
  }
}

// Gauss points and weights of the bilinear map of the quad with corners P
// (counter-clockwise; a repeated corner collapses it to a triangle)
__device__ void quad_cell_points(const Gauss& g, const double (*P)[3], double* cqx, double* cqw) {
  const int n = g.n;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const double s = g.x[a], t = g.x[b];
      const double N[4] = {(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t};
      const double Ns[4] = {-(1 - t), 1 - t, t, -t};
      const double Nt[4] = {-(1 - s), -s, s, 1 - s};
      double X[2] = {0, 0}, J00 = 0, J01 = 0, J10 = 0, J11 = 0;
      for (int k = 0; k < 4; ++k) {
        X[0] += N[k] * P[k][0];
        X[1] += N[k] * P[k][1];
        J00 += Ns[k] * P[k][0];
        J01 += Nt[k] * P[k][0];
        J10 += Ns[k] * P[k][1];
        J11 += Nt[k] * P[k][1];
      }
      const int q = a * n + b;
      cqx[q * 3 + 0] = X[0];
      cqx[q * 3 + 1] = X[1];
      cqx[q * 3 + 2] = 0.0;
      cqw[q] = g.w[a] * g.w[b] * fabs(J00 * J11 - J01 * J10);
    }
}

// Gauss points and weights of the trilinear map of the hex with corners P
// (repeated corners collapse it to a tetrahedron)
__device__ void hex_cell_points(const Gauss& g, const double (*P)[3], double* cqx, double* cqw) {
  const int n = g.n;
  const int R3[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                        {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int e = 0; e < n; ++e) {
        const double s[3] = {g.x[a], g.x[b], g.x[e]};
        double X[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int k = 0; k < 8; ++k) {
          double f[3], dr[3];
          for (int r = 0; r < 3; ++r) {
            f[r] = R3[k][r] ? s[r] : 1 - s[r];
            dr[r] = R3[k][r] ? 1.0 : -1.0;
          }
          const double N = f[0] * f[1] * f[2];
          const double dN[3] = {dr[0] * f[1] * f[2], f[0] * dr[1] * f[2], f[0] * f[1] * dr[2]};
          for (int r = 0; r < 3; ++r) {
            X[r] += N * P[k][r];
            for (int t = 0; t < 3; ++t) J[r][t] += dN[t] * P[k][r];
          }
        }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const int q = (a * n + b) * n + e;
        for (int r = 0; r < 3; ++r) cqx[q * 3 + r] = X[r];
        cqw[q] = g.w[a] * g.w[b] * g.w[e] * fabs(det);
      }
}

// volume and centroid from the divergence theorem over the cell's own
// outward faces; Gauss points of the bilinear / trilinear cell map.  A
// polygon (poly: corners padded with -1 up to nv) uses its sides as faces
// and, for the cell rule, the fan of collapsed triangles from its corners'
// average, one block of n^2 points per slot (zero weight past the last side).
__global__ void k_cell_geometry(int dim, bool simplex, bool poly, int nv, int nlf, int nfv, int Q,
                                int QC, int64_t nc, Gauss g, const double* __restrict__ x,
                                const int32_t* __restrict__ cnodes, double* xc, double* vol,
                                double* cqx, double* cqw) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int nk = nv;  // corners present
  if (poly) {
    nk = 0;
    while (nk < nv && cnodes[c * nv + nk] >= 0) ++nk;
  }
  double cx[8][3];
  for (int k = 0; k < nk; ++k)
    for (int a = 0; a < 3; ++a) cx[k][a] = x[3 * (int64_t)cnodes[c * nv + k] + a];
  double V = 0, M2[3] = {0, 0, 0};
  const int nfaces = poly ? nk : nlf;
  for (int lf = 0; lf < nfaces; ++lf) {
    double corner[12];
    for (int k = 0; k < nfv; ++k) {
      const int node = poly ? (lf + k) % nk : local_face_node(dim, simplex, lf, k);
      for (int a = 0; a < 3; ++a) corner[3 * k + a] = cx[node][a];
    }
    if (dim == 3 && nfv == 3)
      for (int a = 0; a < 3; ++a) corner[9 + a] = corner[a];
    double pq[3 * kMaxQ], pa[3 * kMaxQ];
    face_points(dim, g, corner, pq, pa);
    for (int q = 0; q < Q; ++q)
      for (int a = 0; a < dim; ++a) {
        V += pq[3 * q + a] * pa[3 * q + a];
        M2[a] += pq[3 * q + a] * pq[3 * q + a] * pa[3 * q + a];
      }
  }
  V /= dim;
  vol[c] = V;
  for (int a = 0; a < 3; ++a) xc[3 * c + a] = a < dim ? M2[a] / (2.0 * V) : 0.0;
  const int n = g.n;
  if (poly) {
    double xb[3] = {0, 0, 0};
    for (int k = 0; k < nk; ++k)
      for (int a = 0; a < 2; ++a) xb[a] += cx[k][a];
    for (int a = 0; a < 2; ++a) xb[a] /= nk;
    for (int t = 0; t < nlf; ++t) {
      double* qx = cqx + (c * QC + t * n * n) * 3;
      double* qw = cqw + c * QC + t * n * n;
      if (t >= nk) {
        for (int q = 0; q < n * n; ++q) {
          for (int a = 0; a < 3; ++a) qx[3 * q + a] = xb[a];
          qw[q] = 0.0;
        }
        continue;
      }
      const int t1 = (t + 1) % nk;
      const double P[4][3] = {{xb[0], xb[1], 0.0},
                              {cx[t][0], cx[t][1], 0.0},
                              {cx[t1][0], cx[t1][1], 0.0},
                              {xb[0], xb[1], 0.0}};
      quad_cell_points(g, P, qx, qw);
    }
    return;
  }
  if (simplex) {  // corners of the collapsed square / cube
    double s[8][3];
    const int nm = dim == 2 ? 4 : 8;
    for (int k = 0; k < nm; ++k)
      for (int a = 0; a < 3; ++a) s[k][a] = cx[dim == 2 ? c_tri_map[k] : c_tet_map[k]][a];
    for (int k = 0; k < nm; ++k)
      for (int a = 0; a < 3; ++a) cx[k][a] = s[k][a];
  }
  if (dim == 2) {
    quad_cell_points(g, cx, cqx + c * QC * 3, cqw + c * QC);
    return;
  }
  hex_cell_points(g, cx, cqx + c * QC * 3, cqw + c * QC);
}

// ---------------------------------------------------------------------
// polyhedra given face by face (corners padded with -1 up to nfv): a face
// is the fan of triangles from its corners' average cb, each the collapsed
// patch (cb, v_t, v_t+1, cb) with n^2 points (zero area at cb in the slots
// past its last corner); a cell's volume and centroid come from the
// divergence theorem over its faces' points, its rule from the fan of
// tetrahedra (xb, cb_f, v_t, v_t+1), xb the average of its faces' cb.
// ---------------------------------------------------------------------
__device__ __forceinline__ int face_corners_fan(const int32_t* __restrict__ fn, int nfv,
                                                const double* __restrict__ x, double* cb) {
  int k = 0;
  while (k < nfv && fn[k] >= 0) ++k;
  for (int a = 0; a < 3; ++a) cb[a] = 0.0;
  for (int t = 0; t < k; ++t)
    for (int a = 0; a < 3; ++a) cb[a] += x[3 * (int64_t)fn[t] + a];
  for (int a = 0; a < 3; ++a) cb[a] /= k;
  return k;
}

__global__ void k_face_geometry_fan(int nfv, int Q, int64_t nf, Gauss g,
                                    const double* __restrict__ x,
                                    const int32_t* __restrict__ fnodes, double* xq, double* aq,
                                    double* xf, double* nrm, double* gam) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int32_t* fn = fnodes + f * nfv;
  double cb[3];
  const int k = face_corners_fan(fn, nfv, x, cb);
  const int n2 = g.n * g.n;
  double G = 0, A[3] = {0, 0, 0}, X[3] = {0, 0, 0};
  for (int t = 0; t < nfv; ++t) {
    double pq[3 * kMaxQ], pa[3 * kMaxQ];
    if (t < k) {
      double corner[12];
      const int32_t v0 = fn[t], v1 = fn[(t + 1) % k];
      for (int a = 0; a < 3; ++a) {
        corner[a] = cb[a];
        corner[3 + a] = x[3 * (int64_t)v0 + a];
        corner[6 + a] = x[3 * (int64_t)v1 + a];
        corner[9 + a] = cb[a];
      }
      face_points(3, g, corner, pq, pa);
    } else {
      for (int q = 0; q < n2; ++q)
        for (int a = 0; a < 3; ++a) {
          pq[3 * q + a] = cb[a];
          pa[3 * q + a] = 0.0;
        }
    }
    for (int q = 0; q < n2; ++q) {
      const double m = sqrt(pa[3 * q] * pa[3 * q] + pa[3 * q + 1] * pa[3 * q + 1] +
                            pa[3 * q + 2] * pa[3 * q + 2]);
      G += m;
      const int64_t o = (f * Q + t * n2 + q) * 3;
      for (int a = 0; a < 3; ++a) {
        A[a] += pa[3 * q + a];
        X[a] += m * pq[3 * q + a];
        xq[o + a] = pq[3 * q + a];
        aq[o + a] = pa[3 * q + a];
      }
    }
  }
  const double An = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
  gam[f] = G;
  for (int a = 0; a < 3; ++a) {
    xf[3 * f + a] = X[a] / G;
    nrm[3 * f + a] = A[a] / An;
  }
}

__global__ void k_cell_geometry_fan(int nlf, int nfv, int Q, int QC, int maxtets, int64_t nc,
                                    Gauss g, const double* __restrict__ x,
                                    const int32_t* __restrict__ fnodes,
                                    const int64_t* __restrict__ cf,
                                    const int32_t* __restrict__ fown,
                                    const double* __restrict__ xq, const double* __restrict__ aq,
                                    double* xc, double* vol, double* cqx, double* cqw) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double V = 0, M2[3] = {0, 0, 0}, xb[3] = {0, 0, 0};
  int nfc = 0;
  for (int lf = 0; lf < nlf; ++lf) {
    const int64_t f = cf[c * nlf + lf];
    if (f < 0) continue;
    const double sg = fown[f] == c ? 1.0 : -1.0;
    for (int q = 0; q < Q; ++q)
      for (int a = 0; a < 3; ++a) {
        const double xv = xq[(f * Q + q) * 3 + a], av = sg * aq[(f * Q + q) * 3 + a];
        V += xv * av;
        M2[a] += xv * xv * av;
      }
    double cb[3];
    face_corners_fan(fnodes + f * nfv, nfv, x, cb);
    for (int a = 0; a < 3; ++a) xb[a] += cb[a];
    ++nfc;
  }
  V /= 3;
  vol[c] = V;
  for (int a = 0; a < 3; ++a) xc[3 * c + a] = M2[a] / (2.0 * V);
  for (int a = 0; a < 3; ++a) xb[a] /= nfc;
  const int n3 = g.n * g.n * g.n;
  int slot = 0;
  for (int lf = 0; lf < nlf; ++lf) {
    const int64_t f = cf[c * nlf + lf];
    if (f < 0) continue;
    const int32_t* fn = fnodes + f * nfv;
    double cb[3];
    const int k = face_corners_fan(fn, nfv, x, cb);
    for (int t = 0; t < k && slot < maxtets; ++t, ++slot) {
      const int32_t v0 = fn[t], v1 = fn[(t + 1) % k];
      double P[8][3];
      for (int a = 0; a < 3; ++a) {
        P[0][a] = P[3][a] = P[4][a] = P[7][a] = xb[a];
        P[1][a] = P[5][a] = cb[a];
        P[2][a] = x[3 * (int64_t)v0 + a];
        P[6][a] = x[3 * (int64_t)v1 + a];
      }
      hex_cell_points(g, P, cqx + (c * QC + slot * n3) * 3, cqw + c * QC + slot * n3);
    }
  }
  for (; slot < maxtets; ++slot)
    for (int q = 0; q < n3; ++q) {
      for (int a = 0; a < 3; ++a) cqx[(c * QC + slot * n3 + q) * 3 + a] = xb[a];
      cqw[c * QC + slot * n3 + q] = 0.0;
    }
}

static Gauss make_gauss(const hofv_ctx* c) {
  Gauss g;
  g.n = c->q1;
  for (int i = 0; i < 4; ++i) {
    g.x[i] = c->gl_x[i];
    g.w[i] = c->gl_w[i];
  }
  return g;
}

int run_geometry(hofv_ctx* c) {
  Gauss g = make_gauss(c);
  const int T = 128;
  if (c->polyh) {
    k_face_geometry_fan<<<(unsigned)((c->nf + T - 1) / T), T, 0, c->stream>>>(
        c->nfv, c->Q, c->nf, g, c->d_x, c->d_fnodes, c->d_xq, c->d_aq, c->d_xf, c->d_nrm,
        c->d_gam);
    HOFV_CUDA(c, cudaGetLastError());
    k_cell_geometry_fan<<<(unsigned)((c->nc + T - 1) / T), T, 0, c->stream>>>(
        c->nlf, c->nfv, c->Q, c->QC, c->maxtets, c->nc, g, c->d_x, c->d_fnodes, c->d_cf,
        c->d_fown, c->d_xq, c->d_aq, c->d_xc, c->d_vol, c->d_cqx, c->d_cqw);
    HOFV_CUDA(c, cudaGetLastError());
    HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
    return 0;
  }
  k_face_geometry<<<(unsigned)((c->nf + T - 1) / T), T, 0, c->stream>>>(
      c->dim, c->nfv, c->Q, c->nf, g, c->d_x, c->d_fnodes, c->d_xq, c->d_aq, c->d_xf, c->d_nrm,
      c->d_gam);
  HOFV_CUDA(c, cudaGetLastError());
  k_cell_geometry<<<(unsigned)((c->nc + T - 1) / T), T, 0, c->stream>>>(
      c->dim, c->simplex, c->poly, c->nv, c->nlf, c->nfv, c->Q, c->QC, c->nc, g, c->d_x, c->d_cnodes, c->d_xc,
      c->d_vol, c->d_cqx, c->d_cqw);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

}  // namespace hofv
