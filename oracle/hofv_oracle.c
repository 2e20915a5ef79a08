/*
 * hofv_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file;
 * only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no code, header or table with the CUDA library.
 *
 * It restates, step by step, the high-order cell-centred finite-volume
 * discretisation of Batistic, Castrillo & Cardiff (arXiv 2601.18417):
 *   - face / cell geometry and Gaussian quadrature        (Sec. 3.1-3.3)
 *   - nearest-neighbour stencils                          (Sec. 3.5.2)
 *   - least-squares Taylor reconstruction, eqs. (te)-(lsA), weight (weightFunc)
 *   - displacement-boundary ghost node                    (Sec. 3.5.3)
 *   - face-qp gradients, eq. (faceQuadGrad)               (Sec. 3.5.4)
 *   - linear elastic and neo-Hookean laws                 (App. A)
 *   - surface quadrature of the traction, eq. (divStressDiscret)
 *   - alpha stabilisation, eqs. (alpha), (alphaJump), App. B
 *   - residual R(u) and the compact approximate Jacobian  (Sec. 4.1)
 *
 * Conventions shared with the library only through the documented API:
 *   grad[i][j] = d u_j / d x_i  (the paper writes grad u = sum c (x) u);
 *   vectors are component-major: u[j*n_cells + cell];
 *   internal faces are ordered by (owner, owner local face), owner < neighbour;
 *   boundary faces follow: displacement, symmetry, then traction faces, each
 *   in input order; local faces of a quad / hex are x-, x+, y-, y+ (, z-,
 *   z+), local face k of a triangle joins nodes k and k+1 mod 3, local face
 *   k of a tetrahedron lies opposite node 3 - k, local face k of a polygon
 *   joins corners k and k+1 (8 slots per polygon, -1 past its last side).
 *
 * Readings of the paper taken here (the paper is silent or its setting differs):
 *   - faces are bilinear patches with tensor Gauss-Legendre points; each point
 *     carries its own vector area (the paper fan-triangulates planar faces);
 *     a triangular face is the patch with a repeated corner and a triangle
 *     or tetrahedron cell the collapsed square / cube (Duffy's map), so the
 *     same tensor rules serve unstructured simplex meshes; a polygon cell is
 *     the fan of triangles from its corners' average, each so collapsed; a
 *     polyhedron's polygonal face is the fan of triangles from its corners'
 *     average and its cell rule the fan of tetrahedra from the average of
 *     its face averages (the paper's fan triangulation and tetrahedral
 *     decomposition, with collapsed tensor rules instead of Dunavant's);
 *   - stencil ties are broken by a quantised squared distance (quantum
 *     2^-24 of the squared reference cell size) then by cell id;
 *   - the reconstruction is solved from the normal equations, eq. (maQw), in
 *     extended precision (the paper uses Householder QR; the result is the same
 *     in exact arithmetic).
 *
 * Compile with -ffp-contract=off so that squared distances round exactly as
 * written.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long double ld;

/* ------------------------------------------------------------------ */
/* mesh object                                                         */
/* ------------------------------------------------------------------ */
typedef struct {
  int dim, simplex, poly, polyh, nv, nlf, nfv;
  int maxtets;     /* polyhedra: most fan tetrahedra of one cell */
  int64_t nn, nc, nb;
  double *x;       /* [nn][3] */
  int64_t *cn;     /* [nc][nv]; polygons: corners, -1 past the last */
  int *cnv;        /* polygons: [nc] number of corners (= sides) */
  /* faces */
  int64_t nf, nfi, nfd, nfy, nft;
  int64_t *fown, *fnei;
  int *flf, *ftag; /* owner local face; -1 internal, 0 disp, 1 traction, 2 symmetry */
  int64_t *fnodes; /* [nf][nfv] in the owner's outward order (polyhedra: -1 past the last) */
  int *fcnt;       /* polyhedra: [nf] corners of each face */
  int64_t *cf;     /* [nc][nlf] face id of each local face */
  /* scheme */
  int have_scheme, p, nplus, q1, S, Nt, Q, QC;
  double kw, alpha;
  /* geometry */
  int have_geom;
  double *xc, *vol;        /* [nc][3], [nc] */
  double *xq, *aq;         /* [nf][Q][3] */
  double *xf, *nrm, *gam;  /* [nf][3], [nf][3], [nf] */
  double *cqx, *cqw;       /* [nc][QC][3], [nc][QC] */
  double gl_x[8], gl_w[8];
  int href_exp;
  /* subset data */
  int64_t *fslot, *cslot;  /* -1 if not prepared */
  int64_t nfs, ncs;
  int64_t *fst;            /* [nfs][S] */
  double *fco;             /* [nfs][Q][S+1][3]  (slot S: ghost node) */
  double *fcond;           /* [nfs][Q] */
  int64_t *cst;            /* [ncs][S] */
  double *cex;             /* [ncs][nlf][S] */
  double *ccond;           /* [ncs] */
} orc_mesh;

/* local faces of a quad (nodes counter-clockwise) and of a hex, as node
   positions within the cell, ordered so the normal points outward */
static const int QUAD_LF[4][2] = {{3, 0}, {1, 2}, {0, 1}, {2, 3}};
static const int HEX_LF[6][4] = {{0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4},
                                 {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};

/* local faces of a triangle (nodes counter-clockwise) and of a tetrahedron
   (positive orientation: (x1-x0) . ((x2-x0) x (x3-x0)) > 0), outward order;
   local face k of a tetrahedron is the one opposite node 3 - k */
static const int TRI_LF[3][2] = {{0, 1}, {1, 2}, {2, 0}};
static const int TET_LF[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};

static int lf_node(const orc_mesh* m, int lf, int k) {
  if (m->simplex) return m->dim == 2 ? TRI_LF[lf][k] : TET_LF[lf][k];
  return m->dim == 2 ? QUAD_LF[lf][k] : HEX_LF[lf][k];
}

/* a polygon has as many local faces as corners; local face k runs from
   corner k to corner k+1.  Slots past the last side hold no face. */
#define POLY_MAX_SIDES 8

static int face_exists(const orc_mesh* m, int64_t c, int lf) {
  return !m->poly || lf < m->cnv[c];
}

/* node k of local face lf of cell c (the face must exist) */
static int64_t cell_face_node(const orc_mesh* m, int64_t c, int lf, int k) {
  if (m->poly) return m->cn[c * m->nv + (lf + k) % m->cnv[c]];
  return m->cn[c * m->nv + lf_node(m, lf, k)];
}

/* corner coordinates [4][3] of a face for face_quadrature: a triangle is
   the bilinear patch whose fourth corner coincides with its first, i.e.
   the collapsed square of Duffy's transformation */
static void face_corners(const orc_mesh* m, const int64_t* nodes, double* corner) {
  for (int k = 0; k < m->nfv; ++k)
    for (int a = 0; a < 3; ++a) corner[3 * k + a] = m->x[3 * nodes[k] + a];
  if (m->dim == 3 && m->nfv == 3)
    for (int a = 0; a < 3; ++a) corner[9 + a] = corner[a];
}

/* node ids of the bilinear / trilinear map of cell c: a quad or hex as
   given; a triangle or tetrahedron as the degenerate quad (0,1,2,0) or hex
   (0,1,2,0, 0,1,3,0), which is the collapsed-cube (Duffy) map
   x = x0 + s (x1 - x0) + s t (x2 - x1) [+ s t r (x3 - x2)] */
static void cell_map_nodes(const orc_mesh* m, int64_t c, int64_t* out) {
  static const int TRI_MAP[4] = {0, 1, 2, 0};
  static const int TET_MAP[8] = {0, 1, 2, 0, 0, 1, 3, 0};
  const int64_t* cn = m->cn + c * m->nv;
  int n = m->dim == 2 ? 4 : 8;
  for (int k = 0; k < n; ++k)
    out[k] = !m->simplex ? cn[k] : cn[m->dim == 2 ? TRI_MAP[k] : TET_MAP[k]];
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rules on [0,1] (closed forms of the 1..4 point rules) */
/* ------------------------------------------------------------------ */
int orc_gauss_legendre(int n, double* x, double* w) {
  double t[4], c[4];
  if (n == 1) {
    t[0] = 0.0; c[0] = 2.0;
  } else if (n == 2) {
    t[0] = -1.0 / sqrt(3.0); t[1] = -t[0]; c[0] = c[1] = 1.0;
  } else if (n == 3) {
    t[0] = -sqrt(3.0 / 5.0); t[1] = 0.0; t[2] = -t[0];
    c[0] = c[2] = 5.0 / 9.0; c[1] = 8.0 / 9.0;
  } else if (n == 4) {
    double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
    double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    t[0] = -b; t[1] = -a; t[2] = a; t[3] = b;
    c[1] = c[2] = (18.0 + sqrt(30.0)) / 36.0;
    c[0] = c[3] = (18.0 - sqrt(30.0)) / 36.0;
  } else {
    return -1;
  }
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (t[i] + 1.0);
    w[i] = 0.5 * c[i];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* construction and face extraction                                    */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t key[4];
  int64_t cell;
  int lf;
} face_rec;

static int cmp_key(const int64_t* a, const int64_t* b) {
  for (int i = 0; i < 4; ++i) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}
static int cmp_rec(const void* pa, const void* pb) {
  const face_rec* a = (const face_rec*)pa;
  const face_rec* b = (const face_rec*)pb;
  int c = cmp_key(a->key, b->key);
  if (c) return c;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  return a->lf - b->lf;
}
static void sorted_key(const int64_t* nodes, int n, int64_t* key) {
  int64_t t[4] = {-1, -1, -1, -1};
  for (int i = 0; i < n; ++i) t[i] = nodes[i];
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (t[j] < t[i]) { int64_t s = t[i]; t[i] = t[j]; t[j] = s; }
  for (int i = 0; i < 4; ++i) key[i] = t[i];
}

void orc_free(orc_mesh* m);

/* faces of the mesh from the cells' local faces: equal node sets pair up
   into internal faces, the rest must be the boundary list */
static orc_mesh* build_faces(orc_mesh* m, int64_t nb, const int64_t* bface_nodes,
                             const int* bface_tag) {
  int64_t nc = m->nc, nslot = nc * m->nlf, nrec = 0;
  for (int64_t c = 0; c < nc; ++c)
    for (int lf = 0; lf < m->nlf; ++lf) nrec += face_exists(m, c, lf);
  /* every local face of every cell, sorted by its node set */
  face_rec* rec = (face_rec*)malloc(sizeof(face_rec) * (nrec > 0 ? nrec : 1));
  int64_t r_ = 0;
  for (int64_t c = 0; c < nc; ++c)
    for (int lf = 0; lf < m->nlf; ++lf) {
      if (!face_exists(m, c, lf)) continue;
      int64_t nodes[4];
      for (int k = 0; k < m->nfv; ++k) nodes[k] = cell_face_node(m, c, lf, k);
      face_rec* r = &rec[r_++];
      sorted_key(nodes, m->nfv, r->key);
      r->cell = c;
      r->lf = lf;
    }
  qsort(rec, nrec, sizeof(face_rec), cmp_rec);
  /* partner of each local face slot c*nlf+lf: pairs of equal keys are internal faces */
  int64_t* partner = (int64_t*)malloc(sizeof(int64_t) * nslot);
  for (int64_t i = 0; i < nslot; ++i) partner[i] = -1;
  int ok = 1;
  for (int64_t i = 0; i + 1 < nrec; ++i)
    if (cmp_key(rec[i].key, rec[i + 1].key) == 0) {
      if (i + 2 < nrec && cmp_key(rec[i].key, rec[i + 2].key) == 0) ok = 0;
      partner[rec[i].cell * m->nlf + rec[i].lf] = rec[i + 1].cell * m->nlf + rec[i + 1].lf;
      partner[rec[i + 1].cell * m->nlf + rec[i + 1].lf] = rec[i].cell * m->nlf + rec[i].lf;
    }
  /* boundary faces: find the owning local face of each */
  int64_t* bown = (int64_t*)malloc(sizeof(int64_t) * (nb > 0 ? nb : 1));
  for (int64_t b = 0; b < nb && ok; ++b) {
    face_rec q;
    sorted_key(bface_nodes + b * m->nfv, m->nfv, q.key);
    int64_t lo = 0, hi = nrec - 1, hit = -1;
    while (lo <= hi) {
      int64_t mid = (lo + hi) / 2;
      int c = cmp_key(rec[mid].key, q.key);
      if (c == 0) { hit = mid; break; }
      if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    if (hit < 0) { ok = 0; break; }
    int64_t id = rec[hit].cell * m->nlf + rec[hit].lf;
    if (partner[id] >= 0) { ok = 0; break; }
    bown[b] = id;
  }
  int64_t nfi = 0, nbound = 0;
  for (int64_t i = 0; i < nslot; ++i) {
    if (!face_exists(m, i / m->nlf, (int)(i % m->nlf))) continue;
    if (partner[i] > i) ++nfi;
    if (partner[i] < 0) ++nbound;
  }
  if (nbound != nb) ok = 0;
  int64_t nfd = 0, nft = 0, nfy = 0;
  for (int64_t b = 0; b < nb; ++b) {
    if (bface_tag[b] == 0) ++nfd;
    else if (bface_tag[b] == 1) ++nft;
    else if (bface_tag[b] == 2) ++nfy;
    else ok = 0;
  }
  if (!ok) {
    free(rec); free(partner); free(bown); orc_free(m);
    return NULL;
  }
  m->nfi = nfi; m->nfd = nfd; m->nfy = nfy; m->nft = nft;
  m->nf = nfi + nfd + nfy + nft;
  m->fown = (int64_t*)malloc(sizeof(int64_t) * m->nf);
  m->fnei = (int64_t*)malloc(sizeof(int64_t) * m->nf);
  m->flf = (int*)malloc(sizeof(int) * m->nf);
  m->ftag = (int*)malloc(sizeof(int) * m->nf);
  m->fnodes = (int64_t*)malloc(sizeof(int64_t) * m->nf * m->nfv);
  m->cf = (int64_t*)malloc(sizeof(int64_t) * nslot);
  for (int64_t i = 0; i < nslot; ++i) m->cf[i] = -1;
  int64_t f = 0;
  for (int64_t c = 0; c < nc; ++c)
    for (int lf = 0; lf < m->nlf; ++lf) {
      int64_t id = c * m->nlf + lf, pid = partner[id];
      if (pid >= 0 && pid / m->nlf > c) {
        m->fown[f] = c; m->fnei[f] = pid / m->nlf; m->flf[f] = lf; m->ftag[f] = -1;
        m->cf[id] = f; m->cf[pid] = f;
        ++f;
      }
    }
  static const int ORDER[3] = {0, 2, 1};  /* displacement, symmetry, traction */
  for (int o = 0; o < 3; ++o)
    for (int64_t b = 0; b < nb; ++b)
      if (bface_tag[b] == ORDER[o]) {
        int tag = ORDER[o];
        int64_t id = bown[b];
        m->fown[f] = id / m->nlf; m->fnei[f] = -1; m->flf[f] = (int)(id % m->nlf);
        m->ftag[f] = tag; m->cf[id] = f;
        ++f;
      }
  for (f = 0; f < m->nf; ++f)
    for (int k = 0; k < m->nfv; ++k)
      m->fnodes[f * m->nfv + k] = cell_face_node(m, m->fown[f], m->flf[f], k);
  free(rec); free(partner); free(bown);
  return m;
}

/* simplex = 0: quads / hexes; 1: triangles / tetrahedra */
orc_mesh* orc_create_cells(int dim, int simplex, int64_t nn, const double* xyz, int64_t nc,
                           const int64_t* cell_nodes, int64_t nb,
                           const int64_t* bface_nodes, const int* bface_tag) {
  if (dim != 2 && dim != 3) return NULL;
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  m->dim = dim;
  m->simplex = simplex ? 1 : 0;
  m->nv = simplex ? dim + 1 : (dim == 2 ? 4 : 8);
  m->nlf = simplex ? dim + 1 : 2 * dim;
  m->nfv = simplex ? dim : (dim == 2 ? 2 : 4);
  m->nn = nn; m->nc = nc; m->nb = nb;
  m->x = (double*)calloc((size_t)nn * 3, sizeof(double));
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < dim; ++a) m->x[3 * i + a] = xyz[dim * i + a];
  m->cn = (int64_t*)malloc(sizeof(int64_t) * nc * m->nv);
  memcpy(m->cn, cell_nodes, sizeof(int64_t) * nc * m->nv);
  return build_faces(m, nb, bface_nodes, bface_tag);
}

/* 2-D polygons (counter-clockwise corners, 3..POLY_MAX_SIDES of them):
   cell c has corners cell_nodes[cell_ptr[c] .. cell_ptr[c+1]) */
orc_mesh* orc_create_poly(int64_t nn, const double* xyz, int64_t nc, const int64_t* cell_ptr,
                          const int64_t* cell_nodes, int64_t nb, const int64_t* bface_nodes,
                          const int* bface_tag) {
  for (int64_t c = 0; c < nc; ++c) {
    int64_t k = cell_ptr[c + 1] - cell_ptr[c];
    if (k < 3 || k > POLY_MAX_SIDES) return NULL;
  }
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  m->dim = 2;
  m->poly = 1;
  m->nv = m->nlf = POLY_MAX_SIDES;
  m->nfv = 2;
  m->nn = nn; m->nc = nc; m->nb = nb;
  m->x = (double*)calloc((size_t)nn * 3, sizeof(double));
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < 2; ++a) m->x[3 * i + a] = xyz[2 * i + a];
  m->cn = (int64_t*)malloc(sizeof(int64_t) * nc * m->nv);
  m->cnv = (int*)malloc(sizeof(int) * nc);
  for (int64_t c = 0; c < nc; ++c) {
    m->cnv[c] = (int)(cell_ptr[c + 1] - cell_ptr[c]);
    for (int k = 0; k < m->nv; ++k)
      m->cn[c * m->nv + k] = k < m->cnv[c] ? cell_nodes[cell_ptr[c] + k] : -1;
  }
  return build_faces(m, nb, bface_nodes, bface_tag);
}

orc_mesh* orc_create(int dim, int64_t nn, const double* xyz, int64_t nc,
                     const int64_t* cell_nodes, int64_t nb,
                     const int64_t* bface_nodes, const int* bface_tag) {
  return orc_create_cells(dim, 0, nn, xyz, nc, cell_nodes, nb, bface_nodes, bface_tag);
}

void orc_free_subset(orc_mesh* m) {
  free(m->fslot); free(m->cslot); free(m->fst); free(m->fco); free(m->fcond);
  free(m->cst); free(m->cex); free(m->ccond);
  m->fslot = m->cslot = m->fst = m->cst = NULL;
  m->fco = m->fcond = m->cex = m->ccond = NULL;
  m->nfs = m->ncs = 0;
}

void orc_free(orc_mesh* m) {
  if (!m) return;
  free(m->x); free(m->cn); free(m->cnv); free(m->fcnt); free(m->fown); free(m->fnei); free(m->flf); free(m->ftag);
  free(m->fnodes); free(m->cf); free(m->xc); free(m->vol); free(m->xq); free(m->aq);
  free(m->xf); free(m->nrm); free(m->gam); free(m->cqx); free(m->cqw);
  orc_free_subset(m);
  free(m);
}

void orc_counts(const orc_mesh* m, int64_t* out) {
  out[0] = m->nf; out[1] = m->nfi; out[2] = m->nfd; out[3] = m->nft;
  out[4] = m->nc; out[5] = m->Q; out[6] = m->S; out[7] = m->QC; out[8] = m->nfy;
}

int orc_set_scheme(orc_mesh* m, int p, int nplus, int q1, double kw, double alpha) {
  if (p < 1 || p > 3 || q1 < 1 || q1 > 4 || nplus < 0) return -1;
  m->p = p; m->nplus = nplus; m->q1 = q1; m->kw = kw; m->alpha = alpha;
  int nt = 1;
  for (int i = 1; i <= m->dim; ++i) nt = nt * (p + i) / i;   /* C(d+p, d) */
  m->Nt = nt;
  m->S = nt + nplus;
  m->Q = m->polyh ? m->nfv * q1 * q1 : m->dim == 2 ? q1 : q1 * q1;
  m->QC = m->polyh ? m->maxtets * q1 * q1 * q1
        : m->poly ? m->nlf * q1 * q1 : m->dim == 2 ? q1 * q1 : q1 * q1 * q1;
  if (m->S > m->nc) return -2;
  orc_gauss_legendre(q1, m->gl_x, m->gl_w);
  m->have_scheme = 1;
  m->have_geom = 0;
  orc_free_subset(m);
  return 0;
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* quadrature points and vector-area elements of one face given its corner
   coordinates in outward order (Sec. 3.2, surface quadrature) */
static void face_quadrature(const orc_mesh* m, const double* corner /*[nfv][3]*/,
                            double* xq, double* aq) {
  int n = m->q1;
  if (m->dim == 2) {
    const double* c0 = corner;
    const double* c1 = corner + 3;
    double t[3] = {c1[0] - c0[0], c1[1] - c0[1], 0.0};
    for (int a = 0; a < n; ++a) {
      double s = m->gl_x[a];
      for (int k = 0; k < 3; ++k) xq[3 * a + k] = (1.0 - s) * c0[k] + s * c1[k];
      aq[3 * a + 0] = m->gl_w[a] * t[1];
      aq[3 * a + 1] = -m->gl_w[a] * t[0];
      aq[3 * a + 2] = 0.0;
    }
    return;
  }
  const double *c0 = corner, *c1 = corner + 3, *c2 = corner + 6, *c3 = corner + 9;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double xi = m->gl_x[a], eta = m->gl_x[b];
      int q = a * n + b;
      double xs[3], xe[3], cr[3];
      for (int k = 0; k < 3; ++k) {
        xq[3 * q + k] = (1 - xi) * (1 - eta) * c0[k] + xi * (1 - eta) * c1[k] +
                        xi * eta * c2[k] + (1 - xi) * eta * c3[k];
        xs[k] = (1 - eta) * (c1[k] - c0[k]) + eta * (c2[k] - c3[k]);
        xe[k] = (1 - xi) * (c3[k] - c0[k]) + xi * (c2[k] - c1[k]);
      }
      cross3(xs, xe, cr);
      double w = m->gl_w[a] * m->gl_w[b];
      for (int k = 0; k < 3; ++k) aq[3 * q + k] = w * cr[k];
    }
}

/* Gauss points and weights of the bilinear map of the quad with corners
   P (counter-clockwise; a repeated corner collapses it to a triangle) */
static void quad_rule(const orc_mesh* m, const double P[4][2], double* cqx, double* cqw) {
  static const double R2[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
  int n = m->q1;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double s[2] = {m->gl_x[a], m->gl_x[b]};
      double X2[3] = {0, 0, 0}, J[2][2] = {{0, 0}, {0, 0}};
      for (int k = 0; k < 4; ++k) {
        double f0 = R2[k][0] ? s[0] : 1 - s[0], f1 = R2[k][1] ? s[1] : 1 - s[1];
        double d0 = R2[k][0] ? 1 : -1, d1 = R2[k][1] ? 1 : -1;
        double N = f0 * f1, dN0 = d0 * f1, dN1 = f0 * d1;
        for (int e = 0; e < 2; ++e) {
          double xv = P[k][e];
          X2[e] += N * xv;
          J[e][0] += dN0 * xv;
          J[e][1] += dN1 * xv;
        }
      }
      double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      int q = a * n + b;
      for (int e = 0; e < 3; ++e) cqx[q * 3 + e] = X2[e];
      cqw[q] = m->gl_w[a] * m->gl_w[b] * fabs(det);
    }
}

/* Gauss points and weights of the trilinear map of the hex with corners P
   (repeated corners collapse it to a tetrahedron) */
static void hex_rule(const orc_mesh* m, const double P[8][3], double* cqx, double* cqw) {
  static const double R3[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                  {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  int n = m->q1;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int g = 0; g < n; ++g) {
        double s[3] = {m->gl_x[a], m->gl_x[b], m->gl_x[g]};
        double X3[3] = {0, 0, 0}, J[3][3] = {{0}};
        for (int k = 0; k < 8; ++k) {
          double fct[3], dr[3];
          for (int e = 0; e < 3; ++e) {
            fct[e] = R3[k][e] ? s[e] : 1 - s[e];
            dr[e] = R3[k][e] ? 1 : -1;
          }
          double N = fct[0] * fct[1] * fct[2];
          double dN[3] = {dr[0] * fct[1] * fct[2], fct[0] * dr[1] * fct[2],
                          fct[0] * fct[1] * dr[2]};
          for (int e = 0; e < 3; ++e) {
            double xv = P[k][e];
            X3[e] += N * xv;
            for (int r = 0; r < 3; ++r) J[e][r] += dN[r] * xv;
          }
        }
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        int q = (a * n + b) * n + g;
        for (int e = 0; e < 3; ++e) cqx[q * 3 + e] = X3[e];
        cqw[q] = m->gl_w[a] * m->gl_w[b] * m->gl_w[g] * fabs(det);
      }
}

/* reference length for the stencil tie key: a power of two near the mean
   cell size, from the node bounding box */
static void set_href(orc_mesh* m) {
  int d = m->dim;
  double vbox = 1.0;
  for (int a = 0; a < d; ++a) {
    double lo = m->x[a], hi = m->x[a];
    for (int64_t i = 1; i < m->nn; ++i) {
      double v = m->x[3 * i + a];
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
    vbox *= (hi - lo);
  }
  int e = ilogb(vbox / (double)m->nc);
  m->href_exp = e >= 0 ? e / d : -((-e + d - 1) / d); /* floor(e / d) */
}

static int geometry_polyhedra(orc_mesh* m);

int orc_geometry(orc_mesh* m) {
  if (!m->have_scheme) return -1;
  int d = m->dim, Q = m->Q, nfv = m->nfv;
  free(m->xc); free(m->vol); free(m->xq); free(m->aq); free(m->xf); free(m->nrm);
  free(m->gam); free(m->cqx); free(m->cqw);
  m->xc = (double*)calloc(m->nc * 3, sizeof(double));
  m->vol = (double*)calloc(m->nc, sizeof(double));
  m->xq = (double*)calloc(m->nf * Q * 3, sizeof(double));
  m->aq = (double*)calloc(m->nf * Q * 3, sizeof(double));
  m->xf = (double*)calloc(m->nf * 3, sizeof(double));
  m->nrm = (double*)calloc(m->nf * 3, sizeof(double));
  m->gam = (double*)calloc(m->nf, sizeof(double));
  m->cqx = (double*)calloc(m->nc * m->QC * 3, sizeof(double));
  m->cqw = (double*)calloc(m->nc * m->QC, sizeof(double));
  double corner[12], xq[16 * 3], aq[16 * 3];
  if (m->polyh) return geometry_polyhedra(m);
  /* faces */
  for (int64_t f = 0; f < m->nf; ++f) {
    face_corners(m, m->fnodes + f * nfv, corner);
    face_quadrature(m, corner, m->xq + f * Q * 3, m->aq + f * Q * 3);
    double G = 0, A[3] = {0, 0, 0}, X[3] = {0, 0, 0};
    for (int q = 0; q < Q; ++q) {
      const double* a = m->aq + (f * Q + q) * 3;
      double mag = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      G += mag;
      for (int k = 0; k < 3; ++k) {
        A[k] += a[k];
        X[k] += mag * m->xq[(f * Q + q) * 3 + k];
      }
    }
    double An = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    m->gam[f] = G;
    for (int k = 0; k < 3; ++k) {
      m->xf[3 * f + k] = X[k] / G;
      m->nrm[3 * f + k] = A[k] / An;
    }
  }
  /* cells: volume and centroid from the divergence theorem over the cell's
     own outward faces, with the same face quadrature */
  for (int64_t c = 0; c < m->nc; ++c) {
    double V = 0, M2[3] = {0, 0, 0};
    for (int lf = 0; lf < m->nlf; ++lf) {
      if (!face_exists(m, c, lf)) continue;
      int64_t fn[4];
      for (int k = 0; k < nfv; ++k) fn[k] = cell_face_node(m, c, lf, k);
      face_corners(m, fn, corner);
      face_quadrature(m, corner, xq, aq);
      for (int q = 0; q < Q; ++q)
        for (int a = 0; a < d; ++a) {
          V += xq[3 * q + a] * aq[3 * q + a];
          M2[a] += xq[3 * q + a] * xq[3 * q + a] * aq[3 * q + a];
        }
    }
    V /= d;
    m->vol[c] = V;
    for (int a = 0; a < d; ++a) m->xc[3 * c + a] = M2[a] / (2.0 * V);
    /* cell quadrature for volume integrals (tensor Gauss on the
       bilinear / trilinear map), eq. (bodyTerm) */
    int n = m->q1;
    int64_t cn[8];
    if (m->poly) {
      /* fan of triangles (xbar, corner t, corner t+1) from the corners'
         average, each on the collapsed square; unused slots weigh zero */
      double xb[2] = {0, 0};
      int k = m->cnv[c];
      for (int t = 0; t < k; ++t)
        for (int e = 0; e < 2; ++e) xb[e] += m->x[3 * m->cn[c * m->nv + t] + e];
      for (int e = 0; e < 2; ++e) xb[e] /= k;
      for (int t = 0; t < m->nlf; ++t) {
        double* qx = m->cqx + (c * m->QC + t * n * n) * 3;
        double* qw = m->cqw + c * m->QC + t * n * n;
        if (t >= k) {
          for (int q = 0; q < n * n; ++q) {
            qx[3 * q] = xb[0]; qx[3 * q + 1] = xb[1]; qx[3 * q + 2] = 0.0;
            qw[q] = 0.0;
          }
          continue;
        }
        const double* v0 = m->x + 3 * m->cn[c * m->nv + t];
        const double* v1 = m->x + 3 * m->cn[c * m->nv + (t + 1) % k];
        double P4[4][2] = {{xb[0], xb[1]}, {v0[0], v0[1]}, {v1[0], v1[1]}, {xb[0], xb[1]}};
        quad_rule(m, P4, qx, qw);
      }
    } else if (d == 2) {
      cell_map_nodes(m, c, cn);
      double P4[4][2];
      for (int k = 0; k < 4; ++k)
        for (int e = 0; e < 2; ++e) P4[k][e] = m->x[3 * cn[k] + e];
      quad_rule(m, P4, m->cqx + c * m->QC * 3, m->cqw + c * m->QC);
    } else {
      cell_map_nodes(m, c, cn);
      double P8[8][3];
      for (int k = 0; k < 8; ++k)
        for (int e = 0; e < 3; ++e) P8[k][e] = m->x[3 * cn[k] + e];
      hex_rule(m, P8, m->cqx + c * m->QC * 3, m->cqw + c * m->QC);
    }
  }
  set_href(m);
  m->have_geom = 1;
  return 0;
}

/* Polyhedra (faces given as polygons): each face is the fan of triangles
   from its corners' average cbar_f to its sides, each triangle the bilinear
   patch (cbar_f, v_t, v_t+1, cbar_f) with q1 x q1 points (Q = nfv q1^2, zero
   area past a face's last side).  Volume and centroid by the divergence
   theorem over those points, each face counted outward; the cell rule is
   the fan of tetrahedra (xbar_c, cbar_f, v_t, v_t+1) from the average xbar_c
   of the cell's face averages, each the collapsed cube (q1^3 points). */
static int geometry_polyhedra(orc_mesh* m) {
  int Q = m->Q, n2 = m->q1 * m->q1, n3 = n2 * m->q1;
  double* cbar = (double*)calloc(m->nf * 3, sizeof(double));
  for (int64_t f = 0; f < m->nf; ++f) {
    int k = m->fcnt[f];
    const int64_t* fn = m->fnodes + f * m->nfv;
    double* cb = cbar + 3 * f;
    for (int t = 0; t < k; ++t)
      for (int e = 0; e < 3; ++e) cb[e] += m->x[3 * fn[t] + e];
    for (int e = 0; e < 3; ++e) cb[e] /= k;
    for (int t = 0; t < m->nfv; ++t) {
      double* xq = m->xq + (f * Q + t * n2) * 3;
      double* aq = m->aq + (f * Q + t * n2) * 3;
      if (t >= k) {
        for (int q = 0; q < n2; ++q)
          for (int e = 0; e < 3; ++e) { xq[3 * q + e] = cb[e]; aq[3 * q + e] = 0.0; }
        continue;
      }
      double corner[12];
      for (int e = 0; e < 3; ++e) {
        corner[e] = cb[e];
        corner[3 + e] = m->x[3 * fn[t] + e];
        corner[6 + e] = m->x[3 * fn[(t + 1) % k] + e];
        corner[9 + e] = cb[e];
      }
      face_quadrature(m, corner, xq, aq);
    }
    double G = 0, A[3] = {0, 0, 0}, X[3] = {0, 0, 0};
    for (int q = 0; q < Q; ++q) {
      const double* a = m->aq + (f * Q + q) * 3;
      double mag = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      G += mag;
      for (int e = 0; e < 3; ++e) {
        A[e] += a[e];
        X[e] += mag * m->xq[(f * Q + q) * 3 + e];
      }
    }
    double An = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    m->gam[f] = G;
    for (int e = 0; e < 3; ++e) {
      m->xf[3 * f + e] = X[e] / G;
      m->nrm[3 * f + e] = A[e] / An;
    }
  }
  for (int64_t c = 0; c < m->nc; ++c) {
    double V = 0, M2[3] = {0, 0, 0}, xb[3] = {0, 0, 0};
    int nfc = 0;
    for (int lf = 0; lf < m->nlf; ++lf) {
      int64_t f = m->cf[c * m->nlf + lf];
      if (f < 0) continue;
      double sg = m->fown[f] == c ? 1.0 : -1.0;
      for (int q = 0; q < Q; ++q)
        for (int a = 0; a < 3; ++a) {
          const double xv = m->xq[(f * Q + q) * 3 + a], av = sg * m->aq[(f * Q + q) * 3 + a];
          V += xv * av;
          M2[a] += xv * xv * av;
        }
      for (int e = 0; e < 3; ++e) xb[e] += cbar[3 * f + e];
      ++nfc;
    }
    V /= 3;
    m->vol[c] = V;
    for (int a = 0; a < 3; ++a) m->xc[3 * c + a] = M2[a] / (2.0 * V);
    for (int e = 0; e < 3; ++e) xb[e] /= nfc;
    int slot = 0;
    for (int lf = 0; lf < m->nlf; ++lf) {
      int64_t f = m->cf[c * m->nlf + lf];
      if (f < 0) continue;
      int k = m->fcnt[f];
      const int64_t* fn = m->fnodes + f * m->nfv;
      for (int t = 0; t < k; ++t, ++slot) {
        double P8[8][3];
        for (int e = 0; e < 3; ++e) {
          P8[0][e] = P8[3][e] = P8[4][e] = P8[7][e] = xb[e];
          P8[1][e] = P8[5][e] = cbar[3 * f + e];
          P8[2][e] = m->x[3 * fn[t] + e];
          P8[6][e] = m->x[3 * fn[(t + 1) % k] + e];
        }
        hex_rule(m, P8, m->cqx + (c * m->QC + slot * n3) * 3, m->cqw + c * m->QC + slot * n3);
      }
    }
    for (; slot < m->maxtets; ++slot)
      for (int q = 0; q < n3; ++q) {
        for (int e = 0; e < 3; ++e) m->cqx[(c * m->QC + slot * n3 + q) * 3 + e] = xb[e];
        m->cqw[c * m->QC + slot * n3 + q] = 0.0;
      }
  }
  free(cbar);
  set_href(m);
  m->have_geom = 1;
  return 0;
}

/* 3-D polyhedra from a face list (the polyMesh layout): face i has corners
   face_nodes[face_ptr[i] .. face_ptr[i+1]) (3..8 of them), its normal by the
   right-hand rule pointing out of owner[i]; neighbour[i] = -1 and
   face_tag[i] in {0, 1, 2} on the boundary.  A cell's local faces are its
   faces in input order; internal faces are renumbered by (owner, local face)
   with owner < neighbour (a face is flipped where needed), boundary faces
   follow by tag (displacement, symmetry, traction), each in input order. */
orc_mesh* orc_create_faces(int64_t nn, const double* xyz, int64_t nc, int64_t nfin,
                           const int64_t* face_ptr, const int64_t* face_nodes,
                           const int64_t* owner, const int64_t* neighbour, const int* face_tag) {
  int maxfv = 0;
  for (int64_t i = 0; i < nfin; ++i) {
    int64_t k = face_ptr[i + 1] - face_ptr[i];
    if (k < 3 || k > POLY_MAX_SIDES) return NULL;
    if (owner[i] < 0 || owner[i] >= nc || neighbour[i] >= nc || neighbour[i] == owner[i]) return NULL;
    if (neighbour[i] < 0 && (face_tag[i] < 0 || face_tag[i] > 2)) return NULL;
    if (k > maxfv) maxfv = (int)k;
  }
  int* nfc = (int*)calloc(nc, sizeof(int));
  for (int64_t i = 0; i < nfin; ++i) {
    nfc[owner[i]]++;
    if (neighbour[i] >= 0) nfc[neighbour[i]]++;
  }
  int maxf = 0;
  for (int64_t c = 0; c < nc; ++c) {
    if (nfc[c] < 4) { free(nfc); return NULL; }
    if (nfc[c] > maxf) maxf = nfc[c];
  }
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  m->dim = 3;
  m->polyh = 1;
  m->nlf = maxf;
  m->nfv = maxfv;
  m->nv = 0;
  m->nn = nn; m->nc = nc;
  m->x = (double*)calloc((size_t)nn * 3, sizeof(double));
  for (int64_t i = 0; i < nn * 3; ++i) m->x[i] = xyz[i];
  /* orientation: owner the lower id */
  int64_t* own = (int64_t*)malloc(sizeof(int64_t) * nfin);
  int64_t* nei = (int64_t*)malloc(sizeof(int64_t) * nfin);
  int* flip = (int*)calloc(nfin, sizeof(int));
  for (int64_t i = 0; i < nfin; ++i) {
    own[i] = owner[i]; nei[i] = neighbour[i];
    if (nei[i] >= 0 && nei[i] < own[i]) { own[i] = neighbour[i]; nei[i] = owner[i]; flip[i] = 1; }
  }
  /* local faces: each cell's faces in input order */
  int* fill = (int*)calloc(nc, sizeof(int));
  int* lf_own = (int*)malloc(sizeof(int) * nfin);
  int* lf_nei = (int*)malloc(sizeof(int) * nfin);
  for (int64_t i = 0; i < nfin; ++i) {
    lf_own[i] = fill[own[i]]++;
    lf_nei[i] = nei[i] >= 0 ? fill[nei[i]]++ : -1;
  }
  /* canonical order: internal by (owner, local face), then boundary by tag */
  int64_t nfi = 0, nfd = 0, nfy = 0, nft = 0;
  for (int64_t i = 0; i < nfin; ++i) {
    if (nei[i] >= 0) ++nfi;
    else if (face_tag[i] == 0) ++nfd;
    else if (face_tag[i] == 2) ++nfy;
    else ++nft;
  }
  m->nfi = nfi; m->nfd = nfd; m->nfy = nfy; m->nft = nft; m->nb = nfd + nfy + nft;
  m->nf = nfin;
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * nfin);
  int64_t f = 0;
  for (int64_t c = 0; c < nc; ++c)           /* internal, by owner then local face */
    for (int64_t i = 0; i < nfin; ++i)
      if (nei[i] >= 0 && own[i] == c) order[f++] = i;
  static const int ORDER[3] = {0, 2, 1};
  for (int o = 0; o < 3; ++o)
    for (int64_t i = 0; i < nfin; ++i)
      if (nei[i] < 0 && face_tag[i] == ORDER[o]) order[f++] = i;
  m->fown = (int64_t*)malloc(sizeof(int64_t) * m->nf);
  m->fnei = (int64_t*)malloc(sizeof(int64_t) * m->nf);
  m->flf = (int*)malloc(sizeof(int) * m->nf);
  m->ftag = (int*)malloc(sizeof(int) * m->nf);
  m->fcnt = (int*)malloc(sizeof(int) * m->nf);
  m->fnodes = (int64_t*)malloc(sizeof(int64_t) * m->nf * m->nfv);
  m->cf = (int64_t*)malloc(sizeof(int64_t) * nc * m->nlf);
  for (int64_t i = 0; i < nc * m->nlf; ++i) m->cf[i] = -1;
  for (f = 0; f < m->nf; ++f) {
    int64_t i = order[f];
    int k = (int)(face_ptr[i + 1] - face_ptr[i]);
    m->fown[f] = own[i]; m->fnei[f] = nei[i]; m->flf[f] = lf_own[i];
    m->ftag[f] = nei[i] >= 0 ? -1 : face_tag[i];
    m->fcnt[f] = k;
    for (int t = 0; t < m->nfv; ++t)
      m->fnodes[f * m->nfv + t] =
          t < k ? face_nodes[face_ptr[i] + (flip[i] ? k - 1 - t : t)] : -1;
    m->cf[own[i] * m->nlf + lf_own[i]] = f;
    if (nei[i] >= 0) m->cf[nei[i] * m->nlf + lf_nei[i]] = f;
  }
  m->maxtets = 0;
  for (int64_t c = 0; c < nc; ++c) {
    int t = 0;
    for (int lf = 0; lf < m->nlf; ++lf)
      if (m->cf[c * m->nlf + lf] >= 0) t += m->fcnt[m->cf[c * m->nlf + lf]];
    if (t > m->maxtets) m->maxtets = t;
  }
  free(nfc); free(own); free(nei); free(flip); free(fill); free(lf_own); free(lf_nei); free(order);
  return m;
}

/* accessors ---------------------------------------------------------- */
#define GETTER(name, field, count)                                        \
  void name(const orc_mesh* m, double* out) {                             \
    memcpy(out, m->field, sizeof(double) * (size_t)(count));              \
  }
GETTER(orc_get_xc, xc, m->nc * 3)
GETTER(orc_get_vol, vol, m->nc)
GETTER(orc_get_xq, xq, m->nf * m->Q * 3)
GETTER(orc_get_aq, aq, m->nf * m->Q * 3)
GETTER(orc_get_xf, xf, m->nf * 3)
GETTER(orc_get_nrm, nrm, m->nf * 3)
GETTER(orc_get_gam, gam, m->nf)
GETTER(orc_get_cqx, cqx, m->nc * m->QC * 3)
GETTER(orc_get_cqw, cqw, m->nc * m->QC)

void orc_get_faces(const orc_mesh* m, int64_t* own, int64_t* nei, int* lf, int* tag) {
  memcpy(own, m->fown, sizeof(int64_t) * m->nf);
  memcpy(nei, m->fnei, sizeof(int64_t) * m->nf);
  memcpy(lf, m->flf, sizeof(int) * m->nf);
  memcpy(tag, m->ftag, sizeof(int) * m->nf);
}
void orc_get_cell_faces(const orc_mesh* m, int64_t* cf) {
  memcpy(cf, m->cf, sizeof(int64_t) * m->nc * m->nlf);
}
int orc_href_exp(const orc_mesh* m) { return m->href_exp; }
int orc_nlf(const orc_mesh* m) { return m->nlf; }

/* ------------------------------------------------------------------ */
/* stencils (Sec. 3.5.2): the |S| cell centroids nearest to the         */
/* reference point, ties ordered by a quantised squared distance and    */
/* then by cell id.  Exhaustive search over all cells.                   */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t key, id;
} cand;
static int cmp_cand(const void* pa, const void* pb) {
  const cand* a = (const cand*)pa;
  const cand* b = (const cand*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->id < b->id ? -1 : (a->id > b->id);
}

static int64_t dist_key(const orc_mesh* m, const double* xr, int64_t cell) {
  double dx = m->xc[3 * cell] - xr[0];
  double dy = m->xc[3 * cell + 1] - xr[1];
  double d2 = dx * dx + dy * dy;
  if (m->dim == 3) {
    double dz = m->xc[3 * cell + 2] - xr[2];
    d2 = d2 + dz * dz;
  }
  double s = ldexp(d2, 24 - 2 * m->href_exp);
  return (int64_t)floor(s + 0.5);
}

/* uniform bucket grid over the centroids, used only to prune the
   exhaustive search: the result equals a sort of all cells */
typedef struct {
  int nb[3];
  double lo[3], bs;
  int64_t *start, *items;
} buckets;

static void build_buckets(const orc_mesh* m, buckets* B) {
  int d = m->dim;
  B->bs = ldexp(1.0, m->href_exp);
  int64_t total = 1;
  for (int a = 0; a < 3; ++a) {
    if (a >= d) { B->nb[a] = 1; B->lo[a] = 0; continue; }
    double lo = m->xc[a], hi = m->xc[a];
    for (int64_t c = 1; c < m->nc; ++c) {
      double v = m->xc[3 * c + a];
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
    B->lo[a] = lo;
    B->nb[a] = (int)floor((hi - lo) / B->bs) + 1;
    total *= B->nb[a];
  }
  B->start = (int64_t*)calloc(total + 1, sizeof(int64_t));
  B->items = (int64_t*)malloc(sizeof(int64_t) * m->nc);
  int64_t* bid = (int64_t*)malloc(sizeof(int64_t) * m->nc);
  for (int64_t c = 0; c < m->nc; ++c) {
    int64_t id = 0;
    for (int a = d - 1; a >= 0; --a) {
      int i = (int)floor((m->xc[3 * c + a] - B->lo[a]) / B->bs);
      if (i < 0) i = 0;
      if (i >= B->nb[a]) i = B->nb[a] - 1;
      id = id * B->nb[a] + i;
    }
    bid[c] = id;
    B->start[id + 1]++;
  }
  for (int64_t i = 0; i < total; ++i) B->start[i + 1] += B->start[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * total);
  for (int64_t i = 0; i < total; ++i) fill[i] = B->start[i];
  for (int64_t c = 0; c < m->nc; ++c) B->items[fill[bid[c]]++] = c;
  free(fill);
  free(bid);
}
static void free_buckets(buckets* B) { free(B->start); free(B->items); }

/* exhaustive version: sort every cell */
int orc_stencil_bruteforce(const orc_mesh* m, const double* xr, int64_t* out) {
  cand* all = (cand*)malloc(sizeof(cand) * m->nc);
  for (int64_t c = 0; c < m->nc; ++c) {
    all[c].key = dist_key(m, xr, c);
    all[c].id = c;
  }
  qsort(all, m->nc, sizeof(cand), cmp_cand);
  for (int i = 0; i < m->S; ++i) out[i] = all[i].id;
  free(all);
  return 0;
}

static int stencil_search_n(const orc_mesh* m, const buckets* B, const double* xr, int S,
                            int64_t* out) {
  int d = m->dim;
  int ib[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    int i = (int)floor((xr[a] - B->lo[a]) / B->bs);
    if (i < 0) i = 0;
    if (i >= B->nb[a]) i = B->nb[a] - 1;
    ib[a] = i;
  }
  int maxr = B->nb[0] + B->nb[1] + B->nb[2];
  size_t cap = 1024;
  cand* cs = (cand*)malloc(sizeof(cand) * cap);
  for (int r = 1; r <= maxr; ++r) {
    size_t n = 0;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = a < d ? ib[a] - r : 0;
      hi[a] = a < d ? ib[a] + r : 0;
      if (lo[a] < 0) lo[a] = 0;
      if (hi[a] >= B->nb[a]) hi[a] = B->nb[a] - 1;
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          int64_t id = ((int64_t)k * B->nb[1] + j) * B->nb[0] + i;
          for (int64_t t = B->start[id]; t < B->start[id + 1]; ++t) {
            if (n == cap) { cap *= 2; cs = (cand*)realloc(cs, sizeof(cand) * cap); }
            cs[n].id = B->items[t];
            cs[n].key = dist_key(m, xr, cs[n].id);
            ++n;
          }
        }
    if ((int64_t)n < S && (int64_t)n < m->nc) continue;
    qsort(cs, n, sizeof(cand), cmp_cand);
    /* everything outside the searched block lies farther than the distance
       from xr to the block's faces; accept when the S-th key is clearly
       inside that radius (or the block already covers every cell) */
    int whole = 1;
    double reach = 1e300;
    for (int a = 0; a < d; ++a) {
      if (lo[a] > 0) { whole = 0; double g = xr[a] - (B->lo[a] + lo[a] * B->bs); if (g < reach) reach = g; }
      if (hi[a] < B->nb[a] - 1) { whole = 0; double g = (B->lo[a] + (hi[a] + 1) * B->bs) - xr[a]; if (g < reach) reach = g; }
    }
    int64_t kmax = cs[S - 1].key;
    double reach_key = ldexp(reach * reach, 24 - 2 * m->href_exp);
    if (whole || (double)kmax + 2.0 < reach_key) {
      for (int i = 0; i < S; ++i) out[i] = cs[i].id;
      free(cs);
      return 0;
    }
  }
  free(cs);
  return -1;
}

static int stencil_search(const orc_mesh* m, const buckets* B, const double* xr,
                          int64_t* out) {
  return stencil_search_n(m, B, xr, m->S, out);
}

/* mirror image of x in the plane of face f (its centre and unit normal) */
static void mirror_point(const orc_mesh* m, int64_t f, const double* x, double* y) {
  double dn = 0;
  for (int a = 0; a < 3; ++a) dn += (x[a] - m->xf[3 * f + a]) * m->nrm[3 * f + a];
  for (int a = 0; a < 3; ++a) y[a] = x[a] - 2.0 * dn * m->nrm[3 * f + a];
}

/* R v = v - 2 n (n . v), the reflection across the plane of face f */
static void reflect(const orc_mesh* m, int64_t f, const double* v, double* w) {
  double dn = 0;
  for (int a = 0; a < m->dim; ++a) dn += v[a] * m->nrm[3 * f + a];
  for (int a = 0; a < m->dim; ++a) w[a] = v[a] - 2.0 * dn * m->nrm[3 * f + a];
}

/* ------------------------------------------------------------------ */
/* least-squares Taylor reconstruction, eqs. (te)-(lsA)                */
/* ------------------------------------------------------------------ */

/* scaled Taylor basis q(X) in graded order with 1/(a! b! c!) factors */
static void taylor_basis(int dim, int p, const double* X, double* q) {
  static const double fact[4] = {1, 1, 2, 6};
  int t = 0;
  for (int deg = 0; deg <= p; ++deg) {
    if (dim == 2) {
      for (int a = deg; a >= 0; --a) {
        int b = deg - a;
        q[t++] = pow(X[0], a) * pow(X[1], b) / (fact[a] * fact[b]);
      }
    } else {
      for (int a = deg; a >= 0; --a)
        for (int b = deg - a; b >= 0; --b) {
          int c = deg - a - b;
          q[t++] = pow(X[0], a) * pow(X[1], b) * pow(X[2], c) / (fact[a] * fact[b] * fact[c]);
        }
    }
  }
}

/* Solve M X = B (n x n, n x ncol) by Gaussian elimination with partial
   pivoting, in extended precision.  Returns 0, or -1 if singular. */
static int ld_solve(int n, ld* M, int ncol, ld* B) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    ld best = fabsl(M[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabsl(M[i * n + k]) > best) { best = fabsl(M[i * n + k]); piv = i; }
    if (best == 0.0L) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { ld s = M[k * n + j]; M[k * n + j] = M[piv * n + j]; M[piv * n + j] = s; }
      for (int j = 0; j < ncol; ++j) { ld s = B[k * ncol + j]; B[k * ncol + j] = B[piv * ncol + j]; B[piv * ncol + j] = s; }
    }
    for (int i = k + 1; i < n; ++i) {
      ld f = M[i * n + k] / M[k * n + k];
      if (f == 0.0L) continue;
      for (int j = k; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
      for (int j = 0; j < ncol; ++j) B[i * ncol + j] -= f * B[k * ncol + j];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = 0; j < ncol; ++j) {
      ld s = B[k * ncol + j];
      for (int i = k + 1; i < n; ++i) s -= M[k * n + i] * B[i * ncol + j];
      B[k * ncol + j] = s / M[k * n + k];
    }
  }
  return 0;
}

/* Reconstruction matrix Abar = M^{-1} Q W for the reference point xt and the
   stencil cells st[0..S-1], plus (ghost=1) a node co-located with xt with
   basis [1,0,...] and unit weight.  Abar is written [Nt][ncol] with
   ncol = S + ghost, in the scaled basis; *h_out receives h = 2 r_s and
   *cond_out the 1-norm condition number of M. */
static int reconstruct_pts(const orc_mesh* m, const double* xt, const double* pts, int ghost,
                           double* Abar, double* h_out, double* cond_out) {
  int d = m->dim, S = m->S, Nt = m->Nt, ncol = S + ghost;
  double rs = 0.0;
  for (int i = 0; i < S; ++i) {
    double s = 0;
    for (int a = 0; a < d; ++a) {
      double e = pts[3 * i + a] - xt[a];
      s += e * e;
    }
    s = sqrt(s);
    if (s > rs) rs = s;
  }
  double h = 2.0 * rs; /* stencil diameter d_s, also the basis scale */
  double k2 = m->kw * m->kw;
  double ek = exp(-k2);
  ld* Qm = (ld*)malloc(sizeof(ld) * Nt * ncol);
  ld* W = (ld*)malloc(sizeof(ld) * ncol);
  double X[3] = {0, 0, 0}, q[20];
  for (int i = 0; i < S; ++i) {
    double dd = 0;
    for (int a = 0; a < d; ++a) {
      X[a] = (pts[3 * i + a] - xt[a]) / h;
      dd += X[a] * X[a];
    }
    /* eq. (weightFunc) with dtilde = |xt - x_N| / d_s */
    W[i] = (exp(-dd * k2) - ek) / (1.0 - ek);
    taylor_basis(d, m->p, X, q);
    for (int t = 0; t < Nt; ++t) Qm[t * ncol + i] = q[t];
  }
  if (ghost) {
    W[S] = 1.0L;
    for (int t = 0; t < Nt; ++t) Qm[t * ncol + S] = t == 0 ? 1.0L : 0.0L;
  }
  ld* M = (ld*)calloc(Nt * Nt, sizeof(ld));
  ld* Mc = (ld*)calloc(Nt * Nt, sizeof(ld));
  ld* B = (ld*)malloc(sizeof(ld) * Nt * ncol);
  for (int r = 0; r < Nt; ++r)
    for (int c = 0; c < Nt; ++c) {
      ld s = 0;
      for (int i = 0; i < ncol; ++i) s += Qm[r * ncol + i] * W[i] * Qm[c * ncol + i];
      M[r * Nt + c] = s;
    }
  memcpy(Mc, M, sizeof(ld) * Nt * Nt);
  for (int r = 0; r < Nt; ++r)
    for (int i = 0; i < ncol; ++i) B[r * ncol + i] = Qm[r * ncol + i] * W[i];
  int rc = ld_solve(Nt, M, ncol, B);
  if (rc == 0 && cond_out) {
    /* ||M||_1 * ||M^{-1}||_1 */
    ld* I = (ld*)calloc(Nt * Nt, sizeof(ld));
    for (int i = 0; i < Nt; ++i) I[i * Nt + i] = 1.0L;
    ld* Mc2 = (ld*)malloc(sizeof(ld) * Nt * Nt);
    memcpy(Mc2, Mc, sizeof(ld) * Nt * Nt);
    ld_solve(Nt, Mc2, Nt, I);
    ld n1 = 0, ni = 0;
    for (int c = 0; c < Nt; ++c) {
      ld s1 = 0, s2 = 0;
      for (int r = 0; r < Nt; ++r) { s1 += fabsl(Mc[r * Nt + c]); s2 += fabsl(I[r * Nt + c]); }
      if (s1 > n1) n1 = s1;
      if (s2 > ni) ni = s2;
    }
    *cond_out = (double)(n1 * ni);
    free(I); free(Mc2);
  }
  for (int r = 0; r < Nt; ++r)
    for (int i = 0; i < ncol; ++i) Abar[r * ncol + i] = (double)B[r * ncol + i];
  *h_out = h;
  free(Qm); free(W); free(M); free(Mc); free(B);
  return rc;
}

/* the same for stencil cells given by id (their centroids) */
static int reconstruct(const orc_mesh* m, const double* xt, const int64_t* st, int ghost,
                       double* Abar, double* h_out, double* cond_out) {
  double* pts = (double*)malloc(sizeof(double) * 3 * m->S);
  for (int i = 0; i < m->S; ++i)
    for (int a = 0; a < 3; ++a) pts[3 * i + a] = m->xc[3 * st[i] + a];
  int rc = reconstruct_pts(m, xt, pts, ghost, Abar, h_out, cond_out);
  free(pts);
  return rc;
}

/* ------------------------------------------------------------------ */
/* prepare stencils and coefficients for a subset of cells              */
/* ------------------------------------------------------------------ */
int orc_prepare(orc_mesh* m, int64_t nsub, const int64_t* cells) {
  if (!m->have_geom) return -1;
  orc_free_subset(m);
  int d = m->dim, S = m->S, Q = m->Q, Nt = m->Nt, nlf = m->nlf;
  m->fslot = (int64_t*)malloc(sizeof(int64_t) * m->nf);
  m->cslot = (int64_t*)malloc(sizeof(int64_t) * m->nc);
  for (int64_t f = 0; f < m->nf; ++f) m->fslot[f] = -1;
  for (int64_t c = 0; c < m->nc; ++c) m->cslot[c] = -1;
  /* needed: faces of subset cells (with stencils unless traction), the
     subset cells and their face neighbours (cell stencils for the jump) */
  int64_t nfs = 0, ncs = 0;
  int64_t ns = nsub < 0 ? m->nc : nsub;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t c = nsub < 0 ? s : cells[s];
    if (c < 0 || c >= m->nc) return -2;
    if (m->cslot[c] < 0) m->cslot[c] = ncs++;
    for (int lf = 0; lf < nlf; ++lf) {
      int64_t f = m->cf[c * nlf + lf];
      if (f < 0 || m->ftag[f] == 1) continue;
      if (m->fslot[f] < 0) m->fslot[f] = nfs++;
      if (m->ftag[f] < 0) {
        int64_t o = m->fown[f] == c ? m->fnei[f] : m->fown[f];
        if (m->cslot[o] < 0) m->cslot[o] = ncs++;
      }
    }
  }
  m->nfs = nfs; m->ncs = ncs;
  m->fst = (int64_t*)malloc(sizeof(int64_t) * (nfs * S + 1));
  m->fco = (double*)calloc(nfs * Q * (S + 1) * 3 + 1, sizeof(double));
  m->fcond = (double*)calloc(nfs * Q + 1, sizeof(double));
  m->cst = (int64_t*)malloc(sizeof(int64_t) * (ncs * S + 1));
  m->cex = (double*)calloc(ncs * nlf * S + 1, sizeof(double));
  m->ccond = (double*)calloc(ncs + 1, sizeof(double));
  buckets B;
  build_buckets(m, &B);
  int rc = 0;
  /* faces and cells are independent: OpenMP threads take whole ones */
#pragma omp parallel
  {
  double* Abar = (double*)malloc(sizeof(double) * Nt * (S + 1));
  double* pts = (double*)malloc(sizeof(double) * 3 * S);
#pragma omp for schedule(dynamic, 8)
  for (int64_t f = 0; f < m->nf; ++f) {
    int64_t sl = m->fslot[f];
    if (sl < 0) continue;
    int err;
#pragma omp atomic read
    err = rc;
    if (err) continue;
    int64_t* st = m->fst + sl * S;
    int ghost = m->ftag[f] == 0;
    /* symmetry face (Sec. 3.5.2): the ceil(S/2) nearest cells and the mirror
       images of the floor(S/2) nearest of them; slot half + k holds the
       source cell of mirror k */
    int half = m->ftag[f] == 2 ? (S + 1) / 2 : S;
    if (stencil_search_n(m, &B, m->xf + 3 * f, half, st)) {
#pragma omp atomic write
      rc = -3;
      continue;
    }
    for (int k = 0; k < S - half; ++k) st[half + k] = st[k];
    for (int i = 0; i < S; ++i) {
      if (i < half)
        for (int a = 0; a < 3; ++a) pts[3 * i + a] = m->xc[3 * st[i] + a];
      else
        mirror_point(m, f, m->xc + 3 * st[i], pts + 3 * i);
    }
    for (int q = 0; q < Q; ++q) {
      double h;
      if (reconstruct_pts(m, m->xq + (f * Q + q) * 3, pts, ghost, Abar, &h,
                          &m->fcond[sl * Q + q])) {
#pragma omp atomic write
        rc = -4;
        break;
      }
      int ncol = S + ghost;
      /* gradient rows of Abar, rescaled from the scaled basis (App. B) */
      for (int i = 0; i < ncol; ++i)
        for (int a = 0; a < d; ++a)
          m->fco[((sl * Q + q) * (S + 1) + i) * 3 + a] = Abar[(1 + a) * ncol + i] / h;
    }
  }
#pragma omp for schedule(dynamic, 8)
  for (int64_t c = 0; c < m->nc; ++c) {
    int64_t sl = m->cslot[c];
    if (sl < 0) continue;
    int err;
#pragma omp atomic read
    err = rc;
    if (err) continue;
    int64_t* st = m->cst + sl * S;
    if (stencil_search(m, &B, m->xc + 3 * c, st)) {
#pragma omp atomic write
      rc = -3;
      continue;
    }
    double h;
    if (reconstruct(m, m->xc + 3 * c, st, 0, Abar, &h, &m->ccond[sl])) {
#pragma omp atomic write
      rc = -4;
      continue;
    }
    /* extrapolation to each face centre, eq. (alphaJump): the Taylor terms
       of order 1..p evaluated at d_Pf, applied to the derivative rows */
    for (int lf = 0; lf < nlf; ++lf) {
      int64_t f = m->cf[c * nlf + lf];
      if (f < 0) continue;  /* polygon slot past its last side */
      double X[3] = {0, 0, 0}, g[20];
      for (int a = 0; a < d; ++a) X[a] = (m->xf[3 * f + a] - m->xc[3 * c + a]) / h;
      taylor_basis(d, m->p, X, g);
      for (int i = 0; i < S; ++i) {
        double e = 0;
        for (int t = 1; t < Nt; ++t) e += g[t] * Abar[t * S + i];
        m->cex[(sl * nlf + lf) * S + i] = e;
      }
    }
  }
  free(Abar);
  free(pts);
  }
  free_buckets(&B);
  return rc;
}

/* threads of the parallel loops (0: OpenMP's default); returns the count in
   use, 1 when built without OpenMP */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_face_slot(const orc_mesh* m, int64_t f) { return m->fslot ? (int)m->fslot[f] : -1; }
int orc_cell_slot(const orc_mesh* m, int64_t c) { return m->cslot ? (int)m->cslot[c] : -1; }
void orc_get_face_stencil(const orc_mesh* m, int64_t slot, int64_t* out) {
  memcpy(out, m->fst + slot * m->S, sizeof(int64_t) * m->S);
}
void orc_get_face_coef(const orc_mesh* m, int64_t slot, double* out) {
  memcpy(out, m->fco + slot * m->Q * (m->S + 1) * 3, sizeof(double) * m->Q * (m->S + 1) * 3);
}
void orc_get_face_cond(const orc_mesh* m, int64_t slot, double* out) {
  memcpy(out, m->fcond + slot * m->Q, sizeof(double) * m->Q);
}
void orc_get_cell_stencil(const orc_mesh* m, int64_t slot, int64_t* out) {
  memcpy(out, m->cst + slot * m->S, sizeof(int64_t) * m->S);
}
void orc_get_cell_ext(const orc_mesh* m, int64_t slot, double* out) {
  memcpy(out, m->cex + slot * m->nlf * m->S, sizeof(double) * m->nlf * m->S);
}
double orc_get_cell_cond(const orc_mesh* m, int64_t slot) { return m->ccond[slot]; }

/* Full reconstruction matrix for an arbitrary point and stencil (tests):
   Abar [Nt][S+ghost] in the scaled basis, and h. */
int orc_reconstruct(const orc_mesh* m, const double* xt, const int64_t* st, int ghost,
                    double* Abar, double* h, double* cond) {
  return reconstruct(m, xt, st, ghost, Abar, h, cond);
}
int orc_stencil(const orc_mesh* m, const double* xr, int64_t* out) {
  buckets B;
  build_buckets(m, &B);
  int rc = stencil_search(m, &B, xr, out);
  free_buckets(&B);
  return rc;
}

/* ------------------------------------------------------------------ */
/* mechanical laws (App. A)                                            */
/* ------------------------------------------------------------------ */
static double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}
static void inv3(const double A[3][3], double B[3][3]) {
  double dt = det3(A);
  B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / dt;
  B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / dt;
  B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / dt;
  B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / dt;
  B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / dt;
  B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / dt;
  B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / dt;
  B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / dt;
  B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / dt;
}

/* Stress tensor T at a quadrature point from G[i][j] = d u_j / d x_i
   (3x3, zero rows/cols beyond dim), such that the face traction is
   t_i = sum_j T[i][j] a_j.  law 0: engineering stress sigma_s (symmetric);
   law 1: first Piola-Kirchhoff P = J sigma F^{-T} with neo-Hookean sigma. */
void orc_stress(int law, double mu, double lam, const double G[3][3], double T[3][3]) {
  if (law == 0) {
    double tr = G[0][0] + G[1][1] + G[2][2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) T[i][j] = mu * (G[i][j] + G[j][i]) + (i == j ? lam * tr : 0.0);
    return;
  }
  double F[3][3], b[3][3], Finv[3][3], s[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) F[i][j] = (i == j ? 1.0 : 0.0) + G[j][i]; /* F = I + grad(u)^T */
  double J = det3(F);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = 0;
      for (int k = 0; k < 3; ++k) t += F[i][k] * F[j][k];
      b[i][j] = pow(J, -2.0 / 3.0) * t;           /* isochoric b-bar */
    }
  double trb = (b[0][0] + b[1][1] + b[2][2]) / 3.0;
  double kappa = lam + 2.0 * mu / 3.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      s[i][j] = (mu / J) * (b[i][j] - (i == j ? trb : 0.0)) +
                (i == j ? 0.5 * kappa * (J * J - 1.0) / J : 0.0);
  inv3(F, Finv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = 0;
      for (int k = 0; k < 3; ++k) t += s[i][k] * Finv[j][k]; /* sigma F^{-T} */
      T[i][j] = J * t;
    }
}

/* ------------------------------------------------------------------ */
/* residual R(u), eqs. (divStressDiscret), (alpha), (bodyTerm)          */
/* Computes R at the prepared subset cells (in slot order of `cells`).  */
/*  u    [d][nc]                                                        */
/*  ubq  [nfd][Q][d]   prescribed displacement at disp-face points      */
/*  ubf  [nfd][d]      prescribed displacement at disp-face centres     */
/*  tbq  [nft][Q][d]   prescribed traction at traction-face points      */
/*  bsrc [d][nc]       integrated body force per cell (may be NULL)     */
/*  R    [d][nsub]                                                      */
/* ------------------------------------------------------------------ */
static void face_flux(const orc_mesh* m, int64_t f, int law, double mu, double lam,
                      const double* u, const double* ubq, const double* ubf,
                      const double* tbq, double* flux) {
  int d = m->dim, S = m->S, Q = m->Q, nlf = m->nlf;
  int64_t nc = m->nc;
  for (int a = 0; a < 3; ++a) flux[a] = 0.0;
  if (m->ftag[f] == 1) {
    int64_t b = f - m->nfi - m->nfd - m->nfy;
    for (int q = 0; q < Q; ++q) {
      const double* a = m->aq + (f * Q + q) * 3;
      double mag = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      for (int j = 0; j < d; ++j) flux[j] += mag * tbq[(b * Q + q) * d + j];
    }
    return;
  }
  int64_t sl = m->fslot[f];
  const int64_t* st = m->fst + sl * S;
  int64_t bd = m->ftag[f] == 0 ? f - m->nfi : -1;
  int sym = m->ftag[f] == 2;
  int half = sym ? (S + 1) / 2 : S;
  for (int q = 0; q < Q; ++q) {
    double G[3][3] = {{0}};
    const double* co = m->fco + (sl * Q + q) * (S + 1) * 3;
    for (int i = 0; i < S; ++i) {
      double un[3] = {0, 0, 0}, w[3];
      for (int j = 0; j < d; ++j) un[j] = u[j * nc + st[i]];
      if (i >= half) {  /* mirrored node: the reflected state R u_N */
        reflect(m, f, un, w);
        for (int j = 0; j < d; ++j) un[j] = w[j];
      }
      for (int a = 0; a < d; ++a)
        for (int j = 0; j < d; ++j) G[a][j] += co[i * 3 + a] * un[j];
    }
    if (bd >= 0)
      for (int a = 0; a < d; ++a)
        for (int j = 0; j < d; ++j) G[a][j] += co[S * 3 + a] * ubq[(bd * Q + q) * d + j];
    double T[3][3];
    orc_stress(law, mu, lam, G, T);
    const double* aq = m->aq + (f * Q + q) * 3;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) flux[i] += T[i][j] * aq[j];
  }
  /* alpha stabilisation: jump of the values extrapolated to the face centre */
  double Kbar = 2.0 * mu + lam;
  int64_t P = m->fown[f];
  int64_t cp = m->cslot[P];
  double uP[3];
  for (int j = 0; j < d; ++j) {
    double s = u[j * nc + P];
    const double* e = m->cex + (cp * nlf + m->flf[f]) * S;
    const int64_t* sp = m->cst + cp * S;
    for (int i = 0; i < S; ++i) s += e[i] * u[j * nc + sp[i]];
    uP[j] = s;
  }
  double dvec[3] = {0, 0, 0}, other[3];
  if (sym) {
    /* the other side of a symmetry face is the mirror of this one */
    reflect(m, f, uP, other);
    for (int a = 0; a < d; ++a) dvec[a] = m->xf[3 * f + a] - m->xc[3 * P + a];
  } else if (bd < 0) {
    int64_t N = m->fnei[f];
    int64_t cn_ = m->cslot[N];
    int lfN = -1;
    for (int lf = 0; lf < nlf; ++lf)
      if (m->cf[N * nlf + lf] == f) lfN = lf;
    for (int j = 0; j < d; ++j) {
      double s = u[j * nc + N];
      const double* e = m->cex + (cn_ * nlf + lfN) * S;
      const int64_t* sn = m->cst + cn_ * S;
      for (int i = 0; i < S; ++i) s += e[i] * u[j * nc + sn[i]];
      other[j] = s;
    }
    for (int a = 0; a < d; ++a) dvec[a] = m->xc[3 * N + a] - m->xc[3 * P + a];
  } else {
    for (int j = 0; j < d; ++j) other[j] = ubf[bd * d + j];
    for (int a = 0; a < d; ++a) dvec[a] = m->xf[3 * f + a] - m->xc[3 * P + a];
  }
  double dn = 0;
  for (int a = 0; a < d; ++a) dn += dvec[a] * m->nrm[3 * f + a];
  double coef = m->alpha * Kbar / fabs(dn) * m->gam[f];
  for (int j = 0; j < d; ++j) flux[j] += coef * (other[j] - uP[j]);
}

int orc_residual(const orc_mesh* m, int law, double mu, double lam, const double* u,
                 const double* ubq, const double* ubf, const double* tbq,
                 const double* bsrc, int64_t nsub, const int64_t* cells, double* R) {
  int d = m->dim, nlf = m->nlf;
  int64_t ns = nsub < 0 ? m->nc : nsub;
  for (int64_t s = 0; s < ns; ++s)
    if (m->cslot[nsub < 0 ? s : cells[s]] < 0) return -1;
  /* cells are independent: each thread takes whole cells (OpenMP when built
     with it; the arithmetic of a cell does not depend on the thread count) */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < ns; ++s) {
    int64_t c = nsub < 0 ? s : cells[s];
    double r[3] = {0, 0, 0}, fl[3];
    for (int lf = 0; lf < nlf; ++lf) {
      int64_t f = m->cf[c * nlf + lf];
      if (f < 0) continue;
      face_flux(m, f, law, mu, lam, u, ubq, ubf, tbq, fl);
      double sg = m->fown[f] == c ? 1.0 : -1.0;
      for (int j = 0; j < d; ++j) r[j] += sg * fl[j];
    }
    for (int j = 0; j < d; ++j) R[j * ns + s] = r[j] + (bsrc ? bsrc[j * m->nc + c] : 0.0);
  }
  return 0;
}

/* per-face flux for the prepared faces of the subset (tests of the
   face-level quantities); flux [nf][3] filled for prepared faces only */
int orc_face_fluxes(const orc_mesh* m, int law, double mu, double lam, const double* u,
                    const double* ubq, const double* ubf, const double* tbq, double* flux) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t f = 0; f < m->nf; ++f) {
    if (m->ftag[f] != 1 && m->fslot[f] < 0) continue;
    face_flux(m, f, law, mu, lam, u, ubq, ubf, tbq, flux + 3 * f);
  }
  return 0;
}

/* body-force integral per cell, eq. (bodyTerm): fq [nc][QC][d] -> b [d][nc] */
void orc_integrate_cells(const orc_mesh* m, const double* fq, double* b) {
  int d = m->dim;
  for (int64_t c = 0; c < m->nc; ++c)
    for (int j = 0; j < d; ++j) {
      double s = 0;
      for (int q = 0; q < m->QC; ++q) s += m->cqw[c * m->QC + q] * fq[(c * m->QC + q) * d + j];
      b[j * m->nc + c] = s;
    }
}

/* ------------------------------------------------------------------ */
/* compact-stencil approximate Jacobian (Sec. 4.1): scalar operator     */
/*   (A v)_P = sum_int a_PN (v_N - v_P) - sum_disp a_Pb v_P             */
/*   a_PN = Kbar Gamma_f |Delta_f| / |d_PN|,  Delta_f = d/(d.n)          */
/* diag [nc]; off [nfi] (entry of internal face f couples own/nei)       */
/* ------------------------------------------------------------------ */
void orc_aj(const orc_mesh* m, double Kbar, double* diag, double* off) {
  int d = m->dim;
  for (int64_t c = 0; c < m->nc; ++c) diag[c] = 0.0;
  for (int64_t f = 0; f < m->nfi + m->nfd + m->nfy; ++f) {
    int64_t P = m->fown[f];
    double dv[3] = {0, 0, 0}, dn = 0, dl = 0;
    for (int a = 0; a < d; ++a) {
      dv[a] = (f < m->nfi ? m->xc[3 * m->fnei[f] + a] : m->xf[3 * f + a]) - m->xc[3 * P + a];
      dn += dv[a] * m->nrm[3 * f + a];
      dl += dv[a] * dv[a];
    }
    dl = sqrt(dl);
    double Delta = 0;  /* |Delta_f| = |d| / |d.n| */
    Delta = dl / fabs(dn);
    double a = Kbar * Delta / dl * m->gam[f];
    if (f < m->nfi) {
      off[f] = a;
      diag[P] -= a;
      diag[m->fnei[f]] -= a;
    } else {
      diag[P] -= a;
    }
  }
}
