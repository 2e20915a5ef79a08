// api.cu -- the C ABI of libhofv (include/hofv.h): context, mesh and face
// extraction, set-up orchestration, evaluation entry points and the
// Jacobian-free Newton-Krylov driver (arXiv 2601.18417, Sec. 4.1).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <numeric>

#include "hofv_internal.cuh"

#define TRY(x)                 \
  do {                         \
    int rc_ = (x);             \
    if (rc_ != 0) return rc_;  \
  } while (0)

namespace hofv {

int fail(hofv_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(hofv_ctx* c, cudaError_t e, const char* what) {
  return fail(c, HOFV_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void dev_free(hofv_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) c->allocs.erase(it);
  cudaFree(p);
}

DevMesh dev_mesh(const hofv_ctx* c) {
  DevMesh m;
  m.dim = c->dim;
  m.nlf = c->nlf;
  m.S = c->S;
  m.Q = c->Q;
  m.R = c->Q * c->dim;
  m.nc = c->nc;
  m.nf = c->nf;
  m.nfi = c->nfi;
  m.nfd = c->nfd;
  m.nft = c->nft;
  m.nfid = c->nfid;
  m.nftile = c->nftile;
  m.nctile = c->nctile;
  m.fst = c->d_fst;
  m.fco = c->d_fco;
  m.gco = c->d_gco;
  m.aq = c->d_aq;
  m.fstar = c->d_fstar;
  m.fstab = c->d_fstab;
  m.fql = c->d_fql;
  m.pgrp = c->d_pgrp;
  m.npg = c->npg;
  m.cst = c->d_cst;
  m.cex = c->d_cex;
  m.cface = c->d_cface;
  m.tco = (c->contract && c->tco_valid && c->mat.law == HOFV_LAW_LINEAR) ? c->d_tco : nullptr;
  m.nfy = c->nfy;
  m.ng = c->ng;
  m.wst = c->nc + c->ng;
  m.gsrc = c->d_gsrc;
  m.gface = c->d_gface;
  m.nrm = c->d_nrm;
  m.wext = c->d_wext;
  m.ubfw = c->d_ubf;
  m.mscale = c->inertia ? c->d_mscale : nullptr;
  m.cmass = (c->inertia && !c->one_point) ? c->d_cmass : nullptr;
  m.inert = c->d_inert;
  m.prec = c->prec;
  m.su = c->d_su;
  m.sv = c->d_sv;
  m.ustar_v = c->d_ustar_v;
  m.vext = c->d_vext;
  m.gcache = c->d_gcache;
  m.tcache = c->d_tcache;
  m.kerr = c->d_bar ? c->d_bar + 3 : nullptr;
  m.fcsum = c->d_fcsum;
  return m;
}

// local faces of the reference quad / hex and of the triangle /
// tetrahedron as node positions, outward order (face k of a tetrahedron lies
// opposite its node 3 - k)
static const int kQuadLF[4][2] = {{3, 0}, {1, 2}, {0, 1}, {2, 3}};
static const int kHexLF[6][4] = {{0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4},
                                 {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};
static const int kTriLF[3][2] = {{0, 1}, {1, 2}, {2, 0}};
static const int kTetLF[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};

static int lf_node(const hofv_ctx* c, int lf, int k) {
  if (c->simplex) return c->dim == 2 ? kTriLF[lf][k] : kTetLF[lf][k];
  return c->dim == 2 ? kQuadLF[lf][k] : kHexLF[lf][k];
}

// a polygon has one local face per side, from corner k to corner k+1;
// slots past its last side hold no face
static bool face_exists(const hofv_ctx* c, int64_t cell, int lf) {
  return !c->poly || lf < c->cnv[cell];
}

static int64_t cell_face_node(const hofv_ctx* c, int64_t cell, int lf, int k) {
  if (c->poly) return c->cn[cell * c->nv + (lf + k) % c->cnv[cell]];
  return c->cn[cell * c->nv + lf_node(c, lf, k)];
}

// Gauss-Legendre rule on [0, 1] (closed forms of the 1..4 point rules on
// [-1, 1], mapped by x = (t + 1) / 2, w = c / 2)
static void gauss_rule(int n, double* x, double* w) {
  double t[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
  switch (n) {
    case 1: t[0] = 0.0; c[0] = 2.0; break;
    case 2: t[0] = -1.0 / sqrt(3.0); t[1] = -t[0]; c[0] = c[1] = 1.0; break;
    case 3:
      t[0] = -sqrt(3.0 / 5.0); t[1] = 0.0; t[2] = -t[0];
      c[0] = c[2] = 5.0 / 9.0; c[1] = 8.0 / 9.0;
      break;
    default: {
      const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
      const double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
      t[0] = -b; t[1] = -a; t[2] = a; t[3] = b;
      c[1] = c[2] = (18.0 + sqrt(30.0)) / 36.0;
      c[0] = c[3] = (18.0 - sqrt(30.0)) / 36.0;
    }
  }
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (t[i] + 1.0);
    w[i] = 0.5 * c[i];
  }
}

static void graphs_clear(hofv_ctx* c);

// kernel arguments baked into captured graphs change: drop the graphs
static void invalidate_graphs(hofv_ctx* c) {
  c->gen++;
  graphs_clear(c);
}

static void free_built(hofv_ctx* c) {
  invalidate_graphs(c);
  gnn_release(c);
  mg_release(c);
  nej_release(c);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->device_bytes = 0;
  c->d_x = nullptr; c->d_fnodes = nullptr; c->d_cnodes = nullptr;
  c->d_xc = c->d_vol = c->d_xq = c->d_aq = c->d_xf = c->d_nrm = c->d_gam = nullptr;
  c->d_cqx = c->d_cqw = nullptr;
  c->d_cf = nullptr; c->d_ftag = c->d_fown = c->d_fnei = nullptr;
  c->d_fst = c->d_cst = c->d_fstar = c->d_cface = nullptr;
  c->d_fco = c->d_gco = c->d_cex = c->d_fstab = nullptr;
  c->d_fql = nullptr;
  c->d_pgrp = nullptr;
  c->npg = 0;
  c->d_ubq = c->d_ubf = c->d_tbq = c->d_body = c->d_src = nullptr;
  c->d_tco = c->d_gflux = nullptr;
  c->tco_valid = false;
  c->d_xce = c->d_wext = nullptr;
  c->d_gsrc = c->d_gface = nullptr;
  c->ng = 0;
  c->gsrc_host.clear();
  c->inertia = false;
  c->hist_set = false;
  c->d_cmass = c->d_mscale = c->d_inert = c->d_hist = nullptr;
  c->d_ustar = c->d_flux = c->d_w = c->d_red = c->d_scal = nullptr;
  c->d_su = c->d_sv = nullptr;
  c->d_ustar_v = c->d_vext = nullptr;
  c->d_gcache = c->d_tcache = nullptr;
  c->d_fcsum = nullptr;
  c->jv_u = c->jv_R = nullptr;
  c->jv_cur++;
  c->d_count = nullptr;
  c->d_aj_diag = c->d_aj_off = nullptr;
  c->d_aj_col = nullptr;
  c->d_aj_diag32 = c->d_aj_off32 = nullptr;
  c->d_aj_invd = nullptr;
  c->d_aj_invd32 = nullptr;
  c->d_bar = nullptr;
  c->d_cg64 = nullptr;
  c->d_cg32 = nullptr;
  c->d_V = c->d_Z = c->d_kvec = c->d_h = nullptr;
  c->kry_m = 0;
  c->built = false;
}

// rewrite the face and cell coefficient arrays as double-float pairs
// (to_df = 1) or back to doubles (0), in place
static int coef_format(hofv_ctx* c, int to_df) {
  const int64_t nfco = std::max<int64_t>(c->nftile, 1) * c->S * kTile * c->Q * c->dim;
  const int64_t ncex = c->nctile * c->S * kTile * c->nlf;
  launch_coef_format(c->d_fco, nfco, to_df, c->stream);
  launch_coef_format(c->d_cex, ncex, to_df, c->stream);
  c->prec = to_df ? HOFV_PREC_DF64 : HOFV_PREC_FP64;  // the arrays' format from here on
  if (to_df) launch_row_sums(dev_mesh(c), c->d_fcsum, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

// ---- linearisation cache of the neo-Hookean double-float Jv ----
static bool jv_uses_cache(const hofv_ctx* c) {
  return c->prec == HOFV_PREC_DF64 && c->have_mat && c->mat.law == HOFV_LAW_NEOHOOKEAN;
}

// storage of the cache, allocated by the set-up calls that make it needed
static int ensure_jv_storage(hofv_ctx* c) {
  if (!c->built || !jv_uses_cache(c) || c->d_gcache) return 0;
  const int64_t nf = std::max<int64_t>(c->nftile, 1) * kTile;
  TRY(dev_alloc(c, &c->d_gcache, nf * c->Q * c->dim * c->dim));
  TRY(dev_alloc(c, &c->d_tcache, nf * c->Q * c->dim));
  return 0;
}

// the cache no longer describes any state (data, material or coefficients
// changed, or the state it was filled from may have been overwritten)
static void jv_invalidate(hofv_ctx* c) {
  c->jv_cur++;
  c->jv_u = c->jv_R = nullptr;
}

// a residual evaluation at u: the caller may have changed u in place
static void jv_touch(hofv_ctx* c, const double* u) {
  if (u == c->jv_u) jv_invalidate(c);
}

// gradient rows and tractions at u, for the Jv calls about (u, R(u)) that
// follow; refilled when (u, Ru) differs from the last fill or after an
// invalidation.  Host-side check plus, on a miss, one launch sequence:
// call outside stream capture.
int ensure_jv_cache(hofv_ctx* c, const double* u, const double* Ru) {
  if (!jv_uses_cache(c)) return 0;
  if (c->jv_u == u && c->jv_R == Ru && c->jv_gen == c->jv_cur) return 0;
  TRY(ensure_jv_storage(c));
  launch_jv_cache_fill(dev_mesh(c), c->mat, u, c->d_ubq, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  c->jv_u = u;
  c->jv_R = Ru;
  c->jv_gen = c->jv_cur;
  return 0;
}

// contracted linear-elastic face matrices for the current material
static int build_contraction(hofv_ctx* c) {
  if (!c->contract || !c->have_mat || c->mat.law != HOFV_LAW_LINEAR || !c->built) return 0;
  const int64_t count = std::max<int64_t>(c->nftile, 1) * c->S * kTile * c->dim * c->dim;
  if (!c->d_tco) TRY(dev_alloc(c, &c->d_tco, count));
  if (!c->d_gflux) TRY(dev_alloc(c, &c->d_gflux, std::max<int64_t>(c->nfd, 1) * c->dim));
  DevMesh m = dev_mesh(c);
  launch_build_tco(m, c->mat.mu, c->mat.lam, c->d_tco, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->tco_valid = true;
  return 0;
}

// the contracted matrices for the current material, whether or not the
// residual uses the contracted form (the near-exact Jacobian is made of them)
int ensure_tco(hofv_ctx* c) {
  if (c->tco_valid) return 0;
  if (!c->have_mat || c->mat.law != HOFV_LAW_LINEAR || !c->built)
    return fail(c, HOFV_ESTATE, "linear-elastic material and stencils must be set first");
  const int64_t count = std::max<int64_t>(c->nftile, 1) * c->S * kTile * c->dim * c->dim;
  if (!c->d_tco) TRY(dev_alloc(c, &c->d_tco, count));
  launch_build_tco(dev_mesh(c), c->mat.mu, c->mat.lam, c->d_tco, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->tco_valid = true;
  return 0;
}

int refresh_source(hofv_ctx* c) {
  if (!c->built) return 0;
  if (c->contract && c->tco_valid && c->have_mat && c->mat.law == HOFV_LAW_LINEAR)
    launch_ghost_flux(dev_mesh(c), c->mat.mu, c->mat.lam, c->d_ubq, c->d_gflux, c->stream);
  launch_source(c, c->stream);
  if (c->inertia)  // history part of the BDF2 acceleration, a constant per time step
    launch_combine4(c->nc * c->dim, 1.0, c->d_src, 1.0, c->d_hist, 0.0, nullptr, 0.0, nullptr,
                    c->d_src, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

}  // namespace hofv

using namespace hofv;

extern "C" {

int hofv_set_contraction(hofv_ctx* c, int on) {
  if (!c) return HOFV_EINVAL;
  invalidate_graphs(c);
  c->contract = on != 0;
  if (!c->contract) {
    c->tco_valid = false;
    return refresh_source(c);
  }
  TRY(build_contraction(c));
  return refresh_source(c);
}

int hofv_set_precision(hofv_ctx* c, int prec) {
  if (!c) return HOFV_EINVAL;
  if (prec != HOFV_PREC_FP64 && prec != HOFV_PREC_DF64) return fail(c, HOFV_EINVAL, "unknown precision");
  if (prec == c->prec) return HOFV_OK;
  invalidate_graphs(c);
  jv_invalidate(c);
  if (c->built) {
    HOFV_CUDA(c, cudaSetDevice(c->device));
    TRY(coef_format(c, prec == HOFV_PREC_DF64 ? 1 : 0));
  }
  c->prec = prec;
  return ensure_jv_storage(c);
}

int hofv_get_precision(const hofv_ctx* c) { return c ? c->prec : HOFV_EINVAL; }

const char* hofv_version(void) { return "hofv 0.2 (sm_103a)"; }

int hofv_create(hofv_ctx** out, int device, void* stream) {
  if (!out) return HOFV_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return HOFV_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return HOFV_ECUDA;
  hofv_ctx* c = new hofv_ctx();
  c->device = device;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      c->sm_count < 1)
    c->sm_count = 1;
  c->stream = static_cast<cudaStream_t>(stream);
  // default arithmetic of the gradient contraction
  const char* pe = getenv("HOFV_PRECISION");
  if (pe && (strcmp(pe, "df64") == 0 || strcmp(pe, "DF64") == 0)) c->prec = HOFV_PREC_DF64;
  *out = c;
  return HOFV_OK;
}

void hofv_destroy(hofv_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_built(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

const char* hofv_last_error(const hofv_ctx* c) { return c ? c->err.c_str() : "null context"; }

// faces from the cells' local faces: equal node sets pair up into internal
// faces, the rest must be exactly the boundary list
static int build_faces(hofv_ctx* c, int64_t nb, const int64_t* bface_nodes,
                       const int32_t* bface_tag) {
  for (int64_t b = 0; b < nb; ++b) {
    if (bface_tag[b] < 0 || bface_tag[b] > 2) return fail(c, HOFV_EINVAL, "bad boundary tag");
  }
  // local faces keyed by their sorted node ids
  const int64_t nc = c->nc;
  const int nlf = c->nlf, nfv = c->nfv;
  struct Rec {
    std::array<int64_t, 4> key;
    int64_t id;  // cell * nlf + lf
  };
  auto make_key = [&](const int64_t* nodes) {
    std::array<int64_t, 4> k = {-1, -1, -1, -1};
    for (int i = 0; i < nfv; ++i) k[i] = nodes[i];
    std::sort(k.begin(), k.begin() + nfv);
    return k;
  };
  std::vector<Rec> recs;
  recs.reserve((size_t)nc * nlf);
  for (int64_t cell = 0; cell < nc; ++cell)
    for (int lf = 0; lf < nlf; ++lf) {
      if (!face_exists(c, cell, lf)) continue;
      int64_t nodes[4];
      for (int k = 0; k < nfv; ++k) nodes[k] = cell_face_node(c, cell, lf, k);
      recs.push_back({make_key(nodes), cell * nlf + lf});
    }
  std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
    return a.key != b.key ? a.key < b.key : a.id < b.id;
  });
  std::vector<int64_t> partner((size_t)nc * nlf, -1);
  for (size_t i = 0; i + 1 < recs.size(); ++i)
    if (recs[i].key == recs[i + 1].key) {
      if (i + 2 < recs.size() && recs[i + 2].key == recs[i].key)
        return fail(c, HOFV_EINVAL, "a face is shared by more than two cells");
      partner[recs[i].id] = recs[i + 1].id;
      partner[recs[i + 1].id] = recs[i].id;
    }
  int64_t nbound = 0;
  for (int64_t i = 0; i < nc * nlf; ++i) nbound += partner[i] < 0 && face_exists(c, i / nlf, (int)(i % nlf));
  if (nbound != nb) return fail(c, HOFV_EINVAL, "boundary face list does not match the mesh boundary");
  std::vector<int64_t> bown((size_t)nb);
  std::vector<char> seen((size_t)nc * nlf, 0);
  for (int64_t b = 0; b < nb; ++b) {
    Rec q{make_key(bface_nodes + b * nfv), -1};
    auto itr = std::lower_bound(recs.begin(), recs.end(), q, [](const Rec& a, const Rec& b) {
      return a.key < b.key;
    });
    if (itr == recs.end() || itr->key != q.key) return fail(c, HOFV_EINVAL, "boundary face not in mesh");
    if (partner[itr->id] >= 0) return fail(c, HOFV_EINVAL, "boundary face is an internal face");
    if (seen[itr->id]) return fail(c, HOFV_EINVAL, "boundary face listed twice");
    seen[itr->id] = 1;
    bown[b] = itr->id;
  }
  int64_t nfi = 0, nfd = 0, nft = 0, nfy = 0;
  for (int64_t i = 0; i < nc * nlf; ++i) nfi += partner[i] > i;
  for (int64_t b = 0; b < nb; ++b)
    (bface_tag[b] == 0 ? nfd : bface_tag[b] == 1 ? nft : nfy)++;
  c->nfi = nfi;
  c->nfd = nfd;
  c->nfy = nfy;
  c->nft = nft;
  c->nfid = nfi + nfd + nfy;  // faces with a stencil and a flux
  c->nf = nfi + nfd + nfy + nft;
  c->fown.assign(c->nf, -1);
  c->fnei.assign(c->nf, -1);
  c->flf.assign(c->nf, 0);
  c->ftag.assign(c->nf, -1);
  c->cf.assign((size_t)nc * nlf, -1);
  int64_t f = 0;
  for (int64_t cell = 0; cell < nc; ++cell)
    for (int lf = 0; lf < nlf; ++lf) {
      const int64_t id = cell * nlf + lf, pid = partner[id];
      if (pid >= 0 && pid / nlf > cell) {
        c->fown[f] = cell;
        c->fnei[f] = pid / nlf;
        c->flf[f] = lf;
        c->cf[id] = f;
        c->cf[pid] = f;
        ++f;
      }
    }
  for (int tag : {0, 2, 1})  // displacement, symmetry, traction
    for (int64_t b = 0; b < nb; ++b)
      if (bface_tag[b] == tag) {
        const int64_t id = bown[b];
        c->fown[f] = id / nlf;
        c->flf[f] = (int)(id % nlf);
        c->ftag[f] = tag;
        c->cf[id] = f;
        ++f;
      }
  c->fnodes.assign((size_t)c->nf * nfv, 0);
  for (f = 0; f < c->nf; ++f)
    for (int k = 0; k < nfv; ++k) {
      const int lf = c->flf[f];
      c->fnodes[f * nfv + k] = (int32_t)cell_face_node(c, c->fown[f], lf, k);
    }
  c->have_mesh = true;
  c->built = false;
  return HOFV_OK;
}

int hofv_set_mesh(hofv_ctx* c, int dim, int64_t nn, const double* xyz, int64_t nc,
                  const int64_t* cell_nodes, int64_t nb, const int64_t* bface_nodes,
                  const int32_t* bface_tag) {
  return hofv_set_mesh_cells(c, dim, HOFV_CELL_TENSOR, nn, xyz, nc, cell_nodes, nb, bface_nodes,
                             bface_tag);
}

int hofv_set_mesh_cells(hofv_ctx* c, int dim, int cell_kind, int64_t nn, const double* xyz,
                        int64_t nc, const int64_t* cell_nodes, int64_t nb,
                        const int64_t* bface_nodes, const int32_t* bface_tag) {
  if (!c) return HOFV_EINVAL;
  invalidate_graphs(c);
  if (dim != 2 && dim != 3) return fail(c, HOFV_EINVAL, "dim must be 2 or 3");
  if (cell_kind != HOFV_CELL_TENSOR && cell_kind != HOFV_CELL_SIMPLEX)
    return fail(c, HOFV_EINVAL, "cell_kind must be HOFV_CELL_TENSOR or HOFV_CELL_SIMPLEX");
  if (nn <= 0 || nc <= 0 || !xyz || !cell_nodes || nb < 0 || (nb > 0 && (!bface_nodes || !bface_tag)))
    return fail(c, HOFV_EINVAL, "empty mesh or null array");
  if (nn >= (int64_t)1 << 31 || nc >= (int64_t)1 << 30)
    return fail(c, HOFV_EINVAL, "mesh too large for 32-bit ids");
  free_built(c);
  c->have_mesh = false;
  c->dim = dim;
  c->poly = false;
  c->polyh = false;
  c->cnv.clear();
  c->simplex = cell_kind == HOFV_CELL_SIMPLEX;
  c->nv = c->simplex ? dim + 1 : (dim == 2 ? 4 : 8);
  c->nlf = c->simplex ? dim + 1 : 2 * dim;
  c->nfv = c->simplex ? dim : (dim == 2 ? 2 : 4);
  c->nn = nn;
  c->nc = nc;
  c->nb = nb;
  c->x.assign((size_t)nn * 3, 0.0);
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < dim; ++a) c->x[3 * i + a] = xyz[dim * i + a];
  c->cn.assign(cell_nodes, cell_nodes + nc * c->nv);
  for (int64_t i = 0; i < nc * c->nv; ++i)
    if (c->cn[i] < 0 || c->cn[i] >= nn) return fail(c, HOFV_EINVAL, "cell node id out of range");
  if (c->simplex)
    for (int64_t cell = 0; cell < nc; ++cell) {
      const int64_t* v = &c->cn[cell * c->nv];
      double e[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int k = 1; k <= dim; ++k)
        for (int a = 0; a < dim; ++a) e[k - 1][a] = c->x[3 * v[k] + a] - c->x[3 * v[0] + a];
      const double det = dim == 2 ? e[0][0] * e[1][1] - e[0][1] * e[1][0]
                                  : e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                                        e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                                        e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
      if (!(det > 0)) return fail(c, HOFV_EINVAL, "simplex cell not positively oriented");
    }
  return build_faces(c, nb, bface_nodes, bface_tag);
}

int hofv_set_mesh_polygons(hofv_ctx* c, int64_t nn, const double* xyz, int64_t nc,
                           const int64_t* cell_ptr, const int64_t* cell_nodes, int64_t nb,
                           const int64_t* bface_nodes, const int32_t* bface_tag) {
  if (!c) return HOFV_EINVAL;
  invalidate_graphs(c);
  if (nn <= 0 || nc <= 0 || !xyz || !cell_ptr || !cell_nodes || nb < 0 ||
      (nb > 0 && (!bface_nodes || !bface_tag)))
    return fail(c, HOFV_EINVAL, "empty mesh or null array");
  if (nn >= (int64_t)1 << 31 || nc >= (int64_t)1 << 30)
    return fail(c, HOFV_EINVAL, "mesh too large for 32-bit ids");
  if (cell_ptr[0] != 0) return fail(c, HOFV_EINVAL, "cell_ptr[0] must be 0");
  for (int64_t cell = 0; cell < nc; ++cell) {
    const int64_t k = cell_ptr[cell + 1] - cell_ptr[cell];
    if (k < 3 || k > kPolyMaxSides)
      return fail(c, HOFV_EINVAL, "a polygon must have 3 to 8 corners");
  }
  free_built(c);
  c->have_mesh = false;
  c->dim = 2;
  c->simplex = false;
  c->polyh = false;
  c->poly = true;
  c->nv = c->nlf = kPolyMaxSides;
  c->nfv = 2;
  c->nn = nn;
  c->nc = nc;
  c->nb = nb;
  c->x.assign((size_t)nn * 3, 0.0);
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < 2; ++a) c->x[3 * i + a] = xyz[2 * i + a];
  c->cn.assign((size_t)nc * c->nv, -1);
  c->cnv.assign((size_t)nc, 0);
  for (int64_t cell = 0; cell < nc; ++cell) {
    const int64_t k = cell_ptr[cell + 1] - cell_ptr[cell];
    c->cnv[cell] = (int32_t)k;
    for (int64_t j = 0; j < k; ++j) {
      const int64_t v = cell_nodes[cell_ptr[cell] + j];
      if (v < 0 || v >= nn) return fail(c, HOFV_EINVAL, "cell node id out of range");
      c->cn[cell * c->nv + j] = v;
    }
    // every fan triangle (corner average, corner j, corner j+1) positively oriented
    double xb[2] = {0, 0};
    for (int64_t j = 0; j < k; ++j)
      for (int a = 0; a < 2; ++a) xb[a] += c->x[3 * c->cn[cell * c->nv + j] + a];
    for (int a = 0; a < 2; ++a) xb[a] /= (double)k;
    for (int64_t j = 0; j < k; ++j) {
      const double* p0 = &c->x[3 * c->cn[cell * c->nv + j]];
      const double* p1 = &c->x[3 * c->cn[cell * c->nv + (j + 1) % k]];
      const double cr = (p0[0] - xb[0]) * (p1[1] - xb[1]) - (p0[1] - xb[1]) * (p1[0] - xb[0]);
      if (!(cr > 0))
        return fail(c, HOFV_EINVAL, "polygon not counter-clockwise and star-shaped about its corners' average");
    }
  }
  return build_faces(c, nb, bface_nodes, bface_tag);
}

int hofv_set_mesh_faces(hofv_ctx* c, int64_t nn, const double* xyz, int64_t nc, int64_t nf,
                        const int64_t* face_ptr, const int64_t* face_nodes, const int64_t* owner,
                        const int64_t* neighbour, const int32_t* face_tag) {
  if (!c) return HOFV_EINVAL;
  invalidate_graphs(c);
  if (nn <= 0 || nc <= 0 || nf <= 0 || !xyz || !face_ptr || !face_nodes || !owner || !neighbour ||
      !face_tag)
    return fail(c, HOFV_EINVAL, "empty mesh or null array");
  if (nn >= (int64_t)1 << 31 || nc >= (int64_t)1 << 30 || nf >= (int64_t)1 << 30)
    return fail(c, HOFV_EINVAL, "mesh too large for 32-bit ids");
  if (face_ptr[0] != 0) return fail(c, HOFV_EINVAL, "face_ptr[0] must be 0");
  int maxfv = 0;
  for (int64_t i = 0; i < nf; ++i) {
    const int64_t k = face_ptr[i + 1] - face_ptr[i];
    if (k < 3 || k > kPolyFaceMaxCorners)
      return fail(c, HOFV_EINVAL, "a face must have 3 to 8 corners");
    for (int64_t j = face_ptr[i]; j < face_ptr[i + 1]; ++j)
      if (face_nodes[j] < 0 || face_nodes[j] >= nn)
        return fail(c, HOFV_EINVAL, "face node id out of range");
    if (owner[i] < 0 || owner[i] >= nc || neighbour[i] >= nc || neighbour[i] == owner[i])
      return fail(c, HOFV_EINVAL, "bad owner or neighbour");
    if (neighbour[i] < 0 && (face_tag[i] < 0 || face_tag[i] > 2))
      return fail(c, HOFV_EINVAL, "bad boundary tag");
    maxfv = std::max(maxfv, (int)k);
  }
  std::vector<int> nfc((size_t)nc, 0);
  for (int64_t i = 0; i < nf; ++i) {
    ++nfc[owner[i]];
    if (neighbour[i] >= 0) ++nfc[neighbour[i]];
  }
  for (int64_t cell = 0; cell < nc; ++cell)
    if (nfc[cell] < 4 || nfc[cell] > kPolyhedronMaxFaces)
      return fail(c, HOFV_EINVAL, "a cell must have 4 to 16 faces");
  free_built(c);
  c->have_mesh = false;
  c->dim = 3;
  c->simplex = false;
  c->poly = false;
  c->polyh = true;
  c->cnv.clear();
  c->nv = 0;
  c->nlf = kPolyhedronMaxFaces;
  // corner slots of a face: 4 or 8, so that the face kernels see one of a
  // few point counts (slots past a face's last corner carry zero area)
  const int nfv = maxfv <= 4 ? 4 : kPolyFaceMaxCorners;
  c->nfv = nfv;
  c->nn = nn;
  c->nc = nc;
  c->x.assign(xyz, xyz + nn * 3);
  c->cn.clear();
  // owner = the lower cell id (the face flipped where the input's owner is
  // the higher one); a cell's local faces are its faces in input order
  std::vector<int64_t> own((size_t)nf), nei((size_t)nf);
  std::vector<char> flip((size_t)nf, 0);
  std::vector<int> fill((size_t)nc, 0), lfo((size_t)nf), lfn((size_t)nf, -1);
  int64_t nfi = 0, nfd = 0, nfy = 0, nft = 0;
  for (int64_t i = 0; i < nf; ++i) {
    own[i] = owner[i];
    nei[i] = neighbour[i];
    if (nei[i] >= 0 && nei[i] < own[i]) {
      std::swap(own[i], nei[i]);
      flip[i] = 1;
    }
    lfo[i] = fill[own[i]]++;
    if (nei[i] >= 0) lfn[i] = fill[nei[i]]++;
    if (nei[i] >= 0) ++nfi;
    else if (face_tag[i] == 0) ++nfd;
    else if (face_tag[i] == 2) ++nfy;
    else ++nft;
  }
  // canonical order: internal faces by (owner, owner's local face), then
  // displacement, symmetry and traction faces in input order
  std::vector<int64_t> order;
  order.reserve((size_t)nf);
  for (int64_t i = 0; i < nf; ++i)
    if (nei[i] >= 0) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return own[a] != own[b] ? own[a] < own[b] : lfo[a] < lfo[b];
  });
  for (int tag : {0, 2, 1})
    for (int64_t i = 0; i < nf; ++i)
      if (nei[i] < 0 && face_tag[i] == tag) order.push_back(i);
  c->nb = nfd + nfy + nft;
  c->nfi = nfi;
  c->nfd = nfd;
  c->nfy = nfy;
  c->nft = nft;
  c->nfid = nfi + nfd + nfy;
  c->nf = nf;
  c->fown.assign(nf, -1);
  c->fnei.assign(nf, -1);
  c->flf.assign(nf, 0);
  c->ftag.assign(nf, -1);
  c->cf.assign((size_t)nc * c->nlf, -1);
  c->fnodes.assign((size_t)nf * nfv, -1);
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t i = order[f];
    const int64_t k = face_ptr[i + 1] - face_ptr[i];
    c->fown[f] = own[i];
    c->fnei[f] = nei[i];
    c->flf[f] = lfo[i];
    c->ftag[f] = nei[i] >= 0 ? -1 : face_tag[i];
    for (int64_t t = 0; t < k; ++t)
      c->fnodes[f * nfv + t] = (int32_t)face_nodes[face_ptr[i] + (flip[i] ? k - 1 - t : t)];
    c->cf[own[i] * c->nlf + lfo[i]] = f;
    if (nei[i] >= 0) c->cf[nei[i] * c->nlf + lfn[i]] = f;
  }
  c->maxtets = 0;
  for (int64_t cell = 0; cell < nc; ++cell) {
    int t = 0;
    for (int lf = 0; lf < c->nlf; ++lf) {
      const int64_t f = c->cf[cell * c->nlf + lf];
      if (f < 0) continue;
      int k = 0;
      while (k < nfv && c->fnodes[f * nfv + k] >= 0) ++k;
      t += k;
    }
    c->maxtets = std::max(c->maxtets, t);
  }
  c->have_mesh = true;
  c->built = false;
  return HOFV_OK;
}

int hofv_set_scheme(hofv_ctx* c, int p, int n_plus, int q1, double k_weight, double alpha) {
  if (!c) return HOFV_EINVAL;
  invalidate_graphs(c);
  if (!c->have_mesh) return fail(c, HOFV_ESTATE, "hofv_set_mesh must come first");
  if (p < 1 || p > 3) return fail(c, HOFV_EINVAL, "p must be 1..3");
  if (q1 < 1 || q1 > 4 || (c->dim == 3 && q1 > 3))
    return fail(c, HOFV_EINVAL, "q_per_dir must be 1..4 in 2-D and 1..3 in 3-D");
  if (c->polyh && q1 > 2)
    return fail(c, HOFV_EINVAL, "q_per_dir must be 1..2 on polyhedra (8 q^2 points a face)");
  if (n_plus < 0 || !(k_weight > 0) || !(alpha >= 0)) return fail(c, HOFV_EINVAL, "bad scheme parameter");
  int nt = 1;
  for (int i = 1; i <= c->dim; ++i) nt = nt * (p + i) / i;
  if (nt + n_plus + 1 > kMaxS) return fail(c, HOFV_EINVAL, "stencil too large");
  if (nt + n_plus > c->nc) return fail(c, HOFV_EINVAL, "stencil larger than the mesh");
  free_built(c);
  c->p = p;
  c->nplus = n_plus;
  c->q1 = q1;
  c->Nt = nt;
  c->S = nt + n_plus;
  c->Q = c->polyh ? c->nfv * q1 * q1 : c->dim == 2 ? q1 : q1 * q1;
  c->QC = c->polyh  ? c->maxtets * q1 * q1 * q1
          : c->poly ? c->nlf * q1 * q1
          : c->dim == 2 ? q1 * q1 : q1 * q1 * q1;
  c->kw = k_weight;
  c->alpha = alpha;
  gauss_rule(q1, c->gl_x, c->gl_w);
  c->have_scheme = true;
  return HOFV_OK;
}


int hofv_build_stencils(hofv_ctx* c) {
  if (!c) return HOFV_EINVAL;
  if (!c->have_mesh || !c->have_scheme) return fail(c, HOFV_ESTATE, "mesh and scheme must be set first");
  HOFV_CUDA(c, cudaSetDevice(c->device));
  const auto t0 = std::chrono::steady_clock::now();
  free_built(c);
  const int d = c->dim, nlf = c->nlf;
  const int64_t nc = c->nc, nf = c->nf;
  c->nftile = (c->nfid + kTile - 1) / kTile;
  c->nctile = (nc + kTile - 1) / kTile;
  const int R = c->Q * d;
  // ---- uploads ----
  TRY(dev_alloc(c, &c->d_x, c->nn * 3));
  TRY(dev_alloc(c, &c->d_fnodes, nf * c->nfv));
  TRY(dev_alloc(c, &c->d_cnodes, nc * c->nv));
  TRY(dev_alloc(c, &c->d_cf, nc * nlf));
  TRY(dev_alloc(c, &c->d_ftag, nf));
  TRY(dev_alloc(c, &c->d_fown, nf));
  TRY(dev_alloc(c, &c->d_fnei, nf));
  TRY(dev_alloc(c, &c->d_cface, nc * nlf));
  std::vector<int32_t> tmp32((size_t)std::max(nc * c->nv, std::max(nc * nlf, nf)));
  HOFV_CUDA(c, cudaMemcpy(c->d_x, c->x.data(), sizeof(double) * c->nn * 3, cudaMemcpyHostToDevice));
  HOFV_CUDA(c, cudaMemcpy(c->d_fnodes, c->fnodes.data(), sizeof(int32_t) * nf * c->nfv,
                          cudaMemcpyHostToDevice));
  for (int64_t i = 0; i < nc * c->nv; ++i) tmp32[i] = (int32_t)c->cn[i];
  HOFV_CUDA(c, cudaMemcpy(c->d_cnodes, tmp32.data(), sizeof(int32_t) * nc * c->nv, cudaMemcpyHostToDevice));
  HOFV_CUDA(c, cudaMemcpy(c->d_cf, c->cf.data(), sizeof(int64_t) * nc * nlf, cudaMemcpyHostToDevice));
  HOFV_CUDA(c, cudaMemcpy(c->d_ftag, c->ftag.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice));
  for (int64_t i = 0; i < nf; ++i) tmp32[i] = (int32_t)c->fown[i];
  HOFV_CUDA(c, cudaMemcpy(c->d_fown, tmp32.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice));
  for (int64_t i = 0; i < nf; ++i) tmp32[i] = (int32_t)c->fnei[i];
  HOFV_CUDA(c, cudaMemcpy(c->d_fnei, tmp32.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice));
  for (int64_t cell = 0; cell < nc; ++cell)
    for (int lf = 0; lf < nlf; ++lf) {
      const int64_t f = c->cf[cell * nlf + lf];  // -1: polygon slot without a face
      tmp32[cell * nlf + lf] = f < 0 || c->ftag[f] == 1 ? 0 : (c->fown[f] == cell ? (int32_t)(f + 1) : -(int32_t)(f + 1));
    }
  HOFV_CUDA(c, cudaMemcpy(c->d_cface, tmp32.data(), sizeof(int32_t) * nc * nlf, cudaMemcpyHostToDevice));
  std::vector<int32_t>().swap(tmp32);
  // ---- geometry ----
  TRY(dev_alloc(c, &c->d_xc, nc * 3));
  TRY(dev_alloc(c, &c->d_vol, nc));
  TRY(dev_alloc(c, &c->d_xq, nf * c->Q * 3));
  TRY(dev_alloc(c, &c->d_aq, nf * c->Q * 3));
  TRY(dev_alloc(c, &c->d_xf, nf * 3));
  TRY(dev_alloc(c, &c->d_nrm, nf * 3));
  TRY(dev_alloc(c, &c->d_gam, nf));
  TRY(dev_alloc(c, &c->d_cqx, nc * c->QC * 3));
  TRY(dev_alloc(c, &c->d_cqw, nc * c->QC));
  TRY(run_geometry(c));
  // faces with more rows than one thread per (face, row) of a 32-face tile
  // allows take the strided FP64 face kernel, whose shared memory is raised
  if (kTile * c->Q * d > (d == 3 ? 864 : 256) &&
      (d != 3 || c->Q > kPolyFaceMaxCorners * 4 || flux_wide_prepare() != 0))
    return fail(c, HOFV_ENOTSUP, "too many face points for the face kernel");
  // reference length: power of two near the mean cell size (node bounding box)
  double vbox = 1.0;
  for (int a = 0; a < d; ++a) {
    double lo = c->x[a], hi = c->x[a];
    for (int64_t i = 1; i < c->nn; ++i) {
      lo = std::min(lo, c->x[3 * i + a]);
      hi = std::max(hi, c->x[3 * i + a]);
    }
    vbox *= (hi - lo);
  }
  {
    const int e = ilogb(vbox / (double)nc);
    c->href_exp = (int)floor((double)e / d);
  }
  // ---- buckets of centroids (host) ----
  std::vector<double> xc((size_t)nc * 3);
  HOFV_CUDA(c, cudaMemcpy(xc.data(), c->d_xc, sizeof(double) * nc * 3, cudaMemcpyDeviceToHost));
  const double bs = ldexp(1.0, c->href_exp);
  int nb[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    double l = xc[a], h = xc[a];
    for (int64_t i = 1; i < nc; ++i) {
      l = std::min(l, xc[3 * i + a]);
      h = std::max(h, xc[3 * i + a]);
    }
    lo[a] = l;
    nb[a] = (int)floor((h - l) / bs) + 1;
  }
  const int64_t nbk = (int64_t)nb[0] * nb[1] * nb[2];
  std::vector<int64_t> bstart((size_t)nbk + 1, 0);
  std::vector<int64_t> bid((size_t)nc);
  for (int64_t i = 0; i < nc; ++i) {
    int64_t id = 0;
    for (int a = d - 1; a >= 0; --a) {
      int k = (int)floor((xc[3 * i + a] - lo[a]) / bs);
      k = std::min(std::max(k, 0), nb[a] - 1);
      id = id * nb[a] + k;
    }
    bid[i] = id;
    bstart[id + 1]++;
  }
  for (int64_t i = 0; i < nbk; ++i) bstart[i + 1] += bstart[i];
  std::vector<int32_t> bitems((size_t)nc);
  {
    std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
    for (int64_t i = 0; i < nc; ++i) bitems[fill[bid[i]]++] = (int32_t)i;
  }
  // ---- stencils ----
  TRY(dev_alloc(c, &c->d_fst, std::max<int64_t>(c->nftile, 1) * c->S * kTile));
  TRY(dev_alloc(c, &c->d_cst, c->nctile * c->S * kTile));
  HOFV_CUDA(c, cudaMemset(c->d_fst, 0, sizeof(int32_t) * std::max<int64_t>(c->nftile, 1) * c->S * kTile));
  HOFV_CUDA(c, cudaMemset(c->d_cst, 0, sizeof(int32_t) * c->nctile * c->S * kTile));
  TRY(run_stencils(c, bstart, bitems, nb, lo, bs));
  // ---- reconstruction coefficients ----
  const int64_t nfco = std::max<int64_t>(c->nftile, 1) * c->S * kTile * R;
  TRY(dev_alloc(c, &c->d_fco, nfco));
  HOFV_CUDA(c, cudaMemset(c->d_fco, 0, sizeof(double) * nfco));
  TRY(dev_alloc(c, &c->d_gco, std::max<int64_t>(c->nfd + c->nfy, 1) * R));
  HOFV_CUDA(c, cudaMemset(c->d_gco, 0, sizeof(double) * std::max<int64_t>(c->nfd + c->nfy, 1) * R));
  TRY(run_ghosts(c));
  const int64_t ncex = c->nctile * c->S * kTile * nlf;
  TRY(dev_alloc(c, &c->d_cex, ncex));
  HOFV_CUDA(c, cudaMemset(c->d_cex, 0, sizeof(double) * ncex));
  TRY(run_lsq(c));
  // ---- per-face data and approximate Jacobian ----
  TRY(dev_alloc(c, &c->d_fstar, std::max<int64_t>(c->nfid, 1) * 2));
  TRY(dev_alloc(c, &c->d_fstab, std::max<int64_t>(c->nfid, 1)));
  if (c->polyh) {
    // points of each face with area: its corners x q^2 (the fan slots past a
    // face's last corner carry none); the face kernels skip the other rows
    const int64_t nfp = std::max<int64_t>(c->nftile, 1) * kTile;
    std::vector<int32_t> ql((size_t)nfp, 0);
    for (int64_t f = 0; f < std::min<int64_t>(c->nf, nfp); ++f) {
      int k = 0;
      while (k < c->nfv && c->fnodes[f * c->nfv + k] >= 0) ++k;
      ql[f] = k * c->q1 * c->q1;
    }
    TRY(dev_alloc(c, &c->d_fql, nfp));
    HOFV_CUDA(c, cudaMemcpy(c->d_fql, ql.data(), sizeof(int32_t) * nfp, cudaMemcpyHostToDevice));
    if (c->Q == 32) {
      // faces of 8 fan slots (Q = 32): consecutive faces of a tile packed into
      // groups whose rows with area fill the packed kernel's threads
      std::vector<int32_t> grp;
      for (int64_t t0 = 0; t0 < c->nfid; t0 += kTile) {
        const int64_t t1 = std::min<int64_t>(t0 + kTile, c->nfid);
        int64_t f = t0;
        while (f < t1) {
          int rows = 0, n = 0;
          while (f + n < t1 && n < kPackMaxFaces && rows + ql[f + n] * c->dim <= kPackThreads) {
            rows += ql[f + n] * c->dim;
            ++n;
          }
          if (n == 0) return fail(c, HOFV_EINVAL, "a polyhedral face has more points than a packed group");
          grp.push_back((int32_t)f);
          grp.push_back(n);
          f += n;
        }
      }
      c->npg = (int64_t)grp.size() / 2;
      TRY(dev_alloc(c, &c->d_pgrp, std::max<int64_t>(c->npg, 1) * 2));
      if (c->npg > 0)
        HOFV_CUDA(c, cudaMemcpy(c->d_pgrp, grp.data(), sizeof(int32_t) * grp.size(), cudaMemcpyHostToDevice));
    }
  }
  TRY(dev_alloc(c, &c->d_aj_diag, nc));
  TRY(dev_alloc(c, &c->d_aj_col, nc * nlf));
  TRY(dev_alloc(c, &c->d_aj_off, nc * nlf));
  TRY(dev_alloc(c, &c->d_aj_diag32, nc));
  TRY(dev_alloc(c, &c->d_aj_off32, nc * nlf));
  TRY(dev_alloc(c, &c->d_aj_invd, nc));
  TRY(dev_alloc(c, &c->d_bar, 4));
  HOFV_CUDA(c, cudaMemset(c->d_bar, 0, 4 * sizeof(unsigned int)));
  TRY(dev_alloc(c, &c->d_aj_invd32, nc));
  TRY(run_face_aux(c));
  // ---- boundary data, sources and scratch ----
  // displacement-face data, then (library-owned) symmetry-face slots
  const int64_t nfb = std::max<int64_t>(c->nfd + c->nfy, 1);
  TRY(dev_alloc(c, &c->d_ubq, nfb * c->Q * d));
  TRY(dev_alloc(c, &c->d_ubf, nfb * d));
  TRY(dev_alloc(c, &c->d_tbq, std::max<int64_t>(c->nft, 1) * c->Q * d));
  TRY(dev_alloc(c, &c->d_body, nc * d));
  TRY(dev_alloc(c, &c->d_src, nc * d));
  HOFV_CUDA(c, cudaMemset(c->d_ubq, 0, sizeof(double) * nfb * c->Q * d));
  HOFV_CUDA(c, cudaMemset(c->d_ubf, 0, sizeof(double) * nfb * d));
  HOFV_CUDA(c, cudaMemset(c->d_tbq, 0, sizeof(double) * std::max<int64_t>(c->nft, 1) * c->Q * d));
  HOFV_CUDA(c, cudaMemset(c->d_body, 0, sizeof(double) * nc * d));
  HOFV_CUDA(c, cudaMemset(c->d_src, 0, sizeof(double) * nc * d));
  TRY(dev_alloc(c, &c->d_ustar, nc * nlf * d));
  TRY(dev_alloc(c, &c->d_flux, std::max<int64_t>(c->nfid, 1) * d));
  TRY(dev_alloc(c, &c->d_w, nc * d));
  if (c->ng > 0) TRY(dev_alloc(c, &c->d_wext, (nc + c->ng) * d));
  // double-float scratch: split state and Jv direction, extrapolated values
  // of the direction, its extended copy
  TRY(dev_alloc(c, &c->d_su, (nc + c->ng) * split4(d)));
  TRY(dev_alloc(c, &c->d_sv, (nc + c->ng) * split4(d)));
  TRY(dev_alloc(c, &c->d_ustar_v, nc * nlf * d));
  TRY(dev_alloc(c, &c->d_fcsum, std::max<int64_t>(c->nftile, 1) * kTile * R));
  if (c->ng > 0) TRY(dev_alloc(c, &c->d_vext, (nc + c->ng) * d));
  {
    const int e = setup_df_kernels();
    if (e != 0) return cuda_fail(c, (cudaError_t)e, "cudaFuncSetAttribute(face kernels)");
  }
  if (c->prec == HOFV_PREC_DF64) TRY(coef_format(c, 1));
  c->red_blocks = 4 * c->sm_count;
  TRY(dev_alloc(c, &c->d_red, (int64_t)c->red_blocks * 128));
  TRY(dev_alloc(c, &c->d_count, 256));
  TRY(dev_alloc(c, &c->d_scal, 256));
  HOFV_CUDA(c, cudaMemset(c->d_count, 0, sizeof(unsigned int) * 256));
  HOFV_CUDA(c, cudaMemset(c->d_scal, 0, sizeof(double) * 256));
  TRY(dev_alloc(c, &c->d_cg64, 8 * nc * d));
  TRY(dev_alloc(c, &c->d_cg32, 8 * nc * d));
  HOFV_CUDA(c, cudaDeviceSynchronize());
  c->src_dirty = false;
  c->built = true;
  c->tco_valid = false;
  TRY(build_contraction(c));
  TRY(ensure_jv_storage(c));
  c->setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return HOFV_OK;
}

int hofv_get_layout(const hofv_ctx* c, hofv_layout* out) {
  if (!c || !out) return HOFV_EINVAL;
  if (!c->have_mesh || !c->have_scheme) return HOFV_ESTATE;
  out->dim = c->dim;
  out->p = c->p;
  out->stencil = c->S;
  out->n_t = c->Nt;
  out->q_face = c->Q;
  out->q_cell = c->QC;
  out->n_cells = c->nc;
  out->n_faces = c->nf;
  out->n_internal = c->nfi;
  out->n_disp = c->nfd;
  out->n_trac = c->nft;
  out->n_symm = c->nfy;
  out->max_cond = c->max_cond;
  out->setup_seconds = c->setup_seconds;
  out->device_bytes = c->device_bytes;
  return HOFV_OK;
}

int hofv_get_points(hofv_ctx* c, int kind, double* out) {
  if (!c || !out) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  const int d = c->dim, Q = c->Q;
  std::vector<double> buf;
  auto fetch = [&](const double* src, int64_t count) -> int {
    buf.resize((size_t)count);
    HOFV_CUDA(c, cudaMemcpy(buf.data(), src, sizeof(double) * count, cudaMemcpyDeviceToHost));
    return 0;
  };
  switch (kind) {
    case HOFV_PTS_CELL_CENTROID:
      TRY(fetch(c->d_xc, c->nc * 3));
      for (int64_t i = 0; i < c->nc; ++i)
        for (int a = 0; a < d; ++a) out[i * d + a] = buf[3 * i + a];
      return 0;
    case HOFV_PTS_CELL_VOLUME:
      TRY(fetch(c->d_vol, c->nc));
      memcpy(out, buf.data(), sizeof(double) * c->nc);
      return 0;
    case HOFV_PTS_CELL_QP:
      TRY(fetch(c->d_cqx, c->nc * c->QC * 3));
      for (int64_t i = 0; i < c->nc * c->QC; ++i)
        for (int a = 0; a < d; ++a) out[i * d + a] = buf[3 * i + a];
      return 0;
    case HOFV_PTS_FACE_CENTRE:
    case HOFV_PTS_DISP_CENTRE: {
      TRY(fetch(c->d_xf, c->nf * 3));
      const int64_t f0 = kind == HOFV_PTS_DISP_CENTRE ? c->nfi : 0;
      const int64_t nfx = kind == HOFV_PTS_DISP_CENTRE ? c->nfd : c->nf;
      for (int64_t i = 0; i < nfx; ++i)
        for (int a = 0; a < d; ++a) out[i * d + a] = buf[3 * (f0 + i) + a];
      return 0;
    }
    case HOFV_PTS_FACE_QP:
    case HOFV_PTS_DISP_QP:
    case HOFV_PTS_TRAC_QP:
    case HOFV_PTS_FACE_AREA: {
      TRY(fetch(kind == HOFV_PTS_FACE_AREA ? c->d_aq : c->d_xq, c->nf * Q * 3));
      int64_t f0 = 0, nfx = c->nf;
      if (kind == HOFV_PTS_DISP_QP) { f0 = c->nfi; nfx = c->nfd; }
      if (kind == HOFV_PTS_TRAC_QP) { f0 = c->nfi + c->nfd + c->nfy; nfx = c->nft; }
      for (int64_t i = 0; i < nfx * Q; ++i)
        for (int a = 0; a < d; ++a) out[i * d + a] = buf[3 * (f0 * Q + i) + a];
      return 0;
    }
    default:
      return fail(c, HOFV_EINVAL, "unknown point set");
  }
}

int hofv_set_material(hofv_ctx* c, int law, double mu, double lambda) {
  if (!c) return HOFV_EINVAL;
  if (law != HOFV_LAW_LINEAR && law != HOFV_LAW_NEOHOOKEAN) return fail(c, HOFV_EINVAL, "unknown law");
  if (!(mu > 0) || !(lambda > -2.0 * mu / 3.0)) return fail(c, HOFV_EINVAL, "bad material constants");
  invalidate_graphs(c);
  c->mat.law = law;
  c->mat.mu = mu;
  c->mat.lam = lambda;
  c->mat.kappa = lambda + 2.0 * mu / 3.0;
  c->mat.kbar = 2.0 * mu + lambda;
  c->mat.alpha = c->alpha;
  c->have_mat = true;
  c->tco_valid = false;
  jv_invalidate(c);
  TRY(ensure_jv_storage(c));
  if (c->built) {
    TRY(build_contraction(c));
    TRY(refresh_source(c));
    if (c->inertia) {  // the inertia diagonal of the AJ is scaled by 1 / Kbar
      TRY(run_aj_rows(c));
      mg_drop(c);
    }
  }
  return HOFV_OK;
}

int hofv_set_bc(hofv_ctx* c, const double* ubq, const double* ubf, const double* tbq,
                const double* body) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  const int d = c->dim;
  auto put = [&](double* dst, const double* src, int64_t count) -> int {
    if (count <= 0) return 0;
    if (src)
      HOFV_CUDA(c, cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToDevice, c->stream));
    else
      HOFV_CUDA(c, cudaMemsetAsync(dst, 0, sizeof(double) * count, c->stream));
    return 0;
  };
  TRY(put(c->d_ubq, ubq, c->nfd * c->Q * d));
  TRY(put(c->d_ubf, ubf, c->nfd * d));
  TRY(put(c->d_tbq, tbq, c->nft * c->Q * d));
  TRY(put(c->d_body, body, c->nc * d));
  jv_invalidate(c);  // the ghost-node data enter the cached gradients
  TRY(refresh_source(c));
  return HOFV_OK;
}

}  // extern "C"

namespace hofv {
__global__ void k_integrate(int dim, int QC, int64_t nc, const double* __restrict__ w,
                            const double* __restrict__ f, double* __restrict__ b) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  for (int j = 0; j < dim; ++j) {
    double s = 0.0;
    for (int q = 0; q < QC; ++q) s = fma(w[c * QC + q], f[(c * QC + q) * dim + j], s);
    b[j * nc + c] = s;
  }
}
}  // namespace hofv

extern "C" {

int hofv_integrate_cells(hofv_ctx* c, const double* f_qp, double* b) {
  if (!c || !f_qp || !b) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  k_integrate<<<(unsigned)((c->nc + 127) / 128), 128, 0, c->stream>>>(c->dim, c->QC, c->nc, c->d_cqw,
                                                                       f_qp, b);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}

static int check_eval(hofv_ctx* c) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (!c->have_mat) return fail(c, HOFV_ESTATE, "hofv_set_material must come first");
  c->mat.alpha = c->alpha;
  return 0;
}

int hofv_residual(hofv_ctx* c, const double* u, double* R) {
  TRY(check_eval(c));
  if (!u || !R) return fail(c, HOFV_EINVAL, "null vector");
  jv_touch(c, u);
  launch_residual(dev_mesh(c), c->mat, u, nullptr, nullptr, nullptr, R, c->d_ustar, c->d_flux,
                  c->d_ubq, c->d_ubf, c->d_src, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}

// Jv with ||u|| already in d_scal[0]: computes ||v||, eps, w = u + eps v and
// (R(w) - Ru) / eps into Jv.  eps stays in d_scal[2].
static int jvp_impl(hofv_ctx* c, const double* u, const double* Ru, const double* v, double* Jv,
                    cudaEvent_t* ev = nullptr) {
  const int64_t n = c->nc * c->dim;
  double* sc = c->d_scal;
  launch_norm2(v, n, c->d_red, c->d_count, sc + 1, c->red_blocks, c->stream);
  launch_jv_eps(sc + 0, sc + 1, sc + 2, c->stream);
  if (c->prec == HOFV_PREC_DF64) {  // the caller made the linearisation cache valid
    launch_jv_df(dev_mesh(c), c->mat, v, sc + 2, Jv, c->d_flux, c->stream, ev);
    HOFV_CUDA(c, cudaGetLastError());
    return 0;
  }
  launch_waxpy_dev(c->d_w, u, v, sc + 2, 1.0, n, c->stream);
  launch_residual(dev_mesh(c), c->mat, c->d_w, nullptr, sc + 2, Ru, Jv, c->d_ustar, c->d_flux,
                  c->d_ubq, c->d_ubf, c->d_src, c->stream, ev);
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

int hofv_jvp(hofv_ctx* c, const double* u, const double* Ru, const double* v, double* Jv,
             double* eps_used) {
  TRY(check_eval(c));
  if (!u || !Ru || !v || !Jv) return fail(c, HOFV_EINVAL, "null vector");
  const int64_t n = c->nc * c->dim;
  launch_norm2(u, n, c->d_red, c->d_count, c->d_scal + 0, c->red_blocks, c->stream);
  TRY(ensure_jv_cache(c, u, Ru));
  TRY(jvp_impl(c, u, Ru, v, Jv));
  if (eps_used) {
    HOFV_CUDA(c, cudaMemcpyAsync(eps_used, c->d_scal + 2, sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
    HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return HOFV_OK;
}

int hofv_jvp_timed(hofv_ctx* c, const double* u, const double* Ru, const double* v, double* Jv,
                   float* ms) {
  TRY(check_eval(c));
  if (!u || !Ru || !v || !Jv || !ms) return fail(c, HOFV_EINVAL, "null argument");
  const int64_t n = c->nc * c->dim;
  launch_norm2(u, n, c->d_red, c->d_count, c->d_scal + 0, c->red_blocks, c->stream);
  TRY(ensure_jv_cache(c, u, Ru));
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) HOFV_CUDA(c, cudaEventCreate(&ev[i]));
  const int rc = jvp_impl(c, u, Ru, v, Jv, ev);
  cudaError_t e = rc == 0 ? cudaEventSynchronize(ev[3]) : cudaSuccess;
  for (int i = 0; i < 3 && rc == 0 && e == cudaSuccess; ++i)
    e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  if (rc != 0) return rc;
  HOFV_CUDA(c, e);
  return HOFV_OK;
}

int hofv_precondition(hofv_ctx* c, int kind, int iters, const double* v, double* z) {
  TRY(check_eval(c));
  if (!v || !z) return fail(c, HOFV_EINVAL, "null vector");
  if (iters < 0 || iters > 100000) return fail(c, HOFV_EINVAL, "bad inner iteration count");
  const int64_t n = c->nc * c->dim;
  switch (kind) {
    case HOFV_PC_NONE:
      HOFV_CUDA(c, cudaMemcpyAsync(z, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      return HOFV_OK;
    case HOFV_PC_AJ64:
    case HOFV_PC_AJ32:
      return aj_precondition(c, kind, iters, v, z);
    case HOFV_PC_AJMG:
      return mg_precondition(c, iters, v, z);
    case HOFV_PC_NEJ:
      return nej_precondition(c, iters, v, z);
    case HOFV_PC_GNN: {
      if (!c->gnn) return fail(c, HOFV_ESTATE, "no learned preconditioner loaded");
      TRY(aj_precondition(c, HOFV_PC_AJ32, iters, v, z));
      return gnn_apply(c, v, z, z);
    }
    default:
      return fail(c, HOFV_EINVAL, "unknown preconditioner");
  }
}

void hofv_default_opts(hofv_solve_opts* o) {
  if (!o) return;
  o->max_newton = 30;
  o->rtol = 1e-8;
  o->atol = 0.0;
  o->ftol = 0.0;
  o->restart = 30;
  o->max_krylov = 300;
  o->eta_max = 1e-2;
  o->precond = HOFV_PC_AJ32;
  o->inner_iters = 30;
  o->line_search_max = 10;
  o->verbose = 0;
  o->record_pairs = 0;
  o->gnn_judge = 1;
}

}  // extern "C"

namespace hofv {

// ---------------------------------------------------------------------
// The device part of one flexible Arnoldi step, z_j = M v_j, w = J z_j,
// w -= V (V^T w) twice, |w| (and, for the stand-alone step, v_{j+1} =
// w / |w|), is 20-30 kernel launches whose arguments stay the same for a
// given basis index j as long as the mesh, scheme, material and buffers do.
// It is captured once per such key into a CUDA graph and replayed with one
// launch; a change of any of them (the context's generation) drops the
// graphs.  Captured only for the preconditioners made of plain kernel
// launches (none, multigrid); capture happens on a private stream, so the
// caller's stream may be the legacy default stream.
// ---------------------------------------------------------------------
struct ArnoldiKey {
  uint64_t gen;
  int kind, inner, j, with_unorm, with_scale;
  const double *u, *Ru, *V, *Z, *w, *dh;
  int64_t ld, dstride;
  bool operator==(const ArnoldiKey& o) const {
    return gen == o.gen && kind == o.kind && inner == o.inner && j == o.j &&
           with_unorm == o.with_unorm && with_scale == o.with_scale && u == o.u && Ru == o.Ru &&
           V == o.V && Z == o.Z && w == o.w && dh == o.dh && ld == o.ld && dstride == o.dstride;
  }
};
struct GraphCache {
  std::vector<std::pair<ArnoldiKey, cudaGraphExec_t>> items;
  bool broken = false;  // a capture failed once: launch directly from then on
};
constexpr size_t kMaxGraphs = 128;

static void graphs_clear(hofv_ctx* c) {
  GraphCache* g = static_cast<GraphCache*>(c->graphs);
  if (!g) return;
  for (auto& it : g->items) cudaGraphExecDestroy(it.second);
  delete g;
  c->graphs = nullptr;
}

static int apply_pc(hofv_ctx* c, const hofv_solve_opts& o, const double* v, double* z,
                    hofv_stats* st);
static int arnoldi_launch(hofv_ctx* c, const hofv_solve_opts& o, const ArnoldiKey& k,
                          hofv_stats* st) {
  const int64_t n = c->nc * c->dim;
  double* V = const_cast<double*>(k.V);
  double* Z = const_cast<double*>(k.Z);
  double* w = const_cast<double*>(k.w);
  double* dh = const_cast<double*>(k.dh);
  double* Vj = V + (int64_t)k.j * k.ld;
  double* Zj = Z + (int64_t)k.j * k.ld;
  const int nv = k.j + 1;
  TRY(apply_pc(c, o, Vj, Zj, st));
  if (k.with_unorm) launch_norm2(k.u, n, c->d_red, c->d_count, c->d_scal + 0, c->red_blocks, c->stream);
  TRY(jvp_impl(c, k.u, k.Ru, Zj, w));
  launch_dots(V, k.ld, w, nv, n, c->d_red, c->d_count, dh, c->red_blocks, c->stream, 0);
  launch_multi_axpy(w, V, dh, nv, n, k.ld, c->stream);
  launch_dots(V, k.ld, w, nv, n, c->d_red, c->d_count, dh + k.dstride, c->red_blocks, c->stream, 0);
  launch_multi_axpy(w, V, dh + k.dstride, nv, n, k.ld, c->stream);
  launch_norm2(w, n, c->d_red, c->d_count, dh + 2 * k.dstride, c->red_blocks, c->stream);
  if (k.with_scale)
    launch_scale_copy(V + (int64_t)(k.j + 1) * k.ld, w, dh + 2 * k.dstride, 1, n, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

static bool graphs_enabled() {
  const char* e = getenv("HOFV_GRAPHS");
  return !(e && e[0] == '0');
}

static int arnoldi_device(hofv_ctx* c, const hofv_solve_opts& o, const ArnoldiKey& k,
                          hofv_stats* st) {
  const bool graphable = (o.precond == HOFV_PC_NONE || o.precond == HOFV_PC_AJMG) &&
                         graphs_enabled();
  GraphCache* g = static_cast<GraphCache*>(c->graphs);
  if (!graphable || (g && g->broken)) return arnoldi_launch(c, o, k, st);
  if (!g) c->graphs = g = new GraphCache();
  for (auto& it : g->items) {
    if (it.first == k) {
      st->precond_applies++;
      HOFV_CUDA(c, cudaGraphLaunch(it.second, c->stream));
      return 0;
    }
  }
  if (o.precond == HOFV_PC_AJMG) TRY(mg_ensure(c));  // synchronising set-up, outside capture
  if (!c->cap) HOFV_CUDA(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (g->items.size() >= kMaxGraphs) {
    for (auto& it : g->items) cudaGraphExecDestroy(it.second);
    g->items.clear();
  }
  cudaStream_t user = c->stream;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  int rc = 0;
  if (e == cudaSuccess) {
    c->stream = c->cap;
    hofv_stats dummy = *st;
    rc = arnoldi_launch(c, o, k, &dummy);
    c->stream = user;
    e = cudaStreamEndCapture(c->cap, &graph);
  }
  if (e == cudaSuccess && rc == 0) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || rc != 0 || !exec) {
    cudaGetLastError();  // clear the capture error and launch directly from now on
    g->broken = true;
    return arnoldi_launch(c, o, k, st);
  }
  g->items.emplace_back(k, exec);
  st->precond_applies++;
  HOFV_CUDA(c, cudaGraphLaunch(exec, c->stream));
  return 0;
}

// host-side FGMRES state for one linear solve J x = b
struct Fgmres {
  std::vector<double> H;   // [(m+1) x m] column-major
  std::vector<double> cs, sn, g, y, hbuf;
};

static int ensure_krylov(hofv_ctx* c, int m) {
  if (c->kry_m >= m) return 0;
  const int64_t n = c->nc * c->dim;
  dev_free(c, c->d_V);
  dev_free(c, c->d_Z);
  dev_free(c, c->d_kvec);
  dev_free(c, c->d_h);
  c->d_V = c->d_Z = c->d_kvec = c->d_h = nullptr;
  TRY(dev_alloc(c, &c->d_V, (int64_t)(m + 1) * n));
  TRY(dev_alloc(c, &c->d_Z, (int64_t)m * n));
  TRY(dev_alloc(c, &c->d_kvec, 6 * n));
  TRY(dev_alloc(c, &c->d_h, 4 * (int64_t)(std::max(m, 100) + 2)));
  c->kry_m = m;
  return 0;
}

static int apply_pc(hofv_ctx* c, const hofv_solve_opts& o, const double* v, double* z,
                    hofv_stats* st) {
  st->precond_applies++;
  if (o.precond == HOFV_PC_NONE) {
    HOFV_CUDA(c, cudaMemcpyAsync(z, v, sizeof(double) * c->nc * c->dim, cudaMemcpyDeviceToDevice,
                                 c->stream));
    return 0;
  }
  if (o.precond == HOFV_PC_GNN && c->gnn) {
    TRY(aj_precondition(c, HOFV_PC_AJ32, o.inner_iters, v, z));
    return gnn_apply(c, v, z, z);
  }
  if (o.precond == HOFV_PC_AJMG) return mg_precondition(c, o.inner_iters, v, z);
  if (o.precond == HOFV_PC_NEJ) return nej_precondition(c, o.inner_iters, v, z);
  return aj_precondition(c, o.precond == HOFV_PC_AJ64 ? HOFV_PC_AJ64 : HOFV_PC_AJ32, o.inner_iters, v,
                         z);
}

static double dev_norm(hofv_ctx* c, const double* x, int64_t n) {
  launch_norm2(x, n, c->d_red, c->d_count, c->d_scal + 16, c->red_blocks, c->stream);
  double v = 0;
  cudaMemcpyAsync(&v, c->d_scal + 16, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return v;
}

// Solve J x = b (b = -R(u)), x zero on entry, to ||b - J x|| <= tol.
// Flexible GMRES(m), right preconditioning, classical Gram-Schmidt with one
// re-orthogonalisation; Jv by forward differences about u (||u|| in d_scal[0]).
static int fgmres(hofv_ctx* c, const hofv_solve_opts& o, const double* u, const double* Ru,
                  const double* b, double* x, double tol, int max_it, hofv_stats* st,
                  int* its_out, double* res_out) {
  const int64_t n = c->nc * c->dim;
  const int m = o.restart;
  double* V = c->d_V;
  double* Z = c->d_Z;
  double* w = c->d_kvec;
  double* r = c->d_kvec + n;
  double* dh = c->d_h;
  Fgmres F;
  F.H.assign((size_t)(m + 1) * m, 0.0);
  F.cs.assign(m, 0.0);
  F.sn.assign(m, 0.0);
  F.g.assign(m + 1, 0.0);
  F.y.assign(m, 0.0);
  F.hbuf.assign(2 * (m + 2), 0.0);
  HOFV_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
  HOFV_CUDA(c, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  TRY(ensure_jv_cache(c, u, Ru));
  int total = 0;
  double res = dev_norm(c, r, n);
  const double res0 = res;
  // the learned preconditioner stays on only while its restart cycles reduce
  // the residual at least as fast per iteration as the last AJ cycle did
  hofv_solve_opts oc = o;
  if (oc.precond == HOFV_PC_GNN && !c->gnn) oc.precond = HOFV_PC_AJ32;
  while (total < max_it) {
    if (res <= tol || res == 0.0) break;
    const double beta = res;
    const bool cycle_gnn = oc.precond == HOFV_PC_GNN;
    bool broken = false;
    HOFV_CUDA(c, cudaMemcpyAsync(c->d_scal + 20, &beta, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_scale_copy(V, r, c->d_scal + 20, 1, n, c->stream);
    std::fill(F.g.begin(), F.g.end(), 0.0);
    F.g[0] = beta;
    int j = 0;
    for (; j < m && total < max_it; ++j) {
      double* Vj = V + (int64_t)j * n;
      double* Zj = Z + (int64_t)j * n;
      // (J z, z) is an exact pair of the inverse Jacobian: keep a few from
      // the Krylov space as training data for the learned preconditioner
      const bool rec =
          o.record_pairs >= 2 && !cycle_gnn && (j == 0 || j == 3 || j == 8 || j == 15 || j == 24);
      if (rec) {
        TRY(apply_pc(c, oc, Vj, Zj, st));
        TRY(jvp_impl(c, u, Ru, Zj, w));
        TRY(hofv_gnn_record(c, w, Zj));
        // classical Gram-Schmidt, twice
        launch_dots(V, n, w, j + 1, n, c->d_red, c->d_count, dh, c->red_blocks, c->stream, 0);
        launch_multi_axpy(w, V, dh, j + 1, n, n, c->stream);
        launch_dots(V, n, w, j + 1, n, c->d_red, c->d_count, dh + (m + 2), c->red_blocks, c->stream, 0);
        launch_multi_axpy(w, V, dh + (m + 2), j + 1, n, n, c->stream);
        launch_norm2(w, n, c->d_red, c->d_count, dh + 2 * (m + 2), c->red_blocks, c->stream);
      } else {
        const ArnoldiKey key{c->gen, oc.precond, oc.inner_iters, j, 0, 0, u, Ru, V, Z, w, dh,
                             n, m + 2};
        TRY(arnoldi_device(c, oc, key, st));
      }
      st->residual_evals++;
      HOFV_CUDA(c, cudaMemcpyAsync(F.hbuf.data(), dh, sizeof(double) * 2 * (m + 2),
                                   cudaMemcpyDeviceToHost, c->stream));
      double hn = 0.0;
      HOFV_CUDA(c, cudaMemcpyAsync(&hn, dh + 2 * (m + 2), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
      TRY(check_pc_barrier(c));
      if (!std::isfinite(hn) && cycle_gnn) {
        // learned preconditioner failed: drop this cycle, continue with AJ
        oc.precond = HOFV_PC_AJ32;
        st->gnn_fallbacks++;
        broken = true;
        break;
      }
      if (!std::isfinite(hn)) return fail(c, HOFV_ENAN, "non-finite value in the Krylov basis");
      double* Hc = F.H.data() + (size_t)j * (m + 1);
      for (int i = 0; i <= j; ++i) Hc[i] = F.hbuf[i] + F.hbuf[(m + 2) + i];
      Hc[j + 1] = hn;
      if (hn > 0.0) launch_scale_copy(V + (int64_t)(j + 1) * n, w, dh + 2 * (m + 2), 1, n, c->stream);
      for (int i = 0; i < j; ++i) {  // previous rotations
        const double t = F.cs[i] * Hc[i] + F.sn[i] * Hc[i + 1];
        Hc[i + 1] = -F.sn[i] * Hc[i] + F.cs[i] * Hc[i + 1];
        Hc[i] = t;
      }
      const double den = hypot(Hc[j], Hc[j + 1]);
      F.cs[j] = den > 0 ? Hc[j] / den : 1.0;
      F.sn[j] = den > 0 ? Hc[j + 1] / den : 0.0;
      Hc[j] = den;
      Hc[j + 1] = 0.0;
      F.g[j + 1] = -F.sn[j] * F.g[j];
      F.g[j] = F.cs[j] * F.g[j];
      res = fabs(F.g[j + 1]);
      ++total;
      st->krylov_iters++;
      if (res <= tol || hn == 0.0) {
        ++j;
        break;
      }
    }
    if (broken) {
      // restart from the current x without the failed cycle
      TRY(jvp_impl(c, u, Ru, x, w));
      st->residual_evals++;
      HOFV_CUDA(c, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      launch_axpby(r, -1.0, w, 1.0, n, c->stream);
      res = dev_norm(c, r, n);
      continue;
    }
    if (j > 0 && beta > 0.0 && cycle_gnn && o.gnn_judge) {
      const double rate = pow(std::max(res, 1e-300) / beta, 1.0 / j);
      const double judge = c->aj_rate > 0.0 ? c->aj_rate : 0.98;
      if (!(rate <= judge)) {
        oc.precond = HOFV_PC_AJ32;
        st->gnn_fallbacks++;
      }
    }
    // y = H^{-1} g (upper triangular j x j)
    for (int i = j - 1; i >= 0; --i) {
      double s = F.g[i];
      for (int k = i + 1; k < j; ++k) s -= F.H[(size_t)k * (m + 1) + i] * F.y[k];
      const double dgl = F.H[(size_t)i * (m + 1) + i];
      F.y[i] = dgl != 0.0 ? s / dgl : 0.0;
    }
    HOFV_CUDA(c, cudaMemcpyAsync(dh, F.y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, c->stream));
    launch_combine(x, Z, dh, j, n, n, c->stream);
    if (res <= tol || total >= max_it) break;
    // restart: r = b - J x
    TRY(jvp_impl(c, u, Ru, x, w));
    st->residual_evals++;
    HOFV_CUDA(c, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    launch_axpby(r, -1.0, w, 1.0, n, c->stream);
    res = dev_norm(c, r, n);
  }
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (o.precond != HOFV_PC_GNN && o.precond != HOFV_PC_NONE && total > 0 && res0 > 0.0)
    c->aj_rate = pow(std::max(res, 1e-300) / res0, 1.0 / total);
  *its_out = total;
  *res_out = res;
  return 0;
}

}  // namespace hofv

extern "C" int hofv_newton_solve(hofv_ctx* c, double* u, const hofv_solve_opts* opts,
                                 hofv_stats* stats) {
  TRY(check_eval(c));
  if (!u) return fail(c, HOFV_EINVAL, "null vector");
  hofv_solve_opts o;
  hofv_default_opts(&o);
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 100 || o.max_krylov < 1 || o.max_newton < 0 ||
      o.precond < HOFV_PC_NONE || o.precond > HOFV_PC_NEJ)
    return fail(c, HOFV_EINVAL, "bad solver options");
  hofv_stats st;
  memset(&st, 0, sizeof(st));
  const auto t0 = std::chrono::steady_clock::now();
  TRY(ensure_krylov(c, o.restart));
  hofv_solve_opts on = o;
  const int64_t n = c->nc * c->dim;
  double* R = c->d_kvec + 2 * n;
  double* du = c->d_kvec + 3 * n;
  double* ut = c->d_kvec + 4 * n;
  double* Rt = c->d_kvec + 5 * n;
  double atol = o.atol;
  if (o.ftol > 0.0) {
    double fs = 0.0;
    TRY(hofv_force_scale(c, u, &fs));
    st.residual_evals++;
    atol = std::max(atol, o.ftol * fs * sqrt((double)n));
  }
  TRY(hofv_residual(c, u, R));
  st.residual_evals++;
  double rn = dev_norm(c, R, n);
  const double r0 = rn;
  st.r0 = r0;
  if (o.verbose) fprintf(stderr, "[hofv] |R0| %.6e  absolute floor %.3e\n", r0, atol);
  int status = HOFV_WNOTCONV;
  if (!std::isfinite(rn)) {
    status = fail(c, HOFV_ENAN, "non-finite initial residual");
  } else {
    for (int it = 0; it <= o.max_newton; ++it) {
      if (rn <= o.rtol * r0 || rn <= atol || rn == 0.0) {
        status = HOFV_OK;
        break;
      }
      if (it == o.max_newton) break;
      // rhs -R into Rt, ||u|| into d_scal[0]
      HOFV_CUDA(c, cudaMemcpyAsync(Rt, R, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      launch_axpby(Rt, 0.0, Rt, -1.0, n, c->stream);
      launch_norm2(u, n, c->d_red, c->d_count, c->d_scal + 0, c->red_blocks, c->stream);
      const double eta = std::min(o.eta_max, rn / r0);
      const double tol = std::max(eta * rn, 0.5 * o.rtol * r0);
      int its = 0;
      double lres = 0.0;
      // once the learned preconditioner has lost to AJ in this solve, keep AJ
      const int fb0 = st.gnn_fallbacks;
      int rc = fgmres(c, on, u, R, Rt, du, tol, o.max_krylov, &st, &its, &lres);
      if (st.gnn_fallbacks > fb0) on.precond = HOFV_PC_AJ32;
      if (rc < 0) { status = rc; break; }
      if (o.record_pairs) {
        rc = hofv_gnn_record(c, Rt, du);  // (-R(u_k), du_k)
        if (rc < 0) { status = rc; break; }
      }
      if (o.verbose >= 2) {
        // true linear residual ||R + J du|| and its FD estimate with a 100x larger step
        double* w = c->d_kvec;
        TRY(ensure_jv_cache(c, u, R));
        TRY(jvp_impl(c, u, R, du, w));
        launch_axpby(w, 1.0, R, 1.0, n, c->stream);
        const double tr = dev_norm(c, w, n);
        const double dn = dev_norm(c, du, n);
        fprintf(stderr, "[hofv]   true linear residual %.3e (estimate %.3e, tol %.3e)  |du| %.3e\n", tr,
                lres, tol, dn);
      }
      // backtracking line search on ||R||
      double lam = 1.0, rt = 0.0;
      bool ok = false;
      for (int ls = 0; ls <= o.line_search_max; ++ls) {
        HOFV_CUDA(c, cudaMemcpyAsync(ut, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        launch_axpby(ut, lam, du, 1.0, n, c->stream);
        TRY(hofv_residual(c, ut, Rt));
        st.residual_evals++;
        rt = dev_norm(c, Rt, n);
        if (std::isfinite(rt) && rt <= (1.0 - 1e-4 * lam) * rn) {
          ok = true;
          break;
        }
        lam *= 0.5;
      }
      if (o.verbose)
        fprintf(stderr, "[hofv] newton %d |R| %.3e -> %.3e  krylov %d (lin res %.2e)  lambda %.3g\n", it,
                rn, rt, its, lres, lam);
      if (!ok) {
        status = fail(c, HOFV_WNOTCONV, "line search failed to reduce the residual");
        break;
      }
      HOFV_CUDA(c, cudaMemcpyAsync(u, ut, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      HOFV_CUDA(c, cudaMemcpyAsync(R, Rt, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      jv_invalidate(c);  // u moved
      rn = rt;
      st.newton_iters++;
    }
  }
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  st.r_final = rn;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  st.status = status;
  if (stats) *stats = st;
  return status;
}

// host copy of a coefficient array held as double-float pairs -> doubles
static void df_to_double(std::vector<double>& a) {
  for (double& x : a) {
    float hl[2];
    memcpy(hl, &x, sizeof(hl));
    x = (double)hl[0] + (double)hl[1];
  }
}

extern "C" {

int hofv_get_face_data(hofv_ctx* c, int64_t first, int64_t count, int32_t* stencil, double* coef) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (first < 0 || count < 0 || first + count > c->nf) return fail(c, HOFV_EINVAL, "face range");
  const int S = c->S, Q = c->Q, d = c->dim, R = Q * d;
  const int64_t hi = std::min(first + count, c->nfid);
  if (hi <= first) return HOFV_OK;
  const int64_t t0 = first / kTile, t1 = (hi - 1) / kTile + 1;
  std::vector<int32_t> st((size_t)(t1 - t0) * S * kTile);
  HOFV_CUDA(c, cudaMemcpy(st.data(), c->d_fst + t0 * S * kTile, sizeof(int32_t) * st.size(),
                          cudaMemcpyDeviceToHost));
  std::vector<double> co;
  std::vector<double> gc;
  if (coef) {
    co.resize((size_t)(t1 - t0) * S * kTile * R);
    HOFV_CUDA(c, cudaMemcpy(co.data(), c->d_fco + t0 * S * kTile * R, sizeof(double) * co.size(),
                            cudaMemcpyDeviceToHost));
    if (c->prec == HOFV_PREC_DF64) df_to_double(co);
    if (c->nfd + c->nfy > 0) {
      gc.resize((size_t)(c->nfd + c->nfy) * R);
      HOFV_CUDA(c, cudaMemcpy(gc.data(), c->d_gco, sizeof(double) * gc.size(), cudaMemcpyDeviceToHost));
    }
  }
  for (int64_t f = first; f < hi; ++f) {
    const int64_t t = f / kTile - t0, fi = f % kTile, o = f - first;
    for (int nn = 0; nn < S; ++nn) {
      int32_t id = st[(t * S + nn) * kTile + fi];
      if (id >= c->nc) id = c->gsrc_host[id - c->nc];  // a mirror node: report its source cell
      if (stencil) stencil[o * S + nn] = id;
      if (coef)
        for (int q = 0; q < Q; ++q)
          for (int i = 0; i < d; ++i)
            coef[((o * Q + q) * (S + 1) + nn) * d + i] = co[((t * S + nn) * kTile + fi) * R + q * d + i];
    }
    if (coef)
      for (int q = 0; q < Q; ++q)
        for (int i = 0; i < d; ++i)
          coef[((o * Q + q) * (S + 1) + S) * d + i] = f >= c->nfi ? gc[(f - c->nfi) * R + q * d + i] : 0.0;
  }
  return HOFV_OK;
}

int hofv_get_cell_data(hofv_ctx* c, int64_t first, int64_t count, int32_t* stencil, double* ext) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (first < 0 || count < 0 || first + count > c->nc) return fail(c, HOFV_EINVAL, "cell range");
  if (count == 0) return HOFV_OK;
  const int S = c->S, nlf = c->nlf;
  const int64_t hi = first + count;
  const int64_t t0 = first / kTile, t1 = (hi - 1) / kTile + 1;
  std::vector<int32_t> st((size_t)(t1 - t0) * S * kTile);
  HOFV_CUDA(c, cudaMemcpy(st.data(), c->d_cst + t0 * S * kTile, sizeof(int32_t) * st.size(),
                          cudaMemcpyDeviceToHost));
  std::vector<double> ex;
  if (ext) {
    ex.resize((size_t)(t1 - t0) * S * kTile * nlf);
    HOFV_CUDA(c, cudaMemcpy(ex.data(), c->d_cex + t0 * S * kTile * nlf, sizeof(double) * ex.size(),
                            cudaMemcpyDeviceToHost));
    if (c->prec == HOFV_PREC_DF64) df_to_double(ex);
  }
  for (int64_t cell = first; cell < hi; ++cell) {
    const int64_t t = cell / kTile - t0, ci = cell % kTile, o = cell - first;
    for (int nn = 0; nn < S; ++nn) {
      if (stencil) stencil[o * S + nn] = st[(t * S + nn) * kTile + ci];
      if (ext)
        for (int lf = 0; lf < nlf; ++lf)
          ext[(o * nlf + lf) * S + nn] = ex[((t * S + nn) * kTile + ci) * nlf + lf];
    }
  }
  return HOFV_OK;
}

int hofv_get_faces(hofv_ctx* c, int64_t* owner, int64_t* nei, int32_t* lf, int32_t* tag) {
  if (!c) return HOFV_EINVAL;
  if (!c->have_mesh) return fail(c, HOFV_ESTATE, "hofv_set_mesh must come first");
  if (owner) memcpy(owner, c->fown.data(), sizeof(int64_t) * c->nf);
  if (nei) memcpy(nei, c->fnei.data(), sizeof(int64_t) * c->nf);
  if (lf) memcpy(lf, c->flf.data(), sizeof(int32_t) * c->nf);
  if (tag) memcpy(tag, c->ftag.data(), sizeof(int32_t) * c->nf);
  return HOFV_OK;
}

int hofv_get_aj(hofv_ctx* c, double* diag, double* off) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (diag) HOFV_CUDA(c, cudaMemcpy(diag, c->d_aj_diag, sizeof(double) * c->nc, cudaMemcpyDeviceToHost));
  if (off && c->nfi > 0) {
    std::vector<double> fs((size_t)c->nfi);
    HOFV_CUDA(c, cudaMemcpy(fs.data(), c->d_fstab, sizeof(double) * c->nfi, cudaMemcpyDeviceToHost));
    memcpy(off, fs.data(), sizeof(double) * c->nfi);
  }
  return HOFV_OK;
}

}  // extern "C"

extern "C" int hofv_arnoldi_step(hofv_ctx* c, const double* u, const double* Ru, int kind,
                                 int inner_iters, double* V, double* Z, int64_t ld, int j,
                                 double* h) {
  TRY(check_eval(c));
  if (!u || !Ru || !V || !Z || !h) return fail(c, HOFV_EINVAL, "null argument");
  const int64_t n = c->nc * c->dim;
  if (j < 0 || j > 99 || ld < n) return fail(c, HOFV_EINVAL, "bad Arnoldi index or leading dimension");
  if (kind != HOFV_PC_NONE && kind != HOFV_PC_AJ64 && kind != HOFV_PC_AJ32 && kind != HOFV_PC_GNN &&
      kind != HOFV_PC_AJMG && kind != HOFV_PC_NEJ)
    return fail(c, HOFV_EINVAL, "unknown preconditioner");
  if (kind == HOFV_PC_GNN && !c->gnn) return fail(c, HOFV_ESTATE, "no learned preconditioner loaded");
  TRY(ensure_krylov(c, 1));
  double* w = c->d_kvec;
  double* dh = c->d_h;
  hofv_solve_opts o;
  hofv_default_opts(&o);
  o.precond = kind;
  o.inner_iters = inner_iters;
  hofv_stats st;
  memset(&st, 0, sizeof(st));
  const int k = j + 1;
  const ArnoldiKey key{c->gen, kind, inner_iters, j, 1, 1, u, Ru, V, Z, w, dh, ld, k};
  TRY(ensure_jv_cache(c, u, Ru));
  TRY(arnoldi_device(c, o, key, &st));
  std::vector<double> hb((size_t)(2 * k + 1));
  HOFV_CUDA(c, cudaMemcpyAsync(hb.data(), dh, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost,
                               c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  TRY(check_pc_barrier(c));
  for (int i = 0; i < k; ++i) h[i] = hb[i] + hb[k + i];
  h[k] = hb[2 * k];
  if (!std::isfinite(h[k])) return fail(c, HOFV_ENAN, "non-finite value in the Arnoldi step");
  return HOFV_OK;
}

extern "C" int hofv_residual_timed(hofv_ctx* c, const double* u, double* R, float* ms) {
  TRY(check_eval(c));
  if (!u || !R || !ms) return fail(c, HOFV_EINVAL, "null argument");
  jv_touch(c, u);
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) HOFV_CUDA(c, cudaEventCreate(&ev[i]));
  launch_residual(dev_mesh(c), c->mat, u, nullptr, nullptr, nullptr, R, c->d_ustar, c->d_flux,
                  c->d_ubq, c->d_ubf, c->d_src, c->stream, ev);
  cudaError_t e = cudaEventSynchronize(ev[3]);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  HOFV_CUDA(c, e);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}

extern "C" int hofv_force_scale(hofv_ctx* c, const double* u, double* fs) {
  TRY(check_eval(c));
  if (!u || !fs) return fail(c, HOFV_EINVAL, "null argument");
  jv_touch(c, u);
  launch_residual(dev_mesh(c), c->mat, u, nullptr, nullptr, nullptr, c->d_w, c->d_ustar, c->d_flux,
                  c->d_ubq, c->d_ubf, c->d_src, c->stream);
  launch_flux_scale(dev_mesh(c), c->d_flux, c->d_w, c->stream);
  std::vector<double> per((size_t)c->nc);
  HOFV_CUDA(c, cudaMemcpyAsync(per.data(), c->d_w, sizeof(double) * c->nc, cudaMemcpyDeviceToHost,
                               c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  double m = 0.0;
  for (double v : per) m = std::isnan(v) ? v : std::max(m, v);
  *fs = m;
  if (!std::isfinite(m)) return fail(c, HOFV_ENAN, "non-finite face flux");
  return HOFV_OK;
}

namespace hofv {
int check_pc_barrier(hofv_ctx* c) {
  if (!c->d_bar) return 0;
  int err = 0;
  HOFV_CUDA(c, cudaMemcpy(&err, c->d_bar + 2, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    HOFV_CUDA(c, cudaMemset(c->d_bar, 0, 4 * sizeof(unsigned int)));
    return fail(c, HOFV_ECUDA, "approximate-Jacobian solve: grid barrier timed out");
  }
  HOFV_CUDA(c, cudaMemcpy(&err, c->d_bar + 3, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    HOFV_CUDA(c, cudaMemset(c->d_bar + 3, 0, sizeof(unsigned int)));
    return fail(c, HOFV_ECUDA, "face kernel: a shared-memory copy did not complete in time");
  }
  return 0;
}
}  // namespace hofv

extern "C" int hofv_selftest_barrier(hofv_ctx* c, int32_t* timed_out) {
  if (!c || !timed_out) return HOFV_EINVAL;
  int t = 0;
  TRY(barrier_selftest(c, &t));
  *timed_out = t;
  return HOFV_OK;
}

extern "C" int hofv_mg_info(hofv_ctx* c, int32_t* levels, int64_t* sizes, int32_t max_sizes,
                            int64_t* nnz, double* setup_seconds) {
  if (!c || !levels || !nnz || !setup_seconds || (max_sizes > 0 && !sizes)) return HOFV_EINVAL;
  if (!c->built) return hofv::fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  TRY(hofv::mg_info(c, levels, sizes, max_sizes, nnz, setup_seconds));
  return HOFV_OK;
}

// ---------------------------------------------------------------------
// inertia term with BDF2 in time (eq. inertiaTerm, App. time integration)
// ---------------------------------------------------------------------
// cell-average weights of the cell fit, computed on first use
static int ensure_cmass(hofv_ctx* c) {
  if (c->d_cmass) return 0;
  const size_t count = (size_t)c->nctile * c->S * kTile;
  TRY(dev_alloc(c, &c->d_cmass, count));
  HOFV_CUDA(c, cudaMemsetAsync(c->d_cmass, 0, sizeof(double) * count, c->stream));
  return run_cell_mass(c);
}

extern "C" int hofv_set_inertia(hofv_ctx* c, double rho, double dt, int one_point) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return hofv::fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (!(rho >= 0.0) || (rho > 0.0 && !(dt > 0.0)) || !std::isfinite(rho) || !std::isfinite(dt))
    return hofv::fail(c, HOFV_EINVAL, "bad density or time step");
  invalidate_graphs(c);
  const int64_t n = c->nc * c->dim;
  if (rho == 0.0) {
    c->inertia = false;
    c->hist_set = false;
  } else {
    if (!c->d_mscale) {
      TRY(dev_alloc(c, &c->d_mscale, c->nc));
      TRY(dev_alloc(c, &c->d_inert, n));
      TRY(dev_alloc(c, &c->d_hist, n));
    }
    if (!one_point) TRY(ensure_cmass(c));
    const double c2 = 9.0 / (4.0 * dt * dt);
    c->rho = rho;
    c->dt = dt;
    c->one_point = one_point ? 1 : 0;
    c->inertia = true;
    c->hist_set = false;
    launch_combine4(c->nc, -rho * c2, c->d_vol, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr,
                    c->d_mscale, c->stream);
    HOFV_CUDA(c, cudaMemsetAsync(c->d_hist, 0, sizeof(double) * n, c->stream));
  }
  TRY(refresh_source(c));
  TRY(run_aj_rows(c));
  mg_drop(c);
  return HOFV_OK;
}

static const double* avg_weights(hofv_ctx* c) { return c->one_point ? nullptr : c->d_cmass; }

extern "C" int hofv_set_history(hofv_ctx* c, const double* u_t, const double* u_tm1,
                                const double* v_t, const double* v_tm1) {
  if (!c) return HOFV_EINVAL;
  if (!c->inertia) return hofv::fail(c, HOFV_ESTATE, "hofv_set_inertia must come first");
  if (!u_t) return hofv::fail(c, HOFV_EINVAL, "null displacement");
  if (!u_tm1) u_tm1 = u_t;
  DevMesh m = dev_mesh(c);
  m.cmass = avg_weights(c);
  const int64_t n = c->nc * c->dim;
  const double dt = c->dt;
  launch_cell_average(m, u_t, c->d_inert, c->stream);
  launch_cell_average(m, u_tm1, c->d_hist, c->stream);
  // h / c2 with h = (-12 ubar^t + 3 ubar^{t-1}) / (4 dt^2) + (-4 v^t + v^{t-1}) / (2 dt)
  launch_combine4(n, -4.0 / 3.0, c->d_inert, 1.0 / 3.0, c->d_hist, -8.0 * dt / 9.0, v_t,
                  2.0 * dt / 9.0, v_tm1, c->d_hist, c->stream);
  launch_scale_rows(c->dim, c->nc, c->d_mscale, c->d_hist, c->stream);
  c->hist_set = true;
  TRY(refresh_source(c));
  return HOFV_OK;
}

extern "C" int hofv_bdf2_velocity(hofv_ctx* c, const double* u_tp1, const double* u_t,
                                  const double* u_tm1, double* v_out) {
  if (!c) return HOFV_EINVAL;
  if (!c->inertia) return hofv::fail(c, HOFV_ESTATE, "hofv_set_inertia must come first");
  if (!u_tp1 || !u_t || !v_out) return hofv::fail(c, HOFV_EINVAL, "null vector");
  if (!u_tm1) u_tm1 = u_t;
  DevMesh m = dev_mesh(c);
  m.cmass = avg_weights(c);
  const int64_t n = c->nc * c->dim;
  const double k = 1.0 / (2.0 * c->dt);
  launch_cell_average(m, u_tp1, v_out, c->stream);
  launch_cell_average(m, u_t, c->d_inert, c->stream);
  launch_combine4(n, 3.0 * k, v_out, -4.0 * k, c->d_inert, 0.0, nullptr, 0.0, nullptr, v_out,
                  c->stream);
  launch_cell_average(m, u_tm1, c->d_inert, c->stream);
  launch_combine4(n, 1.0, v_out, k, c->d_inert, 0.0, nullptr, 0.0, nullptr, v_out, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}

extern "C" int hofv_cell_average(hofv_ctx* c, const double* u, double* ubar) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return hofv::fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (!u || !ubar) return hofv::fail(c, HOFV_EINVAL, "null vector");
  TRY(ensure_cmass(c));
  DevMesh m = dev_mesh(c);
  m.cmass = c->d_cmass;
  launch_cell_average(m, u, ubar, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}

extern "C" int hofv_nej_apply(hofv_ctx* c, const double* x, double* y) {
  if (!c) return HOFV_EINVAL;
  if (!c->built || !c->have_mat) return hofv::fail(c, HOFV_ESTATE, "stencils and material must be set first");
  if (!x || !y) return hofv::fail(c, HOFV_EINVAL, "null vector");
  TRY(hofv::nej_apply(c, x, y));
  return HOFV_OK;
}

// ---------------------------------------------------------------------
// caller-supplied stencils, solver preparation, load path
// ---------------------------------------------------------------------
namespace hofv {

// tiled stencil arrays [tiles][S][kTile] <-> row-major [count][S]
static void tile_rows(const int32_t* rows, int64_t count, int S, std::vector<int32_t>& tiled) {
  const int64_t tiles = (count + kTile - 1) / kTile;
  tiled.assign((size_t)std::max<int64_t>(tiles, 1) * S * kTile, 0);
  for (int64_t i = 0; i < count; ++i)
    for (int n = 0; n < S; ++n)
      tiled[((i / kTile) * S + n) * kTile + i % kTile] = rows[i * S + n];
}

// recompute everything derived from the stencils: reconstruction
// coefficients and stabilisation weights, their double-float form, the cell
// averages of the inertia term, the contracted matrices; the near-exact
// Jacobian (built from them) is rebuilt on its next use
static int rebuild_from_stencils(hofv_ctx* c) {
  invalidate_graphs(c);
  jv_invalidate(c);
  TRY(run_lsq(c));
  if (c->prec == HOFV_PREC_DF64) TRY(coef_format(c, 1));
  if (c->d_cmass) TRY(run_cell_mass(c));
  c->tco_valid = false;
  nej_release(c);
  TRY(build_contraction(c));
  return refresh_source(c);
}

}  // namespace hofv

extern "C" int hofv_set_stencils(hofv_ctx* c, const int32_t* face_stencils,
                                 const int32_t* cell_stencils) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (c->nfy > 0)
    return fail(c, HOFV_ENOTSUP, "stencils cannot be replaced on meshes with symmetry faces");
  const int S = c->S;
  auto check = [&](const int32_t* rows, int64_t count) -> bool {
    for (int64_t i = 0; i < count * S; ++i)
      if (rows[i] < 0 || rows[i] >= c->nc) return false;
    return true;
  };
  if ((face_stencils && !check(face_stencils, c->nfid)) ||
      (cell_stencils && !check(cell_stencils, c->nc)))
    return fail(c, HOFV_EINVAL, "stencil cell id out of range");
  HOFV_CUDA(c, cudaSetDevice(c->device));
  const size_t nfst = (size_t)std::max<int64_t>(c->nftile, 1) * S * kTile;
  const size_t ncst = (size_t)c->nctile * S * kTile;
  std::vector<int32_t> old_f(nfst), old_c(ncst), t;
  HOFV_CUDA(c, cudaMemcpy(old_f.data(), c->d_fst, sizeof(int32_t) * nfst, cudaMemcpyDeviceToHost));
  HOFV_CUDA(c, cudaMemcpy(old_c.data(), c->d_cst, sizeof(int32_t) * ncst, cudaMemcpyDeviceToHost));
  if (face_stencils) {
    tile_rows(face_stencils, c->nfid, S, t);
    HOFV_CUDA(c, cudaMemcpy(c->d_fst, t.data(), sizeof(int32_t) * nfst, cudaMemcpyHostToDevice));
  }
  if (cell_stencils) {
    tile_rows(cell_stencils, c->nc, S, t);
    HOFV_CUDA(c, cudaMemcpy(c->d_cst, t.data(), sizeof(int32_t) * ncst, cudaMemcpyHostToDevice));
  }
  const int rc = rebuild_from_stencils(c);
  if (rc < 0) {  // keep the context usable: back to the previous stencils
    const std::string msg = c->err;
    cudaMemcpy(c->d_fst, old_f.data(), sizeof(int32_t) * nfst, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_cst, old_c.data(), sizeof(int32_t) * ncst, cudaMemcpyHostToDevice);
    rebuild_from_stencils(c);
    return fail(c, rc, msg + " (previous stencils restored)");
  }
  return HOFV_OK;
}

extern "C" int hofv_prepare_solver(hofv_ctx* c, const hofv_solve_opts* opts) {
  TRY(check_eval(c));
  hofv_solve_opts o;
  hofv_default_opts(&o);
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 100 || o.precond < HOFV_PC_NONE || o.precond > HOFV_PC_NEJ)
    return fail(c, HOFV_EINVAL, "bad solver options");
  HOFV_CUDA(c, cudaSetDevice(c->device));
  TRY(ensure_krylov(c, o.restart));
  if (o.precond == HOFV_PC_AJMG || o.precond == HOFV_PC_NEJ) TRY(mg_ensure(c));
  if (o.precond == HOFV_PC_NEJ) {
    if (c->mat.law != HOFV_LAW_LINEAR)
      return fail(c, HOFV_ENOTSUP, "the near-exact Jacobian is defined for the linear law");
    TRY(ensure_tco(c));
    TRY(nej_prepare(c, o.inner_iters));
  }
  TRY(ensure_jv_storage(c));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOFV_OK;
}

extern "C" int hofv_solve_load_path(hofv_ctx* c, double* u, const double* u_bq1,
                                    const double* u_bf1, const double* t_bq1, const double* body1,
                                    const double* du_dlambda, int32_t n_steps,
                                    int32_t max_halvings, const hofv_solve_opts* opts,
                                    hofv_stats* stats, int32_t* steps_done) {
  TRY(check_eval(c));
  if (!u) return fail(c, HOFV_EINVAL, "null vector");
  if (n_steps < 1 || n_steps > 1000000 || max_halvings < 0 || max_halvings > 30)
    return fail(c, HOFV_EINVAL, "bad step count or halving limit");
  const auto t0 = std::chrono::steady_clock::now();
  const int d = c->dim;
  const int64_t n = c->nc * d;
  // data at load factors 0 (the context's current data) and 1; state before
  // the increment; previous converged state (secant predictor)
  const int64_t nbq = c->nfd * c->Q * d, nbf = c->nfd * d, ntq = c->nft * c->Q * d, nbd = n;
  const int64_t ndat = nbq + nbf + ntq + nbd;
  double* buf = nullptr;
  HOFV_CUDA(c, cudaMalloc(&buf, sizeof(double) * (2 * ndat + 3 * n + 1)));
  double* d0 = buf;
  double* d1 = buf + ndat;
  double* u_last = d1 + ndat;   // last converged state
  double* u_prev = u_last + n;  // the one before (secant predictor)
  double* u_try = u_prev + n;
  struct Part { double* ctxp; const double* one; int64_t off, cnt; };
  const Part parts[4] = {{c->d_ubq, u_bq1, 0, nbq},
                         {c->d_ubf, u_bf1, nbq, nbf},
                         {c->d_tbq, t_bq1, nbq + nbf, ntq},
                         {c->d_body, body1, nbq + nbf + ntq, nbd}};
  int rc = 0;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == 0) rc = cuda_fail(c, e, what);
  };
  for (const Part& p : parts) {
    if (p.cnt <= 0) continue;
    cu(cudaMemcpyAsync(d0 + p.off, p.ctxp, sizeof(double) * p.cnt, cudaMemcpyDeviceToDevice,
                       c->stream), "load path: copy of the initial data");
    cu(cudaMemcpyAsync(d1 + p.off, p.one ? p.one : p.ctxp, sizeof(double) * p.cnt,
                       cudaMemcpyDeviceToDevice, c->stream), "load path: copy of the final data");
  }
  cu(cudaMemcpyAsync(u_last, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream),
     "load path: state copy");
  auto set_data = [&](double lam) -> int {  // data(lam) = (1 - lam) d0 + lam d1
    for (const Part& p : parts)
      if (p.cnt > 0)
        launch_combine4(p.cnt, 1.0 - lam, d0 + p.off, lam, d1 + p.off, 0.0, nullptr, 0.0, nullptr,
                        p.ctxp, c->stream);
    HOFV_CUDA(c, cudaGetLastError());
    jv_invalidate(c);
    return refresh_source(c);
  };
  hofv_stats tot;
  memset(&tot, 0, sizeof(tot));
  const double nominal = 1.0 / n_steps;
  double lam = 0.0, dlam = nominal, dlam_prev = 0.0;
  int halvings = 0, accepted = 0;
  int status = HOFV_OK;
  while (rc == 0 && lam < 1.0 - 1e-15) {
    const double step = std::min(dlam, 1.0 - lam);
    rc = set_data(lam + step);
    if (rc) break;
    // predictor: the caller's direction per unit load factor, else the
    // secant through the last two converged states, else the last state
    if (du_dlambda)
      launch_combine4(n, 1.0, u_last, step, du_dlambda, 0.0, nullptr, 0.0, nullptr, u_try,
                      c->stream);
    else if (accepted > 0 && dlam_prev > 0.0)
      launch_combine4(n, 1.0 + step / dlam_prev, u_last, -step / dlam_prev, u_prev, 0.0, nullptr,
                      0.0, nullptr, u_try, c->stream);
    else
      cu(cudaMemcpyAsync(u_try, u_last, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream),
         "load path: predictor");
    if (rc) break;
    hofv_stats st;
    memset(&st, 0, sizeof(st));
    const int s = hofv_newton_solve(c, u_try, opts, &st);
    tot.newton_iters += st.newton_iters;
    tot.krylov_iters += st.krylov_iters;
    tot.residual_evals += st.residual_evals;
    tot.precond_applies += st.precond_applies;
    tot.gnn_fallbacks += st.gnn_fallbacks;
    if (accepted == 0 && halvings == 0) tot.r0 = st.r0;
    tot.r_final = st.r_final;
    if (s == HOFV_OK) {
      cu(cudaMemcpyAsync(u_prev, u_last, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream),
         "load path: state copy");
      cu(cudaMemcpyAsync(u_last, u_try, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream),
         "load path: state copy");
      lam += step;
      dlam_prev = step;
      ++accepted;
      halvings = 0;
      dlam = std::min(nominal, 2.0 * dlam);  // grow back after a halved increment
    } else if (s == HOFV_WNOTCONV || s == HOFV_ENAN) {
      if (halvings >= max_halvings) {
        status = HOFV_WNOTCONV;
        fail(c, HOFV_WNOTCONV, "load path: an increment failed after the allowed halvings");
        break;
      }
      ++halvings;
      dlam = 0.5 * step;
    } else {
      rc = s;  // a hard error of the solver
    }
  }
  if (rc == 0 && status != HOFV_OK) rc = set_data(lam);  // the data of the state returned
  cu(cudaMemcpyAsync(u, u_last, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream),
     "load path: result copy");
  cu(cudaStreamSynchronize(c->stream), "load path: synchronisation");
  cudaFree(buf);
  if (steps_done) *steps_done = accepted;
  tot.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  tot.status = rc ? rc : status;
  if (stats) *stats = tot;
  return rc ? rc : status;
}
