// hofv_internal.cuh -- context layout and kernel launchers shared by the
// translation units of libhofv (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hofv.h"

namespace hofv {

constexpr int kTile = 32;        // faces / cells per tile of the tiled layouts
constexpr int kMaxS = 128;       // largest supported stencil (+ ghost)
constexpr int kMaxNt = 20;       // Taylor terms of a cubic in 3-D
constexpr int kMaxQ = 16;        // Gauss points per face (4 x 4)
constexpr int kMaxQC = 64;       // Gauss points per cell (4^3)
constexpr int kPolyMaxSides = 8; // face slots of a polygon cell
constexpr int kPolyhedronMaxFaces = 16;  // face slots of a polyhedral cell
constexpr int kPolyFaceMaxCorners = 8;   // corners of a polyhedral face
constexpr int kPackThreads = 384;        // threads (rows with area) of a packed face group
constexpr int kPackMaxFaces = 8;         // faces of a packed face group

// J^{-1/3} for the neo-Hookean law, with one FP64 correction of a
// single-precision estimate instead of the full double-precision routine:
// with r = rcbrtf(J) and h = 1 - J r^3 (|h| ~ 1e-7), J^{-1/3} = r (1 - h)^{-1/3}
// = r (1 + h/3 + 2 h^2/9 + O(h^3)) (binomial series; one step of
// Householder's third-order iteration for r^-3 = J), exact to rounding since
// h^3 ~ 1e-21.  Outside 1e-30 < J < 1e30 (beyond the float range of the
// estimate) and for J <= 0 it defers to rcbrt (NaN for J <= 0).
#if defined(__CUDACC__)
__device__ __forceinline__ double inv_cbrt(double J) {
  if (!(J > 1e-30 && J < 1e30)) return J > 0.0 ? rcbrt(J) : __longlong_as_double(0x7ff8000000000000LL);
  const double r = (double)rcbrtf((float)J);
  const double h = fma(-J, r * r * r, 1.0);
  return fma(r, h * fma(h, 2.0 / 9.0, 1.0 / 3.0), r);
}
#endif

// Device-side description of the discretisation used by the residual
// kernels.  All pointers are device addresses owned by the context.
struct DevMesh {
  int dim, nlf, S, Q, R;          // R = Q * dim rows per face
  int64_t nc, nf, nfi, nfd, nft;
  int64_t nfid;                   // internal + displacement faces
  int64_t nftile;                 // face tiles of kTile (internal + disp)
  int64_t nctile;                 // cell tiles of kTile
  // faces (internal + displacement), index f in [0, nfid)
  const int32_t* fst;     // [nftile][S][kTile]                stencil cell ids
  const double* fco;      // [nftile][S][kTile][R]             gradient coefficients
  const double* gco;      // [nfd][R]                          ghost coefficients
  const double* aq;       // [nf][Q][3]                        vector areas
  const int32_t* fstar;   // [nfid][2]  u* slots (cell*nlf+lf) owner, neighbour (-1 disp)
  const double* fstab;    // [nfid]     Gamma_f / |d . n|
  const int32_t* fql;     // [nftile * kTile] points of each face that carry area (polyhedral
                          // fans with fewer corners than slots), or nullptr: all Q
  const int32_t* pgrp;    // [npg][2] polyhedral faces with 8 fan slots packed by their
                          // points with area: first face and face count of each group
                          // (consecutive faces of one tile), or nullptr
  int64_t npg;            // groups in pgrp
  // cells
  const int32_t* cst;     // [nctile][S][kTile]
  const double* cex;      // [nctile][S][kTile][nlf]
  const int32_t* cface;   // [nc][nlf]  +(f+1) owner, -(f+1) neighbour, 0 traction
  const double* tco;      // [nftile][S][kTile][dim][dim] contracted linear-elastic
                          // face matrices, or nullptr (then the per-point form is used)
  // symmetry faces [nfi + nfd, nfid): their stencils end in mirror images of
  // cells ("ghosts", ids nc + g); the state is then read from an extended
  // copy [dim][wst] holding the reflected values R u_src after the cells
  int64_t nfy, ng, wst;   // symmetry faces, ghosts, stride of the state read
  const int32_t* gsrc;    // [ng] source cell of each ghost
  const int32_t* gface;   // [ng] symmetry face whose plane mirrors it
  const double* nrm;      // [nf][3] unit face normals
  double* wext;           // [dim][nc + ng] extended state (scratch), or nullptr
  double* ubfw;           // [nfd + nfy][dim] face-centre values; the symmetry
                          // slots are rewritten by each residual call
  // inertia (BDF2): R_P -= rho Omega_P c2 ubar_P(u), ubar_P = u_P + sum_N cmass_N u_N
  const double* mscale;   // [nc] -rho Omega_P c2, or nullptr (no inertia term)
  const double* cmass;    // [nctile][S][kTile] cell-average weights, or nullptr (ubar = u_P)
  double* inert;          // [dim][nc] scratch: the inertia term of the current call
  // gradient contraction precision (HOFV_PREC_*).  With HOFV_PREC_DF64 every
  // 8-byte slot of fco and cex holds a double-float pair (float hi, float lo),
  // and the state is split into such pairs before the contraction
  int prec;
  float4* su;             // [wst][dim] split state (scratch): (hi, mid, lo, 0) per component
  float4* sv;             // [wst][dim] split Jv direction (scratch)
  double* ustar_v;        // [nc][nlf][dim] extrapolated values of the Jv direction (scratch)
  double* vext;           // [dim][wst] extended Jv direction (symmetry faces; scratch)
  // linearisation of the neo-Hookean law at u for the double-float Jv:
  // gradient rows and Gauss-point tractions of every face at u
  double* gcache;         // [nftile * kTile][R][dim]
  double* tcache;         // [nftile * kTile][Q][dim]
  unsigned int* kerr;     // set to 1 by a face kernel whose bounded wait ran out
  const double* fcsum;    // [nftile * kTile][R] sums over the stencil of the stored
                          // (double-float) gradient coefficients of each row
};

// float4 slots per cell of a split state: one per component, the value
// split exactly into three floats (hi, mid, lo, 0), hi + mid + lo = value
__host__ __device__ constexpr int split4(int dim) { return dim; }

struct Material {
  int law;
  double mu, lam, kappa, kbar, alpha;
};

}  // namespace hofv

struct hofv_ctx {
  int device = 0;
  int sm_count = 1;                 // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  std::string err;
  // ---- mesh (host) ----
  bool have_mesh = false, have_scheme = false, built = false, have_mat = false;
  int dim = 0, nv = 0, nlf = 0, nfv = 0;
  bool simplex = false;            // triangles / tetrahedra instead of quads / hexes
  bool poly = false;               // 2-D polygons: nlf = nv = kPolyMaxSides slots per cell
  std::vector<int32_t> cnv;        // polygons: [nc] corners (= sides) of each cell
  bool polyh = false;              // 3-D polyhedra given face by face: nlf = kPolyhedronMaxFaces
                                   // slots, nfv = 4 or 8 corner slots a face (-1 past its last)
  int maxtets = 0;                 // polyhedra: most fan tetrahedra of one cell
  int64_t nn = 0, nc = 0, nb = 0;
  std::vector<double> x;            // [nn][3]
  std::vector<int64_t> cn;          // [nc][nv]
  int64_t nf = 0, nfi = 0, nfd = 0, nft = 0, nfid = 0;
  int64_t nfy = 0;                  // symmetry faces, after the displacement faces
  std::vector<int64_t> fown, fnei;
  std::vector<int32_t> flf, ftag;
  std::vector<int32_t> fnodes;      // [nf][nfv]
  std::vector<int64_t> cf;          // [nc][nlf]
  // ---- scheme ----
  int p = 0, nplus = 0, q1 = 0, S = 0, Nt = 0, Q = 0, QC = 0;
  double kw = 6.0, alpha = 0.1;
  int href_exp = 0;
  double gl_x[4] = {0}, gl_w[4] = {0};
  // ---- material ----
  hofv::Material mat{};
  // ---- device geometry ----
  double* d_x = nullptr;            // [nn][3]
  int32_t* d_fnodes = nullptr;      // [nf][nfv]
  int32_t* d_cnodes = nullptr;      // [nc][nv]
  double *d_xc = nullptr, *d_vol = nullptr;        // [nc][3], [nc]
  double *d_xq = nullptr, *d_aq = nullptr;         // [nf][Q][3]
  double *d_xf = nullptr, *d_nrm = nullptr, *d_gam = nullptr;  // [nf][3],[nf][3],[nf]
  double *d_cqx = nullptr, *d_cqw = nullptr;       // [nc][QC][3], [nc][QC]
  int64_t* d_cf = nullptr;          // [nc][nlf] face of each local face
  int32_t* d_ftag = nullptr;        // [nf]
  int32_t* d_fown = nullptr;        // [nf]
  int32_t* d_fnei = nullptr;        // [nf]
  // ---- stencils / coefficients ----
  int64_t nftile = 0, nctile = 0;
  int32_t* d_fst = nullptr;
  double* d_fco = nullptr;
  double* d_gco = nullptr;
  int32_t* d_cst = nullptr;
  double* d_cex = nullptr;
  int32_t* d_fstar = nullptr;
  double* d_fstab = nullptr;
  int32_t* d_fql = nullptr;
  int32_t* d_pgrp = nullptr;        // packed face groups (polyhedra, 8 fan slots)
  int64_t npg = 0;
  int32_t* d_cface = nullptr;
  double max_cond = 0.0;
  double setup_seconds = 0.0;
  // ---- boundary data ----
  double* d_ubq = nullptr;          // [nfd][Q][dim]
  double* d_ubf = nullptr;          // [nfd][dim]
  double* d_tbq = nullptr;          // [nft][Q][dim]
  double* d_body = nullptr;         // [dim][nc]
  double* d_src = nullptr;          // [dim][nc]  body + traction-face fluxes
  // contracted linear-elastic form (per face and stencil cell d x d matrices)
  bool contract = false;            // requested by the caller
  bool tco_valid = false;           // d_tco holds the matrices for the current mu, lambda
  double* d_tco = nullptr;
  double* d_gflux = nullptr;        // [nfd][dim] ghost-node flux (constant per load step)
  bool src_dirty = true;
  // ---- gradient contraction precision (HOFV_PREC_*) ----
  int prec = HOFV_PREC_FP64;
  float4* d_su = nullptr;           // [nc + ng][split4] split state
  float4* d_sv = nullptr;           // [nc + ng][split4] split Jv direction
  double* d_ustar_v = nullptr;      // [nc][nlf][dim]
  double* d_fcsum = nullptr;        // [nftile * kTile][R] row sums of the stored coefficients
  double* d_vext = nullptr;         // [dim][nc + ng]
  // neo-Hookean double-float Jv: face gradients and tractions at u, valid
  // for the state / residual pair (jv_u, jv_R) while jv_gen == jv_cur
  double* d_gcache = nullptr;
  double* d_tcache = nullptr;
  const double* jv_u = nullptr;
  const double* jv_R = nullptr;
  uint64_t jv_gen = 0, jv_cur = 1;
  // ---- scratch for the residual ----
  double* d_ustar = nullptr;        // [nc][nlf][dim]
  double* d_flux = nullptr;         // [nfid][dim]
  double* d_w = nullptr;            // [dim][nc]
  double* d_red = nullptr;          // reduction partials
  unsigned int* d_count = nullptr;  // last-block counters
  double* d_scal = nullptr;         // device scalars (eps, norms, CG alpha/beta)
  int red_blocks = 0;
  // ---- approximate Jacobian (Kbar = 1) ----
  double* d_aj_diag = nullptr;      // [nc]
  int32_t* d_aj_col = nullptr;      // [nc][nlf]  neighbour id or -1
  double* d_aj_off = nullptr;       // [nc][nlf]
  float* d_aj_diag32 = nullptr;
  float* d_aj_off32 = nullptr;
  unsigned int* d_bar = nullptr;    // grid barrier of the persistent CG: count, generation, error
  double* d_aj_invd = nullptr;      // 1 / (-diag), FP64 and FP32
  float* d_aj_invd32 = nullptr;
  // CG work vectors (sized dim*nc each)
  double *d_cg64 = nullptr;         // 5 vectors FP64
  float *d_cg32 = nullptr;          // 5 vectors FP32
  // ---- Krylov ----
  int kry_m = 0;
  double* d_V = nullptr;            // [(m+1)][n]
  double* d_Z = nullptr;            // [m][n]
  double* d_kvec = nullptr;         // work vectors
  double* d_h = nullptr;            // [m+2] projections
  // ---- learned preconditioner ----
  void* gnn = nullptr;
  // ---- multigrid hierarchy of the approximate Jacobian ----
  void* mg = nullptr;
  // ---- symmetry faces: mirrored stencil nodes ----
  int64_t ng = 0;                   // ghosts = nfy * floor(S / 2)
  double* d_xce = nullptr;          // [nc + ng][3] centroids and ghost positions
  int32_t* d_gsrc = nullptr;        // [ng]
  int32_t* d_gface = nullptr;       // [ng]
  double* d_wext = nullptr;         // [dim][nc + ng]
  std::vector<int32_t> gsrc_host;
  // ---- inertia term, BDF2 in time (App. time integration) ----
  bool inertia = false;
  double rho = 0.0, dt = 0.0;
  int one_point = 0;
  double* d_cmass = nullptr;        // cell-average weights over the cell stencil
  double* d_mscale = nullptr;       // [nc] -rho Omega c2
  double* d_inert = nullptr;        // [dim][nc] scratch
  double* d_hist = nullptr;         // [dim][nc] -rho Omega (history part of the acceleration)
  bool hist_set = false;
  // ---- near-exact Jacobian preconditioner (nej.cu) ----
  void* nej = nullptr;
  // ---- CUDA graphs of the device part of an Arnoldi step ----
  uint64_t gen = 1;                 // bumped by every call that changes kernel arguments
  void* graphs = nullptr;           // cache of instantiated graphs (api.cu)
  cudaStream_t cap = nullptr;       // private stream used only for capturing
  double aj_rate = -1.0;            // mean per-iteration residual reduction of the last AJ cycle
  int64_t device_bytes = 0;
  std::vector<void*> allocs;
};

namespace hofv {

// error helpers
int fail(hofv_ctx* c, int code, const std::string& msg);
int cuda_fail(hofv_ctx* c, cudaError_t e, const char* what);
#define HOFV_CUDA(ctx, call)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return hofv::cuda_fail(ctx, e_, #call); \
  } while (0)

template <typename T>
int dev_alloc(hofv_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  size_t bytes = count * sizeof(T) + 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, HOFV_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  c->device_bytes += (int64_t)bytes;
  *p = static_cast<T*>(q);
  return 0;
}
void dev_free(hofv_ctx* c, void* p);

DevMesh dev_mesh(const hofv_ctx* c);

// ---- set-up kernels (setup.cu) ----
int run_geometry(hofv_ctx* c);
int flux_wide_prepare();
int run_stencils(hofv_ctx* c, const std::vector<int64_t>& bucket_start,
                 const std::vector<int32_t>& bucket_items, const int nb[3], const double lo[3],
                 double bs);
int run_lsq(hofv_ctx* c);
// ghost (mirrored) stencil nodes of the symmetry faces: sources, planes, positions
int run_ghosts(hofv_ctx* c);
int run_face_aux(hofv_ctx* c);
// cell-average weights of the cell fit over the cell's Gauss points
int run_cell_mass(hofv_ctx* c);
// rebuild the approximate Jacobian rows, with the inertia diagonal if enabled
int run_aj_rows(hofv_ctx* c);

// ---- residual kernels (residual.cu) ----
// R = residual(w) where w = u (+ eps * v when v != nullptr, eps read from
// *d_eps on the device); when R0 != nullptr the output is (R(w) - R0) / eps.
void launch_residual(const DevMesh& m, const Material& mat, const double* u, const double* v,
                     const double* d_eps, const double* R0, double* out, double* ustar,
                     double* flux, const double* ubq, const double* ubf, const double* src,
                     cudaStream_t st, cudaEvent_t* ev = nullptr);
// Jv with HOFV_PREC_DF64 (eps read from *d_eps on the device).  Linear law:
// the residual is affine, so (R(u + eps v) - R(u)) / eps is evaluated exactly
// as its homogeneous part at v (no boundary data, no sources).  Neo-Hookean:
// the face kernels contract v alone and difference the tractions of
// grad u + eps grad v and grad u in FP64, grad u and its tractions read from
// the linearisation cache (launch_jv_cache_fill), so the rounding of the
// double-float contraction of u cancels exactly
void launch_jv_df(const DevMesh& m, const Material& mat, const double* v, const double* d_eps,
                  double* out, double* flux, cudaStream_t st, cudaEvent_t* ev = nullptr);
// the neo-Hookean linearisation at u for launch_jv_df: face gradient rows
// (with the ghost-node data) and Gauss-point tractions into m.gcache,
// m.tcache
void launch_jv_cache_fill(const DevMesh& m, const Material& mat, const double* u,
                          const double* ubq, cudaStream_t st);
// rewrites the n 8-byte slots of a coefficient array in place: to_df != 0
// turns each double into the double-float pair (float hi, float lo) with
// hi + lo its value rounded to 48 significant bits; to_df == 0 turns the pairs
// back into doubles (exactly)
void launch_coef_format(double* a, int64_t n, int to_df, cudaStream_t st);
// fcsum[f][r] = sum over the stencil slots of the stored coefficient of face
// f, row r (double-float pairs summed in FP64, in slot order)
void launch_row_sums(const DevMesh& m, double* fcsum, cudaStream_t st);
// raises the dynamic shared-memory limit of the double-float face kernels
// (once per process, at set-up); 0 or a cudaError_t
int setup_df_kernels();
void launch_source(const hofv_ctx* c, cudaStream_t st);
void launch_build_tco(const DevMesh& m, double mu, double lam, double* tco, cudaStream_t st);
void launch_ghost_flux(const DevMesh& m, double mu, double lam, const double* ubq, double* gflux,
                       cudaStream_t st);
void launch_tflux(const DevMesh& m, const double* tco, double alpha_kbar, const double* w,
                  const double* ustar, const double* ubf, double* flux, cudaStream_t st);
// recompute the constant cell source (body, traction faces and, for the
// contracted linear form, the ghost-node fluxes)
int refresh_source(hofv_ctx* c);
// ubar[j][c] = u_P + sum_N cmass_N u_N (u_P alone when m.cmass is null)
void launch_cell_average(const DevMesh& m, const double* u, double* ubar, cudaStream_t st);
// out = a * x + b * y + g * z + e * w (component vectors [dim][nc]; null terms skipped)
void launch_combine4(int64_t n, double a, const double* x, double b, const double* y, double g,
                     const double* z, double e, const double* w, double* out, cudaStream_t st);
// out[j][c] *= s[c]
void launch_scale_rows(int dim, int64_t nc, const double* s, double* out, cudaStream_t st);
// out[cell] = sum over the cell's internal/displacement faces of |flux_f|
void launch_flux_scale(const DevMesh& m, const double* flux, double* out, cudaStream_t st);

// ---- vector kernels (krylov.cu) ----
// out[i] = sum over blocks of partial dot products, deterministic order
// out[k] = X_k . y (mode 0) for k < nvec with X_k = X + k * ldx; mode 1: sqrt
void launch_dots(const double* X, int64_t ldx, const double* y, int nvec, int64_t n, double* red,
                 unsigned int* count, double* out, int blocks, cudaStream_t st, int mode);
void launch_norm2(const double* x, int64_t n, double* red, unsigned int* count, double* out,
                  int blocks, cudaStream_t st);
void launch_jv_eps(const double* u_norm, const double* v_norm, double* eps, cudaStream_t st);
// y = x + sign * alpha[0] * v
void launch_waxpy_dev(double* y, const double* x, const double* v, const double* alpha,
                      double sign, int64_t n, cudaStream_t st);
void launch_scale_copy(double* y, const double* x, const double* s, int invert, int64_t n,
                       cudaStream_t st);
void launch_multi_axpy(double* w, const double* V, const double* coef, int k, int64_t n,
                       int64_t ld, cudaStream_t st);
void launch_combine(double* x, const double* Z, const double* y, int k, int64_t n, int64_t ld,
                    cudaStream_t st);
void launch_axpby(double* y, double a, const double* x, double b, int64_t n, cudaStream_t st);
int aj_precondition(hofv_ctx* c, int kind, int iters, const double* v, double* z);
// error of a timed-out persistent-CG grid barrier since the last check
// (reads the flag: call after a stream synchronisation), then clears it
int check_pc_barrier(hofv_ctx* c);
// bounded-wait self-test of the grid barrier (see hofv_selftest_barrier)
int barrier_selftest(hofv_ctx* c, int* timed_out);

// ---- multigrid inner solve of the approximate Jacobian (multigrid.cu) ----
int mg_precondition(hofv_ctx* c, int iters, const double* v, double* z);
// builds the hierarchy if it does not exist yet (synchronises)
int mg_ensure(hofv_ctx* c);
int mg_info(hofv_ctx* c, int32_t* levels, int64_t* sizes, int max_sizes, int64_t* nnz,
            double* setup_s);
void mg_release(hofv_ctx* c);
// frees the hierarchy's device memory too (the approximate Jacobian changed)
void mg_drop(hofv_ctx* c);

// ---- near-exact Jacobian (nej.cu) ----
// contracted linear-elastic matrices for the current material (api.cu)
int ensure_tco(hofv_ctx* c);
int nej_ensure(hofv_ctx* c);
int nej_apply(hofv_ctx* c, const double* x, double* y);
int nej_precondition(hofv_ctx* c, int iters, const double* v, double* z);
// the structure, values and inner-solver storage for `iters` inner iterations
int nej_prepare(hofv_ctx* c, int iters);
void nej_release(hofv_ctx* c);

// ---- learned preconditioner (gnn.cu) ----
int gnn_apply(hofv_ctx* c, const double* v, const double* z_aj, double* z);
void gnn_release(hofv_ctx* c);

}  // namespace hofv
