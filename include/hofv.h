/*
 * hofv.h -- C ABI of the GB300 (sm_103a) high-order finite-volume JFNK
 * library for solid mechanics.
 *
 * The method is the cell-centred finite-volume discretisation of
 * Batistic, Castrillo & Cardiff, "High-order finite volume solid mechanics
 * with Jacobian-free Newton-Krylov" (arXiv 2601.18417): point values at
 * cell centroids, least-squares Taylor reconstruction of the displacement
 * gradient at face Gauss points, Gaussian face quadrature of the traction,
 * alpha stabilisation, a Jacobian-free Newton-Krylov solver and the
 * compact-stencil approximate Jacobian as preconditioner.
 *
 * Conventions (all entry points)
 *   - Return value: 0 OK; > 0 warning (HOFV_WNOTCONV); < 0 error.  Errors
 *     never abort the process; hofv_last_error() gives the message.
 *   - Vectors over cells are FP64, component-major: x[c * n_cells + cell].
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device, owned by the caller; the library never frees them.  The
 *     library owns mesh, stencil, coefficient, preconditioner and Krylov
 *     storage, allocated by the set-up calls; the evaluation calls
 *     (residual, jvp, precondition) allocate nothing, except that the first
 *     use of a preconditioner builds its data (multigrid hierarchy,
 *     near-exact Jacobian) and the first Arnoldi step of a kind captures
 *     its CUDA graph; hofv_prepare_solver does all of that up front.
 *   - Asynchrony: evaluation calls enqueue work on the context stream and
 *     return; set-up calls and hofv_newton_solve synchronise that stream.
 *   - Faces: internal faces first, ordered by (owner, owner local face) with
 *     owner < neighbour; then displacement, symmetry and traction faces, each
 *     in the order of the boundary-face list given to hofv_set_mesh.  Local
 *     faces of a quad / hex are x-, x+, y-, y+ (, z-, z+) of its reference
 *     element; local face k of a triangle runs from node k to node k+1 mod 3,
 *     local face k of a tetrahedron is the face opposite node 3 - k, and
 *     local face k of a polygon runs from its corner k to corner k+1.
 *   - Gradients: grad[i][j] = d u_j / d x_i, the paper's sum of c (x) u
 *     (Sec. 3.5.4, eq. faceQuadGrad).
 */
#ifndef HOFV_H
#define HOFV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HOFV_OK 0
#define HOFV_WNOTCONV 1      /* solver stopped before reaching its tolerance */
#define HOFV_EINVAL (-1)     /* bad argument */
#define HOFV_ENOMEM (-2)     /* device or host allocation failed */
#define HOFV_ECUDA (-3)      /* CUDA runtime error */
#define HOFV_EILLCOND (-4)   /* singular / ill-conditioned reconstruction */
#define HOFV_ENAN (-5)       /* non-finite value met */
#define HOFV_ENOTSUP (-6)    /* feature not supported */
#define HOFV_ESTATE (-7)     /* call out of order (e.g. residual before set-up) */

/* laws (App. A) */
#define HOFV_LAW_LINEAR 0       /* small-strain Hooke's law, eq. (linearElastic) */
#define HOFV_LAW_NEOHOOKEAN 1   /* total-Lagrangian neo-Hookean, eq. (neoHook) */

/* preconditioners for hofv_precondition / hofv_newton_solve */
#define HOFV_PC_NONE (-1)
#define HOFV_PC_AJ64 0   /* compact approximate Jacobian, FP64 inner solve */
#define HOFV_PC_AJ32 1   /* same operator stored and applied in FP32 */
#define HOFV_PC_GNN 2    /* learned graph network on top of AJ32 */
#define HOFV_PC_AJMG 3   /* same operator (FP32), CG with an algebraic-multigrid V-cycle */
#define HOFV_PC_NEJ 4    /* near-exact Jacobian (linear law), inner GMRES with AJMG */

/* arithmetic of the gradient contraction (hofv_set_precision) */
#define HOFV_PREC_FP64 0   /* FP64 fused multiply-adds (default) */
#define HOFV_PREC_DF64 1   /* double-float pairs on the FP32 pipe, everything else FP64 */

/* point sets for hofv_get_points */
#define HOFV_PTS_CELL_CENTROID 0   /* [n_cells][dim] */
#define HOFV_PTS_DISP_QP 1         /* [n_disp][Q][dim]  displacement-face Gauss points */
#define HOFV_PTS_DISP_CENTRE 2     /* [n_disp][dim]     displacement-face centres */
#define HOFV_PTS_TRAC_QP 3         /* [n_trac][Q][dim]  traction-face Gauss points */
#define HOFV_PTS_CELL_QP 4         /* [n_cells][QC][dim] cell Gauss points */
#define HOFV_PTS_FACE_CENTRE 5     /* [n_faces][dim] all face centres */
#define HOFV_PTS_FACE_QP 6         /* [n_faces][Q][dim] all face Gauss points */
#define HOFV_PTS_FACE_AREA 7       /* [n_faces][Q][dim] vector area of each Gauss point */
#define HOFV_PTS_CELL_VOLUME 8     /* [n_cells] */

typedef struct hofv_ctx hofv_ctx;

typedef struct {
  int32_t dim;
  int32_t p;            /* reconstruction degree */
  int32_t stencil;      /* |S| = N_t + n_plus */
  int32_t n_t;          /* number of Taylor terms N_t = (d+p)! / (d! p!) */
  int32_t q_face;       /* Gauss points per face Q */
  int32_t q_cell;       /* Gauss points per cell QC */
  int64_t n_cells, n_faces, n_internal, n_disp, n_trac;
  double max_cond;      /* largest 2-norm condition-number estimate of the
                           scaled, weighted LSQ matrix W^1/2 Q^T seen at set-up */
  double setup_seconds; /* wall time of hofv_build_stencils */
  int64_t device_bytes; /* device memory held by the context */
  int64_t n_symm;       /* symmetry faces (after the displacement faces) */
} hofv_layout;

typedef struct {
  int32_t max_newton;      /* Newton iterations per call (default 30) */
  double rtol;             /* stop when ||R|| <= rtol * ||R(u_in)|| (default 1e-8) */
  double atol;             /* ... or ||R|| <= atol (default 0) */
  double ftol;             /* ... or ||R|| <= ftol * F_s * sqrt(dim * n_cells), F_s the force
                              scale of the entry state (hofv_force_scale): a floor for the
                              rounding noise of the FP64 residual (default 0 = off) */
  int32_t restart;         /* FGMRES restart length m (default 30, max 100) */
  int32_t max_krylov;      /* Krylov iterations per Newton step (default 300) */
  double eta_max;          /* forcing term cap (default 1e-2) */
  int32_t precond;         /* HOFV_PC_* (default HOFV_PC_AJ32) */
  int32_t inner_iters;     /* inner iterations per apply (default 30): CG for AJ64/AJ32,
                              V-cycles (1) or multigrid-CG for AJMG, GMRES for NEJ */
  int32_t line_search_max; /* backtracking halvings (default 10) */
  int32_t verbose;         /* 1: one line per Newton step on stderr */
  int32_t record_pairs;    /* 1: keep (-R(u_k), du_k) of every Newton step as a training
                              pair of the learned preconditioner (hofv_gnn_train); 2: also
                              keep (J z, z) for the preconditioned Krylov vectors z of a few
                              Arnoldi steps (exact inverse-Jacobian pairs, one Jv each) */
  int32_t gnn_judge;       /* 1 (default): a learned-preconditioner restart cycle whose mean
                              per-iteration residual reduction is worse than that of the last
                              FGMRES solve preconditioned by AJ alone switches the rest of the
                              Newton solve to AJ; 0: never switch (non-finite output still does) */
} hofv_solve_opts;

typedef struct {
  int32_t newton_iters;
  int32_t krylov_iters;    /* total over the call */
  int32_t residual_evals;  /* R evaluations incl. those inside Jv */
  int32_t precond_applies;
  int32_t gnn_fallbacks;   /* learned-preconditioner cycles replaced by AJ */
  double r0, r_final;      /* ||R|| at entry and exit */
  double seconds;
  int32_t status;          /* same as the return value */
} hofv_stats;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
   (NULL = the legacy default stream) on which all work is enqueued. */
int hofv_create(hofv_ctx** out, int device, void* cuda_stream);
void hofv_destroy(hofv_ctx* ctx);
/* Message of the last error on this context (never NULL). */
const char* hofv_last_error(const hofv_ctx* ctx);
/* Library version string. */
const char* hofv_version(void);

/* ---- set-up ------------------------------------------------------------ */

/* Mesh of straight-edged quads (dim 2, unit depth, nodes counter-clockwise)
   or hexahedra (dim 3, bottom face counter-clockwise seen from +z, then the
   top face).  All arrays are HOST arrays, copied in:
     xyz         [n_nodes][dim]
     cell_nodes  [n_cells][2^dim]
     bface_nodes [n_bfaces][2^(dim-1)]   every boundary face exactly once
     bface_tag   [n_bfaces]  0 = prescribed displacement, 1 = prescribed
                             traction, 2 = symmetry (a plane of mirror
                             symmetry: zero normal displacement and shear
                             traction; Sec. 3.5.2-3.5.3)
   Face sets of Sec. 3.1; faces are numbered internal, displacement,
   symmetry, traction.  A symmetry face's stencil holds the ceil(S/2) cells
   nearest its centre and the mirror images of the floor(S/2) nearest of
   them, whose values are the reflected states (I - 2 n n) u.  Errors:
   EINVAL if a boundary face is missing, duplicated or not on the boundary,
   or a tag is unknown. */
int hofv_set_mesh(hofv_ctx* ctx, int dim, int64_t n_nodes, const double* xyz,
                  int64_t n_cells, const int64_t* cell_nodes, int64_t n_bfaces,
                  const int64_t* bface_nodes, const int32_t* bface_tag);

/* cell kinds for hofv_set_mesh_cells */
#define HOFV_CELL_TENSOR 0   /* quadrilaterals (dim 2) / hexahedra (dim 3) */
#define HOFV_CELL_SIMPLEX 1  /* triangles (dim 2) / tetrahedra (dim 3) */

/* hofv_set_mesh for a given cell kind; HOFV_CELL_TENSOR is hofv_set_mesh.
   HOFV_CELL_SIMPLEX takes unstructured triangles (counter-clockwise) or
   tetrahedra (positively oriented: (x1-x0) . ((x2-x0) x (x3-x0)) > 0) with
     cell_nodes  [n_cells][dim + 1]
     bface_nodes [n_bfaces][dim]
   Their faces are straight edges or flat triangles; the face rule keeps
   q_per_dir^(dim-1) points, a triangle being the bilinear patch with a
   repeated corner (the collapsed square of Duffy's transformation), and the
   cell rule keeps q_per_dir^dim points on the collapsed square / cube.
   Every other call works unchanged on such meshes.  Errors as
   hofv_set_mesh; EINVAL for an unknown cell_kind. */
int hofv_set_mesh_cells(hofv_ctx* ctx, int dim, int cell_kind, int64_t n_nodes,
                        const double* xyz, int64_t n_cells, const int64_t* cell_nodes,
                        int64_t n_bfaces, const int64_t* bface_nodes,
                        const int32_t* bface_tag);

/* hofv_set_mesh for a 2-D mesh of polygons with 3 to 8 corners each, e.g.
   the dual of a triangle mesh.  HOST arrays, copied in:
     xyz         [n_nodes][2]
     cell_ptr    [n_cells + 1], cell_ptr[0] = 0; cell c has the corners
                 cell_nodes[cell_ptr[c] .. cell_ptr[c+1]), counter-clockwise
     bface_nodes [n_bfaces][2], bface_tag [n_bfaces] as hofv_set_mesh
   Local face k of a cell runs from its corner k to corner k+1; every cell
   keeps 8 face slots (ext rows of hofv_get_cell_data), those past its last
   side holding no face.  Faces are straight edges with q_per_dir Gauss
   points; the cell rule is the fan of triangles from the corners' average
   to each side, q_per_dir^2 points on each (collapsed square), 8 q_per_dir^2
   points per cell with zero weights past the last side.  Errors as
   hofv_set_mesh; EINVAL for a polygon with fewer than 3 or more than 8
   corners, or one that is not counter-clockwise and star-shaped about its
   corners' average. */
int hofv_set_mesh_polygons(hofv_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_cells,
                           const int64_t* cell_ptr, const int64_t* cell_nodes,
                           int64_t n_bfaces, const int64_t* bface_nodes,
                           const int32_t* bface_tag);

/* hofv_set_mesh for a 3-D mesh of polyhedra given face by face (the layout
   of a polyMesh; arbitrary convex polyhedra, Sec. 3.1-3.3, with their faces
   split into triangles and their cells into tetrahedra).  HOST arrays,
   copied in:
     xyz        [n_nodes][3]
     face_ptr   [n_faces + 1], face_ptr[0] = 0; face i has the corners
                face_nodes[face_ptr[i] .. face_ptr[i+1]) (3 to 8), ordered so
                that the right-hand-rule normal points out of owner[i]
     owner      [n_faces] cell ids in [0, n_cells)
     neighbour  [n_faces] the other cell, -1 for a boundary face
     face_tag   [n_faces] boundary tag as hofv_set_mesh (read only where
                neighbour is -1)
   Each cell needs 4 to 16 faces; its local faces are its faces in input
   order (16 slots, ext rows of hofv_get_cell_data, empty past its last
   face).  Faces are renumbered as everywhere: internal faces by (owner,
   owner's local face) with owner < neighbour (a face whose owner has the
   higher id is flipped), then displacement, symmetry and traction faces in
   input order.  A face is the fan of triangles from its corners' average,
   each the collapsed square with q_per_dir^2 points; a face has 4 corner
   slots when no face of the mesh has more than 4 corners, else 8, so
   Q = q_per_dir^2 * slots, and the points of slots past a face's last
   corner sit at its corners' average with zero area.  A cell's rule is the
   fan of tetrahedra (its faces' fan triangles joined to the average of its
   faces' corner averages), each the collapsed cube with q_per_dir^3
   points.  q_per_dir must be 1 or 2 (hofv_set_scheme).  Errors: EINVAL for
   a bad count, id or tag. */
int hofv_set_mesh_faces(hofv_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_cells,
                        int64_t n_faces, const int64_t* face_ptr, const int64_t* face_nodes,
                        const int64_t* owner, const int64_t* neighbour,
                        const int32_t* face_tag);

/* Scheme (Sec. 3.5): reconstruction degree p in 1..3, surplus stencil nodes
   n_plus (|S| = N_t + n_plus; the paper uses 10 in 2-D and 45/55/65 in 3-D),
   Gauss points per face direction q_per_dir in 1..4 in 2-D, 1..3 in 3-D and
   1..2 on polyhedra (faces are bilinear patches with q_per_dir^(dim-1)
   tensor Gauss-Legendre points; polyhedral faces fans of them), weight shape
   k_weight (eq. weightFunc, paper: 6) and stabilisation factor alpha
   (eq. alpha, paper: 0.1). */
int hofv_set_scheme(hofv_ctx* ctx, int p, int n_plus, int q_per_dir,
                    double k_weight, double alpha);

/* Build everything that depends only on the mesh, on the device: geometry
   and quadrature, nearest-neighbour stencils (Sec. 3.5.2), the
   least-squares reconstruction coefficients by Householder QR (eqs. ls-lsA),
   the alpha-stabilisation extrapolation weights (eq. alphaJump, App. B) and
   the compact approximate Jacobian (Sec. 4.1).  Synchronises.
   Errors: ESTATE before set_mesh/set_scheme, ENOMEM, EILLCOND. */
int hofv_build_stencils(hofv_ctx* ctx);

/* Replace the nearest-neighbour stencils (Sec. 3.5.2) by the caller's and
   recompute everything made from them (reconstruction coefficients, the
   stabilisation extrapolation weights of eq. alphaJump, the cell averages of
   the inertia term, the contracted linear-elastic matrices; the near-exact
   Jacobian is rebuilt on its next use).  HOST int32 cell ids, row-major,
   copied in:
     face_stencils [n_internal + n_disp][S]   (NULL: keep the current ones)
     cell_stencils [n_cells][S]               (NULL: keep the current ones)
   The order of the ids within a stencil does not matter; the caller keeps
   them distinct.  Needs hofv_build_stencils first (ESTATE).  Errors: EINVAL
   for an id outside [0, n_cells), ENOTSUP on meshes with symmetry faces
   (their stencils hold mirror nodes), EILLCOND when a fit is singular; on
   any error the previous stencils are restored.  Synchronises. */
int hofv_set_stencils(hofv_ctx* ctx, const int32_t* face_stencils,
                      const int32_t* cell_stencils);

int hofv_get_layout(const hofv_ctx* ctx, hofv_layout* out);

/* Copy a point set (HOFV_PTS_*) to the HOST array `out` (layouts above),
   so the caller can evaluate boundary data and body forces. */
int hofv_get_points(hofv_ctx* ctx, int kind, double* out);

/* Material (App. A).  For neo-Hookean the bulk modulus is
   kappa = lambda + 2 mu / 3; the stabilisation stiffness is
   Kbar = 2 mu + lambda in both laws (Sec. 3.4). */
int hofv_set_material(hofv_ctx* ctx, int law, double mu, double lambda);

/* Evaluate the linear-elastic flux in contracted form (on = 1) or per Gauss
   point (on = 0, default).  With Hooke's law the traction of a face is linear
   in the stencil values, so the law and the Gauss quadrature of
   eq. divStressDiscret fold exactly into one d x d matrix per face and
   stencil cell, T_N = sum_q mu c_qN (x) a_q + mu (c_qN . a_q) I +
   lambda a_q (x) c_qN, built when the material is set (extra device memory:
   |S| d^2 doubles per face).  Results equal the per-point form up to
   rounding; the neo-Hookean law always uses the per-point form. */
int hofv_set_contraction(hofv_ctx* ctx, int on);

/* Arithmetic of the dominant step of the residual, the contraction of the
   reconstruction coefficients with the stencil values (the displacement
   gradient at every face Gauss point, eq. faceQuadGrad, and the
   extrapolated face values of the stabilisation, eq. alphaJump).
   HOFV_PREC_FP64 (default) uses FP64 fused multiply-adds.  HOFV_PREC_DF64
   stores each coefficient as a pair of floats (hi, lo), hi + lo its value
   rounded to 48 significant bits, splits the state exactly into three
   floats, and forms each product exactly (TwoProduct by FMA, Dekker 1971)
   and the sums with TwoSum and a compensation term (Dot2, Ogita, Rump &
   Oishi 2005) on the FP32 pipe.  The face gradients contract the
   differences to each face's nearest stencil cell (exact differences of the
   splits) and add back that cell's value times the FP64 sum of the stored
   coefficients, so the rounding acts on the local variation of the field
   and not on its magnitude.  Each gradient is then converted to FP64; the
   law, quadrature, stabilisation jump, assembly and every solver vector stay
   FP64.  With HOFV_PREC_DF64, hofv_jvp evaluates the forward difference
   without differencing two separately rounded residuals: for the linear law
   the residual is affine and (R(u + eps v) - R(u)) / eps is its
   homogeneous part at v; for the neo-Hookean law the face kernels contract
   v alone and difference, in FP64, the tractions at grad u + eps grad v and
   at grad u, with grad u and its tractions cached per (u, Ru) pair (filled
   on the first Jv after the state or the data change; hofv_residual at u
   marks it stale).  Ru is not read.  Callable at any time: after
   hofv_build_stencils the coefficient arrays are rewritten in place
   (synchronises); switching back to FP64 keeps the 48-bit values until the
   next hofv_build_stencils.  The environment variable HOFV_PRECISION
   (fp64 / df64) sets the default of new contexts.  EINVAL for an unknown
   mode. */
int hofv_set_precision(hofv_ctx* ctx, int prec);
/* The current HOFV_PREC_* of the context (or EINVAL for NULL). */
int hofv_get_precision(const hofv_ctx* ctx);

/* y = J_NEJ x with the near-exact Jacobian of the appendix on the
   near-exact-Jacobian preconditioner: the Jacobian of the face fluxes of
   the linear-elastic law without the stabilisation term (ghost-node and
   traction contributions are constants and drop out).  Assembled on first
   use (and after a material change) as block CSR with d x d FP32 blocks,
   columns = the union of each cell's face stencils; products accumulate in
   FP32.  x, y: DEVICE [dim][n_cells].  HOFV_ENOTSUP for the neo-Hookean
   law and for meshes with symmetry faces. */
int hofv_nej_apply(hofv_ctx* ctx, const double* x, double* y);

/* Inertia term for dynamics (eq. inertiaTerm; BDF2 of the appendix on time
   integration): the residual becomes R(u) - int_Omega rho u_tt dOmega with
   the acceleration of every cell Gauss point
     a = (3 v^{t+1} - 4 v^t + v^{t-1}) / (2 dt),
     v^{t+1} = (3 u^{t+1} - 4 u^t + u^{t-1}) / (2 dt),
   and the point values extrapolated from the cell centroid with the Taylor
   terms of the cell fit (as in eq. alphaJump).  rho is constant, so the sum
   over the Gauss points reduces to cell averages ubar = u_P + sum_N m_N u_N
   of the fit; one_point = 1 uses the centroid alone (ubar = u_P, one
   integration point per cell), 0 the cell's q_per_dir^d Gauss points.
   rho > 0 and dt > 0 enable the term; rho = 0 disables it.  The compact
   approximate Jacobian gains -rho Omega_P 9/(4 dt^2) on its diagonal.  The
   history starts at rest (zero) until hofv_set_history.  HOFV_ESTATE before
   hofv_build_stencils. */
int hofv_set_inertia(hofv_ctx* ctx, double rho, double dt, int one_point);

/* History of the current time step: displacements u^t, u^{t-1} (DEVICE
   [dim][n_cells], cell centroid values; u_tm1 NULL = u_t) and cell-average
   velocities v^t, v^{t-1} (DEVICE [dim][n_cells] as returned by
   hofv_bdf2_velocity; NULL = zero).  Folded into the constant source of
   the residual.  HOFV_ESTATE unless the inertia term is enabled. */
int hofv_set_history(hofv_ctx* ctx, const double* u_t, const double* u_tm1, const double* v_t,
                     const double* v_tm1);

/* Cell-average velocity after a solved step, v^{t+1} = (3 ubar^{t+1} -
   4 ubar^t + ubar^{t-1}) / (2 dt) (u_tm1 NULL = u_t).  DEVICE [dim][n_cells]
   vectors; enqueued on the context stream. */
int hofv_bdf2_velocity(hofv_ctx* ctx, const double* u_tp1, const double* u_t, const double* u_tm1,
                       double* v_out);

/* Cell averages of the cell least-squares fit over each cell's Gauss points,
   ubar = u_P + sum_N m_N u_N (the weights are computed on first use).
   DEVICE [dim][n_cells]. */
int hofv_cell_average(hofv_ctx* ctx, const double* u, double* ubar);

/* Boundary data and sources, DEVICE arrays copied into the context (any may
   be NULL = zero):
     u_bq  [n_disp][Q][dim]  prescribed displacement at displacement-face Gauss points
     u_bf  [n_disp][dim]     prescribed displacement at displacement-face centres
     t_bq  [n_trac][Q][dim]  prescribed traction at traction-face Gauss points
     body  [dim][n_cells]    integrated body force per cell (eq. bodyTerm) */
int hofv_set_bc(hofv_ctx* ctx, const double* u_bq, const double* u_bf,
                const double* t_bq, const double* body);

/* Gauss quadrature over each cell, eq. (bodyTerm): f_qp [n_cells][QC][dim]
   (DEVICE) -> b [dim][n_cells] (DEVICE). */
int hofv_integrate_cells(hofv_ctx* ctx, const double* f_qp, double* b);

/* ---- evaluation (hot path) -------------------------------------------- */

/* R(u) = sum of face tractions (Gauss quadrature, eq. divStressDiscret) +
   alpha stabilisation (eq. alpha) + traction-boundary and body sources.
   u, R: DEVICE [dim][n_cells].  Enqueued on the context stream. */
int hofv_residual(hofv_ctx* ctx, const double* u, double* R);

/* Jacobian-vector product by forward difference (Sec. 4.1):
   Jv = (R(u + eps v) - R(u)) / eps with
   eps = sqrt(2^-52) (1 + ||u||_2) / ||v||_2 computed on the device.
   Ru must hold R(u) (with HOFV_PREC_DF64 it is not read: see
   hofv_set_precision).  u, Ru, v, Jv: DEVICE [dim][n_cells].  eps_used: HOST
   pointer or NULL; when non-NULL the call synchronises to return eps. */
int hofv_jvp(hofv_ctx* ctx, const double* u, const double* Ru, const double* v,
             double* Jv, double* eps_used);

/* z ~= P^{-1} v with the compact approximate Jacobian P (Sec. 4.1) applied
   to every displacement component: HOFV_PC_AJ64 / AJ32 run `inner_iters`
   Jacobi-preconditioned CG iterations in FP64 / FP32; HOFV_PC_AJMG applies
   one V-cycle of smoothed-aggregation multigrid on P (FP32) when
   inner_iters <= 1, else runs `inner_iters` CG iterations preconditioned by
   that V-cycle (hierarchy built on first use, once per mesh; the paper
   leaves the inner solve of P to its linear-algebra library); HOFV_PC_NEJ
   approximates the inverse of the near-exact Jacobian instead (linear law
   only, HOFV_ENOTSUP otherwise; see hofv_nej_apply) by `inner_iters` GMRES
   iterations right-preconditioned by one AJMG V-cycle; HOFV_PC_GNN adds the learned correction (needs hofv_gnn_load or
   hofv_gnn_train first).  v, z: DEVICE [dim][n_cells]. */
int hofv_precondition(hofv_ctx* ctx, int kind, int inner_iters, const double* v, double* z);

/* Newton-Krylov solve of R(u) = 0 from the DEVICE vector u (updated in
   place): flexible GMRES(m), right preconditioned, Jv by forward
   differences, backtracking line search on ||R||_2.  opts/stats are HOST
   pointers (opts NULL = defaults).  Returns 0, HOFV_WNOTCONV, or an error.
   Synchronises. */
int hofv_newton_solve(hofv_ctx* ctx, double* u, const hofv_solve_opts* opts,
                      hofv_stats* stats);

/* Everything hofv_newton_solve and hofv_arnoldi_step allocate or build on
   first use, done now for the options `opts` (NULL = defaults): the Krylov
   basis of opts->restart vectors, the multigrid hierarchy (HOFV_PC_AJMG,
   HOFV_PC_NEJ) and the near-exact Jacobian (HOFV_PC_NEJ), the linearisation
   cache of the double-float neo-Hookean Jv.  After it the evaluation calls
   and solves with these options allocate nothing (the first Arnoldi step of
   a kind still captures its CUDA graph).  Synchronises. */
int hofv_prepare_solver(hofv_ctx* ctx, const hofv_solve_opts* opts);

/* Load incrementation (the paper's load steps of its hyperelastic cases,
   Sec. 5) with automatic cut-back.  The context's current boundary data
   (hofv_set_bc) are the data at load factor 0, where u (DEVICE
   [dim][n_cells], updated in place) is a converged state; the DEVICE arrays
   u_bq1, u_bf1, t_bq1, body1 (layouts of hofv_set_bc; NULL = unchanged)
   are the data at factor 1.  The factor advances in n_steps equal
   increments; the data of each are interpolated linearly and the step is
   solved by hofv_newton_solve with `opts` from a predictor: u +
   increment * du_dlambda (DEVICE [dim][n_cells], the state's derivative
   with respect to the factor as the caller estimates it) when du_dlambda
   is not NULL, else the secant through the last two converged states.  A
   step whose solve fails (HOFV_WNOTCONV or HOFV_ENAN) is retried from the
   last converged state with half the increment, up to max_halvings times
   in a row; after a success the increment doubles back towards the
   nominal one.  On return u holds the last converged state and the
   context's data are those of its load factor; *steps_done (HOST, may be
   NULL) counts the accepted increments and *stats (HOST, may be NULL)
   sums the solver counts.  Returns 0 at factor 1, HOFV_WNOTCONV if an
   increment still failed after max_halvings halvings, or an error.
   Allocates two copies of the boundary data and three state vectors for
   the duration of the call; synchronises. */
int hofv_solve_load_path(hofv_ctx* ctx, double* u, const double* u_bq1, const double* u_bf1,
                         const double* t_bq1, const double* body1, const double* du_dlambda,
                         int32_t n_steps, int32_t max_halvings, const hofv_solve_opts* opts,
                         hofv_stats* stats, int32_t* steps_done);

/* ---- learned preconditioner ---------------------------------------------
   A graph network over the cell adjacency (no counterpart in the paper):
   nodes are cells, neighbours are face neighbours weighted by the
   normalised compact approximate Jacobian, w_ij = a_ij / sqrt(D_i D_j).
   Inputs per cell: v / rms(v), z / rms(z) with z = P_AJ^{-1} v, and the
   fractions of displacement and traction faces (16 features, zero-padded);
   encoder 16 -> 64 (ReLU), four message-passing layers
   h += ReLU(W [h ; sum_j w_ij h_j] + b) with W 64 x 128, decoder 64 -> dim.
   The preconditioned vector is z + rms(z) * y.  Node-wise products run on
   the tensor cores in BF16 with FP32 accumulation; parameters are FP32.
   Parameter order (flat): W0 [64][16], b0 [64], then per layer W [64][128],
   b [64], then Wd [dim][64], bd [dim].  Training minimises
   |z + rms(z) y - delta|^2 / |delta|^2 over recorded (residual, Newton
   correction) pairs with Adam.  All entry points need hofv_build_stencils;
   changing the mesh or scheme discards the network. */

typedef struct {
  int32_t epochs;       /* passes over the recorded pairs */
  int32_t batch;        /* pairs per Adam step */
  double lr;            /* Adam learning rate */
  int32_t inner_iters;  /* CG iterations of the AJ preconditioner feeding the network */
  uint64_t seed;        /* shuffling seed */
  int32_t verbose;
} hofv_train_opts;

typedef struct {
  int32_t pairs, epochs;
  double loss_first, loss_last;  /* mean loss of the first and last epoch */
  double seconds;
} hofv_train_stats;

/* Random initialisation (seeded); the output layer is scaled by out_scale
   (0 gives the identity correction z_out = z). */
int hofv_gnn_init(hofv_ctx* ctx, uint64_t seed, double out_scale);
int hofv_gnn_num_params(hofv_ctx* ctx, int64_t* n);
/* Copy the FP32 parameters to / from a HOST array of hofv_gnn_num_params. */
int hofv_gnn_get_params(hofv_ctx* ctx, float* host, int64_t n);
int hofv_gnn_set_params(hofv_ctx* ctx, const float* host, int64_t n);
/* Save / load the parameters (binary file with a dimension check). */
int hofv_gnn_save(hofv_ctx* ctx, const char* path);
int hofv_gnn_load(hofv_ctx* ctx, const char* path);
/* zout = z + rms(z) G(v, z): DEVICE [dim][n_cells]; zout may alias z. */
int hofv_gnn_forward(hofv_ctx* ctx, const double* v, const double* z, double* zout);
/* Loss of one sample (v, z, delta DEVICE) and its gradient (HOST float
   array of hofv_gnn_num_params, may be NULL); *loss HOST.  Synchronises. */
int hofv_gnn_loss_grad(hofv_ctx* ctx, const double* v, const double* z, const double* delta,
                       double* loss, float* grad);
/* Record one training pair (r, delta), DEVICE vectors copied in. */
int hofv_gnn_record(hofv_ctx* ctx, const double* r, const double* delta);
int hofv_gnn_pairs(hofv_ctx* ctx, int32_t* count);
int hofv_gnn_clear_pairs(hofv_ctx* ctx);
/* Train on the recorded pairs (Adam, FP32 master weights).  Synchronises. */
int hofv_gnn_train(hofv_ctx* ctx, const hofv_train_opts* opts, hofv_train_stats* stats);

/* Fill `opts` with the defaults listed in hofv_solve_opts. */
void hofv_default_opts(hofv_solve_opts* opts);

/* Force scale F_s = max over cells of the sum over the cell's internal and
   displacement faces of |flux_f| at the state u (DEVICE [dim][n_cells]); the
   magnitude against which the rounding error of R(u) is measured.  *fs is
   a HOST pointer.  Synchronises. */
int hofv_force_scale(hofv_ctx* ctx, const double* u, double* fs);

/* One flexible-GMRES Arnoldi step of the JFNK solver (Sec. 4.1, right
   preconditioning): Z_j = P^{-1} V_j (preconditioner `kind`, `inner_iters`),
   w = J Z_j by forward differences about u (Ru = R(u)), w orthogonalised
   against V_0..V_j by classical Gram-Schmidt applied twice, and
   V_{j+1} = w / ||w||.  This is one pass over every kernel of the hot path.
     V  DEVICE [(j+2)][ld], columns 0..j given, column j+1 written
     Z  DEVICE [(j+1)][ld], column j written
     ld >= dim * n_cells (elements between columns)
     h  HOST [j+2] receives the Hessenberg column (h[j+1] = ||w||)
   Synchronises.  j must be in 0..99. */
int hofv_arnoldi_step(hofv_ctx* ctx, const double* u, const double* Ru, int kind,
                      int inner_iters, double* V, double* Z, int64_t ld, int j, double* h);

/* Same result as hofv_residual, for callers that must not have device memory
   allocated on their behalf (for example code running while a stream is
   captured into a CUDA graph, real-time loops that forbid allocation after
   start-up, or frameworks that own every device allocation).  The paper has
   no counterpart: this is a property of the library, not of the method.
   The call allocates nothing: its scratch is one fixed device array of
   32 MiB (4 Mi doubles) compiled into the library and held on every GPU
   that loads it until exit.  A mesh needs n_cells * F * dim doubles
   (F = face slots per cell: dim + 1 for triangles / tetrahedra, 2 dim for
   quads / hexes, 8 for polygons), rounded up to a multiple of 32, plus
   (n_internal + n_disp + n_symm) * dim, rounded up to 32, plus with
   HOFV_PREC_DF64 (n_cells + mirror nodes) * 4 (2-D) or 6 (3-D) for the
   split state, rounded up to 32; larger meshes get HOFV_EINVAL.  All calls share the array:
   calls that overlap on the GPU race and must be serialised by the caller.
   Like every evaluation call it also writes buffers of its own context
   (extended state and mirrored face values of symmetry faces, the inertia
   term), so it must be ordered with the context's other evaluation calls
   issued from other streams.  The first call on a device resolves the
   array's address (cudaGetSymbolAddress), again after the device's CUDA
   context has changed (e.g. after cudaDeviceReset); that first call should
   come before any stream capture.  u, R: DEVICE [dim][n_cells]. */
int hofv_residual_noalloc(hofv_ctx* ctx, const double* u, double* R);

/* The multigrid hierarchy of HOFV_PC_AJMG (built here if not yet built):
   number of levels, the cell count of the first min(levels, max_sizes)
   levels into sizes (HOST), stored non-zeros over all levels, and the host
   seconds its construction took.  Synchronises. */
int hofv_mg_info(hofv_ctx* ctx, int32_t* levels, int64_t* sizes, int32_t max_sizes,
                 int64_t* nnz, double* setup_seconds);

/* Self-test of the bounded waits: the approximate-Jacobian solve runs as one
   cooperative launch whose blocks meet at grid barriers; each wait gives up
   after a bounded number of polls, latches an error flag and returns, and
   the host reports HOFV_ECUDA at its next synchronisation.  This launches
   two blocks that wait for a third arrival that never comes; on return
   *timed_out (HOST) is 1 when the wait ran out and was latched, and the
   flag has been cleared so the context stays usable.  Synchronises. */
int hofv_selftest_barrier(hofv_ctx* ctx, int32_t* timed_out);

/* hofv_residual with each of its three kernels timed by CUDA events on the
   context stream: ms[0] stabilisation extrapolation (cell-ordered), ms[1]
   face fluxes, ms[2] cell assembly (HOST array of 3).  Synchronises. */
int hofv_residual_timed(hofv_ctx* ctx, const double* u, double* R, float* ms);

/* hofv_jvp (Sec. 4.1) with its kernels timed by CUDA events on the context
   stream: ms[0] the direction's split and stabilisation extrapolation (or,
   in FP64 mode, the residual's extrapolation after u + eps v is formed),
   ms[1] the face fluxes, ms[2] the cell assembly (HOST array of 3).  The
   same arguments, layouts and errors as hofv_jvp.  Synchronises. */
int hofv_jvp_timed(hofv_ctx* ctx, const double* u, const double* Ru, const double* v, double* Jv,
                   float* ms);

/* ---- measurement ----------------------------------------------------------- */

/* Arithmetic peaks of the context's device, measured: FP64 and FP32 fused
   multiply-add throughput in TFLOP/s (2 flops per FMA) from register-only
   kernels on every SM, timed with CUDA events on the context stream, and
   the number of SMs.  The denominators of the benchmark's ALU rooflines;
   no counterpart in the paper.  Any output pointer may be NULL (that peak
   is not measured).  Allocates 64 bytes for the duration of the call and
   synchronises. */
int hofv_probe_peaks(hofv_ctx* ctx, double* fp64_tflops, double* fp32_tflops, int32_t* sm_count);

/* The neo-Hookean law's J^{-1/3} (App. A, eq. neoHook: the isochoric factor
   J^{-2/3} and the volumetric term use r = J^{-1/3}) as the face kernels
   evaluate it -- a single-precision estimate corrected once in FP64 by the
   binomial series of (1 - h)^{-1/3}, h = 1 - J r^3 -- next to CUDA's
   double-precision rcbrt, for n values J (DEVICE arrays of n doubles; r_own
   and r_lib DEVICE outputs of n doubles, either may be NULL).  Checks the
   law's own routine against the library's error bound; no counterpart in
   the paper.  HOFV_EINVAL for n < 0 or a NULL J with n > 0.  Synchronises. */
int hofv_probe_inv_cbrt(hofv_ctx* ctx, const double* J, double* r_own, double* r_lib, int64_t n);

/* ---- inspection (tests) -------------------------------------------------- */

/* Face data for faces [first, first + count) to HOST arrays (any may be NULL):
     stencil [count][S]        int32 cell ids (internal and displacement faces)
     coef    [count][Q][S+1][dim]  gradient coefficients; slot S = ghost node
   Traction faces have no stencil; their rows are left untouched. */
int hofv_get_face_data(hofv_ctx* ctx, int64_t first, int64_t count, int32_t* stencil,
                       double* coef);

/* Cell data for cells [first, first + count) to HOST arrays (any may be NULL):
     stencil [count][S] int32;  ext [count][F][S] weights e with
     u*_{f,P} = u_P + sum_N e_N u_N (eq. alphaJump); F = faces per cell
     (2 dim for quads / hexes, dim + 1 for triangles / tetrahedra, 8 slots
     for polygons, 16 for polyhedra, zero rows past a cell's last face). */
int hofv_get_cell_data(hofv_ctx* ctx, int64_t first, int64_t count, int32_t* stencil,
                       double* ext);

/* Faces: owner, neighbour (-1 on the boundary), owner local face, tag
   (-1 internal, 0 displacement, 1 traction); HOST arrays [n_faces]. */
int hofv_get_faces(hofv_ctx* ctx, int64_t* owner, int64_t* neighbour, int32_t* local_face,
                   int32_t* tag);

/* Approximate Jacobian (Sec. 4.1) in FP64: diag [n_cells], off [n_internal]
   (entry coupling owner and neighbour of internal face f); HOST arrays. */
int hofv_get_aj(hofv_ctx* ctx, double* diag, double* off);

#ifdef __cplusplus
}
#endif
#endif /* HOFV_H */
