"""Thin Python binding of libhofv (C ABI in ``include/hofv.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device vectors are torch CUDA tensors (FP64, component-major
``[dim, n_cells]``); torch provides device memory and the stream.  The
library must have been built (``paper_2601_18417_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhofv.so")

OK, WNOTCONV = 0, 1
EINVAL, ENOMEM, ECUDA, EILLCOND, ENAN, ENOTSUP, ESTATE = -1, -2, -3, -4, -5, -6, -7
LAW_LINEAR, LAW_NEOHOOKEAN = 0, 1
PC_NONE, PC_AJ64, PC_AJ32, PC_GNN, PC_AJMG, PC_NEJ = -1, 0, 1, 2, 3, 4
PREC_FP64, PREC_DF64 = 0, 1
CELL_TENSOR, CELL_SIMPLEX = 0, 1
POLY_SLOTS = 8  # face slots of a polygon cell
POLYHEDRON_SLOTS = 16  # face slots of a polyhedral cell
PTS_CELL_CENTROID, PTS_DISP_QP, PTS_DISP_CENTRE, PTS_TRAC_QP, PTS_CELL_QP = 0, 1, 2, 3, 4
PTS_FACE_CENTRE, PTS_FACE_QP, PTS_FACE_AREA, PTS_CELL_VOLUME = 5, 6, 7, 8


class HofvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hofv error {code}: {msg}")
        self.code = code


class Layout(C.Structure):
    _fields_ = [("dim", C.c_int32), ("p", C.c_int32), ("stencil", C.c_int32), ("n_t", C.c_int32),
                ("q_face", C.c_int32), ("q_cell", C.c_int32), ("n_cells", C.c_int64),
                ("n_faces", C.c_int64), ("n_internal", C.c_int64), ("n_disp", C.c_int64),
                ("n_trac", C.c_int64), ("max_cond", C.c_double), ("setup_seconds", C.c_double),
                ("device_bytes", C.c_int64), ("n_symm", C.c_int64)]


class SolveOpts(C.Structure):
    _fields_ = [("max_newton", C.c_int32), ("rtol", C.c_double), ("atol", C.c_double),
                ("ftol", C.c_double),
                ("restart", C.c_int32), ("max_krylov", C.c_int32), ("eta_max", C.c_double),
                ("precond", C.c_int32), ("inner_iters", C.c_int32),
                ("line_search_max", C.c_int32), ("verbose", C.c_int32),
                ("record_pairs", C.c_int32), ("gnn_judge", C.c_int32)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("inner_iters", C.c_int32), ("seed", C.c_uint64), ("verbose", C.c_int32)]


class TrainStats(C.Structure):
    _fields_ = [("pairs", C.c_int32), ("epochs", C.c_int32), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("krylov_iters", C.c_int32),
                ("residual_evals", C.c_int32), ("precond_applies", C.c_int32),
                ("gnn_fallbacks", C.c_int32), ("r0", C.c_double), ("r_final", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# exported entry points and their argument types
_P, _I, _I64, _D = C.c_void_p, C.c_int, C.c_int64, C.c_double
SIGNATURES = {
    "hofv_create": (_I, [C.POINTER(_P), _I, _P]),
    "hofv_destroy": (None, [_P]),
    "hofv_last_error": (C.c_char_p, [_P]),
    "hofv_version": (C.c_char_p, []),
    "hofv_set_mesh": (_I, [_P, _I, _I64, _P, _I64, _P, _I64, _P, _P]),
    "hofv_set_mesh_cells": (_I, [_P, _I, _I, _I64, _P, _I64, _P, _I64, _P, _P]),
    "hofv_set_mesh_polygons": (_I, [_P, _I64, _P, _I64, _P, _P, _I64, _P, _P]),
    "hofv_set_mesh_faces": (_I, [_P, _I64, _P, _I64, _I64, _P, _P, _P, _P, _P]),
    "hofv_set_scheme": (_I, [_P, _I, _I, _I, _D, _D]),
    "hofv_build_stencils": (_I, [_P]),
    "hofv_get_layout": (_I, [_P, C.POINTER(Layout)]),
    "hofv_get_points": (_I, [_P, _I, _P]),
    "hofv_set_material": (_I, [_P, _I, _D, _D]),
    "hofv_set_bc": (_I, [_P, _P, _P, _P, _P]),
    "hofv_integrate_cells": (_I, [_P, _P, _P]),
    "hofv_residual": (_I, [_P, _P, _P]),
    "hofv_jvp": (_I, [_P, _P, _P, _P, _P, C.POINTER(_D)]),
    "hofv_precondition": (_I, [_P, _I, _I, _P, _P]),
    "hofv_newton_solve": (_I, [_P, _P, C.POINTER(SolveOpts), C.POINTER(Stats)]),
    "hofv_default_opts": (None, [C.POINTER(SolveOpts)]),
    "hofv_get_face_data": (_I, [_P, _I64, _I64, _P, _P]),
    "hofv_get_cell_data": (_I, [_P, _I64, _I64, _P, _P]),
    "hofv_get_faces": (_I, [_P, _P, _P, _P, _P]),
    "hofv_get_aj": (_I, [_P, _P, _P]),
    "hofv_arnoldi_step": (_I, [_P, _P, _P, _I, _I, _P, _P, _I64, _I, _P]),
    "hofv_residual_timed": (_I, [_P, _P, _P, _P]),
    "hofv_jvp_timed": (_I, [_P, _P, _P, _P, _P, _P]),
    "hofv_residual_noalloc": (_I, [_P, _P, _P]),
    "hofv_force_scale": (_I, [_P, _P, C.POINTER(_D)]),
    "hofv_set_contraction": (_I, [_P, _I]),
    "hofv_set_precision": (_I, [_P, _I]),
    "hofv_probe_peaks": (_I, [_P, C.POINTER(_D), C.POINTER(_D), C.POINTER(C.c_int32)]),
    "hofv_probe_inv_cbrt": (_I, [_P, _P, _P, _P, C.c_int64]),
    "hofv_set_stencils": (_I, [_P, _P, _P]),
    "hofv_prepare_solver": (_I, [_P, C.POINTER(SolveOpts)]),
    "hofv_solve_load_path": (_I, [_P, _P, _P, _P, _P, _P, _P, C.c_int32, C.c_int32,
                                  C.POINTER(SolveOpts), C.POINTER(Stats), C.POINTER(C.c_int32)]),
    "hofv_get_precision": (_I, [_P]),
    "hofv_selftest_barrier": (_I, [_P, C.POINTER(C.c_int32)]),
    "hofv_nej_apply": (_I, [_P, _P, _P]),
    "hofv_set_inertia": (_I, [_P, C.c_double, C.c_double, _I]),
    "hofv_set_history": (_I, [_P, _P, _P, _P, _P]),
    "hofv_bdf2_velocity": (_I, [_P, _P, _P, _P, _P]),
    "hofv_cell_average": (_I, [_P, _P, _P]),
    "hofv_mg_info": (_I, [_P, C.POINTER(C.c_int32), _P, C.c_int32, C.POINTER(C.c_int64),
                          C.POINTER(C.c_double)]),
    "hofv_gnn_init": (_I, [_P, C.c_uint64, _D]),
    "hofv_gnn_num_params": (_I, [_P, C.POINTER(_I64)]),
    "hofv_gnn_get_params": (_I, [_P, _P, _I64]),
    "hofv_gnn_set_params": (_I, [_P, _P, _I64]),
    "hofv_gnn_save": (_I, [_P, C.c_char_p]),
    "hofv_gnn_load": (_I, [_P, C.c_char_p]),
    "hofv_gnn_forward": (_I, [_P, _P, _P, _P]),
    "hofv_gnn_loss_grad": (_I, [_P, _P, _P, _P, C.POINTER(_D), _P]),
    "hofv_gnn_record": (_I, [_P, _P, _P]),
    "hofv_gnn_pairs": (_I, [_P, C.POINTER(C.c_int32)]),
    "hofv_gnn_clear_pairs": (_I, [_P]),
    "hofv_gnn_train": (_I, [_P, C.POINTER(TrainOpts), C.POINTER(TrainStats)]),
}


def load():
    """Load libhofv.so (no fallback: raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2601_18417_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _dev(t, dtype_name="float64"):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == f"torch.{dtype_name}"):
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor")
    return t


class Context:
    """One hofv context on a CUDA device and stream (torch's current stream
    unless given)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        L = load()
        self._L = L
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        rc = L.hofv_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise HofvError(rc, "hofv_create failed (no CUDA device?)")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self._L.hofv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow_warn=False):
        if rc < 0 or (rc > 0 and not allow_warn):
            raise HofvError(rc, self._L.hofv_last_error(self.h).decode())
        return rc

    # ---- set-up --------------------------------------------------------
    def set_mesh(self, mesh, bface_tag):
        """Quads / hexes, simplices (mesh.simplex), 2-D polygons (mesh.cell_ptr)
        or polyhedra given face by face (mesh.face_ptr; bface_tag then holds
        one tag per face, read on boundary faces)."""
        if hasattr(mesh, "face_ptr"):
            return self._set_mesh_faces(mesh, bface_tag)
        xyz = np.ascontiguousarray(mesh.xyz, np.float64)
        cn = np.ascontiguousarray(mesh.cell_nodes, np.int64)
        bn = np.ascontiguousarray(mesh.bface_nodes, np.int64)
        tag = np.ascontiguousarray(bface_tag, np.int32)
        self.dim = mesh.dim
        if getattr(mesh, "cell_ptr", None) is not None:  # 2-D polygons
            ptr = np.ascontiguousarray(mesh.cell_ptr, np.int64)
            self.faces_per_cell = POLY_SLOTS
            return self._check(self._L.hofv_set_mesh_polygons(
                self.h, xyz.shape[0], _ptr(xyz), ptr.shape[0] - 1, _ptr(ptr), _ptr(cn),
                bn.shape[0], _ptr(bn), _ptr(tag)))
        kind = CELL_SIMPLEX if getattr(mesh, "simplex", False) else CELL_TENSOR
        self.faces_per_cell = mesh.dim + 1 if kind == CELL_SIMPLEX else 2 * mesh.dim
        return self._check(self._L.hofv_set_mesh_cells(self.h, mesh.dim, kind, xyz.shape[0],
                                                       _ptr(xyz), cn.shape[0], _ptr(cn),
                                                       bn.shape[0], _ptr(bn), _ptr(tag)))

    def _set_mesh_faces(self, mesh, face_tag):
        xyz = np.ascontiguousarray(mesh.xyz, np.float64)
        ptr = np.ascontiguousarray(mesh.face_ptr, np.int64)
        fn = np.ascontiguousarray(mesh.face_nodes, np.int64)
        own = np.ascontiguousarray(mesh.owner, np.int64)
        nei = np.ascontiguousarray(mesh.neighbour, np.int64)
        tag = np.ascontiguousarray(face_tag, np.int32)
        self.dim = 3
        self.faces_per_cell = POLYHEDRON_SLOTS
        return self._check(self._L.hofv_set_mesh_faces(
            self.h, xyz.shape[0], _ptr(xyz), mesh.n_cells, ptr.shape[0] - 1, _ptr(ptr), _ptr(fn),
            _ptr(own), _ptr(nei), _ptr(tag)))

    def set_scheme(self, p, n_plus, q_per_dir, k_weight=6.0, alpha=0.1):
        return self._check(self._L.hofv_set_scheme(self.h, p, n_plus, q_per_dir, k_weight, alpha))

    def build_stencils(self):
        self._check(self._L.hofv_build_stencils(self.h))
        self.layout = self.get_layout()
        return self.layout

    def get_layout(self) -> Layout:
        lay = Layout()
        self._check(self._L.hofv_get_layout(self.h, C.byref(lay)))
        return lay

    def get_points(self, kind):
        lay = self.layout
        d = lay.dim
        shapes = {PTS_CELL_CENTROID: (lay.n_cells, d), PTS_DISP_QP: (lay.n_disp, lay.q_face, d),
                  PTS_DISP_CENTRE: (lay.n_disp, d), PTS_TRAC_QP: (lay.n_trac, lay.q_face, d),
                  PTS_CELL_QP: (lay.n_cells, lay.q_cell, d), PTS_FACE_CENTRE: (lay.n_faces, d),
                  PTS_FACE_QP: (lay.n_faces, lay.q_face, d),
                  PTS_FACE_AREA: (lay.n_faces, lay.q_face, d), PTS_CELL_VOLUME: (lay.n_cells,)}
        out = np.zeros(shapes[kind])
        self._check(self._L.hofv_get_points(self.h, kind, _ptr(out)))
        return out

    def set_material(self, law, mu, lam):
        return self._check(self._L.hofv_set_material(self.h, law, mu, lam))

    def nej_apply(self, x, y):
        """y = near-exact Jacobian times x (linear law)."""
        return self._check(self._L.hofv_nej_apply(self.h, _ptr(_dev(x)), _ptr(_dev(y))))

    # ---- dynamics (BDF2 inertia term) ------------------------------------
    def set_inertia(self, rho, dt, one_point=False):
        return self._check(self._L.hofv_set_inertia(self.h, rho, dt, int(bool(one_point))))

    def set_history(self, u_t, u_tm1=None, v_t=None, v_tm1=None):
        args = [_dev(t) for t in (u_t, u_tm1, v_t, v_tm1)]
        return self._check(self._L.hofv_set_history(self.h, *[_ptr(a) for a in args]))

    def bdf2_velocity(self, u_tp1, u_t, u_tm1, v_out):
        return self._check(self._L.hofv_bdf2_velocity(self.h, _ptr(_dev(u_tp1)), _ptr(_dev(u_t)),
                                                      _ptr(_dev(u_tm1)), _ptr(_dev(v_out))))

    def cell_average(self, u, ubar):
        return self._check(self._L.hofv_cell_average(self.h, _ptr(_dev(u)), _ptr(_dev(ubar))))

    def mg_info(self):
        """Multigrid hierarchy of PC_AJMG: level sizes, non-zeros, set-up s."""
        lv = C.c_int32(0)
        sizes = np.zeros(32, np.int64)
        nnz = C.c_int64(0)
        sec = C.c_double(0.0)
        self._check(self._L.hofv_mg_info(self.h, C.byref(lv), _ptr(sizes), sizes.size,
                                         C.byref(nnz), C.byref(sec)))
        return {"levels": lv.value, "sizes": sizes[: lv.value].tolist(), "nnz": nnz.value,
                "setup_s": sec.value}

    def selftest_barrier(self):
        t = C.c_int32(0)
        self._check(self._L.hofv_selftest_barrier(self.h, C.byref(t)))
        return bool(t.value)

    def set_contraction(self, on=True):
        return self._check(self._L.hofv_set_contraction(self.h, int(bool(on))))

    def set_precision(self, prec):
        """HOFV_PREC_FP64 or HOFV_PREC_DF64 for the gradient contraction."""
        return self._check(self._L.hofv_set_precision(self.h, int(prec)))

    def probe_peaks(self):
        """Measured FP64 / FP32 FMA throughput (TFLOP/s) and SM count."""
        d, f, n = C.c_double(), C.c_double(), C.c_int32()
        self._check(self._L.hofv_probe_peaks(self.h, C.byref(d), C.byref(f), C.byref(n)))
        return {"fp64_tflops": d.value, "fp32_tflops": f.value, "sm_count": n.value}

    def probe_inv_cbrt(self, J, r_own, r_lib):
        """The law's J^{-1/3} and CUDA's rcbrt of the device vector J."""
        self._check(self._L.hofv_probe_inv_cbrt(self.h, _ptr(_dev(J)), _ptr(_dev(r_own)),
                                                _ptr(_dev(r_lib)), int(J.numel())))

    @property
    def precision(self):
        rc = self._L.hofv_get_precision(self.h)
        if rc < 0:
            self._check(rc)
        return rc

    def set_bc(self, u_bq=None, u_bf=None, t_bq=None, body=None):
        args = [_dev(t) for t in (u_bq, u_bf, t_bq, body)]
        return self._check(self._L.hofv_set_bc(self.h, *[_ptr(a) for a in args]))

    def integrate_cells(self, f_qp, out):
        return self._check(self._L.hofv_integrate_cells(self.h, _ptr(_dev(f_qp)), _ptr(_dev(out))))

    # ---- evaluation ------------------------------------------------------
    def residual(self, u, R):
        return self._check(self._L.hofv_residual(self.h, _ptr(_dev(u)), _ptr(_dev(R))))

    def jvp(self, u, Ru, v, Jv, want_eps=False):
        eps = C.c_double(0.0)
        self._check(self._L.hofv_jvp(self.h, _ptr(_dev(u)), _ptr(_dev(Ru)), _ptr(_dev(v)),
                                     _ptr(_dev(Jv)), C.byref(eps) if want_eps else None))
        return eps.value if want_eps else None

    def precondition(self, kind, inner_iters, v, z):
        return self._check(self._L.hofv_precondition(self.h, kind, inner_iters, _ptr(_dev(v)),
                                                     _ptr(_dev(z))))

    def newton_solve(self, u, **opts):
        o = SolveOpts()
        self._L.hofv_default_opts(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        st = Stats()
        rc = self._L.hofv_newton_solve(self.h, _ptr(_dev(u)), C.byref(o), C.byref(st))
        self._check(rc, allow_warn=True)
        return st.as_dict()

    def prepare_solver(self, **opts):
        """Allocate and build up front what a solve with these options uses."""
        o = SolveOpts()
        self._L.hofv_default_opts(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        return self._check(self._L.hofv_prepare_solver(self.h, C.byref(o)))

    def solve_load_path(self, u, n_steps, u_bq1=None, u_bf1=None, t_bq1=None, body1=None,
                        du_dlambda=None, max_halvings=6, **opts):
        """hofv_solve_load_path; returns (stats dict, accepted increments)."""
        o = SolveOpts()
        self._L.hofv_default_opts(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        st = Stats()
        done = C.c_int32(0)
        args = [_ptr(_dev(a)) if a is not None else None
                for a in (u_bq1, u_bf1, t_bq1, body1, du_dlambda)]
        rc = self._L.hofv_solve_load_path(self.h, _ptr(_dev(u)), *args, int(n_steps),
                                          int(max_halvings), C.byref(o), C.byref(st),
                                          C.byref(done))
        self._check(rc, allow_warn=True)
        return st.as_dict(), done.value

    def set_stencils(self, face_stencils=None, cell_stencils=None):
        """Replace the stencils (HOST int32 [n_faces_with_stencil][S], [n_cells][S])."""
        f = None if face_stencils is None else np.ascontiguousarray(face_stencils, np.int32)
        c = None if cell_stencils is None else np.ascontiguousarray(cell_stencils, np.int32)
        return self._check(self._L.hofv_set_stencils(self.h, _ptr(f), _ptr(c)))

    def arnoldi_step(self, u, Ru, kind, inner_iters, V, Z, j):
        """One flexible Arnoldi step; V [(j+2), n], Z [(j+1), n] CUDA FP64.
        Returns the Hessenberg column (numpy, length j+2)."""
        h = np.zeros(j + 2)
        ld = V.stride(0)
        self._check(self._L.hofv_arnoldi_step(self.h, _ptr(_dev(u)), _ptr(_dev(Ru)), kind,
                                              inner_iters, _ptr(V), _ptr(Z), ld, j, _ptr(h)))
        return h

    def force_scale(self, u):
        """F_s = max over cells of the sum of |face flux| at state u."""
        fs = C.c_double(0.0)
        self._check(self._L.hofv_force_scale(self.h, _ptr(_dev(u)), C.byref(fs)))
        return fs.value

    def residual_noalloc(self, u, R):
        """hofv_residual through the variant that allocates nothing."""
        return self._check(self._L.hofv_residual_noalloc(self.h, _ptr(_dev(u)), _ptr(_dev(R))))

    def residual_timed(self, u, R):
        """Residual with per-kernel CUDA-event times (ms): u*, flux, cell."""
        ms = (C.c_float * 3)()
        self._check(self._L.hofv_residual_timed(self.h, _ptr(_dev(u)), _ptr(_dev(R)), ms))
        return [float(x) for x in ms]

    def jvp_timed(self, u, Ru, v, Jv):
        """Jacobian-vector product with per-kernel CUDA-event times (ms):
        extrapolation, flux, cell."""
        ms = (C.c_float * 3)()
        self._check(self._L.hofv_jvp_timed(self.h, _ptr(_dev(u)), _ptr(_dev(Ru)), _ptr(_dev(v)),
                                           _ptr(_dev(Jv)), ms))
        return [float(x) for x in ms]

    # ---- learned preconditioner -------------------------------------------
    def gnn_init(self, seed=0, out_scale=0.0):
        return self._check(self._L.hofv_gnn_init(self.h, seed, out_scale))

    def gnn_num_params(self):
        n = C.c_int64(0)
        self._check(self._L.hofv_gnn_num_params(self.h, C.byref(n)))
        return n.value

    def gnn_get_params(self):
        out = np.zeros(self.gnn_num_params(), np.float32)
        self._check(self._L.hofv_gnn_get_params(self.h, _ptr(out), out.size))
        return out

    def gnn_set_params(self, theta):
        theta = np.ascontiguousarray(theta, np.float32)
        return self._check(self._L.hofv_gnn_set_params(self.h, _ptr(theta), theta.size))

    def gnn_save(self, path):
        return self._check(self._L.hofv_gnn_save(self.h, str(path).encode()))

    def gnn_load(self, path):
        return self._check(self._L.hofv_gnn_load(self.h, str(path).encode()))

    def gnn_forward(self, v, z, zout):
        return self._check(self._L.hofv_gnn_forward(self.h, _ptr(_dev(v)), _ptr(_dev(z)),
                                                    _ptr(_dev(zout))))

    def gnn_loss_grad(self, v, z, delta):
        loss = C.c_double(0.0)
        g = np.zeros(self.gnn_num_params(), np.float32)
        self._check(self._L.hofv_gnn_loss_grad(self.h, _ptr(_dev(v)), _ptr(_dev(z)),
                                               _ptr(_dev(delta)), C.byref(loss), _ptr(g)))
        return loss.value, g

    def gnn_record(self, r, delta):
        return self._check(self._L.hofv_gnn_record(self.h, _ptr(_dev(r)), _ptr(_dev(delta))))

    def gnn_pairs(self):
        n = C.c_int32(0)
        self._check(self._L.hofv_gnn_pairs(self.h, C.byref(n)))
        return n.value

    def gnn_clear_pairs(self):
        return self._check(self._L.hofv_gnn_clear_pairs(self.h))

    def gnn_train(self, epochs=20, batch=4, lr=1e-3, inner_iters=20, seed=0, verbose=0):
        o = TrainOpts(epochs, batch, lr, inner_iters, seed, verbose)
        st = TrainStats()
        self._check(self._L.hofv_gnn_train(self.h, C.byref(o), C.byref(st)))
        return st.as_dict()

    # ---- inspection --------------------------------------------------------
    def get_face_data(self, first, count, coef=True):
        lay = self.layout
        st = np.zeros((count, lay.stencil), np.int32)
        co = np.zeros((count, lay.q_face, lay.stencil + 1, lay.dim)) if coef else None
        self._check(self._L.hofv_get_face_data(self.h, first, count, _ptr(st), _ptr(co)))
        return st, co

    def get_cell_data(self, first, count, ext=True):
        lay = self.layout
        st = np.zeros((count, lay.stencil), np.int32)
        ex = np.zeros((count, self.faces_per_cell, lay.stencil)) if ext else None
        self._check(self._L.hofv_get_cell_data(self.h, first, count, _ptr(st), _ptr(ex)))
        return st, ex

    def get_faces(self):
        n = self.layout.n_faces
        own = np.zeros(n, np.int64)
        nei = np.zeros(n, np.int64)
        lf = np.zeros(n, np.int32)
        tag = np.zeros(n, np.int32)
        self._check(self._L.hofv_get_faces(self.h, _ptr(own), _ptr(nei), _ptr(lf), _ptr(tag)))
        return own, nei, lf, tag

    def get_aj(self):
        lay = self.layout
        diag = np.zeros(lay.n_cells)
        off = np.zeros(max(lay.n_internal, 1))
        self._check(self._L.hofv_get_aj(self.h, _ptr(diag), _ptr(off)))
        return diag, off[: lay.n_internal]
