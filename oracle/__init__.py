"""Python access to the plain-C FP64 oracle (``hofv_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may load this module; the product path never does.  It
shares no code with the CUDA library.

Every function follows a passage of arXiv 2601.18417 (cited in the C source):
geometry and quadrature (Sec. 3.1-3.3), stencils (Sec. 3.5.2), least-squares
reconstruction (eqs. te-lsA, weightFunc), boundary ghost node (Sec. 3.5.3),
face gradients (eq. faceQuadGrad), laws (App. A), alpha stabilisation
(eqs. alpha, alphaJump, App. B), residual and approximate Jacobian (Sec. 4.1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hofv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, as the source asks)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P, I64, D = C.c_void_p, C.c_int64, C.c_double
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.c_int, I64, P, I64, P, I64, P, P]
        L.orc_create_cells.restype = P
        L.orc_create_cells.argtypes = [C.c_int, C.c_int, I64, P, I64, P, I64, P, P]
        L.orc_create_poly.restype = P
        L.orc_create_poly.argtypes = [I64, P, I64, P, P, I64, P, P]
        L.orc_create_faces.restype = P
        L.orc_create_faces.argtypes = [I64, P, I64, I64, P, P, P, P, P]
        L.orc_free.argtypes = [P]
        L.orc_counts.argtypes = [P, P]
        L.orc_set_scheme.argtypes = [P, C.c_int, C.c_int, C.c_int, D, D]
        L.orc_geometry.argtypes = [P]
        for n in ("xc", "vol", "xq", "aq", "xf", "nrm", "gam", "cqx", "cqw"):
            getattr(L, f"orc_get_{n}").argtypes = [P, P]
        L.orc_get_faces.argtypes = [P, P, P, P, P]
        L.orc_get_cell_faces.argtypes = [P, P]
        L.orc_href_exp.argtypes = [P]
        L.orc_nlf.argtypes = [P]
        L.orc_prepare.argtypes = [P, I64, P]
        L.orc_face_slot.argtypes = [P, I64]
        L.orc_cell_slot.argtypes = [P, I64]
        for n in ("face_stencil", "face_coef", "face_cond", "cell_stencil", "cell_ext"):
            getattr(L, f"orc_get_{n}").argtypes = [P, I64, P]
        L.orc_get_cell_cond.argtypes = [P, I64]
        L.orc_get_cell_cond.restype = D
        L.orc_reconstruct.argtypes = [P, P, P, C.c_int, P, P, P]
        L.orc_stencil.argtypes = [P, P, P]
        L.orc_stencil_bruteforce.argtypes = [P, P, P]
        L.orc_stress.argtypes = [C.c_int, D, D, P, P]
        L.orc_residual.argtypes = [P, C.c_int, D, D, P, P, P, P, P, I64, P, P]
        L.orc_face_fluxes.argtypes = [P, C.c_int, D, D, P, P, P, P, P]
        L.orc_integrate_cells.argtypes = [P, P, P]
        L.orc_aj.argtypes = [P, D, P, P]
        L.orc_gauss_legendre.argtypes = [C.c_int, P, P]
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def set_threads(n: int = 0) -> int:
    """OpenMP threads of the oracle's loops over cells and faces (0 = all
    cores); returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    x = np.zeros(8)
    w = np.zeros(8)
    if lib().orc_gauss_legendre(n, _p(x), _p(w)) != 0:
        raise ValueError("unsupported rule")
    return x[:n].copy(), w[:n].copy()


def stress(law: int, mu: float, lam: float, G: np.ndarray) -> np.ndarray:
    """Stress tensor T (traction t = T a) from G[i][j] = du_j/dx_i (3x3)."""
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(3, 3)
    T = np.zeros((3, 3))
    lib().orc_stress(law, mu, lam, _p(G), _p(T))
    return T


class OracleMesh:
    """One mesh + scheme in the oracle.  Arrays use the library's layouts."""

    def __init__(self, mesh, tags_per_side, p: int, n_plus: int, q1: int,
                 k_weight: float = 6.0, alpha: float = 0.1):
        L = lib()
        self.dim = mesh.dim
        self.mesh = mesh
        self.simplex = self.polygon = False
        self.polyhedral = hasattr(mesh, "face_ptr")
        if self.polyhedral:
            self._init_faces(L, mesh, tags_per_side)
            self._finish(L, p, n_plus, q1, k_weight, alpha)
            return
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        cn = np.ascontiguousarray(mesh.cell_nodes, dtype=np.int64)
        bn = np.ascontiguousarray(mesh.bface_nodes, dtype=np.int64)
        tags = np.ascontiguousarray(np.asarray(tags_per_side, np.int32)[mesh.bface_side])
        self.bface_tag = tags
        self._keep = (xyz, cn, bn, tags)
        self.simplex = bool(getattr(mesh, "simplex", False))
        self.polygon = getattr(mesh, "cell_ptr", None) is not None
        if self.polygon:
            ptr = np.ascontiguousarray(mesh.cell_ptr, dtype=np.int64)
            self._keep += (ptr,)
            self.h = L.orc_create_poly(xyz.shape[0], _p(xyz), ptr.shape[0] - 1, _p(ptr), _p(cn),
                                       bn.shape[0], _p(bn), _p(tags))
        else:
            self.h = L.orc_create_cells(self.dim, int(self.simplex), xyz.shape[0], _p(xyz),
                                        cn.shape[0], _p(cn), bn.shape[0], _p(bn), _p(tags))
        if not self.h:
            raise ValueError("oracle rejected the mesh")
        self._finish(L, p, n_plus, q1, k_weight, alpha)

    def _init_faces(self, L, mesh, tags_per_side):
        """A face-based polyhedral mesh (inputs.FaceMesh)."""
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        ptr = np.ascontiguousarray(mesh.face_ptr, dtype=np.int64)
        fn = np.ascontiguousarray(mesh.face_nodes, dtype=np.int64)
        own = np.ascontiguousarray(mesh.owner, dtype=np.int64)
        nei = np.ascontiguousarray(mesh.neighbour, dtype=np.int64)
        side = np.asarray(mesh.face_side)
        tags = np.ascontiguousarray(np.where(side >= 0, np.asarray(tags_per_side, np.int32)[
            np.maximum(side, 0)], -1).astype(np.int32))
        self.bface_tag = tags  # per input face, -1 inside
        self._keep = (xyz, ptr, fn, own, nei, tags)
        self.h = L.orc_create_faces(xyz.shape[0], _p(xyz), mesh.n_cells, ptr.shape[0] - 1,
                                    _p(ptr), _p(fn), _p(own), _p(nei), _p(tags))
        if not self.h:
            raise ValueError("oracle rejected the mesh")

    def _finish(self, L, p, n_plus, q1, k_weight, alpha):
        rc = L.orc_set_scheme(self.h, p, n_plus, q1, k_weight, alpha)
        if rc != 0:
            raise ValueError(f"oracle rejected the scheme ({rc})")
        if L.orc_geometry(self.h) != 0:
            raise RuntimeError("geometry failed")
        cnt = np.zeros(9, dtype=np.int64)
        L.orc_counts(self.h, _p(cnt))
        (self.nf, self.nfi, self.nfd, self.nft, self.nc, self.Q, self.S, self.QC, self.nfy) = (
            int(v) for v in cnt)
        self.p, self.n_plus, self.q1 = p, n_plus, q1
        # faces per cell; polygons keep 8 slots, -1 past a cell's last side,
        # polyhedra as many slots as the cell with most faces
        if self.polyhedral:
            self.nlf = int(L.orc_nlf(self.h))
        else:
            self.nlf = 8 if self.polygon else self.dim + 1 if self.simplex else 2 * self.dim
        self._subset = None

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_free(self.h)
            self.h = None

    # geometry ---------------------------------------------------------
    def _get(self, name, shape):
        out = np.zeros(shape)
        getattr(lib(), f"orc_get_{name}")(self.h, _p(out))
        return out

    @property
    def xc(self):
        return self._get("xc", (self.nc, 3))[:, : self.dim]

    @property
    def vol(self):
        return self._get("vol", (self.nc,))

    @property
    def xq(self):
        return self._get("xq", (self.nf, self.Q, 3))[..., : self.dim]

    @property
    def aq(self):
        return self._get("aq", (self.nf, self.Q, 3))[..., : self.dim]

    @property
    def xf(self):
        return self._get("xf", (self.nf, 3))[:, : self.dim]

    @property
    def normal(self):
        return self._get("nrm", (self.nf, 3))[:, : self.dim]

    @property
    def gamma(self):
        return self._get("gam", (self.nf,))

    @property
    def cell_qp(self):
        return self._get("cqx", (self.nc, self.QC, 3))[..., : self.dim]

    @property
    def cell_qw(self):
        return self._get("cqw", (self.nc, self.QC))

    def faces(self):
        own = np.zeros(self.nf, np.int64)
        nei = np.zeros(self.nf, np.int64)
        lf = np.zeros(self.nf, np.int32)
        tag = np.zeros(self.nf, np.int32)
        lib().orc_get_faces(self.h, _p(own), _p(nei), _p(lf), _p(tag))
        return own, nei, lf, tag

    def cell_faces(self):
        cf = np.zeros((self.nc, self.nlf), np.int64)
        lib().orc_get_cell_faces(self.h, _p(cf))
        return cf

    @property
    def href_exp(self) -> int:
        return int(lib().orc_href_exp(self.h))

    # stencils and coefficients ------------------------------------------
    def prepare(self, cells=None):
        if cells is None:
            rc = lib().orc_prepare(self.h, -1, None)
            self._subset = None
        else:
            cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
            rc = lib().orc_prepare(self.h, cells.shape[0], _p(cells))
            self._subset = cells
        if rc != 0:
            raise RuntimeError(f"oracle prepare failed ({rc})")

    def face_slot(self, f):
        return int(lib().orc_face_slot(self.h, int(f)))

    def cell_slot(self, c):
        return int(lib().orc_cell_slot(self.h, int(c)))

    def face_stencil(self, f):
        s = self.face_slot(f)
        out = np.zeros(self.S, np.int64)
        lib().orc_get_face_stencil(self.h, s, _p(out))
        return out

    def face_coef(self, f):
        """[Q][S+1][d] gradient coefficients; slot S is the ghost node."""
        s = self.face_slot(f)
        out = np.zeros((self.Q, self.S + 1, 3))
        lib().orc_get_face_coef(self.h, s, _p(out))
        return out[..., : self.dim]

    def face_cond(self, f):
        out = np.zeros(self.Q)
        lib().orc_get_face_cond(self.h, self.face_slot(f), _p(out))
        return out

    def cell_stencil(self, c):
        out = np.zeros(self.S, np.int64)
        lib().orc_get_cell_stencil(self.h, self.cell_slot(c), _p(out))
        return out

    def cell_ext(self, c):
        """[2d][S] weights e with u*_{f,P} = u_P + sum_N e_N u_N."""
        out = np.zeros((self.nlf, self.S))
        lib().orc_get_cell_ext(self.h, self.cell_slot(c), _p(out))
        return out

    def cell_cond(self, c):
        return float(lib().orc_get_cell_cond(self.h, self.cell_slot(c)))

    def reconstruct(self, xt, stencil, ghost=False):
        xt3 = np.zeros(3)
        xt3[: self.dim] = xt
        st = np.ascontiguousarray(np.asarray(stencil, np.int64))
        nt = self.S - self.n_plus
        A = np.zeros((nt, self.S + int(ghost)))
        h = np.zeros(1)
        cond = np.zeros(1)
        rc = lib().orc_reconstruct(self.h, _p(xt3), _p(st), int(ghost), _p(A), _p(h), _p(cond))
        if rc != 0:
            raise RuntimeError("singular reconstruction")
        return A, float(h[0]), float(cond[0])

    def stencil(self, xr, brute=False):
        xr3 = np.zeros(3)
        xr3[: self.dim] = xr
        out = np.zeros(self.S, np.int64)
        fn = lib().orc_stencil_bruteforce if brute else lib().orc_stencil
        if fn(self.h, _p(xr3), _p(out)) != 0:
            raise RuntimeError("stencil search failed")
        return out

    # residual -------------------------------------------------------------
    def residual(self, law, mu, lam, u, ubq=None, ubf=None, tbq=None, bsrc=None,
                 cells=None):
        """R [d][n] at `cells` (all cells if None).  u is [d][nc]."""
        d = self.dim
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(d, self.nc)
        ubq = np.ascontiguousarray(np.zeros((max(self.nfd, 1), self.Q, d)) if ubq is None else ubq, dtype=np.float64)
        ubf = np.ascontiguousarray(np.zeros((max(self.nfd, 1), d)) if ubf is None else ubf, dtype=np.float64)
        tbq = np.ascontiguousarray(np.zeros((max(self.nft, 1), self.Q, d)) if tbq is None else tbq, dtype=np.float64)
        b = None if bsrc is None else np.ascontiguousarray(bsrc, dtype=np.float64).reshape(d, self.nc)
        if cells is None:
            ns, cp = -1, None
            R = np.zeros((d, self.nc))
        else:
            cells = np.ascontiguousarray(np.asarray(cells, np.int64))
            ns, cp = cells.shape[0], cells
            R = np.zeros((d, ns))
        rc = lib().orc_residual(self.h, law, mu, lam, _p(u), _p(ubq), _p(ubf), _p(tbq),
                                _p(b), ns, _p(cp), _p(R))
        if rc != 0:
            raise RuntimeError("residual requested at unprepared cells")
        return R

    def face_fluxes(self, law, mu, lam, u, ubq=None, ubf=None, tbq=None):
        d = self.dim
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(d, self.nc)
        ubq = np.ascontiguousarray(np.zeros((max(self.nfd, 1), self.Q, d)) if ubq is None else ubq, dtype=np.float64)
        ubf = np.ascontiguousarray(np.zeros((max(self.nfd, 1), d)) if ubf is None else ubf, dtype=np.float64)
        tbq = np.ascontiguousarray(np.zeros((max(self.nft, 1), self.Q, d)) if tbq is None else tbq, dtype=np.float64)
        out = np.zeros((self.nf, 3))
        lib().orc_face_fluxes(self.h, law, mu, lam, _p(u), _p(ubq), _p(ubf), _p(tbq), _p(out))
        return out[:, :d]

    def integrate_cells(self, fq):
        """fq [nc][QC][d] -> [d][nc]"""
        fq = np.ascontiguousarray(fq, dtype=np.float64)
        b = np.zeros((self.dim, self.nc))
        lib().orc_integrate_cells(self.h, _p(fq), _p(b))
        return b

    def aj(self, kbar):
        diag = np.zeros(self.nc)
        off = np.zeros(max(self.nfi, 1))
        lib().orc_aj(self.h, kbar, _p(diag), _p(off))
        return diag, off[: self.nfi]

    def aj_matrix(self, kbar):
        """The scalar approximate Jacobian as a scipy CSR matrix."""
        import scipy.sparse as sp
        diag, off = self.aj(kbar)
        own, nei, _, _ = self.faces()
        i = np.concatenate([np.arange(self.nc), own[: self.nfi], nei[: self.nfi]])
        j = np.concatenate([np.arange(self.nc), nei[: self.nfi], own[: self.nfi]])
        v = np.concatenate([diag, off, off])
        return sp.csr_matrix((v, (i, j)), shape=(self.nc, self.nc))

    # boundary data helpers -------------------------------------------------
    def disp_faces(self):
        return np.arange(self.nfi, self.nfi + self.nfd)

    def symm_faces(self):
        return np.arange(self.nfi + self.nfd, self.nfi + self.nfd + self.nfy)

    def trac_faces(self):
        return np.arange(self.nfi + self.nfd + self.nfy, self.nf)
