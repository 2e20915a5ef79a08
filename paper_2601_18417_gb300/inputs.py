"""Seeded synthetic inputs: meshes, manufactured fields and random vectors.

This module holds no arithmetic of the finite-volume method itself.  It builds
structured quad/hex meshes (optionally with seeded interior-node jitter), the
triangle / tetrahedron meshes cut from them, their polygonal duals and those
duals extruded into polyhedra,
evaluates closed-form displacement fields together with their exact
derivatives and the matching body force of linear elasticity, and draws
seeded random vectors.  Both the CUDA path and the oracle consume these inputs;
neither imports the other.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: value i of stream s is splitmix64(seed_mix(s) + i * golden_gamma).

Workloads follow the paper's manufactured-solution case (Section 5.1.1, Case 1)
and the block-compression loading used for the neo-Hookean runs; the dataclass
``Workload`` records each one's mesh, order and material.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied to 64-bit counters (vectorised)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from counter-based SplitMix64 (53 high bits)."""
    base = splitmix64(np.array([seed * 1_000_003 + stream], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        ctr = base + np.arange(n, dtype=np.uint64) * _GAMMA
    bits = splitmix64(ctr) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n standard normal doubles (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, n, 2 * stream + 1)
    u2 = uniform(seed, n, 2 * stream + 2)
    u1 = np.maximum(u1, 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Mesh:
    """Unstructured description of a grid of quads (d=2) or hexes (d=3), or
    of triangles / tetrahedra (simplex=True) on the same nodes.

    xyz          [n_nodes, d] node coordinates
    cell_nodes   [n_cells, 2**d] node ids; quads counter-clockwise, hexes with
                 the bottom face (z-) counter-clockwise seen from +z, then top;
                 simplex meshes: [n_cells, d+1], triangles counter-clockwise,
                 tetrahedra positively oriented
    bface_nodes  [n_bfaces, 2**(d-1)] (simplex: [n_bfaces, d]) node ids of
                 boundary faces, outward order
    bface_side   [n_bfaces] domain side: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+
    cell_ptr     polygon meshes (d = 2) only: [n_cells + 1] offsets into the
                 flat cell_nodes, each polygon counter-clockwise
    """

    dim: int
    n: int
    xyz: np.ndarray
    cell_nodes: np.ndarray
    bface_nodes: np.ndarray
    bface_side: np.ndarray
    length: float = 1.0
    simplex: bool = False
    cell_ptr: np.ndarray | None = None   # polygon meshes: cell c is cell_nodes[ptr[c]:ptr[c+1]]

    @property
    def n_cells(self) -> int:
        if self.cell_ptr is not None:
            return int(self.cell_ptr.shape[0] - 1)
        return int(self.cell_nodes.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])


def structured_mesh(dim: int, n: int, length: float = 1.0, jitter: float = 0.0,
                    seed: int = 0) -> Mesh:
    """n^d cells on [0, length]^d; interior nodes moved by U(-jitter*h, jitter*h)
    per coordinate, boundary nodes fixed (boundary-normal motion would change
    the domain; tangential motion of boundary nodes is also left out)."""
    h = length / n
    m = n + 1
    if dim == 2:
        j, i = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        xyz = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
        nid = lambda i, j: i + m * j  # noqa: E731
        cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        ci, cj = ci.ravel(), cj.ravel()
        cell_nodes = np.stack([nid(ci, cj), nid(ci + 1, cj), nid(ci + 1, cj + 1),
                               nid(ci, cj + 1)], axis=1)
        interior = (i.ravel() > 0) & (i.ravel() < n) & (j.ravel() > 0) & (j.ravel() < n)
        r = np.arange(n)
        faces, sides = [], []
        # x- (i=0): outward order (0,3) -> nodes (0,j+1),(0,j)
        faces.append(np.stack([nid(0, r + 1), nid(0, r)], 1)); sides.append(np.full(n, 0))
        faces.append(np.stack([nid(n, r), nid(n, r + 1)], 1)); sides.append(np.full(n, 1))
        faces.append(np.stack([nid(r, 0), nid(r + 1, 0)], 1)); sides.append(np.full(n, 2))
        faces.append(np.stack([nid(r + 1, n), nid(r, n)], 1)); sides.append(np.full(n, 3))
    elif dim == 3:
        k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
        xyz = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)
        nid = lambda i, j, k: i + m * (j + m * k)  # noqa: E731
        ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
        cell_nodes = np.stack([
            nid(ci, cj, ck), nid(ci + 1, cj, ck), nid(ci + 1, cj + 1, ck), nid(ci, cj + 1, ck),
            nid(ci, cj, ck + 1), nid(ci + 1, cj, ck + 1), nid(ci + 1, cj + 1, ck + 1),
            nid(ci, cj + 1, ck + 1)], axis=1)
        iv, jv, kv = i.ravel(), j.ravel(), k.ravel()
        interior = ((iv > 0) & (iv < n) & (jv > 0) & (jv < n) & (kv > 0) & (kv < n))
        b, a = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        a, b = a.ravel(), b.ravel()
        faces, sides = [], []
        nf = n * n
        # outward node orders mirror the hex's local faces
        faces.append(np.stack([nid(0, a, b), nid(0, a, b + 1), nid(0, a + 1, b + 1), nid(0, a + 1, b)], 1)); sides.append(np.full(nf, 0))
        faces.append(np.stack([nid(n, a, b), nid(n, a + 1, b), nid(n, a + 1, b + 1), nid(n, a, b + 1)], 1)); sides.append(np.full(nf, 1))
        faces.append(np.stack([nid(a, 0, b), nid(a + 1, 0, b), nid(a + 1, 0, b + 1), nid(a, 0, b + 1)], 1)); sides.append(np.full(nf, 2))
        faces.append(np.stack([nid(a, n, b), nid(a, n, b + 1), nid(a + 1, n, b + 1), nid(a + 1, n, b)], 1)); sides.append(np.full(nf, 3))
        faces.append(np.stack([nid(a, b, 0), nid(a, b + 1, 0), nid(a + 1, b + 1, 0), nid(a + 1, b, 0)], 1)); sides.append(np.full(nf, 4))
        faces.append(np.stack([nid(a, b, n), nid(a + 1, b, n), nid(a + 1, b + 1, n), nid(a, b + 1, n)], 1)); sides.append(np.full(nf, 5))
    else:
        raise ValueError("dim must be 2 or 3")
    if jitter > 0.0:
        nn = xyz.shape[0]
        shift = (2.0 * uniform(seed, nn * dim, stream=7) - 1.0).reshape(nn, dim) * (jitter * h)
        xyz = xyz + np.where(interior[:, None], shift, 0.0)
    return Mesh(dim=dim, n=n, xyz=np.ascontiguousarray(xyz),
                cell_nodes=np.ascontiguousarray(cell_nodes.astype(np.int64)),
                bface_nodes=np.ascontiguousarray(np.concatenate(faces).astype(np.int64)),
                bface_side=np.concatenate(sides).astype(np.int32), length=length)


# local faces of a triangle / tetrahedron in outward node order (a
# tetrahedron's face k lies opposite its node 3 - k)
SIMPLEX_LOCAL_FACES = {2: ((0, 1), (1, 2), (2, 0)),
                       3: ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))}


def _signed_measure(xyz: np.ndarray, cells: np.ndarray) -> np.ndarray:
    x0 = xyz[cells[:, 0]]
    E = np.stack([xyz[cells[:, k]] - x0 for k in range(1, cells.shape[1])], axis=1)
    return np.linalg.det(E)


def simplex_mesh(dim: int, n: int, length: float = 1.0, jitter: float = 0.0,
                 seed: int = 0) -> Mesh:
    """Triangles (2 n^2) or tetrahedra (6 n^3) on the nodes of
    structured_mesh(dim, n, length, jitter, seed).  Each square is cut along
    one of its diagonals, picked by a seeded coin per square; each cube is cut
    into the six tetrahedra of its Kuhn (Freudenthal) subdivision, the paths
    from its (0,0,0) corner to its (1,1,1) corner along the edges, which
    meet conformingly across neighbouring cubes.  Every cell is positively
    oriented (raises if the jitter inverted one); boundary faces are the cell
    faces that no other cell shares, ordered by domain side and then by cell,
    in outward order."""
    base = structured_mesh(dim, n, length, jitter, seed)
    cn = base.cell_nodes
    if dim == 2:
        flip = uniform(seed, cn.shape[0], stream=11) < 0.5
        t0 = np.where(flip[:, None], cn[:, [0, 1, 3]], cn[:, [0, 1, 2]])
        t1 = np.where(flip[:, None], cn[:, [1, 2, 3]], cn[:, [0, 2, 3]])
        cells = np.stack([t0, t1], axis=1).reshape(-1, 3)
    elif dim == 3:
        corner = {(0, 0, 0): 0, (1, 0, 0): 1, (1, 1, 0): 2, (0, 1, 0): 3,
                  (0, 0, 1): 4, (1, 0, 1): 5, (1, 1, 1): 6, (0, 1, 1): 7}
        paths = []
        for perm in itertools.permutations(range(3)):
            r = [0, 0, 0]
            path = [corner[tuple(r)]]
            for ax in perm:
                r[ax] = 1
                path.append(corner[tuple(r)])
            paths.append(path)
        cells = cn[:, paths].reshape(-1, 4)
    else:
        raise ValueError("dim must be 2 or 3")
    # orientation from the unjittered grid, then checked on the jittered one
    grid = structured_mesh(dim, n, length, 0.0, seed).xyz
    neg = _signed_measure(grid, cells) < 0
    cells[neg, 1], cells[neg, 2] = cells[neg, 2].copy(), cells[neg, 1].copy()
    if np.any(_signed_measure(base.xyz, cells) <= 0):
        raise ValueError("jitter inverted a simplex; lower it")
    # boundary faces: local faces met once
    lfs = np.asarray(SIMPLEX_LOCAL_FACES[dim])
    fn = cells[:, lfs]                                   # [nc, d+1, d]
    keys = np.sort(fn, axis=2).reshape(-1, dim)
    _, inv, cnt = np.unique(keys, axis=0, return_inverse=True, return_counts=True)
    once = cnt[inv.ravel()] == 1
    bnodes = fn.reshape(-1, dim)[once]
    m = n + 1
    ijk = np.stack([(bnodes // m ** a) % m for a in range(dim)], axis=-1)   # [nb, d, dim]
    side = np.full(bnodes.shape[0], -1, np.int64)
    for a in range(dim):
        side = np.where(np.all(ijk[:, :, a] == 0, axis=1), 2 * a, side)
        side = np.where(np.all(ijk[:, :, a] == n, axis=1), 2 * a + 1, side)
    if np.any(side < 0):
        raise AssertionError("boundary face off the domain sides")
    order = np.argsort(side, kind="stable")
    return Mesh(dim=dim, n=n, xyz=base.xyz, cell_nodes=np.ascontiguousarray(cells.astype(np.int64)),
                bface_nodes=np.ascontiguousarray(bnodes[order].astype(np.int64)),
                bface_side=side[order].astype(np.int32), length=length, simplex=True)


def polygon_mesh(n: int, length: float = 1.0, jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Polygonal cells: the dual of simplex_mesh(2, n, ...), built the way a
    dual mesh generator builds it.  Each node of the triangle mesh becomes a
    cell whose corners are the centroids of its triangles, in turn around
    it; a node on the boundary also keeps itself and the midpoints of its two
    boundary edges as corners, so the dual covers the square exactly.
    Interior cells have 4 to 8 sides (one per triangle at the node).  Every
    fan triangle from a cell's vertex average to one of its sides is checked
    to be positively oriented (raises otherwise)."""
    tri = simplex_mesh(2, n, length, jitter, seed)
    X, T = tri.xyz, tri.cell_nodes
    nn, nt = X.shape[0], T.shape[0]
    cent = X[T].mean(axis=1)
    bn = tri.bface_nodes                          # [nb, 2], outward (counter-clockwise)
    nbe = bn.shape[0]
    mid = 0.5 * (X[bn[:, 0]] + X[bn[:, 1]])
    bnodes = np.unique(bn.ravel())
    # dual node ids: triangle centroids, boundary-edge midpoints, boundary nodes
    mid0, bn0 = nt, nt + nbe
    bnode_id = np.full(nn, -1, np.int64)
    bnode_id[bnodes] = bn0 + np.arange(bnodes.size)
    xyz = np.concatenate([cent, mid, X[bnodes]])
    # (cell = triangle-mesh node, corner = dual node) pairs
    node = np.concatenate([T.ravel(), bn[:, 0], bn[:, 1], bnodes])
    corner = np.concatenate([np.repeat(np.arange(nt), 3), mid0 + np.arange(nbe),
                             mid0 + np.arange(nbe), bnode_id[bnodes]])
    cnt = np.bincount(node, minlength=nn)
    c = np.stack([np.bincount(node, weights=xyz[corner, a], minlength=nn) for a in range(2)],
                 axis=1) / cnt[:, None]
    d = xyz[corner] - c[node]
    order = np.lexsort((np.arctan2(d[:, 1], d[:, 0]), node))
    flat = corner[order].astype(np.int64)
    ptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    # star-shaped about the corners' average, counter-clockwise
    nxt = np.arange(flat.size) + 1
    nxt[ptr[1:] - 1] = ptr[:-1]
    own = np.repeat(np.arange(nn), cnt)
    e0 = xyz[flat] - c[own]
    e1 = xyz[flat[nxt]] - c[own]
    if np.any(e0[:, 0] * e1[:, 1] - e0[:, 1] * e1[:, 0] <= 0):
        raise ValueError("a dual cell is not star-shaped about its vertex average")
    # boundary faces: the halves of each boundary edge, (a, mid) for cell a and
    # (mid, b) for cell b, on the edge's domain side
    e = np.arange(nbe)
    faces = np.stack([np.stack([bnode_id[bn[:, 0]], mid0 + e], axis=1),
                      np.stack([mid0 + e, bnode_id[bn[:, 1]]], axis=1)], axis=1).reshape(-1, 2)
    sides = np.repeat(tri.bface_side, 2)
    return Mesh(dim=2, n=n, xyz=np.ascontiguousarray(xyz), cell_nodes=flat,
                bface_nodes=faces.astype(np.int64), bface_side=sides.astype(np.int32),
                length=length, cell_ptr=ptr)


@dataclasses.dataclass
class FaceMesh:
    """Face-based description of a 3-D polyhedral mesh (the layout of a
    polyMesh): every face once, as a polygon whose normal by the right-hand
    rule points out of its owner.

    xyz         [n_nodes, 3]
    face_ptr    [n_faces + 1] offsets into face_nodes (3 to 8 corners a face)
    face_nodes  flat corner lists
    owner       [n_faces] owning cell; neighbour [n_faces], -1 on the boundary
    face_side   [n_faces] domain side 0..5 of a boundary face, -1 inside
    cell_grid   [n_cells, 3] integer position of each cell in its generator's
                grid (used to colour cells, not by the method)
    """

    dim: int
    n: int
    xyz: np.ndarray
    face_ptr: np.ndarray
    face_nodes: np.ndarray
    owner: np.ndarray
    neighbour: np.ndarray
    face_side: np.ndarray
    n_cells: int
    cell_grid: np.ndarray
    length: float = 1.0

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])


def prism_mesh(n: int, nz: int | None = None, length: float = 1.0, jitter: float = 0.0,
               seed: int = 0) -> FaceMesh:
    """Polyhedra: the dual polygons of polygon_mesh(n, ...) extruded through
    nz layers of the cube [0, length]^3.  A cell has its polygon (4 to 8
    corners) as bottom and top face and one quadrilateral per side; interior
    node levels move by U(-jitter, jitter) of the layer height, so top,
    bottom and side faces are not planar.  Faces are listed bottom to top:
    the horizontal faces of each level, then the side faces of each layer;
    an internal face is owned by the lower cell id."""
    nz = n if nz is None else nz
    base = polygon_mesh(n, length, jitter, seed)
    P2, ptr2, cn2 = base.xyz, base.cell_ptr, base.cell_nodes
    np2, nc2 = P2.shape[0], ptr2.shape[0] - 1
    hz = length / nz
    z = np.tile((np.arange(nz + 1) * hz)[:, None], (1, np2))
    if jitter > 0.0:
        dz = (2.0 * uniform(seed, (nz + 1) * np2, stream=13) - 1.0).reshape(nz + 1, np2)
        z[1:nz] += jitter * hz * dz[1:nz]
    xyz = np.concatenate([np.concatenate([P2, z[k][:, None]], axis=1) for k in range(nz + 1)])
    nid = lambda p, k: k * np2 + p  # noqa: E731
    cid = lambda c, k: k * nc2 + c  # noqa: E731
    # 2-D edges with the cells on their left (counter-clockwise) and right
    edge_left = {}
    for c in range(nc2):
        cs = cn2[ptr2[c]:ptr2[c + 1]]
        for j in range(cs.size):
            edge_left[(int(cs[j]), int(cs[(j + 1) % cs.size]))] = c
    side_of = {}
    for (a, b), sd in zip(map(tuple, base.bface_nodes), base.bface_side):
        side_of[(int(a), int(b))] = int(sd)
    faces, own, nei, side = [], [], [], []

    def add(nodes, o, nb, sd):
        if nb >= 0 and nb < o:  # owner is the lower id: flip the face
            o, nb = nb, o
            nodes = nodes[::-1]
        faces.append(np.asarray(nodes, np.int64))
        own.append(o)
        nei.append(nb)
        side.append(sd)

    for k in range(nz + 1):          # horizontal faces, normal +z out of the lower cell
        for c in range(nc2):
            cs = [nid(int(p), k) for p in cn2[ptr2[c]:ptr2[c + 1]]]
            if k == 0:
                add(cs[::-1], cid(c, 0), -1, 4)
            elif k == nz:
                add(cs, cid(c, nz - 1), -1, 5)
            else:
                add(cs, cid(c, k - 1), cid(c, k), -1)
    for k in range(nz):              # side faces, out of the cell on the edge's left
        for (a, b), c in edge_left.items():
            quad = [nid(a, k), nid(b, k), nid(b, k + 1), nid(a, k + 1)]
            other = edge_left.get((b, a), -1)
            if other >= 0:
                if c < other:
                    add(quad, cid(c, k), cid(other, k), -1)
            else:
                add(quad, cid(c, k), -1, side_of[(a, b)])
    fptr = np.concatenate([[0], np.cumsum([f.size for f in faces])]).astype(np.int64)
    grid = np.stack([np.tile(np.arange(nc2) % (n + 1), nz), np.tile(np.arange(nc2) // (n + 1), nz),
                     np.repeat(np.arange(nz), nc2)], axis=1).astype(np.int64)
    return FaceMesh(dim=3, n=n, xyz=np.ascontiguousarray(xyz), face_ptr=fptr,
                    face_nodes=np.concatenate(faces), owner=np.asarray(own, np.int64),
                    neighbour=np.asarray(nei, np.int64), face_side=np.asarray(side, np.int32),
                    n_cells=nc2 * nz, cell_grid=grid, length=length)


# outward corner order of each local face of a hex (nodes 0-3 the bottom,
# counter-clockwise seen from +z, 4-7 the top): x-, x+, y-, y+, z-, z+
_HEX_FACES = ((0, 4, 7, 3), (1, 2, 6, 5), (0, 1, 5, 4), (3, 7, 6, 2), (0, 3, 2, 1), (4, 5, 6, 7))


def hex_face_mesh(n: int, length: float = 1.0, jitter: float = 0.0, seed: int = 0) -> FaceMesh:
    """structured_mesh(3, n, ...) described face by face: every hex face a
    quadrilateral polygon, owned by the lower cell id, listed in the order
    cells and their local faces first meet it; boundary faces keep their
    domain side."""
    base = structured_mesh(3, n, length, jitter, seed)
    cn = base.cell_nodes
    seen = {}
    faces, own, nei, side = [], [], [], []
    for c in range(cn.shape[0]):
        for lf, loc in enumerate(_HEX_FACES):
            nodes = [int(cn[c, k]) for k in loc]
            key = tuple(sorted(nodes))
            if key in seen:
                nei[seen[key]] = c
                continue
            seen[key] = len(faces)
            faces.append(np.asarray(nodes, np.int64))
            own.append(c)
            nei.append(-1)
            side.append(lf)
    nei = np.asarray(nei, np.int64)
    side = np.where(nei >= 0, -1, np.asarray(side)).astype(np.int32)
    fptr = np.arange(len(faces) + 1, dtype=np.int64) * 4
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    grid = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1).astype(np.int64)
    return FaceMesh(dim=3, n=n, xyz=base.xyz, face_ptr=fptr, face_nodes=np.concatenate(faces),
                    owner=np.asarray(own, np.int64), neighbour=nei, face_side=side,
                    n_cells=cn.shape[0], cell_grid=grid, length=length)


def make_mesh(dim: int, n: int, length: float = 1.0, jitter: float = 0.0, seed: int = 0,
              cells: str = "tensor") -> Mesh:
    """structured_mesh (cells="tensor"), simplex_mesh (cells="simplex"), in
    2-D polygon_mesh (cells="polygon", (n + 1)^2 cells), in 3-D prism_mesh
    (cells="polyhedron", (n + 1)^2 n cells) and hex_face_mesh (cells="hexfaces",
    n^3 hexes given face by face)."""
    if cells == "simplex":
        return simplex_mesh(dim, n, length, jitter, seed)
    if cells == "polygon":
        if dim != 2:
            raise ValueError("polygon meshes are two-dimensional")
        return polygon_mesh(n, length, jitter, seed)
    if cells == "polyhedron":
        if dim != 3:
            raise ValueError("polyhedral meshes are three-dimensional")
        return prism_mesh(n, n, length, jitter, seed)
    if cells == "hexfaces":
        if dim != 3:
            raise ValueError("hexes given face by face are three-dimensional")
        return hex_face_mesh(n, length, jitter, seed)
    if cells != "tensor":
        raise ValueError("cells must be 'tensor', 'simplex', 'polygon', 'polyhedron' or 'hexfaces'")
    return structured_mesh(dim, n, length, jitter, seed)


# --------------------------------------------------------------------------
# material constants
# --------------------------------------------------------------------------

def lame_from_young(E: float, nu: float) -> tuple[float, float]:
    """(mu, lambda) from Young's modulus and Poisson's ratio (Appendix A)."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


# --------------------------------------------------------------------------
# closed-form displacement fields: value, gradient, Hessian
# grad[..., i, j] = d u_j / d x_i ; hess[..., j, a, b] = d^2 u_j / dx_a dx_b
# --------------------------------------------------------------------------

class Field:
    dim: int

    def value(self, x):  # pragma: no cover - interface
        raise NotImplementedError

    def grad(self, x):  # pragma: no cover
        raise NotImplementedError

    def hess(self, x):  # pragma: no cover
        raise NotImplementedError

    def body_force(self, x, mu, lam):
        """f_b = -div(sigma(u)) for linear elasticity:
        -(mu * lap(u) + (mu + lam) * grad(div u))."""
        H = self.hess(x)
        lap = np.einsum("...jaa->...j", H)
        grad_div = np.einsum("...iji->...j", H)
        return -(mu * lap + (mu + lam) * grad_div)


class Trig2D(Field):
    """u = a sin(4 pi x) sin(2 pi y): the paper's 3-D trigonometric field
    (Case 1) with the z factor dropped, a = (2, 4) micrometres."""
    dim = 2

    def __init__(self, a=(2e-6, 4e-6)):
        self.a = np.asarray(a, dtype=np.float64)

    def _parts(self, x):
        X, Y = x[..., 0], x[..., 1]
        kx, ky = 4 * math.pi, 2 * math.pi
        return X, Y, kx, ky

    def value(self, x):
        X, Y, kx, ky = self._parts(x)
        s = np.sin(kx * X) * np.sin(ky * Y)
        return s[..., None] * self.a

    def grad(self, x):
        X, Y, kx, ky = self._parts(x)
        dx = kx * np.cos(kx * X) * np.sin(ky * Y)
        dy = ky * np.sin(kx * X) * np.cos(ky * Y)
        g = np.stack([dx, dy], axis=-1)  # d s / d x_i
        return g[..., :, None] * self.a[None, :]

    def hess(self, x):
        X, Y, kx, ky = self._parts(x)
        sxx = -kx * kx * np.sin(kx * X) * np.sin(ky * Y)
        syy = -ky * ky * np.sin(kx * X) * np.sin(ky * Y)
        sxy = kx * ky * np.cos(kx * X) * np.cos(ky * Y)
        Hs = np.stack([np.stack([sxx, sxy], -1), np.stack([sxy, syy], -1)], -2)
        return self.a[:, None, None] * Hs[..., None, :, :]


class Mixed2D(Field):
    """The paper's 2-D manufactured field (Case 1):
    u_x = exp(x^2) sin(y),  u_y = ln(3 + y) cos(x) + sin(y)."""
    dim = 2

    def value(self, x):
        X, Y = x[..., 0], x[..., 1]
        return np.stack([np.exp(X * X) * np.sin(Y),
                         np.log(3 + Y) * np.cos(X) + np.sin(Y)], axis=-1)

    def grad(self, x):
        X, Y = x[..., 0], x[..., 1]
        e = np.exp(X * X)
        dux_dx = 2 * X * e * np.sin(Y)
        dux_dy = e * np.cos(Y)
        duy_dx = -np.log(3 + Y) * np.sin(X)
        duy_dy = np.cos(X) / (3 + Y) + np.cos(Y)
        g = np.empty(x.shape[:-1] + (2, 2))
        g[..., 0, 0], g[..., 1, 0] = dux_dx, dux_dy
        g[..., 0, 1], g[..., 1, 1] = duy_dx, duy_dy
        return g

    def hess(self, x):
        X, Y = x[..., 0], x[..., 1]
        e = np.exp(X * X)
        H = np.empty(x.shape[:-1] + (2, 2, 2))
        H[..., 0, 0, 0] = (2 + 4 * X * X) * e * np.sin(Y)
        H[..., 0, 0, 1] = H[..., 0, 1, 0] = 2 * X * e * np.cos(Y)
        H[..., 0, 1, 1] = -e * np.sin(Y)
        H[..., 1, 0, 0] = -np.log(3 + Y) * np.cos(X)
        H[..., 1, 0, 1] = H[..., 1, 1, 0] = -np.sin(X) / (3 + Y)
        H[..., 1, 1, 1] = -np.cos(X) / (3 + Y) ** 2 - np.sin(Y)
        return H


class Trig3D(Field):
    """The paper's 3-D manufactured field (Case 1):
    u = a sin(4 pi x) sin(2 pi y) sin(pi z), a = (2, 4, 6) micrometres."""
    dim = 3

    def __init__(self, a=(2e-6, 4e-6, 6e-6)):
        self.a = np.asarray(a, dtype=np.float64)
        self.k = np.array([4 * math.pi, 2 * math.pi, math.pi])

    def _sc(self, x):
        s = np.sin(self.k * x)
        c = np.cos(self.k * x)
        return s, c

    def value(self, x):
        s, _ = self._sc(x)
        return np.prod(s, axis=-1)[..., None] * self.a

    def grad(self, x):
        s, c = self._sc(x)
        k = self.k
        g = np.stack([k[0] * c[..., 0] * s[..., 1] * s[..., 2],
                      k[1] * s[..., 0] * c[..., 1] * s[..., 2],
                      k[2] * s[..., 0] * s[..., 1] * c[..., 2]], axis=-1)
        return g[..., :, None] * self.a

    def hess(self, x):
        s, c = self._sc(x)
        k = self.k
        Hs = np.empty(x.shape[:-1] + (3, 3))
        for a_ in range(3):
            for b_ in range(3):
                f = np.ones(x.shape[:-1])
                for m in range(3):
                    if m == a_ and m == b_:
                        f = f * (-k[m] * k[m] * s[..., m])
                    elif m == a_ or m == b_:
                        f = f * (k[m] * c[..., m])
                    else:
                        f = f * s[..., m]
                Hs[..., a_, b_] = f
        return self.a[:, None, None] * Hs[..., None, :, :]


def monomial_exponents(dim: int, p: int) -> list[tuple[int, ...]]:
    """Exponent tuples of all monomials of total degree <= p, graded order."""
    out = []
    for deg in range(p + 1):
        if dim == 2:
            for a in range(deg, -1, -1):
                out.append((a, deg - a))
        else:
            for a in range(deg, -1, -1):
                for b in range(deg - a, -1, -1):
                    out.append((a, b, deg - a - b))
    return out


class Polynomial(Field):
    """Vector polynomial field with seeded coefficients of total degree <= p.
    coef[m, j] multiplies monomial m in component j."""

    def __init__(self, dim: int, p: int, seed: int = 0, scale: float = 1.0,
                 center=None):
        self.dim = dim
        self.exps = monomial_exponents(dim, p)
        self.coef = (2.0 * uniform(seed, len(self.exps) * dim, stream=11) - 1.0).reshape(
            len(self.exps), dim) * scale
        self.center = np.zeros(dim) if center is None else np.asarray(center, float)

    def _mono(self, x, deriv):
        y = x - self.center
        out = []
        for e in self.exps:
            f = np.ones(x.shape[:-1])
            for ax in range(self.dim):
                n_d = deriv.count(ax)
                ee = e[ax]
                if n_d > ee:
                    f = f * 0.0
                    continue
                fac = 1.0
                for t in range(n_d):
                    fac *= (ee - t)
                f = f * fac * y[..., ax] ** (ee - n_d)
            out.append(f)
        return np.stack(out, axis=-1)

    def value(self, x):
        return self._mono(x, ()) @ self.coef

    def grad(self, x):
        return np.stack([self._mono(x, (i,)) @ self.coef for i in range(self.dim)], axis=-2)

    def hess(self, x):
        d = self.dim
        H = np.empty(x.shape[:-1] + (d, d, d))
        for a in range(d):
            for b in range(d):
                H[..., :, a, b] = self._mono(x, (a, b)) @ self.coef
        return H


class RigidBody(Field):
    """u = c + W x with W skew-symmetric (an infinitesimal rigid motion)."""

    def __init__(self, dim: int, seed: int = 0, scale: float = 1e-3):
        self.dim = dim
        r = 2.0 * uniform(seed, 4, stream=13) - 1.0
        self.c = r[:dim] * scale
        W = np.zeros((dim, dim))
        if dim == 2:
            W[0, 1], W[1, 0] = r[3] * scale, -r[3] * scale
        else:
            w = r[1:4] * scale
            W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        self.W = W

    def value(self, x):
        return self.c + x @ self.W.T

    def grad(self, x):
        return np.broadcast_to(self.W.T, x.shape[:-1] + (self.dim, self.dim)).copy()

    def hess(self, x):
        return np.zeros(x.shape[:-1] + (self.dim,) * 3)


class FiniteRotation(Field):
    """u = (Q - I) x for a proper rotation Q (a finite rigid motion)."""

    def __init__(self, dim: int, angle: float = 0.3, axis=(1.0, 2.0, 2.0)):
        self.dim = dim
        if dim == 2:
            c, s = math.cos(angle), math.sin(angle)
            Q = np.array([[c, -s], [s, c]])
        else:
            a = np.asarray(axis, float)
            a = a / np.linalg.norm(a)
            K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
            Q = np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)
        self.Q = Q

    def value(self, x):
        return x @ (self.Q - np.eye(self.dim)).T

    def grad(self, x):
        return np.broadcast_to((self.Q - np.eye(self.dim)).T,
                               x.shape[:-1] + (self.dim, self.dim)).copy()

    def hess(self, x):
        return np.zeros(x.shape[:-1] + (self.dim,) * 3)


# --------------------------------------------------------------------------
# workloads (the paper's Case 1 fields; the block-compression loading)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    n: int
    p: int
    n_plus: int
    q1: int
    jitter: float
    law: int            # 0 linear elastic, 1 neo-Hookean
    mu: float
    lam: float
    problem: str        # "mms-trig2d", "mms-mixed2d", "mms-trig3d", "block"
    mesh_seed: int
    load_steps: int = 1
    alpha: float = 0.1
    k_weight: float = 6.0
    length: float = 1.0      # edge of the square / cube
    cells: str = "tensor"    # "tensor" (quads / hexes), "simplex" (triangles / tetrahedra),
    #                          "polygon" (2-D dual polygons), "polyhedron" (extruded dual
    #                          polygons, given face by face) or "hexfaces"

    @property
    def n_cells(self) -> int:
        if self.cells == "polygon":
            return (self.n + 1) ** 2
        if self.cells == "polyhedron":
            return (self.n + 1) ** 2 * self.n
        if self.cells == "hexfaces":
            return self.n ** 3
        per = (2 if self.dim == 2 else 6) if self.cells == "simplex" else 1
        return per * self.n ** self.dim

    def mesh(self) -> Mesh:
        return make_mesh(self.dim, self.n, length=self.length, jitter=self.jitter,
                         seed=self.mesh_seed, cells=self.cells)

    @property
    def n_t(self) -> int:
        return math.comb(self.dim + self.p, self.dim)

    @property
    def stencil(self) -> int:
        return self.n_t + self.n_plus


_MU_S, _LAM_S = lame_from_young(200e9, 0.3)
_MU_1G, _LAM_1G = lame_from_young(1e9, 0.3)

WORKLOADS = {
    # 2-D plane strain, E=200 GPa, nu=0.3, 32x32 quads, quadratic LSQ, 2 Gauss pts/face
    "quad32-p2-trig": Workload("quad32-p2-trig", 2, 32, 2, 10, 2, 0.0, 0, _MU_S, _LAM_S,
                               "mms-trig2d", 1234),
    # 2-D, cubic LSQ, 3 Gauss pts/face, 512x512 quads jittered 25 %
    "quad512j-p3-mixed": Workload("quad512j-p3-mixed", 2, 512, 3, 10, 3, 0.25, 0, _MU_S,
                                  _LAM_S, "mms-mixed2d", 1235),
    # 3-D linear elastic cube, 96^3 hexes, cubic LSQ, 3x3 Gauss pts/face, E=1 GPa
    "hex96-p3-trig": Workload("hex96-p3-trig", 3, 96, 3, 65, 3, 0.0, 0, _MU_1G, _LAM_1G,
                              "mms-trig3d", 1236),
    # small 3-D cube of the same scheme (profiling-sized: ~2 GB of coefficients)
    "hex32-p3-trig": Workload("hex32-p3-trig", 3, 32, 3, 65, 3, 0.0, 0, _MU_1G, _LAM_1G,
                              "mms-trig3d", 1239),
    "hex32j-p3-nh": Workload("hex32j-p3-nh", 3, 32, 3, 65, 3, 0.20, 1, 1e6, 4e6, "block",
                             1240, load_steps=10),
    # the paper's largest regular-hex manufactured-solution mesh (Table 1): 45^3 hexes on a
    # 0.2 m cube, E=200 GPa, nu=0.3, cubic LSQ, 3x3 Gauss pts/face
    "hex45-p3-trig": Workload("hex45-p3-trig", 3, 45, 3, 65, 3, 0.0, 0, _MU_S, _LAM_S,
                              "mms-trig3d", 1241, length=0.2),
    # 3-D neo-Hookean block mu=1 MPa lambda=4 MPa, 64^3 hexes jittered 20 %, quadratic LSQ
    "hex64j-p2-nh": Workload("hex64j-p2-nh", 3, 64, 2, 55, 2, 0.20, 1, 1e6, 4e6, "block",
                             1237, load_steps=10),
    # unstructured simplex meshes: 2 x 512^2 jittered triangles, cubic LSQ (the 2-D
    # mixed field); 6 x 32^3 jittered tetrahedra, quadratic LSQ (the 3-D field)
    "tri512j-p3-mixed": Workload("tri512j-p3-mixed", 2, 512, 3, 10, 3, 0.15, 0, _MU_S, _LAM_S,
                                 "mms-mixed2d", 1242, cells="simplex"),
    "tet32j-p2-trig": Workload("tet32j-p2-trig", 3, 32, 2, 55, 2, 0.1, 0, _MU_1G, _LAM_1G,
                               "mms-trig3d", 1243, cells="simplex"),
    # the dual of the 2 x 512^2 triangle mesh: 513^2 polygons of 4-8 sides, cubic LSQ
    "poly512j-p3-mixed": Workload("poly512j-p3-mixed", 2, 512, 3, 10, 3, 0.15, 0, _MU_S, _LAM_S,
                                  "mms-mixed2d", 1244, cells="polygon"),
    # polyhedra: the dual polygons of 2 x 48^2 triangles extruded through 48 layers
    # (49^2 x 48 cells of 6 to 10 faces, non-planar faces of 4 to 8 corners), quadratic LSQ,
    # 2 x 2 points per fan triangle
    "prism48j-p2-trig": Workload("prism48j-p2-trig", 3, 48, 2, 55, 2, 0.1, 0, _MU_1G, _LAM_1G,
                                 "mms-trig3d", 1245, cells="polyhedron"),
    "prism24j-p2-trig": Workload("prism24j-p2-trig", 3, 24, 2, 55, 2, 0.1, 0, _MU_1G, _LAM_1G,
                                 "mms-trig3d", 1246, cells="polyhedron"),
    # the 64^3 jittered hexes described face by face (every face 4 corners: the
    # polyhedral path without padded fan slots), quadratic LSQ
    "hexf64j-p2-trig": Workload("hexf64j-p2-trig", 3, 64, 2, 55, 2, 0.2, 0, _MU_1G, _LAM_1G,
                                "mms-trig3d", 1247, cells="hexfaces"),
    # 3-D neo-Hookean, 128^3 jittered hexes, cubic LSQ
    "hex128j-p3-nh": Workload("hex128j-p3-nh", 3, 128, 3, 65, 3, 0.20, 1, 1e6, 4e6, "block",
                              1238, load_steps=10),
}


def field_for(problem: str, dim: int) -> Field | None:
    if problem == "mms-trig2d":
        return Trig2D()
    if problem == "mms-mixed2d":
        return Mixed2D()
    if problem == "mms-trig3d":
        return Trig3D()
    return None


def side_tags(problem: str, dim: int) -> np.ndarray:
    """Boundary condition tag per domain side: 0 displacement, 1 traction.
    Manufactured cases prescribe displacement on every side; the block has a
    fixed bottom (z-), a displaced top (z+) and traction-free sides."""
    if problem == "block":
        t = np.ones(2 * dim, dtype=np.int32)
        t[2 * dim - 2] = 0
        t[2 * dim - 1] = 0
        return t
    return np.zeros(2 * dim, dtype=np.int32)


def block_top_displacement(step: int, n_steps: int, dim: int, total: float = 0.3) -> np.ndarray:
    """Prescribed top-face displacement at load step `step` of `n_steps`:
    a compression of `total` of the unit height, in equal increments."""
    u = np.zeros(dim)
    u[dim - 1] = -total * step / n_steps
    return u
