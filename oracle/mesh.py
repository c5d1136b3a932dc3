"""Generic triangle meshes, Cartesian cube grids and TPFA geometry for the oracle (Sec. 2.1 of the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Everything here works on an explicit vertex / triangle list: edges, areas,
circumcentres and the two-level injection are computed from coordinates,
without using the structure of the square grid.  The only structured step is
the canonical renumbering of the refined mesh, which locates each fine
triangle by its centroid.

Readings taken where the paper is silent, ambiguous or inconsistent:
  R1  cell points are circumcentres (Sec. 2.1).  On right triangles two cells
      that share a hypotenuse have the same circumcentre; for such an edge
      (|w| < 1e-12 |e|) the distance |w| is replaced by the distance between
      the two barycentres and the reconstruction weight by 1/2.
  R2  the arithmetic-mean reconstruction weight of Sec. 2.1 is
      lambda_{e,K} = d_{K,e} / |w_e|, with d_{K,e} the distance from the point
      of K to the line of e (the share of the diamond of e lying in K).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class TriMesh:
    """A triangle mesh with interior-edge TPFA geometry."""

    xy: np.ndarray          # (nv, 2) vertex coordinates
    tri: np.ndarray         # (nt, 3) vertex indices, counter-clockwise
    area: np.ndarray        # (nt,) |c|
    centre: np.ndarray      # (nt, 2) circumcentres
    bary: np.ndarray        # (nt, 2) barycentres
    edge_cells: np.ndarray  # (ne, 2) [left, right] cell of each interior edge
    edge_len: np.ndarray    # (ne,) |e|
    edge_dist: np.ndarray   # (ne,) |w| (distance between cell points)
    edge_lambda: np.ndarray  # (ne,) weight of the left cell in the edge average
    degenerate: np.ndarray  # (ne,) True where rule R1 replaced |w|

    @property
    def ncell(self) -> int:
        return self.tri.shape[0]

    @property
    def nedge(self) -> int:
        return self.edge_cells.shape[0]


def _circumcentre(p: np.ndarray) -> np.ndarray:
    a, b, c = p[:, 0], p[:, 1], p[:, 2]
    d = 2.0 * (a[:, 0] * (b[:, 1] - c[:, 1]) + b[:, 0] * (c[:, 1] - a[:, 1]) + c[:, 0] * (a[:, 1] - b[:, 1]))
    a2, b2, c2 = (a ** 2).sum(1), (b ** 2).sum(1), (c ** 2).sum(1)
    ux = (a2 * (b[:, 1] - c[:, 1]) + b2 * (c[:, 1] - a[:, 1]) + c2 * (a[:, 1] - b[:, 1])) / d
    uy = (a2 * (c[:, 0] - b[:, 0]) + b2 * (a[:, 0] - c[:, 0]) + c2 * (b[:, 0] - a[:, 0])) / d
    return np.stack([ux, uy], 1)


def _point_line_distance(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    t = b - a
    cross = t[:, 0] * (p[:, 1] - a[:, 1]) - t[:, 1] * (p[:, 0] - a[:, 0])
    return np.abs(cross) / np.hypot(t[:, 0], t[:, 1])


def build_mesh(xy: np.ndarray, tri: np.ndarray) -> TriMesh:
    """Compute areas, cell points and interior-edge geometry of a triangle list."""
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    p = xy[tri]
    e1, e2 = p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    if np.any(area <= 0):
        raise ValueError("triangles must be counter-clockwise and non-degenerate")
    centre = _circumcentre(p)
    bary = p.mean(1)

    # interior edges = vertex pairs shared by two triangles
    owner: dict[tuple[int, int], int] = {}
    cells, verts = [], []
    for c in range(tri.shape[0]):
        for a, b in ((0, 1), (1, 2), (2, 0)):
            key = tuple(sorted((int(tri[c, a]), int(tri[c, b]))))
            if key in owner:
                cells.append((owner.pop(key), c))
                verts.append(key)
            else:
                owner[key] = c
    edge_cells = np.array(cells, dtype=np.int64).reshape(-1, 2)
    ev = np.array(verts, dtype=np.int64).reshape(-1, 2)
    va, vb = xy[ev[:, 0]], xy[ev[:, 1]]
    edge_len = np.hypot(*(vb - va).T)

    left, right = edge_cells[:, 0], edge_cells[:, 1]
    dist = np.hypot(*(centre[left] - centre[right]).T)
    degenerate = dist < 1e-12 * edge_len
    bdist = np.hypot(*(bary[left] - bary[right]).T)
    edge_dist = np.where(degenerate, bdist, dist)
    d_left = _point_line_distance(centre[left], va, vb)
    lam = np.where(degenerate, 0.5, d_left / np.where(degenerate, 1.0, dist))
    return TriMesh(xy, tri, area, centre, bary, edge_cells, edge_len, edge_dist, lam, degenerate)


def square_grid(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit square, n x n squares, each split by its (0,0)->(1,1) diagonal.

    Triangle (t, i, j) has index t n^2 + j n + i; t = 0 is the lower-right
    triangle (i,j),(i+1,j),(i+1,j+1), t = 1 the upper-left (i,j),(i+1,j+1),(i,j+1).
    """
    vid = lambda i, j: j * (n + 1) + i  # noqa: E731
    xs = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    tri = np.zeros((2 * n * n, 3), dtype=np.int64)
    for j in range(n):
        for i in range(n):
            tri[j * n + i] = (vid(i, j), vid(i + 1, j), vid(i + 1, j + 1))
            tri[n * n + j * n + i] = (vid(i, j), vid(i + 1, j + 1), vid(i, j + 1))
    return xy, tri


def refine4(xy: np.ndarray, tri: np.ndarray):
    """Midpoint 4-split of every triangle.

    Returns (xy_fine, tri_fine, parent) where parent[f] is the coarse triangle
    containing fine triangle f.  Fine triangles keep counter-clockwise order.
    """
    xy = list(map(tuple, np.asarray(xy, dtype=np.float64)))
    index = {p: k for k, p in enumerate(xy)}
    mid: dict[tuple[int, int], int] = {}

    def midpoint(a: int, b: int) -> int:
        key = (min(a, b), max(a, b))
        if key not in mid:
            p = ((xy[a][0] + xy[b][0]) / 2, (xy[a][1] + xy[b][1]) / 2)
            if p not in index:
                index[p] = len(xy)
                xy.append(p)
            mid[key] = index[p]
        return mid[key]

    fine, parent = [], []
    for c, (a, b, d) in enumerate(np.asarray(tri)):
        ab, bd, da = midpoint(a, b), midpoint(b, d), midpoint(d, a)
        for t in ((a, ab, da), (ab, b, bd), (da, bd, d), (ab, bd, da)):
            fine.append(t)
            parent.append(c)
    return np.array(xy), np.array(fine, dtype=np.int64), np.array(parent, dtype=np.int64)


def canonical_square_order(xy: np.ndarray, tri: np.ndarray, m: int) -> np.ndarray:
    """Permutation putting the triangles of a refined m x m diagonal grid in canonical order.

    Returns perm with perm[canonical index] = position in ``tri``.  Each triangle
    is located by its centroid: square (I, J) = floor(centroid * m), and it is
    the lower-right one (t = 0) when its centroid lies below the diagonal.
    """
    g = np.asarray(xy)[np.asarray(tri)].mean(1)
    I = np.floor(g[:, 0] * m).astype(np.int64)
    J = np.floor(g[:, 1] * m).astype(np.int64)
    below = (g[:, 0] * m - I) > (g[:, 1] * m - J)
    t = np.where(below, 0, 1)
    canon = t * m * m + J * m + I
    perm = np.empty(len(canon), dtype=np.int64)
    perm[canon] = np.arange(len(canon))
    if len(np.unique(canon)) != len(canon):
        raise ValueError("refined mesh is not the canonical diagonal grid")
    return perm


@dataclass
class TwoLevelMesh:
    """Coarse mesh T' (density, slack) and fine mesh T (potential), Sec. 2.1."""

    coarse: TriMesh
    fine: TriMesh
    parent: np.ndarray  # (N,) coarse cell of each fine cell: the injection J
    n: int              # squares per side of the coarse grid


def two_level_square(n: int) -> TwoLevelMesh:
    """Coarse n x n right-triangle grid and its midpoint 4-split, both in canonical order."""
    xy, tri = square_grid(n)
    coarse = build_mesh(xy, tri)
    fxy, ftri, parent = refine4(xy, tri)
    perm = canonical_square_order(fxy, ftri, 2 * n)
    fine = build_mesh(fxy, ftri[perm])
    return TwoLevelMesh(coarse, fine, parent[perm], n)


# ---------------------------------------------------------------- cube grids (3D)
@dataclass
class CubeMesh:
    """A uniform grid of n^3 cubes of side h = 1/n on [0,1]^3, with the same
    TPFA fields as TriMesh so that the operators apply unchanged: `area` holds
    the cell measure h^3, each interior face is an `edge` with measure
    edge_len = h^2, cell-point distance edge_dist = h and weight 1/2 (the
    cube centres are the cell points; every face is orthogonal to the segment
    joining them)."""

    n: int
    area: np.ndarray        # (nc,) cell volumes
    centre: np.ndarray      # (nc, 3) cube centres
    bary: np.ndarray        # (nc, 3) the same points
    edge_cells: np.ndarray  # (nf, 2) [lower, upper] cell along the face normal
    edge_len: np.ndarray    # (nf,) face areas
    edge_dist: np.ndarray   # (nf,) distance between the two centres
    edge_lambda: np.ndarray  # (nf,) 1/2
    degenerate: np.ndarray  # (nf,) False
    edge_axis: np.ndarray   # (nf,) 0, 1, 2: normal direction x, y, z

    @property
    def ncell(self) -> int:
        return self.area.shape[0]

    @property
    def nedge(self) -> int:
        return self.edge_cells.shape[0]


def cube_grid(n: int) -> CubeMesh:
    """n^3 cubes, cell (i, j, k) at index (k n + j) n + i (x fastest)."""
    h = 1.0 / n
    idx = lambda i, j, k: (k * n + j) * n + i  # noqa: E731
    g = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    centre = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    cells, axes = [], []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                if i + 1 < n:
                    cells.append((idx(i, j, k), idx(i + 1, j, k)))
                    axes.append(0)
                if j + 1 < n:
                    cells.append((idx(i, j, k), idx(i, j + 1, k)))
                    axes.append(1)
                if k + 1 < n:
                    cells.append((idx(i, j, k), idx(i, j, k + 1)))
                    axes.append(2)
    nf = len(cells)
    edge_cells = np.array(cells, dtype=np.int64).reshape(-1, 2)
    return CubeMesh(n, np.full(n ** 3, h ** 3), centre, centre.copy(), edge_cells, np.full(nf, h * h),
                    np.full(nf, h), np.full(nf, 0.5), np.zeros(nf, dtype=bool), np.array(axes, dtype=np.int64))


def one_level_cube(n: int) -> TwoLevelMesh:
    """The Cartesian case of the paper's test 4: density and potential on the same
    n^3 grid, so the injection J is the identity."""
    m = cube_grid(n)
    return TwoLevelMesh(m, m, np.arange(m.ncell, dtype=np.int64), n)
