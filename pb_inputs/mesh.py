"""Seeded synthetic surface meshes: icospheres and Gaussian-density isosurfaces.

These produce the flat-triangle discretisation the method consumes (Section 2.2:
flat triangles with centroid collocation; Section 2.4: faces/vertices converted to
centroids, normals and areas).  The paper's meshes come from MSMS, which is not
available, so a subdivided icosahedron stands in for the spherical cavity of
Section 3.2 and a marching-tetrahedra isosurface of summed atom Gaussians stands
in for the protein surfaces of Section 3.3.

Nothing here evaluates the boundary-integral method: it only builds triangles.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Surface:
    """A closed triangulated surface in collocation form.

    centroids: (N, 3) float64, triangle centroids in Angstrom.
    normals:   (N, 3) float64, unit normals pointing out of the solute (Omega_1).
    areas:     (N,)   float64, triangle areas in Angstrom^2 (the weights W_j).
    vertices/faces: the underlying triangle mesh (kept for inspection).
    """

    centroids: np.ndarray
    normals: np.ndarray
    areas: np.ndarray
    vertices: np.ndarray | None = None
    faces: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.areas.shape[0])

    def transformed(self, rot: np.ndarray | None = None, shift=None, scale: float = 1.0) -> "Surface":
        """Rigid motion plus uniform scaling: x -> scale * R x + shift."""
        rot = np.eye(3) if rot is None else np.asarray(rot, dtype=np.float64)
        shift = np.zeros(3) if shift is None else np.asarray(shift, dtype=np.float64)
        c = scale * self.centroids @ rot.T + shift
        nrm = self.normals @ rot.T
        a = self.areas * scale * scale
        v = None if self.vertices is None else scale * self.vertices @ rot.T + shift
        return Surface(np.ascontiguousarray(c), np.ascontiguousarray(nrm),
                       np.ascontiguousarray(a), v, self.faces)

    def subset(self, idx) -> "Surface":
        idx = np.asarray(idx)
        return Surface(np.ascontiguousarray(self.centroids[idx]), np.ascontiguousarray(self.normals[idx]),
                       np.ascontiguousarray(self.areas[idx]))


def triangles_to_surface(vertices: np.ndarray, faces: np.ndarray, min_area: float = 1e-10) -> Surface:
    """Centroid, unit normal (right-hand rule on the face order) and area per face.

    Faces with area below ``min_area`` are dropped (degenerate triangles).
    """
    v = np.asarray(vertices, dtype=np.float64)
    f = np.asarray(faces, dtype=np.int64)
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    twice_area = np.sqrt(np.einsum("ij,ij->i", cr, cr))
    keep = 0.5 * twice_area >= min_area
    cr, twice_area, f = cr[keep], twice_area[keep], f[keep]
    p0, p1, p2 = p0[keep], p1[keep], p2[keep]
    centroids = (p0 + p1 + p2) / 3.0
    normals = cr / twice_area[:, None]
    return Surface(np.ascontiguousarray(centroids), np.ascontiguousarray(normals),
                   np.ascontiguousarray(0.5 * twice_area), v, f)


def _icosahedron():
    t = (1.0 + np.sqrt(5.0)) / 2.0
    verts = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                      [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                      [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    faces = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                      [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                      [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                      [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    return verts, faces


def icosphere(radius: float, level: int, center=(0.0, 0.0, 0.0)) -> Surface:
    """Icosahedron subdivided ``level`` times (20 * 4**level flat faces).

    Every edge midpoint is pushed out to the sphere, so all vertices lie on the
    sphere of the given radius and the flat faces sit slightly inside it.  Faces
    are ordered so that their right-hand normals point outward.
    """
    verts, faces = _icosahedron()
    vlist = [v for v in verts]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            k = cache.get(key)
            if k is None:
                m = vlist[a] + vlist[b]
                m = m / np.linalg.norm(m)
                vlist.append(m)
                k = len(vlist) - 1
                cache[key] = k
            return k

        nf = np.empty((faces.shape[0] * 4, 3), dtype=np.int64)
        for fi, (a, b, c) in enumerate(faces):
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf[4 * fi + 0] = (a, ab, ca)
            nf[4 * fi + 1] = (b, bc, ab)
            nf[4 * fi + 2] = (c, ca, bc)
            nf[4 * fi + 3] = (ab, bc, ca)
        faces = nf
    v = np.asarray(vlist) * float(radius) + np.asarray(center, dtype=np.float64)
    # orient outward: the face normal must point away from the centre
    p0, p1, p2 = v[faces[:, 0]], v[faces[:, 1]], v[faces[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    inward = np.einsum("ij,ij->i", cr, (p0 + p1 + p2) / 3.0 - np.asarray(center)) < 0
    faces[inward] = faces[inward][:, ::-1]
    return triangles_to_surface(v, faces)


# --- marching tetrahedra ----------------------------------------------------
# Each grid cube is split into the six tetrahedra that share its main diagonal
# (corner 0 -> corner 7).  Corner c of a cube has offset ((c>>0)&1, (c>>1)&1, (c>>2)&1).
_CUBE_TETS = np.array([[0, 1, 3, 7], [0, 3, 2, 7], [0, 2, 6, 7],
                       [0, 6, 4, 7], [0, 4, 5, 7], [0, 5, 1, 7]], dtype=np.int64)
_TET_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _edge_index(a: int, b: int) -> int:
    return _TET_EDGES.index((a, b) if a < b else (b, a))


def _tet_case_table():
    """For each of the 16 inside/outside patterns of a tetrahedron, the list of
    triangles given as triples of tetrahedron-edge indices (unoriented)."""
    table = []
    for case in range(16):
        inside = [i for i in range(4) if (case >> i) & 1]
        outside = [i for i in range(4) if not (case >> i) & 1]
        tris = []
        if len(inside) in (1, 3):
            lone = inside[0] if len(inside) == 1 else outside[0]
            others = [i for i in range(4) if i != lone]
            tris.append(tuple(_edge_index(lone, o) for o in others))
        elif len(inside) == 2:
            a, b = inside
            c, d = outside
            e_ac, e_ad, e_bc, e_bd = (_edge_index(a, c), _edge_index(a, d),
                                      _edge_index(b, c), _edge_index(b, d))
            # quad a-c, a-d, b-d, b-c split into two triangles
            tris.append((e_ac, e_ad, e_bd))
            tris.append((e_ac, e_bd, e_bc))
        table.append(tris)
    return table


_TET_TABLE = _tet_case_table()


def isosurface(field: np.ndarray, origin, spacing: float, level: float, min_area: float = 1e-10,
               value_and_grad=None, relax_iterations: int = 8) -> Surface:
    """Marching-tetrahedra isosurface {field == level} of a sampled scalar field.

    ``field[i, j, k]`` is the value at origin + spacing * (i, j, k).  The region
    field >= level is the inside; every triangle is oriented so that its normal
    points toward decreasing field (outward).  Vertices on shared edges are
    merged, so the output is a closed, consistently triangulated surface when the
    inside region does not touch the grid boundary.

    Marching tetrahedra leaves many slivers, and slivers make the collocation
    system badly conditioned.  When ``value_and_grad`` (the exact field and its
    gradient) is given, the vertices are relaxed along the level set with
    ``relax_on_level_set`` before the collocation data are computed.
    """
    f = np.asarray(field, dtype=np.float64)
    nx, ny, nz = f.shape
    origin = np.asarray(origin, dtype=np.float64)
    inside = f >= level

    # global index of grid point (i, j, k)
    def gid(i, j, k):
        return (i * ny + j) * nz + k

    # keep only cubes that straddle the level
    any_in = np.zeros((nx - 1, ny - 1, nz - 1), dtype=bool)
    all_in = np.ones((nx - 1, ny - 1, nz - 1), dtype=bool)
    for c in range(8):
        dx, dy, dz = (c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1
        sl = inside[dx:nx - 1 + dx, dy:ny - 1 + dy, dz:nz - 1 + dz]
        any_in |= sl
        all_in &= sl
    ci, cj, ck = np.nonzero(any_in & ~all_in)
    ci, cj, ck = ci.astype(np.int64), cj.astype(np.int64), ck.astype(np.int64)
    corner_ids = np.stack([gid(ci + ((c >> 0) & 1), cj + ((c >> 1) & 1), ck + ((c >> 2) & 1)) for c in range(8)], 1)
    ins_flat = inside.ravel()
    fflat = f.ravel()

    edge_keys = []   # (tri, 3) pairs of grid ids per triangle vertex
    for tet in _CUBE_TETS:
        tv = corner_ids[:, tet]                       # (M, 4) grid ids
        tin = ins_flat[tv]
        case = (tin[:, 0].astype(np.int64) | (tin[:, 1] << 1) | (tin[:, 2] << 2) | (tin[:, 3] << 3))
        for cs in range(1, 15):
            sel = case == cs
            if not sel.any():
                continue
            tvs = tv[sel]
            for tri in _TET_TABLE[cs]:
                ends = []
                for e in tri:
                    a, b = _TET_EDGES[e]
                    ga, gb = tvs[:, a], tvs[:, b]
                    ends.append(np.stack([np.minimum(ga, gb), np.maximum(ga, gb)], 1))
                edge_keys.append(np.stack(ends, 1))   # (m, 3, 2)
    if not edge_keys:
        raise ValueError("isosurface: the level set is empty on this grid")
    ek = np.concatenate(edge_keys, 0)
    flat = ek.reshape(-1, 2)
    uniq, inv = np.unique(flat[:, 0] * (nx * ny * nz) + flat[:, 1], return_inverse=True)
    ga = uniq // (nx * ny * nz)
    gb = uniq % (nx * ny * nz)

    def coords(g):
        i = g // (ny * nz)
        j = (g // nz) % ny
        k = g % nz
        return origin + spacing * np.stack([i, j, k], 1).astype(np.float64)

    fa, fb = fflat[ga], fflat[gb]
    t = (level - fa) / (fb - fa)
    verts = coords(ga) + t[:, None] * (coords(gb) - coords(ga))
    faces = inv.reshape(-1, 3).astype(np.int64)

    # orient: outward = toward lower field.  The plane of each triangle crosses
    # the edge of its first vertex, so the triangle normal must point from that
    # edge's inside end to its outside end.
    p0, p1, p2 = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    e0 = ek[:, 0, :]
    in_end = np.where(ins_flat[e0[:, 0]], e0[:, 0], e0[:, 1])
    out_end = np.where(ins_flat[e0[:, 0]], e0[:, 1], e0[:, 0])
    outward_dir = coords(out_end) - coords(in_end)
    flip = np.einsum("ij,ij->i", cr, outward_dir) < 0
    faces[flip] = faces[flip][:, ::-1]

    if value_and_grad is not None and relax_iterations > 0:
        verts = relax_on_level_set(verts, faces, value_and_grad, level, relax_iterations)
    # drop collapsed faces before computing geometry
    ok = (faces[:, 0] != faces[:, 1]) & (faces[:, 1] != faces[:, 2]) & (faces[:, 0] != faces[:, 2])
    return triangles_to_surface(verts, faces[ok], min_area=min_area)


def relax_on_level_set(vertices: np.ndarray, faces: np.ndarray, value_and_grad, level: float,
                       iterations: int = 8, weight: float = 0.5, newton_steps: int = 3) -> np.ndarray:
    """Improve triangle shapes while keeping every vertex on {f = level}.

    Each iteration moves every vertex a fraction ``weight`` toward the mean of
    its edge neighbours (uniform Laplacian smoothing) and then projects it back
    onto the level set with Newton steps along the gradient,
    x <- x - (f(x) - level) grad f / |grad f|^2.  ``value_and_grad(x)`` returns
    (f (n,), grad f (n,3)).  Connectivity is unchanged.
    """
    v = np.array(vertices, dtype=np.float64, copy=True)
    f = np.asarray(faces, dtype=np.int64)
    nv = v.shape[0]
    src = np.concatenate([f[:, 0], f[:, 1], f[:, 2], f[:, 1], f[:, 2], f[:, 0]])
    dst = np.concatenate([f[:, 1], f[:, 2], f[:, 0], f[:, 0], f[:, 1], f[:, 2]])
    key = np.unique(src * nv + dst)
    src, dst = key // nv, key % nv
    deg = np.bincount(src, minlength=nv).astype(np.float64)
    used = deg > 0
    for _ in range(iterations):
        mean = np.zeros_like(v)
        for d in range(3):
            mean[:, d] = np.bincount(src, weights=v[dst, d], minlength=nv)
        mean[used] /= deg[used, None]
        v[used] += weight * (mean[used] - v[used])
        for _ in range(newton_steps):
            val, grad = value_and_grad(v[used])
            g2 = np.einsum("ij,ij->i", grad, grad)
            step = np.where(g2 > 0, (val - level) / np.where(g2 > 0, g2, 1.0), 0.0)
            v[used] -= step[:, None] * grad
    return v


def enclosed_volume(surface: Surface) -> float:
    """Signed volume (divergence theorem with the centroid rule); > 0 when the
    normals point outward."""
    return float(np.sum(np.einsum("ij,ij->i", surface.centroids, surface.normals) * surface.areas) / 3.0)
