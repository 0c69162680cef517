"""Workload recipes: seeded synthetic stand-ins for the paper's test problems.

* ``kirkwood_sphere_single``: spherical cavity, one central unit charge (the Born
  problem), icosphere radius 2 A at level 4 = 5,120 triangles.
* ``kirkwood_sphere_multi``: icosphere radius 20 A at level 6 = 81,920 triangles
  with 20 charges uniform in the ball of radius 16 A, Q ~ U[-1, 1] (seed 2).
* ``protein_like``: a compact 2,000-atom chain; the surface is the isosurface
  of summed atom Gaussians, about 300,000 triangles.
* ``helix_sphere``: the nine-charge helix in a radius-4 A sphere (Section 3.2).

Physical parameters for all of them: eps1 = 1, eps2 = 80, kappa = 0.1257 1/A
(about 0.15 M monovalent salt), GMRES restart 10.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .charges import ball_charges, compact_chain, helix_charges
from .mesh import Surface, icosphere, isosurface

EPS1 = 1.0
EPS2 = 80.0
KAPPA = 0.1257


@dataclasses.dataclass
class Problem:
    name: str
    surface: Surface
    charges: np.ndarray          # (Nc, 4): x, y, z, Q
    eps1: float = EPS1
    eps2: float = EPS2
    kappa: float = KAPPA
    sphere_radius: float | None = None   # set for spherical cavities centred at the origin

    @property
    def n(self) -> int:
        return self.surface.n

    @property
    def nc(self) -> int:
        return int(self.charges.shape[0])


def kirkwood_sphere_single(level: int = 4, radius: float = 2.0, kappa: float = KAPPA) -> Problem:
    surf = icosphere(radius, level)
    ch = np.array([[0.0, 0.0, 0.0, 1.0]])
    return Problem(f"born_sphere_R{radius:g}_L{level}", surf, ch, kappa=kappa, sphere_radius=radius)


def kirkwood_sphere_multi(level: int = 6, radius: float = 20.0, n_charges: int = 20, seed: int = 2,
                          kappa: float = KAPPA) -> Problem:
    surf = icosphere(radius, level)
    ch = ball_charges(n_charges, 0.8 * radius, seed)
    return Problem(f"kirkwood_sphere_R{radius:g}_L{level}_q{n_charges}", surf, ch, kappa=kappa,
                   sphere_radius=radius)


def helix_sphere(level: int = 4, radius: float = 4.0, kappa: float = 0.0) -> Problem:
    surf = icosphere(radius, level)
    ch = helix_charges()
    return Problem(f"helix_sphere_R{radius:g}_L{level}", surf, ch, kappa=kappa, sphere_radius=radius)


def gaussian_density(pos: np.ndarray, radii: np.ndarray, origin: np.ndarray, spacing: float,
                     shape, beta: float = 2.0, cutoff: float = 1e-7) -> np.ndarray:
    """Sum over atoms of exp(-beta (|x - c|^2 / r^2 - 1)) sampled on a grid."""
    field = np.zeros(shape)
    for c, r in zip(pos, radii):
        # exp(-beta (d^2/r^2 - 1)) < cutoff beyond d^2 = r^2 (1 - ln(cutoff)/beta)
        rc = r * np.sqrt(1.0 - np.log(cutoff) / beta)
        lo = np.maximum(np.floor((c - rc - origin) / spacing).astype(int), 0)
        hi = np.minimum(np.ceil((c + rc - origin) / spacing).astype(int) + 1, np.asarray(shape))
        gx = origin[0] + spacing * np.arange(lo[0], hi[0]) - c[0]
        gy = origin[1] + spacing * np.arange(lo[1], hi[1]) - c[1]
        gz = origin[2] + spacing * np.arange(lo[2], hi[2]) - c[2]
        d2 = gx[:, None, None] ** 2 + gy[None, :, None] ** 2 + gz[None, None, :] ** 2
        field[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += np.exp(-beta * (d2 / (r * r) - 1.0))
    return field


def gaussian_value_and_grad(pos: np.ndarray, radii: np.ndarray, beta: float = 2.0, cutoff: float = 1e-7,
                            max_neighbors: int = 96):
    """Exact summed-Gaussian field and its gradient at arbitrary points (atoms
    beyond the same cutoff radius as ``gaussian_density`` are ignored)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(pos)
    rc = float(radii.max()) * np.sqrt(1.0 - np.log(cutoff) / beta)
    k = min(max_neighbors, pos.shape[0])

    def fg(x):
        d, idx = tree.query(x, k=k, distance_upper_bound=rc)
        d = np.asarray(d).reshape(x.shape[0], k)
        idx = np.asarray(idx).reshape(x.shape[0], k)
        ok = np.isfinite(d)
        ii = np.where(ok, idx, 0)
        r2 = radii[ii] ** 2
        diff = x[:, None, :] - pos[ii]
        dd = np.einsum("ijk,ijk->ij", diff, diff)
        w = np.where(ok, np.exp(-beta * (dd / r2 - 1.0)), 0.0)
        val = w.sum(1)
        grad = np.einsum("ij,ijk->ik", w * (-2.0 * beta / r2), diff)
        return val, grad
    return fg


SOLUTE_LEVELS = (1.0, 0.95, 1.05, 0.9, 1.1)


def _folded_facets(surf: Surface, value_and_grad) -> int:
    """Facets whose geometric normal opposes the smooth surface's normal
    (-grad f) at their centroid."""
    v = surf.vertices[surf.faces]
    fn = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    _, g = value_and_grad(surf.centroids)
    return int(np.sum(np.einsum("ij,ij->i", fn, -g) <= 0.0))


def solute_surface(pos: np.ndarray, radii: np.ndarray, spacing: float, beta: float = 2.0,
                   relax_iterations: int = 8, analytic_normals: bool = True,
                   levels=SOLUTE_LEVELS) -> Surface:
    """Isosurface of the summed atom Gaussians, relaxed on the exact level set.

    The level is the first of ``levels`` (1 first) whose triangulation has no
    folded facet, else the one with the fewest: where a critical value of the
    field lies close to the level, the level set has a pinch finer than the
    grid and the piecewise-linear surface folds there; a slightly different
    level moves off it.

    With ``analytic_normals`` every element's normal is the unit outward normal
    of the smooth surface at its centroid, -grad f / |grad f|, instead of the
    flat facet's normal; the two agree on an unfolded mesh up to the facet's
    tilt."""
    margin = float(radii.max()) * 2.0 + 2.0 * spacing
    origin = pos.min(0) - margin
    shape = tuple(int(np.ceil(e / spacing)) + 1 for e in (pos.max(0) + margin - origin))
    field = gaussian_density(pos, radii, origin, spacing, shape, beta=beta)
    fg = gaussian_value_and_grad(pos, radii, beta)
    best, best_folds = None, None
    for level in levels:
        cand = isosurface(field, origin, spacing, level, value_and_grad=fg, relax_iterations=relax_iterations)
        folds = _folded_facets(cand, fg)
        if best is None or folds < best_folds:
            best, best_folds = cand, folds
        if folds == 0:
            break
    surf = best
    if analytic_normals:
        _, g = fg(surf.centroids)
        gn = np.linalg.norm(g, axis=1, keepdims=True)
        ok = gn[:, 0] > 0
        nrm = surf.normals.copy()
        nrm[ok] = -g[ok] / gn[ok]
        surf = Surface(surf.centroids, np.ascontiguousarray(nrm), surf.areas, surf.vertices, surf.faces)
    return surf


PROBE_RADIUS = 1.4


def protein_like(n_atoms: int = 2000, seed: int = 3, target_triangles: int | None = 300_000,
                 spacing: float | None = None, beta: float = 0.4, probe: float = PROBE_RADIUS) -> Problem:
    """Seeded protein-like solute.

    The surface is the level-1 set of summed Gaussians whose radii are the atom
    radii plus a solvent-probe radius (1.4 A), so that crevices narrower than a
    water molecule are filled, as on a probe-traced molecular surface (Section 1).
    Without the probe the bead-chain surface has thin necks between atoms and
    the collocation system converges very slowly.  The soft Gaussians
    (beta = 0.4) keep the surface's curvature resolved at the coarse grid
    spacings (up to about 2 A) that 40 triangles per atom need: with beta = 1
    such meshes had folded facets, facets whose orientation opposes the smooth
    surface's, and some of them stalled restarted GMRES.  With
    ``target_triangles`` the grid spacing is chosen from a coarse trial surface
    so that the final triangle count lands near the target (the count scales
    like area / spacing^2)."""
    pos, radii, q = compact_chain(n_atoms, seed)
    rs = radii + probe
    if spacing is None:
        trial = 1.2
        n_trial = solute_surface(pos, rs, trial, beta, relax_iterations=0, levels=(1.0,)).n
        spacing = trial * np.sqrt(n_trial / float(target_triangles))
    surf = solute_surface(pos, rs, spacing, beta, relax_iterations=10)
    ch = np.concatenate([pos, q[:, None]], 1)
    return Problem(f"protein_like_a{n_atoms}_s{seed}", surf, ch)


def by_name(name: str) -> Problem:
    """The named synthetic workloads used by the tests and the benchmark."""
    if name == "sphere1":
        return kirkwood_sphere_single()
    if name == "sphere2":
        return kirkwood_sphere_multi()
    if name == "sphere2_salt_free":
        return kirkwood_sphere_multi(kappa=0.0)
    if name == "protein300k":
        return protein_like()
    raise KeyError(name)
