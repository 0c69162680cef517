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


def batch_specs(n: int = 64, seed: int = 4):
    """The batched-solve workload's solutes: atom counts floor(exp U[ln 50,
    ln 1500]) with about 40 triangles per atom (N ~ 2k-60k).  Returns
    [(n_atoms, chain seed, target triangles)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    atoms = np.floor(np.exp(rng.uniform(np.log(50), np.log(1500), size=n))).astype(int)
    return [(int(a), 1000 + i, int(40 * a)) for i, a in enumerate(atoms)]


def serve_specs(n: int = 64, seed: int = 5):
    """The serving workload's solute pool: N log-uniform in [5k, 300k], atom
    count N/150 (the 2,000-atom solute gives ~300k).  Returns
    [(n_atoms, chain seed, target triangles)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(np.log(5e3), np.log(3e5), size=n))
    return [(max(20, int(x / 150)), 2000 + i, int(x)) for i, x in enumerate(ns)]


def solute_from_spec(spec, kappa: float = KAPPA) -> Problem:
    n_atoms, seed, target = spec
    p = protein_like(n_atoms=n_atoms, seed=seed, target_triangles=target)
    return Problem(p.name, p.surface, p.charges, kappa=kappa)


def batch_problem(k: int, r: int) -> Problem:
    """Solute k of the 64-solute batch with its charge variant r (of 8; the
    variants drawn with seed 3000 + k)."""
    from .charges import charge_variants
    p = solute_from_spec(batch_specs(64)[k])
    q = charge_variants(p.charges, 8, seed=3000 + k)[r]
    return Problem(f"{p.name}_set{r}", p.surface, q, p.eps1, p.eps2, p.kappa)


def by_name(name: str) -> Problem:
    """The named synthetic workloads used by the tests and the benchmark.
    ``serve<k>_kappa<0|1>``: solute k of the 64-solute serving pool with
    kappa 0 or 0.1257; ``batch<k>_set<r>``: solute k of the 64-solute batch
    with charge variant r."""
    if name.startswith("batch") and "_set" in name:
        k, r = name[len("batch"):].split("_set")
        return batch_problem(int(k), int(r))
    if name.startswith("serve") and "_kappa" in name:
        k, kap = name[len("serve"):].split("_kappa")
        return solute_from_spec(serve_specs(64)[int(k)], kappa=(0.0 if kap == "0" else KAPPA))
    if name == "sphere1":
        return kirkwood_sphere_single()
    if name == "sphere2":
        return kirkwood_sphere_multi()
    if name == "sphere2_salt_free":
        return kirkwood_sphere_multi(kappa=0.0)
    if name == "protein300k":
        return protein_like()
    raise KeyError(name)


def md_frames(base: Problem, n_frames: int = 20, seed: int = 7, amplitude: float = 0.2, wavelength: float = 25.0,
              phase_step: float = 0.15, q_sigma: float = 0.02) -> list:
    """A sequence of perturbed copies of a solute, standing in for the frames
    of a molecular-dynamics trajectory that are solved one after another.

    Frame f moves every point by a smooth displacement
    g_f(x) = sum_m c_m [sin(w_m . x + phi_m + f omega_m) - sin(w_m . x + phi_m)]
    (three modes, |c_m| = ``amplitude``, |w_m| = 2 pi / ``wavelength``, phases
    advancing by about ``phase_step`` per frame), zero at frame 0.  Element centroids and charge positions move
    with it; normals and areas follow the deformation gradient J = I + grad g
    (Nanson's relation: n' dA' = det(J) J^-T n dA).  The partial charges get
    seeded N(0, q_sigma) jitter per frame, shifted to keep the net charge.
    Frame 0 is the undeformed solute with its own charges."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = 2.0 * np.pi / wavelength
    dirs = rng.normal(size=(3, 3))
    w = k * dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    cvec = rng.normal(size=(3, 3))
    cvec = amplitude * cvec / np.linalg.norm(cvec, axis=1, keepdims=True)
    phi0 = rng.uniform(0.0, 2.0 * np.pi, size=3)
    omega = phase_step * rng.uniform(0.5, 1.5, size=3)
    s = base.surface
    q0 = base.charges
    frames = []
    for f in range(n_frames):
        if f == 0:
            frames.append(Problem(f"{base.name}_frame0", s, q0.copy(), base.eps1, base.eps2, base.kappa,
                                  base.sphere_radius))
            continue

        def disp(x):
            arg0 = x @ w.T + phi0                    # (n, 3 modes)
            arg = arg0 + f * omega
            return (np.sin(arg) - np.sin(arg0)) @ cvec, np.cos(arg) - np.cos(arg0)

        d, cosv = disp(s.centroids)
        cen = s.centroids + d
        # J = I + sum_m c_m ((cos_m(f) - cos_m(0)) w_m)^T per point
        J = np.eye(3)[None] + np.einsum("nm,mi,mj->nij", cosv, cvec, w)
        Jit = np.linalg.inv(J).transpose(0, 2, 1)
        m = np.einsum("nij,nj->ni", Jit, s.normals)
        mn = np.linalg.norm(m, axis=1)
        nrm = m / mn[:, None]
        area = s.areas * np.linalg.det(J) * mn
        dq, _ = disp(q0[:, :3])
        q = q0.copy()
        q[:, :3] += dq
        jit = rng.normal(0.0, q_sigma, size=q.shape[0])
        q[:, 3] += jit - jit.mean()
        frames.append(Problem(f"{base.name}_frame{f}", Surface(np.ascontiguousarray(cen), np.ascontiguousarray(nrm),
                                                                np.ascontiguousarray(area)),
                              q, base.eps1, base.eps2, base.kappa, base.sphere_radius))
    return frames
