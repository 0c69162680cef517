"""The seeded input generators: shapes, closure, orientation and determinism."""
import math
from collections import Counter

import numpy as np
import pytest

import pb_inputs as pi


@pytest.mark.parametrize("level", [0, 1, 3])
def test_icosphere_counts_orientation_and_area(level):
    s = pi.icosphere(2.5, level)
    assert s.n == 20 * 4 ** level
    assert np.allclose(np.linalg.norm(s.vertices, axis=1), 2.5)
    assert np.all(np.einsum("ij,ij->i", s.normals, s.centroids) > 0)       # outward
    assert np.allclose(np.linalg.norm(s.normals, axis=1), 1.0)
    assert 0.6 * 4 * math.pi * 2.5 ** 2 < s.areas.sum() < 4 * math.pi * 2.5 ** 2
    assert pi.enclosed_volume(s) > 0


def _edge_use(faces):
    c = Counter()
    for a, b, d in faces:
        for e in ((a, b), (b, d), (d, a)):
            c[e] += 1
    return c


def test_icosphere_is_closed_and_consistently_oriented():
    use = _edge_use(pi.icosphere(1.0, 2).faces)
    assert all(v == 1 for v in use.values())
    assert all((b, a) in use for (a, b) in use)


def test_solute_isosurface_is_closed_oriented_and_encloses_its_atoms():
    import oracle
    p = pi.protein_like(n_atoms=12, seed=5, target_triangles=None, spacing=1.5)
    use = _edge_use(p.surface.faces)
    assert all(v == 1 for v in use.values())
    assert all((b, a) in use for (a, b) in use)
    g = oracle.gauss_sums(p.surface, p.charges[:, :3])
    assert np.all(np.abs(g + 1.0) < 0.02)
    assert abs(round(p.charges[:, 3].sum()) - p.charges[:, 3].sum()) < 1e-12


def test_coarse_solute_mesh_has_no_folded_facets():
    """At about 40 triangles per atom (grid spacing near 1.9 A) every facet is
    oriented like the smooth surface through it: its geometric normal makes an
    acute angle with -grad f at its centroid (the element normal)."""
    p = pi.protein_like(n_atoms=150, seed=1010, target_triangles=6000)
    s = p.surface
    v = s.vertices[s.faces]
    fn = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    fn /= np.linalg.norm(fn, axis=1)[:, None]
    cos = np.einsum("ij,ij->i", fn, s.normals)
    assert cos.min() > 0.2
    h = np.sqrt(s.areas.mean())
    assert s.areas.min() > 0.02 * h * h


def test_generators_are_deterministic():
    a = pi.ball_charges(20, 16.0, 2)
    b = pi.ball_charges(20, 16.0, 2)
    assert np.array_equal(a, b)
    assert np.all(np.linalg.norm(a[:, :3], axis=1) <= 16.0)
    assert np.all(np.abs(a[:, 3]) <= 1.0)
    p1, r1, q1 = pi.compact_chain(40, 9)
    p2, r2, q2 = pi.compact_chain(40, 9)
    assert np.array_equal(p1, p2) and np.array_equal(q1, q2)
    d = np.linalg.norm(np.diff(p1, axis=0), axis=1)
    assert np.allclose(d, 3.8)
    dm = np.linalg.norm(p1[:, None] - p1[None], axis=2) + np.eye(40) * 10
    assert dm.min() >= 3.0 - 1e-9


def test_charge_variants():
    base = pi.ball_charges(40, 10.0, 1)
    v = pi.charge_variants(base, 8, seed=4)
    assert v.shape == (8, 40, 4)
    assert np.array_equal(v[0], base)
    for r in range(1, 8):
        diff = v[r, :, 3] - base[:, 3]
        assert np.count_nonzero(diff) == 2
        assert np.allclose(np.abs(diff[diff != 0]), 0.5)
        assert np.array_equal(v[r, :, :3], base[:, :3])


def test_helix_charges():
    h = pi.helix_charges()
    assert h.shape == (9, 4)
    assert np.allclose(h[:, 3], np.arange(1, 10) / 10)
    assert np.allclose(h[-1, :3], [3 / (4 * math.pi), 0.0, 2.0])


def test_md_frames_are_small_smooth_perturbations_keeping_charges_inside():
    import oracle
    base = pi.protein_like(n_atoms=8, seed=1, target_triangles=None, spacing=1.6)
    frames = pi.md_frames(base, 4)
    assert np.array_equal(frames[0].surface.centroids, base.surface.centroids)
    disp = [float(np.abs(f.surface.centroids - base.surface.centroids).max()) for f in frames]
    assert disp[0] == 0.0 and 0.0 < disp[1] < disp[2] < disp[3] < 0.5
    for f in frames:
        assert np.allclose(np.linalg.norm(f.surface.normals, axis=1), 1.0)
        assert np.all(f.surface.areas > 0)
        assert abs(f.surface.areas.sum() / base.surface.areas.sum() - 1.0) < 0.01
        assert f.charges[:, 3].sum() == pytest.approx(base.charges[:, 3].sum(), abs=1e-12)
        g = oracle.gauss_sums(f.surface, f.charges[:, :3])
        assert np.all(np.abs(g + 1.0) < 0.02)          # every charge still inside
