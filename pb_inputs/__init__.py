"""Seeded synthetic inputs (surfaces and charge sets) shared by the tests, the
benchmark and the oracle checks.  This package only builds geometry and charges;
it evaluates no part of the boundary-integral method."""
from .charges import ball_charges, charge_variants, compact_chain, helix_charges  # noqa: F401
from .mesh import Surface, enclosed_volume, icosphere, isosurface, triangles_to_surface  # noqa: F401
from .workloads import (EPS1, EPS2, KAPPA, Problem, batch_specs, by_name, helix_sphere,  # noqa: F401
                        kirkwood_sphere_multi, kirkwood_sphere_single, md_frames, protein_like, serve_specs,
                        solute_from_spec)
