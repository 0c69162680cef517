"""Parity checks of a product y = Au block by block.

The two row blocks of Eqs. (12)-(13) differ in size by about the ratio of
their diagonals: the phi rows carry (1+eps)/2 phi_i (40.5 phi_i at eps = 80),
the psi rows (1+1/eps)/2 psi_i (about 0.51 psi_i) plus the K3/K4 sums.  A norm
over the concatenated vector would let the psi block be wrong by far more than
the stated tolerance, so every product is compared per block: a relative L2
bound and an element-wise bound against that block's own largest entry.
"""
import numpy as np

# (relative L2, element-wise against the block's max) per product precision
TOL_FP64 = (1e-10, 1e-9)
TOL_FP32PAIR = (2e-5, 1e-4)


def block_errors(y, ref):
    """[(rel_l2, rel_elem)] for the phi block and the psi block."""
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    n = ref.size // 2
    out = []
    for sl in (slice(0, n), slice(n, 2 * n)):
        d = y[sl] - ref[sl]
        r = ref[sl]
        nr = float(np.linalg.norm(r))
        mr = float(np.max(np.abs(r))) if r.size else 0.0
        out.append((float(np.linalg.norm(d)) / nr if nr > 0 else float(np.linalg.norm(d)),
                    float(np.max(np.abs(d))) / mr if mr > 0 else float(np.max(np.abs(d), initial=0.0))))
    return out


def assert_blocks_close(y, ref, tol, what=""):
    """Both row blocks within (relative L2, element-wise) = tol of ref."""
    y = np.asarray(y, dtype=np.float64)
    assert y.shape == np.shape(ref), what
    assert np.all(np.isfinite(y)), what
    l2, el = tol
    for name, (e2, ee) in zip(("phi", "psi"), block_errors(y, ref)):
        assert e2 <= l2, f"{what} {name} block: relative L2 {e2:.3e} > {l2:g}"
        assert ee <= el, f"{what} {name} block: element-wise {ee:.3e} > {el:g}"


def assert_rows_close(got_phi, got_psi, ref_phi, ref_psi, tol, what=""):
    """Sampled rows: the phi rows and the psi rows compared separately."""
    assert_blocks_close(np.concatenate([got_phi, got_psi]), np.concatenate([ref_phi, ref_psi]), tol, what)
