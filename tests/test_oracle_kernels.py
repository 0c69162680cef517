"""Pins for the oracle's Green's-function derivatives and kernels K1..K4.

The oracle evaluates closed forms of dG/dnu_x, dG/dnu_y and d2G/dnu_x dnu_y.
These tests check them against central finite differences of the two
fundamental solutions of Eq. (5) themselves, so a dropped term, a wrong sign
or swapped normals in the closed forms fails here.
"""
import math

import numpy as np
import pytest

import oracle


def G0(x, y):
    return 1.0 / (4.0 * math.pi * np.linalg.norm(np.asarray(x) - np.asarray(y)))


def Gk(x, y, kappa):
    d = np.linalg.norm(np.asarray(x) - np.asarray(y))
    return math.exp(-kappa * d) / (4.0 * math.pi * d)


def _unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


def _cases(n=25, seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(n):
        x = rng.normal(size=3)
        y = x + _unit(rng.normal(size=3)) * rng.uniform(0.3, 4.0)
        yield x, _unit(rng.normal(size=3)), y, _unit(rng.normal(size=3)), rng.uniform(0.0, 1.5)


def _fd_first(f, x, nx, y, ny, h=1e-5):
    dny = (f(x, y + h * ny) - f(x, y - h * ny)) / (2 * h)
    dnx = (f(x + h * nx, y) - f(x - h * nx, y)) / (2 * h)
    return dnx, dny


def _fd_mixed(f, x, nx, y, ny, h=2e-4):
    return (f(x + h * nx, y + h * ny) - f(x + h * nx, y - h * ny)
            - f(x - h * nx, y + h * ny) + f(x - h * nx, y - h * ny)) / (4 * h * h)


@pytest.mark.parametrize("case", list(_cases()))
def test_green_derivatives_match_finite_differences(case):
    x, nx, y, ny, kappa = case
    g = oracle.green(x, nx, y, ny, kappa)
    gk = lambda a, b: Gk(a, b, kappa)  # noqa: E731
    assert g[0] == pytest.approx(G0(x, y), rel=1e-14)
    assert g[1] == pytest.approx(gk(x, y), rel=1e-14)
    d0x, d0y = _fd_first(G0, x, nx, y, ny)
    dkx, dky = _fd_first(gk, x, nx, y, ny)
    scale0 = abs(G0(x, y)) / np.linalg.norm(x - y)
    assert abs(g[2] - d0y) < 1e-7 * scale0
    assert abs(g[3] - dky) < 1e-7 * scale0
    assert abs(g[4] - d0x) < 1e-7 * scale0
    assert abs(g[5] - dkx) < 1e-7 * scale0
    scale2 = scale0 / np.linalg.norm(x - y)
    assert abs(g[6] - _fd_mixed(G0, x, nx, y, ny)) < 2e-6 * scale2
    assert abs(g[7] - _fd_mixed(gk, x, nx, y, ny)) < 2e-6 * scale2


@pytest.mark.parametrize("case", list(_cases(12, seed=5)))
def test_kernels_are_the_combinations_of_eq10(case):
    """K1 = G0 - Gk, K2 = eps dGk/dny - dG0/dny, K3 = dG0/dnx - dGk/dnx / eps,
    K4 = d2Gk - d2G0, each checked against finite differences of Eq. (5)."""
    x, nx, y, ny, kappa = case
    eps = 80.0
    K = oracle.kernels(x, nx, y, ny, eps, kappa)
    gk = lambda a, b: Gk(a, b, kappa)  # noqa: E731
    d0x, d0y = _fd_first(G0, x, nx, y, ny)
    dkx, dky = _fd_first(gk, x, nx, y, ny)
    s = abs(G0(x, y)) / np.linalg.norm(x - y)
    assert K[0] == pytest.approx(G0(x, y) - gk(x, y), rel=1e-12, abs=1e-15)
    assert abs(K[1] - (eps * dky - d0y)) < 1e-7 * s * eps
    assert abs(K[2] - (d0x - dkx / eps)) < 1e-7 * s
    assert abs(K[3] - (_fd_mixed(gk, x, nx, y, ny) - _fd_mixed(G0, x, nx, y, ny))) < 4e-6 * s / np.linalg.norm(x - y)


def test_kernel_symmetries():
    """K1 and K4 are symmetric under exchanging (x, nu_x) with (y, nu_y)."""
    for x, nx, y, ny, kappa in _cases(10, seed=3):
        a = oracle.kernels(x, nx, y, ny, 80.0, kappa)
        b = oracle.kernels(y, ny, x, nx, 80.0, kappa)
        assert a[0] == pytest.approx(b[0], rel=1e-13)
        assert a[3] == pytest.approx(b[3], rel=1e-12, abs=1e-15)


def test_kernels_vanish_without_dielectric_jump_or_salt():
    """eps = 1 and kappa = 0 make G_kappa = G0, so K1..K4 are exactly zero."""
    for x, nx, y, ny, _ in _cases(10, seed=9):
        K = oracle.kernels(x, nx, y, ny, 1.0, 0.0)
        assert np.all(K == 0.0)
