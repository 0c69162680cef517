"""FP64 CPU oracle for the direct-sum boundary-integral linear PB method.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only code that may import this package.  It shares no
code with the CUDA library and is never a fallback for it.

What it computes, with the passage each function follows:
  kernels / green        Eq. (5) and the kernels K1..K4 of Eq. (10)
  matvec / matvec_rows   the discrete product Au of Eqs. (12)-(13)
  assemble               the same A as a dense 2N x 2N matrix
  source                 b = [S1(x_i); S2(x_i)] of Eq. (11)
  reaction_energy        E_sol of Eq. (14), in kcal/mol
  gmres                  restarted GMRES (Saad & Schultz), x0 = 0, restart from the
                         previous approximation (Section 2.4)
  solve / solve_dense    GMRES or dense LU on Au = b, then Eq. (14)
  kirkwood_*             the analytic spherical-cavity solution (Section 3.2)
  error_linf / order     Eqs. (15)-(16)
  yl_*                   the straightforward system of Eqs. (6)-(7) (Yoon and
                         Lenhoff), which the paper sets aside as ill-conditioned:
                         a CPU-only conditioning contrast, not on the GPU path

Readings where the paper is silent or inconsistent:
  * eps = eps2/eps1 (the text after Eq. (11) prints eps1/eps2; only eps2/eps1
    makes Eqs. (8)-(9) follow from Eqs. (6)-(7) with the jump conditions (3)).
  * S1, S2 carry Q_k/eps1 (Eq. (1) has eps1 on its left-hand side).
  * kappa in G_kappa is the inverse Debye length (A^-1).
  * E[kcal/mol] = 4 pi * 332.0636 * (1/2) sum_k Q_k phi_reac(x_k), since G0
    carries 1/(4 pi) and e_c^2/(4 pi eps_0 A) = 332.0636 kcal/mol.
"""
from __future__ import annotations

import ctypes
import math
from fractions import Fraction

import numpy as np

from . import build as _build

COULOMB_KCAL = 332.0636          # e_c^2 / (4 pi eps_0 * 1 Angstrom) in kcal/mol
ENERGY_FACTOR = 4.0 * math.pi * COULOMB_KCAL

_LIB = None
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        lib.oracle_green.argtypes = [_D, _D, _D, _D, ctypes.c_double, _D]
        lib.oracle_kernels.argtypes = [_D, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_matvec.argtypes = [_I64, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.oracle_matvec_rows.argtypes = [_I64, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D,
                                           _I64, ctypes.POINTER(ctypes.c_int64), _D]
        lib.oracle_assemble.argtypes = [_I64, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_source.argtypes = [_I64, _D, _D, _I64, _D, ctypes.c_double, _D]
        lib.oracle_energy.argtypes = [_I64, _D, _D, _D, _I64, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.oracle_energy.restype = ctypes.c_double
        lib.oracle_gauss.argtypes = [_I64, _D, _D, _D, _I64, _D, _D]
        lib.oracle_yl_matvec.argtypes = [_I64, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.oracle_yl_energy.argtypes = [_I64, _D, _D, _D, _I64, _D, _D]
        lib.oracle_yl_energy.restype = ctypes.c_double
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _LIB = lib
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (a timing knob; results do not change)."""
    _lib().oracle_set_num_threads(int(n))


def _geom(surface):
    c = _f64(surface.centroids).reshape(-1, 3)
    n = _f64(surface.normals).reshape(-1, 3)
    a = _f64(surface.areas).reshape(-1)
    if not (c.shape[0] == n.shape[0] == a.shape[0]):
        raise ValueError("centroids, normals and areas disagree in length")
    return c, n, a


# --- Eq. (5), Eq. (10) -------------------------------------------------------
def green(x, nx, y, ny, kappa: float) -> np.ndarray:
    """[G0, Gk, dG0/dny, dGk/dny, dG0/dnx, dGk/dnx, d2G0/dnxdny, d2Gk/dnxdny] at (x, y)."""
    g = np.zeros(8)
    _lib().oracle_green(_p(_f64(x)), _p(_f64(nx)), _p(_f64(y)), _p(_f64(ny)), float(kappa), _p(g))
    return g


def kernels(x, nx, y, ny, eps: float, kappa: float) -> np.ndarray:
    """[K1, K2, K3, K4] of Eq. (10) at target x (normal nx), source y (normal ny)."""
    k = np.zeros(4)
    _lib().oracle_kernels(_p(_f64(x)), _p(_f64(nx)), _p(_f64(y)), _p(_f64(ny)), float(eps), float(kappa), _p(k))
    return k


# --- Eqs. (11)-(14) ------------------------------------------------------------
def matvec(surface, eps: float, kappa: float, u) -> np.ndarray:
    c, n, a = _geom(surface)
    u = _f64(u)
    N = a.shape[0]
    if u.shape != (2 * N,):
        raise ValueError("u must have length 2N")
    y = np.empty(2 * N)
    _lib().oracle_matvec(N, _p(c), _p(n), _p(a), float(eps), float(kappa), _p(u), _p(y))
    return y


def matvec_rows(surface, eps: float, kappa: float, u, rows) -> tuple[np.ndarray, np.ndarray]:
    """Rows i and N+i of Au for each i in ``rows``: returns (y[rows], y[N+rows])."""
    c, n, a = _geom(surface)
    u = _f64(u)
    N = a.shape[0]
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.empty(2 * rows.size)
    _lib().oracle_matvec_rows(N, _p(c), _p(n), _p(a), float(eps), float(kappa), _p(u), rows.size,
                              rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(out))
    return out[0::2].copy(), out[1::2].copy()


def assemble(surface, eps: float, kappa: float) -> np.ndarray:
    c, n, a = _geom(surface)
    N = a.shape[0]
    A = np.empty((2 * N, 2 * N))
    _lib().oracle_assemble(N, _p(c), _p(n), _p(a), float(eps), float(kappa), _p(A))
    return A


def source(surface, charges, eps1: float) -> np.ndarray:
    c, n, _ = _geom(surface)
    ch = _f64(charges).reshape(-1, 4)
    N = c.shape[0]
    b = np.empty(2 * N)
    _lib().oracle_source(N, _p(c), _p(n), ch.shape[0], _p(ch), float(eps1), _p(b))
    return b


def reaction_potential(surface, charges, eps: float, kappa: float, u) -> np.ndarray:
    """phi_reac(x_k) for every charge (Eq. (14), the integral part), in e_c/A units
    that include the 1/(4 pi) of G0."""
    c, n, a = _geom(surface)
    ch = _f64(charges).reshape(-1, 4)
    out = np.empty(ch.shape[0])
    _lib().oracle_energy(a.shape[0], _p(c), _p(n), _p(a), ch.shape[0], _p(ch), float(eps), float(kappa),
                         _p(_f64(u)), _p(out))
    return out


def reaction_energy(surface, charges, eps: float, kappa: float, u) -> float:
    """E_sol of Eq. (14) in kcal/mol."""
    c, n, a = _geom(surface)
    ch = _f64(charges).reshape(-1, 4)
    e = _lib().oracle_energy(a.shape[0], _p(c), _p(n), _p(a), ch.shape[0], _p(ch), float(eps), float(kappa),
                             _p(_f64(u)), None)
    return ENERGY_FACTOR * e


def gauss_sums(surface, points) -> np.ndarray:
    """sum_j W_j dG0(p, x_j)/dnu_j at each point p."""
    c, n, a = _geom(surface)
    pts = _f64(points).reshape(-1, 3)
    out = np.empty(pts.shape[0])
    _lib().oracle_gauss(a.shape[0], _p(c), _p(n), _p(a), pts.shape[0], _p(pts), _p(out))
    return out


# --- GMRES ---------------------------------------------------------------------
def gmres(apply_A, b, restart: int = 10, tol: float = 1e-10, maxit: int = 1000, x0=None,
          callback=None):
    """Restarted GMRES(m) of Saad & Schultz: modified Gram-Schmidt Arnoldi, Givens
    rotations, back substitution, x += V y.  Unpreconditioned; starts from x0
    (zero by default) and restarts from the current approximation.  Stops when
    the true relative residual ||b - Ax|| / ||b|| <= tol, checked at every restart;
    inside a cycle the Givens estimate ends the cycle early.  One iteration is one
    Arnoldi step (one product with A).

    ``callback(x, iterations, rel_resid)``, if given, is called after each true
    residual (at every restart) and does not change the iteration: a run
    restarted from that x continues exactly as the uninterrupted one would.

    Returns (x, iterations, history of true relative residuals, converged)."""
    b = _f64(b)
    n = b.size
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), 0, [0.0], True
    m = int(restart)
    iters = 0
    history = []
    converged = False
    first = True
    while True:
        r = b.copy() if (first and x0 is None) else b - apply_A(x)
        first = False
        beta = float(np.linalg.norm(r))
        history.append(beta / bnorm)
        if callback is not None:
            callback(x, iters, beta / bnorm)
        if not np.isfinite(beta):
            break
        if beta / bnorm <= tol:
            converged = True
            break
        if iters >= maxit:
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply_A(V[k])
            iters += 1
            for i in range(k + 1):
                H[i, k] = float(np.dot(V[i], w))
                w = w - H[i, k] * V[i]
            H[k + 1, k] = float(np.linalg.norm(w))
            breakdown = H[k + 1, k] == 0.0
            if not breakdown:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            d = math.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / d
            sn[k] = H[k + 1, k] / d
            H[k, k] = d
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            if abs(g[k + 1]) / bnorm <= tol or iters >= maxit or breakdown:
                break
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):
            y[i] = (g[i] - float(np.dot(H[i, i + 1:k_used], y[i + 1:]))) / H[i, i]
        x = x + V[:k_used].T @ y
    return x, iters, history, converged


def solve(surface, charges, eps1: float, eps2: float, kappa: float, restart: int = 10,
          tol: float = 1e-10, maxit: int = 1000, x0=None, callback=None) -> dict:
    """b from Eq. (11), GMRES on Eqs. (12)-(13), E_sol from Eq. (14)."""
    eps = eps2 / eps1
    b = source(surface, charges, eps1)
    u, iters, hist, conv = gmres(lambda v: matvec(surface, eps, kappa, v), b, restart, tol, maxit, x0,
                                 callback)
    E = reaction_energy(surface, charges, eps, kappa, u)
    return {"u": u, "b": b, "energy": E, "iters": iters, "history": hist, "converged": conv}


def solve_dense(surface, charges, eps1: float, eps2: float, kappa: float) -> dict:
    """Assemble A and solve with LU (small N only)."""
    eps = eps2 / eps1
    b = source(surface, charges, eps1)
    A = assemble(surface, eps, kappa)
    u = np.linalg.solve(A, b)
    return {"u": u, "b": b, "A": A, "energy": reaction_energy(surface, charges, eps, kappa, u)}


# --- the straightforward (Yoon-Lenhoff) system, a conditioning contrast ----------
def yl_matvec(surface, eps: float, kappa: float, u) -> np.ndarray:
    """The collocated Eqs. (6)-(7) on the surface (see oracle_yl_matvec)."""
    c, n, a = _geom(surface)
    u = _f64(u)
    N = a.shape[0]
    if u.shape != (2 * N,):
        raise ValueError("u must have length 2N")
    y = np.empty(2 * N)
    _lib().oracle_yl_matvec(N, _p(c), _p(n), _p(a), float(eps), float(kappa), _p(u), _p(y))
    return y


def yl_assemble(surface, eps: float, kappa: float) -> np.ndarray:
    """The straightforward system's dense matrix, column by column (small N)."""
    N = _geom(surface)[2].shape[0]
    A = np.empty((2 * N, 2 * N))
    e = np.zeros(2 * N)
    for j in range(2 * N):
        e[j] = 1.0
        A[:, j] = yl_matvec(surface, eps, kappa, e)
        e[j] = 0.0
    return A


def yl_solve(surface, charges, eps1: float, eps2: float, kappa: float, restart: int = 10, tol: float = 1e-10,
             maxit: int = 5000) -> dict:
    """b = [S1; 0], GMRES on the straightforward system, and its reaction energy (kcal/mol)."""
    eps = eps2 / eps1
    c, n, a = _geom(surface)
    ch = _f64(charges).reshape(-1, 4)
    N = a.shape[0]
    b = np.concatenate([source(surface, charges, eps1)[:N], np.zeros(N)])
    u, iters, hist, conv = gmres(lambda v: yl_matvec(surface, eps, kappa, v), b, restart, tol, maxit)
    e = _lib().oracle_yl_energy(N, _p(c), _p(n), _p(a), ch.shape[0], _p(ch), _p(_f64(u)))
    return {"u": u, "b": b, "energy": ENERGY_FACTOR * e, "iters": iters, "history": hist, "converged": conv}


# --- analytic spherical cavity (Kirkwood) ---------------------------------------
def born_energy(Q: float, a: float, eps1: float, eps2: float, kappa: float) -> float:
    """One charge Q at the centre of a sphere of radius a, kcal/mol."""
    return -0.5 * COULOMB_KCAL * Q * Q * (1.0 / (eps1 * a) - 1.0 / (eps2 * a * (1.0 + kappa * a)))


def khat_coeffs(n: int) -> list[float]:
    """Coefficients of the polynomial khat_n(x) = sum_s 2^s n! (2n-s)! / (s! (2n)! (n-s)!) x^s,
    with e^-x khat_n(x) / x^(n+1) proportional to the modified spherical Bessel
    function k_n(x) and khat_n(0) = 1."""
    out = []
    for s in range(n + 1):
        f = Fraction(2 ** s * math.factorial(n) * math.factorial(2 * n - s),
                     math.factorial(s) * math.factorial(2 * n) * math.factorial(n - s))
        out.append(float(f))
    return out


def kirkwood_g(n: int, x: float) -> float:
    """g_n = a f_n'(a) / f_n(a) for the decaying exterior radial solution
    f_n(r) = e^{-kappa r} khat_n(kappa r) / r^{n+1}, x = kappa a."""
    if x == 0.0:
        return -(n + 1.0)
    c = khat_coeffs(n)
    k = sum(cs * x ** s for s, cs in enumerate(c))
    kp = sum(s * cs * x ** (s - 1) for s, cs in enumerate(c) if s > 0)
    return -(n + 1.0) - x + x * kp / k


def kirkwood_R(n: int, a: float, eps1: float, eps2: float, kappa: float) -> float:
    """Reaction coefficient of order n: the interior reaction field of a source
    multipole E_n r^-(n+1) is E_n R_n r^n / a^(2n+1)."""
    g = kirkwood_g(n, kappa * a)
    return (eps2 * g + (n + 1) * eps1) / (n * eps1 - eps2 * g)


def _cos_matrix(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    rp = np.linalg.norm(p, axis=1)
    rq = np.linalg.norm(q, axis=1)
    dot = p @ q.T
    den = np.outer(rp, rq)
    with np.errstate(invalid="ignore", divide="ignore"):
        cg = np.where(den > 0, dot / np.where(den > 0, den, 1.0), 1.0)
    return np.clip(cg, -1.0, 1.0)


def kirkwood_energy(charges, a: float, eps1: float, eps2: float, kappa: float, L: int = 60) -> float:
    """Solvation energy (kcal/mol) of point charges inside a sphere of radius a
    centred at the origin: matching interior and exterior series at r = a
    term by term in Legendre order n, truncated at n = L."""
    from scipy.special import eval_legendre
    ch = _f64(charges).reshape(-1, 4)
    pos, Q = ch[:, :3], ch[:, 3]
    r = np.linalg.norm(pos, axis=1)
    if np.any(r >= a):
        raise ValueError("all charges must lie strictly inside the sphere")
    cg = _cos_matrix(pos, pos)
    rr = np.outer(r, r)
    QQ = np.outer(Q, Q)
    total = 0.0
    for n in range(L + 1):
        Rn = kirkwood_R(n, a, eps1, eps2, kappa)
        total += Rn * float(np.sum(QQ * rr ** n * eval_legendre(n, cg))) / a ** (2 * n + 1)
    return 0.5 * COULOMB_KCAL / eps1 * total


def kirkwood_surface(points, charges, a: float, eps1: float, eps2: float, kappa: float, L: int = 60):
    """Exact phi and dphi/dnu (interior side) on the sphere r = a in the directions
    of ``points``, in the units of the discrete unknowns (G0 with its 1/(4 pi))."""
    from scipy.special import eval_legendre
    ch = _f64(charges).reshape(-1, 4)
    pos, Q = ch[:, :3], ch[:, 3]
    rk = np.linalg.norm(pos, axis=1)
    pts = _f64(points).reshape(-1, 3)
    cg = _cos_matrix(pts, pos)
    phi = np.zeros(pts.shape[0])
    dphi = np.zeros(pts.shape[0])
    for n in range(L + 1):
        Rn = kirkwood_R(n, a, eps1, eps2, kappa)
        s = (eval_legendre(n, cg) * (Q * rk ** n)[None, :]).sum(1) / (4.0 * math.pi * eps1)
        phi += (1.0 + Rn) * s / a ** (n + 1)
        dphi += (n * Rn - (n + 1)) * s / a ** (n + 2)
    return phi, dphi


def error_linf(phi_num, phi_exact) -> float:
    """Eq. (15): relative L-infinity error of the surface potential."""
    return float(np.max(np.abs(np.asarray(phi_num) - np.asarray(phi_exact))) / np.max(np.abs(phi_exact)))


def order(err_coarse: float, err_fine: float, mesh_ratio: float) -> float:
    """Eq. (16): log base (coarse/fine mesh parameter) of e_coarse / e_fine."""
    return math.log(err_coarse / err_fine) / math.log(mesh_ratio)
