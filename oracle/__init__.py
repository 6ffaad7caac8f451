"""FP64 CPU oracle for the truncated short-range P2P gravity (arXiv:2107.14008).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2107_14008_gb300``): the pair sums are plain C
(``psr_oracle.c``), the finite-difference helper below is numpy.  The product
path never calls it.

Definitions (paper, Section 2): x = r/(2 r_s); T(x) = erfc(x) + (2x/sqrt(pi))
exp(-x^2) (Eq. tr); pair acceleration G m_j d T/|d|^3 with d = x_j + nL - x_i,
summed over all periodic images with 0 < |d| < r_c.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)
_LP = ctypes.POINTER(ctypes.c_int64)

T_EXACT, T_LINEAR, T_CUBIC, T_TAYLOR = 0, 1, 2, 3


def lib():
    """Load (building on first use) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_T.restype = ctypes.c_double
        L.oracle_T.argtypes = [ctypes.c_double]
        L.oracle_E.restype = ctypes.c_double
        L.oracle_E.argtypes = [ctypes.c_double]
        L.oracle_prefactor.restype = ctypes.c_double
        L.oracle_prefactor.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.oracle_prefactor_newton.restype = ctypes.c_double
        L.oracle_prefactor_newton.argtypes = [ctypes.c_int, ctypes.c_double]
        L.oracle_T_interp.restype = ctypes.c_double
        L.oracle_T_interp.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int]
        L.oracle_T_array.restype = None
        L.oracle_T_array.argtypes = [_I64, _DP, _DP, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int]
        L.oracle_forces.restype = ctypes.c_int
        L.oracle_forces.argtypes = [_I64, _DP, _DP, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, _I64, _LP, _DP, _LP, _LP,
                                    ctypes.c_int, ctypes.c_int]
        L.oracle_adjoint.restype = ctypes.c_int
        L.oracle_adjoint.argtypes = [_I64, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _I64, _LP, _DP, _DP,
                                     ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _lp(a):
    return a.ctypes.data_as(_LP)


def default_threads():
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
               else (os.cpu_count() or 1))


def T(x, mode=T_EXACT, table_n=1024, x_c=2.25, level=4):
    """T(x) (Eq. tr) or one of its interpolants, elementwise, FP64."""
    x = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    out = np.empty_like(x)
    lib().oracle_T_array(x.size, _dp(x), _dp(out), int(mode), int(table_n), float(x_c),
                         int(level))
    return out


def E(x):
    """E(x) = -4 exp(-x^2)/sqrt(pi) (Section 3.3)."""
    return lib().oracle_E(float(x))


def prefactor(n, r, r_s):
    """Truncated prefactor f_(n)(r) of Section 2 (general n)."""
    return lib().oracle_prefactor(int(n), float(r), float(r_s))


def prefactor_newton(n, r):
    """Newtonian prefactor f^inv_(n)(r) = (-1)^n (2n-1)!!/r^(2n+1)."""
    return lib().oracle_prefactor_newton(int(n), float(r))


def _prep(pos, mass, L):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mass = np.ascontiguousarray(mass, dtype=np.float64).reshape(-1)
    if mass.shape[0] != pos.shape[0]:
        raise ValueError("mass and pos lengths differ")
    return pos, mass


def forces(pos, mass, L, r_s, r_c, G=1.0, targets=None, t_mode=T_EXACT, table_n=1024,
           level=4, cells=False, threads=None):
    """Accelerations a_i of the listed targets (all if None), FP64.

    Returns (acc[n_t,3], pairs[n_t], zero_pairs[n_t]): `pairs` counts the
    within-cutoff images summed, `zero_pairs` the distinct pairs at r == 0.
    """
    pos, mass = _prep(pos, mass, L)
    n = pos.shape[0]
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = targets.size, _lp(targets)
    acc = np.zeros((nt, 3))
    pairs = np.zeros(nt, dtype=np.int64)
    zero = np.zeros(nt, dtype=np.int64)
    rc = lib().oracle_forces(n, _dp(pos), _dp(mass), L, r_s, r_c, G, int(t_mode),
                             int(table_n), int(level), nt, tp, _dp(acc), _lp(pairs),
                             _lp(zero), int(bool(cells)), int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_forces failed (%d): need 0 < r_c <= L, pos in [0,L)" % rc)
    return acc, pairs, zero


def adjoint(pos, mass, cot, L, r_s, r_c, G=1.0, targets=None, cells=False, threads=None):
    """dL/dx (n_t x 3) and dL/dm (n_t) of L = sum_i cot_i . a_i, FP64, exact T."""
    pos, mass = _prep(pos, mass, L)
    cot = np.ascontiguousarray(cot, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = targets.size, _lp(targets)
    gx = np.zeros((nt, 3))
    gm = np.zeros(nt)
    rc = lib().oracle_adjoint(n, _dp(pos), _dp(mass), _dp(cot), L, r_s, r_c, G, nt, tp,
                              _dp(gx), _dp(gm), int(bool(cells)),
                              int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_adjoint failed (%d)" % rc)
    return gx, gm


# ------------------------------------------------------------------------------
# Finite differences of the loss with the set of interacting pairs frozen.
# Only pairs that touch particle p depend on x_p or m_p, so
#   L_p(x_p) = G sum_{(j,n) within r_c at the unperturbed positions}
#              g(r_pj) d_pj . (m_j c_p - m_p c_j),   d_pj = x_j + nL - x_p,
# where the first term is c_p . a_p and the second collects c_j . a_j's term
# from source p (d_jp = -d_pj).  T is evaluated with scipy's erfc.
# ------------------------------------------------------------------------------

def _neighbours(pos, p, L, r_c):
    d0 = pos - pos[p]
    js, ds = [], []
    for nx in (-1, 0, 1):
        for ny in (-1, 0, 1):
            for nz in (-1, 0, 1):
                d = d0 + np.array([nx, ny, nz], dtype=np.float64) * L
                r2 = np.einsum("ij,ij->i", d, d)
                ok = (r2 < r_c * r_c) & (r2 > 0.0)
                idx = np.nonzero(ok)[0]
                js.append(idx)
                ds.append(np.repeat(np.array([[nx, ny, nz]], dtype=np.float64), idx.size, 0))
    return np.concatenate(js), np.concatenate(ds)


def local_loss_factory(pos, mass, cot, p, L, r_s, r_c, G=1.0):
    """Return f(x_p, m_p) -> L_p on the pair set frozen at the given positions."""
    from scipy.special import erfc
    pos = np.asarray(pos, dtype=np.float64)
    js, shifts = _neighbours(pos, p, L, r_c)
    xj = pos[js] + shifts * L
    mj = np.asarray(mass, dtype=np.float64)[js]
    cj = np.asarray(cot, dtype=np.float64)[js]
    cp = np.asarray(cot, dtype=np.float64)[p]

    def f(xp, mp):
        d = xj - xp
        r2 = np.einsum("ij,ij->i", d, d)
        r = np.sqrt(r2)
        x = r / (2.0 * r_s)
        Tv = erfc(x) + 2.0 * x / np.sqrt(np.pi) * np.exp(-x * x)
        g = Tv / (r2 * r)
        w = mj[:, None] * cp[None, :] - mp * cj
        return G * np.sum(g * np.einsum("ij,ij->i", d, w))

    return f


def fd_gradient(pos, mass, cot, p, L, r_s, r_c, G=1.0, h=None, richardson=False):
    """Central finite differences of L_p in x_p (3) and m_p, frozen pair set."""
    pos = np.asarray(pos, dtype=np.float64)
    f = local_loss_factory(pos, mass, cot, p, L, r_s, r_c, G)
    h = 1e-6 * L if h is None else h
    xp = pos[p].copy()
    mp = float(mass[p])

    def cd(hh):
        g = np.zeros(3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = hh
            g[a] = (f(xp + e, mp) - f(xp - e, mp)) / (2 * hh)
        return g

    gx = cd(h)
    if richardson:
        gx = (4.0 * cd(h / 2) - gx) / 3.0
    hm = 1e-6 * max(mp, 1e-300)
    gm = (f(xp, mp + hm) - f(xp, mp - hm)) / (2 * hm)
    return gx, gm
