"""FP64 CPU oracle for the truncated multipole operators of the PM-FMM short
range (arXiv:2107.14008, Section 2: P2M, M2L with the truncated prefactors
f_(n), L2P).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` and the CPU legs of ``bench.py``
may import this module.  It shares no code with the CUDA library.

Kernel: psi(r) = erfc(r / 2 r_s) / r, the short-range potential per unit mass
(the acceleration it gives, G m grad psi(x - x_j), is the pair force of Eq.
tr).  Its prefactors f_(k) = (1/r d/dr)^k psi are the paper's f_(n) (the
closed form is in the C oracle, ``oracle.prefactor``).  Because psi depends on
s = r^2/2 only, and d/ds = (1/r) d/dr, every Cartesian derivative is a
polynomial in R times the f_(k):

  D_n(R) = d^n psi(R) = sum_{j <= n/2} prod_a n_a! / (2^j_a j_a! (n_a - 2 j_a)!)
                        R^(n - 2j) f_(|n| - |j|)(|R|)

Expansions (multi-indices n, m; |n| = n1 + n2 + n3 <= p; n! = n1! n2! n3!):
  P2M  M_m = sum_j m_j (z_A - x_j)^m / m!             about the source centre z_A
  M2L  L_n = sum_{|m| <= p - |n|} M_m D_{n+m}(z_B - z_A)  about the target centre z_B
  L2P  a_c(x) = G sum_{|k| <= p-1} L_{k + e_c} (x - z_B)^k / k!
so that a(x) approximates G sum_j m_j grad psi(x - x_j) over the source cell
(no cutoff: the operators expand the smooth truncated kernel itself).

Coefficient order (the library's layout too): graded by |n|, then n1
descending, then n2 descending.
"""
import math

import numpy as np

import oracle


def multi_indices(p):
    """All (n1, n2, n3) with n1 + n2 + n3 <= p, in the graded order."""
    out = []
    for k in range(p + 1):
        for a in range(k, -1, -1):
            for b in range(k - a, -1, -1):
                out.append((a, b, k - a - b))
    return out


def _fact(n):
    return math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2])


def prefactors(r, r_s, kmax):
    """f_(0..kmax)(r) for psi = erfc(r/2 r_s)/r (f_(0) = psi)."""
    f = [math.erfc(r / (2.0 * r_s)) / r]
    for k in range(1, kmax + 1):
        f.append(oracle.prefactor(k, r, r_s))
    return f


def derivatives(R, r_s, order):
    """D_n(R) for every |n| <= order (dict keyed by n), from the f_(k)."""
    R = np.asarray(R, dtype=np.float64)
    r = float(np.sqrt(np.sum(R * R)))
    f = prefactors(r, r_s, order)
    D = {}
    for n in multi_indices(order):
        s = 0.0
        for j0 in range(n[0] // 2 + 1):
            for j1 in range(n[1] // 2 + 1):
                for j2 in range(n[2] // 2 + 1):
                    j = (j0, j1, j2)
                    c = 1.0
                    mono = 1.0
                    for a in range(3):
                        c *= math.factorial(n[a]) / (2.0 ** j[a] * math.factorial(j[a]) *
                                                     math.factorial(n[a] - 2 * j[a]))
                        mono *= R[a] ** (n[a] - 2 * j[a])
                    s += c * mono * f[sum(n) - sum(j)]
        D[n] = s
    return D


def p2m(pos, mass, centre, p):
    """Multipole moments M_m = sum_j m_j (z_A - x_j)^m / m!, graded order."""
    v = np.asarray(centre, dtype=np.float64)[None, :] - np.asarray(pos, dtype=np.float64)
    m = np.asarray(mass, dtype=np.float64)
    return np.array([np.sum(m * np.prod(v ** np.array(n), axis=1)) / _fact(n)
                     for n in multi_indices(p)])


def m2l(M, R, r_s, p):
    """Local coefficients L_n about z_B from moments M about z_A, R = z_B - z_A."""
    idx = multi_indices(p)
    D = derivatives(R, r_s, 2 * p)
    L = np.zeros(len(idx))
    for a, n in enumerate(idx):
        for b, m in enumerate(idx):
            if sum(n) + sum(m) <= p:
                L[a] += M[b] * D[(n[0] + m[0], n[1] + m[1], n[2] + m[2])]
    return L


def l2p(L, centre, pos, p, G=1.0):
    """Accelerations G grad of sum_n L_n (x - z_B)^n / n! at the positions."""
    idx = multi_indices(p)
    where = {n: a for a, n in enumerate(idx)}
    u = np.asarray(pos, dtype=np.float64) - np.asarray(centre, dtype=np.float64)[None, :]
    acc = np.zeros((len(u), 3))
    for k in multi_indices(p - 1):
        mono = np.prod(u ** np.array(k), axis=1) / _fact(k)
        for c in range(3):
            kc = list(k)
            kc[c] += 1
            acc[:, c] += L[where[tuple(kc)]] * mono
    return G * acc


def direct(src_pos, src_mass, targets, r_s, G=1.0):
    """G sum_j m_j grad psi(x - x_j) with no cutoff (what the operators expand)."""
    t = np.asarray(targets, dtype=np.float64)
    acc = np.zeros((len(t), 3))
    for x, m in zip(np.asarray(src_pos, dtype=np.float64), np.asarray(src_mass, dtype=np.float64)):
        d = t - x[None, :]
        r = np.sqrt(np.sum(d * d, axis=1))
        f1 = np.array([oracle.prefactor(1, ri, r_s) for ri in r])
        acc += G * m * f1[:, None] * d
    return acc
