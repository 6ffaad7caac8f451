"""Pins of the truncated multipole oracle (oracle/fmm.py; paper Section 2:
M2L with the truncated prefactors f_(n)) against facts outside its code.

- D_n(R) = d^n psi(R), psi = erfc(r/2 r_s)/r, equals high-precision numerical
  derivatives (mpmath) for every |n| <= 4: pins the radial-derivative formula
  and the paper's closed form for f_(n) together.
- The trace D_(2,0,0) + D_(0,2,0) + D_(0,0,2) is the Laplacian of psi, which
  for r > 0 is 4 pi times a normalised Gaussian of variance 2 r_s^2; it is not
  zero (the paper calls D traceless, which holds for the Newtonian kernel
  only), and in the Newtonian limit r << r_s it does go to zero relative to
  the second derivatives.
- A point mass at the source centre seen at the target centre: L2P gives
  G m f_(1)(R) (-R), the exact pair force, at every order.
- P2M -> M2L -> L2P converges geometrically to the direct sum in the order p.
- The dipole moment about the centre of mass vanishes.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fmm

mp = pytest.importorskip("mpmath")


def _psi_mp(x, y, z, r_s):
    r = mp.sqrt(x * x + y * y + z * z)
    return mp.erfc(r / (2 * r_s)) / r


@pytest.mark.parametrize("R", [(1.3, -0.7, 0.4), (0.35, 0.2, -0.9)])
def test_derivative_tensors_equal_numerical_derivatives(R):
    r_s = 0.8
    D = fmm.derivatives(R, r_s, 4)
    mp.mp.dps = 40
    for n in fmm.multi_indices(4):
        num = mp.diff(lambda x, y, z: _psi_mp(x, y, z, mp.mpf(r_s)),
                      (mp.mpf(R[0]), mp.mpf(R[1]), mp.mpf(R[2])), n)
        assert abs(D[n] - float(num)) <= 1e-9 * max(1.0, abs(float(num))), n


def test_trace_is_the_gaussian_source_and_vanishes_in_the_newtonian_limit():
    r_s = 0.6
    for R in ([0.5, 0.2, -0.3], [1.5, 0.9, 0.4]):
        D = fmm.derivatives(R, r_s, 2)
        r2 = float(np.dot(R, R))
        trace = D[(2, 0, 0)] + D[(0, 2, 0)] + D[(0, 0, 2)]
        gauss = 4.0 * math.pi * (4.0 * math.pi * r_s * r_s) ** -1.5 * math.exp(-r2 / (4 * r_s * r_s))
        assert trace == pytest.approx(gauss, rel=1e-9)
    D = fmm.derivatives([1e-3, 2e-3, -1.5e-3], 10.0, 2)
    trace = D[(2, 0, 0)] + D[(0, 2, 0)] + D[(0, 0, 2)]
    assert abs(trace) < 1e-9 * abs(D[(2, 0, 0)])


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_point_mass_at_the_centres_gives_the_pair_force(p):
    r_s, m = 0.7, 2.5
    zA, R = np.array([0.1, -0.2, 0.3]), np.array([1.1, 0.6, -0.8])
    M = fmm.p2m(zA[None, :], [m], zA, p)
    L = fmm.m2l(M, R, r_s, p)
    a = fmm.l2p(L, zA + R, (zA + R)[None, :], p, G=1.3)[0]
    r = float(np.linalg.norm(R))
    want = 1.3 * m * oracle.prefactor(1, r, r_s) * R  # G m grad psi at R
    assert np.allclose(a, want, rtol=1e-12, atol=0)
    assert np.allclose(a, fmm.direct(zA[None, :], [m], (zA + R)[None, :], r_s, G=1.3)[0],
                       rtol=1e-12, atol=0)


def test_expansion_converges_geometrically_in_the_order():
    rng = np.random.default_rng(0)
    r_s, h = 1.0, 0.5
    src, ms = rng.uniform(-h, h, (40, 3)), rng.uniform(0.5, 1.5, 40)
    R = np.array([2.2, 1.0, -0.6])
    tg = R + rng.uniform(-h, h, (30, 3))
    ref = fmm.direct(src, ms, tg, r_s)
    errs = []
    for p in range(1, 7):
        L = fmm.m2l(fmm.p2m(src, ms, np.zeros(3), p), R, r_s, p)
        a = fmm.l2p(L, R, tg, p)
        errs.append(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2)))
    assert all(e1 < 0.7 * e0 for e0, e1 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2


def test_dipole_about_the_centre_of_mass_vanishes():
    rng = np.random.default_rng(1)
    x, m = rng.random((25, 3)), rng.uniform(0.2, 2.0, 25)
    com = (m[:, None] * x).sum(0) / m.sum()
    M = fmm.p2m(x, m, com, 2)
    assert M[0] == pytest.approx(m.sum(), rel=1e-14)
    assert np.max(np.abs(M[1:4])) < 1e-13 * m.sum()
