"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: quadrature of
the paper's integral form of T, high-precision derivatives, the paper's
printed Taylor coefficients (tests/golden), the paper's general prefactor
formula, closed-form isolated pairs, and symmetries of the periodic sum.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQRT_PI = math.sqrt(math.pi)


# ----------------------------------------------------------------- T(x) ------

def test_T_matches_integral_form_by_quadrature():
    """Section 3.3: T(x) = (4/sqrt(pi)) int_x^inf u^2 exp(-u^2) du."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    xs = [0.0, 1e-3, 0.1, 0.37, 0.5, 1.0, 1.5, 2.0, 2.25, 3.0, 4.5]
    for x in xs:
        q = mp.quad(lambda u: u * u * mp.exp(-u * u), [x, x + 1, x + 3, mp.inf])
        ref = float(4 / mp.sqrt(mp.pi) * q)
        assert abs(oracle.T(x)[0] - ref) <= 2e-16 * 8 + 1e-15 * ref, x


def test_T_limits_and_small_x_series():
    assert oracle.T(0.0)[0] == 1.0
    assert oracle.T(30.0)[0] == 0.0
    # T(x) = 1 - (4/sqrt(pi)) (x^3/3 - x^5/5 + x^7/14 - ...) from the integral form
    for x in [1e-3, 1e-2, 3e-2]:
        series = 1.0 - 4.0 / SQRT_PI * (x ** 3 / 3.0 - x ** 5 / 5.0 + x ** 7 / 14.0)
        assert abs(oracle.T(x)[0] - series) < 1e-13


def test_T_derivative_is_x2_E():
    """First Taylor term of Eq. (int): dT/dx = x^2 E(x)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    Tm = lambda x: mp.erfc(x) + 2 * x / mp.sqrt(mp.pi) * mp.exp(-x * x)
    for x in [0.2, 0.9, 1.7, 2.2]:
        d = float(mp.diff(Tm, x))
        assert abs(d - x * x * oracle.E(x)) < 1e-14


def _golden_taylor():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_taylor_coefficients.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            rows[int(parts[0])] = [Fraction(p) for p in parts[1:]]
    return rows


def test_paper_taylor_coefficients_are_derivatives_of_T():
    """The printed T_[1..4] of Eq. (int) equal T^(k)(x_i)/k! (golden file)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    Tm = lambda x: mp.erfc(x) + 2 * x / mp.sqrt(mp.pi) * mp.exp(-x * x)
    rows = _golden_taylor()
    assert sorted(rows) == [1, 2, 3, 4]
    for xi in [0.0, 0.3, 1.0, 1.4, 2.0, 2.9]:
        Ei = -4 * mp.exp(-mp.mpf(xi) ** 2) / mp.sqrt(mp.pi)
        for k, coef in rows.items():
            poly = sum(mp.mpf(c.numerator) / c.denominator * mp.mpf(xi) ** p
                       for p, c in enumerate(coef))
            deriv = mp.diff(Tm, mp.mpf(xi), k) / mp.factorial(k)
            assert abs(float(poly * Ei - deriv)) < 1e-25, (k, xi)


def test_oracle_taylor_table_follows_eq_int():
    """Mode 3 of the oracle is the truncated series of Eq. (int) about the
    nearest node: compare with mpmath's Taylor polynomial of T."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    Tm = lambda x: mp.erfc(x) + 2 * x / mp.sqrt(mp.pi) * mp.exp(-x * x)
    N, xc = 512, 3.0
    h = xc / N
    rng = np.random.default_rng(1)
    for x in rng.uniform(0.0, 2.99, 12):
        k = int(math.floor(x / h + 0.5))
        xi = k * h
        eps = x - xi
        coeffs = mp.taylor(Tm, mp.mpf(xi), 4)
        for level in range(5):
            ref = float(sum(coeffs[m] * mp.mpf(eps) ** m for m in range(level + 1)))
            got = oracle.T(x, oracle.T_TAYLOR, N, xc, level)[0]
            assert abs(got - ref) < 2e-15, (x, level)


def test_taylor_table_error_envelope_ordering():
    """Fig. 2 ordering: the max error falls with each added term, and by
    roughly (h/2)^(level+1) per level."""
    x = np.linspace(0.0, 2.999, 200001)
    exact = oracle.T(x)
    errs = [np.max(np.abs(oracle.T(x, oracle.T_TAYLOR, 512, 3.0, lv) - exact))
            for lv in range(5)]
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.05
    assert errs[2] < 1e-7   # "adequate for single precision"
    assert errs[4] < 1e-12  # "for double precision"


@pytest.mark.parametrize("mode,N,bound,order", [
    (oracle.T_LINEAR, 1024, 8.1e-7, 2), (oracle.T_LINEAR, 4096, 5.1e-8, 2),
    (oracle.T_CUBIC, 1024, 8.7e-13, 4), (oracle.T_CUBIC, 256, 2.3e-10, 4)])
def test_interpolation_error_floor(mode, N, bound, order):
    """Linear: max|T''| h^2/8; cubic Hermite: max|T''''| h^4/384, x_c = 2.25."""
    xc = 2.25
    x = np.linspace(0.0, xc * (1 - 1e-9), 400001)
    exact = oracle.T(x)
    e1 = np.max(np.abs(oracle.T(x, mode, N, xc) - exact))
    e2 = np.max(np.abs(oracle.T(x, mode, 2 * N, xc) - exact))
    assert e1 <= bound
    ratio = e1 / max(e2, 1e-300)
    assert 0.7 * 2 ** order < ratio < 1.3 * 2 ** order or e2 < 1e-15
    # beyond the cutoff every interpolant is zero
    assert oracle.T(xc, mode, N, xc)[0] == 0.0


# --------------------------------------------------------- prefactors --------

def test_prefactor_n1_is_minus_T_over_r3():
    """The paper's f_(n) at n = 1 reduces to -T/r^3 (force of Section 2)."""
    r_s = 3.75
    for r in [0.01, 0.5, 3.0, 7.5, 16.0]:
        x = r / (2 * r_s)
        assert math.isclose(oracle.prefactor(1, r, r_s), -oracle.T(x)[0] / r ** 3,
                            rel_tol=1e-13)


def test_prefactor_newtonian_limit():
    """f_(n) -> f^inv_(n) = (-1)^n (2n-1)!!/r^(2n+1) as r/r_s -> 0."""
    r_s = 1.0
    for n in range(1, 5):
        r = 1e-3
        a, b = oracle.prefactor(n, r, r_s), oracle.prefactor_newton(n, r)
        assert abs(a / b - 1.0) < 1e-8, n


def test_prefactor_recursion_f2_is_derivative_of_f1():
    """f_(2) = (1/r) d f_(1)/dr: the tidal term used by the adjoint."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    r_s = mp.mpf("2.5")

    def f1(r):
        x = r / (2 * r_s)
        return -(mp.erfc(x) + 2 * x / mp.sqrt(mp.pi) * mp.exp(-x * x)) / r ** 3

    for r in [0.05, 1.0, 4.0, 9.0]:
        ref = float(mp.diff(f1, mp.mpf(r)) / r)
        got = oracle.prefactor(2, r, float(r_s))
        assert abs(got / ref - 1.0) < 1e-12


# ------------------------------------------------------------ pair sums -------

def _two(d, m=(0.7, 0.3), L=1000.0, r_s=3.0, r_c=13.5, base=(500.0, 500.0, 500.0)):
    p0 = np.array(base)
    pos = np.stack([p0, p0 + np.asarray(d, dtype=np.float64)])
    return pos, np.array(m), L, r_s, r_c


def _T_ref(x):
    from scipy.special import erfc
    return erfc(x) + 2 * x / SQRT_PI * math.exp(-x * x)


def test_isolated_pair_closed_form_and_sign():
    """a_0 = G m_1 d T/r^3 towards particle 1, a_1 = -G m_0 d T/r^3."""
    d = np.array([2.0, -1.0, 0.5])
    pos, m, L, r_s, r_c = _two(d)
    G = 2.5
    acc, pairs, _ = oracle.forces(pos, m, L, r_s, r_c, G)
    r = np.linalg.norm(d)
    g = _T_ref(r / (2 * r_s)) / r ** 3
    np.testing.assert_allclose(acc[0], G * m[1] * g * d, rtol=1e-14)
    np.testing.assert_allclose(acc[1], -G * m[0] * g * d, rtol=1e-14)
    assert np.dot(acc[0], d) > 0  # attractive
    assert list(pairs) == [1, 1]


def test_isolated_pair_cutoff_is_hard_and_strict():
    r_c = 13.5
    for r, inside in [(r_c * (1 - 1e-12), True), (r_c, False), (r_c * (1 + 1e-9), False)]:
        pos, m, L, r_s, _ = _two([r, 0, 0])
        acc, pairs, _ = oracle.forces(pos, m, L, r_s, r_c)
        assert (np.abs(acc).sum() > 0) == inside
        assert pairs[0] == int(inside)
    # just inside: the jump equals G m T(x_c)/r_c^2
    pos, m, L, r_s, _ = _two([r_c * (1 - 1e-12), 0, 0])
    acc, _, _ = oracle.forces(pos, m, L, r_s, r_c)
    assert math.isclose(acc[0, 0], m[1] * _T_ref(2.25) / r_c ** 2, rel_tol=1e-9)


def test_newtonian_limit_of_pair_force():
    """For r << r_s: |a| = G m/r^2 (1 - (4/(3 sqrt(pi))) x^3 + O(x^5))."""
    r_s = 3.0
    for r in [1e-3, 1e-2, 5e-2]:
        pos, m, L, _, r_c = _two([0, r, 0], r_s=r_s)
        acc, _, _ = oracle.forces(pos, m, L, r_s, r_c)
        x = r / (2 * r_s)
        newton = m[1] / r ** 2
        assert abs(acc[0, 1] / newton - (1 - 4 / (3 * SQRT_PI) * x ** 3)) < 1e-9


def test_periodic_image_across_the_face():
    """A pair straddling x = 0 interacts through the image n = (-1,0,0)."""
    L, r_s, r_c = 100.0, 3.75, 16.875
    pos = np.array([[0.5, 50.0, 50.0], [99.0, 50.0, 50.0]])
    m = np.array([1.0, 1.0])
    acc, pairs, _ = oracle.forces(pos, m, L, r_s, r_c)
    r = 1.5
    g = _T_ref(r / (2 * r_s)) / r ** 3
    np.testing.assert_allclose(acc[0], [-g * r, 0, 0], rtol=1e-14)
    assert list(pairs) == [1, 1]


def _numpy_all_images(pos, mass, L, r_s, r_c, nimg=2):
    """Independent brute force over images n in {-nimg..nimg}^3 (small n)."""
    n = pos.shape[0]
    acc = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    rng = range(-nimg, nimg + 1)
    for i in range(n):
        for nx in rng:
            for ny in rng:
                for nz in rng:
                    d = pos + np.array([nx, ny, nz]) * L - pos[i]
                    r2 = np.einsum("ij,ij->i", d, d)
                    ok = (r2 < r_c * r_c) & (r2 > 0)
                    r = np.sqrt(r2[ok])
                    x = r / (2 * r_s)
                    from scipy.special import erfc
                    Tv = erfc(x) + 2 * x / SQRT_PI * np.exp(-x * x)
                    acc[i] += np.sum((mass[ok] * Tv / r ** 3)[:, None] * d[ok], axis=0)
                    cnt[i] += ok.sum()
    return acc, cnt


def test_images_complete_when_cutoff_exceeds_half_box():
    """r_c = 0.675 L (the smallest boxes of the batch workload): several images
    of one source lie within r_c; {-1,0,1}^3 must find them all."""
    rng = np.random.default_rng(7)
    L = 10.0
    r_c = 0.675 * L
    r_s = r_c / 4.5
    pos = rng.random((40, 3)) * L
    mass = rng.uniform(0.5, 1.5, 40)
    acc, cnt, _ = oracle.forces(pos, mass, L, r_s, r_c)
    ref, rcnt = _numpy_all_images(pos, mass, L, r_s, r_c)
    np.testing.assert_array_equal(cnt, rcnt)
    np.testing.assert_allclose(acc, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def _clustered(n=3000, L=60.0, seed=3):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, 5, rng)
    mass = rng.uniform(0.2, 2.0, n)
    return pos, mass, L


def test_momentum_conservation_unequal_masses():
    pos, mass, L = _clustered()
    r_s = 1.2 * L / 16
    r_c = 4.5 * r_s
    acc, _, _ = oracle.forces(pos, mass, L, r_s, r_c, cells=True)
    tot = (mass[:, None] * acc).sum(0)
    scale = (mass[:, None] * np.abs(acc)).sum(0)
    assert np.all(np.abs(tot) < 1e-13 * scale)


def test_translation_invariance_periodic_shift():
    pos, mass, L = _clustered()
    r_s, r_c = 1.2 * L / 16, 5.4 * L / 16
    a0, _, _ = oracle.forces(pos, mass, L, r_s, r_c, cells=True)
    shifted = np.mod(pos + np.array([17.3, -41.9, 29.05]), L)
    shifted = np.where(shifted >= L, 0.0, shifted)
    a1, _, _ = oracle.forces(shifted, mass, L, r_s, r_c, cells=True)
    # positions are rounded by the shift, so close pairs move by ~1e-16 L
    assert np.sqrt(np.sum((a1 - a0) ** 2) / np.sum(a0 ** 2)) < 1e-10


def test_reflection_flips_accelerations():
    pos, mass, L = _clustered()
    r_s, r_c = 1.2 * L / 16, 5.4 * L / 16
    a0, _, _ = oracle.forces(pos, mass, L, r_s, r_c, cells=True)
    refl = np.mod(L - pos, L)
    refl = np.where(refl >= L, 0.0, refl)
    a1, _, _ = oracle.forces(refl, mass, L, r_s, r_c, cells=True)
    assert np.sqrt(np.sum((a1 + a0) ** 2) / np.sum(a0 ** 2)) < 1e-10


def test_scale_invariance():
    """(x, L, r_s, r_c) -> lam (x, L, r_s, r_c) gives a -> a / lam^2."""
    pos, mass, L = _clustered(n=1500)
    r_s, r_c = 1.2 * L / 16, 5.4 * L / 16
    lam = 3.0
    a0, _, _ = oracle.forces(pos, mass, L, r_s, r_c)
    a1, _, _ = oracle.forces(pos * lam, mass, L * lam, r_s * lam, r_c * lam)
    np.testing.assert_allclose(a1 * lam ** 2, a0, rtol=1e-11, atol=1e-12 * np.abs(a0).max())


def test_linearity_in_source_masses():
    pos, mass, L = _clustered(n=1500)
    r_s, r_c = 1.2 * L / 16, 5.4 * L / 16
    rng = np.random.default_rng(11)
    m2 = rng.uniform(0, 1, mass.size)
    a1, _, _ = oracle.forces(pos, mass, L, r_s, r_c)
    a2, _, _ = oracle.forces(pos, m2, L, r_s, r_c)
    a3, _, _ = oracle.forces(pos, mass + 2 * m2, L, r_s, r_c)
    np.testing.assert_allclose(a3, a1 + 2 * a2, rtol=1e-11, atol=1e-12 * np.abs(a3).max())


def test_perfect_lattice_has_zero_force():
    nside, L = 12, 24.0
    pos = synth.lattice(nside, L)
    mass = np.full(pos.shape[0], 1.0)
    r_s = 1.2 * L / nside
    for r_c in [4.5 * r_s, 2.0 * r_s]:
        acc, pairs, _ = oracle.forces(pos, mass, L, r_s, r_c, cells=True)
        one = 1.0 / (L / nside) ** 2  # a single nearest-neighbour Newtonian term
        assert np.abs(acc).max() < 1e-12 * one
        assert np.all(pairs == pairs[0])


def test_cells_equal_brute_force():
    pos, mass, L = _clustered(n=2500)
    r_s, r_c = 1.2 * L / 16, 5.4 * L / 16
    tg = np.arange(0, 2500, 7)
    a0, p0, z0 = oracle.forces(pos, mass, L, r_s, r_c, targets=tg)
    a1, p1, z1 = oracle.forces(pos, mass, L, r_s, r_c, targets=tg, cells=True)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_allclose(a1, a0, rtol=1e-12, atol=1e-14 * np.abs(a0).max())


def test_coincident_distinct_pair_contributes_zero():
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0], [6.0, 5.0, 5.0]])
    mass = np.array([1.0, 1.0, 1.0])
    acc, pairs, zero = oracle.forces(pos, mass, 50.0, 1.0, 4.5)
    assert list(zero) == [1, 1, 0]
    g = _T_ref(0.5)  # r = 1
    np.testing.assert_allclose(acc[0], [g, 0, 0], rtol=1e-14)
    np.testing.assert_allclose(acc[2], [-2 * g, 0, 0], rtol=1e-14)


def test_rejects_cutoff_beyond_box():
    pos = np.array([[1.0, 1.0, 1.0]])
    with pytest.raises(ValueError):
        oracle.forces(pos, np.ones(1), 10.0, 3.0, 10.5)


# ------------------------------------------------------------- adjoint -------

def test_adjoint_isolated_pair_closed_form():
    """Two particles: dL/dx_0 = G K(d) (m_0 c_1 - m_1 c_0) with
    K = g I + (g'/r) d d^T and g = T/r^3 differentiated by mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    d = np.array([1.5, -0.4, 2.2])
    pos, m, L, r_s, r_c = _two(d)
    cot = np.array([[0.3, -1.2, 0.8], [-0.5, 0.9, 0.1]])
    gx, gm = oracle.adjoint(pos, m, cot, L, r_s, r_c, G=1.7)
    r = float(np.linalg.norm(d))

    def gfun(rr):
        x = rr / (2 * mp.mpf(r_s))
        return (mp.erfc(x) + 2 * x / mp.sqrt(mp.pi) * mp.exp(-x * x)) / rr ** 3

    g = float(gfun(mp.mpf(r)))
    gp = float(mp.diff(gfun, mp.mpf(r)))
    K = g * np.eye(3) + gp / r * np.outer(d, d)
    np.testing.assert_allclose(gx[0], 1.7 * K @ (m[0] * cot[1] - m[1] * cot[0]), rtol=1e-12)
    np.testing.assert_allclose(gx[1], 1.7 * K @ (m[1] * cot[0] - m[0] * cot[1]), rtol=1e-12)
    np.testing.assert_allclose(gm[0], -1.7 * g * np.dot(d, cot[1]), rtol=1e-12)
    np.testing.assert_allclose(gm[1], -1.7 * g * np.dot(-d, cot[0]), rtol=1e-12)


def test_adjoint_matches_finite_differences():
    pos, mass, L = _clustered(n=2000, L=40.0, seed=5)
    r_s, r_c = 1.2 * L / 16, 5.4 * L / 16
    cot = synth.cotangent(pos.shape[0], 99)
    tg = np.arange(0, 2000, 97)
    gx, gm = oracle.adjoint(pos, mass, cot, L, r_s, r_c, targets=tg)
    fx = np.zeros_like(gx)
    fm = np.zeros_like(gm)
    for k, p in enumerate(tg):
        fx[k], fm[k] = oracle.fd_gradient(pos, mass, cot, p, L, r_s, r_c, richardson=True)
    assert np.sqrt(np.sum((fx - gx) ** 2) / np.sum(gx ** 2)) < 1e-6
    np.testing.assert_allclose(fm, gm, rtol=1e-7, atol=1e-9 * np.abs(gm).max())
