"""Pins of the long-range PM oracle (oracle/pm.py) against facts that do not
come from its own code (paper, Section 2: phi = phi_long + phi_short with the
Gaussian split; the reading of the filter is exp(-k^2 r_s^2)).

- Short + long is the full periodic Newtonian force, whatever the split
  radius: the short-range oracle (the C pair sum, erfc kernel, cutoff far in
  the tail) plus the Ewald k-space sum at r_s and at r_s' agree to rounding.
  A wrong sign, a dropped 4 pi / L^3, or a filter exp(-k^2/4r_s^2) breaks it.
- Two bodies: the long-range force is G m (1 - T(x)) / r^2 (the complement of
  Eq. tr) plus the periodic background term -(4 pi/3) G m r / L^3.
- Momentum: sum_i m_i a_i = 0.
- The mesh method converges to the Ewald sum: at the paper's split
  r_s = 1.2 L/N_PM within 3 % RMS with CIC deconvolution, and closer on a
  finer mesh; CIC conserves mass, puts a particle at a grid point on one
  point, and interpolates trilinear fields exactly; a lattice on the grid
  points feels no force; a shift by one cell shifts the solution.
"""
import numpy as np
import pytest
from scipy.special import erfc

import oracle
from oracle import pm


def _T(x):
    return erfc(x) + 2.0 * x / np.sqrt(np.pi) * np.exp(-x * x)


def _rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def test_short_plus_long_is_independent_of_the_split():
    rng = np.random.default_rng(1)
    L, n = 1.0, 40
    pos, mass = rng.random((n, 3)), rng.uniform(0.5, 1.5, n)
    tot = []
    for r_s in (0.03, 0.04):
        short, _, _ = oracle.forces(pos, mass, L, r_s, 11.0 * r_s, 1.0)  # T(5.5) ~ 1e-13
        tot.append(short + pm.ewald_long(pos, mass, L, r_s))
    assert _rel(tot[0], tot[1]) < 1e-12
    # the split is not trivial: each part alone changes a lot
    assert _rel(pm.ewald_long(pos, mass, L, 0.03), pm.ewald_long(pos, mass, L, 0.04)) > 0.1


def test_long_range_conserves_momentum():
    rng = np.random.default_rng(2)
    pos, mass = rng.random((60, 3)) * 3.0, rng.uniform(0.1, 2.0, 60)
    a = pm.ewald_long(pos, mass, 3.0, 0.08)
    p = (mass[:, None] * a).sum(axis=0)
    assert np.max(np.abs(p)) < 1e-12 * np.sum(mass * np.linalg.norm(a, axis=1))


@pytest.mark.parametrize("r", [0.005, 0.02, 0.05])
def test_two_body_long_range_force(r):
    L, r_s, m1 = 1.0, 0.01, 2.0
    p = np.array([[0.3, 0.4, 0.5], [0.3 + r, 0.4, 0.5]])
    a = pm.ewald_long(p, np.array([1.0, m1]), L, r_s)
    closed = m1 * (1.0 - _T(r / (2.0 * r_s))) / r ** 2 - 4.0 * np.pi / 3.0 * m1 * r / L ** 3
    assert abs(a[0, 0] - closed) < 1e-5 * abs(closed)
    assert np.all(np.abs(a[0, 1:]) < 1e-9 * abs(closed))
    assert abs(a[1, 0] + a[0, 0] / m1) < 1e-9 * abs(a[0, 0])


def test_cic_mass_points_and_trilinear_fields():
    rng = np.random.default_rng(3)
    L, n = 2.0, 8
    pos, mass = rng.random((100, 3)) * L, rng.uniform(0.5, 1.5, 100)
    rho = pm.cic_deposit(pos, mass, L, n)
    assert abs(rho.sum() * (L / n) ** 3 - mass.sum()) < 1e-12 * mass.sum()
    one = pm.cic_deposit(np.array([[3, 5, 1]]) * (L / n), np.array([2.0]), L, n)
    assert one[3, 5, 1] == pytest.approx(2.0 / (L / n) ** 3, rel=1e-14)
    assert np.count_nonzero(one) == 1
    g = np.arange(n, dtype=float)
    field = 2.0 * g[:, None, None] - 3.0 * g[None, :, None] + 0.5 * g[None, None, :] + 1.0
    inner = rng.random((50, 3)) * (n - 1) * (L / n)  # away from the periodic seam
    u = inner / (L / n)
    want = 2.0 * u[:, 0] - 3.0 * u[:, 1] + 0.5 * u[:, 2] + 1.0
    assert np.allclose(pm.cic_interp(field, inner, L), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n_pm,r_s_cells,bound", [(32, 1.2, 3e-2), (64, 2.4, 6e-3)])
def test_mesh_converges_to_the_ewald_sum(n_pm, r_s_cells, bound):
    rng = np.random.default_rng(4)
    L, N = 1.0, 400
    pos, mass = rng.random((N, 3)), np.full(N, 1.0 / N)
    r_s = r_s_cells * L / n_pm
    exact = pm.ewald_long(pos, mass, L, r_s)
    with_dec = _rel(pm.pm_forces(pos, mass, L, r_s, n_pm), exact)
    without = _rel(pm.pm_forces(pos, mass, L, r_s, n_pm, deconvolve=False), exact)
    assert with_dec < bound
    assert without > 2.0 * with_dec  # deconvolution of the CIC windows helps


def test_mesh_error_falls_with_resolution_at_fixed_split():
    rng = np.random.default_rng(5)
    L, N, r_s = 1.0, 300, 1.2 / 32
    pos, mass = rng.random((N, 3)), rng.uniform(0.5, 1.5, N)
    exact = pm.ewald_long(pos, mass, L, r_s)
    e32 = _rel(pm.pm_forces(pos, mass, L, r_s, 32), exact)
    e64 = _rel(pm.pm_forces(pos, mass, L, r_s, 64), exact)
    assert e64 < 0.3 * e32


def test_mesh_symmetries():
    n, L = 16, 1.0
    g = (np.arange(n) + 0.0) * (L / n)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    a = pm.pm_forces(lat, np.ones(len(lat)), L, 1.2 * L / n, n)
    assert np.max(np.abs(a)) < 1e-10
    rng = np.random.default_rng(6)
    pos, mass = rng.random((200, 3)), rng.uniform(0.5, 1.5, 200)
    a0 = pm.pm_forces(pos, mass, L, 0.05, n)
    a1 = pm.pm_forces(pos + np.array([L / n, 0.0, -2 * L / n]), mass, L, 0.05, n)
    assert np.max(np.abs(a1 - a0)) < 1e-10 * np.max(np.abs(a0))
    a2 = pm.pm_forces(pos, 2.0 * mass, L, 0.05, n)
    assert np.allclose(a2, 2.0 * a0, rtol=1e-12, atol=1e-12 * np.max(np.abs(a0)))
