"""The seeded input generators (CPU): the NFW radius inversion against plain
bisection of the enclosed-mass profile, and the workload recipes' sizes."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("conc", [1.0, 4.0, 10.0, 30.0])
def test_nfw_radius_inversion_matches_bisection(conc):
    rng = np.random.default_rng(7)
    u = np.concatenate([[0.0, 1e-300, 1e-12, 0.5, 1.0 - 1e-16, 1.0], rng.random(20000)])
    s = synth._nfw_radii(u, conc)
    target = u * synth._nfw_mu(conc)
    lo, hi = np.zeros_like(u), np.full_like(u, conc)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        below = synth._nfw_mu(mid) < target
        lo, hi = np.where(below, mid, lo), np.where(below, hi, mid)
    ref = 0.5 * (lo + hi)
    assert np.all((s >= 0.0) & (s <= conc))
    assert np.max(np.abs(s - ref)) < 1e-12 * conc
    assert np.max(np.abs(synth._nfw_mu(s) - target)) < 1e-14


def test_nfw_clustered_is_seeded_and_in_the_box():
    a, ma = synth.nfw_clustered(5000, 50.0, 0.6, 7, np.random.default_rng(3))
    b, mb = synth.nfw_clustered(5000, 50.0, 0.6, 7, np.random.default_rng(3))
    assert np.array_equal(a, b) and ma == mb
    assert np.all((a >= 0.0) & (a < 50.0))
    assert ma["halo_particles"] == pytest.approx(0.6 * 5000, abs=7)
