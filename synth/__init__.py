"""Seeded synthetic particle sets shaped like the paper's runs.

This module holds the input generators shared by the tests, the benchmark and
the smoke check.  It contains none of the force method's arithmetic: it draws
positions and masses and states each workload's box parameters.

The paper's own runs start from 2LPTic / Zel'dovich initial conditions with
CAMB spectra (Section 4), which are not available here; uniform and
NFW-clustered sets stand in for them.  Workloads:

* ``small``      32^3 uniform, L=100, N_PM=32, leaves <= 32
* ``precision``  128^3, L=500, N_PM=128, 60 % of the mass in 4000 NFW halos
                 (concentration 10, halo masses from dN/dM ~ M^-1.9 on
                 [1e-5, 1e-2] of the total, rescaled to the stated fraction),
                 40 % uniform, leaves <= 32
* ``batch``      64 boxes, N log-uniform in [8^3, 64^3], L ~ U[50, 400],
                 N_PM = max(8, round(N^(1/3))), even boxes uniform, odd boxes
                 NFW-clustered as in ``precision``
* ``adjoint``    64^3 NFW-clustered, L=200, N_PM=64
* ``large``      512^3, L=1000, N_PM=512, 70 % of the mass in 200000 halos,
                 leaves <= 64

In every workload G = 1, particle masses are equal (1/N, total mass 1), the
split radius is r_s = 1.2 L / N_PM and the cutoff is r_c = 4.5 r_s.
Seeds are 12345 + workload index (+ box index for ``batch``).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

SPLIT_FACTOR = 1.2   # r_s = 1.2 * L / N_PM
CUTOFF_FACTOR = 4.5  # r_c = 4.5 * r_s


@dataclass
class Box:
    """One periodic box: positions (n,3) in [0,L), masses (n,), parameters."""
    pos: np.ndarray
    mass: np.ndarray
    L: float
    n_pm: int
    r_s: float
    r_c: float
    G: float = 1.0
    max_leaf: int = 32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.pos.shape[0])


def box_params(L, n_pm):
    """(r_s, r_c) of a workload with box side L and PM grid n_pm."""
    r_s = SPLIT_FACTOR * float(L) / float(n_pm)
    return r_s, CUTOFF_FACTOR * r_s


def uniform(n, L, rng):
    """n positions uniform in [0, L)^3."""
    p = rng.random((n, 3)) * L
    return np.where(p >= L, 0.0, p)


def lattice(nside, L, offset=0.5):
    """Perfect cubic lattice of nside^3 points, spacing L/nside."""
    g = (np.arange(nside, dtype=np.float64) + offset) * (L / nside)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _nfw_mu(s):
    return np.log1p(s) - s / (1.0 + s)


def _nfw_radii(u, conc, nodes=4096, newton_steps=3):
    """Radii in units of the NFW scale radius, inverting the enclosed-mass
    profile mu(s) = ln(1+s) - s/(1+s) on [0, conc]: mu(s) = u mu(conc).
    The inverse is tabulated by bisection on nodes uniform in sqrt(u) (near
    u = 0 the radius grows like sqrt(u), since mu ~ s^2/2), interpolated
    linearly, and refined by Newton steps with mu'(s) = s/(1+s)^2; the result
    solves the equation to a few units in the last place (checked against
    bisection in the tests)."""
    mc = _nfw_mu(conc)
    xk = np.arange(nodes + 1, dtype=np.float64) / nodes
    tk = xk * xk * mc
    lo, hi = np.zeros_like(xk), np.full_like(xk, float(conc))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = _nfw_mu(mid) < tk
        lo, hi = np.where(below, mid, lo), np.where(below, hi, mid)
    sk = 0.5 * (lo + hi)
    x = np.sqrt(u) * nodes
    k = np.minimum(x.astype(np.int64), nodes - 1)
    f = x - k
    s = sk[k] + f * (sk[k + 1] - sk[k])
    target = u * mc
    for _ in range(newton_steps):
        d = s / (1.0 + s) ** 2
        s = np.clip(s - (_nfw_mu(s) - target) / np.maximum(d, 1e-300), 0.0, float(conc))
    return s


def halo_masses(n_halos, frac, rng, slope=-1.9, mlo=1e-5, mhi=1e-2):
    """Halo masses (fractions of the total) from dN/dM ~ M^slope on
    [mlo, mhi], rescaled so that they sum to `frac`."""
    a = slope + 1.0
    u = rng.random(n_halos)
    m = (mlo ** a + u * (mhi ** a - mlo ** a)) ** (1.0 / a)
    return m * (frac / m.sum())


def nfw_clustered(n, L, frac, n_halos, rng, conc=10.0, chunk=1 << 22):
    """n positions: `frac` of them in NFW halos, the rest uniform.

    Each halo gets round(M_h n) particles; its R_200 encloses a mean density
    of 200 times the box mean, its scale radius is R_200 / conc, radii follow
    the NFW enclosed mass out to R_200, directions are isotropic, centres are
    uniform in the box, and all positions wrap periodically.
    """
    n_halos = max(1, int(n_halos))
    mh = halo_masses(n_halos, frac, rng)
    counts = np.rint(mh * n).astype(np.int64)
    over = counts.sum() - n
    if over > 0:  # rounding can only overshoot by a handful; trim the largest
        order = np.argsort(-counts)
        for k in range(int(over)):
            counts[order[k % n_halos]] -= 1
    centres = rng.random((n_halos, 3)) * L
    r200 = (3.0 * (counts / float(n)) * L ** 3 / (4.0 * np.pi * 200.0)) ** (1.0 / 3.0)
    n_h = int(counts.sum())
    pos = np.empty((n, 3))
    hid = np.repeat(np.arange(n_halos), counts)
    for s in range(0, n_h, chunk):
        e = min(n_h, s + chunk)
        h = hid[s:e]
        rad = _nfw_radii(rng.random(e - s), conc) * (r200[h] / conc)
        cz = 2.0 * rng.random(e - s) - 1.0
        ph = 2.0 * np.pi * rng.random(e - s)
        sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
        d = np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1) * rad[:, None]
        pos[s:e] = centres[h] + d
    pos[n_h:] = rng.random((n - n_h, 3)) * L
    pos = np.mod(pos, L)
    pos = np.where(pos >= L, 0.0, pos)
    return pos, {"n_halos": n_halos, "halo_particles": n_h,
                 "largest_halo": int(counts.max()) if n_halos else 0}


def _box(name, pos, L, n_pm, max_leaf, meta=None):
    n = pos.shape[0]
    r_s, r_c = box_params(L, n_pm)
    return Box(pos=pos, mass=np.full(n, 1.0 / n), L=float(L), n_pm=int(n_pm), r_s=r_s,
               r_c=r_c, G=1.0, max_leaf=max_leaf, name=name, meta=meta or {})


def small(seed=12345, nside=32):
    rng = np.random.default_rng(seed)
    n = nside ** 3
    return _box("uniform %d^3 L=100 N_PM=%d" % (nside, nside), uniform(n, 100.0, rng),
                100.0, nside, 32)


def precision(seed=12346, nside=128, L=500.0, frac=0.6, n_halos=4000):
    rng = np.random.default_rng(seed)
    n = nside ** 3
    pos, meta = nfw_clustered(n, L, frac, n_halos, rng)
    return _box("NFW %d^3 L=%g N_PM=%d %d halos" % (nside, L, nside, n_halos), pos, L,
                nside, 32, meta)


def batch(seed=12347, nbox=64, nmin=8 ** 3, nmax=64 ** 3) -> List[Box]:
    boxes = []
    for b in range(nbox):
        rng = np.random.default_rng(seed + b)
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        L = float(rng.uniform(50.0, 400.0))
        n_pm = max(8, int(round(n ** (1.0 / 3.0))))
        if b % 2 == 0:
            pos, meta = uniform(n, L, rng), {"kind": "uniform"}
        else:
            pos, meta = nfw_clustered(n, L, 0.6, max(1, round(4000 * n / 128 ** 3)), rng)
            meta["kind"] = "nfw"
        boxes.append(_box("batch box %d" % b, pos, L, n_pm, 32, meta))
    return boxes


def adjoint(seed=12348, nside=64, L=200.0):
    rng = np.random.default_rng(seed)
    n = nside ** 3
    pos, meta = nfw_clustered(n, L, 0.6, max(1, round(4000 * n / 128 ** 3)), rng)
    return _box("NFW %d^3 L=%g N_PM=%d" % (nside, L, nside), pos, L, nside, 32, meta)


def large(seed=12349, nside=512, L=1000.0, frac=0.7, n_halos=200000):
    rng = np.random.default_rng(seed)
    n = nside ** 3
    pos, meta = nfw_clustered(n, L, frac, n_halos, rng)
    return _box("NFW %d^3 L=%g N_PM=%d" % (nside, L, nside), pos, L, nside, 64, meta)


def cotangent(n, seed):
    """Seeded N(0,1) cotangent on every force component."""
    return np.random.default_rng(seed).standard_normal((n, 3))
