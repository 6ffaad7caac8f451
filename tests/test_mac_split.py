"""Multipole split of the device pair walk (psr_device_build_split; paper,
Section 2: well-separated cell pairs interact through M2L, the others
through P2P) and the far part of the short range on it (psr_fmm_forces).

- The near and far lists of every target leaf partition, entry for entry,
  the list psr_device_build writes for the same input.
- Every far entry is well separated and wholly inside r_c, and every near
  entry is not, by the acceptance test recomputed here in FP64 from the
  leaves' particle boxes; the device decides in FP32 (rigorously for the
  cutoff side, from boxes rounded outward to FP32), so entries within a
  relative 1e-4 of a threshold may fall either way; no far entry may have a
  point pair at r_c or beyond.
- The expansion centres are the box centres and half-diagonals.
- fmm_forces against the oracle: on sampled target leaves the far part is
  the direct sum of the smooth truncated kernel (oracle fmm.direct: within
  r_c the hard cutoff changes nothing) over the far list's particles, to
  within the expansion's error bound, which shrinks with the order; near
  part (P2P, FP64) plus far part against the FP64 oracle's total force.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import fmm as ofmm

torch = pytest.importorskip("torch")
psr = pytest.importorskip("paper_2107_14008_gb300")
from paper_2107_14008_gb300 import capi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14008_gb300 import build
    build.build()


def _clustered(n, L=60.0, seed=3, n_pm=16, halos=6, max_leaf=32):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, halos, rng)
    r_s, r_c = synth.box_params(L, n_pm)
    return synth.Box(pos=pos, mass=rng.uniform(0.2, 2.0, n), L=L, n_pm=n_pm, r_s=r_s, r_c=r_c,
                     max_leaf=max_leaf)


CASES = {
    "uniform32": lambda: synth.small(nside=32),
    "clustered": lambda: _clustered(20000),
    "clustered_leaf8": lambda: _clustered(8000, seed=8, max_leaf=8),
    "small_box": lambda: _clustered(3000, L=10.0, seed=9, n_pm=8),  # r_c = 0.675 L: images
}


def _builds(b, theta, fp64=True, gaussian=False):
    dev = torch.device("cuda")
    pos = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    mass = torch.tensor(b.mass, dtype=torch.float64, device=dev)
    full = psr.Leaves.device_build(pos, mass, b.L, b.r_s, b.r_c, b.G, b.max_leaf, fp64=fp64)
    split = psr.Leaves.device_build(pos, mass, b.L, b.r_s, b.r_c, b.G, b.max_leaf, fp64=fp64,
                                    theta=theta, gaussian_mac=gaussian)
    return full, split


def _shifts(code, L):
    code = np.asarray(code, dtype=np.int64)
    return np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], axis=-1) * L


def _leaf_boxes(D):
    pd, leaf = D["pd"], D["leaf"]
    first = leaf[:, 0].astype(np.int64)
    lo = np.minimum.reduceat(pd[:, :3], first, axis=0)
    hi = np.maximum.reduceat(pd[:, :3], first, axis=0)
    return lo, hi


def _rows(rowptr, pairs):
    I = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return I, (pairs >> 5).astype(np.int64), (pairs & 31).astype(np.int64)


def _accept(lo, hi, I, J, code, L, theta, r_c, r_s, gaussian):
    """The split's test in FP64: (largest point-pair distance^2 / r_c^2,
    theta^2 l^2 / (rho_I + rho_J)^2, |R|^2), l = |R|, or with the Gaussian
    term min(|R|, 2 r_s^2 / |R|)."""
    sh = _shifts(code, L)
    d2 = m2 = ra2 = rb2 = np.zeros(len(I))
    for a in range(3):
        ea = 0.5 * (hi[I, a] - lo[I, a])
        eb = 0.5 * (hi[J, a] - lo[J, a])
        d = 0.5 * (lo[J, a] + hi[J, a]) + sh[:, a] - 0.5 * (lo[I, a] + hi[I, a])
        mx = np.abs(d) + ea + eb
        d2, m2 = d2 + d * d, m2 + mx * mx
        ra2, rb2 = ra2 + ea * ea, rb2 + eb * eb
    s2 = (np.sqrt(ra2) + np.sqrt(rb2)) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        scale2 = np.minimum(d2, (2 * r_s * r_s) ** 2 / d2) if gaussian else d2
        mac = np.where(s2 > 0, theta * theta * scale2 / s2, np.inf)
    return m2 / (r_c * r_c), mac, d2


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("theta", [0.4, 0.7])
@pytest.mark.parametrize("gaussian", [False, True])
def test_split_partitions_the_pair_list_by_the_acceptance_test(case, theta, gaussian):
    b = CASES[case]()
    full, split = _builds(b, theta, gaussian=gaussian)
    full.check()
    split.check()
    fi, si = full.info, split.info
    assert si.theta == theta and fi.n_far == 0
    assert si.n_leaves == fi.n_leaves
    # both count walks record the same kept ranges in the pair cache
    assert si.rows_walked_twice == fi.rows_walked_twice
    assert si.n_pairs + si.n_far == fi.n_pairs
    DF, DS, F = full.device_arrays(), split.device_arrays(), split.far_arrays()
    for k in ("leaf", "lcen", "perm"):
        assert np.array_equal(DF[k], DS[k]), k
    # partition: the union of the two lists is the full list, row by row
    nl = int(fi.n_leaves)
    key = lambda rp, pr: np.sort(np.repeat(np.arange(nl, dtype=np.uint64), np.diff(rp)) << 32
                                 | pr.astype(np.uint64))
    got = np.sort(np.concatenate([key(DS["rowptr"], DS["pairs"]), key(F["frow"], F["fpairs"])]))
    assert np.array_equal(got, key(DF["rowptr"], DF["pairs"]))
    # each side is the acceptance test
    lo, hi = _leaf_boxes(DS)
    I, J, code = _rows(F["frow"], F["fpairs"])
    inside, mac, d2 = _accept(lo, hi, I, J, code, b.L, theta, b.r_c, b.r_s, gaussian)
    assert np.all(inside < 1.0) and np.all(d2 > 0)
    assert np.all(mac >= 1.0 - 1e-5)
    I, J, code = _rows(DS["rowptr"], DS["pairs"])
    inside, mac, d2 = _accept(lo, hi, I, J, code, b.L, theta, b.r_c, b.r_s, gaussian)
    far_by_margin = (inside < 1.0 - 1e-4) & (mac > 1.0 + 1e-4) & (d2 > 0)
    assert not far_by_margin.any(), np.flatnonzero(far_by_margin)[:10]
    # expansion centres
    cen = 0.5 * (lo + hi)
    rad = np.sqrt(np.sum((0.5 * (hi - lo)) ** 2, axis=1))
    assert np.allclose(F["fcen"][:, :3], cen, rtol=0, atol=1e-12 * b.L)
    assert np.allclose(F["fcen"][:, 3], rad, rtol=1e-14, atol=1e-14 * b.L)
    # the FP32 offsets from the cell centres reproduce the FP64 centres
    unit = b.L / 2.0 ** 22
    back = DS["lcen"][:, :3].astype(np.float64) * unit + F["fofs"][:, :3].astype(np.float64)
    assert np.allclose(back, F["fcen"][:, :3], rtol=0, atol=4e-7 * b.L)
    if case.startswith("clustered") and not gaussian:  # dense halos: small, well separated leaves
        assert si.n_far > 0


def _far_direct(b, DS, F, rows):
    """Oracle far part of the sorted targets of the given target leaves."""
    pd, leaf = DS["pd"], DS["leaf"]
    out = {}
    for I in rows:
        f, c = leaf[I, 0], leaf[I, 1]
        tgt = pd[f:f + c, :3]
        src, m = [], []
        for e in range(F["frow"][I], F["frow"][I + 1]):
            J, code = int(F["fpairs"][e]) >> 5, int(F["fpairs"][e]) & 31
            fj, cj = leaf[J, 0], leaf[J, 1]
            src.append(pd[fj:fj + cj, :3] + _shifts(code, b.L))
            m.append(pd[fj:fj + cj, 3])
        out[I] = (np.arange(f, f + c), ofmm.direct(np.concatenate(src), np.concatenate(m), tgt,
                                                   b.r_s, b.G) if src else np.zeros((c, 3)))
    return out


@pytest.mark.parametrize("case", ["clustered", "clustered_leaf8"])
def test_fmm_forces_far_part_converges_to_the_direct_sum(case):
    """Relative RMS error of the far part over sampled target leaves, below
    2 theta^(p+1) / (1 - theta) (the order-p remainder of a pair whose radii
    sum to theta |R|) and falling with p."""
    theta = 0.5
    b = CASES[case]()
    _, split = _builds(b, theta)
    DS, F = split.device_arrays(), split.far_arrays()
    perm = DS["perm"].astype(np.int64)
    lens = np.diff(F["frow"])
    rows = np.random.default_rng(1).permutation(np.flatnonzero(lens > 0))[:12]
    ref = _far_direct(b, DS, F, rows)
    errs = []
    for p in (2, 4, 6):
        out = split.fmm_forces(p, fp64=True).cpu().numpy()
        num = den = 0.0
        for I, (idx, r) in ref.items():
            num += np.sum((out[perm[idx]] - r) ** 2)
            den += np.sum(r ** 2)
        err = np.sqrt(num / den)
        assert err < 2 * theta ** (p + 1) / (1 - theta), (p, err)
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]


def test_near_plus_far_matches_the_oracle_total():
    b = _clustered(20000, seed=4)
    _, split = _builds(b, 0.5)
    ref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, cells=True)
    errs = []
    for p in (2, 4, 6):
        acc = split.forces(psr.Options(precision=psr.PSR_FP64))
        split.fmm_forces(p, out=acc, accumulate=True, fp64=True)
        a = acc.cpu().numpy()
        errs.append(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3, errs
    # FP32 output: the same far part, accumulated in FP32
    a32 = split.forces(psr.Options())
    split.fmm_forces(6, out=a32, accumulate=True)
    e32 = np.sqrt(np.sum((a32.double().cpu().numpy() - ref) ** 2) / np.sum(ref ** 2))
    assert e32 < errs[2] + 2e-5


def test_split_states_and_arguments():
    b = _clustered(3000, seed=5)
    full, split = _builds(b, 0.5)
    with pytest.raises(psr.PsrError) as e:
        full.fmm_forces(4)
    assert e.value.code == capi.PSR_E_STATE
    _, nofp64 = _builds(b, 0.5, fp64=False)
    with pytest.raises(psr.PsrError) as e:
        nofp64.fmm_forces(4)
    assert e.value.code == capi.PSR_E_STATE
    for bad in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(psr.PsrError) as e:
            _builds(b, bad)
        assert e.value.code == capi.PSR_E_ARG
    with pytest.raises(psr.PsrError):
        split.fmm_forces(7)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    split.fmm_forces(3, status=status)
    assert int(status.item()) == 0


def test_split_build_is_deterministic():
    """The warp-cooperative split walk writes every row in walk order: two
    builds of the same input give identical workspaces, and the near + far
    forces repeat bit for bit."""
    b = CASES["clustered"]()
    dev = torch.device("cuda")
    pos = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    mass = torch.tensor(b.mass, dtype=torch.float64, device=dev)
    runs = []
    for _ in range(2):
        sp = psr.Leaves.device_build(pos, mass, b.L, b.r_s, b.r_c, b.G, b.max_leaf, theta=0.5)
        acc = sp.forces(psr.Options())
        sp.fmm_forces(4, out=acc, accumulate=True)
        runs.append((sp.device_arrays(), sp.far_arrays(), acc.cpu().numpy()))
        sp.check()
    (D1, F1, a1), (D2, F2, a2) = runs
    for k in ("leaf", "lcen", "rowptr", "pairs", "items", "perm"):
        assert np.array_equal(D1[k], D2[k]), k
    for k in ("frow", "fpairs", "fcen", "fofs"):
        assert np.array_equal(F1[k], F2[k]), k
    assert np.array_equal(a1, a2)
