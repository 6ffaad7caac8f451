"""GPU leaf builder (psr_device_build / psr_device_build_finish) against the
host builder: the workspace it writes must equal, array by array and bit by
bit, what psr_upload sends for the host-built handle of the same input (the
host builder is itself checked against the oracle's pair counts and the
paper's leaf rules in test_builder.py).  Integer and index arrays are
compared exactly; the FP32/FP64 payloads too, since both builders take the
same FP64 operations in the same order.
"""
import numpy as np
import pytest

import synth

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


def _box(pos, L, n_pm, mass=None, max_leaf=32):
    r_s, r_c = synth.box_params(L, n_pm)
    n = pos.shape[0]
    m = np.full(n, 1.0 / n) if mass is None else mass
    return synth.Box(pos=pos, mass=m, L=L, n_pm=n_pm, r_s=r_s, r_c=r_c, max_leaf=max_leaf)


def _clustered(n, L=60.0, seed=3, n_pm=16, halos=6):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, halos, rng)
    return _box(pos, L, n_pm, rng.uniform(0.2, 2.0, n))


def _coincident(n_same=1000, n_rest=3000, seed=5):
    """A pack of identical positions (one finest cell, cut into chunks) in a
    uniform background."""
    rng = np.random.default_rng(seed)
    L = 40.0
    pos = np.concatenate([np.tile([[11.3, 7.9, 30.2]], (n_same, 1)), rng.random((n_rest, 3)) * L])
    pos = pos[rng.permutation(pos.shape[0])]
    return _box(pos, L, 12, rng.uniform(0.5, 1.5, pos.shape[0]), max_leaf=8)


def _wrapped(seed=6):
    """Positions outside [0, L): negative, beyond L, exact multiples of L."""
    rng = np.random.default_rng(seed)
    L = 25.0
    pos = rng.uniform(-3 * L, 4 * L, (4000, 3))
    pos[:5] = [[0.0, L, -L], [2 * L, 0.5, -0.0], [L - 1e-13, 1e-300, 3.0], [-1e-17, 1, 2],
               [5 * L, -7 * L, 12.5]]
    return _box(pos, L, 8)


def _lattice_at_cutoff(max_leaf, nside=24):
    """Unit lattice with r_c^2 (1 + 1e-5) = 9: many leaf-box gaps^2 equal the
    threshold to rounding, where only the FP64 leaf test can decide."""
    pos = synth.lattice(nside, float(nside))
    r_c = 3.0 / np.sqrt(1.0 + 1e-5)
    n = pos.shape[0]
    return synth.Box(pos=pos, mass=np.full(n, 1.0 / n), L=float(nside), n_pm=nside,
                     r_s=r_c / 4.5, r_c=r_c, max_leaf=max_leaf)


CASES = {
    "lattice_cutoff1": lambda: _lattice_at_cutoff(1),
    "lattice_cutoff8": lambda: _lattice_at_cutoff(8),
    "uniform20": lambda: synth.small(nside=20),
    "clustered": lambda: _clustered(6000),
    "clustered_leaf1": lambda: _set_leaf(_clustered(3000, seed=7), 1),
    "clustered_leaf8": lambda: _set_leaf(_clustered(6000, seed=8), 8),
    "clustered_leaf64": lambda: _set_leaf(_clustered(20000, seed=9), 64),
    "coincident": _coincident,
    "wrapped": _wrapped,
    "nfw64": lambda: synth.adjoint(nside=64),
    "one": lambda: _box(np.array([[1.0, 2.0, 3.0]]), 10.0, 8),
    "two": lambda: _box(np.array([[1.0, 2.0, 3.0], [1.5, 2.0, 3.0]]), 10.0, 8),
    "three_same": lambda: _box(np.array([[4.0, 4.0, 4.0]] * 3), 10.0, 8, max_leaf=1),
}


def _set_leaf(b, max_leaf):
    b.max_leaf = max_leaf
    return b


def _build_both(b, fp64=True, masses=True):
    dev = torch.device("cuda")
    m = b.mass if masses else None
    host = psr.Leaves.build(b.pos, m, b.L, b.r_s, b.r_c, b.G, b.max_leaf, fp64=fp64)
    host.upload(dev)
    pos_d = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    mass_d = torch.tensor(b.mass, dtype=torch.float64, device=dev) if masses else None
    gpu = psr.Leaves.device_build(pos_d, mass_d, b.L, b.r_s, b.r_c, b.G, b.max_leaf, fp64=fp64)
    return host, gpu


def _compare(host, gpu):
    gpu.check()  # the pair write kernel reports row mismatches here
    hi, gi = host.info, gpu.info
    for k in ("n", "n_leaves", "n_pairs", "n_items", "nbox", "evaluated_pairs", "device_bytes",
              "max_leaf", "max_row"):
        assert getattr(gi, k) == getattr(hi, k), k
    H, D = host.host_arrays(), gpu.device_arrays()
    for k in ("leaf", "lcen", "rowptr", "pairs", "items"):
        assert H[k].shape == D[k].shape, k
        mism = np.flatnonzero(np.any((H[k] != D[k]).reshape(H[k].shape[0], -1), axis=1))
        assert mism.size == 0, (k, mism[:10])
    assert np.array_equal(H["pf"].view(np.uint32), D["pf"].view(np.uint32))
    if H["pd"] is None:
        assert D["pd"] is None
    else:
        assert np.array_equal(H["pd"].view(np.uint64), D["pd"].view(np.uint64))
    assert np.array_equal(host.perm, D["perm"].astype(np.int64))
    assert np.array_equal(gpu.perm, host.perm)


def _runs_per_row(A):
    """Maximal runs of consecutive leaves of one image code in each row."""
    rp, p = A["rowptr"], A["pairs"].astype(np.int64)
    if p.size == 0:
        return np.zeros(rp.size - 1, np.int64)
    brk = np.ones(p.size, bool)
    brk[1:] = p[1:] != p[:-1] + 32  # next leaf, same code
    starts = rp[:-1]
    brk[starts[starts < p.size]] = True
    cs = np.concatenate([[0], np.cumsum(brk)])
    return cs[rp[1:]] - cs[rp[:-1]]


def _check_pair_cache(b, host, gpu):
    """The count walk keeps a row as its runs in a slot of floor(8 n / n_leaves)
    runs (the cache is unused below 16); rows with more runs are walked a second
    time.  The walk's runs are the maximal runs of the final row, so the host's
    list fixes how many rows that is."""
    nl = host.info.n_leaves
    kslot = min(8 * max(b.n, 1) // nl, 1 << 20)
    want = nl if kslot < 16 else int(np.sum(_runs_per_row(host.host_arrays()) > kslot))
    assert gpu.info.rows_walked_twice == want
    return want


@pytest.mark.parametrize("case", sorted(CASES))
def test_device_build_equals_host_build(case):
    """Bit for bit, whether the pair rows come from the count walk's cache
    (clustered, nfw64, ...), from a second walk (clustered_leaf1 and
    lattice_cutoff1: slots below 16 runs) or from both (clustered_leaf8)."""
    b = CASES[case]()
    host, gpu = _build_both(b)
    _compare(host, gpu)
    twice = _check_pair_cache(b, host, gpu)
    if case == "clustered_leaf8":
        assert 0 < twice < host.info.n_leaves
    if case in ("clustered", "nfw64", "uniform20"):
        assert twice == 0


@pytest.mark.parametrize("fp64,masses", [(False, True), (True, False)])
def test_device_build_flags_and_default_masses(fp64, masses):
    b = _clustered(5000, seed=11)
    host, gpu = _build_both(b, fp64=fp64, masses=masses)
    _compare(host, gpu)


def test_device_build_precision_workload():
    """2.1M clustered particles: many sort tiles, scan tiles and top-level
    scan entries."""
    b = synth.precision()
    host, gpu = _build_both(b)
    _compare(host, gpu)


@pytest.mark.parametrize("precision", [psr.PSR_FP32_TABLE, psr.PSR_FP64])
def test_forces_from_device_build_are_bitwise_equal(precision):
    b = _clustered(8000, seed=12)
    host, gpu = _build_both(b)
    o = psr.Options(precision=precision)
    a_h = host.forces(o).cpu().numpy()
    a_g = gpu.forces(o).cpu().numpy()
    assert np.array_equal(a_h, a_g)
    cot = torch.tensor(synth.cotangent(b.n, 3), device="cuda")
    gh = [t.cpu().numpy() for t in host.adjoint(cot, o)]
    gg = [t.cpu().numpy() for t in gpu.adjoint(cot, o)]
    assert np.array_equal(gh[0], gg[0]) and np.array_equal(gh[1], gg[1])


def test_device_build_state_and_argument_errors():
    b = _clustered(2000, seed=13)
    _, gpu = _build_both(b)
    with pytest.raises(capi.PsrError) as e:
        gpu.upload()
    assert e.value.code == capi.PSR_E_STATE
    with pytest.raises(capi.PsrError) as e:
        gpu.host_arrays()
    assert e.value.code == capi.PSR_E_STATE
    with pytest.raises(capi.PsrError) as e:  # the build is no longer pending
        capi.psr_device_build_finish(gpu._h, gpu.workspace.data_ptr(), gpu.workspace.numel(),
                                     torch.cuda.current_stream().cuda_stream)
    assert e.value.code == capi.PSR_E_STATE
    bad = torch.tensor(b.pos, device="cuda")
    bad[17, 1] = float("nan")
    with pytest.raises(capi.PsrError) as e:
        psr.Leaves.device_build(bad, None, b.L, b.r_s, b.r_c)
    assert e.value.code == capi.PSR_E_ARG
    badm = torch.ones(b.n, dtype=torch.float64, device="cuda")
    badm[3] = float("inf")
    with pytest.raises(capi.PsrError) as e:
        psr.Leaves.device_build(torch.tensor(b.pos, device="cuda"), badm, b.L, b.r_s, b.r_c)
    assert e.value.code == capi.PSR_E_ARG
    # scratch too small
    n = b.n
    need = capi.psr_device_build_scratch_bytes(n)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    pos = torch.tensor(b.pos, device="cuda")
    with pytest.raises(capi.PsrError) as e:
        capi.psr_device_build(pos.data_ptr(), 0, n, psr._box(b.L, b.r_s, b.r_c), 32, 0,
                              small.data_ptr(), small.numel(),
                              torch.cuda.current_stream().cuda_stream, 1000)
    assert e.value.code == capi.PSR_E_WORKSPACE


def test_device_build_on_a_side_stream_and_sharded_launch():
    b = _clustered(6000, seed=14)
    host, _ = _build_both(b)
    s = torch.cuda.Stream()
    pos = torch.tensor(b.pos, device="cuda")
    mass = torch.tensor(b.mass, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        gpu = psr.Leaves.device_build(pos, mass, b.L, b.r_s, b.r_c, b.G, b.max_leaf, stream=s)
        full = gpu.forces(psr.Options(), stream=s)
        parts = torch.zeros_like(full)
        for k in range(3):
            gpu.forces(psr.Options(shard_count=3, shard_index=k), out=parts, stream=s)
    s.synchronize()
    assert torch.equal(full, parts)
    assert np.array_equal(full.cpu().numpy(), host.forces(psr.Options()).cpu().numpy())
    t0 = gpu.shard_targets(3, 0)
    assert np.array_equal(t0, host.shard_targets(3, 0))


@pytest.mark.parametrize("case", ["clustered", "coincident", "lattice_cutoff8", "nfw64"])
def test_device_build_unpacked_equals_host_unpacked(case):
    """PSR_BUILD_UNPACKED on both builders: plain octree leaves, bit for bit."""
    b = CASES[case]()
    dev = torch.device("cuda")
    host = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, b.max_leaf, pack=False)
    host.upload(dev)
    pos_d = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    mass_d = torch.tensor(b.mass, dtype=torch.float64, device=dev)
    gpu = psr.Leaves.device_build(pos_d, mass_d, b.L, b.r_s, b.r_c, b.G, b.max_leaf, pack=False)
    _compare(host, gpu)
    _check_pair_cache(b, host, gpu)
    packed = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, b.max_leaf)
    assert packed.info.n_leaves <= host.info.n_leaves


# ------------------------------------------------- device build vs oracle ---

def _rel_rms(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(np.sum((a - ref) ** 2) / max(np.sum(ref ** 2), 1e-300)))


@pytest.mark.parametrize("case", ["uniform20", "clustered", "clustered_leaf8", "clustered_leaf64",
                                  "coincident", "wrapped", "lattice_cutoff8"])
def test_device_build_against_the_oracle(case):
    """The leaf set built on the GPU, checked directly against the FP64
    oracle (not only through the host builder): the FP64 kernel's count of
    within-cutoff pairs equals the oracle's exactly (the leaf-pair list lost
    no pair within r_c), its forces match to 1e-6 rel RMS (1e-9 elementwise),
    and the FP32 table path's to 2e-5 (on the lattice, where every force is
    zero, both stay at rounding level)."""
    import oracle
    b = CASES[case]()
    pos = np.mod(b.pos, b.L)
    pos = np.where(pos >= b.L, 0.0, pos)
    ref, pairs, _ = oracle.forces(pos, b.mass, b.L, b.r_s, b.r_c, b.G, cells=True)
    dev = torch.device("cuda")
    gpu = psr.Leaves.device_build(torch.tensor(b.pos, dtype=torch.float64, device=dev),
                                  torch.tensor(b.mass, dtype=torch.float64, device=dev),
                                  b.L, b.r_s, b.r_c, b.G, b.max_leaf, fp64=True)
    a64 = gpu.forces(psr.Options(precision=psr.PSR_FP64)).cpu().numpy()
    a32 = gpu.forces(psr.Options(precision=psr.PSR_FP32_TABLE)).double().cpu().numpy()
    if case.startswith("lattice"):
        # a perfect lattice: every acceleration is zero by symmetry, so the
        # sums are compared with the size of one unit-spacing pair term
        unit = b.G * b.mass.max()
        assert np.abs(ref).max() < 1e-12 * unit
        assert np.abs(a64).max() < 1e-12 * unit
        assert np.abs(a32).max() < 1e-4 * unit
    else:
        assert _rel_rms(a64, ref) < 1e-6
        np.testing.assert_allclose(a64, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
        assert _rel_rms(a32, ref) < 2e-5
    gpu.forces(psr.Options(precision=psr.PSR_FP64, count_pairs=True))
    assert gpu.pair_count() == int(pairs.sum())
    gpu.check()
