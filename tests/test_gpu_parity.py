"""GPU parity: libpsr's kernels, called through the C ABI, against the FP64
oracle on the same seeded inputs.

Tolerances (relative RMS over all compared particles,
sqrt(sum |da|^2 / sum |a|^2)):
  FP64 path                   1e-6   (spec bound; observed ~1e-14)
  FP32 paths vs exact oracle  2e-5   (spec bound)
  FP32 table vs the oracle's interpolated T of the same table: 2e-6 (what
  remains is FP32 rounding of coordinates and sums)
  FP32 adjoint (dL/dx and dL/dm) vs the oracle gradient: 2e-5, the FP32
  force tolerance
Per particle, on the workloads' sampled targets: max over targets of
|da_i| / max(|a_i|, 1e-3 rms|a|) below MAX_REL_FP32 (see there).
"""
import numpy as np
import pytest

import oracle
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


# Largest per-particle error allowed on the FP32 paths.  The error of one
# target is dominated by its closest pairs, whose FP32 coordinates (leaf-local,
# measured from the parent cell's centre for packed leaves) round to ~1e-7 of
# the cell size: the worst of 100 000 sampled targets of the 128^3 workload
# measured 7.6e-5 (99th percentile 2e-6); the bound keeps a 3.3x margin.
MAX_REL_FP32 = 2.5e-4


def max_rel(a, ref):
    """max_i |a_i - ref_i| / max(|ref_i|, 1e-3 rms|ref|)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nr = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(nr * nr))
    return float(np.max(np.linalg.norm(a - ref, axis=1) / np.maximum(nr, floor)))


def rel_rms(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(np.sum((a - ref) ** 2) / max(np.sum(ref ** 2), 1e-300)))


def _clustered(n=6000, L=60.0, seed=3, n_pm=16, halos=6):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, halos, rng)
    r_s, r_c = synth.box_params(L, n_pm)
    return synth.Box(pos=pos, mass=rng.uniform(0.2, 2.0, n), L=L, n_pm=n_pm, r_s=r_s, r_c=r_c)


def _small_box():
    rng = np.random.default_rng(4)
    L, n = 10.0, 500
    r_s, r_c = synth.box_params(L, 8)
    return synth.Box(pos=rng.random((n, 3)) * L, mass=rng.uniform(0.5, 1.5, n), L=L, n_pm=8,
                     r_s=r_s, r_c=r_c)


CASES = {
    "uniform": lambda: synth.small(nside=20),
    "clustered": _clustered,
    "small_box": _small_box,
}

_oracle_cache = {}


def oracle_acc(b, key, t_mode=oracle.T_EXACT, table_n=1024, level=4):
    k = (key, t_mode, table_n, level)
    if k not in _oracle_cache:
        _oracle_cache[k] = oracle.forces(b.pos % b.L, b.mass, b.L, b.r_s, b.r_c, b.G,
                                         t_mode=t_mode, table_n=table_n, level=level, cells=True)
    return _oracle_cache[k]


def gpu_forces(b, opts, max_leaf=32):
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf).upload()
    acc = lv.forces(opts)
    lv.check()
    return acc.double().cpu().numpy(), lv


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("max_leaf", [1, 8, 32, 64])
def test_fp64_path_matches_oracle(case, max_leaf):
    b = CASES[case]()
    ref, _, _ = oracle_acc(b, case)
    acc, _ = gpu_forces(b, psr.Options(precision=psr.PSR_FP64), max_leaf)
    assert rel_rms(acc, ref) < 1e-6
    np.testing.assert_allclose(acc, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


FP32_VARIANTS = [
    ("exact", dict(precision=psr.PSR_FP32_EXACT)),
    ("lin1024", dict(precision=psr.PSR_FP32_TABLE, table_n=1024, interp=psr.PSR_LINEAR)),
    ("lin4096", dict(precision=psr.PSR_FP32_TABLE, table_n=4096, interp=psr.PSR_LINEAR)),
    ("cub1024", dict(precision=psr.PSR_FP32_TABLE, table_n=1024, interp=psr.PSR_CUBIC)),
    ("cub4096", dict(precision=psr.PSR_FP32_TABLE, table_n=4096, interp=psr.PSR_CUBIC)),
]


KERNELS = [psr.PSR_KERNEL_SCALAR, psr.PSR_KERNEL_PACKED, psr.PSR_KERNEL_PAPER]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("name,kw", FP32_VARIANTS)
@pytest.mark.parametrize("accum", [psr.PSR_ACC_FP64, psr.PSR_ACC_KAHAN32])
@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_paths_match_oracle(case, name, kw, accum, kernel):
    b = CASES[case]()
    ref, _, _ = oracle_acc(b, case)
    acc, _ = gpu_forces(b, psr.Options(accum=accum, kernel=kernel, **kw), 32)
    assert rel_rms(acc, ref) < 2e-5, name


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("interp", [psr.PSR_LINEAR, psr.PSR_CUBIC])
def test_wide_leaves_two_targets_per_lane(case, kernel, interp):
    """max_leaf 64: leaves above 32 particles put two targets on each lane."""
    b = CASES[case]()
    ref, _, _ = oracle_acc(b, case)
    acc, lv = gpu_forces(b, psr.Options(kernel=kernel, interp=interp), 64)
    assert rel_rms(acc, ref) < 2e-5


@pytest.mark.parametrize("tile", [64, 128, 256])
@pytest.mark.parametrize("accum", [psr.PSR_ACC_FP64, psr.PSR_ACC_KAHAN32])
def test_each_targets_per_lane_class(tile, accum):
    """The scalar kernel puts 1, 2 or 3 targets on a lane by leaf size (3 for
    leaves of 3, 6, 9, 11-12, 17-18, 21-24 and 33-48 particles with tiles of
    128 or more, 2 for 19-20 and 49-64; with 64-particle tiles only 1 or 2).
    Each group of leaf sizes is checked on its own targets, so one wrong path
    cannot hide in the mean over all particles."""
    b = CASES["clustered"]()
    ref, _, _ = oracle_acc(b, "clustered")
    acc, lv = gpu_forces(b, psr.Options(accum=accum, source_tile=tile), 64)
    leaf, perm = lv.host_arrays()["leaf"], lv.perm
    size = np.zeros(b.n, np.int64)
    for first, cnt in leaf[:, :2]:
        size[perm[first:first + cnt]] = cnt
    three = [3, 6, 9, 11, 12, 17, 18, 21, 22, 23, 24] + list(range(33, 49))
    classes = {"three": np.isin(size, three), "two": np.isin(size, [19, 20] + list(range(49, 65)))}
    classes["one"] = ~(classes["three"] | classes["two"])
    for name, sel in classes.items():
        assert sel.sum() > 100, name
        assert rel_rms(acc[sel], ref[sel]) < 2e-5, name


@pytest.mark.parametrize("case", ["uniform", "clustered"])
@pytest.mark.parametrize("interp,mode", [(psr.PSR_LINEAR, oracle.T_LINEAR),
                                         (psr.PSR_CUBIC, oracle.T_CUBIC)])
@pytest.mark.parametrize("table_n", [256, 1024])
@pytest.mark.parametrize("kernel", KERNELS)
def test_table_path_matches_interpolated_oracle(case, interp, mode, table_n, kernel):
    b = CASES[case]()
    ref, _, _ = oracle_acc(b, case, mode, table_n)
    acc, _ = gpu_forces(b, psr.Options(precision=psr.PSR_FP32_TABLE, table_n=table_n,
                                       interp=interp, kernel=kernel), 16)
    assert rel_rms(acc, ref) < 2e-6


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision,kernel", [(psr.PSR_FP64, 0), (psr.PSR_FP32_TABLE, 1),
                                              (psr.PSR_FP32_TABLE, 2), (psr.PSR_FP32_EXACT, 1),
                                              (psr.PSR_FP32_TABLE, 3)])
def test_pair_count_matches_oracle(case, precision, kernel):
    b = CASES[case]()
    _, pairs, _ = oracle_acc(b, case)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=16).upload()
    lv.forces(psr.Options(precision=precision, count_pairs=True, kernel=kernel))
    got = lv.pair_count()
    # FP32 distances can move a pair within one rounding of r_c across it
    tol = 0 if precision == psr.PSR_FP64 else max(2, int(1e-6 * pairs.sum()))
    assert abs(got - int(pairs.sum())) <= tol
    # pair terms the kernel evaluated: every leaf-tile pair for the FP64 and
    # block-per-leaf kernels; the warp-per-leaf kernels drop sources at least
    # r_c from the target box, so they evaluate fewer, never fewer than the
    # pairs within the cutoff plus the self pairs
    ev, tiles = lv.evaluated_count(), lv.evaluated_pairs
    if precision == psr.PSR_FP64 or kernel == psr.PSR_KERNEL_PAPER:
        assert ev == tiles
    else:
        assert int(pairs.sum()) + b.n <= ev <= tiles


@pytest.mark.parametrize("interp,mode", [(psr.PSR_LINEAR, oracle.T_LINEAR),
                                         (psr.PSR_CUBIC, oracle.T_CUBIC)])
@pytest.mark.parametrize("table_n", [64, 1024, 4096])
def test_table_kernel_values(interp, mode, table_n):
    x_c = 2.25
    out = torch.zeros((table_n + 1, 4), dtype=torch.float32, device="cuda")
    capi.psr_table(table_n, interp, x_c, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    tab = out.double().cpu().numpy()
    assert np.all(tab[table_n] == 0.0)
    h = x_c / table_n
    x = np.linspace(0, x_c * (1 - 1e-9), 20011)
    k = np.minimum(np.floor(x / h).astype(int), table_n - 1)
    f = (x - k * h) / h - 0.5
    c = tab[k]
    if interp == psr.PSR_LINEAR:
        val = c[:, 0] + f * c[:, 1]
        # the intercept form the forward kernel evaluates: A_k + (k + f) D_k
        val2 = c[:, 2] + (k + f) * c[:, 1]
        ref2 = oracle.T(x, mode, table_n, x_c)
        assert np.max(np.abs(val2 - ref2)) < 4e-7 + 2.0 ** -24 * np.max(np.abs(k * c[:, 1]))
        assert np.all(tab[table_n] == 0.0)
    else:
        val = c[:, 0] + f * (c[:, 1] + f * (c[:, 2] + f * c[:, 3]))
    ref = oracle.T(x, mode, table_n, x_c)
    assert np.max(np.abs(val - ref)) < 4e-7  # FP32 rounding of the coefficients


def test_isolated_pair_and_single_particle():
    L = 100.0
    r_s, r_c = 3.0, 13.5
    d = np.array([2.0, -1.0, 0.5])
    pos = np.array([[50.0, 50.0, 50.0], [50.0, 50.0, 50.0] + d])
    m = np.array([0.7, 0.3])
    ref, _, _ = oracle.forces(pos, m, L, r_s, r_c)
    for prec in (psr.PSR_FP64, psr.PSR_FP32_EXACT, psr.PSR_FP32_TABLE):
        lv = psr.Leaves.build(pos, m, L, r_s, r_c).upload()
        acc = lv.forces(psr.Options(precision=prec)).double().cpu().numpy()
        tol = 1e-12 if prec == psr.PSR_FP64 else 1e-6
        np.testing.assert_allclose(acc, ref, rtol=tol)
    one = psr.Leaves.build(pos[:1], m[:1], L, r_s, r_c).upload()
    for prec in (psr.PSR_FP64, psr.PSR_FP32_TABLE):
        assert np.all(one.forces(psr.Options(precision=prec)).cpu().numpy() == 0.0)


def test_coincident_particles_give_finite_forces():
    pos = np.vstack([np.full((70, 3), 3.0), np.random.default_rng(1).random((50, 3)) * 20])
    m = np.ones(120)
    r_s, r_c = synth.box_params(20.0, 8)
    ref, _, _ = oracle.forces(pos, m, 20.0, r_s, r_c)
    for prec in (psr.PSR_FP64, psr.PSR_FP32_TABLE, psr.PSR_FP32_EXACT):
        lv = psr.Leaves.build(pos, m, 20.0, r_s, r_c).upload()
        acc = lv.forces(psr.Options(precision=prec)).double().cpu().numpy()
        assert np.all(np.isfinite(acc))
        assert rel_rms(acc, ref) < (1e-9 if prec == psr.PSR_FP64 else 2e-5)


@pytest.mark.parametrize("kernel", [psr.PSR_KERNEL_SCALAR, psr.PSR_KERNEL_PACKED])
def test_coincident_particles_give_finite_adjoint(kernel):
    """Coincident pairs contribute nothing to either gradient (r = 0: the
    linear path's table coordinate reaches the zero entry, the others take
    1/r = 0); every other pair of the 70 coincident particles and the 50
    scattered ones must still match the oracle."""
    pos = np.vstack([np.full((70, 3), 3.0), np.random.default_rng(1).random((50, 3)) * 20])
    m = np.linspace(0.5, 1.5, 120)
    r_s, r_c = synth.box_params(20.0, 8)
    cot = synth.cotangent(120, 7)
    gx_ref, gm_ref = oracle.adjoint(pos, m, cot, 20.0, r_s, r_c, 1.0, cells=True)
    for prec in (psr.PSR_FP64, psr.PSR_FP32_TABLE, psr.PSR_FP32_EXACT):
        lv = psr.Leaves.build(pos, m, 20.0, r_s, r_c).upload()
        gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(precision=prec, kernel=kernel))
        lv.check()
        gx, gm = gx.double().cpu().numpy(), gm.double().cpu().numpy()
        assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gm))
        tol = 1e-9 if prec == psr.PSR_FP64 else 2e-5
        assert rel_rms(gx, gx_ref) < tol, prec
        assert rel_rms(gm, gm_ref) < tol, prec


@pytest.mark.parametrize("equal", [False, True])
def test_deterministic_and_batch_equals_single_boxes(equal):
    """A batch gives each box the forces of that box alone, bit for bit, and
    repeats them bit for bit: with per-particle masses (the general per-pair
    form), and with one mass per box (every box takes the equal-mass path,
    alone as in the batch)."""
    small = synth.small(nside=12)
    if equal:
        boxes = [small, synth.small(seed=9, nside=10), synth.precision(nside=16, L=60.0, n_halos=4)]
    else:
        varied = synth.Box(pos=small.pos, mass=np.linspace(0.5, 1.5, small.n), L=small.L,
                           n_pm=small.n_pm, r_s=small.r_s, r_c=small.r_c)
        boxes = [varied, _clustered(n=3000), _small_box()]
    opts = psr.Options(precision=psr.PSR_FP32_TABLE)
    lv = psr.Leaves.build_batch([(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G) for b in boxes],
                                max_leaf=32).upload()
    assert lv.info.equal_mass == int(equal)
    a1 = lv.forces(opts).cpu().numpy()
    a2 = lv.forces(opts).cpu().numpy()
    np.testing.assert_array_equal(a1, a2)
    off = 0
    for b in boxes:
        single, one = gpu_forces(b, opts, 32)
        assert one.info.equal_mass == int(equal)
        np.testing.assert_array_equal(a1[off:off + b.n], single.astype(np.float32))
        off += b.n


def test_cuda_graph_replay_matches_eager():
    b = _clustered()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    opts = psr.Options(precision=psr.PSR_FP32_TABLE)
    eager = lv.forces(opts).clone()
    out = torch.zeros_like(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lv.forces(opts, out=out)  # warm-up (builds nothing new)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lv.forces(opts, out=out)
    for _ in range(3):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
    lv.check()


def test_small_workload_all_targets():
    """32^3 uniform, L=100, N_PM=32: every particle against the oracle."""
    b = synth.small()
    ref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, cells=True)
    acc64, _ = gpu_forces(b, psr.Options(precision=psr.PSR_FP64))
    assert rel_rms(acc64, ref) < 1e-6
    acc32, _ = gpu_forces(b, psr.Options(precision=psr.PSR_FP32_TABLE))
    assert rel_rms(acc32, ref) < 2e-5
    assert max_rel(acc32, ref) < MAX_REL_FP32


@pytest.fixture(scope="module")
def precision_workload():
    b = synth.precision()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
    rng = np.random.default_rng(777)
    tg = np.sort(rng.choice(b.n, 2000, replace=False))
    ref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, targets=tg, cells=True)
    return b, lv, tg, ref


@pytest.mark.parametrize("name,kw", FP32_VARIANTS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_precision_workload_sampled(precision_workload, name, kw, kernel):
    """128^3 NFW (60 % in 4000 halos), L=500: 2000 sampled targets, the full
    launch the benchmark times."""
    b, lv, tg, ref = precision_workload
    acc = lv.forces(psr.Options(kernel=kernel, **kw)).double().cpu().numpy()
    lv.check()
    assert np.all(np.isfinite(acc))
    assert rel_rms(acc[tg], ref) < 2e-5, name
    assert max_rel(acc[tg], ref) < MAX_REL_FP32, name


def test_precision_workload_fp64_sampled(precision_workload):
    b, lv, tg, ref = precision_workload
    acc = lv.forces(psr.Options(precision=psr.PSR_FP64)).cpu().numpy()
    assert rel_rms(acc[tg], ref) < 1e-6


# ------------------------------------------------------------------ adjoint --

@pytest.mark.parametrize("case", ["uniform", "clustered", "small_box"])
def test_adjoint_fp64_matches_oracle(case):
    b = CASES[case]()
    cot = synth.cotangent(b.n, 5)
    gx_ref, gm_ref = oracle.adjoint(b.pos % b.L, b.mass, cot, b.L, b.r_s, b.r_c, b.G, cells=True)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(precision=psr.PSR_FP64))
    lv.check()
    assert rel_rms(gx.cpu().numpy(), gx_ref) < 1e-6
    assert rel_rms(gm.cpu().numpy(), gm_ref) < 1e-6


@pytest.mark.parametrize("case", ["uniform", "clustered", "small_box"])
@pytest.mark.parametrize("name,kw", FP32_VARIANTS)
@pytest.mark.parametrize("kernel", [psr.PSR_KERNEL_SCALAR, psr.PSR_KERNEL_PACKED])
def test_adjoint_fp32_matches_oracle(case, name, kw, kernel):
    b = CASES[case]()
    cot = synth.cotangent(b.n, 5)
    gx_ref, gm_ref = oracle.adjoint(b.pos % b.L, b.mass, cot, b.L, b.r_s, b.r_c, b.G, cells=True)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(kernel=kernel, **kw))
    lv.check()
    assert rel_rms(gx.double().cpu().numpy(), gx_ref) < 2e-5, name
    assert rel_rms(gm.double().cpu().numpy(), gm_ref) < 2e-5, name


def test_adjoint_fp64_matches_finite_differences():
    b = _clustered(n=4000, L=40.0, seed=5)
    cot = synth.cotangent(b.n, 99)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(precision=psr.PSR_FP64))
    gx, gm = gx.cpu().numpy(), gm.cpu().numpy()
    tg = np.arange(0, b.n, 41)
    fx = np.array([oracle.fd_gradient(b.pos % b.L, b.mass, cot, p, b.L, b.r_s, b.r_c,
                                      richardson=True)[0] for p in tg])
    assert rel_rms(gx[tg], fx) < 1e-5


def test_autograd_function_backward_is_adjoint():
    b = _clustered(n=2000)
    pos = torch.tensor(b.pos, device="cuda", requires_grad=True)
    mass = torch.tensor(b.mass, device="cuda", requires_grad=True)
    opts = psr.Options(precision=psr.PSR_FP64)
    acc = psr.forces(pos, mass, b.L, b.r_s, b.r_c, b.G, opts)
    cot = torch.tensor(synth.cotangent(b.n, 3), device="cuda")
    (acc * cot).sum().backward()
    gx_ref, gm_ref = oracle.adjoint(b.pos % b.L, b.mass, cot.cpu().numpy(), b.L, b.r_s, b.r_c,
                                    b.G, cells=True)
    assert rel_rms(pos.grad.cpu().numpy(), gx_ref) < 1e-6
    assert rel_rms(mass.grad.cpu().numpy(), gm_ref) < 1e-6


# -------------------------------------------------------- tiles, autotune ---

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("tile", [64, 128, 256])
def test_source_tile_sizes(kernel, tile):
    b = CASES["clustered"]()
    ref, _, _ = oracle_acc(b, "clustered")
    acc, _ = gpu_forces(b, psr.Options(kernel=kernel, source_tile=tile), 32)
    assert rel_rms(acc, ref) < 2e-5
    cot = synth.cotangent(b.n, 5)
    gx_ref, gm_ref = oracle.adjoint(b.pos % b.L, b.mass, cot, b.L, b.r_s, b.r_c, b.G, cells=True)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(source_tile=tile))
    assert rel_rms(gx.double().cpu().numpy(), gx_ref) < 2e-5
    assert rel_rms(gm.double().cpu().numpy(), gm_ref) < 2e-5


def test_source_tile_values_are_checked():
    b = CASES["uniform"]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    for bad in (32, 100, 512):
        with pytest.raises(capi.PsrError) as e:
            lv.forces(psr.Options(source_tile=bad))
        assert e.value.code == capi.PSR_E_ARG


def test_autotune_picks_a_valid_tile_shape():
    b = CASES["clustered"]()
    ref, _, _ = oracle_acc(b, "clustered")
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    best, ms = lv.autotune(psr.Options(), reps=2)
    assert ms > 0
    assert best.kernel in KERNELS and best.warps_per_block in (4, 8)
    assert best.source_tile in (64, 128, 256)
    acc = lv.forces(best).double().cpu().numpy()
    assert rel_rms(acc, ref) < 2e-5


# ------------------------------------------------------- batched workload ---

def test_batch_workload_graph_replay_sampled():
    """64 boxes, N log-uniform in [8^3, 64^3], L in [50, 400], half uniform and
    half NFW-clustered: one persistent launch, autotuned, replayed from a CUDA
    graph; every box checked against the oracle on sampled targets."""
    boxes = synth.batch()
    lv = psr.Leaves.build_batch([(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G) for b in boxes],
                                max_leaf=32).upload()
    best, _ = lv.autotune(psr.Options(), reps=1)
    out = torch.zeros((lv.n, 3), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lv.forces(best, out=out)
    torch.cuda.current_stream().wait_stream(s)
    eager = out.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lv.forces(best, out=out)
    out.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    lv.check()
    acc = out.double().cpu().numpy()
    off = 0
    rng = np.random.default_rng(31)
    num = den = 0.0
    for b in boxes:
        tg = np.sort(rng.choice(b.n, min(200, b.n), replace=False))
        ref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, targets=tg, cells=True)
        d = acc[off + tg] - ref
        assert rel_rms(acc[off + tg], ref) < 5e-5, b.name
        num += np.sum(d * d)
        den += np.sum(ref * ref)
        off += b.n
    assert np.sqrt(num / den) < 2e-5


# --------------------------------------------------------------- sharding ---

@pytest.mark.parametrize("precision", [psr.PSR_FP32_TABLE, psr.PSR_FP64])
@pytest.mark.parametrize("nshard", [2, 3])
def test_shards_run_in_sequence_reproduce_the_full_launch(precision, nshard):
    """Each shard writes only its own targets, with the same arithmetic as
    the full launch: the shards run one after another on one GPU rebuild the
    full result bit for bit (forward and adjoint)."""
    b = CASES["clustered"]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    full = lv.forces(psr.Options(precision=precision)).clone()
    out = torch.full_like(full, float("nan"))
    for r in range(nshard):
        lv.forces(psr.Options(precision=precision, shard_count=nshard, shard_index=r), out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, full)
    cot = torch.tensor(synth.cotangent(b.n, 2))
    g_full, m_full = lv.adjoint(cot, psr.Options(precision=precision))
    g_full, m_full = g_full.clone(), m_full.clone()
    gp = torch.full_like(g_full, float("nan"))
    gm = torch.full_like(m_full, float("nan"))
    for r in range(nshard):
        lv.adjoint(cot, psr.Options(precision=precision, shard_count=nshard, shard_index=r), gp, gm)
    torch.cuda.synchronize()
    assert torch.equal(gp, g_full) and torch.equal(gm, m_full)
    lv.check()


def test_empty_handle_and_empty_box_in_a_batch():
    e = psr.Leaves.build(np.zeros((0, 3)), None, 10.0, 1.0, 4.5).upload()
    for prec in (psr.PSR_FP64, psr.PSR_FP32_TABLE):
        assert e.forces(psr.Options(precision=prec)).shape == (0, 3)
        gx, gm = e.adjoint(torch.zeros((0, 3)), psr.Options(precision=prec))
        assert gx.shape == (0, 3) and gm.shape == (0,)
    e.check()
    b1, b2 = _clustered(n=1500), _small_box()
    parts = [(b1.pos, b1.mass, b1.L, b1.r_s, b1.r_c, b1.G),
             (np.zeros((0, 3)), None, 40.0, b1.r_s, b1.r_c, 1.0),
             (b2.pos, b2.mass, b2.L, b2.r_s, b2.r_c, b2.G)]
    lv = psr.Leaves.build_batch(parts).upload()
    acc = lv.forces(psr.Options()).cpu().numpy()
    a1, _ = gpu_forces(b1, psr.Options())
    a2, _ = gpu_forces(b2, psr.Options())
    np.testing.assert_array_equal(acc[:b1.n], a1.astype(np.float32))
    np.testing.assert_array_equal(acc[b1.n:], a2.astype(np.float32))


# ---- the paper's Taylor table (Section 3.3, Eq. int), forward only -------

TAYLOR = [(psr.PSR_TAYLOR2, 2), (psr.PSR_TAYLOR4, 4)]


@pytest.mark.parametrize("case", ["uniform", "clustered", "small_box"])
@pytest.mark.parametrize("interp,level", TAYLOR)
@pytest.mark.parametrize("table_n", [384, 1000])
@pytest.mark.parametrize("kernel", KERNELS)
def test_taylor_table_matches_interpolated_oracle(case, interp, level, table_n, kernel):
    """Same nodes, level and nearest-node rule as the oracle's Taylor mode: what
    remains is FP32 rounding (table_n 384 is the paper's spacing 3/512)."""
    b = CASES[case]()
    ref, _, _ = oracle_acc(b, case, oracle.T_TAYLOR, table_n, level)
    acc, _ = gpu_forces(b, psr.Options(precision=psr.PSR_FP32_TABLE, table_n=table_n,
                                       interp=interp, kernel=kernel), 32)
    assert rel_rms(acc, ref) < 2e-6
    exact, _, _ = oracle_acc(b, case)
    assert rel_rms(acc, exact) < 2e-5


@pytest.mark.parametrize("interp,level", TAYLOR)
@pytest.mark.parametrize("accum", [psr.PSR_ACC_FP64, psr.PSR_ACC_KAHAN32])
def test_taylor_table_wide_leaves_and_counts(interp, level, accum):
    b = CASES["clustered"]()
    ref, pairs, _ = oracle_acc(b, "clustered", oracle.T_TAYLOR, 384, level)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=64).upload()
    o = psr.Options(precision=psr.PSR_FP32_TABLE, table_n=384, interp=interp, accum=accum)
    acc = lv.forces(o).double().cpu().numpy()
    assert rel_rms(acc, ref) < 2e-6
    lv.forces(psr.Options(precision=o.precision, table_n=384, interp=interp, count_pairs=True))
    assert abs(lv.pair_count() - int(pairs.sum())) <= max(2, int(1e-6 * pairs.sum()))
    lv.check()


@pytest.mark.parametrize("interp,level", TAYLOR)
@pytest.mark.parametrize("table_n", [64, 384, 2048])
def test_taylor_table_values(interp, level, table_n):
    x_c = 2.25
    out = torch.zeros((2 * (table_n + 1), 4), dtype=torch.float32, device="cuda")
    capi.psr_table(table_n, interp, x_c, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    tab = out.double().cpu().numpy().reshape(table_n + 1, 8)
    if level == 2:
        assert np.all(tab[:, 3:5] == 0.0)
    h = x_c / table_n
    x = np.linspace(0, x_c * (1 - 1e-9), 20011)
    k = np.rint(x / h).astype(int)
    f = x / h - k
    c = tab[k]
    val = c[:, 0] + f * (c[:, 1] + f * (c[:, 2] + f * (c[:, 3] + f * c[:, 4])))
    ref = oracle.T(x, oracle.T_TAYLOR, table_n, x_c, level)
    assert np.max(np.abs(val - ref)) < 4e-7  # FP32 rounding of the coefficients


def test_taylor_table_is_forward_only_and_runs_without_allocation():
    b = CASES["small_box"]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G).upload()
    o = psr.Options(precision=psr.PSR_FP32_TABLE, table_n=384, interp=psr.PSR_TAYLOR2)
    with pytest.raises(capi.PsrError) as e:
        lv.adjoint(torch.zeros((b.n, 3), device="cuda"), o)
    assert e.value.code == capi.PSR_E_ARG
    a1 = lv.forces(o)
    a2 = torch.empty_like(a1)
    capi.psr_p2p_forces_noalloc(lv._h, o.c(), a2.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert torch.equal(a1, a2)
    big = psr.Options(precision=psr.PSR_FP32_TABLE, table_n=2048, interp=psr.PSR_TAYLOR4)
    a3 = lv.forces(big)
    capi.psr_p2p_forces_noalloc(lv._h, big.c(), a2.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert torch.equal(a3, a2)
    lv.check()


@pytest.mark.parametrize("case", ["uniform", "clustered"])
@pytest.mark.parametrize("name,kw", [("lin1024", dict(precision=psr.PSR_FP32_TABLE)),
                                     ("exact", dict(precision=psr.PSR_FP32_EXACT))])
@pytest.mark.parametrize("accum", [psr.PSR_ACC_FP64, psr.PSR_ACC_KAHAN32])
@pytest.mark.parametrize("max_leaf", [16, 64])
@pytest.mark.parametrize("kernel", [psr.PSR_KERNEL_SCALAR, psr.PSR_KERNEL_PACKED])
def test_adjoint_fp32_two_targets_per_lane(case, name, kw, accum, max_leaf, kernel):
    """The FP32 adjoint's two-targets-per-lane path (leaves of 11-12 and 17-20
    particles at max_leaf 16/32, every leaf above 32 at max_leaf 64), both
    accumulations: every target slot of a lane must reduce correctly."""
    b = CASES[case]()
    cot = synth.cotangent(b.n, 6)
    gx_ref, gm_ref = oracle.adjoint(b.pos % b.L, b.mass, cot, b.L, b.r_s, b.r_c, b.G, cells=True)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf).upload()
    gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(accum=accum, kernel=kernel, **kw))
    lv.check()
    assert rel_rms(gx.double().cpu().numpy(), gx_ref) < 2e-5, name
    assert rel_rms(gm.double().cpu().numpy(), gm_ref) < 2e-5, name


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("max_leaf", [8, 32, 64])
def test_orb_leaves_match_oracle(case, max_leaf):
    """The paper's ORB tree (PSR_BUILD_ORB) feeds the same sum: FP64 path to
    1e-9, the FP32 table path (warp-per-leaf and the paper's block-per-leaf
    kernel) to the table tolerance."""
    b = CASES[case]()
    ref, _, _ = oracle_acc(b, case)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf,
                          orb=True).upload()
    a64 = lv.forces(psr.Options(precision=psr.PSR_FP64)).cpu().numpy()
    np.testing.assert_allclose(a64, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    for kernel in KERNELS:
        a32 = lv.forces(psr.Options(kernel=kernel)).double().cpu().numpy()
        assert rel_rms(a32, ref) < 2e-5, kernel
    lv.check()


def test_paper_kernel_sharded_and_graph_replayed():
    """Sharded launches of the block-per-leaf kernel cover every target once;
    a CUDA graph replays it."""
    b = CASES["clustered"]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
    o = psr.Options(kernel=psr.PSR_KERNEL_PAPER)
    whole = lv.forces(o).cpu().numpy()
    out = torch.full((b.n, 3), float("nan"), dtype=torch.float32, device="cuda")
    for k in range(3):
        lv.forces(psr.Options(kernel=psr.PSR_KERNEL_PAPER, shard_count=3, shard_index=k), out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), whole)
    out2 = torch.zeros((b.n, 3), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lv.forces(o, out=out2)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lv.forces(o, out=out2)
    out2.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out2.cpu().numpy(), whole)
    lv.check()


@pytest.mark.parametrize("case", ["uniform", "clustered", "small_box"])
@pytest.mark.parametrize("interp,level", TAYLOR)
@pytest.mark.parametrize("table_n", [384, 1000])
def test_fp64_taylor_table_matches_interpolated_oracle(case, interp, level, table_n):
    """PSR_FP64 with a Taylor level: the paper's double-precision table path
    (Section 3.3).  Against the oracle's Taylor mode (same nodes, level and
    nearest node) only FP64 rounding remains; against the exact oracle the
    level's truncation: T_[4] at the paper's spacing is below 1e-11, T_[2]
    below 1e-7."""
    b = CASES[case]()
    ref, pairs, _ = oracle_acc(b, case, oracle.T_TAYLOR, table_n, level)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
    o = psr.Options(precision=psr.PSR_FP64, table_n=table_n, interp=interp)
    acc = lv.forces(o).cpu().numpy()
    lv.check()
    assert acc.dtype == np.float64
    assert rel_rms(acc, ref) < 1e-12
    exact, _, _ = oracle_acc(b, case)
    assert rel_rms(acc, exact) < (1e-11 if level == 4 else 1e-7)
    lv.forces(psr.Options(precision=psr.PSR_FP64, table_n=table_n, interp=interp,
                          count_pairs=True))
    assert lv.pair_count() == int(pairs.sum())


def test_fp64_taylor_table_argument_rules():
    """Forward-only: the adjoint and the allocation-free entry point refuse
    it; switching between table kinds rebuilds the table each time."""
    b = CASES["clustered"]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
    o64 = psr.Options(precision=psr.PSR_FP64, interp=psr.PSR_TAYLOR4)
    cot = torch.zeros((b.n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(psr.PsrError) as e:
        lv.adjoint(cot, o64)
    assert e.value.code == capi.PSR_E_ARG
    out = torch.empty((b.n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(capi.PsrError) as e:
        capi.psr_p2p_forces_noalloc(lv._h, o64.c(), out.data_ptr(), 0)
    assert e.value.code == capi.PSR_E_ARG
    a1 = lv.forces(o64).cpu().numpy()
    lv.forces(psr.Options(precision=psr.PSR_FP32_TABLE, interp=psr.PSR_TAYLOR4))
    a2 = lv.forces(o64).cpu().numpy()
    np.testing.assert_array_equal(a1, a2)


def test_fp32_peak_probe_measures_a_positive_rate():
    """psr_fp32_peak: a short run gives a finite, positive FMA rate below
    twice the rate the unit counts allow at the device's largest clock, the
    sink holds the chains' finite sums, and a sink too small is refused."""
    props = torch.cuda.get_device_properties(0)
    sink = torch.full((1 << 20,), float("nan"), dtype=torch.float32, device="cuda")
    rate = capi.psr_fp32_peak(sink.data_ptr(), sink.numel() * 4, 64, 2, 0, 30000)
    nominal = props.multi_processor_count * 128 * 2 * 2.5e9
    assert 0.0 < rate < 2.0 * nominal
    used = props.multi_processor_count * 4 * 256
    assert torch.isfinite(sink[:used]).all()
    with pytest.raises(capi.PsrError) as e:
        capi.psr_fp32_peak(sink.data_ptr(), used * 4 - 4, 64, 1, 0, 30000)
    assert e.value.code == capi.PSR_E_ARG


@pytest.mark.parametrize("kernel", [psr.PSR_KERNEL_SCALAR, psr.PSR_KERNEL_PACKED,
                                    psr.PSR_KERNEL_PAPER])
@pytest.mark.parametrize("accum", [psr.PSR_ACC_FP64, psr.PSR_ACC_KAHAN32])
@pytest.mark.parametrize("max_leaf", [32, 64])
def test_equal_mass_path_matches_the_general_path(kernel, accum, max_leaf):
    """With one mass for every particle (psr_info.equal_mass) the FP32
    forward and adjoint kernels apply it once per target; the same positions
    with one mass changed by a part in 10^12 take the general per-pair form.
    Forces and both gradients agree to FP32 rounding, and the equal-mass
    results match the oracle within the FP32 tolerances."""
    b = _clustered()
    m = np.full(b.n, 0.7)
    m2 = m.copy()
    m2[5] *= 1.0 + 1e-12
    lv1 = psr.Leaves.build(b.pos, m, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf).upload()
    lv2 = psr.Leaves.build(b.pos, m2, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf).upload()
    assert lv1.info.equal_mass == 1 and lv2.info.equal_mass == 0
    o = psr.Options(kernel=kernel, accum=accum)
    a1 = lv1.forces(o).double().cpu().numpy()
    a2 = lv2.forces(o).double().cpu().numpy()
    lv1.check()
    lv2.check()
    assert rel_rms(a1, a2) < 1e-6
    ref, _, _ = oracle.forces(b.pos % b.L, m, b.L, b.r_s, b.r_c, b.G)
    assert rel_rms(a1, ref) < 2e-5
    assert max_rel(a1, ref) < MAX_REL_FP32
    cot = synth.cotangent(b.n, 9)
    g1, h1 = lv1.adjoint(torch.tensor(cot), o)
    g2, h2 = lv2.adjoint(torch.tensor(cot), o)
    g1, h1 = g1.double().cpu().numpy(), h1.double().cpu().numpy()
    g2, h2 = g2.double().cpu().numpy(), h2.double().cpu().numpy()
    assert rel_rms(g1, g2) < 1e-6 and rel_rms(h1, h2) < 1e-6
    gref, href = oracle.adjoint(b.pos % b.L, m, cot, b.L, b.r_s, b.r_c, b.G, cells=True)
    assert rel_rms(g1, gref) < 2e-5 and rel_rms(h1, href) < 2e-5


def test_equal_mass_flag_of_a_device_built_leaf_set():
    """The GPU builder detects one mass for all particles as the host builder
    does, and the forces of both leaf sets agree bit for bit."""
    b = synth.small(nside=16)
    pos = torch.tensor(b.pos, device="cuda")
    for mass in (b.mass, np.linspace(0.5, 1.5, b.n)):
        dv = psr.Leaves.device_build(pos, torch.tensor(mass, device="cuda"), b.L, b.r_s, b.r_c,
                                     b.G, max_leaf=32)
        hv = psr.Leaves.build(b.pos, mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
        eq = int(np.all(mass == mass[0]))
        assert dv.info.equal_mass == eq and hv.info.equal_mass == eq
        o = psr.Options(precision=psr.PSR_FP32_TABLE)
        assert torch.equal(dv.forces(o), hv.forces(o))
        dv.check()
    dv = psr.Leaves.device_build(pos, None, b.L, b.r_s, b.r_c, b.G, max_leaf=32)
    assert dv.info.equal_mass == 1

