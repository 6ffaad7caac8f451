"""Host-side tests of libpsr: exported symbols, leaf partition, pair-list
completeness against the oracle's within-cutoff pair counts, and argument
errors.  No GPU is touched (psr_build_leaves is host code)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

psr = pytest.importorskip("paper_2107_14008_gb300")
from paper_2107_14008_gb300 import capi  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2107_14008_gb300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    text = open(os.path.join(ROOT, "include", "psr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    declared = sorted(set(re.findall(r"\b(psr_[a-z0-9_]+)\s*\(", text)))
    assert declared, "no declarations found"
    assert sorted(capi.EXPORTS) == declared
    lib = ctypes.CDLL(capi.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert capi.psr_version().startswith("psr")


def _build(b, max_leaf=32, fp64=True):
    return psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf, fp64=fp64)


def _clustered(n=4000, L=60.0, seed=3, n_pm=16):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, 6, rng)
    r_s, r_c = synth.box_params(L, n_pm)
    return synth.Box(pos=pos, mass=rng.uniform(0.2, 2.0, n), L=L, n_pm=n_pm, r_s=r_s, r_c=r_c)


def _small_box():
    # r_c = 0.675 L: two images of one source can lie within r_c
    rng = np.random.default_rng(4)
    L, n = 10.0, 300
    r_s, r_c = synth.box_params(L, 8)
    return synth.Box(pos=rng.random((n, 3)) * L, mass=np.full(n, 1.0 / n), L=L, n_pm=8,
                     r_s=r_s, r_c=r_c)


CASES = {
    "uniform": lambda: synth.small(nside=16),
    "clustered": _clustered,
    "small_box": _small_box,
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("max_leaf", [1, 8, 32, 64])
def test_leaf_partition_and_local_coordinates(case, max_leaf):
    b = CASES[case]()
    lv = _build(b, max_leaf)
    A = lv.host_arrays()
    perm = lv.perm
    n = b.n
    assert np.array_equal(np.sort(perm), np.arange(n))
    leaf = A["leaf"]
    assert leaf[0, 0] == 0
    assert np.all(leaf[1:, 0] == leaf[:-1, 0] + leaf[:-1, 1])  # contiguous packs
    assert leaf[-1, 0] + leaf[-1, 1] == n
    assert leaf[:, 1].min() >= 1 and leaf[:, 1].max() <= max_leaf
    assert lv.info.max_leaf == leaf[:, 1].max()
    # FP64 copy is the wrapped position in sorted order
    wrapped = np.mod(b.pos, b.L)
    np.testing.assert_array_equal(A["pd"][:, :3], wrapped[perm])
    np.testing.assert_array_equal(A["pd"][:, 3], b.mass[perm])
    # FP32 local coordinates: (x - cell centre) / (2 r_s), inside the cell
    unit = b.L / 2.0 ** 22
    owner = np.repeat(np.arange(leaf.shape[0]), leaf[:, 1])
    cen = A["lcen"][owner, :3] * unit
    half = 0.5 * b.L / 2.0 ** A["lcen"][owner, 3]
    loc = A["pf"][:, :3].astype(np.float64) * 2 * b.r_s
    assert np.all(np.abs(loc) <= half[:, None] * (1 + 1e-6) + 1e-12)
    # one FP32 rounding of a coordinate bounded by the cell's half side
    err = np.abs(loc + cen - wrapped[perm])
    assert np.all(err <= 1.2e-7 * half[:, None] + 1e-12 * b.L)
    # centres are odd multiples of 2^(21 - level)
    lc = A["lcen"]
    step = 2 ** (21 - lc[:, 3])
    assert np.all((lc[:, :3] // step[:, None]) % 2 == 1)


def _count_listed_pairs(lv, b):
    """Within-cutoff pairs per sorted target, summed over the leaf-pair list."""
    A = lv.host_arrays()
    pd, leaf, rowptr, pairs = A["pd"], A["leaf"], A["rowptr"], A["pairs"]
    counts = np.zeros(b.n, dtype=np.int64)
    for I in range(leaf.shape[0]):
        f, c = leaf[I, 0], leaf[I, 1]
        xi = pd[f:f + c, :3]
        ent = pairs[rowptr[I]:rowptr[I + 1]]
        seen = set()
        for e in ent:
            J, code = int(e >> 5), int(e & 31)
            assert code < 27 and J < leaf.shape[0]
            assert (J, code) not in seen
            seen.add((J, code))
            nvec = np.array([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1]) * b.L
            xj = pd[leaf[J, 0]:leaf[J, 0] + leaf[J, 1], :3] + nvec
            d = xj[None, :, :] - xi[:, None, :]
            r2 = np.einsum("ijk,ijk->ij", d, d)
            counts[f:f + c] += np.sum((r2 < b.r_c ** 2) & (r2 > 0), axis=1)
        # the self pair (I, I, no shift) is always listed
        assert (I, 13) in seen
    return counts


@pytest.mark.parametrize("case", list(CASES))
def test_pair_list_is_complete(case):
    """Every pair within r_c appears in exactly one listed leaf pair: the
    per-target counts equal the oracle's brute-force counts."""
    b = CASES[case]()
    lv = _build(b, 16)
    counts = _count_listed_pairs(lv, b)
    _, ref, zero = oracle.forces(b.pos % b.L, b.mass, b.L, b.r_s, b.r_c)
    np.testing.assert_array_equal(counts, ref[lv.perm])


def test_coincident_particles_split_into_chunks():
    pos = np.vstack([np.full((100, 3), 3.0), np.random.default_rng(1).random((50, 3)) * 20])
    r_s, r_c = synth.box_params(20.0, 8)
    b = synth.Box(pos=pos, mass=np.ones(150), L=20.0, n_pm=8, r_s=r_s, r_c=r_c)
    lv = _build(b, 32)
    A = lv.host_arrays()
    assert A["leaf"][:, 1].max() <= 32
    counts = _count_listed_pairs(lv, b)
    _, ref, zero = oracle.forces(pos, b.mass, b.L, r_s, r_c)
    np.testing.assert_array_equal(counts, ref[lv.perm])
    assert zero.sum() == 100 * 99


def test_leaf_offsets_are_exact_integers():
    b = _clustered()
    lv = _build(b, 8)
    A = lv.host_arrays()
    lc = A["lcen"][:, :3].astype(np.int64)
    ent = A["pairs"]
    I = np.repeat(np.arange(lc.shape[0]), np.diff(A["rowptr"]))
    J = (ent >> 5).astype(np.int64)
    code = (ent & 31).astype(np.int64)
    nv = np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], 1)
    diff = lc[J] - lc[I] + nv * 2 ** 22
    assert np.abs(diff).max() < 2 ** 24  # exact in FP32
    unit = b.L / 2.0 ** 22
    np.testing.assert_allclose(diff * unit, lc[J] * unit + nv * b.L - lc[I] * unit, atol=1e-9)


def test_schedule_largest_first():
    b = _clustered()
    lv = _build(b, 32)
    A = lv.host_arrays()
    items = A["items"]
    assert np.array_equal(np.sort(items), np.arange(A["leaf"].shape[0]))
    leaf, rowptr, pairs = A["leaf"], A["rowptr"], A["pairs"]
    src = np.array([leaf[(pairs[rowptr[i]:rowptr[i + 1]] >> 5).astype(np.int64), 1].sum()
                    for i in range(leaf.shape[0])])
    cost = src * leaf[:, 1]
    assert np.all(np.diff(cost[items]) <= 0)
    assert lv.evaluated_pairs == cost.sum()


def test_batch_keeps_boxes_apart():
    boxes = [CASES["uniform"](), _clustered(n=1500), _small_box()]
    lv = psr.Leaves.build_batch([(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G) for b in boxes],
                                max_leaf=16)
    A = lv.host_arrays()
    nb = [b.n for b in boxes]
    first = np.concatenate([[0], np.cumsum(nb)])
    perm = lv.perm
    leaf = A["leaf"]
    for k in range(3):  # each box's particles stay in its own contiguous range
        sl = slice(first[k], first[k + 1])
        assert np.all((perm[sl] >= first[k]) & (perm[sl] < first[k + 1]))
    box_of_leaf = leaf[:, 2]
    I = np.repeat(np.arange(leaf.shape[0]), np.diff(A["rowptr"]))
    J = (A["pairs"] >> 5).astype(np.int64)
    assert np.all(box_of_leaf[I] == box_of_leaf[J])
    assert lv.info.nbox == 3


def test_argument_errors():
    b = synth.small(nside=8)
    with pytest.raises(capi.PsrError) as e:
        psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.L * 1.01, 1.0)
    assert e.value.code == capi.PSR_E_CUTOFF
    with pytest.raises(capi.PsrError) as e:
        psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.L, 1.0)
    assert e.value.code == capi.PSR_E_CUTOFF
    bad = b.pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(capi.PsrError) as e:
        psr.Leaves.build(bad, b.mass, b.L, b.r_s, b.r_c)
    assert e.value.code == capi.PSR_E_ARG
    for ml in (0, 65):
        with pytest.raises(capi.PsrError) as e:
            psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, max_leaf=ml)
        assert e.value.code == capi.PSR_E_ARG
    with pytest.raises(capi.PsrError) as e:
        psr.Leaves.build_batch([(b.pos, b.mass, b.L, b.r_s, b.r_c, 1.0),
                                (b.pos, b.mass, b.L, b.r_s, 0.9 * b.r_c, 1.0)])
    assert e.value.code == capi.PSR_E_ARG


def test_positions_outside_box_are_wrapped():
    b = synth.small(nside=8)
    shifted = b.pos + np.array([3 * b.L, -2 * b.L, b.L])
    lv0, lv1 = _build(b), psr.Leaves.build(shifted, b.mass, b.L, b.r_s, b.r_c)
    a0, a1 = lv0.host_arrays(), lv1.host_arrays()
    np.testing.assert_allclose(a1["pd"], a0["pd"], rtol=0, atol=1e-12 * b.L)
    np.testing.assert_array_equal(a1["pairs"], a0["pairs"])


def test_equal_mass_flag():
    """psr_info.equal_mass: 1 when every particle of each box has one mass
    (also for mass = NULL, which means 1/n each), 0 as soon as one differs."""
    b = synth.small(nside=8)
    assert _build(b).info.equal_mass == 1
    assert psr.Leaves.build(b.pos, None, b.L, b.r_s, b.r_c).info.equal_mass == 1
    m = b.mass.copy()
    m[17] *= 1.0 + 1e-12
    assert psr.Leaves.build(b.pos, m, b.L, b.r_s, b.r_c).info.equal_mass == 0
    c = synth.small(seed=7, nside=6)
    both = [(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G), (c.pos, c.mass, c.L, c.r_s, c.r_c, c.G)]
    assert psr.Leaves.build_batch(both).info.equal_mass == 1  # 1/512 and 1/216: one per box
    both[1] = (c.pos, np.linspace(1.0, 2.0, c.n), c.L, c.r_s, c.r_c, c.G)
    assert psr.Leaves.build_batch(both).info.equal_mass == 0


def test_fp32_peak_rejects_bad_arguments_before_any_launch():
    with pytest.raises(capi.PsrError) as e:
        capi.psr_fp32_peak(0, 1 << 20, 16, 1, 0, 1000)
    assert e.value.code == capi.PSR_E_ARG
    with pytest.raises(capi.PsrError) as e:
        capi.psr_fp32_peak(1 << 20, 1 << 20, 0, 1, 0, 1000)
    assert e.value.code == capi.PSR_E_ARG


def test_device_calls_refuse_before_upload():
    b = synth.small(nside=8)
    lv = _build(b)
    with pytest.raises(capi.PsrError) as e:
        lv.forces()
    assert e.value.code == capi.PSR_E_STATE


def test_options_marshal_to_the_c_struct_and_back():
    o = psr.Options(precision=psr.PSR_FP32_EXACT, table_n=4096, interp=psr.PSR_CUBIC,
                    accum=psr.PSR_ACC_KAHAN32, warps_per_block=4, blocks_per_sm=2, fold_every=32,
                    count_pairs=True, kernel=psr.PSR_KERNEL_PACKED, source_tile=128,
                    shard_count=3, shard_index=2)
    c = o.c()
    assert isinstance(c, capi.psr_opts)
    assert (c.precision, c.table_n, c.interp, c.accum, c.warps_per_block, c.blocks_per_sm,
            c.fold_every, c.count_pairs, c.kernel, c.source_tile, c.shard_count,
            c.shard_index) == (1, 4096, 1, 1, 4, 2, 32, 1, 2, 128, 3, 2)
    assert list(c.reserved) == [0] * len(c.reserved)
    assert psr.Options.from_c(c) == o


def test_ctypes_struct_layouts_match_the_header(tmp_path):
    """Compile a C probe against include/psr.h and compare sizes and offsets
    with the ctypes mirrors used by the binding."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    structs = {"psr_box": capi.psr_box, "psr_opts": capi.psr_opts, "psr_info": capi.psr_info,
               "psr_host_arrays": capi.psr_host_arrays, "psr_regions": capi.psr_regions}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "psr.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[name + "." + fname]) == getattr(cls, fname).offset, (name, fname)


def test_empty_inputs():
    """An empty box gives an empty handle; an empty box inside a batch adds
    no leaves and no pairs and does not disturb its neighbours."""
    e = psr.Leaves.build(np.zeros((0, 3)), None, 10.0, 1.0, 4.5)
    assert (e.n, e.info.n_leaves, e.info.n_pairs, e.evaluated_pairs) == (0, 0, 0, 0)
    assert e.perm.size == 0
    b1, b2 = synth.small(nside=8), synth.small(nside=10)
    parts = [(b1.pos, b1.mass, b1.L, b1.r_s, b1.r_c, 1.0),
             (np.zeros((0, 3)), None, 50.0, 0.5 * b1.r_s, 0.5 * b1.r_c, 1.0),
             (b2.pos, b2.mass, b2.L, b2.r_s, b2.r_c, 1.0)]
    lv = psr.Leaves.build_batch(parts, max_leaf=16)
    one = psr.Leaves.build_batch([parts[0], parts[2]], max_leaf=16)
    assert lv.n == b1.n + b2.n and lv.info.nbox == 3
    A, B = lv.host_arrays(), one.host_arrays()
    np.testing.assert_array_equal(A["pairs"], B["pairs"])
    np.testing.assert_array_equal(A["pf"], B["pf"])
    assert np.all(A["leaf"][:, 2] != 1)  # no leaf belongs to the empty box
    np.testing.assert_array_equal(np.sort(lv.perm), np.arange(lv.n))


def test_device_builder_host_side_checks():
    """Arguments psr_device_build rejects before touching a device, and the
    scratch size (a linear function of n, about 430 bytes per particle)."""
    with pytest.raises(capi.PsrError) as e:
        capi.psr_device_build_scratch_bytes(0)
    assert e.value.code == capi.PSR_E_ARG
    with pytest.raises(capi.PsrError):
        capi.psr_device_build_scratch_bytes((1 << 28) + 1)
    b1, b2 = (capi.psr_device_build_scratch_bytes(n) for n in (1 << 20, 1 << 21))
    assert 400 * (1 << 20) < b1 < 460 * (1 << 20) and abs(b2 - 2 * b1) < 1 << 16
    box = capi.psr_box(10.0, 0.5, 2.25, 1.0)
    fake = 1 << 40  # never dereferenced: every check below fails first
    for theta in (0.0, -1.0, 1.01, float("nan")):
        with pytest.raises(capi.PsrError) as e:
            capi.psr_device_build_split(fake, 0, 100, box, 32, 0, theta, fake, b1, 0, 1000)
        assert e.value.code == capi.PSR_E_ARG
    for args, code in [((0, 0, 100, box, 32, 0, fake, b1), capi.PSR_E_ARG),
                       ((fake, 0, 100, box, 0, 0, fake, b1), capi.PSR_E_ARG),
                       ((fake, 0, 100, box, 65, 0, fake, b1), capi.PSR_E_ARG),
                       ((fake, 0, 100, capi.psr_box(10.0, 0.5, 10.0, 1.0), 32, 0, fake, b1),
                        capi.PSR_E_CUTOFF),
                       ((fake, 0, 100, capi.psr_box(2e12, 1e11, 4.5e11, 1.0), 32, 0, fake, b1),
                        capi.PSR_E_ARG),
                       ((fake, 0, 100, box, 32, 0, 0, b1), capi.PSR_E_WORKSPACE),
                       ((fake, 0, 100, box, 32, 0, fake + 8, b1), capi.PSR_E_WORKSPACE),
                       ((fake, 0, 100, box, 32, 0, fake, 1000), capi.PSR_E_WORKSPACE)]:
        with pytest.raises(capi.PsrError) as e:
            capi.psr_device_build(*args, 0, 1000)
        assert e.value.code == code, args
    with pytest.raises(capi.PsrError) as e:
        capi.psr_device_build_finish(None, fake, 1 << 20, 0)
    assert e.value.code == capi.PSR_E_STATE


def test_regions_of_a_host_built_handle():
    """psr_leaves_regions: 256-byte aligned, in layout order, sized for the
    arrays psr_host_arrays describes."""
    rng = np.random.default_rng(2)
    lv = psr.Leaves.build(rng.random((3000, 3)) * 20.0, None, 20.0, 1.5, 6.75)
    r = capi.psr_leaves_regions(lv._h)
    inf = lv.info
    assert inf.rows_walked_twice == 0 and inf.n_far == 0  # device-build fields
    n, nl, npairs = 3000, inf.n_leaves, inf.n_pairs
    order = [("pf", 16 * n), ("pd", 32 * n), ("perm", 4 * n), ("leaf", 16 * nl),
             ("lcen", 16 * nl), ("rowptr", 8 * (nl + 1)), ("pairs", 4 * npairs),
             ("items", 4 * nl)]
    for (a, size), (b, _) in zip(order, order[1:]):
        assert getattr(r, a) % 256 == 0
        assert getattr(r, b) - getattr(r, a) >= size, a
    assert r.total == inf.device_bytes


def test_table_argument_checks():
    """psr_table validates its arguments before any device work: power-of-two
    interval counts for the interval tables, [64, 2048] for the Taylor
    tables (Section 3.3, Eq. int)."""
    fake = 1 << 40  # never written: every call below fails its checks first
    for n, interp in [(384, capi.PSR_LINEAR), (384, capi.PSR_CUBIC), (32, capi.PSR_LINEAR),
                      (16384, capi.PSR_CUBIC), (4096, capi.PSR_TAYLOR2), (63, capi.PSR_TAYLOR4),
                      (1024, 4), (1024, -1)]:
        with pytest.raises(capi.PsrError) as e:
            capi.psr_table(n, interp, 2.25, fake, 0)
        assert e.value.code == capi.PSR_E_ARG, (n, interp)
    with pytest.raises(capi.PsrError) as e:
        capi.psr_table(384, capi.PSR_TAYLOR2, -1.0, fake, 0)
    assert e.value.code == capi.PSR_E_ARG


def _orb_leaf_sizes(n, max_leaf):
    """Leaf sizes of equal-halves bisection (paper, Section 2: a cell's
    particles are split equally between two children until at most
    MAXLEAF remain), in leaf order, by recursion on the counts alone."""
    if n <= max_leaf:
        return [n]
    return _orb_leaf_sizes(n // 2, max_leaf) + _orb_leaf_sizes(n - n // 2, max_leaf)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("max_leaf", [1, 8, 32, 64])
def test_orb_leaves_are_equal_halves(case, max_leaf):
    """PSR_BUILD_ORB: the leaf sizes are those of equal halving (so that no
    two leaves differ by more than one particle for a count that is not a
    power-of-two multiple); each leaf's particles lie in its box; every
    particle once; the FP32 local coordinates round the offset from the
    leaf's reference point (its box centre on the L / 2^22 grid) once."""
    b = CASES[case]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf, orb=True)
    A = lv.host_arrays()
    perm = lv.perm
    assert np.array_equal(np.sort(perm), np.arange(b.n))
    leaf = A["leaf"]
    assert list(leaf[:, 1]) == _orb_leaf_sizes(b.n, max_leaf)
    assert np.all(leaf[1:, 0] == leaf[:-1, 0] + leaf[:-1, 1])
    wrapped = np.mod(b.pos, b.L)[perm]
    np.testing.assert_array_equal(A["pd"][:, :3], wrapped)
    unit = b.L / 2.0 ** 22
    owner = np.repeat(np.arange(leaf.shape[0]), leaf[:, 1])
    lo = np.minimum.reduceat(wrapped, leaf[:, 0], axis=0)
    hi = np.maximum.reduceat(wrapped, leaf[:, 0], axis=0)
    ref = np.clip(np.floor(0.5 * (lo + hi) / unit + 0.5), 0, 2 ** 22 - 1)
    np.testing.assert_array_equal(A["lcen"][:, :3], ref.astype(np.int32))
    loc = A["pf"][:, :3].astype(np.float64) * 2 * b.r_s
    cen = A["lcen"][owner, :3] * unit
    span = np.max(hi - lo, axis=1)[owner] + unit
    assert np.all(np.abs(loc + cen - wrapped) <= 1.2e-7 * span[:, None] + 1e-12 * b.L)


def test_orb_splits_along_the_longest_axis():
    """A slab 8 x 1 x 1: the first three splits cut x (extents 8, 4, 2
    against 1), so the first eighth of the particles in ORB order are those
    of smallest x."""
    rng = np.random.default_rng(9)
    n = 1024
    pos = rng.random((n, 3)) * [8.0, 1.0, 1.0] + [1.0, 1.0, 1.0]
    L = 20.0
    r_s, r_c = synth.box_params(L, 16)
    lv = psr.Leaves.build(pos, None, L, r_s, r_c, 1.0, max_leaf=32, orb=True)
    assert set(lv.perm[:n // 8]) == set(np.argsort(pos[:, 0])[:n // 8])
    assert set(lv.perm[:n // 2]) == set(np.argsort(pos[:, 0])[:n // 2])


@pytest.mark.parametrize("case", list(CASES))
def test_orb_pair_list_is_complete(case):
    b = CASES[case]()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=16, orb=True)
    counts = _count_listed_pairs(lv, b)
    _, ref, zero = oracle.forces(b.pos % b.L, b.mass, b.L, b.r_s, b.r_c)
    np.testing.assert_array_equal(counts, ref[lv.perm])


def test_build_flag_checks():
    b = CASES["uniform"]()
    with pytest.raises(psr.PsrError) as e:
        capi.psr_build_leaves(np.ascontiguousarray(b.pos).ctypes.data_as(
            __import__("ctypes").POINTER(__import__("ctypes").c_double)), None, b.n,
            capi.psr_box(b.L, b.r_s, b.r_c, 1.0), 32, 8)
    assert e.value.code == capi.PSR_E_ARG
    box = capi.psr_box(10.0, 0.5, 2.25, 1.0)
    fake = 1 << 40  # never dereferenced: the flag check fails first
    with pytest.raises(capi.PsrError) as e:
        capi.psr_device_build(fake, 0, 100, box, 32, capi.PSR_BUILD_ORB, fake,
                              capi.psr_device_build_scratch_bytes(100), 0, 1000)
    assert e.value.code == capi.PSR_E_ARG


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("max_leaf", [1, 8, 32])
def test_leaf_packing_merges_consecutive_siblings(case, max_leaf):
    """Default (packed) leaves against PSR_BUILD_UNPACKED on the same input:
    the same particle order; every packed leaf is a run of consecutive
    unpacked leaves of one level L and one parent cell, with the parent's
    cell (level L - 1) when the run has several; runs are greedy: the next
    sibling starts a new pack only when it would take the pack past
    max_leaf."""
    b = CASES[case]()
    pk = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf)
    up = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=max_leaf, pack=False)
    assert np.array_equal(pk.perm, up.perm)
    P, U = pk.host_arrays(), up.host_arrays()
    ustart = {int(f): i for i, f in enumerate(U["leaf"][:, 0])}
    step = lambda lvl: 2 ** (21 - lvl)
    parent = lambda lc: tuple((lc[:3] // (2 * step(lc[3] - 1))).tolist()) + (int(lc[3]) - 1,)
    for g in range(P["leaf"].shape[0]):
        f, c = int(P["leaf"][g, 0]), int(P["leaf"][g, 1])
        i = ustart[f]  # packs start on an unpacked leaf boundary
        j, tot = i, 0
        while tot < c:
            tot += int(U["leaf"][j, 1])
            j += 1
        assert tot == c
        run = U["lcen"][i:j]
        if j - i == 1:
            assert np.array_equal(P["lcen"][g], run[0])
            continue
        assert np.all(run[:, 3] == run[0, 3]) and run[0, 3] >= 1
        assert len({parent(r) for r in run}) == 1
        lv = run[0, 3] - 1
        expect = (np.array(parent(run[0])[:3]) * 2 + 1) * step(lv)
        assert np.array_equal(P["lcen"][g, :3], expect) and P["lcen"][g, 3] == lv
    # greedy: a pack followed by an unpacked sibling of the same parent ends
    # only because that sibling would not fit
    for g in range(P["leaf"].shape[0] - 1):
        f2 = int(P["leaf"][g + 1, 0])
        nxt = ustart[f2]
        prev = nxt - 1
        a, b_ = U["lcen"][prev], U["lcen"][nxt]
        if a[3] == b_[3] and a[3] >= 1 and parent(a) == parent(b_) and \
                int(U["leaf"][nxt, 1]) <= max_leaf:
            # same parent, both plain leaves: the split must be forced by size
            # (or by an over-full finest cell's chunks, which never pack)
            chunk = a[3] == 21 and np.array_equal(a[:3], b_[:3])
            assert chunk or int(P["leaf"][g, 1]) + int(U["leaf"][nxt, 1]) > max_leaf
