"""The large workload at its full size: 512^3 particles (134 M), periodic
L = 1000, N_PM = 512, 70 % of the mass in 200000 NFW halos, leaves <= 64.
The leaf set is built on the GPU (the path the benchmark times), the FP32
table forward and the FP32 adjoint run in the benchmark's launch
configuration, and sampled targets are checked against the FP64 oracle:
forces on 1000 targets at the FP32 tolerance (relative RMS 2e-5, per
particle 2.5e-4 of max(|a_i|, 1e-3 rms|a|)), the adjoint on 200 targets at
2e-5.  The pair-counting launch's counts must be ordered: pairs within the
cutoff, pair terms evaluated after the cull, pairs of the leaf-pair tiles.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
psr = pytest.importorskip("paper_2107_14008_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14008_gb300 import build
    build.build()


def rel(a, ref):
    return float(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2)))


def max_rel(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(nr * nr))
    return float(np.max(np.linalg.norm(a - ref, axis=1) / np.maximum(nr, floor)))


def test_large_workload_sampled_against_oracle():
    b = synth.large()
    dev = torch.device("cuda")
    lv = psr.Leaves.device_build(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.mass).to(dev),
                                 b.L, b.r_s, b.r_c, b.G, max_leaf=b.max_leaf, fp64=False)
    acc = lv.forces(psr.Options()).double().cpu().numpy()
    lv.check()
    rng = np.random.default_rng(512)
    tg = np.sort(rng.choice(b.n, 1000, replace=False))
    ref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, targets=tg, cells=True)
    assert np.all(np.isfinite(acc))
    assert rel(acc[tg], ref) < 2e-5
    assert max_rel(acc[tg], ref) < 2.5e-4
    # the counting launch: pairs within the cutoff <= pair terms evaluated
    # after the cull <= pairs of the leaf-pair tiles
    lv.forces(psr.Options(count_pairs=True))
    within = lv.pair_count()
    assert 0 < within <= lv.evaluated_count() <= lv.evaluated_pairs
    cot = synth.cotangent(b.n, 12349)
    gx, gm = lv.adjoint(torch.from_numpy(cot).to(device=dev, dtype=torch.float32), psr.Options())
    lv.check()
    ta = tg[::5]
    gref, mref = oracle.adjoint(b.pos, b.mass, cot, b.L, b.r_s, b.r_c, b.G, targets=ta, cells=True)
    assert rel(gx.double().cpu().numpy()[ta], gref) < 2e-5
    assert rel(gm.double().cpu().numpy()[ta], mref) < 2e-5
