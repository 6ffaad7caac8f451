"""The differentiation workload: 64^3 particles, 60 % of the mass in NFW halos,
periodic L = 200, N_PM = 64 (r_s = 1.2 L/N_PM, r_c = 4.5 r_s).

Forward forces, then the adjoint of L = sum_i c_i . a_i with a seeded N(0,1)
cotangent on every force component, in FP64 and FP32, on 200 sampled
particles:
  * the FP64 adjoint against central finite differences of L in FP64
    (h = 1e-6 L, Richardson-extrapolated over h and h/2), with the set of
    interacting pairs frozen at the unperturbed positions (the gradient of the
    piecewise sum with its hard cutoff): dL/dx within 1e-5 rel L2 over the
    200 x 3 components, dL/dm (exactly linear in m) within 1e-8;
  * the FP64 adjoint against the oracle's gradient (1e-6) and the FP32
    adjoint against it at the FP32 force tolerance (2e-5);
  * the same through the autograd function on GPU tensors, whose leaf set is
    built on the GPU.
The adjoint's arithmetic is the n = 2 truncated prefactor of Section 2
applied to the pair force of Eq. tr.
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
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2)))


@pytest.fixture(scope="module")
def workload():
    b = synth.adjoint()
    cot = synth.cotangent(b.n, 12348)
    tg = np.sort(np.random.default_rng(200).choice(b.n, 200, replace=False))
    fd = [oracle.fd_gradient(b.pos, b.mass, cot, p, b.L, b.r_s, b.r_c, b.G, richardson=True)
          for p in tg]
    fdx = np.array([g for g, _ in fd])
    fdm = np.array([m for _, m in fd])
    gref, mref = oracle.adjoint(b.pos, b.mass, cot, b.L, b.r_s, b.r_c, b.G, targets=tg,
                                cells=True)
    aref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, targets=tg, cells=True)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=b.max_leaf).upload()
    return b, cot, tg, fdx, fdm, gref, mref, aref, lv


def test_oracle_gradient_agrees_with_finite_differences(workload):
    """The oracle's analytic gradient and the frozen-set finite differences
    are two independent routes to the same derivative."""
    b, cot, tg, fdx, fdm, gref, mref, aref, lv = workload
    assert rel(gref, fdx) < 1e-5
    assert rel(mref, fdm) < 1e-8


def test_forward_on_the_sampled_particles(workload):
    b, cot, tg, fdx, fdm, gref, mref, aref, lv = workload
    a64 = lv.forces(psr.Options(precision=psr.PSR_FP64)).cpu().numpy()
    assert rel(a64[tg], aref) < 1e-6
    a32 = lv.forces(psr.Options()).double().cpu().numpy()
    assert rel(a32[tg], aref) < 2e-5
    lv.check()


def test_fp64_adjoint_against_finite_differences_and_oracle(workload):
    b, cot, tg, fdx, fdm, gref, mref, aref, lv = workload
    gx, gm = lv.adjoint(torch.tensor(cot), psr.Options(precision=psr.PSR_FP64))
    gx, gm = gx.cpu().numpy()[tg], gm.cpu().numpy()[tg]
    lv.check()
    assert rel(gx, fdx) < 1e-5
    assert rel(gm, fdm) < 1e-8
    assert rel(gx, gref) < 1e-6
    assert rel(gm, mref) < 1e-6


@pytest.mark.parametrize("accum", [psr.PSR_ACC_FP64, psr.PSR_ACC_KAHAN32])
@pytest.mark.parametrize("kw", [dict(), dict(precision=psr.PSR_FP32_EXACT),
                                dict(table_n=4096, interp=psr.PSR_CUBIC),
                                dict(kernel=psr.PSR_KERNEL_PACKED)])
def test_fp32_adjoint_against_oracle_and_finite_differences(workload, accum, kw):
    b, cot, tg, fdx, fdm, gref, mref, aref, lv = workload
    gx, gm = lv.adjoint(torch.tensor(cot, dtype=torch.float32), psr.Options(accum=accum, **kw))
    gx, gm = gx.double().cpu().numpy()[tg], gm.double().cpu().numpy()[tg]
    lv.check()
    assert rel(gx, gref) < 2e-5
    assert rel(gm, mref) < 2e-5
    assert rel(gx, fdx) < 2e-5


def test_autograd_on_gpu_tensors_uses_a_device_built_leaf_set(workload):
    """psr.forces on CUDA tensors builds the leaf set on the GPU; backward runs
    the adjoint on it."""
    b, cot, tg, fdx, fdm, gref, mref, aref, lv = workload
    pos = torch.tensor(b.pos, device="cuda", requires_grad=True)
    mass = torch.tensor(b.mass, device="cuda", requires_grad=True)
    acc = psr.forces(pos, mass, b.L, b.r_s, b.r_c, b.G, psr.Options(precision=psr.PSR_FP64))
    (acc * torch.tensor(cot, device="cuda")).sum().backward()
    assert rel(acc.detach().cpu().numpy()[tg], aref) < 1e-6
    assert rel(pos.grad.cpu().numpy()[tg], fdx) < 1e-5
    assert rel(mass.grad.cpu().numpy()[tg], mref) < 1e-6
