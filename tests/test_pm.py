"""Long-range PM part (psr_pm_*, paper Section 2) against the PM oracle.

CPU: argument checks that need no device.  GPU: the mesh method element by
element against oracle.pm.pm_forces (same CIC, Green's function, gradient and
interpolation in FP64), with and without deconvolution, on several mesh
sizes; accumulation into the P2P result; the composition P2P + PM against the
oracle's composition; and the split's accuracy against the exact periodic
Newtonian force (short-range erfc sum far into its tail + Ewald k-space sum).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import pm as opm

psr = pytest.importorskip("paper_2107_14008_gb300")
from paper_2107_14008_gb300 import capi  # noqa: E402


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def test_pm_host_side_checks():
    for n in (0, 6, 7, 1025, 2048):
        with pytest.raises(capi.PsrError) as e:
            capi.psr_pm_create(n)
        assert e.value.code == capi.PSR_E_ARG
    with pytest.raises(capi.PsrError):
        capi.psr_pm_scratch_bytes(None)
    box = capi.psr_box(10.0, 0.5, 2.25, 1.0)
    with pytest.raises(capi.PsrError) as e:
        capi.psr_pm_forces(None, 1 << 40, 0, 10, box, 0, 1 << 40, 1 << 30, 1 << 40, 0)
    assert e.value.code == capi.PSR_E_ARG


def _clustered(n, L, n_pm, seed):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, 8, rng)
    return pos, rng.uniform(0.5, 1.5, n)


@pytest.mark.gpu
@pytest.mark.parametrize("n_pm", [16, 32, 48])
@pytest.mark.parametrize("deconvolve", [True, False])
def test_pm_matches_the_oracle_mesh_method(n_pm, deconvolve):
    import torch
    L = 50.0
    pos, mass = _clustered(4000, L, n_pm, 7 + n_pm)
    pos[:3] += [[-L, 0, 2 * L], [3 * L, -0.5, 0], [0, 0, -1e-12]]  # wrapping
    r_s = 1.2 * L / n_pm
    ref = opm.pm_forces(pos, mass, L, r_s, n_pm, deconvolve=deconvolve)
    pm = psr.PM(n_pm)
    got = pm.forces(torch.tensor(pos, device="cuda"), torch.tensor(mass, device="cuda"), L, r_s,
                    deconvolve=deconvolve).double().cpu().numpy()
    assert _rel(got, ref) < 2e-5
    # default masses are 1/n
    got1 = pm.forces(torch.tensor(pos, device="cuda"), None, L, r_s,
                     deconvolve=deconvolve).double().cpu().numpy()
    ref1 = opm.pm_forces(pos, np.full(len(pos), 1.0 / len(pos)), L, r_s, n_pm,
                         deconvolve=deconvolve)
    assert _rel(got1, ref1) < 2e-5


@pytest.mark.gpu
def test_pm_accumulates_and_handles_empty_and_bad_scratch():
    import torch
    L, n_pm = 30.0, 16
    pos, mass = _clustered(1000, L, n_pm, 3)
    pm = psr.PM(n_pm)
    p, m = torch.tensor(pos, device="cuda"), torch.tensor(mass, device="cuda")
    alone = pm.forces(p, m, L, 1.2 * L / n_pm)
    base = torch.randn((1000, 3), dtype=torch.float32, device="cuda")
    summed = pm.forces(p, m, L, 1.2 * L / n_pm, out=base.clone(), accumulate=True)
    assert torch.allclose(summed, base + alone, rtol=1e-5, atol=1e-6 * alone.abs().max().item())
    empty = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    assert pm.forces(empty, None, L, 1.0).shape == (0, 3)
    with pytest.raises(capi.PsrError) as e:
        capi.psr_pm_forces(pm._h, p.data_ptr(), m.data_ptr(), 1000, psr._box(L, 1.0, 4.5),
                           0, pm.scratch.data_ptr(), pm.scratch.numel() - 256,
                           alone.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == capi.PSR_E_WORKSPACE
    with pytest.raises(capi.PsrError) as e:
        capi.psr_pm_forces(pm._h, p.data_ptr(), m.data_ptr(), 1000, psr._box(L, 1.0, 4.5),
                           8, pm.scratch.data_ptr(), pm.scratch.numel(),
                           alone.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == capi.PSR_E_ARG


@pytest.mark.gpu
def test_p2p_plus_pm_is_the_split_force():
    """The composition on the 32^3 uniform workload (L = 100, N_PM = 32,
    r_s = 1.2 L/N_PM, r_c = 4.5 r_s): parity with the oracle's composition."""
    import torch
    b = synth.small()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
    acc = lv.forces(psr.Options())
    pm = psr.PM(b.n_pm)
    pm.forces(torch.tensor(b.pos, device="cuda"), torch.tensor(b.mass, device="cuda"), b.L,
              b.r_s, b.G, out=acc, accumulate=True)
    got = acc.double().cpu().numpy()
    short, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, cells=True)
    long_mesh = opm.pm_forces(b.pos, b.mass, b.L, b.r_s, b.n_pm, b.G)
    assert _rel(got, short + long_mesh) < 2e-5


@pytest.mark.gpu
def test_split_force_accuracy_against_the_exact_periodic_force():
    """16^3 uniform, L = 100, N_PM = 16: P2P + PM against the exact periodic
    Newtonian force (erfc sum to 11 r_s, where T < 1e-13, plus the Ewald k-space
    sum) on 300 sampled particles.  What remains is the method's error: the
    hard cutoff at T(2.25) = 1.75 % (3.7e-4 of the total here) and the mesh
    error at r_s = 1.2 cells (1.8e-3); the oracle's own composition is 1.8e-3
    from the exact force."""
    import torch
    b = synth.small(nside=16)
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=32).upload()
    acc = lv.forces(psr.Options())
    psr.PM(b.n_pm).forces(torch.tensor(b.pos, device="cuda"), torch.tensor(b.mass, device="cuda"),
                          b.L, b.r_s, b.G, out=acc, accumulate=True)
    got = acc.double().cpu().numpy()
    tg = np.random.default_rng(0).choice(b.n, 300, replace=False)
    full_short, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, 11.0 * b.r_s, b.G, targets=tg)
    exact = full_short + opm.ewald_long(b.pos, b.mass, b.L, b.r_s, b.G, targets=tg)
    assert _rel(got[tg], exact) < 5e-3
