"""Truncated multipole operators (psr_fmm_*, paper Section 2) against the
pinned FP64 oracle (oracle/fmm.py).

CPU: coefficient counts and the argument checks made before any device work.
GPU: P2M moments, M2L local coefficients (with periodic images) and L2P
accelerations element by element against the oracle's operators, in the
library's scaled form (Mh_m = M_m / h^|m|, Lh_n = L_n h^(|n|+1)); the chain
P2M -> M2L -> L2P against the oracle's chain and its convergence to the
direct sum; the status bits for bad entries.
"""
import numpy as np
import pytest

from oracle import fmm as ofmm

psr = pytest.importorskip("paper_2107_14008_gb300")
from paper_2107_14008_gb300 import capi  # noqa: E402


def test_coefficient_counts_and_host_side_checks():
    assert [capi.psr_fmm_ncoef(p) for p in range(7)] == [1, 4, 10, 20, 35, 56, 84]
    assert [len(ofmm.multi_indices(p)) for p in range(7)] == [1, 4, 10, 20, 35, 56, 84]
    with pytest.raises(capi.PsrError):
        capi.psr_fmm_ncoef(7)
    box = capi.psr_box(10.0, 0.5, 2.25, 1.0)
    fake = 1 << 40  # never dereferenced: every call below fails its checks first
    for p, h in [(0, 1.0), (7, 1.0), (3, 0.0), (3, float("nan"))]:
        with pytest.raises(capi.PsrError) as e:
            capi.psr_fmm_p2m(p, h, 10, 2, fake, fake, 0, fake, fake, 0)
        assert e.value.code == capi.PSR_E_ARG
        with pytest.raises(capi.PsrError):
            capi.psr_fmm_m2l(p, h, box, 2, 2, fake, fake, fake, fake, fake, fake, 0, 0)
        with pytest.raises(capi.PsrError):
            capi.psr_fmm_l2p(p, h, box, 2, fake, fake, fake, fake, fake, 0, 0)
    with pytest.raises(capi.PsrError):
        capi.psr_fmm_p2m(3, 1.0, 10, 2, 0, fake, 0, fake, fake, 0)
    with pytest.raises(capi.PsrError):
        capi.psr_fmm_l2p(3, 1.0, box, 2, fake, fake, fake, fake, fake, 4, 0)
    with pytest.raises(capi.PsrError):
        capi.psr_fmm_m2l(3, 1.0, capi.psr_box(10.0, 0.0, 2.25, 1.0), 2, 2, fake, fake, fake,
                         fake, fake, fake, 0, 0)
    with pytest.raises(capi.PsrError) as e:  # no handle
        capi.psr_fmm_forces(None, 4, 0, fake, fake, fake, 0, 0)
    assert e.value.code == capi.PSR_E_ARG


def _scale_M(M, p, h):
    return np.array([M[i] / h ** sum(n) for i, n in enumerate(ofmm.multi_indices(p))])


def _scale_L(L, p, h):
    return np.array([L[i] * h ** (sum(n) + 1) for i, n in enumerate(ofmm.multi_indices(p))])


def _cells(rng, ncell, per, half, spread):
    """Cells of `per` particles within +-half of centres spread over a box."""
    centres = rng.uniform(0, spread, (ncell, 3))
    pos = np.concatenate([c + rng.uniform(-half, half, (per, 3)) for c in centres])
    mass = rng.uniform(0.5, 1.5, ncell * per)
    first = np.arange(ncell + 1, dtype=np.int64) * per
    return centres, pos, mass, first


def _dev(a, dt):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _gpu_p2m(p, h, centres, pos, mass, first):
    import torch
    nc = capi.psr_fmm_ncoef(p)
    M = torch.zeros((len(centres), nc), dtype=torch.float32, device="cuda")
    f, x, m, c = (_dev(first, torch.int64), _dev(pos, torch.float64), _dev(mass, torch.float64),
                  _dev(centres, torch.float64))
    capi.psr_fmm_p2m(p, h, len(pos), len(centres), f.data_ptr(), x.data_ptr(), m.data_ptr(),
                     c.data_ptr(), M.data_ptr(), _stream())
    return M


def _rows(ct, cs, L, min_sep, max_sep, images=True):
    """CSR rows: every (source, image) whose shifted centre lies between
    min_sep and max_sep from the target centre (image codes 13 and, if asked,
    14)."""
    rowptr, pairs, shifts = [0], [], []
    for t in range(len(ct)):
        for s in range(len(cs)):
            for code in ((13, 14) if images else (13,)):
                sh = np.array([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1]) * L
                if min_sep <= np.linalg.norm(ct[t] - cs[s] - sh) <= max_sep:
                    pairs.append((s << 5) | code)
                    shifts.append(sh)
        rowptr.append(len(pairs))
    return np.array(rowptr, np.int64), np.array(pairs, np.uint32)


def _oracle_L(p, r_s, ct, cs, L, rowptr, pairs, Ms):
    out = []
    for t in range(len(ct)):
        acc = np.zeros(len(ofmm.multi_indices(p)))
        for e in range(rowptr[t], rowptr[t + 1]):
            s, code = int(pairs[e]) >> 5, int(pairs[e]) & 31
            sh = np.array([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1]) * L
            acc += ofmm.m2l(Ms[s], ct[t] - (cs[s] + sh), r_s, p)
        out.append(acc)
    return np.array(out)


@pytest.mark.gpu
@pytest.mark.parametrize("p", [1, 3, 6])
def test_p2m_matches_the_oracle(p):
    rng = np.random.default_rng(p)
    h = 0.8
    centres, pos, mass, first = _cells(rng, 12, 20, 0.5 * h, 10.0)
    M = _gpu_p2m(p, h, centres, pos, mass, first).double().cpu().numpy()
    for c in range(len(centres)):
        sl = slice(first[c], first[c + 1])
        ref = _scale_M(ofmm.p2m(pos[sl], mass[sl], centres[c], p), p, h)
        assert np.max(np.abs(M[c] - ref)) <= 2e-6 * np.max(np.abs(ref)), c


@pytest.mark.gpu
@pytest.mark.parametrize("p", [2, 4, 6])
@pytest.mark.parametrize("r_s", [0.6, 1.5, 20.0])
def test_m2l_matches_the_oracle_with_images(p, r_s):
    import torch
    rng = np.random.default_rng(10 + p)
    h, L = 1.0, 12.0
    cs, spos, smass, sfirst = _cells(rng, 10, 8, 0.5 * h, L)
    ct = rng.uniform(0, L, (6, 3))
    rowptr, pairs = _rows(ct, cs, L, 2.5 * h, 4.5 * r_s + 2.0 * h)
    Ms_raw = [ofmm.p2m(spos[sfirst[s]:sfirst[s + 1]], smass[sfirst[s]:sfirst[s + 1]], cs[s], p)
              for s in range(len(cs))]
    ref = np.array([_scale_L(l, p, h) for l in _oracle_L(p, r_s, ct, cs, L, rowptr, pairs, Ms_raw)])
    M = _dev(np.array([_scale_M(m, p, h) for m in Ms_raw]), torch.float32)
    Lg = torch.zeros((len(ct), capi.psr_fmm_ncoef(p)), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rp, pr = _dev(rowptr, torch.int64), _dev(pairs.view(np.int32), torch.int32)
    ctd, csd = _dev(ct, torch.float64), _dev(cs, torch.float64)
    capi.psr_fmm_m2l(p, h, capi.psr_box(L, r_s, 4.5 * r_s, 1.0), len(ct), len(cs), rp.data_ptr(),
                     pr.data_ptr(), ctd.data_ptr(), csd.data_ptr(), M.data_ptr(), Lg.data_ptr(),
                     st.data_ptr(), _stream())
    got = Lg.double().cpu().numpy()
    assert int(st.item()) == 0
    assert rowptr[-1] > 0
    for t in range(len(ct)):
        if rowptr[t + 1] == rowptr[t]:
            assert np.all(got[t] == 0.0)
            continue
        err = np.sqrt(np.sum((got[t] - ref[t]) ** 2) / np.sum(ref[t] ** 2))
        assert err < 1e-4, (t, err)


def _gpu_chain(p, h, r_s, G, L, src, tgt, rowptr, pairs):
    import torch
    (cs, spos, smass, sfirst), (ct, tpos, tfirst) = src, tgt
    M = _gpu_p2m(p, h, cs, spos, smass, sfirst)
    nc = capi.psr_fmm_ncoef(p)
    Lg = torch.zeros((len(ct), nc), dtype=torch.float32, device="cuda")
    rp, pr = _dev(rowptr, torch.int64), _dev(pairs.view(np.int32), torch.int32)
    ctd, csd = _dev(ct, torch.float64), _dev(cs, torch.float64)
    box = capi.psr_box(L, r_s, 4.5 * r_s, G)
    capi.psr_fmm_m2l(p, h, box, len(ct), len(cs), rp.data_ptr(), pr.data_ptr(), ctd.data_ptr(),
                     csd.data_ptr(), M.data_ptr(), Lg.data_ptr(), 0, _stream())
    acc = torch.full((len(tpos), 3), 7.0, dtype=torch.float32, device="cuda")
    tf, tp = _dev(tfirst, torch.int64), _dev(tpos, torch.float64)
    capi.psr_fmm_l2p(p, h, box, len(ct), tf.data_ptr(), tp.data_ptr(), ctd.data_ptr(),
                     Lg.data_ptr(), acc.data_ptr(), capi.PSR_FMM_ACCUMULATE, _stream())
    return acc.double().cpu().numpy() - 7.0


@pytest.mark.gpu
def test_chain_matches_the_oracle_and_converges_to_the_direct_sum():
    rng = np.random.default_rng(3)
    h, r_s, G, L = 1.0, 1.2, 1.7, 1000.0
    cs, spos, smass, sfirst = _cells(rng, 1, 40, 0.5 * h, 0.0)
    ct = np.array([[2.4, 1.1, -0.7]])
    tpos = ct[0] + rng.uniform(-0.5 * h, 0.5 * h, (30, 3))
    tfirst = np.array([0, 30], np.int64)
    rowptr, pairs = np.array([0, 1], np.int64), np.array([13], np.uint32)
    direct = ofmm.direct(spos, smass, tpos, r_s, G)
    errs = []
    for p in range(1, 7):
        got = _gpu_chain(p, h, r_s, G, L, (cs, spos, smass, sfirst), (ct, tpos, tfirst),
                         rowptr, pairs)
        Lo = ofmm.m2l(ofmm.p2m(spos, smass, cs[0], p), ct[0] - cs[0], r_s, p)
        ref = ofmm.l2p(Lo, ct[0], tpos, p, G)
        assert np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2)) < 1e-4, p
        errs.append(np.sqrt(np.sum((got - direct) ** 2) / np.sum(direct ** 2)))
    assert all(e1 < 0.7 * e0 for e0, e1 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2


@pytest.mark.gpu
def test_m2l_status_bits_and_skipped_entries():
    import torch
    rng = np.random.default_rng(4)
    h, r_s, L, p = 1.0, 1.0, 50.0, 3
    cs, spos, smass, sfirst = _cells(rng, 2, 5, 0.5, 0.0)
    cs[1] = cs[0] + [3.0, 0.0, 0.0]
    ct = np.array(cs[:1])
    M = _gpu_p2m(p, h, cs, spos, smass, sfirst)
    good = np.array([(1 << 5) | 13], np.uint32)
    bad = np.array([(1 << 5) | 13, (7 << 5) | 13, (0 << 5) | 13, (1 << 5) | 30], np.uint32)
    out = []
    for pairs in (good, bad):
        Lg = torch.zeros((1, capi.psr_fmm_ncoef(p)), dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        rp, pr = _dev([0, len(pairs)], torch.int64), _dev(pairs.view(np.int32), torch.int32)
        ctd, csd = _dev(ct, torch.float64), _dev(cs, torch.float64)
        capi.psr_fmm_m2l(p, h, capi.psr_box(L, r_s, 4.5, 1.0), 1, 2, rp.data_ptr(), pr.data_ptr(),
                         ctd.data_ptr(), csd.data_ptr(), M.data_ptr(), Lg.data_ptr(), st.data_ptr(),
                         _stream())
        out.append((Lg.cpu().numpy(), int(st.item())))
    assert out[0][1] == 0 and out[1][1] == 3  # out of range, then coincident centres
    assert np.array_equal(out[0][0], out[1][0])  # bad entries skipped, the good one kept


@pytest.mark.gpu
@pytest.mark.parametrize("h", [1.0, 300.0, 0.003])
def test_chain_on_tiny_close_cells_for_any_scale(h):
    """Cells 4e-3 across, 0.05 apart, order 6: at h = 300 the prefactor
    h^13 f_(6)(|R|) alone is far outside FP32; each entry forms its
    derivatives at the scale |R| and rescales, so every h gives the oracle's
    chain."""
    rng = np.random.default_rng(21)
    r_s, G, L, p = 0.7, 1.3, 50.0, 6
    cs, spos, smass, sfirst = _cells(rng, 1, 25, 2e-3, 0.0)
    cs += 10.0
    spos += 10.0
    ct = cs + np.array([[0.03, -0.035, 0.02]])
    tpos = ct[0] + rng.uniform(-2e-3, 2e-3, (20, 3))
    tfirst = np.array([0, 20], np.int64)
    rowptr, pairs = np.array([0, 1], np.int64), np.array([13], np.uint32)
    got = _gpu_chain(p, h, r_s, G, L, (cs, spos, smass, sfirst), (ct, tpos, tfirst), rowptr, pairs)
    Lo = ofmm.m2l(ofmm.p2m(spos, smass, cs[0], p), ct[0] - cs[0], r_s, p)
    ref = ofmm.l2p(Lo, ct[0], tpos, p, G)
    assert np.all(np.isfinite(got))
    assert np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2)) < 1e-4


@pytest.mark.gpu
def test_m2l_ragged_rows_across_lane_groups():
    """Rows of 0 .. 40 entries for 37 targets (not a multiple of the targets
    a warp serves), every entry a well-separated pair inside the cutoff."""
    import torch
    rng = np.random.default_rng(22)
    h, r_s, L, p = 1.0, 8.0, 64.0, 4
    cs, spos, smass, sfirst = _cells(rng, 50, 6, 0.5 * h, L)
    ct = rng.uniform(0, L, (37, 3))
    rowptr, pairs = [0], []
    for t in range(len(ct)):
        cand = [s for s in rng.permutation(len(cs))
                if 2.5 * h < np.linalg.norm(ct[t] - cs[s]) < 4.5 * r_s]
        pairs += [(int(s) << 5) | 13 for s in cand[:(t * 7) % 41]]
        rowptr.append(len(pairs))
    rowptr, pairs = np.array(rowptr, np.int64), np.array(pairs, np.uint32)
    Ms_raw = [ofmm.p2m(spos[sfirst[s]:sfirst[s + 1]], smass[sfirst[s]:sfirst[s + 1]], cs[s], p)
              for s in range(len(cs))]
    ref = np.array([_scale_L(l, p, h) for l in _oracle_L(p, r_s, ct, cs, L, rowptr, pairs, Ms_raw)])
    M = _dev(np.array([_scale_M(m, p, h) for m in Ms_raw]), torch.float32)
    Lg = torch.full((len(ct), capi.psr_fmm_ncoef(p)), 5.0, dtype=torch.float32, device="cuda")
    rp, pr = _dev(rowptr, torch.int64), _dev(pairs.view(np.int32), torch.int32)
    ctd, csd = _dev(ct, torch.float64), _dev(cs, torch.float64)
    capi.psr_fmm_m2l(p, h, capi.psr_box(L, r_s, 4.5 * r_s, 1.0), len(ct), len(cs), rp.data_ptr(),
                     pr.data_ptr(), ctd.data_ptr(), csd.data_ptr(), M.data_ptr(), Lg.data_ptr(), 0,
                     _stream())
    got = Lg.double().cpu().numpy()
    for t in range(len(ct)):
        if rowptr[t + 1] == rowptr[t]:
            assert np.all(got[t] == 0.0), t
        else:
            err = np.sqrt(np.sum((got[t] - ref[t]) ** 2) / np.sum(ref[t] ** 2))
            assert err < 1e-4, (t, err)
