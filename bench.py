#!/usr/bin/env python
"""Benchmark of the truncated short-range P2P gravity on one GB300.

Metric: pair interactions per second (G/s) of the FP32-table forward path,
with the plain FP64 path timed beside it, and % of FP32 peak at the paper's
51 flops per interaction (Section 5).  Workload: 128^3 particles, 60 % of the
mass in 4000 NFW halos + 40 % uniform, periodic L = 500, N_PM = 128 (r_s =
1.2 L/N_PM, r_c = 4.5 r_s), octree leaves <= 32 (seeded synthetic stand-in for
the paper's cosmological initial conditions).

A step is one forward evaluation over the whole particle set (kernel with the
un-permute fused) with the leaf set resident on the device; the leaf build is
host work reported separately and included in the end-to-end number.  Each
timed step is bracketed by CUDA events on the launching stream; L2 is flushed
(256 MB write) between steps.  `--gpus N` (torchrun) gives every rank its own
box of the same workload (weak scaling, no collective on the data path).

`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_INTERACTION = 51  # paper, Section 5
METRIC = "G pair-interactions/s & % FP32 peak, FP32-table vs FP64 path, at stated force err"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="psr", choices=["psr", "reference"])
    p.add_argument("--table-n", type=int, default=1024)
    p.add_argument("--interp", default="linear", choices=["linear", "cubic"])
    p.add_argument("--accum", default="fp64", choices=["fp64", "kahan"])
    p.add_argument("--kernel", default="scalar", choices=["scalar", "packed"],
                   help="FP32 forward inner loop: scalar streams (the default) or packed f32x2 "
                        "pairs")
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--adjoint-steps", type=int, default=3)
    p.add_argument("--batch-steps", type=int, default=10)
    p.add_argument("--fmm-steps", type=int, default=3,
                   help="steps of the truncated multipole operators on the leaves (0: skip)")
    p.add_argument("--fmm-order", type=int, default=4)
    p.add_argument("--split-steps", type=int, default=3,
                   help="timed steps of the split short range (P2P near + multipole far)")
    p.add_argument("--split-theta", default="0.5,0.7",
                   help="opening parameters of the split (the first also with the Gaussian term)")
    p.add_argument("--split-orders", default="4,6")
    p.add_argument("--paper-steps", type=int, default=3,
                   help="timed steps of each prior-art variant (the paper's block-per-leaf "
                        "kernel, ORB leaves)")
    p.add_argument("--pm-steps", type=int, default=5,
                   help="steps of the long-range PM part on the same box (0: skip)")
    p.add_argument("--large-steps", type=int, default=3,
                   help="timed forward and adjoint steps of the 512^3 large workload, built on "
                        "the GPU and validated against the oracle on sampled targets (0: skip)")
    p.add_argument("--large-targets", type=int, default=10000,
                   help="oracle targets that validate the large workload's forces (the adjoint "
                        "takes a tenth of them)")
    p.add_argument("--no-variants", dest="variants", action="store_false",
                   help="skip the precision study (one launch per T variant)")
    p.add_argument("--autograd-steps", type=int, default=5,
                   help="timed forward + backward steps through psr.forces (torch autograd)")
    p.add_argument("--peak-launches", type=int, default=5,
                   help="launches of the FP32 FMA-rate microbenchmark (psr_fp32_peak); 0 skips it")
    p.add_argument("--peak-iters", type=int, default=65536,
                   help="iterations of 64 FMAs per thread in each microbenchmark launch")
    p.add_argument("--cpu-targets", type=int, default=100000,
                   help="targets in the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="precision",
                   choices=["precision", "precision96", "adjoint64", "large"],
                   help="precision: 128^3 NFW, L=500 (the headline); adjoint64: 64^3 NFW, L=200 "
                        "(a small case of the same kernels for profiling); precision96: 96^3 at "
                        "the same density and halo fraction as precision; large: 512^3, "
                        "L=1000, N_PM=512, 70%% of the mass in 200000 halos, leaves <= 64 "
                        "(FP32 paths only)")
    return p.parse_args()


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (the job's time is the slowest
    rank's)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[4:8]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


PRECISION_VARIANTS = [
    ("table linear 1024", dict(table_n=1024, interp=0)),
    ("table linear 4096", dict(table_n=4096, interp=0)),
    ("table cubic 1024", dict(table_n=1024, interp=1)),
    ("table cubic 4096", dict(table_n=4096, interp=1)),
    ("exact erfcf/expf", dict(precision=1)),
    # the paper's Taylor table (Section 3.3, Eq. int), its node spacing 3/512
    ("paper Taylor T[2] 384 nodes", dict(table_n=384, interp=2)),
    ("paper Taylor T[4] 384 nodes", dict(table_n=384, interp=3)),
]


def run_batch(args, psr, torch, dev, stream, flush, check):
    """64 boxes, N log-uniform in [8^3, 64^3], L in [50, 400], half uniform and
    half NFW-clustered, in one handle and one launch per step; with check, the
    forces against the FP64 oracle on 200 sampled targets per box."""
    import synth
    boxes = synth.batch()
    t0 = time.perf_counter()
    lv = psr.Leaves.build_batch([(x.pos, x.mass, x.L, x.r_s, x.r_c, x.G) for x in boxes],
                                max_leaf=32, fp64=False)
    build_s = time.perf_counter() - t0
    lv.upload(dev)
    best, _ = lv.autotune(psr.Options(), reps=2)
    out = torch.empty((lv.n, 3), dtype=torch.float32, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        lv.forces(best, out=out)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lv.forces(best, out=out)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    evs = []
    for k in range(args.batch_steps):
        flush.fill_(k & 255)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        graph.replay()
        s1.record(stream)
        evs.append((s0, s1))
    torch.cuda.synchronize()
    lv.check()
    ms = sum(a.elapsed_time(e) for a, e in evs) / args.batch_steps
    ev = lv.evaluated_pairs
    acc = out.double().cpu().numpy()
    cnt = torch.empty_like(out)
    lv.forces(psr.Options(precision=best.precision, table_n=best.table_n, interp=best.interp,
                          accum=best.accum, kernel=best.kernel, warps_per_block=best.warps_per_block,
                          source_tile=best.source_tile, count_pairs=True), out=cnt)
    within = lv.pair_count()
    err = None
    if check:
        import numpy as np
        import oracle
        rng = np.random.default_rng(31)
        num = den = 0.0
        worst, off = 0.0, 0
        for x in boxes:
            tg = np.sort(rng.choice(x.n, min(200, x.n), replace=False))
            ref, _, _ = oracle.forces(x.pos, x.mass, x.L, x.r_s, x.r_c, x.G, targets=tg, cells=True)
            d = acc[off + tg] - ref
            num += float(np.sum(d * d))
            den += float(np.sum(ref * ref))
            worst = max(worst, float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))))
            off += x.n
        err = {"rel_rms_vs_fp64_oracle": float(np.sqrt(num / den)),
               "worst_box_rel_rms": worst,
               "sampled": "200 random targets per box (all of a smaller box), every box"}
    return {"value": within / (ms / 1e3) / 1e9, "unit": "G pair-interactions/s", "ms_per_step": ms,
            "boxes": len(boxes), "n": int(lv.n), "within_cutoff_per_step": int(within),
            "leaf_tile_pairs_per_step": int(ev), "force_error": err,
            "host_build_s": build_s, "launch": "one persistent launch per step, CUDA graph replay",
            "tile_shape": {"kernel": "packed pairs" if best.kernel == 2 else "scalar streams",
                           "warps_per_block": best.warps_per_block,
                           "source_tile": best.source_tile},
            "path": "FP32, linear 1024 table, FP64 fold"}


def rel_errors(a, ref):
    """Relative RMS, and the max and 99th percentile of the per-particle
    relative error |da_i| / max(|a_i|, 1e-3 rms|a|)."""
    import numpy as np
    d = a - ref
    nr = np.linalg.norm(ref, axis=1)
    rel = np.linalg.norm(d, axis=1) / np.maximum(nr, 1e-3 * np.sqrt(np.mean(nr * nr)))
    return {"rel_rms": float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))),
            "max_rel": float(rel.max()), "p99_rel": float(np.percentile(rel, 99))}


def run_large(args, torch, psr, dev, stream, flush, check, peak_tflops):
    """The large workload: 512^3 particles, 70 % of the mass in 200000 NFW
    halos, L = 1000, N_PM = 512, leaves <= 64.  The leaf set is built on the
    GPU from device positions; FP32-table forward (the headline options) and
    FP32 adjoint, each timed over args.large_steps steps (CUDA events, L2
    flushed between steps); with check, forces against the FP64 oracle on
    args.large_targets random targets and the adjoint on a tenth of them."""
    import numpy as np
    import synth
    t0 = time.perf_counter()
    b = synth.large()
    gen_s = time.perf_counter() - t0
    pos_d = torch.from_numpy(b.pos).to(dev)
    mass_d = torch.from_numpy(b.mass).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lv = psr.Leaves.device_build(pos_d, mass_d, b.L, b.r_s, b.r_c, b.G, max_leaf=b.max_leaf,
                                 fp64=False)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    del pos_d, mass_d
    info = lv.info
    opts = psr.Options(precision=psr.PSR_FP32_TABLE, table_n=args.table_n,
                       interp=psr.PSR_LINEAR if args.interp == "linear" else psr.PSR_CUBIC,
                       accum=psr.PSR_ACC_FP64 if args.accum == "fp64" else psr.PSR_ACC_KAHAN32)

    def timed(fn, steps):
        fn()
        torch.cuda.synchronize()
        ms = 0.0
        for k in range(steps):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / steps

    acc = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
    ms = timed(lambda: lv.forces(opts, out=acc), args.large_steps)
    lv.check()
    acc_h = acc.double().cpu().numpy()
    lv.forces(psr.Options(precision=opts.precision, table_n=opts.table_n, interp=opts.interp,
                          accum=opts.accum, count_pairs=True), out=acc)
    within, kev = lv.pair_count(), lv.evaluated_count()
    achieved = FLOPS_PER_INTERACTION * within / (ms / 1e3) / 1e12
    cot_h = synth.cotangent(b.n, 12349)
    cot = torch.from_numpy(cot_h).to(device=dev, dtype=torch.float32)
    gp = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
    gm = torch.empty((b.n,), dtype=torch.float32, device=dev)
    ms_a = timed(lambda: lv.adjoint(cot, opts, gp, gm), args.large_steps)
    lv.check()
    line = {"workload": "NFW-clustered 512^3, L=1000, N_PM=512, 70%% mass in %d halos, "
                        "r_s=1.2L/N_PM, r_c=4.5r_s, leaves<=64" % b.meta.get("n_halos", 0),
            "n": b.n, "value": within / (ms / 1e3) / 1e9,
            "unit": "G pair-interactions/s (within the cutoff)", "ms_per_step": ms,
            "steps": args.large_steps,
            "within_cutoff_per_step": int(within), "kernel_evaluated_per_step": int(kev),
            "leaf_tile_pairs_per_step": int(info.evaluated_pairs),
            "leaves": int(info.n_leaves), "leaf_pairs": int(info.n_pairs),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "counted": "51 flops per pair within the cutoff"},
            "device_build_ms": build_ms, "generate_s": gen_s,
            "adjoint": {"value": within / (ms_a / 1e3) / 1e9, "ms_per_step": ms_a,
                        "path": "FP32 adjoint (dL/dx, dL/dm), same table and pairs"},
            "path": "leaf set built on the GPU; FP32 pair math, T from a %d-interval %s table, "
                    "%s accumulation" % (args.table_n, args.interp, args.accum)}
    if check:
        import oracle
        rng = np.random.default_rng(2025)
        tg = np.sort(rng.choice(b.n, min(args.large_targets, b.n), replace=False))
        t0 = time.perf_counter()
        ref, _, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, targets=tg, cells=True)
        line["force_error"] = dict(rel_errors(acc_h[tg], ref), targets=int(tg.size),
                                   oracle_s=time.perf_counter() - t0)
        ta = tg[::10]
        gref, mref = oracle.adjoint(b.pos, b.mass, cot_h, b.L, b.r_s, b.r_c, b.G, targets=ta,
                                    cells=True)
        dg = gp.double().cpu().numpy()[ta] - gref
        dm = gm.double().cpu().numpy()[ta] - mref
        line["adjoint"]["rel_rms_vs_fp64_oracle_sampled"] = {
            "targets": int(ta.size),
            "dL_dx": float(np.sqrt(np.sum(dg * dg) / np.sum(gref * gref))),
            "dL_dm": float(np.sqrt(np.sum(dm * dm) / np.sum(mref * mref)))}
    del lv, acc, cot, gp, gm
    torch.cuda.empty_cache()
    return line


def m2l_flops_per_entry(p):
    """Algorithmic FP32 flops of one M2L entry: 2 per multiply-add of the
    contraction L_n += M_m D_(n+m) over |n + m| <= p, 2 per term of the
    derivative tensors D_k = sum_j c u^(k-2j) phi_(|k|-|j|), 1 per tensor
    rescale."""
    contraction = terms = nd = 0
    for K in range(p + 1):
        for a in range(K + 1):
            for b in range(K - a + 1):
                c = K - a - b
                contraction += (a + 1) * (b + 1) * (c + 1)
                terms += (a // 2 + 1) * (b // 2 + 1) * (c // 2 + 1)
                nd += 1
    return 2 * contraction + 2 * terms + nd


def run_fmm(args, torch, dev, b, lv, stream, flush, check):
    """Truncated multipole operators (P2M, M2L with the f_(n) prefactors, L2P)
    on the workload's leaves: P2M on every leaf about its cell centre; M2L on
    the leaf pairs of the near-field list that pass the split's opening test
    with theta = 0.5 (theta min(d, 2 r_s^2 / d) >= rho_I + rho_J, rho the
    cell's half diagonal), for the first 5000 target leaves; L2P on those
    targets."""
    import numpy as np
    from paper_2107_14008_gb300 import capi
    p = args.fmm_order
    A = lv.host_arrays()
    leaf, lcen, rowptr, pairs = A["leaf"], A["lcen"], A["rowptr"], A["pairs"]
    nl = len(leaf)
    centres = lcen[:, :3].astype(np.float64) * (b.L / 2.0 ** 22)
    side = b.L / 2.0 ** lcen[:, 3].astype(np.float64)
    first = np.concatenate([leaf[:, 0], [b.n]]).astype(np.int64)
    perm = lv.perm
    spos = np.mod(b.pos, b.L)[perm]  # wrapped, leaf (Morton) order
    smass = np.asarray(b.mass)[perm]
    nt = min(nl, 5000)
    e1 = int(rowptr[nt])
    tgt = np.repeat(np.arange(nt), np.diff(rowptr[:nt + 1]))
    src = (pairs[:e1] >> 5).astype(np.int64)
    code = (pairs[:e1] & 31).astype(np.int64)
    sh = np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], axis=1) * b.L
    dist = np.linalg.norm(centres[tgt] - centres[src] - sh, axis=1)
    rho = 0.5 * np.sqrt(3.0) * side
    far = 0.5 * np.minimum(dist, 2 * b.r_s ** 2 / np.maximum(dist, 1e-300)) >= rho[tgt] + rho[src]
    frow = np.concatenate([[0], np.cumsum(np.bincount(tgt[far], minlength=nt))]).astype(np.int64)
    fpairs = pairs[:e1][far]
    h = float(np.median(side))
    box = capi.psr_box(b.L, b.r_s, b.r_c, b.G)
    nc = capi.psr_fmm_ncoef(p)
    d = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    pos_d, mass_d = d(spos, torch.float64), d(smass, torch.float64)
    first_d, cen_d = d(first, torch.int64), d(centres, torch.float64)
    rp_d, pr_d = d(frow, torch.int64), d(fpairs.view(np.int32), torch.int32)
    M = torch.empty((nl, nc), dtype=torch.float32, device=dev)
    Lc = torch.empty((nt, nc), dtype=torch.float32, device=dev)
    acc = torch.zeros((b.n, 3), dtype=torch.float32, device=dev)
    st = stream.cuda_stream

    def step():
        capi.psr_fmm_p2m(p, h, b.n, nl, first_d.data_ptr(), pos_d.data_ptr(), mass_d.data_ptr(),
                         cen_d.data_ptr(), M.data_ptr(), st)
        ev[1].record(stream)
        capi.psr_fmm_m2l(p, h, box, nt, nl, rp_d.data_ptr(), pr_d.data_ptr(), cen_d.data_ptr(),
                         cen_d.data_ptr(), M.data_ptr(), Lc.data_ptr(), 0, st)
        ev[2].record(stream)
        capi.psr_fmm_l2p(p, h, box, nt, first_d.data_ptr(), pos_d.data_ptr(), cen_d.data_ptr(),
                         Lc.data_ptr(), acc.data_ptr(), 0, st)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    step()
    torch.cuda.synchronize()
    t = np.zeros(3)
    for k in range(args.fmm_steps):
        flush.fill_(k & 255)
        ev[0].record(stream)
        step()
        ev[3].record(stream)
        torch.cuda.synchronize()
        t += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
    t /= args.fmm_steps
    nfar = int(far.sum())
    out = {"order": p, "scale_h": h, "leaves": nl, "target_leaves": nt, "m2l_entries": nfar,
           "near_entries_of_those_rows": e1 - nfar, "p2m_ms": t[0], "m2l_ms": t[1],
           "l2p_ms": t[2], "m2l_entries_per_s": nfar / (t[1] / 1e3),
           "m2l_flops_per_entry": m2l_flops_per_entry(p),
           "m2l_tflops": m2l_flops_per_entry(p) * nfar / (t[1] / 1e3) / 1e12,
           "mac": "0.5 min(d, 2 r_s^2 / d) >= rho_I + rho_J (cell half diagonals)"}
    if check:
        from oracle import fmm as ofmm
        got = acc.double().cpu().numpy()
        rows = [r for r in np.random.default_rng(3).permutation(nt)[:200]
                if frow[r + 1] > frow[r]][:3]
        num = den = 0.0
        for r in rows:
            tp = spos[first[r]:first[r + 1]]
            sp, sm = [], []
            for e in range(frow[r], frow[r + 1]):
                s_, c_ = int(fpairs[e]) >> 5, int(fpairs[e]) & 31
                shv = np.array([c_ // 9 - 1, (c_ // 3) % 3 - 1, c_ % 3 - 1]) * b.L
                sp.append(spos[first[s_]:first[s_ + 1]] + shv)
                sm.append(smass[first[s_]:first[s_ + 1]])
            ref = ofmm.direct(np.concatenate(sp), np.concatenate(sm), tp, b.r_s, b.G)
            num += np.sum((got[first[r]:first[r + 1]] - ref) ** 2)
            den += np.sum(ref ** 2)
        out["rel_rms_vs_direct_sampled"] = float(np.sqrt(num / den)) if den > 0 else None
        out["sampled_target_leaves"] = len(rows)
    return out


def run_split(args, torch, psr, dev, b, opts, stream, flush, full_ms, full_evaluated):
    """The short range with the multipole split (psr_device_build_split):
    P2P (FP32 table, the headline options) over the near entries plus
    psr_fmm_forces (P2M, M2L, L2P) over the well-separated ones, against the
    plain P2P step over the full list, for the opening-angle test alone and
    with the Gaussian-length term (PSR_BUILD_SPLIT_GAUSSIAN).  Returns the
    bench fields and the total accelerations per (rule, order), for the
    oracle comparison."""
    pos_d = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    mass_d = torch.tensor(b.mass, dtype=torch.float64, device=dev)
    thetas = [float(x) for x in str(args.split_theta).split(",") if x]
    orders = [int(x) for x in args.split_orders.split(",") if x]
    out = {"full_p2p_ms": full_ms, "evaluated_full": int(full_evaluated), "rules": []}
    totals = {}
    runs = [(t, "theta |R| >= rho_I + rho_J, both boxes wholly within r_c", False) for t in thetas]
    runs.append((thetas[0], "theta min(|R|, 2 r_s^2/|R|) >= rho_I + rho_J, both boxes wholly "
                            "within r_c", True))
    for theta, rule, gauss in runs:
        mk = lambda: psr.Leaves.device_build(pos_d, mass_d, b.L, b.r_s, b.r_c, b.G,
                                             max_leaf=b.max_leaf, theta=theta, gaussian_mac=gauss)
        lv = mk()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            lvb = mk()
            torch.cuda.synchronize()
            del lvb
        build_ms = (time.perf_counter() - t0) / 3 * 1e3
        inf = lv.info
        acc = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        nl = int(inf.n_leaves)
        scratch = torch.empty(2 * nl * ((capi_ncoef(max(orders)) + 3) // 4 * 4),
                              dtype=torch.float32, device=dev)
        r = {"theta": theta, "acceptance": rule, "leaves": nl, "near_entries": int(inf.n_pairs),
             "far_entries": int(inf.n_far), "evaluated_near": int(inf.evaluated_pairs),
             "p2p_interactions_moved_to_m2l": 1.0 - inf.evaluated_pairs / full_evaluated,
             "device_build_split_ms": build_ms, "orders": []}
        for p in orders:
            def step():
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                lv.forces(opts, out=acc)
                e[1].record(stream)
                lv.fmm_forces(p, out=acc, accumulate=True, scratch=scratch, status=status)
                e[2].record(stream)
                return e
            for _ in range(2):
                step()
            torch.cuda.synchronize()
            tn = tf = 0.0
            for k in range(args.split_steps):
                flush.fill_(k & 255)
                e = step()
                torch.cuda.synchronize()
                tn += e[0].elapsed_time(e[1])
                tf += e[1].elapsed_time(e[2])
            tn /= args.split_steps
            tf /= args.split_steps
            lv.check()
            totals[(theta, gauss, p)] = acc.double().cpu().numpy()
            r["orders"].append({"order": p, "p2p_near_ms": tn, "fmm_far_ms": tf,
                                "short_range_ms": tn + tf,
                                "speedup_vs_full_p2p": full_ms / (tn + tf),
                                "m2l_entries_per_s_upper_bound_time": inf.n_far / (tf / 1e3),
                                "status": int(status.item()), "_key": [theta, gauss, p]})
        out["rules"].append(r)
        del lv
    return out, totals


def run_paper_design(args, torch, psr, dev, b, lv, opts, stream, flush, full_ms, within):
    """The paper's own design on the same workload (prior art): its
    block-per-target-leaf kernel (Algorithms 1 and 2) with the headline table
    and with its Taylor T[2] table, on the octree leaves and on the paper's
    ORB leaves (host-built, the same leaf limit), beside the warp-per-leaf
    kernel on ORB leaves.  Every variant computes the same forces; ms per
    step is the comparison (evaluated pairs differ between trees)."""
    t0 = time.perf_counter()
    orb = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=b.max_leaf, fp64=False,
                           orb=True)
    orb_build_s = time.perf_counter() - t0
    orb.upload(dev)
    taylor = dict(precision=psr.PSR_FP32_TABLE, table_n=384, interp=psr.PSR_TAYLOR2)
    head = dict(precision=opts.precision, table_n=opts.table_n, interp=opts.interp,
                accum=opts.accum)
    runs = [("octree", lv, "paper block-per-leaf", dict(head, kernel=psr.PSR_KERNEL_PAPER)),
            ("octree", lv, "paper block-per-leaf, Taylor T[2] 384",
             dict(taylor, kernel=psr.PSR_KERNEL_PAPER)),
            ("orb", orb, "warp-per-leaf (headline kernel)", head),
            ("orb", orb, "paper block-per-leaf", dict(head, kernel=psr.PSR_KERNEL_PAPER)),
            ("orb", orb, "paper block-per-leaf, Taylor T[2] 384",
             dict(taylor, kernel=psr.PSR_KERNEL_PAPER))]
    out, accs = [], []
    for tree, L_, name, kw in runs:
        o = psr.Options(**kw)
        acc = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
        for _ in range(2):
            L_.forces(o, out=acc)
        torch.cuda.synchronize()
        ms = 0.0
        for k in range(args.paper_steps):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L_.forces(o, out=acc)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        ms /= args.paper_steps
        L_.check()
        ev = int(L_.info.evaluated_pairs)
        out.append({"tree": tree, "kernel": name, "ms_per_step": ms,
                    "value": within / (ms / 1e3) / 1e9,
                    "unit": "G pair-interactions/s (within the cutoff)",
                    "leaf_tile_pairs": ev, "slowdown_vs_headline": ms / full_ms})
        accs.append(acc.double().cpu().numpy())
    oi = orb.info
    line = {"orb_leaves": int(oi.n_leaves), "orb_leaf_pairs": int(oi.n_pairs),
            "orb_evaluated_pairs": int(oi.evaluated_pairs), "orb_host_build_s": orb_build_s,
            "headline_ms": full_ms, "variants": out}
    del orb
    return line, accs


def capi_ncoef(p):
    from paper_2107_14008_gb300 import capi
    return capi.psr_fmm_ncoef(p)


def cpu_baseline(b, acc_gpu, n_targets, seed=2024, return_ref=False):
    """FP64 oracle on a bounded sample of targets (all sources), host cores."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    tg = np.sort(rng.choice(b.n, min(n_targets, b.n), replace=False))
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    ref, pairs, _ = oracle.forces(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, targets=tg, cells=True,
                                  threads=threads)
    dt = time.perf_counter() - t0
    err = None
    if acc_gpu is not None:
        d = acc_gpu[tg] - ref
        err = float(np.sqrt(np.sum(d * d) / np.sum(ref * ref)))
    res = {"value": float(pairs.sum()) / dt / 1e9, "unit": "G pair-interactions/s",
           "cores": threads, "kind": "oracle",
           "sample": "%d random targets of the workload against all %d sources (within-cutoff "
                     "pairs counted), cell-list FP64 brute force, %.1f s" % (tg.size, b.n, dt),
           "seconds": dt, "pairs": int(pairs.sum())}
    if return_ref:
        return res, err, tg, ref
    return res, err, tg.size


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    b = make_box(args)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(b, None, max(1000, args.cpu_targets // 20))
    for k in range(args.steps):
        cb, _, _ = cpu_baseline(b, None, max(1000, args.cpu_targets // 20), seed=100 + k)
        vals.append(cb)
    pairs = sum(v["pairs"] for v in vals)
    secs = sum(v["seconds"] for v in vals)
    value = pairs / secs / 1e9
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "G pair-interactions/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(workload_config(b, args),
                           path="FP64 CPU oracle (cell list), within-cutoff pairs counted"),
            "cpu_baseline": {"value": value, "unit": "G pair-interactions/s",
                             "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": "each step: %d random targets against all sources"
                                       % max(1000, args.cpu_targets // 20)},
            "e2e": {"value": value, "unit": "G pair-interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


FWD_SOURCES = ["fwd_f32_common.cuh", "p2p_fwd_f32.cu", "p2p_fwd_f32_sc.cu", "p2p_fwd_f32_pk.cu",
               "kcommon.cuh", "psr_internal.h"]


def measured_traffic():
    """DRAM bytes per launch of the forward kernel from the committed ncu
    summary, if the kernel sources are unchanged since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "p2p_fwd_f32_precision128_dram.md")
    try:
        txt = open(path).read()
        want = txt.split("source_sha256:")[1].split()[0]
        nbytes = int(txt.split("dram_bytes_per_launch:")[1].split()[0])
    except Exception:
        return None
    h = hashlib.sha256()
    for f in FWD_SOURCES:
        with open(os.path.join(ROOT, "paper_2107_14008_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return nbytes if h.hexdigest() == want else None


def make_box(args, rank=0):
    import synth
    if args.workload == "adjoint64":
        return synth.adjoint(seed=12348 + rank)
    if args.workload == "large":
        return synth.large(seed=12349 + rank)
    if args.workload == "precision96":
        return synth.precision(seed=12346 + rank, nside=96, L=375.0, n_halos=1688)
    return synth.precision(seed=12346 + rank)


def workload_config(b, args):
    frac = 70 if args.workload == "large" else 60
    return {"workload": "NFW-clustered %d^3, L=%g, N_PM=%d, %d%% mass in %d halos, "
                        "r_s=1.2L/N_PM, r_c=4.5r_s, leaves<=%d"
                        % (b.n_pm, b.L, b.n_pm, frac, b.meta.get("n_halos", 0), b.max_leaf),
            "n": b.n, "L": b.L, "r_s": b.r_s, "r_c": b.r_c, "max_leaf": b.max_leaf,
            "path": "FP32 pair math, T from a %d-interval %s table in shared memory, %s "
                    "accumulation" % (args.table_n, args.interp, args.accum),
            "l2": "flushed between timed steps (256 MB write)"}


def run_psr(args):
    import numpy as np
    import torch

    import paper_2107_14008_gb300 as psr

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    b = make_box(args, rank)
    t0 = time.perf_counter()
    lv = psr.Leaves.build(b.pos, b.mass, b.L, b.r_s, b.r_c, b.G, max_leaf=b.max_leaf,
                          fp64=args.fp64_steps > 0)
    build_s = time.perf_counter() - t0
    lv.upload(dev)
    info = lv.info
    opts = psr.Options(precision=psr.PSR_FP32_TABLE, table_n=args.table_n,
                       interp=psr.PSR_LINEAR if args.interp == "linear" else psr.PSR_CUBIC,
                       accum=psr.PSR_ACC_FP64 if args.accum == "fp64" else psr.PSR_ACC_KAHAN32,
                       kernel=psr.PSR_KERNEL_PACKED if args.kernel == "packed"
                       else psr.PSR_KERNEL_SCALAR)
    acc = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        lv.forces(opts, out=acc)
    lv.check()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(k & 255)
            evs[k][0].record(stream)
            lv.forces(opts, out=acc)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = [a.elapsed_time(e) for a, e in evs]
    total_ms = sum(ms)
    if pg:
        total_ms = max_over_ranks(total_ms, pg, dev)
    lv.check()
    acc32 = acc.double().cpu().numpy()
    # within-cutoff pairs (untimed counting run, after the timed region)
    lv.forces(psr.Options(precision=opts.precision, table_n=opts.table_n, interp=opts.interp,
                          accum=opts.accum, count_pairs=True), out=acc)
    within = lv.pair_count()            # pairs with 0 < r < r_c: the workload's interactions
    kernel_evaluated = lv.evaluated_count()  # pair terms the kernel computed (after its cull)
    evaluated = info.evaluated_pairs    # all pairs of the leaf-pair tiles
    value = world * within * args.steps / (total_ms / 1e3) / 1e9
    mean_ms = total_ms / args.steps

    # FP64 path beside it
    fp64 = None
    if args.fp64_steps > 0:
        o64 = psr.Options(precision=psr.PSR_FP64)
        a64 = torch.empty((b.n, 3), dtype=torch.float64, device=dev)
        lv.forces(o64, out=a64)
        torch.cuda.synchronize()
        e64 = []
        for k in range(args.fp64_steps):
            flush.fill_(k & 255)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            lv.forces(o64, out=a64)
            s1.record(stream)
            e64.append((s0, s1))
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(e) for a, e in e64) / args.fp64_steps
        ref64 = a64.cpu().numpy()
        d = acc32 - ref64
        fp64 = {"value": within / (ms64 / 1e3) / 1e9, "unit": "G pair-interactions/s",
                "ms_per_step": ms64,
                "fp32_table_rel_rms_vs_fp64_path": float(np.sqrt(np.sum(d * d) / np.sum(ref64 ** 2)))}
        # the paper's double-precision table path: FP64 pair arithmetic, T from
        # the Taylor T_[4] table in FP64 (384 nodes), 1/r by Newton-Raphson
        ot = psr.Options(precision=psr.PSR_FP64, interp=psr.PSR_TAYLOR4, table_n=384)
        at = torch.empty((b.n, 3), dtype=torch.float64, device=dev)
        lv.forces(ot, out=at)
        torch.cuda.synchronize()
        et = []
        for k in range(args.fp64_steps):
            flush.fill_(k & 255)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            lv.forces(ot, out=at)
            s1.record(stream)
            et.append((s0, s1))
        torch.cuda.synchronize()
        mst = sum(a.elapsed_time(e) for a, e in et) / args.fp64_steps
        dt_ = at.cpu().numpy() - ref64
        fp64["taylor4_table"] = {
            "value": within / (mst / 1e3) / 1e9, "ms_per_step": mst,
            "rel_rms_vs_plain_fp64_path": float(np.sqrt(np.sum(dt_ * dt_) / np.sum(ref64 ** 2))),
            "path": "FP64, T from the paper's Taylor T[4] table in FP64 (384 nodes), "
                    "1/r by Newton-Raphson from an FP32 estimate"}
        lv.check()

    # adjoint (FP32 table) on the same leaf set, same timing rules
    adj = None
    if args.adjoint_steps > 0:
        cot = torch.tensor(np.random.default_rng(5).standard_normal((b.n, 3)), dtype=torch.float32,
                           device=dev)
        gp = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
        gm = torch.empty((b.n,), dtype=torch.float32, device=dev)
        lv.adjoint(cot, opts, gp, gm)
        torch.cuda.synchronize()
        ea = []
        for k in range(args.adjoint_steps):
            flush.fill_(k & 255)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            lv.adjoint(cot, opts, gp, gm)
            s1.record(stream)
            ea.append((s0, s1))
        torch.cuda.synchronize()
        ms_a = sum(a.elapsed_time(e) for a, e in ea) / args.adjoint_steps
        adj = {"value": within / (ms_a / 1e3) / 1e9, "unit": "G pair-interactions/s",
               "ms_per_step": ms_a, "path": "FP32 adjoint (dL/dx, dL/dm), same table and pairs"}
        if args.fp64_steps > 0:
            g64, m64 = lv.adjoint(cot.double(), psr.Options(precision=psr.PSR_FP64))
            dg = gp.double() - g64
            dm = gm.double() - m64
            adj["rel_rms_vs_fp64_path"] = {
                "dL_dx": float(torch.sqrt((dg * dg).sum() / (g64 * g64).sum())),
                "dL_dm": float(torch.sqrt((dm * dm).sum() / (m64 * m64).sum()))}
        lv.check()
        if rank == 0 and not args.no_cpu_baseline:
            # the FP32 adjoint against the FP64 oracle on sampled targets
            import oracle
            tg = np.sort(np.random.default_rng(11).choice(b.n, min(1000, b.n), replace=False))
            gref, mref = oracle.adjoint(b.pos, b.mass, cot.double().cpu().numpy(), b.L, b.r_s,
                                        b.r_c, b.G, targets=tg, cells=True)
            dg = gp.double().cpu().numpy()[tg] - gref
            dm = gm.double().cpu().numpy()[tg] - mref
            adj["rel_rms_vs_fp64_oracle_sampled"] = {
                "targets": int(tg.size),
                "dL_dx": float(np.sqrt(np.sum(dg * dg) / np.sum(gref * gref))),
                "dL_dm": float(np.sqrt(np.sum(dm * dm) / np.sum(mref * mref)))}

        # the same forward + backward through the differentiable entry point
        # (psr.forces, a torch.autograd.Function): GPU leaf build from the
        # CUDA positions, forward kernel, adjoint kernel, every step
        if args.autograd_steps > 0:
            pos_t = torch.tensor(b.pos, dtype=torch.float64, device=dev, requires_grad=True)
            mass_t = torch.tensor(b.mass, dtype=torch.float64, device=dev, requires_grad=True)
            cot64 = cot.double()

            def ag_step():
                pos_t.grad = mass_t.grad = None
                a_ = psr.forces(pos_t, mass_t, b.L, b.r_s, b.r_c, b.G, opts, b.max_leaf)
                a_.backward(cot64)

            ag_step()  # warm-up (allocator)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for k in range(args.autograd_steps):
                ag_step()
            s1.record(stream)
            torch.cuda.synchronize()
            ms_ag = s0.elapsed_time(s1) / args.autograd_steps
            dg = pos_t.grad.float() - gp
            adj["autograd"] = {
                "ms_per_step": ms_ag, "steps": args.autograd_steps,
                "includes": "psr.forces on CUDA tensors: GPU leaf build, forward kernel; "
                            "backward(): adjoint kernel (L2 not flushed between steps)",
                "resident_forward_plus_adjoint_ms": mean_ms + ms_a,
                "grad_pos_rel_rms_vs_resident_adjoint":
                    float(torch.sqrt((dg * dg).sum() / (gp * gp).sum()))}
            del pos_t, mass_t

    # the precision study: every T variant and accumulation, one launch each
    variants = []
    if args.variants:
        for name, kw in PRECISION_VARIANTS:
            for accn, accv in (("fp64", psr.PSR_ACC_FP64), ("kahan", psr.PSR_ACC_KAHAN32)):
                o = psr.Options(accum=accv, **kw)
                out = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
                lv.forces(o, out=out)
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                lv.forces(o, out=out)
                s1.record(stream)
                torch.cuda.synchronize()
                variants.append({"variant": name, "accum": accn,
                                 "value": within / (s0.elapsed_time(s1) / 1e3) / 1e9,
                                 "acc": out.double().cpu().numpy()})
        lv.check()

    # batched workload: 64 boxes in one persistent launch, autotuned tile shape,
    # replayed from a CUDA graph
    batch = None
    if args.batch_steps > 0:
        batch = run_batch(args, psr, torch, dev, stream, flush,
                          rank == 0 and not args.no_cpu_baseline)

    # end to end through the public API, host buffers, copies inside the region:
    # positions and masses from pinned host memory, leaf/pair build on the GPU
    # (psr_device_build), forward kernel, accelerations back to pinned memory
    e2e = None
    if args.e2e_steps > 0:
        pos_h = torch.from_numpy(np.ascontiguousarray(b.pos)).pin_memory()
        mass_h = torch.from_numpy(np.ascontiguousarray(b.mass)).pin_memory()
        out_h = torch.empty((b.n, 3), dtype=torch.float32).pin_memory()
        pos_d = torch.empty(pos_h.shape, dtype=torch.float64, device=dev)
        mass_d = torch.empty(mass_h.shape, dtype=torch.float64, device=dev)

        def e2e_step():
            pos_d.copy_(pos_h, non_blocking=True)
            mass_d.copy_(mass_h, non_blocking=True)
            lv2 = psr.Leaves.device_build(pos_d, mass_d, b.L, b.r_s, b.r_c, b.G,
                                          max_leaf=b.max_leaf, fp64=False)
            out_h.copy_(lv2.forces(opts), non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()  # warm-up (allocator, table)
        same = bool(np.array_equal(out_h.numpy(), acc.cpu().numpy()))
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            e2e_step()
        dt_serial = (time.perf_counter() - t0) / args.e2e_steps

        # Pipelined steps: the next step's positions and masses are copied in
        # on a copy stream while this step's leaf set is built and its forward
        # kernel runs, and each step's accelerations are copied out on another
        # stream while the next step's leaf set is built.  Every step still
        # copies its own inputs in and its own result out.
        h2d = torch.cuda.Stream(device=dev)
        d2h = torch.cuda.Stream(device=dev)
        main = torch.cuda.current_stream(dev)
        pos_b = [pos_d, torch.empty_like(pos_d)]
        mass_b = [mass_d, torch.empty_like(mass_d)]
        out_b = [out_h, torch.empty_like(out_h).pin_memory()]

        def copy_in(j):
            ev = torch.cuda.Event()
            with torch.cuda.stream(h2d):
                pos_b[j].copy_(pos_h, non_blocking=True)
                mass_b[j].copy_(mass_h, non_blocking=True)
                ev.record(h2d)
            return ev

        def e2e_pipelined(steps):
            ev_in = copy_in(0)
            for k in range(steps):
                j = k & 1
                main.wait_event(ev_in)
                lv2 = psr.Leaves.device_build(pos_b[j], mass_b[j], b.L, b.r_s, b.r_c, b.G,
                                              max_leaf=b.max_leaf, fp64=False)
                # the build waited on the host for the main stream's earlier
                # work, so the last reader of the other input buffers (the
                # previous step's build) is done with them
                if k + 1 < steps:
                    ev_in = copy_in(1 - j)
                a2 = lv2.forces(opts)
                ev_out = torch.cuda.Event()
                ev_out.record(main)
                d2h.wait_event(ev_out)
                with torch.cuda.stream(d2h):
                    out_b[j].copy_(a2, non_blocking=True)
                a2.record_stream(d2h)
            torch.cuda.synchronize()
            return out_b[(steps - 1) & 1]

        e2e_pipelined(2)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last = e2e_pipelined(args.e2e_steps)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        same = same and bool(np.array_equal(last.numpy(), acc.cpu().numpy()))
        # the GPU build alone (it ends with a host wait), for the breakdown
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for k in range(args.e2e_steps):
            lv3 = psr.Leaves.device_build(pos_d, mass_d, b.L, b.r_s, b.r_c, b.G,
                                          max_leaf=b.max_leaf, fp64=False)
            torch.cuda.synchronize()
            del lv3
        build_gpu_ms = (time.perf_counter() - t1) / args.e2e_steps * 1e3
        e2e = {"value": world * within / dt / 1e9, "unit": "G pair-interactions/s",
               "h2d_bytes_per_step": b.n * 4 * 8, "d2h_bytes_per_step": b.n * 3 * 4,
               "ms_per_step": dt * 1e3, "device_build_ms": build_gpu_ms,
               "ms_per_step_unpipelined": dt_serial * 1e3,
               "bitwise_equal_to_device_timed_output": same,
               "includes": "pinned H2D of positions and masses, GPU leaf/pair build "
                           "(psr_device_build + finish), forward kernel, D2H of accelerations, "
                           "every step; copies overlapped with the neighbouring steps' "
                           "kernels on two copy streams (ms_per_step_unpipelined: each "
                           "step alone, synchronised)"}
        # the same path with the host builder instead, for context
        t2 = time.perf_counter()
        lvh = psr.Leaves.build(pos_h.numpy(), mass_h.numpy(), b.L, b.r_s, b.r_c, b.G,
                               max_leaf=b.max_leaf, fp64=False)
        lvh.upload(dev)
        out_h.copy_(lvh.forces(opts))
        torch.cuda.synchronize()
        e2e["host_build_path_ms_per_step"] = (time.perf_counter() - t2) * 1e3
        del lvh

    # long-range PM part on the same box: CIC deposit, FFTs, Green's function,
    # gradient, interpolation (one psr_pm_forces call per step)
    pm_line = None
    if args.pm_steps > 0:
        pmo = psr.PM(b.n_pm, dev)
        pos_d = torch.tensor(b.pos, dtype=torch.float64, device=dev)
        mass_d = torch.tensor(b.mass, dtype=torch.float64, device=dev)
        apm = pmo.forces(pos_d, mass_d, b.L, b.r_s, b.G)
        torch.cuda.synchronize()
        ep = []
        for k in range(args.pm_steps):
            flush.fill_(k & 255)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            pmo.forces(pos_d, mass_d, b.L, b.r_s, b.G, out=apm)
            s1.record(stream)
            ep.append((s0, s1))
        torch.cuda.synchronize()
        ms_pm = sum(a.elapsed_time(e) for a, e in ep) / args.pm_steps
        pm_line = {"ms_per_step": ms_pm, "n_pm": b.n_pm, "particles": b.n,
                   "particles_per_s": b.n / (ms_pm / 1e3),
                   "kernels_per_step": "deposit, R2C, Green, 3 x (gradient, C2R), interpolation",
                   "fraction_of_p2p_step": ms_pm / mean_ms}
        if rank == 0 and not args.no_cpu_baseline and b.n <= (1 << 22):
            from oracle import pm as opm
            ref = opm.pm_forces(b.pos, b.mass, b.L, b.r_s, b.n_pm, b.G)
            d = apm.double().cpu().numpy() - ref
            pm_line["rel_rms_vs_fp64_oracle_mesh"] = float(np.sqrt(np.sum(d * d) / np.sum(ref * ref)))
        del pmo

    fmm_line = None
    if args.fmm_steps > 0 and b.n <= (1 << 22):
        fmm_line = run_fmm(args, torch, dev, b, lv, stream, flush,
                           rank == 0 and not args.no_cpu_baseline)

    paper_line = paper_acc = None
    if args.paper_steps > 0 and b.n <= (1 << 22):
        paper_line, paper_acc = run_paper_design(args, torch, psr, dev, b, lv, opts, stream, flush,
                                                 mean_ms, within)

    split_line = split_acc = None
    if args.split_steps > 0 and b.n <= (1 << 22):
        split_line, split_acc = run_split(args, torch, psr, dev, b, opts, stream, flush, mean_ms,
                                          evaluated)

    pk, pk_src = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12

    # the FP32 FMA rate this GPU reaches (psr_fp32_peak: independent FMA
    # chains on every SM), beside the peak derived from the unit counts
    fma_line = None
    if args.peak_launches > 0:
        sink = torch.empty(1 << 20, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        with Clocks(local) as clk_fma:
            fma = psr.capi.psr_fp32_peak(sink.data_ptr(), sink.numel() * 4, args.peak_iters,
                                         args.peak_launches, stream.cuda_stream, 60000)
        del sink
        fma_line = {"tflops": fma / 1e12, "frac_of_derived_peak": fma / 1e12 / peak_tflops,
                    "launches": args.peak_launches,
                    "per_thread": "8 independent FMA chains x %d steps, (SMs x 4) x 256 threads, "
                                  "best launch" % (8 * args.peak_iters),
                    "clocks": clk_fma.summary()}

    large_line = None
    if args.large_steps > 0 and args.workload != "large":
        large_line = run_large(args, torch, psr, dev, stream, flush,
                               rank == 0 and not args.no_cpu_baseline, peak_tflops)

    cb = err = None
    if rank == 0 and not args.no_cpu_baseline:
        cb, err, tg, ref = cpu_baseline(b, acc32, args.cpu_targets, return_ref=True)
        if paper_line:
            for v, a_ in zip(paper_line["variants"], paper_acc):
                d = a_[tg] - ref
                v["rel_rms_vs_fp64_oracle"] = float(np.sqrt(np.sum(d * d) / np.sum(ref * ref)))
        if split_line:
            for r_ in split_line["rules"]:
                for o in r_["orders"]:
                    d = split_acc[tuple(o["_key"])][tg] - ref
                    o["rel_rms_vs_fp64_oracle"] = float(np.sqrt(np.sum(d * d) / np.sum(ref * ref)))
        for v in variants:
            e_ = rel_errors(v["acc"][tg], ref)
            v["rel_rms_vs_fp64_oracle"] = e_["rel_rms"]
            v["max_rel_err"] = e_["max_rel"]
            v["p99_rel_err"] = e_["p99_rel"]
    if split_line:
        for r_ in split_line["rules"]:
            for o in r_["orders"]:
                o.pop("_key", None)
    for v in variants:
        v.pop("acc", None)
    achieved = FLOPS_PER_INTERACTION * within / (mean_ms / 1e3) / 1e12
    achieved_ev = FLOPS_PER_INTERACTION * kernel_evaluated / (mean_ms / 1e3) / 1e12
    clocks = clk.summary()
    line = {
        "metric": METRIC,
        "value": value, "unit": "G pair-interactions/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": mean_ms,
        "ms_median": statistics.median(ms), "ms_min": min(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(b, args),
        "interactions": {"within_cutoff_per_step": within,
                         "kernel_evaluated_per_step": kernel_evaluated,
                         "leaf_tile_pairs_per_step": evaluated,
                         "within_cutoff_value": value,
                         "kernel_evaluated_value":
                             world * kernel_evaluated * args.steps / (total_ms / 1e3) / 1e9,
                         "leaf_tile_value": world * evaluated * args.steps / (total_ms / 1e3) / 1e9,
                         "counts": "value and every other G/s figure count pairs with 0 < r < r_c "
                                   "(the unit of the oracle's arm); the kernel evaluates "
                                   "kernel_evaluated_per_step pair terms after dropping sources "
                                   "farther than r_c from the target leaf's box, out of the "
                                   "leaf-pair tiles' leaf_tile_pairs_per_step",
                         "leaves": int(info.n_leaves), "leaf_pairs": int(info.n_pairs),
                         "host_build_s": build_s},
        "pct_fp32_peak_51flop": 100.0 * achieved / peak_tflops,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "counted": "51 flops per pair within the cutoff",
                     "frac_on_kernel_evaluated_pairs": achieved_ev / peak_tflops,
                     "frac_on_leaf_tile_pairs":
                         FLOPS_PER_INTERACTION * evaluated / (mean_ms / 1e3) / 1e12 / peak_tflops,
                     "traffic": measured_traffic() if args.workload == "precision" else None,
                     "flops_per_interaction": FLOPS_PER_INTERACTION,
                     "peak_from": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz)"
                                  % (props.multi_processor_count, sm_max, pk_src),
                     "frac_of_measured_fma_rate":
                         None if fma_line is None else achieved / fma_line["tflops"]},
        "fp32_fma_rate_measured": fma_line,
        "fp64_path": fp64,
        "adjoint": adj,
        "batch": batch,
        "large": large_line,
        "pm_long_range": pm_line,
        "fmm_operators": fmm_line,
        "split_short_range": split_line,
        "paper_design": paper_line,
        "precision_variants": variants,
        "force_error": {"rel_rms_vs_fp64_oracle": err,
                        "sampled_targets": None if cb is None else args.cpu_targets,
                        **({} if cb is None else rel_errors(acc32[tg], ref))},
        "e2e": e2e,
        "cpu_baseline": None if cb is None else {k: cb[k] for k in
                                                  ("value", "unit", "cores", "kind", "sample")},
        "gpu_launches": args.steps,
        "tile_shape": {"kernel": "packed f32x2 pairs" if args.kernel == "packed" else "scalar streams", "warps_per_block": 8, "source_tile": 256},
        "clocks": clocks,
        "device": props.name,
    }
    if rank == 0:
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_psr(args)


if __name__ == "__main__":
    main()
