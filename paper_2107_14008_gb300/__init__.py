"""psr: GB300-native truncated short-range P2P gravity (arXiv:2107.14008).

Python layer over libpsr's C ABI: argument marshalling, device memory from
PyTorch, and a torch.autograd.Function.  Every step of the computation runs
in libpsr (host leaf builder in C++, forward/adjoint/table kernels in CUDA
for sm_103a).  There is no CPU fallback: without the built library, or
without a CUDA device, the device calls raise.
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from . import capi
from .capi import (PSR_ACC_FP64, PSR_ACC_KAHAN32, PSR_CUBIC, PSR_FP32_EXACT, PSR_FP32_TABLE,
                   PSR_FP64, PSR_KERNEL_AUTO, PSR_KERNEL_PACKED, PSR_KERNEL_PAPER,
                   PSR_KERNEL_SCALAR, PSR_LINEAR, PSR_TAYLOR2, PSR_TAYLOR4, PsrError)

__all__ = ["Options", "Leaves", "PM", "P2PForce", "forces", "PsrError", "PSR_FP64", "PSR_FP32_EXACT",
           "PSR_FP32_TABLE", "PSR_LINEAR", "PSR_CUBIC", "PSR_TAYLOR2", "PSR_TAYLOR4",
           "PSR_ACC_FP64", "PSR_ACC_KAHAN32",
           "PSR_KERNEL_AUTO", "PSR_KERNEL_SCALAR", "PSR_KERNEL_PACKED", "PSR_KERNEL_PAPER"]


@dataclass
class Options:
    """Kernel options (psr_opts)."""
    precision: int = PSR_FP32_TABLE
    table_n: int = 1024
    interp: int = PSR_LINEAR
    accum: int = PSR_ACC_FP64
    warps_per_block: int = 0
    blocks_per_sm: int = 0
    fold_every: int = 0
    count_pairs: bool = False
    kernel: int = 0
    source_tile: int = 0
    shard_count: int = 0
    shard_index: int = 0

    def c(self):
        o = capi.psr_opts()
        o.precision, o.table_n, o.interp, o.accum = (int(self.precision), int(self.table_n),
                                                     int(self.interp), int(self.accum))
        o.warps_per_block, o.blocks_per_sm = int(self.warps_per_block), int(self.blocks_per_sm)
        o.fold_every, o.count_pairs = int(self.fold_every), int(bool(self.count_pairs))
        o.kernel = int(self.kernel)
        o.source_tile = int(self.source_tile)
        o.shard_count, o.shard_index = int(self.shard_count), int(self.shard_index)
        return o

    @classmethod
    def from_c(cls, o):
        return cls(precision=o.precision, table_n=o.table_n, interp=o.interp, accum=o.accum,
                   warps_per_block=o.warps_per_block, blocks_per_sm=o.blocks_per_sm,
                   fold_every=o.fold_every, count_pairs=bool(o.count_pairs), kernel=o.kernel,
                   source_tile=o.source_tile, shard_count=o.shard_count,
                   shard_index=o.shard_index)

    @property
    def fp64(self):
        return self.precision == PSR_FP64


def _box(L, r_s, r_c, G=1.0):
    return capi.psr_box(float(L), float(r_s), float(r_c), float(G))


def _host_f64(a, cols):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(-1, cols) if cols > 1 else a.reshape(-1)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Leaves:
    """A built leaf set (psr_leaves handle) and, once uploaded, its device
    workspace (a torch uint8 tensor owned by this object)."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = n
        self.workspace = None
        self._info = capi.psr_leaves_info(handle)

    @classmethod
    def build(cls, pos, mass, L, r_s, r_c, G=1.0, max_leaf=32, fp64=True, orb=False, pack=True):
        """Host build (psr_build_leaves): the Morton octree with packed leaves
        (pack=False: plain octree leaves, PSR_BUILD_UNPACKED), or with
        orb=True the paper's ORB tree (PSR_BUILD_ORB)."""
        p = _host_f64(pos, 3)
        m = None if mass is None else _host_f64(mass, 1)
        if m is not None and m.shape[0] != p.shape[0]:
            raise ValueError("mass and pos lengths differ")
        dp = ctypes.POINTER(ctypes.c_double)
        h = capi.psr_build_leaves(p.ctypes.data_as(dp),
                                  None if m is None else m.ctypes.data_as(dp), p.shape[0],
                                  _box(L, r_s, r_c, G), int(max_leaf),
                                  (0 if fp64 else capi.PSR_BUILD_NO_FP64) |
                                  (capi.PSR_BUILD_ORB if orb else 0) |
                                  (0 if pack else capi.PSR_BUILD_UNPACKED))
        return cls(h, p.shape[0])

    @classmethod
    def build_batch(cls, boxes, max_leaf=32, fp64=True):
        """boxes: sequence of (pos, mass, L, r_s, r_c, G)."""
        dp = ctypes.POINTER(ctypes.c_double)
        keep, pp, mm, ns, bx = [], [], [], [], []
        for (pos, mass, L, r_s, r_c, G) in boxes:
            p = _host_f64(pos, 3)
            m = _host_f64(mass, 1) if mass is not None else \
                np.full(p.shape[0], 1.0 / max(p.shape[0], 1))
            keep += [p, m]
            pp.append(p.ctypes.data_as(dp))
            mm.append(m.ctypes.data_as(dp))
            ns.append(p.shape[0])
            bx.append(_box(L, r_s, r_c, G))
        nb = len(boxes)
        h = capi.psr_build_leaves_batch(nb, (dp * nb)(*pp), (dp * nb)(*mm),
                                        (ctypes.c_int64 * nb)(*ns), (capi.psr_box * nb)(*bx),
                                        int(max_leaf), 0 if fp64 else capi.PSR_BUILD_NO_FP64)
        return cls(h, int(sum(ns)))

    @classmethod
    def device_build(cls, pos, mass, L, r_s, r_c, G=1.0, max_leaf=32, fp64=True, stream=None,
                     timeout_ms=60000, theta=None, gaussian_mac=False, pack=True):
        """Build on the GPU from device tensors (psr_device_build and
        psr_device_build_finish): pos (n,3) and mass (n,) or None, on one CUDA
        device.  The result is already resident (no upload()).  With theta in
        (0, 1] the pair list is split (psr_device_build_split): forces() then
        sums the near entries and fmm_forces() the well-separated ones;
        gaussian_mac adds PSR_BUILD_SPLIT_GAUSSIAN, pack=False
        PSR_BUILD_UNPACKED."""
        import torch
        if not (hasattr(pos, "is_cuda") and pos.is_cuda):
            raise ValueError("device_build takes CUDA tensors")
        dev = pos.device
        p = pos.detach().to(torch.float64).contiguous().reshape(-1, 3)
        n = p.shape[0]
        m = None
        if mass is not None:
            m = mass.detach().to(device=dev, dtype=torch.float64).contiguous().reshape(-1)
            if m.shape[0] != n:
                raise ValueError("mass and pos lengths differ")
        with torch.cuda.device(dev):
            st = _stream_handle(stream)
            nbytes = capi.psr_device_build_scratch_bytes(n)
            scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            flags = (0 if fp64 else capi.PSR_BUILD_NO_FP64) | \
                (capi.PSR_BUILD_SPLIT_GAUSSIAN if gaussian_mac else 0) | \
                (0 if pack else capi.PSR_BUILD_UNPACKED)
            if theta is None:
                h = capi.psr_device_build(p.data_ptr(), 0 if m is None else m.data_ptr(), n,
                                          _box(L, r_s, r_c, G), int(max_leaf), flags,
                                          scratch.data_ptr(), nbytes, st, int(timeout_ms))
            else:
                h = capi.psr_device_build_split(p.data_ptr(), 0 if m is None else m.data_ptr(),
                                                n, _box(L, r_s, r_c, G), int(max_leaf), flags,
                                                float(theta), scratch.data_ptr(), nbytes, st,
                                                int(timeout_ms))
            lv = cls(h, n)
            lv.workspace = torch.empty(int(lv._info.device_bytes), dtype=torch.uint8, device=dev)
            capi.psr_device_build_finish(h, lv.workspace.data_ptr(), lv.workspace.numel(), st)
            if stream is not None:  # the scratch is read by work queued on `stream`
                scratch.record_stream(stream)
            del scratch
        return lv

    # -- host-side information -------------------------------------------
    @property
    def info(self):
        return self._info

    @property
    def device_built(self):
        return self.n > 0 and not bool(self._info.perm)

    @property
    def perm(self):
        if self.n == 0:
            return np.zeros(0, dtype=np.int64)
        if self.device_built:
            r = capi.psr_leaves_regions(self._h)
            return self.workspace[r.perm:r.perm + 4 * self.n].view(
                __import__("torch").int32).cpu().numpy().astype(np.int64)
        return np.ctypeslib.as_array(self._info.perm, shape=(self.n,)).copy()

    def device_arrays(self):
        """Copies (numpy) of the workspace arrays, with the names and layouts
        of host_arrays() plus perm; needs the workspace to be written."""
        import torch
        if self.workspace is None:
            raise PsrError(capi.PSR_E_STATE, "the workspace has not been written")
        torch.cuda.synchronize(self.workspace.device)
        r = capi.psr_leaves_regions(self._h)
        inf = self._info
        n, nl, npairs = self.n, int(inf.n_leaves), int(inf.n_pairs)
        ws = self.workspace

        def v(off, count, dt, shape):
            nb = count * torch.empty(0, dtype=dt).element_size()
            return ws[off:off + nb].view(dt).cpu().numpy().reshape(shape)
        out = {"pf": v(r.pf, 4 * n, torch.float32, (n, 4)),
               "perm": v(r.perm, n, torch.int32, (n,)),
               "leaf": v(r.leaf, 4 * nl, torch.int32, (nl, 4)),
               "lcen": v(r.lcen, 4 * nl, torch.int32, (nl, 4)),
               "rowptr": v(r.rowptr, nl + 1, torch.int64, (nl + 1,)),
               "pairs": v(r.pairs, npairs, torch.int32, (npairs,)).view(np.uint32),
               "items": v(r.items, nl, torch.int32, (nl,))}
        has_pd = n > 0 and r.perm - r.pd >= 32 * n  # the FP64 region is empty without it
        out["pd"] = v(r.pd, 4 * n, torch.float64, (n, 4)) if has_pd else None
        return out

    def far_arrays(self):
        """Copies (numpy) of the multipole split's workspace arrays: frow
        (n_leaves+1), fpairs (n_far uint32) and fcen (n_leaves x 4: expansion
        centre, radius)."""
        import torch
        if self.workspace is None or self._info.theta <= 0:
            raise PsrError(capi.PSR_E_STATE, "not a written split handle")
        torch.cuda.synchronize(self.workspace.device)
        r = capi.psr_leaves_regions(self._h)
        nl, nf = int(self._info.n_leaves), int(self._info.n_far)
        ws = self.workspace

        def v(off, count, dt, shape):
            nb = count * torch.empty(0, dtype=dt).element_size()
            return ws[off:off + nb].view(dt).cpu().numpy().reshape(shape)
        return {"frow": v(r.frow, nl + 1, torch.int64, (nl + 1,)),
                "fpairs": v(r.fpairs, nf, torch.int32, (nf,)).view(np.uint32),
                "fcen": v(r.fcen, 4 * nl, torch.float64, (nl, 4)),
                "fofs": v(r.fofs, 4 * nl, torch.float32, (nl, 4))}

    def host_arrays(self):
        """Copies of the host arrays psr_upload sends (see psr_leaves_host_arrays)."""
        a = capi.psr_leaves_host_arrays(self._h)
        inf = self._info
        nl, npairs = int(inf.n_leaves), int(inf.n_pairs)
        def v(p, shape):
            if shape[0] == 0 or not bool(p):
                return np.zeros(shape, dtype=np.dtype(p._type_))
            return np.ctypeslib.as_array(p, shape=shape).copy()
        out = {"pf": v(a.pf, (self.n, 4)), "leaf": v(a.leaf, (nl, 4)), "lcen": v(a.lcen, (nl, 4)),
               "rowptr": v(a.rowptr, (nl + 1,)),
               "pairs": v(a.pairs, (npairs,)) if npairs else np.zeros(0, np.uint32),
               "items": v(a.items, (nl,))}
        out["pd"] = v(a.pd, (self.n, 4)) if bool(a.pd) else None
        return out

    def shard_targets(self, shard_count, shard_index):
        """Sorted-order indices of the particles a launch with this shard
        computes (the host mirror of the kernels' item assignment)."""
        A = self.device_arrays() if self.device_built else self.host_arrays()
        items = A["items"][shard_index::max(1, shard_count)]
        leaf = A["leaf"]
        return np.concatenate([np.arange(leaf[i, 0], leaf[i, 0] + leaf[i, 1]) for i in items]) \
            if len(items) else np.zeros(0, dtype=np.int64)

    @property
    def evaluated_pairs(self):
        return int(self._info.evaluated_pairs)

    # -- device ---------------------------------------------------------------
    def upload(self, device=None, stream=None):
        import torch
        dev = torch.device("cuda") if device is None else torch.device(device)
        nbytes = int(self._info.device_bytes)
        if self.workspace is None or self.workspace.numel() < nbytes or self.workspace.device != dev:
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            capi.psr_upload(self._h, self.workspace.data_ptr(), self.workspace.numel(),
                            _stream_handle(stream))
        return self

    def _dev(self):
        if self.workspace is None:
            raise PsrError(capi.PSR_E_STATE, "upload() has not been called")
        return self.workspace.device

    def forces(self, opts=None, out=None, stream=None):
        """Accelerations (n,3) on the workspace's device, original order."""
        import torch
        opts = opts or Options()
        dt = torch.float64 if opts.fp64 else torch.float32
        dev = self._dev()
        if out is None:
            out = torch.empty((self.n, 3), dtype=dt, device=dev)
        if out.dtype != dt or out.shape != (self.n, 3) or not out.is_contiguous() or out.device != dev:
            raise ValueError("out must be a contiguous (n,3) %s tensor on %s" % (dt, dev))
        with torch.cuda.device(dev):
            capi.psr_p2p_forces(self._h, opts.c(), out.data_ptr(), _stream_handle(stream))
        return out

    def fmm_forces(self, p=4, out=None, accumulate=False, fp64=False, scratch=None, status=None,
                   stream=None):
        """Far part of the short range of a split handle (psr_fmm_forces):
        P2M, M2L over the well-separated entries, L2P; (n,3) in the original
        order, written, or added into `out` with accumulate=True (e.g. onto
        forces()).  scratch: optional float32 tensor of 2 n_leaves ncoef4
        elements (ncoef rounded up to a multiple of 4)."""
        import torch
        dt = torch.float64 if fp64 else torch.float32
        dev = self._dev()
        if out is None:
            if accumulate:
                raise ValueError("accumulate=True needs out")
            out = torch.empty((self.n, 3), dtype=dt, device=dev)
        if out.dtype != dt or out.shape != (self.n, 3) or not out.is_contiguous() or out.device != dev:
            raise ValueError("out must be a contiguous (n,3) %s tensor on %s" % (dt, dev))
        nc = (capi.psr_fmm_ncoef(p) + 3) // 4 * 4
        nl = int(self._info.n_leaves)
        if scratch is None:
            scratch = torch.empty(2 * max(nl, 1) * nc, dtype=torch.float32, device=dev)
        if scratch.dtype != torch.float32 or scratch.numel() < 2 * nl * nc or scratch.device != dev:
            raise ValueError("scratch must be float32 with 2 n_leaves ncoef elements on %s" % dev)
        flags = (capi.PSR_FMM_ACCUMULATE if accumulate else 0) | (capi.PSR_FMM_F64 if fp64 else 0)
        with torch.cuda.device(dev):
            capi.psr_fmm_forces(self._h, p, flags, scratch.data_ptr(),
                                scratch.data_ptr() + 4 * nl * nc, out.data_ptr(),
                                0 if status is None else status.data_ptr(),
                                _stream_handle(stream))
        return out

    def adjoint(self, cot, opts=None, grad_pos=None, grad_mass=None, stream=None):
        """(dL/dx (n,3), dL/dm (n,)) for L = sum_i cot_i . a_i."""
        import torch
        opts = opts or Options()
        dt = torch.float64 if opts.fp64 else torch.float32
        dev = self._dev()
        cot = cot.to(device=dev, dtype=dt).contiguous()
        if cot.shape != (self.n, 3):
            raise ValueError("cotangent must be (n,3)")
        if grad_pos is None:
            grad_pos = torch.empty((self.n, 3), dtype=dt, device=dev)
        if grad_mass is None:
            grad_mass = torch.empty((self.n,), dtype=dt, device=dev)
        with torch.cuda.device(dev):
            capi.psr_p2p_adjoint(self._h, opts.c(), cot.data_ptr(), grad_pos.data_ptr(),
                                 grad_mass.data_ptr(), _stream_handle(stream))
        return grad_pos, grad_mass

    def autotune(self, opts=None, reps=3, timeout_ms=120000, stream=None):
        """Tile shape of the FP32 forward kernel for this leaf set
        (psr_autotune): returns (best Options, best time in ms)."""
        import torch
        opts = opts or Options()
        dev = self._dev()
        out = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            best, ms = capi.psr_autotune(self._h, opts.c(), out.data_ptr(), _stream_handle(stream),
                                         int(reps), int(timeout_ms))
        return Options.from_c(best), ms

    def pair_count(self, stream=None, timeout_ms=60000):
        """Pairs within the cutoff counted by the last count_pairs forward."""
        return capi.psr_pair_count(self._h, _stream_handle(stream), timeout_ms)

    def evaluated_count(self, stream=None, timeout_ms=60000):
        """Pair terms the last count_pairs forward's kernel evaluated."""
        return capi.psr_evaluated_count(self._h, _stream_handle(stream), timeout_ms)

    def check(self, stream=None, timeout_ms=60000):
        return capi.psr_check(self._h, _stream_handle(stream), timeout_ms)

    def close(self):
        if getattr(self, "_h", None) is not None:
            capi.psr_free_leaves(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PM:
    """Long-range particle-mesh accelerations on an n_pm^3 mesh (psr_pm_*):
    the Gaussian-filtered complement of the short-range P2P force.  Holds the
    cuFFT plans and a scratch tensor on one CUDA device."""

    def __init__(self, n_pm, device=None):
        import torch
        self.n_pm = int(n_pm)
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self._h = capi.psr_pm_create(self.n_pm)
        self.scratch = torch.empty(capi.psr_pm_scratch_bytes(self._h), dtype=torch.uint8,
                                   device=self.device)

    def forces(self, pos, mass, L, r_s, G=1.0, out=None, accumulate=False, deconvolve=True,
               stream=None):
        """Accelerations (n, 3) FP32 in the input order; with accumulate=True
        they are added to `out` (e.g. the P2P result)."""
        import torch
        dev = self.device
        p = pos.detach().to(device=dev, dtype=torch.float64).contiguous().reshape(-1, 3)
        n = p.shape[0]
        m = None
        if mass is not None:
            m = mass.detach().to(device=dev, dtype=torch.float64).contiguous().reshape(-1)
            if m.shape[0] != n:
                raise ValueError("mass and pos lengths differ")
        if out is None:
            if accumulate:
                raise ValueError("accumulate=True needs out")
            out = torch.empty((n, 3), dtype=torch.float32, device=dev)
        if out.dtype != torch.float32 or out.shape != (n, 3) or not out.is_contiguous() \
                or out.device != dev:
            raise ValueError("out must be a contiguous (n,3) float32 tensor on %s" % dev)
        flags = (capi.PSR_PM_ACCUMULATE if accumulate else 0) | \
            (0 if deconvolve else capi.PSR_PM_NO_DECONVOLVE)
        with torch.cuda.device(dev):
            capi.psr_pm_forces(self._h, p.data_ptr(), 0 if m is None else m.data_ptr(), n,
                               _box(L, r_s, 1.0, G), flags, self.scratch.data_ptr(),
                               self.scratch.numel(), out.data_ptr(), _stream_handle(stream))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            capi.psr_pm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class P2PForce(torch.autograd.Function):
        """a = P2PForce.apply(pos, mass, L, r_s, r_c, G, opts, max_leaf).

        Forward builds the leaf set from `pos` and runs the forward kernel:
        on the GPU (psr_device_build) when `pos` is a CUDA tensor, else on the
        host (psr_build_leaves) and uploaded to the current CUDA device.
        Backward runs the adjoint kernel on the same pair set (the set is
        frozen at the forward positions, so the gradient is that of the
        piecewise function with the hard cutoff held fixed)."""

        @staticmethod
        def forward(ctx, pos, mass, L, r_s, r_c, G=1.0, opts=None, max_leaf=32):
            opts = opts or Options()
            if pos.is_cuda:
                lv = Leaves.device_build(pos, mass, L, r_s, r_c, G, max_leaf, fp64=opts.fp64)
            else:
                lv = Leaves.build(pos, mass, L, r_s, r_c, G, max_leaf, fp64=opts.fp64)
                lv.upload()
            acc = lv.forces(opts)
            if acc.device != pos.device:
                acc = acc.to(pos.device)
            ctx.leaves, ctx.opts = lv, opts
            ctx.pos_dtype, ctx.mass_dtype = pos.dtype, mass.dtype
            return acc.to(pos.dtype)

        @staticmethod
        def backward(ctx, grad_acc):
            dev = grad_acc.device
            gp, gm = ctx.leaves.adjoint(grad_acc.contiguous(), ctx.opts)
            return (gp.to(device=dev, dtype=ctx.pos_dtype), gm.to(device=dev, dtype=ctx.mass_dtype),
                    None, None, None, None, None, None)

    return P2PForce


class _Lazy:
    _f = None

    def __get__(self, obj, owner):
        if _Lazy._f is None:
            _Lazy._f = _autograd_function()
        return _Lazy._f


class _Namespace:
    P2PForce = _Lazy()


def __getattr__(name):
    if name == "P2PForce":
        return _Namespace.P2PForce
    raise AttributeError(name)


def forces(pos, mass, L, r_s, r_c, G=1.0, opts=None, max_leaf=32):
    """Differentiable accelerations of particles `pos` (torch, CUDA)."""
    return _Namespace.P2PForce.apply(pos, mass, L, r_s, r_c, G, opts, max_leaf)
