"""ctypes binding of libpsr's C ABI (include/psr.h), with the same names.

Argument marshalling only: every step of the computation runs inside
libpsr (host builder in C++, kernels in CUDA).  If the library has not been
built, loading it raises immediately; there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PSR_LIB") or os.path.join(HERE, "_build", "libpsr.so")

PSR_OK = 0
PSR_E_ARG, PSR_E_CUTOFF, PSR_E_WORKSPACE, PSR_E_CUDA = -1, -2, -3, -4
PSR_E_DEVICE, PSR_E_TIMEOUT, PSR_E_NOMEM, PSR_E_STATE = -5, -6, -7, -8
PSR_FP64, PSR_FP32_EXACT, PSR_FP32_TABLE = 0, 1, 2
PSR_LINEAR, PSR_CUBIC, PSR_TAYLOR2, PSR_TAYLOR4 = 0, 1, 2, 3
PSR_ACC_FP64, PSR_ACC_KAHAN32 = 0, 1
PSR_KERNEL_AUTO, PSR_KERNEL_SCALAR, PSR_KERNEL_PACKED, PSR_KERNEL_PAPER = 0, 1, 2, 3
PSR_BUILD_NO_FP64, PSR_BUILD_ORB, PSR_BUILD_UNPACKED, PSR_BUILD_SPLIT_GAUSSIAN = 1, 2, 4, 8
PSR_PM_ACCUMULATE, PSR_PM_NO_DECONVOLVE = 1, 2
PSR_FMM_ACCUMULATE, PSR_FMM_F64 = 1, 2

# every symbol include/psr.h declares
EXPORTS = ["psr_build_leaves", "psr_build_leaves_batch", "psr_leaves_info", "psr_upload",
           "psr_p2p_forces", "psr_p2p_forces_noalloc", "psr_p2p_adjoint", "psr_pair_count",
           "psr_evaluated_count",
           "psr_check", "psr_table", "psr_autotune", "psr_fp32_peak",
           "psr_leaves_host_arrays", "psr_leaves_regions", "psr_device_build_scratch_bytes",
           "psr_device_build", "psr_device_build_finish", "psr_device_build_split",
           "psr_pm_create", "psr_pm_scratch_bytes", "psr_pm_forces", "psr_pm_free",
           "psr_fmm_ncoef", "psr_fmm_p2m", "psr_fmm_m2l", "psr_fmm_l2p", "psr_fmm_forces",
           "psr_free_leaves", "psr_last_error", "psr_version"]


class psr_box(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("r_s", ctypes.c_double), ("r_c", ctypes.c_double),
                ("G", ctypes.c_double)]


class psr_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("table_n", ctypes.c_int), ("interp", ctypes.c_int),
                ("accum", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("fold_every", ctypes.c_int),
                ("count_pairs", ctypes.c_int), ("kernel", ctypes.c_int),
                ("source_tile", ctypes.c_int), ("shard_count", ctypes.c_int),
                ("shard_index", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class psr_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("n_items", ctypes.c_int64), ("nbox", ctypes.c_int64),
                ("evaluated_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("max_leaf", ctypes.c_int), ("max_row", ctypes.c_int),
                ("build_seconds", ctypes.c_double), ("perm", ctypes.POINTER(ctypes.c_int64)),
                ("n_far", ctypes.c_int64), ("theta", ctypes.c_double),
                ("rows_walked_twice", ctypes.c_int64), ("equal_mass", ctypes.c_int)]


class psr_host_arrays(ctypes.Structure):
    _fields_ = [("pf", ctypes.POINTER(ctypes.c_float)), ("pd", ctypes.POINTER(ctypes.c_double)),
                ("leaf", ctypes.POINTER(ctypes.c_int32)), ("lcen", ctypes.POINTER(ctypes.c_int32)),
                ("rowptr", ctypes.POINTER(ctypes.c_int64)),
                ("pairs", ctypes.POINTER(ctypes.c_uint32)),
                ("items", ctypes.POINTER(ctypes.c_int32))]


class psr_regions(ctypes.Structure):
    _fields_ = [(k, ctypes.c_size_t) for k in
                ("pf", "pd", "perm", "leaf", "lcen", "rowptr", "pairs", "items", "frow", "fpairs",
                 "fcen", "fofs", "total")]


class PsrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("psr error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """Load libpsr.so (built in-tree by paper_2107_14008_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpsr.so is not built (%s); run "
                           "`python -m paper_2107_14008_gb300.build`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    L.psr_build_leaves.argtypes = [dp, dp, i64, ctypes.POINTER(psr_box), ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(vp)]
    L.psr_build_leaves_batch.argtypes = [ctypes.c_int, ctypes.POINTER(dp), ctypes.POINTER(dp),
                                         ctypes.POINTER(i64), ctypes.POINTER(psr_box),
                                         ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.psr_leaves_info.argtypes = [vp, ctypes.POINTER(psr_info)]
    L.psr_upload.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.psr_p2p_forces.argtypes = [vp, ctypes.POINTER(psr_opts), vp, vp]
    L.psr_p2p_forces_noalloc.argtypes = [vp, ctypes.POINTER(psr_opts), vp, vp]
    L.psr_p2p_adjoint.argtypes = [vp, ctypes.POINTER(psr_opts), vp, vp, vp, vp]
    L.psr_pair_count.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(i64)]
    L.psr_evaluated_count.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(i64)]
    L.psr_fp32_peak.argtypes = [vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                dp]
    L.psr_autotune.argtypes = [vp, ctypes.POINTER(psr_opts), vp, vp, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(psr_opts), ctypes.POINTER(ctypes.c_float)]
    L.psr_check.argtypes = [vp, vp, ctypes.c_int]
    L.psr_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp]
    L.psr_leaves_host_arrays.argtypes = [vp, ctypes.POINTER(psr_host_arrays)]
    L.psr_leaves_regions.argtypes = [vp, ctypes.POINTER(psr_regions)]
    L.psr_device_build_scratch_bytes.argtypes = [i64, ctypes.POINTER(ctypes.c_size_t)]
    L.psr_device_build.argtypes = [vp, vp, i64, ctypes.POINTER(psr_box), ctypes.c_int,
                                   ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.c_int,
                                   ctypes.POINTER(vp)]
    L.psr_device_build_finish.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.psr_device_build_split.argtypes = [vp, vp, i64, ctypes.POINTER(psr_box), ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, vp, ctypes.c_size_t, vp,
                                         ctypes.c_int, ctypes.POINTER(vp)]
    L.psr_pm_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
    L.psr_pm_scratch_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.psr_pm_forces.argtypes = [vp, vp, vp, i64, ctypes.POINTER(psr_box), ctypes.c_int, vp,
                                ctypes.c_size_t, vp, vp]
    L.psr_pm_free.argtypes = [vp]
    L.psr_pm_free.restype = None
    L.psr_fmm_ncoef.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.psr_fmm_p2m.argtypes = [ctypes.c_int, ctypes.c_double, i64, i64, vp, vp, vp, vp, vp, vp]
    L.psr_fmm_m2l.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.POINTER(psr_box), i64, i64,
                              vp, vp, vp, vp, vp, vp, vp, vp]
    L.psr_fmm_l2p.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.POINTER(psr_box), i64, vp, vp,
                              vp, vp, vp, ctypes.c_int, vp]
    L.psr_fmm_forces.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
    L.psr_free_leaves.argtypes = [vp]
    L.psr_free_leaves.restype = None
    L.psr_last_error.restype = ctypes.c_char_p
    L.psr_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("psr_free_leaves", "psr_pm_free", "psr_last_error", "psr_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(rc):
    if rc != PSR_OK:
        raise PsrError(rc, lib().psr_last_error().decode(errors="replace"))
    return rc


# --- same-name wrappers (raise PsrError on a non-zero status) ---------------

def psr_build_leaves(pos_ptr, mass_ptr, n, box, max_leaf, flags):
    h = ctypes.c_void_p()
    check(lib().psr_build_leaves(pos_ptr, mass_ptr, n, ctypes.byref(box), max_leaf, flags,
                                 ctypes.byref(h)))
    return h


def psr_build_leaves_batch(nbox, pos_ptrs, mass_ptrs, ns, boxes, max_leaf, flags):
    h = ctypes.c_void_p()
    check(lib().psr_build_leaves_batch(nbox, pos_ptrs, mass_ptrs, ns, boxes, max_leaf, flags,
                                       ctypes.byref(h)))
    return h


def psr_leaves_info(h):
    info = psr_info()
    check(lib().psr_leaves_info(h, ctypes.byref(info)))
    return info


def psr_upload(h, d_ws, nbytes, stream):
    return check(lib().psr_upload(h, ctypes.c_void_p(d_ws), nbytes, ctypes.c_void_p(stream)))


def psr_p2p_forces(h, opts, d_acc, stream):
    return check(lib().psr_p2p_forces(h, ctypes.byref(opts), ctypes.c_void_p(d_acc),
                                      ctypes.c_void_p(stream)))


def psr_p2p_forces_noalloc(h, opts, d_acc, stream):
    """psr_p2p_forces without any allocation: its scratch is a fixed array in
    the library (see include/psr.h), for callers that cannot allocate."""
    return check(lib().psr_p2p_forces_noalloc(h, ctypes.byref(opts), ctypes.c_void_p(d_acc),
                                              ctypes.c_void_p(stream)))


def psr_p2p_adjoint(h, opts, d_cot, d_gpos, d_gmass, stream):
    return check(lib().psr_p2p_adjoint(h, ctypes.byref(opts), ctypes.c_void_p(d_cot),
                                       ctypes.c_void_p(d_gpos), ctypes.c_void_p(d_gmass),
                                       ctypes.c_void_p(stream)))


def psr_autotune(h, base, d_acc, stream, reps, timeout_ms):
    best = psr_opts()
    ms = ctypes.c_float()
    check(lib().psr_autotune(h, ctypes.byref(base), ctypes.c_void_p(d_acc), ctypes.c_void_p(stream),
                             reps, timeout_ms, ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


def psr_fp32_peak(d_sink, sink_bytes, iters, launches, stream, timeout_ms):
    v = ctypes.c_double()
    check(lib().psr_fp32_peak(ctypes.c_void_p(d_sink), sink_bytes, iters, launches,
                              ctypes.c_void_p(stream), timeout_ms, ctypes.byref(v)))
    return v.value


def psr_pair_count(h, stream, timeout_ms):
    v = ctypes.c_int64()
    check(lib().psr_pair_count(h, ctypes.c_void_p(stream), timeout_ms, ctypes.byref(v)))
    return v.value


def psr_evaluated_count(h, stream, timeout_ms):
    v = ctypes.c_int64()
    check(lib().psr_evaluated_count(h, ctypes.c_void_p(stream), timeout_ms, ctypes.byref(v)))
    return v.value


def psr_check(h, stream, timeout_ms):
    return check(lib().psr_check(h, ctypes.c_void_p(stream), timeout_ms))


def psr_table(table_n, interp, x_c, d_out, stream):
    return check(lib().psr_table(table_n, interp, x_c, ctypes.c_void_p(d_out),
                                 ctypes.c_void_p(stream)))


def psr_leaves_host_arrays(h):
    a = psr_host_arrays()
    check(lib().psr_leaves_host_arrays(h, ctypes.byref(a)))
    return a


def psr_leaves_regions(h):
    r = psr_regions()
    check(lib().psr_leaves_regions(h, ctypes.byref(r)))
    return r


def psr_device_build_scratch_bytes(n):
    v = ctypes.c_size_t()
    check(lib().psr_device_build_scratch_bytes(n, ctypes.byref(v)))
    return v.value


def psr_device_build(d_pos, d_mass, n, box, max_leaf, flags, d_scratch, scratch_bytes, stream,
                     timeout_ms):
    h = ctypes.c_void_p()
    check(lib().psr_device_build(ctypes.c_void_p(d_pos), ctypes.c_void_p(d_mass), n,
                                 ctypes.byref(box), max_leaf, flags, ctypes.c_void_p(d_scratch),
                                 scratch_bytes, ctypes.c_void_p(stream), timeout_ms,
                                 ctypes.byref(h)))
    return h


def psr_device_build_split(d_pos, d_mass, n, box, max_leaf, flags, theta, d_scratch,
                           scratch_bytes, stream, timeout_ms):
    h = ctypes.c_void_p()
    check(lib().psr_device_build_split(ctypes.c_void_p(d_pos), ctypes.c_void_p(d_mass), n,
                                       ctypes.byref(box), max_leaf, flags, float(theta),
                                       ctypes.c_void_p(d_scratch), scratch_bytes,
                                       ctypes.c_void_p(stream), timeout_ms, ctypes.byref(h)))
    return h


def psr_device_build_finish(h, d_ws, nbytes, stream):
    return check(lib().psr_device_build_finish(h, ctypes.c_void_p(d_ws), nbytes,
                                               ctypes.c_void_p(stream)))


def psr_pm_create(n_pm):
    h = ctypes.c_void_p()
    check(lib().psr_pm_create(int(n_pm), ctypes.byref(h)))
    return h


def psr_pm_scratch_bytes(pm):
    v = ctypes.c_size_t()
    check(lib().psr_pm_scratch_bytes(pm, ctypes.byref(v)))
    return v.value


def psr_pm_forces(pm, d_pos, d_mass, n, box, flags, d_scratch, scratch_bytes, d_acc, stream):
    return check(lib().psr_pm_forces(pm, ctypes.c_void_p(d_pos), ctypes.c_void_p(d_mass), n,
                                     ctypes.byref(box), flags, ctypes.c_void_p(d_scratch),
                                     scratch_bytes, ctypes.c_void_p(d_acc),
                                     ctypes.c_void_p(stream)))


def psr_pm_free(pm):
    lib().psr_pm_free(pm)


def psr_fmm_ncoef(p):
    v = ctypes.c_int()
    check(lib().psr_fmm_ncoef(int(p), ctypes.byref(v)))
    return v.value


def _vp(x):
    return ctypes.c_void_p(x or None)


def psr_fmm_p2m(p, h, n, ncell, d_first, d_pos, d_mass, d_centre, d_M, stream):
    return check(lib().psr_fmm_p2m(int(p), float(h), n, ncell, _vp(d_first), _vp(d_pos),
                                   _vp(d_mass), _vp(d_centre), _vp(d_M), _vp(stream)))


def psr_fmm_m2l(p, h, box, ntarget, nsource, d_rowptr, d_pairs, d_ct, d_cs, d_M, d_L, d_status,
                stream):
    return check(lib().psr_fmm_m2l(int(p), float(h), ctypes.byref(box), ntarget, nsource,
                                   _vp(d_rowptr), _vp(d_pairs), _vp(d_ct), _vp(d_cs), _vp(d_M),
                                   _vp(d_L), _vp(d_status), _vp(stream)))


def psr_fmm_l2p(p, h, box, ncell, d_first, d_pos, d_centre, d_L, d_acc, flags, stream):
    return check(lib().psr_fmm_l2p(int(p), float(h), ctypes.byref(box), ncell, _vp(d_first),
                                   _vp(d_pos), _vp(d_centre), _vp(d_L), _vp(d_acc), int(flags),
                                   _vp(stream)))


def psr_fmm_forces(h, p, flags, d_M, d_L, d_acc, d_status, stream):
    return check(lib().psr_fmm_forces(h, int(p), int(flags), _vp(d_M), _vp(d_L), _vp(d_acc),
                                      _vp(d_status), _vp(stream)))


def psr_free_leaves(h):
    lib().psr_free_leaves(h)


def psr_version():
    return lib().psr_version().decode()
