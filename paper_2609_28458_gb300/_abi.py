"""ctypes binding of libgs.so (include/gs.h). Argument marshalling only.

The library must have been built (``paper_2609_28458_gb300.build.build()``); there is no fallback:
loading raises if ``libgs.so`` is missing or does not export every entry point.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgs.so")

SYSTEMS = {"isochrone": 0, "mw": 1, "precession": 2, "quintessence": 3, "loghalo": 4}
METHODS = {"tsit5": 0, "dopri5": 1, "vern7": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32df": 2, "df64": 3}
KERNELS = {"auto": 0, "plain": 1, "persistent": 2}
ORDERS = {"auto": 0, "natural": 1, "estimate": 2, "hint": 3}
ORDER = {0: 5, 1: 5, 2: 7}

ST_MAX_STEPS, ST_H_UNDERFLOW, ST_NONFINITE, ST_EMPTY_INTERVAL, ST_SAVEAT_OUTSIDE, ST_TAPE_OVERFLOW = 1, 2, 4, 8, 16, 32
ST_NO_CONVERGENCE = 64
ST_FAILED = ST_MAX_STEPS | ST_H_UNDERFLOW | ST_NONFINITE | ST_TAPE_OVERFLOW
GS_OK, GS_ERR_INVALID, GS_ERR_CUDA, GS_ERR_WORKSPACE = 0, 1, 2, 3

EXPORTS = ("gs_default_options", "gs_dims", "gs_solve", "gs_vjp", "gs_jvp", "gs_vjp_noalloc", "gs_workspace_bytes",
           "gs_tape_chunk_bytes", "gs_alu_probe", "gs_selftest",
           "gs_solve_flat", "gs_flat_workspace_bytes", "gs_profile_default_options", "gs_profile_prep_bytes",
           "gs_profile_prepare", "gs_profile_workspace_bytes", "gs_profile_fit", "gs_rhs", "gs_last_error",
           "gs_version")
NOALLOC_SCRATCH_BYTES = 64 << 20
SELFTEST_CHECKS = 9  # GS_SELFTEST_CHECKS


class GsOptions(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("precision", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("safety", ctypes.c_double), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("h0", ctypes.c_double), ("per_traj_saveat", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("record_tape", ctypes.c_int32), ("reuse_tape", ctypes.c_int32), ("tape_capacity", ctypes.c_int32),
                ("sm_limit", ctypes.c_int32), ("graph_safe", ctypes.c_int32), ("order", ctypes.c_int32),
                ("cost_hint", ctypes.c_void_p), ("ckpt_stride", ctypes.c_int32),
                ("ckpt_verify", ctypes.c_int32), ("warp_lanes", ctypes.c_int32)]


class GsProfileOptions(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("precision", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("gtol", ctypes.c_double), ("max_newton", ctypes.c_int32),
                ("n_iter", ctypes.c_int32), ("mu", ctypes.c_double), ("trust_om", ctypes.c_double),
                ("trust_h0", ctypes.c_double), ("start_om", ctypes.c_double), ("start_h0", ctypes.c_double),
                ("orad", ctypes.c_double), ("omega_b", ctypes.c_double), ("omega_nu", ctypes.c_double),
                ("conv_dchi2", ctypes.c_double), ("conv_decrement", ctypes.c_double), ("graph_safe", ctypes.c_int32),
                ("sm_limit", ctypes.c_int32)]


class GsError(RuntimeError):
    pass


_lib = None
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)


def lib():
    """Load libgs.so once; raise if it is missing (no CPU or library fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise GsError("libgs.so is not built (run paper_2609_28458_gb300.build.build()); the ensemble "
                      "solver has no other implementation")
    L = ctypes.CDLL(LIB_PATH)
    for name in EXPORTS:
        if not hasattr(L, name):
            raise GsError("libgs.so does not export %s" % name)
    L.gs_default_options.argtypes = [ctypes.POINTER(GsOptions)]
    L.gs_default_options.restype = None
    L.gs_dims.argtypes = [ctypes.c_int32, _i32p, _i32p]
    L.gs_dims.restype = ctypes.c_int
    L.gs_solve.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                           ctypes.c_int32, _vp, ctypes.POINTER(GsOptions), _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
    L.gs_solve.restype = ctypes.c_int
    L.gs_vjp.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                         ctypes.c_int32, _vp, ctypes.POINTER(GsOptions), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                         ctypes.c_size_t, _vp]
    L.gs_vjp.restype = ctypes.c_int
    L.gs_jvp.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                         ctypes.c_int32, _vp, ctypes.POINTER(GsOptions), ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                         _vp, _vp, ctypes.c_size_t, _vp]
    L.gs_jvp.restype = ctypes.c_int
    L.gs_vjp_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int32, _vp, ctypes.POINTER(GsOptions), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gs_vjp_noalloc.restype = ctypes.c_int
    L.gs_solve_flat.argtypes = [ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                _vp, ctypes.POINTER(GsOptions), ctypes.c_int32, ctypes.c_double, _vp, _vp, _vp, _vp,
                                _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
    L.gs_solve_flat.restype = ctypes.c_int
    L.gs_flat_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32]
    L.gs_flat_workspace_bytes.restype = ctypes.c_size_t
    L.gs_profile_default_options.argtypes = [ctypes.POINTER(GsProfileOptions)]
    L.gs_profile_default_options.restype = None
    L.gs_profile_prep_bytes.argtypes = [ctypes.c_int32] * 4
    L.gs_profile_prep_bytes.restype = ctypes.c_size_t
    L.gs_profile_prepare.argtypes = [ctypes.c_int32, _vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp,
                                     ctypes.c_int32, _vp, _vp, _vp, ctypes.c_size_t, _vp]
    L.gs_profile_prepare.restype = ctypes.c_int
    L.gs_profile_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32]
    L.gs_profile_workspace_bytes.restype = ctypes.c_size_t
    L.gs_profile_fit.argtypes = [ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.POINTER(GsProfileOptions), _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                 _vp, ctypes.c_size_t, _vp]
    L.gs_profile_fit.restype = ctypes.c_int
    L.gs_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(GsOptions),
                                     ctypes.c_int32, ctypes.c_double]
    L.gs_workspace_bytes.restype = ctypes.c_size_t
    L.gs_tape_chunk_bytes.argtypes = [ctypes.c_int32, ctypes.POINTER(GsOptions)]
    L.gs_tape_chunk_bytes.restype = ctypes.c_size_t
    L.gs_alu_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _vp, ctypes.POINTER(ctypes.c_int64), _vp]
    L.gs_alu_probe.restype = ctypes.c_int
    L.gs_selftest.argtypes = [ctypes.c_int64, ctypes.c_uint64, _vp, _vp]
    L.gs_selftest.restype = ctypes.c_int
    L.gs_rhs.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gs_rhs.restype = ctypes.c_int
    L.gs_last_error.argtypes = []
    L.gs_last_error.restype = ctypes.c_char_p
    L.gs_version.argtypes = []
    L.gs_version.restype = ctypes.c_char_p
    _lib = L
    return L


def check(rc):
    if rc != GS_OK:
        raise GsError("libgs error %d: %s" % (rc, lib().gs_last_error().decode()))


def options(method="tsit5", precision="fp64", kernel="auto", **kw):
    o = GsOptions()
    lib().gs_default_options(ctypes.byref(o))
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %s" % k)
        if k == "order" and isinstance(v, str):
            v = ORDERS[v]
        if k == "cost_hint" and v is not None and not isinstance(v, (int, ctypes.c_void_p)):
            v = v.data_ptr()  # a contiguous int32 device tensor kept alive by the caller
        setattr(o, k, v)
    return o


def dims(system):
    d, p = ctypes.c_int32(), ctypes.c_int32()
    check(lib().gs_dims(SYSTEMS[system] if isinstance(system, str) else int(system), ctypes.byref(d), ctypes.byref(p)))
    return d.value, p.value


def profile_options(method="tsit5", precision="fp64", **kw):
    o = GsProfileOptions()
    lib().gs_profile_default_options(ctypes.byref(o))
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown profile option %s" % k)
        setattr(o, k, v)
    return o
