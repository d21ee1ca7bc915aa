"""ctypes binding of libmbf.so (argument marshalling only).

Every name mirrors the C ABI of include/mbf.h.  The binding holds no arithmetic of
the method: construction, packing and every apply run in the library (host FP64
builder, sm_103a kernels).  Loading fails loudly if the library has not been
built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libmbf.so")

MBF_OK, MBF_ERR_INVALID, MBF_ERR_OOM, MBF_ERR_CUDA, MBF_ERR_BUSY, MBF_ERR_TIMEOUT, MBF_ERR_IO, \
    MBF_ERR_NOT_FOUND = range(8)
MBF_TREE_UNIFORM, MBF_TREE_POLAR, MBF_TREE_SQUARE, MBF_TREE_POINTS = 0, 1, 2, 3
MBF_PREC_AUTO, MBF_PREC_FP32_SIMT, MBF_PREC_TF32, MBF_PREC_BF16X3 = 0, 1, 2, 3

_STATUS_NAMES = {0: "MBF_OK", 1: "MBF_ERR_INVALID", 2: "MBF_ERR_OOM", 3: "MBF_ERR_CUDA",
                 4: "MBF_ERR_BUSY", 5: "MBF_ERR_TIMEOUT", 6: "MBF_ERR_IO", 7: "MBF_ERR_NOT_FOUND"}


class MbfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32), ("L", C.c_int32), ("r", C.c_int32),
                ("tree", C.c_int32), ("reserved0", C.c_int32), ("n_w", C.c_int64),
                ("w_index", C.POINTER(C.c_int64)), ("w_lo", C.c_double), ("w_side", C.c_double),
                ("n_x_pts", C.c_int64), ("x_pts", C.POINTER(C.c_double)), ("n_w_pts", C.c_int64),
                ("w_pts", C.POINTER(C.c_double))]


class BuildOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("sample_factor", C.c_int32), ("max_rounds", C.c_int32),
                ("tol", C.c_double), ("threads", C.c_int32), ("reserved", C.c_int32),
                ("factor_file", C.c_char_p)]


class Factors(C.Structure):
    _fields_ = [("dim", C.c_int32), ("L", C.c_int32), ("n_out", C.c_int64), ("n_in", C.c_int64),
                ("n_w", C.c_int64), ("x_perm", C.POINTER(C.c_int64)), ("x_off", C.POINTER(C.c_int64)),
                ("w_perm", C.POINTER(C.c_int64)), ("w_off", C.POINTER(C.c_int64)),
                ("RU", C.POINTER(C.c_int32)), ("RV", C.POINTER(C.c_int32)),
                ("max_leaf_x", C.c_int32), ("max_leaf_w", C.c_int32),
                ("UL", C.POINTER(C.c_double)), ("VL", C.POINTER(C.c_double)),
                ("G", C.POINTER(C.POINTER(C.c_double))), ("H", C.POINTER(C.POINTER(C.c_double))),
                ("S", C.POINTER(C.c_double)), ("nnz", C.c_int64)]


class OpInfo(C.Structure):
    _fields_ = [("dim", C.c_int32), ("L", C.c_int32), ("c", C.c_int32), ("n_stages", C.c_int32),
                ("n_out", C.c_int64), ("n_in", C.c_int64), ("RU", C.c_int32 * 32),
                ("RV", C.c_int32 * 32), ("nnz_algorithmic", C.c_int64),
                ("bytes_algorithmic", C.c_int64), ("bytes_packed", C.c_int64),
                ("bytes_stage", C.c_int64 * 32), ("grid", C.c_int32), ("threads", C.c_int32),
                ("smem", C.c_int32), ("nnz_stage", C.c_int64 * 32), ("nnz_leaf_u", C.c_int64),
                ("tensor_ok", C.c_int32), ("tensor_stages", C.c_int32), ("bytes_tensor", C.c_int64),
                ("tensor_smem", C.c_int32), ("tensor_slots", C.c_int32),
                ("tensor_unavailable", C.c_char * 128), ("eps", C.c_double),
                ("eps_samples", C.c_int32), ("reserved_eps", C.c_int32)]


PROFILE_KINDS = 8


class TuneResult(C.Structure):
    _fields_ = [("n_simt", C.c_int32), ("simt_rhs", C.c_int32 * 8), ("simt_ms", C.c_double * 8),
                ("n_slots", C.c_int32), ("slots", C.c_int32 * 8), ("tc_ms", C.c_double * 8),
                ("tc_slots_chosen", C.c_int32), ("tc_min_rhs", C.c_int32), ("panel_buffers", C.c_int32 * 8),
                ("tc_buffers_chosen", C.c_int32), ("reserved_tune", C.c_int32)]


class ServerOpts(C.Structure):
    _fields_ = [("staging_budget_bytes", C.c_int64), ("max_inflight", C.c_int32),
                ("max_batch_rhs", C.c_int32), ("max_queue", C.c_int32), ("use_graphs", C.c_int32),
                ("max_batch_ops", C.c_int32), ("mix_work_pct", C.c_int32)]


class RequestStatus(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("batch_requests", C.c_int32),
                ("batch_rhs", C.c_int32), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("rejected_busy", C.c_int64), ("batches", C.c_int64), ("coalesced_requests", C.c_int64),
                ("graph_launches", C.c_int64), ("graph_instantiations", C.c_int64),
                ("max_batch_requests", C.c_int32), ("max_concurrent_batches", C.c_int32),
                ("mixed_batches", C.c_int64), ("max_batch_ops", C.c_int32), ("reserved_stats", C.c_int32)]


MBF_REQ_QUEUED, MBF_REQ_RUNNING, MBF_REQ_DONE, MBF_REQ_ERROR = 0, 1, 2, 3


class MsbfInfo(C.Structure):
    _fields_ = [("n_parts", C.c_int32), ("part_t", C.c_int32 * 16), ("part_L", C.c_int32 * 16),
                ("part_points", C.c_int64 * 16), ("part_nnz", C.c_int64 * 16), ("n_out", C.c_int64),
                ("n_in", C.c_int64), ("n_center_points", C.c_int64), ("nnz_algorithmic", C.c_int64),
                ("bytes_algorithmic", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("n_kinds", C.c_int32), ("name", (C.c_char * 32) * PROFILE_KINDS),
                ("launches", C.c_int64 * PROFILE_KINDS), ("ms", C.c_double * PROFILE_KINDS)]


ENTRY_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.c_int64,
                       C.c_int32, C.POINTER(C.c_double), C.c_void_p)
APPLY_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64, C.c_int32, C.c_void_p)

# name -> (restype, argtypes); every entry point declared in include/mbf.h
SIGNATURES = {
    "mbf_build_factors": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.POINTER(BuildOpts),
                                    C.POINTER(C.c_void_p)]),
    "mbf_build_from_applies": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.POINTER(BuildOpts),
                                         C.POINTER(C.c_void_p)]),
    "mbf_factors_view": (C.c_int, [C.c_void_p, C.POINTER(Factors)]),
    "mbf_factors_destroy": (C.c_int, [C.c_void_p]),
    "mbf_factors_save": (C.c_int, [C.POINTER(Factors), C.c_char_p]),
    "mbf_factors_load": (C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
    "mbf_op_create": (C.c_int, [C.POINTER(Factors), C.POINTER(C.c_void_p)]),
    "mbf_build_from_entries": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.c_void_p,
                                         C.POINTER(BuildOpts), C.POINTER(C.c_void_p)]),
    "mbf_op_destroy": (C.c_int, [C.c_void_p]),
    "mbf_op_info": (C.c_int, [C.c_void_p, C.POINTER(OpInfo)]),
    "mbf_op_estimate_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_uint64,
                                        C.c_void_p, C.POINTER(C.c_double)]),
    "mbf_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "mbf_apply_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                    C.c_void_p]),
    "mbf_apply_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                 C.c_void_p]),
    "mbf_apply_host_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                       C.c_void_p]),
    "mbf_op_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mbf_op_debug_stall": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "mbf_debug_fail_alloc": (C.c_int, [C.c_int64]),
    "mbf_apply_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mbf_op_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "mbf_op_tune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(TuneResult)]),
    "mbf_build_msbf": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.POINTER(BuildOpts), C.c_int32,
                                 C.POINTER(C.c_void_p)]),
    "mbf_msbf_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.c_int32, C.POINTER(C.c_void_p)]),
    "mbf_msbf_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "mbf_msbf_apply_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "mbf_msbf_info": (C.c_int, [C.c_void_p, C.POINTER(MsbfInfo)]),
    "mbf_msbf_part": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "mbf_msbf_destroy": (C.c_int, [C.c_void_p]),
    "mbf_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "mbf_debug_form_batch": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_double),
                                       C.c_int32, C.c_int32, C.POINTER(ServerOpts), C.POINTER(C.c_int32)]),
    "mbf_debug_split_sms": (C.c_int, [C.POINTER(C.c_double), C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "mbf_debug_layout_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64]),
    "mbf_factors_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mbf_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                             C.POINTER(C.c_int64)]),
    "mbf_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(RequestStatus)]),
    "mbf_server_drain": (C.c_int, [C.c_void_p, C.c_double]),
    "mbf_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "mbf_server_destroy": (C.c_int, [C.c_void_p]),
    "mbf_op_profile": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "mbf_last_error": (C.c_char_p, []),
    "mbf_version": (C.c_char_p, []),
    "mbf_kernel_dft": (None, [C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.c_int64,
                              C.c_int32, C.POINTER(C.c_double), C.c_void_p]),
    "mbf_kernel_fio_iso": (None, [C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.c_int64,
                                  C.c_int32, C.POINTER(C.c_double), C.c_void_p]),
    "mbf_kernel_fio_ellip": (None, [C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double),
                                    C.c_int64, C.c_int32, C.POINTER(C.c_double), C.c_void_p]),
}

_lib = None


def lib():
    """Load libmbf.so (once).  Raises if it is missing: there is no CPU fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise ImportError(f"{LIBPATH} not built; run __graft_entry__.build() first")
        L = C.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != MBF_OK:
        raise MbfError(code, lib().mbf_last_error().decode())


def builtin_kernel(name: str):
    """Address of a built-in entry function: 'dft', 'fio_iso' or 'fio_ellip'."""
    fn = getattr(lib(), {"dft": "mbf_kernel_dft", "fio_iso": "mbf_kernel_fio_iso",
                         "fio_ellip": "mbf_kernel_fio_ellip"}[name])
    return C.cast(fn, C.c_void_p).value


def _ptr(x, ctype):
    return x.ctypes.data_as(C.POINTER(ctype))


class HostFactors:
    """Padded FP64 factor set in host memory: built by the library
    (`build`) or supplied by the caller (`from_arrays`)."""

    def __init__(self):
        self._handle = None
        self._keep = []
        self.view = Factors()

    @classmethod
    def build(cls, dim, n, L, r, tree=MBF_TREE_UNIFORM, kernel="dft", seed=7, threads=0,
              w_index=None, w_lo=0.0, w_side=0.0, sample_factor=3, max_rounds=3, tol=1e-14,
              factor_file=None, x_pts=None, w_pts=None):
        """Host FP64 construction (mbf_build_factors); with factor_file, loaded from that
        file if it exists, else built and written there.  tree=MBF_TREE_POINTS takes explicit
        point sets x_pts [n_x][dim] in [0,1)^dim and w_pts [n_w][dim] in the square
        [w_lo, w_lo + w_side)^dim (§2.6)."""
        self = cls()
        prob = Problem(dim=dim, n=n, L=L, r=r, tree=tree)
        if x_pts is not None:
            xp = np.ascontiguousarray(x_pts, dtype=np.float64).reshape(-1, dim)
            wp = np.ascontiguousarray(w_pts, dtype=np.float64).reshape(-1, dim)
            self._keep.extend([xp, wp])
            prob.n_x_pts, prob.x_pts = xp.shape[0], _ptr(xp, C.c_double)
            prob.n_w_pts, prob.w_pts = wp.shape[0], _ptr(wp, C.c_double)
            prob.w_lo, prob.w_side = w_lo, w_side
        if w_index is not None:
            wi = np.ascontiguousarray(w_index, dtype=np.int64)
            self._keep.append(wi)
            prob.n_w, prob.w_index, prob.w_lo, prob.w_side = wi.size, _ptr(wi, C.c_int64), w_lo, w_side
        opts = BuildOpts(seed=seed, sample_factor=sample_factor, max_rounds=max_rounds, tol=tol,
                         threads=threads, factor_file=None if factor_file is None else os.fsencode(factor_file))
        fn = builtin_kernel(kernel) if isinstance(kernel, str) else kernel
        h = C.c_void_p()
        _check(lib().mbf_build_factors(C.byref(prob), fn, None, C.byref(opts), C.byref(h)))
        self._handle = h
        _check(lib().mbf_factors_view(h, C.byref(self.view)))
        return self

    @classmethod
    def build_from_applies(cls, dim, n, L, r, apply, n_out, n_in, tree=MBF_TREE_UNIFORM, seed=7, threads=0,
                           tol=1e-14, x_pts=None, w_pts=None, w_lo=0.0, w_side=0.0):
        """Case (i) construction (mbf_build_from_applies): `apply(v, adjoint)` takes a complex
        [nrhs, n_in] array (n_out for the adjoint) and returns K v (or K^* v), [nrhs, n_out]."""
        self = cls()
        prob = Problem(dim=dim, n=n, L=L, r=r, tree=tree)
        if x_pts is not None:
            xp = np.ascontiguousarray(x_pts, dtype=np.float64).reshape(-1, dim)
            wp = np.ascontiguousarray(w_pts, dtype=np.float64).reshape(-1, dim)
            self._keep.extend([xp, wp])
            prob.n_x_pts, prob.x_pts = xp.shape[0], _ptr(xp, C.c_double)
            prob.n_w_pts, prob.w_pts = wp.shape[0], _ptr(wp, C.c_double)
            prob.w_lo, prob.w_side = w_lo, w_side
        opts = BuildOpts(seed=seed, sample_factor=3, max_rounds=3, tol=tol, threads=threads, factor_file=None)
        errors = []

        def cb(pin, pout, nrhs, adjoint, _ctx):
            try:
                li, lo = (n_out, n_in) if adjoint else (n_in, n_out)
                v = np.ctypeslib.as_array(pin, shape=(2 * nrhs * li,)).view(np.complex128).reshape(nrhs, li)
                res = np.ascontiguousarray(apply(v.copy(), bool(adjoint)), dtype=np.complex128).reshape(nrhs, lo)
                np.ctypeslib.as_array(pout, shape=(2 * nrhs * lo,))[:] = res.view(np.float64).ravel()
            except Exception as e:   # no exception may cross the C ABI
                errors.append(e)
        fn = APPLY_FN(cb)
        h = C.c_void_p()
        code = lib().mbf_build_from_applies(C.byref(prob), C.cast(fn, C.c_void_p), None, C.byref(opts), C.byref(h))
        if errors:
            raise errors[0]
        _check(code)
        self._handle = h
        _check(lib().mbf_factors_view(h, C.byref(self.view)))
        return self

    @classmethod
    def from_arrays(cls, d, L, n_out, n_in, x_perm, x_off, w_perm, w_off, RU, RV, UL, VL, G, H, S,
                    nnz=0):
        """Wrap caller arrays (numpy) in the mbf_factors_t layout of include/mbf.h."""
        self = cls()
        k = self._keep
        c64 = lambda a: np.ascontiguousarray(a, dtype=np.complex128)
        arrs = dict(x_perm=np.ascontiguousarray(x_perm, np.int64), x_off=np.ascontiguousarray(x_off, np.int64),
                    w_perm=np.ascontiguousarray(w_perm, np.int64), w_off=np.ascontiguousarray(w_off, np.int64),
                    RU=np.ascontiguousarray(RU, np.int32), RV=np.ascontiguousarray(RV, np.int32),
                    UL=c64(UL), VL=c64(VL), S=np.ascontiguousarray(S, np.float64))
        k.extend(arrs.values())
        Gs = [c64(a) for a in G]
        Hs = [c64(a) for a in H]
        k.extend(Gs + Hs)
        Gp = (C.POINTER(C.c_double) * len(Gs))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in Gs])
        Hp = (C.POINTER(C.c_double) * len(Hs))(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in Hs])
        k.extend([Gp, Hp])
        v = self.view
        v.dim, v.L, v.n_out, v.n_in = d, L, n_out, n_in
        v.n_w = arrs["w_perm"].size
        v.x_perm, v.x_off = _ptr(arrs["x_perm"], C.c_int64), _ptr(arrs["x_off"], C.c_int64)
        v.w_perm, v.w_off = _ptr(arrs["w_perm"], C.c_int64), _ptr(arrs["w_off"], C.c_int64)
        v.RU, v.RV = _ptr(arrs["RU"], C.c_int32), _ptr(arrs["RV"], C.c_int32)
        v.max_leaf_x, v.max_leaf_w = arrs["UL"].shape[1], arrs["VL"].shape[1]
        v.UL = arrs["UL"].ctypes.data_as(C.POINTER(C.c_double))
        v.VL = arrs["VL"].ctypes.data_as(C.POINTER(C.c_double))
        v.G = C.cast(Gp, C.POINTER(C.POINTER(C.c_double)))
        v.H = C.cast(Hp, C.POINTER(C.POINTER(C.c_double)))
        v.S = _ptr(arrs["S"], C.c_double)
        v.nnz = nnz
        return self

    def save(self, path):
        """Write the factor set to a factor file (mbf_factors_save)."""
        _check(lib().mbf_factors_save(C.byref(self.view), os.fsencode(path)))

    @classmethod
    def load(cls, path):
        """Factors read from a factor file (mbf_factors_load)."""
        self = cls()
        h = C.c_void_p()
        _check(lib().mbf_factors_load(os.fsencode(path), C.byref(h)))
        self._handle = h
        _check(lib().mbf_factors_view(h, C.byref(self.view)))
        return self

    # ---- read-only numpy views of the padded arrays (library-built factors)
    def arrays(self, copy=True):
        """The factor set as numpy arrays (the oracle's FactorSet fields); copy=False
        gives views of the library's arrays, valid until close()."""
        v = self.view
        d, L = v.dim, v.L
        c, h = 2 ** d, L // 2
        nL = c ** L
        RU = np.ctypeslib.as_array(v.RU, shape=(L + 1,)).copy()
        RV = np.ctypeslib.as_array(v.RV, shape=(L + 1,)).copy()

        def carr(p, shape):
            n = int(np.prod(shape))
            a = np.ctypeslib.as_array(p, shape=(2 * n,)).view(np.complex128).reshape(shape)
            return a.copy() if copy else a

        out = dict(d=d, L=L, n_out=v.n_out, n_in=v.n_in,
                   x_perm=np.ctypeslib.as_array(v.x_perm, shape=(v.n_out,)).copy(),
                   x_off=np.ctypeslib.as_array(v.x_off, shape=(nL + 1,)).copy(),
                   w_perm=np.ctypeslib.as_array(v.w_perm, shape=(v.n_w,)).copy(),
                   w_off=np.ctypeslib.as_array(v.w_off, shape=(nL + 1,)).copy(), RU=RU, RV=RV,
                   UL=carr(v.UL, (nL, v.max_leaf_x, RU[L])), VL=carr(v.VL, (nL, v.max_leaf_w, RV[L])),
                   S=np.ctypeslib.as_array(v.S, shape=(c ** h * c ** h * RU[h],)).reshape(
                       c ** h, c ** h, RU[h]).copy(), nnz=v.nnz)
        out["G"] = [carr(v.G[q], (c ** l, c ** (L - l - 1), c, RU[l + 1], c, RU[l]))
                    for q, l in enumerate(range(h, L))]
        out["H"] = [carr(v.H[q], (c ** l, c ** (L - l - 1), c, RV[l + 1], c, RV[l]))
                    for q, l in enumerate(range(h, L))]
        return out

    def device_bytes(self):
        """(SIMT arena + item table, tensor tiles) bytes an operator of these factors takes
        on the device (mbf_factors_device_bytes; no device needed)."""
        a, b = C.c_int64(), C.c_int64()
        _check(lib().mbf_factors_device_bytes(C.byref(self.view), C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if self._handle is not None:
            lib().mbf_factors_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """Device-resident packed factorization (mbf_op_t)."""

    def __init__(self, factors: HostFactors):
        self._h = C.c_void_p()
        _check(lib().mbf_op_create(C.byref(factors.view), C.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def info(self) -> OpInfo:
        inf = OpInfo()
        _check(lib().mbf_op_info(self._h, C.byref(inf)))
        return inf

    def estimate_error(self, kernel="dft", n_samples=256, seed=1, stream: int = 0) -> float:
        """Relative error against the direct sum on sampled outputs (mbf_op_estimate_error);
        kernel: a built-in name or an entry-function address."""
        fn = builtin_kernel(kernel) if isinstance(kernel, str) else kernel
        e = C.c_double()
        _check(lib().mbf_op_estimate_error(self._h, fn, None, n_samples, seed, C.c_void_p(stream),
                                           C.byref(e)))
        return e.value

    def apply(self, g_ptr: int, u_ptr: int, nrhs: int, precision=MBF_PREC_AUTO, stream: int = 0):
        """u = K_f g on device pointers (complex64, [nrhs][N])."""
        _check(lib().mbf_apply(self._h, C.c_void_p(g_ptr), C.c_void_p(u_ptr), nrhs, precision,
                               C.c_void_p(stream)))

    def apply_adjoint(self, u_ptr: int, g_ptr: int, nrhs: int, precision=MBF_PREC_AUTO,
                      stream: int = 0):
        _check(lib().mbf_apply_adjoint(self._h, C.c_void_p(u_ptr), C.c_void_p(g_ptr), nrhs,
                                       precision, C.c_void_p(stream)))

    def apply_host(self, g: np.ndarray, nrhs: int, precision=MBF_PREC_AUTO, stream: int = 0):
        """Host complex64 [nrhs][n_in] -> host complex64 [nrhs][n_out] (copies included)."""
        inf = self.info()
        g = np.ascontiguousarray(g, dtype=np.complex64)
        u = np.empty((nrhs, inf.n_out), dtype=np.complex64)
        _check(lib().mbf_apply_host(self._h, g.ctypes.data_as(C.c_void_p),
                                    u.ctypes.data_as(C.c_void_p), nrhs, precision, C.c_void_p(stream)))
        return u

    def apply_host_batch(self, g, nrhs: int, precision=MBF_PREC_AUTO, stream: int = 0, out=None):
        """Host complex64 [nbatch][nrhs][n_in] -> host [nbatch][nrhs][n_out]: the panels
        pipelined through the device (copy engines overlapping the applies).  g and out
        may be numpy arrays or CPU torch tensors (page-locked ones overlap)."""
        inf = self.info()
        if hasattr(g, "data_ptr"):
            if str(g.dtype) != "torch.complex64" or not g.is_contiguous() or g.device.type != "cpu":
                raise ValueError("g must be a contiguous complex64 CPU tensor")
            nb = g.numel() // max(1, nrhs * inf.n_in)
            gp = g.data_ptr()
        else:
            g = np.ascontiguousarray(g, dtype=np.complex64)
            nb = g.size // max(1, nrhs * inf.n_in)
            gp = g.ctypes.data
        if nb * nrhs * inf.n_in != (g.numel() if hasattr(g, "numel") else g.size):
            raise ValueError("g is not nbatch x nrhs x n_in")
        if out is None:
            out = np.empty((nb, nrhs, inf.n_out), dtype=np.complex64)
        if hasattr(out, "data_ptr"):
            if str(out.dtype) != "torch.complex64" or not out.is_contiguous() or out.device.type != "cpu":
                raise ValueError("out must be a contiguous complex64 CPU tensor")
            up = out.data_ptr()
        else:
            if out.dtype != np.complex64 or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a C-contiguous complex64 array")
            up = out.ctypes.data
        osz = out.numel() if hasattr(out, "numel") else out.size
        if osz != nb * nrhs * inf.n_out:
            raise ValueError("out is not nbatch x nrhs x n_out")
        _check(lib().mbf_apply_host_batch(self._h, C.c_void_p(gp), C.c_void_p(up), nb, nrhs, precision,
                                          C.c_void_p(stream)))
        return out

    def set_profiling(self, enable: bool = True):
        _check(lib().mbf_op_set_profiling(self._h, 1 if enable else 0))

    def profile(self) -> dict:
        """{kernel: (launches, total ms)} since profiling was enabled or last read."""
        p = Profile()
        _check(lib().mbf_op_profile(self._h, C.byref(p)))
        return {p.name[k].value.decode(): (int(p.launches[k]), float(p.ms[k])) for k in range(p.n_kinds)}

    def tune(self, stream: int = 0) -> TuneResult:
        """Run the autotuner (blocking); returns its measurements and choices."""
        r = TuneResult()
        _check(lib().mbf_op_tune(self._h, C.c_void_p(stream), C.byref(r)))
        return r

    def check(self, stream: int = 0):
        _check(lib().mbf_op_check(self._h, C.c_void_p(stream)))

    def debug_stall(self, stage: int, wait_ns: int = 0):
        """Failure-detection test hook (mbf_op_debug_stall); stage=-1, wait_ns=0 turn it off."""
        _check(lib().mbf_op_debug_stall(self._h, stage, wait_ns))

    def close(self):
        if self._h:
            lib().mbf_op_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def form_batch(ops, nrhs, op_work, free_slots=1, **opts):
    """The server's batch rule (mbf_debug_form_batch) on a queue of requests on operators
    ops[i] with nrhs[i] RHS, oldest first: the group of the next batch each request joins
    (-1: stays queued).  op_work[k]: factor traffic of operator k per RHS."""
    n = len(ops)
    o = ServerOpts(opts.get("staging_budget_bytes", 0), opts.get("max_inflight", 0), opts.get("max_batch_rhs", 0),
                   opts.get("max_queue", 0), 1, opts.get("max_batch_ops", 0), opts.get("mix_work_pct", 0))
    a_ops = (C.c_int32 * max(n, 1))(*ops)
    a_rhs = (C.c_int64 * max(n, 1))(*nrhs)
    a_w = (C.c_double * max(len(op_work), 1))(*op_work)
    out = (C.c_int32 * max(n, 1))()
    _check(lib().mbf_debug_form_batch(a_ops, a_rhs, n, a_w, len(op_work), free_slots, C.byref(o), out))
    return list(out)[:n]


def split_sms(work, share):
    """The server's split of a batch's SMs among its groups (mbf_debug_split_sms): share
    SMs in proportion to work[k], at least one each, the remainder to the group of most
    work."""
    n = len(work)
    a_w = (C.c_double * max(1, n))(*work)
    out = (C.c_int32 * max(1, n))()
    _check(lib().mbf_debug_split_sms(a_w, n, share, out))
    return list(out)[:n]


class Server:
    """Serving loop (mbf_server_t): continuous batching of applies on resident operators."""

    def __init__(self, staging_budget_bytes: int = 0, max_inflight: int = 0, max_batch_rhs: int = 0,
                 max_queue: int = 0, use_graphs: bool = True, max_batch_ops: int = 0, mix_work_pct: int = 0):
        o = ServerOpts(staging_budget_bytes, max_inflight, max_batch_rhs, max_queue, 1 if use_graphs else 0,
                       max_batch_ops, mix_work_pct)
        self._h = C.c_void_p()
        _check(lib().mbf_server_create(C.byref(o), C.byref(self._h)))

    def submit(self, op: "Operator", g_ptr: int, u_ptr: int, nrhs: int) -> int:
        """Queue u = K_f g (device buffers, caller-owned until DONE).  Raises MbfError with
        code MBF_ERR_BUSY when the queue or the staging budget is full."""
        t = C.c_int64()
        _check(lib().mbf_submit(self._h, op.handle, C.c_void_p(g_ptr), C.c_void_p(u_ptr), nrhs, C.byref(t)))
        return t.value

    def poll(self, ticket: int) -> RequestStatus:
        st = RequestStatus()
        _check(lib().mbf_poll(self._h, ticket, C.byref(st)))
        return st

    def drain(self, timeout_s: float = 60.0):
        _check(lib().mbf_server_drain(self._h, timeout_s))

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(lib().mbf_server_stats(self._h, C.byref(st)))
        return st

    def close(self):
        if self._h:
            _check(lib().mbf_server_destroy(self._h))
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MsBF:
    """Multiscale butterfly factorization (mbf_msbf_t, §4): per-corona operators plus the
    dense centre, applied as the sum of eq. (f1)."""

    def __init__(self):
        self._h = C.c_void_p()
        self._parts = []

    @classmethod
    def build(cls, n, r, kernel="fio_iso", n_center=16, seed=7, threads=0, sample_factor=3, max_rounds=3,
              tol=1e-14, factor_file=None):
        """Host FP64 construction of every part and the centre (mbf_build_msbf); with
        factor_file, corona k's factors are loaded from (or written to) factor_file.t<k>."""
        self = cls()
        prob = Problem(dim=2, n=n, L=2, r=r, tree=MBF_TREE_UNIFORM)
        opts = BuildOpts(seed=seed, sample_factor=sample_factor, max_rounds=max_rounds, tol=tol, threads=threads,
                         factor_file=None if factor_file is None else os.fsencode(factor_file))
        fn = builtin_kernel(kernel) if isinstance(kernel, str) else kernel
        _check(lib().mbf_build_msbf(C.byref(prob), fn, None, C.byref(opts), n_center, C.byref(self._h)))
        return self

    @classmethod
    def create(cls, parts, center_kernel, center_index):
        """From resident operators (kept alive by this object) and the centre kernel
        [n_c][n_out] (complex) on the natural Omega indices center_index."""
        self = cls()
        self._parts = list(parts)
        arr = (C.c_void_p * max(1, len(parts)))(*[p.handle.value for p in parts])
        kc = np.ascontiguousarray(center_kernel, dtype=np.complex128)
        ci = np.ascontiguousarray(center_index, dtype=np.int64)
        _check(lib().mbf_msbf_create(arr, len(parts), kc.ctypes.data_as(C.c_void_p),
                                     ci.ctypes.data_as(C.c_void_p), ci.size, 0, C.byref(self._h)))
        return self

    @property
    def handle(self):
        return self._h

    def info(self) -> MsbfInfo:
        inf = MsbfInfo()
        _check(lib().mbf_msbf_info(self._h, C.byref(inf)))
        return inf

    def apply(self, g_ptr: int, u_ptr: int, nrhs: int, precision=MBF_PREC_AUTO, stream: int = 0):
        _check(lib().mbf_msbf_apply(self._h, C.c_void_p(g_ptr), C.c_void_p(u_ptr), nrhs, precision,
                                    C.c_void_p(stream)))

    def apply_adjoint(self, u_ptr: int, g_ptr: int, nrhs: int, precision=MBF_PREC_AUTO, stream: int = 0):
        _check(lib().mbf_msbf_apply_adjoint(self._h, C.c_void_p(u_ptr), C.c_void_p(g_ptr), nrhs, precision,
                                            C.c_void_p(stream)))

    def part_handle(self, i: int):
        h = C.c_void_p()
        _check(lib().mbf_msbf_part(self._h, i, C.byref(h)))
        return h

    def check(self, stream: int = 0):
        """mbf_op_check on every part (a device wait that ran out of time raises)."""
        for i in range(self.info().n_parts):
            _check(lib().mbf_op_check(self.part_handle(i), C.c_void_p(stream)))

    def close(self):
        if self._h:
            _check(lib().mbf_msbf_destroy(self._h))
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def layout_apply(factors, g, path=0, adjoint=False):
    """Host FP64 apply of the packed device layout (mbf_debug_layout_apply): path 0 the
    SIMT arena, path 1 the tensor tiles; forward or adjoint.  g: complex [nrhs, n] ->
    complex128 [nrhs, n']."""
    g = np.ascontiguousarray(np.atleast_2d(g), dtype=np.complex128)
    v = factors.view
    n_dst = v.n_in if adjoint else v.n_out
    out = np.empty((g.shape[0], n_dst), dtype=np.complex128)
    _check(lib().mbf_debug_layout_apply(C.byref(v), path, 1 if adjoint else 0, g.ctypes.data_as(C.c_void_p),
                                        out.ctypes.data_as(C.c_void_p), g.shape[0]))
    return out
