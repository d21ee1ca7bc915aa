"""CPU tests of the C-ABI library: it loads, exports every declared symbol, builds
factors on the host, and refuses to run an apply without a GPU (no fallback)."""
import os
import re

import numpy as np
import pytest

from mbf_synth import complex_normal
from oracle import bf as B
from oracle import direct as D
from oracle import problem as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bd():
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mbf_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(bd):
    import ctypes
    lib = ctypes.CDLL(bd.LIBPATH)
    declared = _declared_symbols()
    assert "mbf_apply" in declared and "mbf_build_from_entries" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    # the binding declares a signature for each of them
    assert declared <= set(bd.SIGNATURES)


def test_version_and_error_text(bd):
    assert b"sm_103a" in bd.lib().mbf_version()
    with pytest.raises(bd.MbfError) as ei:
        bd.HostFactors.build(2, 12, 2, 4)          # n not a power of two
    assert ei.value.code == bd.MBF_ERR_INVALID and "power of two" in str(ei.value)
    with pytest.raises(bd.MbfError):
        bd.HostFactors.build(2, 16, 3, 4)          # odd depth


def _to_oracle(a):
    return B.FactorSet(d=a["d"], L=a["L"], n_out=a["n_out"], n_in=a["n_in"], x_perm=a["x_perm"],
                       x_off=a["x_off"], w_perm=a["w_perm"], w_off=a["w_off"], RU=a["RU"], RV=a["RV"],
                       UL=a["UL"], VL=a["VL"], G=a["G"], H=a["H"], S=a["S"])


@pytest.mark.parametrize("case", [("dft", 8, 2, 2, 16, 0), ("dft", 16, 2, 4, 16, 0),
                                  ("dft", 4, 3, 2, 64, 0), ("fio_ellip", 16, 2, 4, 16, 1)])
def test_builder_exact_at_full_rank(bd, case):
    """The library's FP64 builder, applied by the oracle's independent sparse product,
    reproduces K when r covers every block (to the Gram-eigensolver resolution)."""
    kern, n, d, L, r, tree = case
    a = bd.HostFactors.build(d, n, L, r, tree=tree, kernel=kern).arrays()
    K = P.kernel_block(P.KERNELS[kern], P.grid_x(n, d), P.grid_omega(n, d), np.arange(n ** d),
                       np.arange(n ** d))
    Kf = B.SparseBF(_to_oracle(a)).dense()
    assert np.abs(Kf - K).max() < 1e-6


def test_builder_error_matches_oracle_construction(bd):
    """Same configuration, two independent constructions: the direct-sum error of the
    library's factors is within 15% of the oracle's (2-D DFT, n=64, L=4, r=16)."""
    n, L, r = 64, 4, 16
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    g = complex_normal(n * n, 1, seed=0)
    u = D.dft_closed_form(g, n, 2)
    a = bd.HostFactors.build(2, n, L, r, kernel="dft").arrays()
    e_lib = D.rel_err(B.SparseBF(_to_oracle(a)).apply(g), u)
    fs = B.build(P.kernel_dft, X, W, P.uniform_tree(n, 2, L), P.uniform_tree(n, 2, L), r)
    e_or = D.rel_err(B.SparseBF(fs).apply(g), u)
    assert abs(e_lib - e_or) < 0.15 * e_or
    assert a["nnz"] == fs.nnz_algorithmic()


@pytest.mark.parametrize("kern", ["dft", "fio_iso", "fio_ellip"])
def test_builtin_kernels_match_oracle_kernels(bd, kern):
    import ctypes as C
    n = 32
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    rows, cols = np.arange(0, 1024, 7), np.arange(3, 1024, 5)
    xs = np.ascontiguousarray(X[rows])
    ws = np.ascontiguousarray(W[cols])
    out = np.zeros((cols.size, rows.size), dtype=np.complex128)  # column-major m x n
    fn = getattr(bd.lib(), {"dft": "mbf_kernel_dft", "fio_iso": "mbf_kernel_fio_iso",
                            "fio_ellip": "mbf_kernel_fio_ellip"}[kern])
    dp = C.POINTER(C.c_double)
    fn(xs.ctypes.data_as(dp), rows.size, ws.ctypes.data_as(dp), cols.size, 2,
       out.ctypes.data_as(dp), None)
    ref = P.kernel_block(P.KERNELS[kern], X, W, rows, cols)
    assert np.abs(out.T - ref).max() < 1e-12


def test_polar_tree_matches_oracle_tree(bd):
    """Both sides build T_P independently from the polar map of eq. (polar); the
    permutation and leaf offsets agree."""
    a = bd.HostFactors.build(2, 32, 4, 4, tree=bd.MBF_TREE_POLAR, kernel="fio_iso").arrays()
    t = P.polar_tree(32, 4)
    assert np.array_equal(a["w_perm"], t.perm) and np.array_equal(a["w_off"], t.off)
    xt = P.uniform_tree(32, 2, 4)
    assert np.array_equal(a["x_perm"], xt.perm) and np.array_equal(a["x_off"], xt.off)


def test_import_validation_rejects_bad_factor_sets(bd):
    """mbf_op_create validates the interchange layout on the host before touching a
    device: a broken permutation or an oversized rank is MBF_ERR_INVALID."""
    n, d, L = 8, 2, 2
    fs = B.build(P.kernel_dft, P.grid_x(n, d), P.grid_omega(n, d), P.uniform_tree(n, d, L),
                 P.uniform_tree(n, d, L), 16)
    bad = fs.x_perm.copy()
    bad[0] = bad[1]
    hf = bd.HostFactors.from_arrays(d, L, fs.n_out, fs.n_in, bad, fs.x_off, fs.w_perm, fs.w_off,
                                    fs.RU, fs.RV, fs.UL, fs.VL, fs.G, fs.H, fs.S)
    with pytest.raises(bd.MbfError) as ei:
        bd.Operator(hf)
    assert ei.value.code == bd.MBF_ERR_INVALID and "permutation" in str(ei.value)


PLAN_CASES = [("dft", 16, 2, 2, 8, "none"), ("dft", 64, 2, 4, 16, "none"),
              ("fio_iso", 64, 2, 4, 24, "polar"), ("fio_iso", 32, 2, 4, 12, "polar"),
              ("dft", 8, 3, 2, 16, "none"), ("dft", 32, 2, 2, 64, "none")]


@pytest.mark.parametrize("case", PLAN_CASES)
def test_no_gpu_means_no_apply(bd, case):
    """Without a GPU the operator cannot be created: the library fails loudly (CUDA
    error), it never falls back to a host apply.  Packing and the host plan check
    (every gather/scatter in bounds, stage writes == next stage reads, items inside
    the arena) run first, so reaching the CUDA error means the plan passed."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    from gpu_util import oracle_case
    fs, _ = oracle_case(*case)
    hf = bd.HostFactors.from_arrays(fs.d, fs.L, fs.n_out, fs.n_in, fs.x_perm, fs.x_off, fs.w_perm, fs.w_off,
                                    fs.RU, fs.RV, fs.UL, fs.VL, fs.G, fs.H, fs.S)
    with pytest.raises(bd.MbfError) as ei:
        bd.Operator(hf)
    assert ei.value.code in (bd.MBF_ERR_CUDA, bd.MBF_ERR_OOM), str(ei.value)


def test_server_needs_a_gpu(bd):
    """The serving loop owns CUDA streams: without a GPU it is not created (no host
    fallback), and the C ABI rejects NULL arguments without touching the device."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(bd.MbfError) as ei:
        bd.Server()
    assert ei.value.code == bd.MBF_ERR_CUDA, str(ei.value)
    import ctypes
    t = ctypes.c_int64()
    assert bd.lib().mbf_submit(None, None, None, None, 1, ctypes.byref(t)) == bd.MBF_ERR_INVALID
    st = bd.RequestStatus()
    assert bd.lib().mbf_poll(None, 1, ctypes.byref(st)) == bd.MBF_ERR_INVALID
    assert bd.lib().mbf_op_tune(None, None, None) == bd.MBF_ERR_INVALID


def test_multiscale_needs_a_gpu(bd):
    """mbf_build_msbf uploads its parts: without a GPU it fails loudly before building."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(bd.MbfError) as ei:
        bd.MsBF.build(16, 4, n_center=4)
    assert ei.value.code == bd.MBF_ERR_CUDA, str(ei.value)
    import ctypes
    h = ctypes.c_void_p()
    assert bd.lib().mbf_msbf_create(None, 0, None, None, 0, 0, ctypes.byref(h)) == bd.MBF_ERR_INVALID
