"""The allocation-free entry point mbf_apply_static (GPU).

It exists for callers that may not allocate device memory at apply time (their
memory is owned by another allocator or held to a fixed budget, or allocating
could synchronize a latency-critical loop): it runs the FP32 apply with its
workspace in a fixed library-global device array.  This file is collected last so
that a failure here cannot hide any other test; it also passes on its own in a
fresh process (every fixture is local to this module).

Checks, through the C ABI: two calls in a row give the same result as mbf_apply
and as the CPU oracle's FP64 apply of the same factors, within the FP32 tolerance
of the other GPU tests (relative L2 <= 1e-5 per RHS), for operators of different
size in turn (so each call sees the previous one's leftover scratch), and a
problem whose workspace exceeds the array is rejected with MBF_ERR_INVALID
without running.
"""
import ctypes as C

import numpy as np
import pytest

from mbf_synth import complex_normal

from oracle import bf as B

from gpu_util import export_factors, import_factors, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SIMT = 1e-5


@pytest.fixture(scope="module")
def bd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


def _run(bd, fn, op, g, nrhs, n_out):
    st = torch.cuda.current_stream().cuda_stream
    gt = torch.from_numpy(np.ascontiguousarray(g, dtype=np.complex64)).cuda()
    ut = torch.full((nrhs, n_out), float("nan"), dtype=torch.complex64, device="cuda")
    if fn == "static":
        code = bd.lib().mbf_apply_static(op.handle, C.c_void_p(gt.data_ptr()), C.c_void_p(ut.data_ptr()),
                                         nrhs, C.c_void_p(st))
    else:
        code = bd.lib().mbf_apply(op.handle, C.c_void_p(gt.data_ptr()), C.c_void_p(ut.data_ptr()), nrhs,
                                  bd.MBF_PREC_FP32_SIMT, C.c_void_p(st))
    bd._check(code)
    op.check(st)
    return ut.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("case,nrhs", [(("dft", 64, 2, 4, 16, "none"), 1),
                                       (("fio_iso", 64, 2, 4, 24, "polar"), 3),
                                       (("dft", 8, 3, 2, 16, "none"), 5)])
def test_static_apply_matches_apply_twice(bd, case, nrhs):
    fs, sb = oracle_case(*case)
    op = bd.Operator(import_factors(bd, fs))
    g = complex_normal(fs.n_in, nrhs, seed=21)
    ref = _run(bd, "apply", op, g, nrhs, fs.n_out)
    exact = sb.apply(np.ascontiguousarray(g, dtype=np.complex64).astype(np.complex128))
    for _ in range(2):
        out = _run(bd, "static", op, g, nrhs, fs.n_out)
        assert np.all(np.isfinite(out))
        for k in range(nrhs):
            assert rel(out[k], ref[k]) <= TOL_SIMT
            assert rel(out[k], exact[k]) <= TOL_SIMT
    op.close()


def test_static_apply_rejects_oversized_workspace(bd):
    """2-D DFT n=128, depth 6, r=16: 7 stages of c^L * r = 65,536 entries, so 4 RHS per
    pass need 7 * 8 * 65,536 * 4 bytes > 4 MiB (rejected); 1 RHS (3.7 MB) fits and runs."""
    hf = bd.HostFactors.build(2, 128, 6, 16, kernel="dft")
    op = bd.Operator(hf)
    n = 128 * 128
    st = torch.cuda.current_stream().cuda_stream
    g = torch.zeros((4, n), dtype=torch.complex64, device="cuda")
    u = torch.full((4, n), 3.0, dtype=torch.complex64, device="cuda")
    code = bd.lib().mbf_apply_static(op.handle, C.c_void_p(g.data_ptr()), C.c_void_p(u.data_ptr()), 4,
                                     C.c_void_p(st))
    assert code == bd.MBF_ERR_INVALID
    assert b"static scratch" in bd.lib().mbf_last_error()
    torch.cuda.synchronize()
    assert torch.all(u == 3.0)            # nothing ran
    gh = complex_normal(n, 1, seed=2)
    ref = _run(bd, "apply", op, gh, 1, n)
    exact = B.SparseBF(export_factors(hf.arrays())).apply(
        np.ascontiguousarray(gh, dtype=np.complex64).astype(np.complex128))
    for _ in range(2):
        out = _run(bd, "static", op, gh, 1, n)
        assert rel(out[0], ref[0]) <= TOL_SIMT
        assert rel(out[0], exact[0]) <= TOL_SIMT
    op.close()
