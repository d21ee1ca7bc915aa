"""GPU parity on explicit non-uniform point sets (§2.6): clustered X and Omega, trees
ragged at every level with empty leaves; the library's factors applied on the GPU
(FP32 SIMT and split-BF16x3 tensor cores, forward and adjoint) against the oracle's
FP64 apply of the same factors, and against the direct sum within the factorization's
own error."""
import numpy as np
import pytest

from oracle import bf as B
from oracle import direct as D
from oracle import problem as P
from paper_1509_07925_gb300.binding import MBF_PREC_BF16X3, MBF_PREC_FP32_SIMT

from gpu_util import export_factors, gpu_apply, rel
from test_points_cpu import clustered_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding as bd
    X, W = clustered_points(6000, 5000, -16.0, 32.0, seed=11)
    hf = bd.HostFactors.build(2, 32, 6, 16, tree=bd.MBF_TREE_POINTS, kernel="fio_iso", x_pts=X, w_pts=W,
                              w_lo=-16.0, w_side=32.0)
    fs = export_factors(hf.arrays())
    op = bd.Operator(hf)
    return bd, op, fs, B.SparseBF(fs), X, W


@pytest.mark.parametrize("nrhs,prec,tol", [(1, MBF_PREC_FP32_SIMT, 1e-5), (3, MBF_PREC_FP32_SIMT, 1e-5),
                                           (64, MBF_PREC_BF16X3, 1e-4)])
def test_points_forward(case, nrhs, prec, tol):
    bd, op, fs, sb, X, W = case
    rng = np.random.default_rng(nrhs)
    g = (rng.standard_normal((nrhs, fs.n_in)) + 1j * rng.standard_normal((nrhs, fs.n_in))) / np.sqrt(2)
    u = gpu_apply(torch, op, g, precision=prec)
    ref = sb.apply(np.asarray(g, np.complex64).astype(np.complex128))
    assert max(rel(u[k], ref[k]) for k in range(nrhs)) <= tol
    if nrhs == 1:
        ud = D.direct_sum(P.kernel_fio_iso, X, W, g)
        eps = D.rel_err(ref, ud)
        assert eps < 1e-3 and D.rel_err(u, ud) <= eps + 1e-5


@pytest.mark.parametrize("nrhs,prec,tol", [(2, MBF_PREC_FP32_SIMT, 1e-5), (64, MBF_PREC_BF16X3, 1e-4)])
def test_points_adjoint(case, nrhs, prec, tol):
    bd, op, fs, sb, X, W = case
    rng = np.random.default_rng(100 + nrhs)
    w = (rng.standard_normal((nrhs, fs.n_out)) + 1j * rng.standard_normal((nrhs, fs.n_out))) / np.sqrt(2)
    ga = gpu_apply(torch, op, w, adjoint=True, precision=prec)
    ref = sb.adjoint(np.asarray(w, np.complex64).astype(np.complex128))
    assert max(rel(ga[k], ref[k]) for k in range(nrhs)) <= tol
