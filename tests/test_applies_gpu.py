"""Case (i) construction with a fast black box (§2.3, §3.3 Example 2): the factors of
K~ = K F K are built from products with K~ and K~^* computed as the paper describes --
K and K^* by this library's own GPU apply (a Case (ii) factorization of the Example-1
FIO), F and F^* by the FFT -- and the resulting factorization is applied on the GPU
(FP32 SIMT and split-BF16x3 tensor cores) against the oracle's FP64 apply of the same
factors, and against the black box within the factorization's own error."""
import numpy as np
import pytest

from mbf_synth import complex_normal
from oracle import bf as B
from paper_1509_07925_gb300.binding import MBF_PREC_BF16X3, MBF_PREC_FP32_SIMT

from gpu_util import export_factors, gpu_apply, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_kfk_from_gpu_applies_and_fft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding as bd
    n, L = 32, 4
    N = n * n
    K = bd.Operator(bd.HostFactors.build(2, n, L, 24, tree=bd.MBF_TREE_POLAR, kernel="fio_ellip"))

    def dft(v, adjoint):
        """F (Omega x X): e^{-2 pi i y . eta}, y = m / n, eta in [-n/2, n/2)^2; F^* its adjoint.
        On the grid, F v is the n x n FFT of v read at eta mod n (natural orders)."""
        m = v.reshape(-1, n, n)
        if not adjoint:
            out = np.fft.fftshift(np.fft.fft2(m), axes=(1, 2))
        else:
            out = np.fft.ifft2(np.fft.ifftshift(m, axes=(1, 2))) * N
        return out.reshape(-1, N)

    def kfk(v, adjoint):
        """K F K v (or K^* F^* K^* v) through the GPU apply of K and the FFT."""
        a = gpu_apply(torch, K, v, adjoint=adjoint, precision=MBF_PREC_FP32_SIMT if v.shape[0] < 8 else MBF_PREC_BF16X3)
        a = dft(a, adjoint)
        return gpu_apply(torch, K, a, adjoint=adjoint,
                         precision=MBF_PREC_FP32_SIMT if v.shape[0] < 8 else MBF_PREC_BF16X3)

    hf = bd.HostFactors.build_from_applies(2, n, L, 20, kfk, N, N, tree=bd.MBF_TREE_POLAR)
    fs = export_factors(hf.arrays())
    op = bd.Operator(hf)
    sb = B.SparseBF(fs)
    for nrhs, prec, tol in ((1, MBF_PREC_FP32_SIMT, 1e-5), (64, MBF_PREC_BF16X3, 1e-4)):
        g = complex_normal(N, nrhs, seed=40 + nrhs)
        u = gpu_apply(torch, op, g, precision=prec)
        ref = sb.apply(np.asarray(g, np.complex64).astype(np.complex128))
        assert max(rel(u[k], ref[k]) for k in range(nrhs)) <= tol
    # against the black box: the factorization's own error, with nothing added on the GPU
    g = complex_normal(N, 2, seed=7)
    ub = kfk(g, False)
    eps = rel(sb.apply(g), ub)
    assert eps < 0.6 and rel(gpu_apply(torch, op, g, precision=MBF_PREC_FP32_SIMT), ub) <= eps + 1e-4
    op.close()
    K.close()
