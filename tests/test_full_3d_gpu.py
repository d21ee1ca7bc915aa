"""GPU parity at the full size of the 3-D workload: the 3-D DFT (§5, the d > 2 case of
the factorization), n = 64 (262,144 points per side), octree depth L = 6 (one-point
leaves), r = 32: 32 RHS on the tensor cores (split-BF16x3, tiles of c r = 256 rows and
columns) and 1 RHS on the FP32 SIMT kernel.

The factors are built by the library's host builder (about 43 GB of complex64 on the
device; the FP64 set is 86 GB on the host, read below as views of the library's arrays so
that it is held once).  The reference is the oracle's level-by-level FP64 apply of the
same factors (`oracle.bf.BlockBF`), compared output by output; against the direct sum on
256 sampled outputs the GPU may add no more than the arithmetic tolerance to the
factorization's own error.

The host construction takes tens of minutes on 16 cores, so the test runs only when
MBF_FULL_SIZE=1 is set; the factors are checkpointed in a factor file
($MBF_FULL_3D_FILE, default /tmp/mbf_dft3_n64_L6_r32), which the benchmark loads with
`bench.py --workload dft3_n64_L6_r32_x32 --factor-file <file> --no-cpu-baseline`."""
import os
import time

import numpy as np
import pytest

from mbf_synth import WORKLOADS, complex_normal, sample_outputs
from oracle import bf as B
from oracle import direct as D
from oracle import problem as P
from paper_1509_07925_gb300.binding import MBF_PREC_BF16X3, MBF_PREC_FP32_SIMT

from gpu_util import export_factors, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("MBF_FULL_SIZE") != "1",
                                 reason="full-size 3-D build takes tens of minutes: set MBF_FULL_SIZE=1")]

WL = WORKLOADS["dft3_n64_L6_r32_x32"]
FILE = os.environ.get("MBF_FULL_3D_FILE", "/tmp/mbf_dft3_n64_L6_r32")
TOL_BF16X3 = 1e-4
TOL_SIMT = 1e-5


def test_full_size_3d_dft_n64_L6_r32():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding as bd
    t0 = time.time()
    hf = bd.HostFactors.build(WL.dim, WL.n, WL.L, WL.r, tree=bd.MBF_TREE_UNIFORM, kernel=WL.kernel,
                              seed=WL.seed_build, factor_file=FILE)
    op = bd.Operator(hf)
    inf = op.info()
    print(f"built / loaded in {time.time() - t0:.0f} s: {inf.nnz_algorithmic / 1e9:.3f} G nonzeros, "
          f"tensor path {'yes' if inf.tensor_ok else 'no'}")
    assert inf.tensor_ok
    fs = export_factors(hf.arrays(copy=False))
    N, R = WL.N, WL.nrhs
    st = torch.cuda.current_stream().cuda_stream

    g = complex_normal(N, R, seed=WL.seed_g)
    gt = torch.from_numpy(g.astype(np.complex64)).cuda()
    ut = torch.full((R, N), float("nan"), dtype=torch.complex64, device="cuda")
    op.apply(gt.data_ptr(), ut.data_ptr(), R, MBF_PREC_BF16X3, st)
    op.check(st)
    u = ut.cpu().numpy().astype(np.complex128)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    ev0.record()
    for _ in range(reps):
        op.apply(gt.data_ptr(), ut.data_ptr(), R, MBF_PREC_BF16X3, st)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    print(f"{R}-RHS apply: {ms:.3f} ms, {N * R / (ms * 1e-3) / 1e9:.2f} G points*RHS/s, "
          f"{8 * inf.nnz_algorithmic / (ms * 1e-3) / 1e9:.0f} GB/s of factor bytes")

    # 1 RHS on the FP32 SIMT kernel
    u1t = torch.full((1, N), float("nan"), dtype=torch.complex64, device="cuda")
    op.apply(gt.data_ptr(), u1t.data_ptr(), 1, MBF_PREC_FP32_SIMT, st)
    op.check(st)
    u1 = u1t.cpu().numpy().astype(np.complex128)

    t0 = time.time()
    ref = B.BlockBF(fs).apply(g)
    print(f"oracle level-by-level FP64 apply of {R} RHS: {time.time() - t0:.0f} s")
    errs = [rel(u[k], ref[k]) for k in range(R)]
    print(f"max rel err vs FP64 factor apply: split-BF16x3 {max(errs):.2e}, "
          f"FP32 SIMT {rel(u1[0], ref[0]):.2e}")
    assert np.all(np.isfinite(u)) and max(errs) <= TOL_BF16X3, max(errs)
    assert np.all(np.isfinite(u1)) and rel(u1[0], ref[0]) <= TOL_SIMT

    X, W = P.grid_x(WL.n, WL.dim), P.grid_omega(WL.n, WL.dim)
    S = sample_outputs(N, WL.n_sample, seed=WL.seed_s)
    ud = D.direct_sum(P.KERNELS[WL.kernel], X, W, g[:4], rows=S)
    eps = D.rel_err(ref[:4, S], ud)
    print(f"factorization error vs direct sum on {WL.n_sample} outputs: {eps:.3e}")
    assert D.rel_err(u[:4, S], ud) <= eps + TOL_BF16X3
    op.close()
    hf.close()
