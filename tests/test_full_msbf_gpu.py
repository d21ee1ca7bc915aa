"""GPU parity at the full size of the multiscale workload: the 2-D isotropic FIO with
the multiscale split of §4 (eq. domaindecomp), n = 512 (262,144 points per side),
r = 24, 16 x 16 centre, coronas t = 0..4 of depths 8, 8, 6, 6, 4, applied to 32 RHS
on the tensor cores (split-BF16x3).

Every part is built by the library's host builder (about 1.25 G nonzeros, 10 GB of
complex64 on the device).  The reference is the oracle's level-by-level FP64 apply of
the same factors (`oracle.bf.BlockBF`, equal to the sparse-factor apply to rounding)
plus the dense centre, compared output by output; against the direct sum on 256
sampled outputs the GPU may add no more than the arithmetic tolerance to the
factorization's own error.

The host construction of this operator takes several minutes on 16 cores, so the test
runs only when MBF_FULL_SIZE=1 is set in the environment; its factors are checkpointed in
factor files ($MBF_FULL_SIZE_FILES.t<k>, default /tmp/mbf_msbf_n512_r24.t<k>), which the
benchmark's multiscale leg (`bench.py --workload fio2_msbf_n512_r24_x32 --factor-file ...`)
loads instead of building again."""
import os
import time

import numpy as np
import pytest

from mbf_synth import complex_normal, sample_outputs
from oracle import bf as B
from oracle import direct as D
from oracle import msbf as MS
from oracle import problem as P
from paper_1509_07925_gb300.binding import MBF_PREC_BF16X3

from gpu_util import export_factors, rel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("MBF_FULL_SIZE") != "1",
                                 reason="full-size multiscale build takes minutes: set MBF_FULL_SIZE=1")]

N_SIDE, RANK, CENTRE, NRHS = 512, 24, 16, 32
FILES = os.environ.get("MBF_FULL_SIZE_FILES", "/tmp/mbf_msbf_n512_r24")


def test_full_size_multiscale_n512_r24_32_rhs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding as bd
    n = N_SIDE
    coronas, centre = MS.corona_sets(n, CENTRE)
    assert [t for t, _ in coronas] == [0, 1, 2, 3, 4] and centre.size == 17 * 17
    L = int(np.log2(n))
    t0 = time.time()
    parts, fsets = [], []
    for t, idx in coronas:
        Lt = 2 * ((L - t) // 2)
        half = n / 2 ** (t + 1)
        hf = bd.HostFactors.build(2, n, Lt, RANK, tree=bd.MBF_TREE_SQUARE, kernel="fio_iso", seed=7 + 101 * (t + 1),
                                  w_index=idx, w_lo=-half, w_side=2 * half, factor_file=f"{FILES}.t{t}")
        fsets.append(export_factors(hf.arrays()))
        parts.append(bd.Operator(hf))
        hf.close()
    t_build = time.time() - t0
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    Kc = P.kernel_fio_iso(X[:, None, :], W[centre][None, :, :])
    m = bd.MsBF.create(parts, Kc.T, centre)
    nnz = sum(p.info().nnz_algorithmic for p in parts)
    print(f"built 5 coronas in {t_build:.0f} s: {nnz / 1e9:.3f} G nonzeros")

    g = complex_normal(n * n, NRHS, seed=0)
    gt = torch.from_numpy(g.astype(np.complex64)).cuda()
    ut = torch.full((NRHS, n * n), float("nan"), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    m.apply(gt.data_ptr(), ut.data_ptr(), NRHS, MBF_PREC_BF16X3, st)
    m.check(st)
    u = ut.cpu().numpy().astype(np.complex128)
    # throughput of the 32-RHS apply (CUDA events, after the first apply above)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    ev0.record()
    for _ in range(reps):
        m.apply(gt.data_ptr(), ut.data_ptr(), NRHS, MBF_PREC_BF16X3, st)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    print(f"32-RHS apply: {ms:.3f} ms, {n * n * NRHS / (ms * 1e-3) / 1e9:.2f} G points*RHS/s, "
          f"{8 * nnz / (ms * 1e-3) / 1e9:.0f} GB/s of factor bytes")

    # reference: FP64 level-by-level apply of every part plus the centre
    ref = (Kc @ g[:, centre].T).T
    for fs in fsets:
        ref = ref + B.BlockBF(fs).apply(g)
    errs = [rel(u[k], ref[k]) for k in range(NRHS)]
    print(f"max rel err vs FP64 factor apply over {NRHS} RHS: {max(errs):.2e}")
    assert np.all(np.isfinite(u)) and max(errs) <= 1e-4, max(errs)
    S = sample_outputs(n * n, 256, seed=1)
    ud = D.direct_sum(P.kernel_fio_iso, X, W, g[:4], rows=S)
    eps = D.rel_err(ref[:4, S], ud)
    print(f"factorization error vs direct sum on 256 outputs: {eps:.3e}")
    assert D.rel_err(u[:4, S], ud) <= eps + 1e-4
    m.close()
