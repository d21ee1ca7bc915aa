"""Failure detection on the GPU, without faulting it.

Every device-side wait of the apply kernels is bounded: when it runs out of time the
kernel sets the operator's status word and its warps leave, and the host learns of
it from mbf_op_check (MBF_ERR_TIMEOUT) or from a served request's error.  These tests
make such a wait run out on purpose through the library's test hook: one dependency
counter waits for a producer the plan does not have, with the wait limit shortened
to 50 ms.  Nothing faults or hangs; the context stays usable and the next apply is
checked against the CPU oracle.  Allocation failures are injected on the host
(mbf_debug_fail_alloc) and must surface as MBF_ERR_OOM with nothing leaked into later
calls.
"""
import time

import numpy as np
import pytest

from mbf_synth import complex_normal

from gpu_util import gpu_apply, import_factors, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SIMT = 1e-5
CASE = ("fio_iso", 64, 2, 4, 24, "polar")


@pytest.fixture(scope="module")
def bd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


def _apply_and_check(bd, op, g):
    """FP32 SIMT apply; gpu_apply reports a device wait that gave up (op.check)."""
    return gpu_apply(torch, op, g, precision=bd.MBF_PREC_FP32_SIMT)


def _launch(bd, op, g, n_out):
    """The apply alone, without the check."""
    gt = torch.from_numpy(np.asarray(g, np.complex64)).cuda()
    ut = torch.empty((g.shape[0], n_out), dtype=torch.complex64, device="cuda")
    op.apply(gt.data_ptr(), ut.data_ptr(), g.shape[0], bd.MBF_PREC_FP32_SIMT,
             torch.cuda.current_stream().cuda_stream)
    return gt, ut


@pytest.mark.parametrize("stage", [1, 3])
def test_stalled_dependency_times_out_and_the_next_apply_is_clean(bd, stage):
    fs, sb = oracle_case(*CASE)
    op = bd.Operator(import_factors(bd, fs))
    g = complex_normal(fs.n_in, 2, seed=31)
    ref = sb.apply(np.asarray(g, np.complex64).astype(np.complex128))
    assert max(rel(o, r) for o, r in zip(_apply_and_check(bd, op, g), ref)) <= TOL_SIMT
    st = torch.cuda.current_stream().cuda_stream
    op.debug_stall(stage, 50_000_000)          # 50 ms limit, one producer missing
    t0 = time.perf_counter()
    keep = _launch(bd, op, g, fs.n_out)
    with pytest.raises(bd.MbfError) as e:
        op.check(st)
    elapsed = time.perf_counter() - t0
    assert e.value.code == bd.MBF_ERR_TIMEOUT and "dependency counter" in str(e.value)
    assert elapsed < 1.5, elapsed              # the short limit, not the default 2 s
    del keep
    op.check(st)                               # the flag was cleared by the report
    op.debug_stall(-1, 0)
    for _ in range(2):
        out = _apply_and_check(bd, op, g)
        assert max(rel(o, r) for o, r in zip(out, ref)) <= TOL_SIMT
    op.close()


def test_served_request_on_a_stalled_operator_fails_alone(bd):
    """The server copies the status word with each batch: a batch whose apply gave up
    fails its own requests with MBF_ERR_TIMEOUT; later batches run normally."""
    fs, sb = oracle_case(*CASE)
    op = bd.Operator(import_factors(bd, fs))
    g = complex_normal(fs.n_in, 1, seed=32)
    ref = sb.apply(np.asarray(g, np.complex64).astype(np.complex128))
    gt = torch.from_numpy(np.asarray(g, np.complex64)).cuda()
    srv = bd.Server(staging_budget_bytes=1 << 26, max_inflight=2, max_batch_rhs=8)

    def serve():
        u = torch.empty((1, fs.n_out), dtype=torch.complex64, device="cuda")
        tk = srv.submit(op, gt.data_ptr(), u.data_ptr(), 1)
        t0 = time.perf_counter()
        while True:
            s = srv.poll(tk)
            if s.state in (bd.MBF_REQ_DONE, bd.MBF_REQ_ERROR):
                return s, u
            assert time.perf_counter() - t0 < 10.0
            time.sleep(0.001)

    op.debug_stall(1, 50_000_000)
    s, _ = serve()
    assert s.state == bd.MBF_REQ_ERROR and s.error == bd.MBF_ERR_TIMEOUT
    op.debug_stall(-1, 0)
    s, u = serve()
    assert s.state == bd.MBF_REQ_DONE
    assert rel(u.cpu().numpy().astype(np.complex128)[0], ref[0]) <= TOL_SIMT
    srv.close()
    op.close()


def test_injected_allocation_failures(bd):
    """Fail the k-th device allocation of operator creation for every k: the call
    reports MBF_ERR_OOM (or, for the tensor path's own arrays, creates an operator
    without it and says why); afterwards a normal operator is created and applies
    correctly."""
    fs, sb = oracle_case(*CASE)
    hf = import_factors(bd, fs)
    ooms, degraded = 0, 0
    try:
        for k in range(16):
            bd._check(bd.lib().mbf_debug_fail_alloc(k))
            try:
                op = bd.Operator(hf)
            except bd.MbfError as e:
                assert e.code == bd.MBF_ERR_OOM, str(e)
                ooms += 1
                continue
            inf = op.info()
            if not inf.tensor_ok:
                assert b"cudaMalloc" in inf.tensor_unavailable
                degraded += 1
            op.close()
    finally:
        bd._check(bd.lib().mbf_debug_fail_alloc(-1))
    assert ooms >= 9 and degraded >= 1
    op = bd.Operator(hf)
    assert op.info().tensor_ok
    g = complex_normal(fs.n_in, 1, seed=33)
    ref = sb.apply(np.asarray(g, np.complex64).astype(np.complex128))
    assert rel(_apply_and_check(bd, op, g)[0], ref[0]) <= TOL_SIMT
    op.close()
