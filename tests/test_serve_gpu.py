"""GPU tests of the serving loop and the autotuner: continuous batching with
same-operator coalescing, graph launches and overlapping batches; every result equals
the oracle's FP64 apply of the same factors (within the split-BF16x3 tolerance, since
a coalesced batch may run on the tensor cores) and equals the same request applied
alone; admission refuses what does not fit the staging budget; ticket lifecycle."""
import numpy as np
import pytest

from mbf_synth import complex_normal

from gpu_util import import_factors, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
OPS = [("dft", 16, 2, 2, 8, "none"), ("fio_iso", 32, 2, 4, 12, "polar"), ("dft", 64, 2, 4, 16, "none"),
       ("fio_iso", 64, 2, 4, 24, "polar")]


@pytest.fixture(scope="module")
def bd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ops(bd):
    out = []
    for case in OPS:
        fs, sb = oracle_case(*case)
        out.append((bd.Operator(import_factors(bd, fs)), fs, sb))
    return out


def _requests(ops, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        k = int(rng.integers(len(ops)))
        nrhs = int(rng.integers(1, 13))
        _, fs, _ = ops[k]
        reqs.append((k, complex_normal(fs.n_in, nrhs, seed=1000 + i)))
    return reqs


def _wait(bd, srv, tickets, timeout=60.0):
    import time
    t0 = time.time()
    out = {}
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            st = srv.poll(t)
            if st.state in (bd.MBF_REQ_DONE, bd.MBF_REQ_ERROR):
                out[t] = st
        assert time.time() - t0 < timeout, "requests did not complete"
    return out


def _run(bd, srv, ops, reqs):
    bufs, tickets = [], []
    for k, g in reqs:
        op, fs, _ = ops[k]
        gt = torch.from_numpy(g.astype(np.complex64)).cuda()
        ut = torch.full((g.shape[0], fs.n_out), float("nan"), dtype=torch.complex64, device="cuda")
        bufs.append((gt, ut))
    torch.cuda.synchronize()
    for (k, g), (gt, ut) in zip(reqs, bufs):
        tickets.append(srv.submit(ops[k][0], gt.data_ptr(), ut.data_ptr(), g.shape[0]))
    sts = _wait(bd, srv, tickets)
    res = [ut.cpu().numpy().astype(np.complex128) for _, ut in bufs]
    return res, [sts[t] for t in tickets]


def test_mix_matches_oracle_and_alone(bd, ops):
    reqs = _requests(ops, 48, seed=5)
    # alone: one request at a time, one slot, no coalescing
    alone_srv = bd.Server(max_inflight=1, max_batch_rhs=1 << 20)
    alone = []
    for r in reqs:
        res, sts = _run(bd, alone_srv, ops, [r])
        assert sts[0].state == bd.MBF_REQ_DONE and sts[0].batch_requests == 1
        alone.append(res[0])
    alone_srv.close()
    # in the mix: all submitted at once, 4 slots, coalescing up to 64 RHS
    srv = bd.Server(max_inflight=4, max_batch_rhs=64)
    mix, sts = _run(bd, srv, ops, reqs)
    stats = srv.stats()
    srv.close()
    for (k, g), a, m, st in zip(reqs, alone, mix, sts):
        assert st.state == bd.MBF_REQ_DONE, st.error
        ref = ops[k][2].apply(g)
        assert np.all(np.isfinite(m))
        assert rel(m, ref) <= TOL, (k, g.shape, rel(m, ref))
        assert rel(a, ref) <= TOL
        assert rel(m, a) <= 2 * TOL
        assert st.t_submit <= st.t_start <= st.t_done
    assert stats.completed == len(reqs) and stats.failed == 0
    assert stats.coalesced_requests > 0 and stats.max_batch_requests > 1
    assert stats.max_concurrent_batches > 1          # batches of different operators overlapped
    assert stats.graph_launches == stats.batches     # every batch was one graph launch


def test_mixed_operators_in_one_graph_launch(bd, ops):
    """Requests of several operators and RHS counts queued together go into one batch,
    one CUDA graph launch with a parallel branch per operator; each result equals the
    oracle and the same request applied alone.  A single slot is held by a blocker (an
    operator whose apply is made to wait 300 ms for a producer it lacks, through the
    failure-detection hook) while the mix is queued behind it."""
    import time
    fs0, _ = oracle_case(*OPS[2])
    blocker = bd.Operator(import_factors(bd, fs0))
    blocker.debug_stall(1, 300_000_000)
    srv = bd.Server(max_inflight=1, max_batch_rhs=64, max_batch_ops=4, mix_work_pct=100000)
    reqs = [(k, complex_normal(ops[k][1].n_in, nrhs, seed=70 + 4 * k + nrhs))
            for k in range(len(ops)) for nrhs in (3, 9)]
    # every buffer exists before the blocker runs (a device synchronize would wait for it)
    bufs = []
    for k, g in reqs:
        gt = torch.from_numpy(g.astype(np.complex64)).cuda()
        ut = torch.full((g.shape[0], ops[k][1].n_out), float("nan"), dtype=torch.complex64, device="cuda")
        bufs.append((gt, ut))
    gb = torch.zeros((1, fs0.n_in), dtype=torch.complex64, device="cuda")
    ub = torch.empty((1, fs0.n_out), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    tb = srv.submit(blocker, gb.data_ptr(), ub.data_ptr(), 1)
    t0 = time.time()
    while srv.poll(tb).state != bd.MBF_REQ_RUNNING:     # the blocker holds the only slot
        assert time.time() - t0 < 10.0
    tickets = [srv.submit(ops[k][0], gt.data_ptr(), ut.data_ptr(), g.shape[0])
               for (k, g), (gt, ut) in zip(reqs, bufs)]
    sts = _wait(bd, srv, tickets)
    sts = [sts[t] for t in tickets]
    stb = _wait(bd, srv, [tb])[tb]
    stats = srv.stats()
    srv.close()
    blocker.close()
    mix = [ut.cpu().numpy().astype(np.complex128) for _, ut in bufs]
    assert stb.state == bd.MBF_REQ_ERROR and stb.error == bd.MBF_ERR_TIMEOUT
    assert stats.mixed_batches >= 1 and stats.max_batch_ops == 4
    assert stats.graph_launches == stats.batches
    assert all(st.batch_requests == len(reqs) for st in sts)   # all of them in one batch
    alone_srv = bd.Server(max_inflight=1)
    for (k, g), m, st in zip(reqs, mix, sts):
        assert st.state == bd.MBF_REQ_DONE, st.error
        ref = ops[k][2].apply(g)
        assert rel(m, ref) <= TOL, (k, g.shape, rel(m, ref))
        a, sa = _run(bd, alone_srv, ops, [(k, g)])
        assert sa[0].batch_requests == 1 and rel(m, a[0]) <= 2 * TOL
    alone_srv.close()


def _queue_behind_blocker(bd, srv, ops, order, seed, nrhs=2):
    """Hold the server's only slot with a stalled blocker, queue requests on the
    operators `order` (in that order, nrhs RHS each) behind it, and wait for all."""
    import time
    fs0, _ = oracle_case(*OPS[2])
    blocker = bd.Operator(import_factors(bd, fs0))
    blocker.debug_stall(1, 200_000_000)
    reqs = [(k, complex_normal(ops[k][1].n_in, nrhs, seed=seed + i)) for i, k in enumerate(order)]
    bufs = []
    for k, g in reqs:
        bufs.append((torch.from_numpy(g.astype(np.complex64)).cuda(),
                     torch.empty((nrhs, ops[k][1].n_out), dtype=torch.complex64, device="cuda")))
    gb = torch.zeros((1, fs0.n_in), dtype=torch.complex64, device="cuda")
    ub = torch.empty((1, fs0.n_out), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    tb = srv.submit(blocker, gb.data_ptr(), ub.data_ptr(), 1)
    t0 = time.time()
    while srv.poll(tb).state != bd.MBF_REQ_RUNNING:
        assert time.time() - t0 < 10.0
    tickets = [srv.submit(ops[k][0], gt.data_ptr(), ut.data_ptr(), nrhs) for (k, _), (gt, ut) in zip(reqs, bufs)]
    sts = _wait(bd, srv, tickets)
    _wait(bd, srv, [tb])
    blocker.close()
    for (k, g), (_, ut), t in zip(reqs, bufs, tickets):
        assert sts[t].state == bd.MBF_REQ_DONE
        assert rel(ut.cpu().numpy().astype(np.complex128), ops[k][2].apply(g)) <= TOL
    return [sts[t] for t in tickets]


def test_batch_policy_work_ratio_and_backlog(bd, ops):
    """Default policy: under a backlog (6 queued > 1 slot x 4 operators per batch) a
    further operator joins a batch only if its factor traffic is at most 25 % of the
    first group's.  A small operator queued first keeps a larger one out of its batch;
    a larger one queued first takes the small one along (one mixed batch).  Without a
    backlog (3 queued) no batch is mixed."""
    small, big = 0, 3          # 2-D DFT n = 16 (256 points), polar FIO n = 64 (4096 points)
    srv = bd.Server(max_inflight=1, max_batch_rhs=64, max_batch_ops=4)
    sts = _queue_behind_blocker(bd, srv, ops, [small] * 3 + [big] * 3, seed=300)
    stats = srv.stats()
    srv.close()
    assert stats.mixed_batches == 0
    assert all(st.batch_requests == 3 for st in sts)
    srv = bd.Server(max_inflight=1, max_batch_rhs=64, max_batch_ops=4)
    sts = _queue_behind_blocker(bd, srv, ops, [big] * 3 + [small] * 3, seed=310)
    stats = srv.stats()
    srv.close()
    assert stats.mixed_batches == 1
    assert all(st.batch_requests == 6 for st in sts)
    srv = bd.Server(max_inflight=1, max_batch_rhs=64, max_batch_ops=4)
    sts = _queue_behind_blocker(bd, srv, ops, [big, small, small], seed=320)
    stats = srv.stats()
    srv.close()
    assert stats.mixed_batches == 0


def test_groups_in_place_and_through_staging(bd, ops):
    """A group of up to 64 RHS is applied in place through a table of the requests' rows;
    a larger one (max_batch_rhs 128: three requests of 30 RHS) through a staging panel.
    Both equal the oracle request by request."""
    for nrhs, rhs_total in ((20, 60), (30, 90)):
        srv = bd.Server(max_inflight=1, max_batch_rhs=128)
        sts = _queue_behind_blocker(bd, srv, ops, [3, 3, 3], seed=400 + nrhs, nrhs=nrhs)
        srv.close()
        assert all(st.batch_requests == 3 and st.batch_rhs == rhs_total for st in sts)


def test_batches_of_one_operator_overlap(bd, ops):
    """With a workspace per slot and operator, batches of the same operator run at the
    same time on different slots; every result still equals the oracle."""
    op, fs, sb = ops[3]
    srv = bd.Server(max_inflight=4, max_batch_rhs=8)
    reqs = [(3, complex_normal(fs.n_in, 8, seed=90 + i)) for i in range(16)]
    res, sts = _run(bd, srv, ops, reqs)
    stats = srv.stats()
    srv.close()
    assert stats.max_concurrent_batches >= 2 and stats.mixed_batches == 0
    for (k, g), m, st in zip(reqs, res, sts):
        assert st.state == bd.MBF_REQ_DONE and st.batch_rhs == 8
        assert rel(m, sb.apply(g)) <= TOL


def test_graphs_off_gives_the_same_results(bd, ops):
    reqs = _requests(ops, 16, seed=9)
    a_srv = bd.Server(max_inflight=2, use_graphs=True)
    a, _ = _run(bd, a_srv, ops, reqs)
    a_srv.close()
    b_srv = bd.Server(max_inflight=2, use_graphs=False)
    b, _ = _run(bd, b_srv, ops, reqs)
    st = b_srv.stats()
    b_srv.close()
    assert st.graph_launches == 0
    for x, y, (k, g) in zip(a, b, reqs):
        ref = ops[k][2].apply(g)
        assert rel(x, ref) <= TOL and rel(y, ref) <= TOL


def test_admission_by_staging_budget(bd, ops):
    op, fs, _ = ops[2]
    need = 2 * 8 * max(fs.n_in, fs.n_out) * 8             # bytes reserved by an 8-RHS request
    srv = bd.Server(staging_budget_bytes=3 * need, max_inflight=1)
    g = torch.zeros((8, fs.n_in), dtype=torch.complex64, device="cuda")
    us = [torch.empty((8, fs.n_out), dtype=torch.complex64, device="cuda") for _ in range(4)]
    tickets, busy = [], 0
    for u in us:
        try:
            tickets.append(srv.submit(op, g.data_ptr(), u.data_ptr(), 8))
        except bd.MbfError as e:
            assert e.code == bd.MBF_ERR_BUSY
            busy += 1
    # at most three fit at once; the fourth is refused unless one already finished
    assert len(tickets) >= 3
    _wait(bd, srv, tickets)
    srv.drain(30.0)
    # the budget is free again
    t = srv.submit(op, g.data_ptr(), us[0].data_ptr(), 8)
    _wait(bd, srv, [t])
    assert srv.stats().rejected_busy == busy
    srv.close()


def test_ticket_lifecycle(bd, ops):
    op, fs, sb = ops[0]
    srv = bd.Server()
    g = complex_normal(fs.n_in, 3, seed=2)
    gt = torch.from_numpy(g.astype(np.complex64)).cuda()
    ut = torch.empty((3, fs.n_out), dtype=torch.complex64, device="cuda")
    t = srv.submit(op, gt.data_ptr(), ut.data_ptr(), 3)
    st = _wait(bd, srv, [t])[t]
    assert st.state == bd.MBF_REQ_DONE and st.batch_rhs == 3
    with pytest.raises(bd.MbfError) as ei:
        srv.poll(t)                                       # forgotten after DONE was reported
    assert ei.value.code == bd.MBF_ERR_NOT_FOUND
    with pytest.raises(bd.MbfError) as ei:
        srv.submit(op, gt.data_ptr(), ut.data_ptr(), 0)
    assert ei.value.code == bd.MBF_ERR_INVALID
    assert rel(ut.cpu().numpy(), sb.apply(g)) <= 1e-5     # 3 RHS: the FP32 SIMT path
    srv.close()


def test_tuner_choices_keep_results(bd, ops):
    op, fs, sb = ops[3]
    st = torch.cuda.current_stream().cuda_stream
    r = op.tune(st)
    assert r.n_simt == 7 and all(r.simt_ms[i] > 0 for i in range(r.n_simt))
    assert r.n_slots >= 1
    tried = list(zip(list(r.slots)[:r.n_slots], list(r.panel_buffers)[:r.n_slots]))
    assert all(b in (2, 3) for _, b in tried) and (r.tc_slots_chosen, r.tc_buffers_chosen) in tried
    assert 1 <= r.tc_min_rhs <= 65
    # SIMT time grows with the RHS count; one tensor panel covers up to 64 RHS
    assert r.simt_ms[r.n_simt - 1] > r.simt_ms[0]
    from gpu_util import gpu_apply
    for nrhs in (r.tc_min_rhs - 1, r.tc_min_rhs, 40):
        if nrhs < 1:
            continue
        g = complex_normal(fs.n_in, nrhs, seed=nrhs)
        u = gpu_apply(torch, op, g, precision=bd.MBF_PREC_AUTO)
        assert rel(u, sb.apply(g)) <= TOL
