"""The serving loop's batch rule (mbf_debug_form_batch: the worker's rule as a pure host
function, no device): which queued requests form the next batch.  Requests are given
oldest first as (operator, RHS); a group's factor traffic is op_work[op] x its RHS."""
import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bd():
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


def test_without_backlog_one_operator_fifo(bd):
    # 4 queued <= 4 slots x 4 operators: no backlog, the oldest request's operator alone
    g = bd.form_batch([1, 0, 1, 0], [2, 2, 2, 2], [1.0, 1.0], free_slots=1)
    assert g == [0, -1, 0, -1]


def test_rhs_cap_skips_a_request_that_does_not_fit_but_takes_later_ones(bd):
    # max_batch_rhs 10: 6 + 8 > 10, so the second request waits; the third (4) still fits
    g = bd.form_batch([0, 0, 0], [6, 8, 4], [1.0], max_batch_rhs=10)
    assert g == [0, -1, 0]
    # the first request always opens the group, even above the cap
    g = bd.form_batch([0, 0], [20, 1], [1.0], max_batch_rhs=10)
    assert g == [0, -1]


def test_backlog_mixes_smaller_operators_only(bd):
    # max_inflight 1 x max_batch_ops 4 = 4 < 6 queued: backlog; 1 free slot takes both
    # operators if the second's traffic is within 25 % of the first's
    small_first = bd.form_batch([0, 0, 0, 1, 1, 1], [2] * 6, [1.0, 100.0], free_slots=1, max_inflight=1)
    assert small_first == [0, 0, 0, -1, -1, -1]
    big_first = bd.form_batch([1, 1, 1, 0, 0, 0], [2] * 6, [1.0, 100.0], free_slots=1, max_inflight=1)
    assert big_first == [0, 0, 0, 1, 1, 1]
    # a ratio limit of 100000 % admits any operator
    g = bd.form_batch([0, 0, 0, 1, 1, 1], [2] * 6, [1.0, 100.0], free_slots=1, max_inflight=1,
                      mix_work_pct=100000)
    assert g == [0, 0, 0, 1, 1, 1]


def test_operators_spread_over_the_free_slots(bd):
    # backlog with 6 operators (equal traffic) and 2 free slots: 3 operators in this batch
    ops = [0, 1, 2, 3, 4, 5] * 2
    g = bd.form_batch(ops, [1] * 12, [1.0] * 6, free_slots=2, max_inflight=2, max_batch_ops=4,
                      mix_work_pct=100)
    assert sorted(set(x for x in g if x >= 0)) == [0, 1, 2]
    assert g[:3] == [0, 1, 2] and g[3:6] == [-1, -1, -1] and g[6:9] == [0, 1, 2]
    # with 1 free slot the cap is max_batch_ops
    g = bd.form_batch(ops, [1] * 12, [1.0] * 6, free_slots=1, max_inflight=2, max_batch_ops=4, mix_work_pct=100)
    assert sorted(set(x for x in g if x >= 0)) == [0, 1, 2, 3]


def test_a_passed_operator_does_not_block_later_ones(bd):
    # backlog; operator 1 is too heavy for operator 0's batch, operator 2 is light and joins
    ops = [0, 1, 2, 0, 1, 2]
    g = bd.form_batch(ops, [2] * 6, [10.0, 1000.0, 1.0], free_slots=1, max_inflight=1)
    assert g == [0, -1, 1, 0, -1, 1]


def test_invalid_arguments(bd):
    with pytest.raises(bd.MbfError):
        bd.form_batch([0, 2], [1, 1], [1.0, 1.0])          # operator index out of range
    with pytest.raises(bd.MbfError):
        bd.form_batch([0], [0], [1.0])                     # nrhs <= 0
    with pytest.raises(bd.MbfError):
        bd.form_batch([0], [1], [1.0], free_slots=0)
    with pytest.raises(bd.MbfError):
        bd.form_batch([0], [1], [1.0], max_batch_ops=9)    # more than 8 operators per batch
    assert bd.form_batch([], [], [1.0]) == []


def test_sm_share_split_by_traffic(bd):
    # proportional shares, the rounding remainder to the group of most work
    assert bd.split_sms([3.0, 1.0], 152) == [114, 38]
    assert bd.split_sms([1.0, 1.0, 1.0], 152) == [52, 50, 50]        # 50 each + 2 to the first
    assert bd.split_sms([1.0, 5.0, 1.0], 100) == [14, 72, 14]
    # one group keeps the share; every group gets at least one SM
    assert bd.split_sms([7.0], 40) == [40]
    g = bd.split_sms([1e-9, 1.0, 1.0], 10)
    assert g[0] == 1 and sum(g) == 10
    for work, share in (([2.0, 3.0, 5.0, 7.0], 152), ([1.0] * 8, 152), ([1.0, 1e6], 152), ([4.0, 4.0], 3)):
        g = bd.split_sms(work, share)
        assert sum(g) == share and min(g) >= 1, (work, share, g)
    # fewer SMs than groups: one each (the groups share SMs)
    assert bd.split_sms([1.0, 2.0, 3.0], 2) == [1, 1, 1]
    assert bd.split_sms([], 10) == []
    for work, share in (([1.0, 0.0], 10), ([1.0, -1.0], 10), ([1.0, float("nan")], 10), ([1.0], 0)):
        with pytest.raises(bd.MbfError):
            bd.split_sms(work, share)
