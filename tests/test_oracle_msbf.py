"""Pins of the oracle's multiscale butterfly factorization (§4, eqs. domaindecomp,
msumd, f1): exact at full rank, the centre-only special case is the dense kernel,
the coronas and the centre partition Omega, the adjoint identity, and the error
against the Eckart-Young floor of the coronas' middle levels (with the paper's Table 4
beside it)."""
import os

import numpy as np
import pytest

from mbf_synth import complex_normal, sample_outputs
from oracle import direct as D
from oracle import msbf as MS
from oracle import problem as P

from floor_util import floor_from_tails, middle_level_tails

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_corona_parts_and_centre_partition_omega():
    n = 32
    coronas, centre = MS.corona_sets(n, 8)
    allidx = np.concatenate([idx for _, idx in coronas] + [centre])
    assert np.array_equal(np.sort(allidx), np.arange(n * n))
    # centre = max|xi_k| <= 4: a 9 x 9 block
    assert centre.size == 81
    # every corona lies in its square [-n/2^(t+1), n/2^(t+1)]^2 and outside the next one
    W = P.grid_omega(n, 2)
    for t, idx in coronas:
        m = np.max(np.abs(W[idx]), axis=1)
        assert np.all(m <= n / 2 ** (t + 1)) and np.all(m > n / 2 ** (t + 2))


def test_msbf_exact_at_full_rank():
    """With the rank at least every block dimension each BF_t reproduces its kernel
    block, so eq. (f1) equals the direct sum."""
    n = 16
    m = MS.build(P.kernel_fio_iso, n, r=64, n_center=4)
    assert [t for t, _, _, _ in m.parts] == [0, 1] and [Lt for _, Lt, _, _ in m.parts] == [4, 2]
    assert m.center.size == 25
    g = complex_normal(n * n, 2, seed=3)
    u = MS.SparseMsBF(m).apply(g)
    ud = D.direct_sum(P.kernel_fio_iso, P.grid_x(n, 2), P.grid_omega(n, 2), g)
    assert D.rel_err(u, ud) < 1e-10


def test_centre_only_is_the_dense_kernel():
    """A centre covering Omega leaves no corona: K_C R_C is all of K (eq. msumd)."""
    n = 8
    m = MS.build(P.kernel_fio_iso, n, r=4, n_center=4 * n)
    assert m.parts == [] and m.center.size == n * n
    g = complex_normal(n * n, 1, seed=1)
    ud = D.direct_sum(P.kernel_fio_iso, P.grid_x(n, 2), P.grid_omega(n, 2), g)
    assert D.rel_err(MS.SparseMsBF(m).apply(g), ud) < 1e-13


def test_msbf_adjoint_identity():
    n = 32
    m = MS.build(P.kernel_fio_iso, n, r=8, n_center=8)
    sm = MS.SparseMsBF(m)
    g = complex_normal(n * n, 1, seed=4)
    h = complex_normal(n * n, 1, seed=5)
    lhs = np.vdot(h, sm.apply(g))
    rhs = np.vdot(sm.adjoint(h), g)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_msbf_error_decreases_with_rank():
    n = 32
    g = complex_normal(n * n, 1, seed=0)
    ud = D.direct_sum(P.kernel_fio_iso, P.grid_x(n, 2), P.grid_omega(n, 2), g)
    errs = [D.rel_err(MS.SparseMsBF(MS.build(P.kernel_fio_iso, n, r=r, n_center=8)).apply(g), ud)
            for r in (4, 8, 16)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.1


@pytest.mark.slow
def test_msbf_error_against_table_4():
    """§4.3, Table 4: MBF-s on the Example-1 FIO (elliptic phase) at n = 64 with a 16 x 16
    centre.

    1. Against the mathematics: the error lies between 0.8x and 4x the Eckart-Young floor
       summed over the middle levels of every corona's factorization (the centre is exact).
    2. Against the paper: at r = 20 the printed error is within 2x of that floor; at r = 12
       it is 2-3x below it, a level no rank-r factorization on these trees reaches for iid
       g (the paper does not state its input), so the comparison with the printed value
       is loose there."""
    tab = np.loadtxt(os.path.join(GOLDEN, "table4_mbf_s.txt"))
    n, L = 64, 6
    S = sample_outputs(n * n, 256, seed=1)
    g = complex_normal(n * n, 1, seed=0)
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    u = D.direct_sum(P.kernel_fio_ellip, X, W, g, rows=S)
    coronas, _ = MS.corona_sets(n, 16)
    tails = {12: 0.0, 20: 0.0}
    for t, idx in coronas:
        Lt = 2 * ((L - t) // 2)
        half = n / 2 ** (t + 1)
        part = middle_level_tails(P.kernel_fio_ellip, X, W, P.uniform_tree(n, 2, Lt),
                                  P.square_tree(W[idx], idx, -half, 2 * half, Lt), (12, 20))
        for r in tails:
            tails[r] += part[r]
    floor = floor_from_tails(tails, n * n, n * n)
    errs = {}
    for r in (12, 20):
        m = MS.build(P.kernel_fio_ellip, n, r=r, n_center=16)
        errs[r] = D.rel_err(MS.SparseMsBF(m).apply(g)[:, S], u)
        assert 0.8 * floor[r] < errs[r] < 4 * floor[r], (r, errs[r], floor[r])
        paper = tab[(tab[:, 0] == n) & (tab[:, 1] == r), 2][0]
        assert floor[r] / 4 < paper < 2 * floor[r], (r, paper, floor[r])
    assert errs[20] < errs[12]
