"""Explicit non-uniform point sets (§2.6: trees built adaptively over arbitrary X and
Omega, empty nodes kept as zero-point nodes): the library's trees equal the oracle's,
its factorization is exact when the rank covers every block, and its error against the
direct sum matches the oracle's own construction on the same points."""
import numpy as np
import pytest

from oracle import bf as B
from oracle import direct as D
from oracle import problem as P

from gpu_util import export_factors


@pytest.fixture(scope="module")
def bd():
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


def clustered_points(nx, nw, lo, side, seed):
    """X: half in a Gaussian blob, half uniform, in [0,1)^2; Omega: half concentrated
    near the origin, half uniform, in [lo, lo + side)^2 -- ragged trees at every level."""
    rng = np.random.default_rng(seed)
    X = np.mod(np.concatenate([rng.normal(0.3, 0.08, (nx // 2, 2)), rng.random((nx - nx // 2, 2))]), 1.0)
    W = np.concatenate([rng.normal(lo + side / 2, side / 10, (nw // 2, 2)),
                        rng.uniform(lo, lo + side, (nw - nw // 2, 2))])
    W = np.clip(W, lo, lo + side * (1 - 1e-9))
    return X, W


def test_explicit_point_trees_match_oracle(bd):
    X, W = clustered_points(1500, 1200, -16.0, 32.0, seed=1)
    a = bd.HostFactors.build(2, 32, 4, 8, tree=bd.MBF_TREE_POINTS, kernel="dft", x_pts=X, w_pts=W,
                             w_lo=-16.0, w_side=32.0).arrays()
    xt, wt = P.unit_cube_tree(X, 4), P.unit_cube_tree((W + 16.0) / 32.0, 4)
    assert a["n_out"] == 1500 and a["n_in"] == 1200
    assert np.array_equal(xt.perm, a["x_perm"]) and np.array_equal(xt.off, a["x_off"])
    assert np.array_equal(wt.perm, a["w_perm"]) and np.array_equal(wt.off, a["w_off"])
    assert (np.diff(a["x_off"]) == 0).any() and (np.diff(a["w_off"]) == 0).any()   # empty leaves


def test_explicit_points_exact_at_full_rank(bd):
    """r at least every block dimension: the factors reproduce K to the builder's
    resolution (§2.4, exact truncations; its Gram eigensolver resolves singular values
    down to about 3e-7 sigma_1), here for the FIO kernel on ragged sets."""
    X, W = clustered_points(160, 140, -8.0, 16.0, seed=2)
    a = bd.HostFactors.build(2, 16, 2, 64, tree=bd.MBF_TREE_POINTS, kernel="fio_iso", x_pts=X, w_pts=W,
                             w_lo=-8.0, w_side=16.0).arrays()
    Kf = B.SparseBF(export_factors(a)).dense()
    K = P.kernel_fio_iso(X[:, None, :], W[None, :, :])
    assert np.abs(Kf - K).max() < 1e-5


def test_explicit_points_error_matches_oracle_construction(bd):
    X, W = clustered_points(1200, 1000, -8.0, 16.0, seed=3)
    a = bd.HostFactors.build(2, 16, 4, 12, tree=bd.MBF_TREE_POINTS, kernel="dft", x_pts=X, w_pts=W,
                             w_lo=-8.0, w_side=16.0).arrays()
    rng = np.random.default_rng(4)
    g = (rng.standard_normal((2, W.shape[0])) + 1j * rng.standard_normal((2, W.shape[0]))) / np.sqrt(2)
    ud = D.direct_sum(P.kernel_dft, X, W, g)
    e_lib = D.rel_err(B.SparseBF(export_factors(a)).apply(g), ud)
    fo = B.build(P.kernel_dft, X, W, P.unit_cube_tree(X, 4), P.unit_cube_tree((W + 8.0) / 16.0, 4), 12)
    e_orc = D.rel_err(B.SparseBF(fo).apply(g), ud)
    assert e_lib < 0.1 and 0.5 < e_lib / e_orc < 2.0, (e_lib, e_orc)


def test_explicit_points_are_validated(bd):
    X, W = clustered_points(100, 100, -8.0, 16.0, seed=5)
    for x, w in ((X + 1.0, W), (X, W + 100.0)):
        with pytest.raises(bd.MbfError) as e:
            bd.HostFactors.build(2, 16, 2, 8, tree=bd.MBF_TREE_POINTS, kernel="dft", x_pts=x, w_pts=w,
                                 w_lo=-8.0, w_side=16.0)
        assert e.value.code == bd.MBF_ERR_INVALID
