"""Pins for the oracle's kernels, point sets, trees, direct sum and error metric."""
import math
import os

import numpy as np
import pytest

from mbf_synth import complex_normal, sample_outputs
from oracle import direct as D
from oracle import problem as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- direct sum


@pytest.mark.parametrize("n,d", [(32, 2), (8, 3), (16, 2)])
def test_direct_sum_equals_closed_form_dft(n, d):
    """The direct sum of the DFT kernel is the separable FFT after the shift xi -> xi + n/2."""
    X, W = P.grid_x(n, d), P.grid_omega(n, d)
    g = complex_normal(n ** d, 2, seed=3)
    u = D.direct_sum(P.kernel_dft, X, W, g)
    ref = D.dft_closed_form(g, n, d)
    assert np.abs(u - ref).max() / np.abs(ref).max() < 1e-12


def test_direct_sum_sampled_rows_match_full():
    n = 16
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    g = complex_normal(n * n, 1, seed=0)
    S = sample_outputs(n * n, 40, seed=1)
    full = D.direct_sum(P.kernel_fio_iso, X, W, g)
    part = D.direct_sum(P.kernel_fio_iso, X, W, g, rows=S)
    assert np.abs(full[:, S] - part).max() < 1e-12


def test_direct_sum_brute_force_loops():
    """Tiny case: every term summed in a pure-Python double loop with cmath."""
    import cmath
    n = 4
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    g = complex_normal(n * n, 1, seed=9)[0]
    u = D.direct_sum(P.kernel_fio_ellip, X, W, g)[0]
    for a in range(n * n):
        acc = 0j
        for b in range(n * n):
            acc += cmath.exp(2j * math.pi * float(P.fio_ellip_phase(X[a], W[b]))) * g[b]
        assert abs(acc - u[a]) < 1e-12


# ---------------------------------------------------------------- kernels


@pytest.mark.parametrize("phase", [P.fio_iso_phase, P.fio_ellip_phase])
def test_phase_homogeneous_degree_one(phase):
    """§3.1: Phi(x, lambda xi) = lambda Phi(x, xi) for lambda > 0."""
    rng = np.random.default_rng(0)
    x = rng.random((50, 2))
    xi = rng.standard_normal((50, 2)) * 20
    for lam in (0.5, 3.0, 17.0):
        assert np.allclose(phase(x, lam * xi), lam * phase(x, xi), rtol=1e-13, atol=1e-11)


def test_phase_special_points():
    """Values the Example-1 formulas fix at special x (§3.3, eq. example1phi):
    at x = 0, c_1 = 2/16 and c_2 = 3/16; at x = (1/4, 1/4), c_1 = 3/16, c_2 = 2/16;
    the isotropic phase has c = 2/16 whenever x_1 = 0."""
    xi = np.array([[3.0, -4.0], [7.0, 0.0], [0.0, -9.0]])
    x0 = np.zeros((3, 2))
    expect0 = np.sqrt((2 / 16) ** 2 * xi[:, 0] ** 2 + (3 / 16) ** 2 * xi[:, 1] ** 2)
    assert np.allclose(P.fio_ellip_phase(x0, xi), expect0, atol=1e-14)
    xq = np.full((3, 2), 0.25)
    expectq = xq @ np.array([1.0, 1.0]) * 0 + np.sum(xq * xi, axis=1) + np.sqrt(
        (3 / 16) ** 2 * xi[:, 0] ** 2 + (2 / 16) ** 2 * xi[:, 1] ** 2)
    assert np.allclose(P.fio_ellip_phase(xq, xi), expectq, atol=1e-13)
    x1 = np.array([[0.0, 0.3], [0.0, 0.7], [0.0, 0.1]])
    assert np.allclose(P.fio_iso_phase(x1, xi) - np.sum(x1 * xi, axis=1),
                       (2 / 16) * np.hypot(xi[:, 0], xi[:, 1]), atol=1e-13)


def test_iso_phase_off_the_axes():
    """The isotropic phase x.xi + c(x)|xi| with c = (2 + sin 2pi x_1 sin 2pi x_2)/16
    (Example 1 of §3.3 with c_1 = c_2) at points where neither sine vanishes:
    c(1/4, 1/4) = 3/16, c(1/4, 3/4) = c(3/4, 1/4) = 1/16, c(1/12, 1/4) = 5/32,
    c(1/4, 1/12) = 5/32, c(1/8, 1/8) = (2 + 1/2)/16.  A cosine in place of either
    sine, a dropped 2pi, a wrong sign or a missing x.xi term fails at least one."""
    pts = np.array([[0.25, 0.25], [0.25, 0.75], [0.75, 0.25], [1 / 12, 0.25], [0.25, 1 / 12],
                    [0.125, 0.125]])
    c = np.array([3 / 16, 1 / 16, 1 / 16, 5 / 32, 5 / 32, 2.5 / 16])
    xi = np.array([[3.0, -4.0], [-12.0, 5.0], [8.0, 6.0], [0.0, 7.0], [-24.0, 0.0], [1.0, 1.0]])
    expect = np.sum(pts * xi, axis=1) + c * np.hypot(xi[:, 0], xi[:, 1])
    assert np.allclose(P.fio_iso_phase(pts, xi), expect, atol=1e-13)
    # the kernel is exp(+2 pi i Phi): at x = (1/4, 1/4), xi = (3, -4) the phase is
    # -1/4 + 15/16 = 11/16
    k = P.kernel_fio_iso(pts[:1], xi[:1])[0]
    assert abs(k - np.exp(2j * np.pi * 11 / 16)) < 1e-13


def test_polar_map_inverts_eq_polar():
    """p(xi) followed by eq. (polar) returns xi; p lies in [0,1]^2 and p_1 = 1 only at
    the corner xi = (-n/2, -n/2) (reading of the closed upper cell)."""
    n = 64
    W = P.grid_omega(n, 2)
    p = P.polar_coords(W, n)
    xi = (np.sqrt(2) / 2) * n * p[:, :1] * np.stack(
        [np.cos(2 * np.pi * p[:, 1]), np.sin(2 * np.pi * p[:, 1])], axis=1)
    assert np.abs(xi - W).max() < 1e-10
    assert p.min() >= 0 and p[:, 0].max() <= 1.0 and p[:, 1].max() < 1.0
    top = np.nonzero(np.isclose(p[:, 0], 1.0))[0]
    assert top.tolist() == [0] and W[0].tolist() == [-n / 2, -n / 2]


def test_polar_kernel_rewrite():
    """eq. (polarsum): e^{2 pi i n Psi(x, p)} with Psi = (sqrt2/2) Phi(x, (cos, sin)) p_1
    reproduces K(x, xi) at every grid point (homogeneity, §3.1)."""
    n = 32
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    p = P.polar_coords(W, n)
    rng = np.random.default_rng(4)
    a = rng.integers(0, n * n, 300)
    b = rng.integers(0, n * n, 300)
    direction = np.stack([np.cos(2 * np.pi * p[b, 1]), np.sin(2 * np.pi * p[b, 1])], axis=1)
    psi = (np.sqrt(2) / 2) * P.fio_iso_phase(X[a], direction) * p[b, 0]
    assert np.allclose(np.exp(2j * np.pi * n * psi), P.kernel_fio_iso(X[a], W[b]), atol=1e-9)


# ---------------------------------------------------------------- trees


def test_zorder_matches_figure_1():
    """Level-2 Z-order numbering read off Fig. 1 (golden fixture)."""
    fig = _load("fig1_zorder_level2.txt").astype(np.int64)
    cells = fig[:, 1:3]
    assert P.morton_leaf(cells, 2).tolist() == fig[:, 0].tolist()
    # children of node i are 4i + t with t = 2 bit(x_1) + bit(x_2) (Fig. 1, middle panel)
    lvl1 = P.morton_leaf(cells >> 1, 1)
    assert (fig[:, 0] // 4).tolist() == lvl1.tolist()


@pytest.mark.parametrize("maker", [
    lambda: P.uniform_tree(16, 2, 4), lambda: P.uniform_tree(64, 2, 4),
    lambda: P.polar_tree(64, 4), lambda: P.uniform_tree(8, 3, 2), lambda: P.polar_tree(32, 5)])
def test_tree_invariants(maker):
    t = maker()
    N = t.perm.shape[0]
    assert np.array_equal(np.sort(t.perm), np.arange(N))
    assert t.off[0] == 0 and t.off[-1] == N and np.all(np.diff(t.off) >= 0)
    # node ranges nest: children partition the parent's range in order
    for level in range(t.L):
        for i in range(t.c ** level):
            a, b = t.node_range(level, i)
            ca, _ = t.node_range(level + 1, t.c * i)
            _, cb = t.node_range(level + 1, t.c * i + t.c - 1)
            assert (a, b) == (ca, cb)


def test_uniform_leaf_holds_its_cell():
    n, L = 64, 4
    t = P.uniform_tree(n, 2, L)
    X = P.grid_x(n, 2)
    side = 2.0 ** -L
    for leaf in (0, 1, 2, 77, 255):
        pts = X[t.node_points(L, leaf)]
        assert pts.shape[0] == (n >> L) ** 2
        # all points of a leaf share one cell
        cell = np.floor(pts / side).astype(int)
        assert np.all(cell == cell[0])
        assert P.morton_leaf(cell[:1], L)[0] == leaf


def test_rel_err_definition():
    u = complex_normal(100, 2, seed=0)
    assert abs(D.rel_err(0.9 * u, u) - 0.1) < 1e-14
    assert D.rel_err(u, u) == 0.0


def test_corona_split_partitions_omega():
    """eq. (domaindecomp): coronas and centre partition Omega; for n=512 and a 16x16
    centre, t = 0..4 and the centre is max|xi_k| <= 8 (17 x 17 points)."""
    n = 512
    W = P.grid_omega(n, 2)
    t = P.corona_index(W, n, 16)
    assert set(np.unique(t).tolist()) == {-1, 0, 1, 2, 3, 4}
    m = np.abs(W).max(axis=1)
    assert np.array_equal(t == -1, m <= 8)
    assert np.count_nonzero(t == -1) == 17 * 17
    for tt in range(5):
        sel = t == tt
        assert np.all(m[sel] > n / 2 ** (tt + 2)) and np.all(m[sel] <= n / 2 ** (tt + 1))
