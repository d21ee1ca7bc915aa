"""Kernels, point sets and hierarchical trees (oracle; test infrastructure only).

Point sets follow §1.1, eqs. (X) and (Omega): X = {(n_1/n, ..., n_d/n)}, Omega =
{(n_1, ..., n_d) : -n/2 <= n_k < n/2}.  Natural (ABI) order is row-major:
x index = sum_k n_k n^(d-1-k); xi index = sum_k (xi_k + n/2) n^(d-1-k).

Trees follow §2.2 and Fig. 1: complete 2^d-ary trees over the unit square/cube,
nodes at each level numbered along the Z-order (Morton) curve, children of node
i numbered c*i + t.  In Fig. 1 the first coordinate x_1 runs downwards and x_2
to the right, and child t = 0, 1, 2, 3 is (x_1 low, x_2 low), (low, high),
(high, low), (high, high): so the first coordinate supplies the most
significant bit of t.  Points inside a leaf are kept in natural order.
Non-uniform point sets (the polar set P, the coronas of §4) use the same cells;
a node with no point is an empty range (§2.6).
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# point sets (§1.1)
# ----------------------------------------------------------------------------


def grid_x(n: int, d: int) -> np.ndarray:
    """X of eq. (X): [N, d] array of (n_1/n, ..., n_d/n) in natural row-major order."""
    idx = np.indices((n,) * d).reshape(d, -1).T
    return idx.astype(np.float64) / n


def grid_omega(n: int, d: int) -> np.ndarray:
    """Omega of eq. (Omega): [N, d] integer frequencies -n/2..n/2-1, natural order."""
    idx = np.indices((n,) * d).reshape(d, -1).T
    return (idx - n // 2).astype(np.float64)


# ----------------------------------------------------------------------------
# kernels
# ----------------------------------------------------------------------------


def kernel_dft(x: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """DFT kernel exp(-2 pi i x.xi) with x in [0,1)^d (§1.1: the multidimensional
    Fourier transform is the model complementary low-rank matrix).  With x = m/n
    for integer m this is exp(-2 pi i m.xi / n)."""
    return np.exp(-2j * np.pi * np.sum(x * xi, axis=-1))


def fio_iso_phase(x: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Phi(x, xi) = x.xi + c(x)|xi|, c(x) = (2 + sin 2pi x_1 sin 2pi x_2)/16.

    The isotropic special case c_1 = c_2 = c of the Example-1 phase (§3.3, eq.
    example1phi); homogeneous of degree 1 in xi as §3.1 requires."""
    c = (2.0 + np.sin(2 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1])) / 16.0
    return np.sum(x * xi, axis=-1) + c * np.sqrt(np.sum(xi * xi, axis=-1))


def fio_ellip_phase(x: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Example 1 (§3.3, eq. example1phi): Phi = x.xi + sqrt(c_1^2 xi_1^2 + c_2^2 xi_2^2),
    c_1 = (2 + sin 2pi x_1 sin 2pi x_2)/16, c_2 = (2 + cos 2pi x_1 cos 2pi x_2)/16."""
    s1, s2 = np.sin(2 * np.pi * x[..., 0]), np.sin(2 * np.pi * x[..., 1])
    k1, k2 = np.cos(2 * np.pi * x[..., 0]), np.cos(2 * np.pi * x[..., 1])
    c1 = (2.0 + s1 * s2) / 16.0
    c2 = (2.0 + k1 * k2) / 16.0
    return np.sum(x * xi, axis=-1) + np.sqrt(c1 ** 2 * xi[..., 0] ** 2 + c2 ** 2 * xi[..., 1] ** 2)


def kernel_fio_iso(x, xi):
    """K = exp(2 pi i Phi) for the isotropic phase (§3.1, eq. fio)."""
    return np.exp(2j * np.pi * fio_iso_phase(x, xi))


def kernel_fio_ellip(x, xi):
    """K = exp(2 pi i Phi) for the Example-1 phase (§3.3, eq. example1fio)."""
    return np.exp(2j * np.pi * fio_ellip_phase(x, xi))


KERNELS = {"dft": kernel_dft, "fio_iso": kernel_fio_iso, "fio_ellip": kernel_fio_ellip}


def kernel_block(kernel, X: np.ndarray, W: np.ndarray, rows, cols) -> np.ndarray:
    """Dense submatrix (K(x_a, xi_b)) for a in rows, b in cols (§2.2, K^l_{i,j})."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    return kernel(X[rows][:, None, :], W[cols][None, :, :])


# ----------------------------------------------------------------------------
# polar map (§3.1, eq. polar) and corona split (§4.1, eq. domaindecomp)
# ----------------------------------------------------------------------------


def polar_coords(xi: np.ndarray, n: int) -> np.ndarray:
    """Invert eq. (polar), xi = (sqrt(2)/2) n p_1 (cos 2pi p_2, sin 2pi p_2):
    p_1 = sqrt(2)|xi|/n in [0,1], p_2 = atan2(xi_2, xi_1)/(2 pi) mod 1; xi = 0 -> (0, 0)."""
    p1 = np.minimum(np.sqrt(2.0) * np.sqrt(np.sum(xi * xi, axis=-1)) / n, 1.0)
    p2 = np.mod(np.arctan2(xi[..., 1], xi[..., 0]) / (2 * np.pi), 1.0)
    p2 = np.where(p2 >= 1.0, 0.0, p2)
    return np.stack([p1, p2], axis=-1)


def corona_index(xi: np.ndarray, n: int, n_center: int) -> np.ndarray:
    """Index t of the corona Omega_t containing xi (eq. domaindecomp):
    n/2^(t+2) < max_k |xi_k| <= n/2^(t+1); -1 for the centre Omega_C.  Coronas are
    kept for t = 0 .. T-1 where T is the count with n/2^(t+2) >= n_center/2;
    all remaining points form Omega_C."""
    m = np.max(np.abs(xi), axis=-1)
    L = int(round(np.log2(n)))
    t = np.full(m.shape, -1, dtype=np.int64)
    for tt in range(L):
        lo, hi = n / 2 ** (tt + 2), n / 2 ** (tt + 1)
        if lo < n_center / 2:
            break
        sel = (m > lo) & (m <= hi)
        t[sel] = tt
    # the face xi_k = -n/2 has |xi_k| = n/2 = n/2^(0+1): inside Omega_0 by the inequality
    return t


# ----------------------------------------------------------------------------
# Z-order trees (§2.2, Fig. 1; non-uniform sets §2.6)
# ----------------------------------------------------------------------------


def morton_leaf(cells: np.ndarray, L: int) -> np.ndarray:
    """Z-order index at level L of integer cell coordinates cells[:, k] in [0, 2^L).

    Digit at each level = sum_k bit(cell_k) 2^(d-1-k): the first coordinate is the
    most significant, matching Fig. 1 (t = 2 bit(x_1) + bit(x_2) in 2-D)."""
    d = cells.shape[1]
    c = 2 ** d
    m = np.zeros(cells.shape[0], dtype=np.int64)
    for b in range(L - 1, -1, -1):
        digit = np.zeros(cells.shape[0], dtype=np.int64)
        for k in range(d):
            digit |= ((cells[:, k] >> b) & 1) << (d - 1 - k)
        m = m * c + digit
    return m


class Tree:
    """Z-order tree of depth L over a point set, stored as a permutation of the
    points (tree order -> natural index) plus leaf offsets.

    Node i at level l owns the leaves [i c^(L-l), (i+1) c^(L-l)) and hence the
    contiguous tree-order range [off[i c^(L-l)], off[(i+1) c^(L-l)])."""

    def __init__(self, leaf_of_point: np.ndarray, d: int, L: int, points_index=None):
        self.d, self.L, self.c = d, L, 2 ** d
        n_leaves = self.c ** L
        natural = (np.arange(leaf_of_point.shape[0], dtype=np.int64)
                   if points_index is None else np.asarray(points_index, dtype=np.int64))
        order = np.lexsort((natural, leaf_of_point))
        self.perm = natural[order]
        counts = np.bincount(leaf_of_point, minlength=n_leaves)
        self.off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)

    def node_range(self, level: int, i: int):
        span = self.c ** (self.L - level)
        return int(self.off[i * span]), int(self.off[(i + 1) * span])

    def node_points(self, level: int, i: int) -> np.ndarray:
        a, b = self.node_range(level, i)
        return self.perm[a:b]

    def leaf_sizes(self) -> np.ndarray:
        return np.diff(self.off)


def uniform_tree(n: int, d: int, L: int) -> Tree:
    """Complete tree of depth L over the n^d grid (X of eq. X, or Omega shifted by n/2)."""
    shift = int(round(np.log2(n))) - L
    if shift < 0:
        raise ValueError("depth L exceeds log2(n)")
    idx = np.indices((n,) * d).reshape(d, -1).T
    cells = idx >> shift
    return Tree(morton_leaf(cells, L), d, L)


def unit_cube_tree(p: np.ndarray, L: int, points_index=None) -> Tree:
    """Tree of depth L over points p in [0,1]^d: cell = floor(p 2^L), the closed
    upper face p_k = 1 assigned to the last cell."""
    d = p.shape[1]
    cells = np.minimum(np.floor(p * 2 ** L).astype(np.int64), 2 ** L - 1)
    cells = np.maximum(cells, 0)
    return Tree(morton_leaf(cells, L), d, L, points_index)


def polar_tree(n: int, L: int) -> Tree:
    """Tree T_P over the polar image P of Omega (§3.1-3.2): Omega points keep their
    natural index; their cells are taken in the p = (p_1, p_2) coordinates."""
    W = grid_omega(n, 2)
    return unit_cube_tree(polar_coords(W, n), L)


def square_tree(xi: np.ndarray, points_index: np.ndarray, lo: float, side: float, L: int) -> Tree:
    """Tree of depth L over the square [lo, lo+side)^d holding the points xi (used for
    the smallest square containing a corona, §4.2)."""
    p = (xi - lo) / side
    return unit_cube_tree(p, L, points_index)
