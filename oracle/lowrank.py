"""Low-rank primitives of §2.1 (oracle; test infrastructure only).

* `truncated_svd`  -- Z ~ U_0 Sigma_0 V_0^* (eq. Z), keeping the r largest singular
  values, and no singular value below `tol * sigma_1`.
* `forms`          -- the three factorizations of eqs. (lowrank1)-(lowrank3).
* `svd_sampling`   -- SVD via random sampling (the second procedure of §2.1).
* `svd_matvec`     -- SVD via random matrix-vector multiplication (the first).

Readings where §2.1 leaves a constant open: the sample sets I_row, I_col and the
random supplements have size `factor * r` (capped by the matrix size), the
representative-set iteration stops when both sets repeat or after `max_rounds`
rounds, and the oversampling constant of the matvec procedure defaults to 8.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

TOL = 1e-14


def truncated_svd(Z: np.ndarray, r: int, tol: float = TOL):
    """Rank-r truncated SVD of Z (eq. Z): returns U_0 (m x k), sigma (k), V_0 (n x k)
    with k = min(r, m, n, #{sigma > tol sigma_1})."""
    m, n = Z.shape
    if m == 0 or n == 0 or r == 0:
        return (np.zeros((m, 0), complex), np.zeros(0), np.zeros((n, 0), complex))
    U, s, Vh = np.linalg.svd(Z, full_matrices=False)
    k = int(min(r, np.count_nonzero(s > tol * s[0]))) if s[0] > 0 else 0
    return U[:, :k], s[:k], Vh[:k].conj().T


def forms(U0, s, V0, which: int):
    """The three low-rank forms of §2.1.

    which=1 (eq. lowrank1): Z ~ U S V^*, U = U_0 Sigma_0, S = Sigma_0^{-1}, V^* = Sigma_0 V_0^*
    which=2 (eq. lowrank2): Z ~ U V^*, U = U_0 Sigma_0, V^* = V_0^*
    which=3 (eq. lowrank3): Z ~ U V^*, U = U_0,         V^* = Sigma_0 V_0^*
    Returns (U, S, V) with S None for forms 2 and 3 (V, not V^*, is returned)."""
    if which == 1:
        return U0 * s, 1.0 / s, V0 * s
    if which == 2:
        return U0 * s, None, V0
    if which == 3:
        return U0, None, V0 * s
    raise ValueError(which)


def _pivoted_cols(A: np.ndarray, k: int) -> np.ndarray:
    """First k pivots of a column-pivoted QR of A (the "pivoted QR" of §2.1)."""
    if A.shape[1] == 0 or A.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    _, _, piv = sla.qr(A, mode="economic", pivoting=True)
    return np.asarray(piv[:min(k, A.shape[1], A.shape[0])], dtype=np.int64)


def _orth(A: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the columns of A from a pivoted QR (§2.1 second step)."""
    Q, R, _ = sla.qr(A, mode="economic", pivoting=True)
    if R.size == 0:
        return Q[:, :0]
    d = np.abs(np.diag(R))
    k = int(np.count_nonzero(d > TOL * d[0])) if d[0] > 0 else 0
    return Q[:, :k]


def _supplement(fixed: np.ndarray, total: int, size: int, rng) -> np.ndarray:
    """fixed indices plus random others, `size` in all (capped at `total`), sorted."""
    size = min(size, total)
    fixed = np.unique(fixed)
    need = size - fixed.shape[0]
    if need <= 0:
        return fixed
    pool = np.setdiff1d(np.arange(total), fixed, assume_unique=True)
    extra = rng.choice(pool, size=min(need, pool.shape[0]), replace=False)
    return np.sort(np.concatenate([fixed, extra]))


def svd_sampling(entries, m: int, n: int, r: int, rng, factor: int = 3, max_rounds: int = 3,
                 tol: float = TOL):
    """Approximate rank-r SVD from entry evaluation: SVD via random sampling, §2.1.

    `entries(rows, cols)` returns the dense submatrix Z[rows][:, cols].
      1. Representative columns and rows are discovered alternately: a pivoted QR
         of Z(I, :) over the current rows I picks columns, a pivoted QR of
         Z(:, J)^* over the current columns J picks rows; each new set is joined
         with random indices to form the next sample; stop when both sets repeat.
      2. Q_col, Q_row: orthonormal bases from pivoted QRs of Z(:, cols_rep) and
         Z(rows_rep, :)^*.
      3. M = Q_col(I_row,:)^+ Z(I_row, I_col) (Q_row(I_col,:)^*)^+ on random sets
         I_row, I_col containing the representatives.
      4. SVD of M gives Z ~ (Q_col U_M) Sigma_M (Q_row V_M)^*.
    When a sample would cover the whole matrix the exact truncated SVD is used.
    Returns (U_0, sigma, V_0)."""
    if m == 0 or n == 0 or r == 0:
        return truncated_svd(np.zeros((m, n), complex), r, tol)
    s = factor * r
    if s >= m or s >= n:
        return truncated_svd(entries(np.arange(m), np.arange(n)), r, tol)
    rows_rep = np.zeros(0, dtype=np.int64)
    cols_rep = np.zeros(0, dtype=np.int64)
    for _ in range(max_rounds):
        I = _supplement(rows_rep, m, s, rng)
        new_cols = np.sort(_pivoted_cols(entries(I, np.arange(n)), r))
        J = _supplement(new_cols, n, s, rng)
        new_rows = np.sort(_pivoted_cols(entries(np.arange(m), J).conj().T, r))
        stable = np.array_equal(new_rows, rows_rep) and np.array_equal(new_cols, cols_rep)
        rows_rep, cols_rep = new_rows, new_cols
        if stable:
            break
    Q_col = _orth(entries(np.arange(m), cols_rep))
    Q_row = _orth(entries(rows_rep, np.arange(n)).conj().T)
    I_row = _supplement(rows_rep, m, s, rng)
    I_col = _supplement(cols_rep, n, s, rng)
    Zs = entries(I_row, I_col)
    M = np.linalg.pinv(Q_col[I_row]) @ Zs @ np.linalg.pinv(Q_row[I_col].conj().T)
    Um, sm, V_m = truncated_svd(M, r, tol)
    return Q_col @ Um, sm, Q_row @ V_m


def svd_matvec(apply_Z, apply_Zh, m: int, n: int, r: int, rng, k: int = 8, tol: float = TOL):
    """Approximate rank-r SVD from products with Z and Z^*: SVD via random
    matrix-vector multiplication, §2.1.

      1. Y = Z C, W = Z^* R with Gaussian C (n x (r+k)), R (m x (r+k)).
      2. Q_col, Q_row from pivoted QRs of Y and W (first r columns).
      3. M = (R^* Q_col)^+ R^* Z C (Q_row^* C)^+ ; note R^* Z C = W^* C.
      4. SVD of M gives Z ~ (Q_col U_M) Sigma_M (Q_row V_M)^*.
    Returns (U_0, sigma, V_0)."""
    p = r + k
    C = (rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p))) / np.sqrt(2)
    R = (rng.standard_normal((m, p)) + 1j * rng.standard_normal((m, p))) / np.sqrt(2)
    Y = apply_Z(C)
    W = apply_Zh(R)
    Q_col = _orth(Y)[:, :r]
    Q_row = _orth(W)[:, :r]
    RZC = W.conj().T @ C
    M = np.linalg.pinv(R.conj().T @ Q_col) @ RZC @ np.linalg.pinv(Q_row.conj().T @ C)
    Um, sm, V_m = truncated_svd(M, r, tol)
    return Q_col @ Um, sm, Q_row @ V_m
