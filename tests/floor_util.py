"""Eckart-Young floor of a butterfly factorization's error, from dense SVDs of the
kernel's middle-level blocks (independent of any construction)."""
import numpy as np


def middle_level_tails(kernel, X, W, xtree, wtree, ranks):
    """{r: sum over the middle-level blocks (A, B) of sum_{k > r} sigma_k(K_{A,B})^2}.

    Every factorization of §2.3-2.4 passes each middle-level block K^h_{i,j} through
    a rank-r core (eq. Kij: K^h_{i,j} ~ U S V^*), so its Frobenius error on that block
    is at least this tail (Eckart-Young).  For g with iid unit-variance entries,
    E|(K - K_f) g|^2 = ||K - K_f||_F^2, which is bounded below by the sum of the tails."""
    L = xtree.L
    h = L // 2
    c = 2 ** xtree.d
    tot = {r: 0.0 for r in ranks}
    for i in range(c ** h):
        rows = xtree.node_points(h, i)
        for j in range(c ** (L - h)):
            cols = wtree.node_points(L - h, j)
            if rows.size == 0 or cols.size == 0:
                continue
            s = np.linalg.svd(kernel(X[rows][:, None, :], W[cols][None, :, :]), compute_uv=False)
            for r in ranks:
                tot[r] += float(np.sum(s[r:] ** 2))
    return tot


def floor_from_tails(tails, n_x, n_xi):
    """Relative floor sqrt(tail / ||K||_F^2); every entry of a DFT or FIO kernel has
    modulus 1, so ||K||_F^2 = n_x n_xi."""
    return {r: float(np.sqrt(v / (n_x * n_xi))) for r, v in tails.items()}
