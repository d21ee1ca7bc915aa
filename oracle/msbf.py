"""Multiscale butterfly factorization (MBF), §4: the corona split of Omega and the
multiscale sum of eqs. (msumd) and (f1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

    K ~ K_C R_C + sum_{t=0}^{T-1} BF_t R_t                                    (eq. f1)

R_t restricts g to the corona Omega_t of eq. (domaindecomp), BF_t is the butterfly
factorization (§2.3-2.4, `bf.build`) of the kernel restricted to X x Omega_t built on
two quadtrees of depth L_t = 2 floor((L - t) / 2): T_X over X and T_{Omega~_t} over the
smallest square Omega~_t = [-n/2^(t+1), n/2^(t+1))^2 holding Omega_t (its upper faces
are closed, so xi_k = n/2^(t+1) lands in the last cell).  K_C R_C is the kernel
restricted to the centre Omega_C, applied as a dense matrix (§4.1: O(1) points there).
"""
from dataclasses import dataclass, field

import numpy as np

from . import bf as B
from . import problem as P


@dataclass
class MsBF:
    n: int
    L: int
    n_center: int
    center: np.ndarray                         # natural Omega indices of Omega_C
    Kc: np.ndarray                             # [N_x, |Omega_C|] complex128
    parts: list = field(default_factory=list)  # (t, L_t, corona indices, FactorSet)


def corona_sets(n: int, n_center: int):
    """[(t, indices of Omega_t)], indices of Omega_C (eq. domaindecomp; `problem.corona_index`)."""
    W = P.grid_omega(n, 2)
    t_of = P.corona_index(W, n, n_center)
    T = int(t_of.max()) + 1 if np.any(t_of >= 0) else 0
    return [(t, np.nonzero(t_of == t)[0]) for t in range(T)], np.nonzero(t_of < 0)[0]


def build(kernel, n: int, r: int, n_center: int = 16, seed: int = 7) -> MsBF:
    """The factorization of §4.2: one BF per corona (step 2) plus the dense centre."""
    L = int(round(np.log2(n)))
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    coronas, center = corona_sets(n, n_center)
    Kc = kernel(X[:, None, :], W[center][None, :, :]) if center.size else np.zeros((X.shape[0], 0), complex)
    m = MsBF(n=n, L=L, n_center=n_center, center=center, Kc=np.asarray(Kc, dtype=np.complex128))
    for t, idx in coronas:
        Lt = 2 * ((L - t) // 2)
        half = n / 2 ** (t + 1)
        xt = P.uniform_tree(n, 2, Lt)
        wt = P.square_tree(W[idx], idx, -half, 2 * half, Lt)
        fs = B.build(kernel, X, W, xt, wt, r, seed=seed + 101 * (t + 1))
        m.parts.append((t, Lt, idx, fs))
    return m


class SparseMsBF:
    """Apply of eq. (f1): u = K_C (R_C g) + sum_t BF_t (R_t g), each BF_t by `bf.SparseBF`
    (its leaf matrix V^L_t only has rows at the points of Omega_t, which is R_t)."""

    def __init__(self, m: MsBF):
        self.m = m
        self.bfs = [B.SparseBF(fs) for _, _, _, fs in m.parts]

    def apply(self, g: np.ndarray) -> np.ndarray:
        g = np.atleast_2d(g)
        u = (self.m.Kc @ g[:, self.m.center].T).T
        for sb in self.bfs:
            u = u + sb.apply(g)
        return u

    def adjoint(self, u: np.ndarray) -> np.ndarray:
        u = np.atleast_2d(u)
        g = np.zeros((u.shape[0], self.m.n ** 2), dtype=np.complex128)
        g[:, self.m.center] = (self.m.Kc.conj().T @ u.T).T
        for sb in self.bfs:
            g = g + sb.adjoint(u)
        return g
