"""Butterfly factorization: construction, factor matrices and apply (oracle; test
infrastructure only).

Construction follows §2.3 (middle level) and §2.4 (recursive factorization) in
the paper's order and notation, with every intermediate U^l_{i,j}, V^l_{j,i}
held in memory (small problems only; §2.5 notes the O(N^{3/2}) peak).

The result is a *padded factor set*: every block of a level is stored in a
dense array whose rank dimension is the largest rank met on that level, with
zeros beyond each block's own rank and beyond each leaf's own point count.
Zero padding leaves every product unchanged.  The same layout is the
interchange format through which the CUDA library imports factors.

The apply assembles each factor as an explicit sparse matrix with the block
structure drawn in §2.3-2.4 (U^L block diagonal as in eq. expression-U; G^l as
in the display after eq. blockF; M^h with its (j,i) sub-blocks S^h_{i,j}) and
multiplies them in the order of eq. (gbf):
    K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .lowrank import TOL, _orth, forms, svd_sampling, truncated_svd


@dataclass
class FactorSet:
    """Padded factors of K ~ U^L G^{L-1}..G^h M^h (H^h)^*..(H^{L-1})^* (V^L)^*.

    Index conventions (c = 2^d children per node, h = L/2):
      UL[i, a, k]     row a of U^L_i (X-leaf i, its a-th point in tree order), column k
      VL[j, a, k]     row a of V^L_j (Omega-leaf j)
      G[l-h][i, jp, t, k2, tp, k]   entry (k2, k) of the column block tp of
                      G^l_{c i + t, jp}  (i in I^l, jp in I^{L-l-1}); column block tp
                      multiplies U^l_{i, c jp + tp}  (eq. RSh2)
      H[l-h][j, ip, t, k2, tp, k]   same for H^l_{c j + t, ip} on the Omega side
      S[i, j, k]      diagonal of S^h_{i,j} (eq. Kij, form of eq. lowrank1)
      RU[l], RV[l]    padded rank of level l on the X / Omega side (l = h..L)
      kU[l], kV[l]    true ranks, arrays [c^l, c^(L-l)]
    """

    d: int
    L: int
    n_out: int
    n_in: int
    x_perm: np.ndarray
    x_off: np.ndarray
    w_perm: np.ndarray
    w_off: np.ndarray
    RU: np.ndarray
    RV: np.ndarray
    UL: np.ndarray
    VL: np.ndarray
    G: list
    H: list
    S: np.ndarray
    kU: dict = field(default_factory=dict)
    kV: dict = field(default_factory=dict)

    @property
    def c(self):
        return 2 ** self.d

    @property
    def h(self):
        return self.L // 2

    def nnz_algorithmic(self) -> int:
        """Nonzero entries of the unpadded factors: the apply cost of §2.5."""
        c, L, h = self.c, self.L, self.h
        x_sz, w_sz = np.diff(self.x_off), np.diff(self.w_off)
        total = int(np.sum(x_sz * self.kU[L][:, 0])) + int(np.sum(w_sz * self.kV[L][:, 0]))
        total += int(np.sum(self.kU[h]))  # the diagonal S blocks
        for side in (self.kU, self.kV):
            for l in range(h, L):
                kin = side[l].reshape(c ** l, c ** (L - l - 1), c).sum(axis=2)    # [i, jp]
                kout = side[l + 1].reshape(c ** l, c, c ** (L - l - 1))          # [i, t, jp]
                total += int(np.sum(kout * kin[:, None, :]))
        return total


# ----------------------------------------------------------------------------
# construction
# ----------------------------------------------------------------------------


def build(kernel, X: np.ndarray, W: np.ndarray, xtree, wtree, r: int, seed: int = 7,
          factor: int = 3, tol: float = TOL) -> FactorSet:
    """Construct the BF of K = (kernel(x, xi)) on trees T_X (xtree) and T_Omega (wtree).

    Case (ii) of §2.3: entries are evaluated on demand and each middle-level block
    is factored by the SVD via random sampling (§2.1).  Per-block generators are
    seeded from (seed, i, j) so the result does not depend on loop order."""
    d, L = xtree.d, xtree.L
    assert wtree.L == L and wtree.d == d and L % 2 == 0 and L >= 2
    c, h = 2 ** d, L // 2

    # ---- middle level, §2.3: K^h_{i,j} ~ U^h_{i,j} S^h_{i,j} (V^h_{j,i})^*  (eq. Kij)
    Ucur, Vcur, S = {}, {}, {}
    for i in range(c ** h):
        rows = xtree.node_points(h, i)
        for j in range(c ** h):
            cols = wtree.node_points(L - h, j)
            rng = np.random.default_rng([seed, 0, i, j])

            def entries(a, b, rows=rows, cols=cols):
                return kernel(X[rows[a]][:, None, :], W[cols[b]][None, :, :])

            U0, s, V0 = svd_sampling(entries, rows.shape[0], cols.shape[0], r, rng,
                                     factor=factor, tol=tol)
            U, Sd, V = forms(U0, s, V0, 1)
            Ucur[i, j], S[i, j], Vcur[j, i] = U, Sd, V
    return _recursive(X.shape[0], W.shape[0], xtree, wtree, r, tol, Ucur, Vcur, S)


def build_from_applies(apply_K, apply_Kh, n_out: int, n_in: int, xtree, wtree, r: int,
                       seed: int = 7, k: int = 8, tol: float = TOL) -> FactorSet:
    """Construct the BF of an operator known only through products with K and K^*
    (Case (i) of §2.3).  apply_K(V) = K V for V of shape [n_in, m], apply_Kh(V) = K^* V.

    For each Omega node j a Gaussian C_j (|B_j| x (r + k)) is zero-padded to C^P_j and
    K C^P_j gives K^h_{i,j} C_j for every i; for each X node i, R_i padded to R^P_i gives
    (K^h_{i,j})^* R_i for every j.  Each block is then factored by the SVD via random
    matrix-vector multiplication (§2.1): Q_col, Q_row from pivoted QRs of the two products
    (first r columns), M = (R_i^* Q_col)^+ (R_i^* K^h_{i,j} C_j) (Q_row^* C_j)^+, and the SVD
    of M; R_i^* K^h_{i,j} C_j is read off as ((K^h_{i,j})^* R_i)^* C_j."""
    d, L = xtree.d, xtree.L
    assert wtree.L == L and wtree.d == d and L % 2 == 0 and L >= 2
    c, h = 2 ** d, L // 2
    p = r + k
    rng = np.random.default_rng([seed, 1])
    C, KC = {}, {}
    for j in range(c ** h):
        cols = wtree.node_points(L - h, j)
        C[j] = (rng.standard_normal((cols.size, p)) + 1j * rng.standard_normal((cols.size, p))) / np.sqrt(2)
        CP = np.zeros((n_in, p), dtype=np.complex128)
        CP[cols] = C[j]
        KC[j] = apply_K(CP)
    R, KhR = {}, {}
    for i in range(c ** h):
        rows = xtree.node_points(h, i)
        R[i] = (rng.standard_normal((rows.size, p)) + 1j * rng.standard_normal((rows.size, p))) / np.sqrt(2)
        RP = np.zeros((n_out, p), dtype=np.complex128)
        RP[rows] = R[i]
        KhR[i] = apply_Kh(RP)
    Ucur, Vcur, S = {}, {}, {}
    for i in range(c ** h):
        rows = xtree.node_points(h, i)
        for j in range(c ** h):
            cols = wtree.node_points(L - h, j)
            Y, Wm = KC[j][rows], KhR[i][cols]
            if rows.size == 0 or cols.size == 0:
                U0, s, V0 = truncated_svd(np.zeros((rows.size, cols.size), complex), r, tol)
            else:
                Qc, Qr = _orth(Y)[:, :r], _orth(Wm)[:, :r]
                M = np.linalg.pinv(R[i].conj().T @ Qc) @ (Wm.conj().T @ C[j]) @ np.linalg.pinv(Qr.conj().T @ C[j])
                Um, s, Vm = truncated_svd(M, r, tol)
                U0, V0 = Qc @ Um, Qr @ Vm
            U, Sd, V = forms(U0, s, V0, 1)
            Ucur[i, j], S[i, j], Vcur[j, i] = U, Sd, V
    return _recursive(n_out, n_in, xtree, wtree, r, tol, Ucur, Vcur, S)


def _recursive(n_out, n_in, xtree, wtree, r, tol, Ucur, Vcur, S) -> FactorSet:
    """§2.4: the recursive factorization of the middle-level factors and the assembly of
    the padded factor set."""
    d, L = xtree.d, xtree.L
    c, h = 2 ** d, L // 2
    kU = {h: np.array([[Ucur[i, j].shape[1] for j in range(c ** h)] for i in range(c ** h)])}
    kV = {h: np.array([[Vcur[j, i].shape[1] for i in range(c ** h)] for j in range(c ** h)])}

    # ---- recursive factorization, §2.4.1 (U side) and §2.4.2 (V side)
    def recurse(cur, tree, kdict):
        mats = []
        for l in range(h, L):
            nxt, Gl = {}, {}
            for i in range(c ** l):
                a0, _ = tree.node_range(l, i)
                for t in range(c):
                    child = c * i + t
                    b0, b1 = tree.node_range(l + 1, child)
                    rows = slice(b0 - a0, b1 - a0)      # splitting, eq. (splitandmerge)
                    for jp in range(c ** (L - l - 1)):
                        parts = [cur[i, c * jp + tp][rows] for tp in range(c)]
                        B = np.hstack(parts)            # merging, eq. (blocks)
                        U0, s, V0 = truncated_svd(B, r, tol)   # truncating
                        Unew, _, Vr = forms(U0, s, V0, 2)      # form of eq. (lowrank2)
                        nxt[child, jp] = Unew
                        Gl[child, jp] = (Vr.conj().T, [p.shape[1] for p in parts])
            kdict[l + 1] = np.array([[nxt[a, b].shape[1] for b in range(c ** (L - l - 1))]
                                     for a in range(c ** (l + 1))])
            mats.append(Gl)
            cur = nxt
        return cur, mats

    Ucur, Gmats = recurse(Ucur, xtree, kU)
    Vcur, Hmats = recurse(Vcur, wtree, kV)

    # ---- padded factor set (assembling)
    RU = np.zeros(L + 1, dtype=np.int64)
    RV = np.zeros(L + 1, dtype=np.int64)
    for l in range(h, L + 1):
        RU[l] = max(1, int(kU[l].max()))
        RV[l] = max(1, int(kV[l].max()))
    RU[h] = RV[h] = max(RU[h], RV[h])

    def leaf_array(cur, tree, R):
        sizes = tree.leaf_sizes()
        mx = max(1, int(sizes.max()))
        A = np.zeros((c ** L, mx, R), dtype=np.complex128)
        for i in range(c ** L):
            B = cur[i, 0]
            A[i, :B.shape[0], :B.shape[1]] = B
        return A

    def level_arrays(mats, R):
        out = []
        for idx, Gl in enumerate(mats):
            l = h + idx
            A = np.zeros((c ** l, c ** (L - l - 1), c, R[l + 1], c, R[l]), dtype=np.complex128)
            for (child, jp), (Gm, sizes) in Gl.items():
                i, t = divmod(child, c)
                off = 0
                for tp in range(c):
                    A[i, jp, t, :Gm.shape[0], tp, :sizes[tp]] = Gm[:, off:off + sizes[tp]]
                    off += sizes[tp]
            out.append(A)
        return out

    Sarr = np.zeros((c ** h, c ** h, RU[h]))
    for (i, j), Sd in S.items():
        Sarr[i, j, :Sd.shape[0]] = Sd

    return FactorSet(d=d, L=L, n_out=n_out, n_in=n_in,
                     x_perm=xtree.perm, x_off=xtree.off, w_perm=wtree.perm, w_off=wtree.off,
                     RU=RU, RV=RV, UL=leaf_array(Ucur, xtree, RU[L]),
                     VL=leaf_array(Vcur, wtree, RV[L]),
                     G=level_arrays(Gmats, RU), H=level_arrays(Hmats, RV), S=Sarr, kU=kU, kV=kV)


# ----------------------------------------------------------------------------
# factors as explicit sparse matrices, apply and adjoint
# ----------------------------------------------------------------------------


def _coo(vals, rows, cols, shape):
    nz = vals != 0
    return sp.csr_matrix((vals[nz], (rows[nz], cols[nz])), shape=shape)


def leaf_matrix(A: np.ndarray, perm: np.ndarray, off: np.ndarray, n_points: int):
    """U^L (or V^L): block diagonal, block i = the leaf basis of leaf i, with rows
    placed at the natural indices of that leaf's points (eq. expression-U at l = L)."""
    n_leaves, mx, R = A.shape
    i, a, k = np.nonzero(A)
    sizes = np.diff(off)
    keep = a < sizes[i]
    i, a, k = i[keep], a[keep], k[keep]
    rows = perm[off[i] + a]
    cols = i * R + k
    return _coo(A[i, a, k], rows, cols, (n_points, n_leaves * R))


def transfer_matrix(A: np.ndarray, c: int, L: int, l: int):
    """G^l (or H^l) of eq. (RSU)/(RSV): rows indexed by (c i + t, jp, k2) -- the
    columns of U^{l+1} -- and columns by (i, c jp + tp, k) -- the columns of U^l.
    Block (c i + t, i) is G^l_{c i + t} = blockdiag_jp(G^l_{c i + t, jp})."""
    ni, njp, _, R2, _, R1 = A.shape
    i, jp, t, k2, tp, k = np.nonzero(A)
    B = c ** (L - l - 1)
    rows = ((c * i + t) * B + jp) * R2 + k2
    cols = (i * c ** (L - l) + c * jp + tp) * R1 + k
    n = c ** L
    return _coo(A[i, jp, t, k2, tp, k], rows, cols, (n * R2, n * R1))


def middle_matrix(S: np.ndarray, c: int, h: int):
    """M^h (§2.3): block (i, j) is zero except its (j, i) sub-block S^h_{i,j}; rows are
    the columns (i, j, k) of U^h, columns the columns (j, i, k) of V^h."""
    ni, nj, R = S.shape
    i, j, k = np.meshgrid(np.arange(ni), np.arange(nj), np.arange(R), indexing="ij")
    rows = (i * c ** h + j) * R + k
    cols = (j * c ** h + i) * R + k
    n = c ** (2 * h)
    return _coo(S.ravel().astype(np.complex128), rows.ravel(), cols.ravel(), (n * R, n * R))


class SparseBF:
    """The factors of a FactorSet as scipy CSR matrices; `apply` multiplies them in
    the order of eq. (gbf), `adjoint` applies K^* = V^L H^{L-1} .. (M^h)^* .. (U^L)^*."""

    def __init__(self, fs: FactorSet):
        c, L, h = fs.c, fs.L, fs.h
        self.fs = fs
        self.UL = leaf_matrix(fs.UL, fs.x_perm, fs.x_off, fs.n_out)
        self.VL = leaf_matrix(fs.VL, fs.w_perm, fs.w_off, fs.n_in)
        self.G = [transfer_matrix(A, c, L, h + q) for q, A in enumerate(fs.G)]
        self.H = [transfer_matrix(A, c, L, h + q) for q, A in enumerate(fs.H)]
        self.M = middle_matrix(fs.S, c, h)

    def factors(self):
        """[U^L, G^{L-1}, ..., G^h, M^h, (H^h)^*, ..., (H^{L-1})^*, (V^L)^*] in order."""
        out = [self.UL] + self.G[::-1] + [self.M]
        out += [H.conj().T.tocsr() for H in self.H] + [self.VL.conj().T.tocsr()]
        return out

    def apply(self, g: np.ndarray) -> np.ndarray:
        """u = K_f g for g of shape [nrhs, n_in]; returns [nrhs, n_out]."""
        v = np.atleast_2d(g).T.astype(np.complex128)
        v = self.VL.conj().T @ v
        for H in self.H[::-1]:                 # (H^{L-1})^* first, (H^h)^* last
            v = H.conj().T @ v
        v = self.M @ v
        for G in self.G:                       # G^h first, G^{L-1} last
            v = G @ v
        v = self.UL @ v
        return np.asarray(v).T

    def adjoint(self, u: np.ndarray) -> np.ndarray:
        """g = K_f^* u for u of shape [nrhs, n_out]; returns [nrhs, n_in]."""
        v = np.atleast_2d(u).T.astype(np.complex128)
        v = self.UL.conj().T @ v
        for G in self.G[::-1]:
            v = G.conj().T @ v
        v = self.M.conj().T @ v
        for H in self.H:
            v = H @ v
        v = self.VL @ v
        return np.asarray(v).T

    def dense(self) -> np.ndarray:
        """Dense product of all factors (brute force, small N only)."""
        fac = self.factors()
        D = fac[-1].toarray()
        for F in fac[-2::-1]:
            D = F @ D
        return np.asarray(D)


class BlockBF:
    """The same product of eq. (gbf) applied level by level on the padded arrays, without
    assembling sparse matrices: memory of one level at a time, for factor sets too large
    for `SparseBF` (test infrastructure; equal to `SparseBF` to rounding, pinned).

    Vector of level l on the X side: [c^l, c^(L-l), R_l] indexed (i, j, k) as the columns
    of U^l; on the Omega side [c^l, c^(L-l), R_l] indexed (j, i, k) as the columns of V^l.
      (V^L)^*:   y[j, 0, k]       = sum_a conj(V^L[j, a, k]) g[w_perm[w_off[j] + a]]
      (H^l)^*:   y_l[j, c ip + tp, k] = sum_{t, k2} conj(H^l[j, ip, t, k2, tp, k]) y_{l+1}[c j + t, ip, k2]
      M^h:       w[i, j, k]       = S[i, j, k] y_h[j, i, k]
      G^l:       w_{l+1}[c i + t, jp, k2] = sum_{tp, k} G^l[i, jp, t, k2, tp, k] w_l[i, c jp + tp, k]
      U^L:       u[x_perm[x_off[i] + a]] = sum_k U^L[i, a, k] w[i, 0, k]
    (the index conventions of `FactorSet`, eqs. RSh2 / VF, lowrank1, expression-U)."""

    def __init__(self, fs: FactorSet):
        self.fs = fs

    @staticmethod
    def _gather_index(perm, off, mx):
        sizes = np.diff(off)
        a = np.arange(mx)[None, :]
        valid = a < sizes[:, None]
        idx = np.where(valid, off[:-1, None] + a, 0)
        return np.where(valid, perm[np.minimum(idx, max(perm.shape[0] - 1, 0))], 0), valid

    def apply(self, g: np.ndarray) -> np.ndarray:
        fs = self.fs
        c, L, h = fs.c, fs.L, fs.h
        nL = c ** L
        g = np.atleast_2d(g)
        nr = g.shape[0]
        gt = np.ascontiguousarray(g.T)                              # [n_in, nrhs]
        gi, gv = self._gather_index(fs.w_perm, fs.w_off, fs.VL.shape[1])
        leaf_in = gt[gi] * gv[..., None]                            # [nL, mx, nrhs]
        y = np.matmul(np.conj(fs.VL).transpose(0, 2, 1), leaf_in)   # [nL, R_L, nrhs]
        for l in range(L - 1, h - 1, -1):
            A = fs.H[l - h]                                         # [c^l, c^(L-l-1), c, R2, c, R1]
            ni, njp, _, R2, _, R1 = A.shape
            yl = y.reshape(ni, c, njp, R2, nr).transpose(0, 2, 1, 3, 4).reshape(ni * njp, c * R2, nr)
            Ah = np.conj(A).reshape(ni * njp, c * R2, c * R1).transpose(0, 2, 1)
            y = np.matmul(Ah, yl).reshape(ni, njp * c, R1, nr)     # (j, c ip + tp, k)
        w = fs.S[..., None] * y.transpose(1, 0, 2, 3)               # [c^h, c^h, R_h, nrhs]
        for l in range(h, L):
            A = fs.G[l - h]
            ni, njp, _, R2, _, R1 = A.shape
            wl = w.reshape(ni * njp, c * R1, nr)                    # (i, jp), (tp, k)
            out = np.matmul(A.reshape(ni * njp, c * R2, c * R1), wl).reshape(ni, njp, c, R2, nr)
            w = out.transpose(0, 2, 1, 3, 4).reshape(ni * c, njp, R2, nr)
        up = np.matmul(fs.UL, w.reshape(nL, -1, nr))                # [nL, mx, nrhs]
        xi, xv = self._gather_index(fs.x_perm, fs.x_off, fs.UL.shape[1])
        u = np.zeros((fs.n_out, nr), dtype=np.complex128)
        u[xi[xv]] = up[xv]
        return u.T
