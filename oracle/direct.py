"""Direct summation, closed-form DFT and the error metric (oracle; test infrastructure only)."""
from __future__ import annotations

import numpy as np

from .problem import kernel_block


def direct_sum(kernel, X: np.ndarray, W: np.ndarray, g: np.ndarray, rows=None,
               block: int = 256) -> np.ndarray:
    """u(x) = sum_{xi in Omega} K(x, xi) g(xi) for x in rows (all of X if None).

    §1.1, eq. (kernel), evaluated by definition in complex128.  g has shape
    [nrhs, N_Omega]; the result has shape [nrhs, len(rows)].  Rows are processed
    in blocks only to bound memory; every term is summed exactly as defined."""
    g = np.atleast_2d(g)
    rows = np.arange(X.shape[0]) if rows is None else np.asarray(rows, dtype=np.int64)
    cols = np.arange(W.shape[0])
    out = np.empty((g.shape[0], rows.shape[0]), dtype=np.complex128)
    for a in range(0, rows.shape[0], block):
        K = kernel_block(kernel, X, W, rows[a:a + block], cols)
        out[:, a:a + block] = (K @ g.T).T
    return out


def dft_closed_form(g: np.ndarray, n: int, d: int) -> np.ndarray:
    """Closed form of the direct sum for the DFT kernel exp(-2 pi i m.xi/n).

    With xi = k - n/2 (k = 0..n-1 per axis), exp(-2 pi i m (k - n/2)/n) =
    exp(-2 pi i m k/n) (-1)^m, so u = (-1)^(m_1+...+m_d) FFT_d(g)[m].  This is the
    library special case that pins the direct sum (and, through it, the BF)."""
    g = np.atleast_2d(g)
    shape = (g.shape[0],) + (n,) * d
    G = g.reshape(shape)
    U = np.fft.fftn(G, axes=tuple(range(1, d + 1)))
    sign = (-1.0) ** np.sum(np.indices((n,) * d), axis=0)
    return (U * sign).reshape(g.shape[0], -1)


def rel_err(u_approx: np.ndarray, u_exact: np.ndarray) -> float:
    """e = sqrt(sum |u^f - u|^2 / sum |u|^2) over the given outputs (and RHS),
    the estimator of §3.3 (e^p) and §4.3 (e^m)."""
    num = np.sum(np.abs(np.asarray(u_approx) - np.asarray(u_exact)) ** 2)
    den = np.sum(np.abs(np.asarray(u_exact)) ** 2)
    return float(np.sqrt(num / den))
