"""Helpers shared by the GPU tests: marshal oracle factor sets into the C ABI and run
applies on torch device buffers."""
import functools

import numpy as np

from oracle import bf as B
from oracle import problem as P


def import_factors(bd, fs):
    """Oracle FactorSet -> library HostFactors (mbf_factors_t view of the same arrays)."""
    return bd.HostFactors.from_arrays(fs.d, fs.L, fs.n_out, fs.n_in, fs.x_perm, fs.x_off, fs.w_perm,
                                      fs.w_off, fs.RU, fs.RV, fs.UL, fs.VL, fs.G, fs.H, fs.S)


def export_factors(a):
    """Library-built arrays -> oracle FactorSet (for the oracle's independent apply)."""
    return B.FactorSet(d=a["d"], L=a["L"], n_out=a["n_out"], n_in=a["n_in"], x_perm=a["x_perm"],
                       x_off=a["x_off"], w_perm=a["w_perm"], w_off=a["w_off"], RU=a["RU"], RV=a["RV"],
                       UL=a["UL"], VL=a["VL"], G=a["G"], H=a["H"], S=a["S"])


@functools.lru_cache(maxsize=None)
def oracle_case(kern, n, d, L, r, tree, seed=7):
    """Factors built by the oracle (numpy FP64) for a small case."""
    X, W = P.grid_x(n, d), P.grid_omega(n, d)
    xt = P.uniform_tree(n, d, L)
    wt = P.polar_tree(n, L) if tree == "polar" else P.uniform_tree(n, d, L)
    fs = B.build(P.KERNELS[kern], X, W, xt, wt, r, seed=seed)
    return fs, B.SparseBF(fs)


def gpu_apply(torch, op, g, adjoint=False, precision=0):
    """g: complex numpy [nrhs, n_in] (forward) or [nrhs, n_out] (adjoint) -> numpy result."""
    inf = op.info()
    nrhs = g.shape[0]
    n_res = inf.n_in if adjoint else inf.n_out
    gt = torch.from_numpy(np.ascontiguousarray(g, dtype=np.complex64)).cuda()
    ut = torch.full((nrhs, n_res), float("nan"), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    if adjoint:
        op.apply_adjoint(gt.data_ptr(), ut.data_ptr(), nrhs, precision, stream)
    else:
        op.apply(gt.data_ptr(), ut.data_ptr(), nrhs, precision, stream)
    op.check(stream)
    return ut.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
