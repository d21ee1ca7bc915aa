"""GPU parity of the multiscale butterfly factorization (§4, eq. f1): the sum of the
per-corona operators (FP32 SIMT or split-BF16x3) and the dense centre, against the
oracle's FP64 multiscale apply of the same factors, forward and adjoint; the
library's own construction (mbf_build_msbf) against the same parts assembled from
the oracle's corona split; and the error against the direct sum."""
import numpy as np
import pytest

from mbf_synth import complex_normal, sample_outputs
from oracle import direct as D
from oracle import msbf as MS
from oracle import problem as P
from paper_1509_07925_gb300.binding import MBF_PREC_BF16X3, MBF_PREC_FP32_SIMT

from gpu_util import export_factors, import_factors, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(32, 8, 8), (64, 12, 16)]      # (n, r, n_center)


@pytest.fixture(scope="module")
def bd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def cases(bd):
    out = {}
    for n, r, nc in CASES:
        m = MS.build(P.kernel_fio_iso, n, r, n_center=nc)
        parts = [bd.Operator(import_factors(bd, fs)) for _, _, _, fs in m.parts]
        gm = bd.MsBF.create(parts, m.Kc.T, m.center)
        out[n] = (m, MS.SparseMsBF(m), gm)
    return out


def _apply(bd, gm, g, n_res, precision, adjoint=False):
    gt = torch.from_numpy(np.ascontiguousarray(g, dtype=np.complex64)).cuda()
    ut = torch.full((g.shape[0], n_res), float("nan"), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    if adjoint:
        gm.apply_adjoint(gt.data_ptr(), ut.data_ptr(), g.shape[0], precision, st)
    else:
        gm.apply(gt.data_ptr(), ut.data_ptr(), g.shape[0], precision, st)
    gm.check(st)
    return ut.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n", [c[0] for c in CASES])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_msbf_forward_simt(bd, cases, n, nrhs):
    m, sm, gm = cases[n]
    g = complex_normal(n * n, nrhs, seed=31)
    u = _apply(bd, gm, g, n * n, MBF_PREC_FP32_SIMT)
    ref = sm.apply(g)
    for k in range(nrhs):
        assert rel(u[k], ref[k]) <= 1e-5


@pytest.mark.parametrize("n", [c[0] for c in CASES])
def test_msbf_forward_tensor(bd, cases, n):
    m, sm, gm = cases[n]
    g = complex_normal(n * n, 64, seed=32)
    u = _apply(bd, gm, g, n * n, MBF_PREC_BF16X3)
    ref = sm.apply(g)
    for k in range(64):
        assert rel(u[k], ref[k]) <= 1e-4


@pytest.mark.parametrize("n", [c[0] for c in CASES])
def test_msbf_adjoint(bd, cases, n):
    m, sm, gm = cases[n]
    w = complex_normal(n * n, 2, seed=33)
    g = _apply(bd, gm, w, n * n, MBF_PREC_FP32_SIMT, adjoint=True)
    ref = sm.adjoint(w)
    for k in range(2):
        assert rel(g[k], ref[k]) <= 1e-5


@pytest.mark.parametrize("n", [c[0] for c in CASES])
def test_msbf_adjoint_tensor(bd, cases, n):
    """The multiscale adjoint with 64 RHS on the tensor cores: each corona's adjoint
    scatters into its own Omega points (zero elsewhere for the first part, accumulated
    for the others), the centre adds its part."""
    m, sm, gm = cases[n]
    w = complex_normal(n * n, 64, seed=35)
    g = _apply(bd, gm, w, n * n, MBF_PREC_BF16X3, adjoint=True)
    ref = sm.adjoint(w)
    for k in range(64):
        assert rel(g[k], ref[k]) <= 1e-4


def test_library_construction_matches_assembled_parts_and_direct_sum(bd):
    """mbf_build_msbf (its own corona split) equals the parts built one by one on the
    oracle's split with the same seeds; the GPU result matches the FP64 apply of the
    exported factors, and its error against the direct sum stays at the factorization's."""
    n, r, nc = 64, 12, 16
    lib_m = bd.MsBF.build(n, r, kernel="fio_iso", n_center=nc, seed=7)
    inf = lib_m.info()
    coronas, centre = MS.corona_sets(n, nc)
    assert inf.n_parts == len(coronas) and inf.n_center_points == centre.size
    parts, hfs = [], []
    L = int(np.log2(n))
    for t, idx in coronas:
        Lt = 2 * ((L - t) // 2)
        half = n / 2 ** (t + 1)
        hf = bd.HostFactors.build(2, n, Lt, r, tree=bd.MBF_TREE_SQUARE, kernel="fio_iso", seed=7 + 101 * (t + 1),
                                  w_index=idx, w_lo=-half, w_side=2 * half)
        hfs.append(hf)
        parts.append(bd.Operator(hf))
        assert inf.part_points[t] == idx.size and inf.part_L[t] == Lt
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    Kc = P.kernel_fio_iso(X[:, None, :], W[centre][None, :, :])
    asm = bd.MsBF.create(parts, Kc.T, centre)
    g = complex_normal(n * n, 2, seed=34)
    u_lib = _apply(bd, lib_m, g, n * n, MBF_PREC_FP32_SIMT)
    u_asm = _apply(bd, asm, g, n * n, MBF_PREC_FP32_SIMT)
    assert np.array_equal(u_lib, u_asm)
    # FP64 apply of the library's factors: sum of the exported parts plus the centre
    ref = (Kc @ g[:, centre].T).T
    from oracle import bf as B
    for hf in hfs:
        ref = ref + B.SparseBF(export_factors(hf.arrays())).apply(g)
    assert rel(u_lib, ref) <= 1e-5
    S = sample_outputs(n * n, 256, seed=1)
    ud = D.direct_sum(P.kernel_fio_iso, X, W, g, rows=S)
    eps = D.rel_err(ref[:, S], ud)
    assert eps < 0.2
    assert D.rel_err(u_lib[:, S], ud) <= eps + 1e-5
    asm.close()
    lib_m.close()


def test_msbf_n256_with_a_tensor_only_corona(bd):
    """n = 256 (coronas t = 0..3): the t = 3 corona's X tree has depth 4, so its leaf groups
    hold 1024 points, beyond the SIMT kernel; that part applies on the tensor cores for
    any RHS count while the others take the SIMT path at 3 RHS.  Parts built one by one
    (library host builder), checked against the FP64 apply of their exported factors
    plus the centre, and against the direct sum on sampled outputs."""
    from oracle import bf as B
    n, r, nc = 256, 12, 16
    coronas, centre = MS.corona_sets(n, nc)
    assert len(coronas) == 4
    L = int(np.log2(n))
    parts, sbs = [], []
    for t, idx in coronas:
        Lt = 2 * ((L - t) // 2)
        half = n / 2 ** (t + 1)
        hf = bd.HostFactors.build(2, n, Lt, r, tree=bd.MBF_TREE_SQUARE, kernel="fio_iso", seed=7 + 101 * (t + 1),
                                  w_index=idx, w_lo=-half, w_side=2 * half)
        sbs.append(B.SparseBF(export_factors(hf.arrays())))
        parts.append(bd.Operator(hf))
    X, W = P.grid_x(n, 2), P.grid_omega(n, 2)
    Kc = P.kernel_fio_iso(X[:, None, :], W[centre][None, :, :])
    m = bd.MsBF.create(parts, Kc.T, centre)
    S = sample_outputs(n * n, 256, seed=1)
    for nrhs, prec in ((3, 0), (64, MBF_PREC_BF16X3)):
        g = complex_normal(n * n, nrhs, seed=80 + nrhs)
        u = _apply(bd, m, g, n * n, prec)
        ref = (Kc @ g[:, centre].T).T
        for sb in sbs:
            ref = ref + sb.apply(g)
        for k in range(nrhs):
            assert rel(u[k], ref[k]) <= 1e-4, (nrhs, k, rel(u[k], ref[k]))
        ud = D.direct_sum(P.kernel_fio_iso, X, W, g, rows=S)
        eps = D.rel_err(ref[:, S], ud)
        assert D.rel_err(u[:, S], ud) <= eps + 1e-4
    w = complex_normal(n * n, 3, seed=90)
    ga = _apply(bd, m, w, n * n, 0, adjoint=True)
    refa = (np.conj(Kc).T @ w.T).T
    refa_full = np.zeros_like(ga)
    refa_full[:, centre] = refa
    for sb in sbs:
        refa_full = refa_full + sb.adjoint(w)
    for k in range(3):
        assert rel(ga[k], refa_full[k]) <= 1e-4
    m.close()
