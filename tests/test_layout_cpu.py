"""The packed device layouts checked on the CPU (mbf_debug_layout_apply): the factor
set is packed on the host by the same packers mbf_op_create uses, and the packed data
applied in FP64 as the layout defines it must give the oracle's FP64 apply of the same
factors.  Path 0 is the FP32 SIMT arena, path 1 the split-BF16x3 tiles of the tensor path
(whose rank padding must hold zeros) with the adjoint plan over them; forward and adjoint.  The cases span
2-D / 3-D, uniform and polar Omega trees (ragged and empty leaves), the corner turn with
S folded into G^h, several tile chunks and the largest tile (c r = 256)."""
import numpy as np
import pytest

from mbf_synth import complex_normal

from gpu_util import import_factors, oracle_case, rel

pytest.importorskip("torch")

CASES = [
    ("dft", 16, 2, 2, 8, "none"),         # L = 2: one H and one G stage
    ("dft", 64, 2, 4, 16, "none"),        # depth 4: two H and two G stages
    ("fio_iso", 64, 2, 4, 24, "polar"),   # ragged polar leaves, empty leaves, ranks not multiples of 8
    ("dft", 8, 3, 2, 16, "none"),         # 3-D octree (c = 8)
    ("dft", 32, 2, 2, 64, "none"),        # c r = 256 (the largest tile)
]

# complex64 entries: each rounded to 2^-24 relative; a few levels of sums
TOL_SIMT = 2e-6
# hi + lo bf16 of each entry: about 2^-17 relative
TOL_TILES = 1e-4


@pytest.fixture(scope="module")
def bd():
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


@pytest.mark.parametrize("case", CASES)
def test_simt_arena_forward_and_adjoint(bd, case):
    fs, sb = oracle_case(*case)
    hf = import_factors(bd, fs)
    g = complex_normal(fs.n_in, 3, seed=11)
    u = bd.layout_apply(hf, g, path=0)
    ref = sb.apply(g)
    for k in range(3):
        assert rel(u[k], ref[k]) <= TOL_SIMT, (k, rel(u[k], ref[k]))
    w = complex_normal(fs.n_out, 2, seed=12)
    gt = bd.layout_apply(hf, w, path=0, adjoint=True)
    ref_t = sb.adjoint(w)
    for k in range(2):
        assert rel(gt[k], ref_t[k]) <= TOL_SIMT, (k, rel(gt[k], ref_t[k]))


@pytest.mark.parametrize("case", CASES)
def test_tensor_tiles_forward_and_adjoint(bd, case):
    """Forward through the tile plan; adjoint through the adjoint plan over the same tiles
    read conjugate-transposed (stage e of it = forward stage S - 1 - e)."""
    fs, sb = oracle_case(*case)
    hf = import_factors(bd, fs)
    g = complex_normal(fs.n_in, 2, seed=13)
    u = bd.layout_apply(hf, g, path=1)
    ref = sb.apply(g)
    for k in range(2):
        assert rel(u[k], ref[k]) <= TOL_TILES, (k, rel(u[k], ref[k]))
    w = complex_normal(fs.n_out, 2, seed=14)
    gt = bd.layout_apply(hf, w, path=1, adjoint=True)
    ref_t = sb.adjoint(w)
    for k in range(2):
        assert rel(gt[k], ref_t[k]) <= TOL_TILES, (k, rel(gt[k], ref_t[k]))


def test_layout_arguments(bd):
    fs, _ = oracle_case("dft", 16, 2, 2, 8, "none")
    hf = import_factors(bd, fs)
    g = complex_normal(fs.n_in, 1, seed=1)
    with pytest.raises(bd.MbfError):
        bd.layout_apply(hf, g, path=2)
    with pytest.raises(bd.MbfError):
        bd.layout_apply(hf, complex_normal(fs.n_out, 1, seed=1), path=-1, adjoint=True)
    assert bd.layout_apply(hf, np.zeros((0, fs.n_in)), path=0).shape == (0, fs.n_out)


def _clustered(nx, nw, lo, side, seed):
    """X half in a blob, half uniform in [0,1)^2; Omega half near the square's centre, half
    uniform: ragged trees with empty nodes at every level (compact segments of 0 lines)."""
    rng = np.random.default_rng(seed)
    X = np.mod(np.concatenate([rng.normal(0.3, 0.08, (nx // 2, 2)), rng.random((nx - nx // 2, 2))]), 1.0)
    W = np.concatenate([rng.normal(lo + side / 2, side / 10, (nw // 2, 2)),
                        rng.uniform(lo, lo + side, (nw - nw // 2, 2))])
    return X, np.clip(W, lo, lo + side * (1 - 1e-9))


def _check_library_factors(bd, hf, rhs=2):
    from gpu_util import export_factors
    from oracle import bf as B
    sb = B.SparseBF(export_factors(hf.arrays()))
    v = hf.view
    g = complex_normal(v.n_in, rhs, seed=21)
    ref = sb.apply(g)
    for path, tol in ((0, TOL_SIMT), (1, TOL_TILES)):
        u = bd.layout_apply(hf, g, path=path)
        for k in range(rhs):
            assert rel(u[k], ref[k]) <= tol, (path, k, rel(u[k], ref[k]))
    w = complex_normal(v.n_out, rhs, seed=22)
    ref_t = sb.adjoint(w)
    for path, tol in ((0, TOL_SIMT), (1, TOL_TILES)):
        gt = bd.layout_apply(hf, w, path=path, adjoint=True)
        for k in range(rhs):
            assert rel(gt[k], ref_t[k]) <= tol, (path, k, rel(gt[k], ref_t[k]))


def test_layouts_of_explicit_point_sets(bd):
    """Explicit non-uniform point sets (§2.6): the library's factors on clustered X and
    Omega, whose trees keep empty nodes."""
    X, W = _clustered(1500, 1200, -16.0, 32.0, seed=3)
    hf = bd.HostFactors.build(2, 32, 4, 8, tree=bd.MBF_TREE_POINTS, kernel="dft", x_pts=X, w_pts=W,
                              w_lo=-16.0, w_side=32.0)
    _check_library_factors(bd, hf)


def test_layouts_of_a_multiscale_corona(bd):
    """Corona t = 0 of the multiscale split of §4 (n = 64): an Omega tree over a square
    holding a hole, so that whole subtrees are empty."""
    from oracle import msbf as MS
    n, r = 64, 12
    coronas, _ = MS.corona_sets(n, 16)
    t, idx = coronas[0]
    half = n / 2 ** (t + 1)
    hf = bd.HostFactors.build(2, n, 4, r, tree=bd.MBF_TREE_SQUARE, kernel="fio_iso", seed=7 + 101 * (t + 1),
                              w_index=idx, w_lo=-half, w_side=2 * half)
    _check_library_factors(bd, hf)


@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[3]])
def test_device_bytes_before_creation(bd, case):
    """mbf_factors_device_bytes: the tiles take sum over the 2 (L - h) G / H stages of
    c^(L-1) groups x (K_pad / 16) chunks x 4 planes x M_t rows x 32 bytes (M_t = c R8_out,
    K_pad = c R8_in rounded up to 16); the SIMT arena holds at least 8 bytes per nonzero
    and at most the full blocks' lines (2 x 4 bytes per entry, plus chunk padding)."""
    fs, _ = oracle_case(*case)
    hf = import_factors(bd, fs)
    simt, tc = hf.device_bytes()
    c, L = 2 ** fs.d, fs.L
    h = L // 2
    r8 = lambda r: (int(r) + 7) // 8 * 8
    want = 0
    for l in range(h, L):
        for R_in, R_out in ((fs.RV[l + 1], fs.RV[l]), (fs.RU[l], fs.RU[l + 1])):
            M_t, K_pad = c * r8(R_out), (c * r8(R_in) + 15) // 16 * 16
            want += c ** (L - 1) * (K_pad // 16) * 4 * M_t * 32
    assert tc == want
    nnz = sum(int(np.count_nonzero(a)) for a in list(fs.G) + list(fs.H) + [fs.UL, fs.VL])
    full = sum(c ** (L - 1) * (c * int(fs.RV[l + 1])) * (c * int(fs.RV[l])) +
               c ** (L - 1) * (c * int(fs.RU[l])) * (c * int(fs.RU[l + 1])) for l in range(h, L))
    full += fs.UL.size + fs.VL.size
    assert 8 * nnz <= simt <= 8 * full * 1.1 + 16 * 4 * c ** L
