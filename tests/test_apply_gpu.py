"""GPU parity: the sm_103a apply (through the C ABI) against the oracle's FP64
apply of the same factors, element by element (relative L2 <= 1e-5 for the FP32
SIMT path), forward and adjoint, several RHS counts, ragged polar leaves, 3-D."""
import numpy as np
import pytest

from mbf_synth import complex_normal
from oracle import bf as B
from oracle import direct as D
from oracle import problem as P
from paper_1509_07925_gb300.binding import MBF_PREC_FP32_SIMT

from gpu_util import export_factors, gpu_apply, import_factors, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SIMT = 1e-5

CASES = [
    ("dft", 16, 2, 2, 8, "none"),         # 4 groups per stage, L = 2 (h = L - 1)
    ("dft", 64, 2, 4, 16, "none"),        # 2-D DFT n=64, depth 4, 4x4-point leaves, r=16
    ("fio_iso", 64, 2, 4, 24, "polar"),   # ragged polar leaves (up to 38 points), empty leaves
    ("fio_iso", 32, 2, 4, 12, "polar"),
    ("dft", 8, 3, 2, 16, "none"),         # 3-D octree (c = 8)
    ("dft", 32, 2, 2, 64, "none"),        # longest line: c r = 256, 256-point leaves
]


@pytest.fixture(scope="module")
def bd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ops(bd):
    cache = {}

    def get(case):
        if case not in cache:
            fs, sb = oracle_case(*case)
            cache[case] = (bd.Operator(import_factors(bd, fs)), fs, sb)
        return cache[case]
    return get


@pytest.mark.parametrize("case", CASES[:3])
def test_nnz_counted_when_factors_do_not_give_it(ops, case):
    """Factors imported without a nonzero count (mbf_factors_t.nnz = 0): the operator reports
    the nonzero entries its packer stored, i.e. the oracle's count of the unpadded factors
    less the diagonal S entries, which are folded into the G^h tiles."""
    op, fs, _ = ops(case)
    nnz = op.info().nnz_algorithmic
    exp = fs.nnz_algorithmic()
    assert exp - int(np.sum(fs.kU[fs.h])) <= nnz <= exp


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nrhs", [1, 3, 4, 9])
def test_forward_matches_oracle(ops, case, nrhs):
    op, fs, sb = ops(case)
    g = complex_normal(fs.n_in, nrhs, seed=11)
    u = gpu_apply(torch, op, g, precision=MBF_PREC_FP32_SIMT)
    ref = sb.apply(g)
    assert u.shape == ref.shape
    assert np.all(np.isfinite(u))
    for k in range(nrhs):
        assert rel(u[k], ref[k]) <= TOL_SIMT, (case, nrhs, k)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nrhs", [1, 2, 5])
def test_adjoint_matches_oracle(ops, case, nrhs):
    op, fs, sb = ops(case)
    w = complex_normal(fs.n_out, nrhs, seed=12)
    g = gpu_apply(torch, op, w, adjoint=True)
    ref = sb.adjoint(w)
    for k in range(nrhs):
        assert rel(g[k], ref[k]) <= TOL_SIMT, (case, nrhs, k)


def test_adjoint_identity_on_gpu(ops):
    """<K_f g, w> = <g, K_f^* w> with both products taken on the GPU."""
    op, fs, sb = ops(("fio_iso", 64, 2, 4, 24, "polar"))
    g = complex_normal(fs.n_in, 1, seed=1)
    w = complex_normal(fs.n_out, 1, seed=2)
    lhs = np.vdot(w, gpu_apply(torch, op, g))
    rhs = np.vdot(gpu_apply(torch, op, w, adjoint=True), g)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_exact_bf_equals_closed_form_dft(ops):
    """Full-rank factors (r covers every block of the 4^3 grid): the GPU apply equals
    the closed-form 3-D DFT to FP32 accuracy."""
    op, fs, sb = ops(("dft", 4, 3, 2, 64, "none"))
    g = complex_normal(fs.n_in, 2, seed=5)
    ref = D.dft_closed_form(g, 4, 3)
    assert rel(gpu_apply(torch, op, g), ref) <= TOL_SIMT


def test_zero_rhs_is_a_noop(ops, bd):
    op, fs, sb = ops(("dft", 16, 2, 2, 8, "none"))
    u = torch.full((1, fs.n_out), 7.0, dtype=torch.complex64, device="cuda")
    g = torch.zeros((1, fs.n_in), dtype=torch.complex64, device="cuda")
    op.apply(g.data_ptr(), u.data_ptr(), 0, 0, torch.cuda.current_stream().cuda_stream)
    op.check(torch.cuda.current_stream().cuda_stream)
    assert torch.all(u == 7.0)


def test_host_buffers_match_device_buffers(ops):
    op, fs, sb = ops(("dft", 64, 2, 4, 16, "none"))
    g = complex_normal(fs.n_in, 3, seed=8)
    u_dev = gpu_apply(torch, op, g)
    torch.cuda.synchronize()
    u_host = op.apply_host(g.astype(np.complex64), 3, 0, torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(u_host, u_dev.astype(np.complex64))


def test_repeated_applies_are_deterministic(ops):
    op, fs, sb = ops(("fio_iso", 64, 2, 4, 24, "polar"))
    g = complex_normal(fs.n_in, 4, seed=3)
    a = gpu_apply(torch, op, g)
    b = gpu_apply(torch, op, g)
    assert np.array_equal(a, b)


def test_library_builder_end_to_end_small(bd):
    """mbf_build_factors (host FP64) -> device apply vs the oracle's FP64 apply of the
    exported factors, and vs the direct sum within the factorization error."""
    hf = bd.HostFactors.build(2, 64, 4, 24, tree=bd.MBF_TREE_POLAR, kernel="fio_iso")
    fs = export_factors(hf.arrays())
    op = bd.Operator(hf)
    sb = B.SparseBF(fs)
    g = complex_normal(fs.n_in, 2, seed=0)
    u = gpu_apply(torch, op, g)
    uf = sb.apply(g)
    assert rel(u, uf) <= TOL_SIMT
    X, W = P.grid_x(64, 2), P.grid_omega(64, 2)
    ud = D.direct_sum(P.kernel_fio_iso, X, W, g)
    eps = D.rel_err(uf, ud)
    assert D.rel_err(u, ud) <= eps + TOL_SIMT


def test_error_estimate_of_an_exact_factorization(bd):
    """At full rank the factorization is exact (§2.4: every truncation keeps all singular
    values), so the §3.3 estimate is the FP32 rounding of the apply alone; with every
    output sampled it equals the relative error against the full direct sum."""
    hf = bd.HostFactors.build(2, 16, 4, 16, kernel="dft")   # 16-point middle-level nodes
    op = bd.Operator(hf)
    assert op.info().eps == -1.0
    e = op.estimate_error("dft", n_samples=256, seed=3)
    assert 0 < e <= 1e-5
    op.close()
