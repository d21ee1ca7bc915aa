"""Factor files (the checkpoint of the host construction), on CPU: a saved and reloaded
factor set is bit-identical to the one built; truncated, foreign or corrupted files and
failed writes are reported as MBF_ERR_IO, never loaded."""
import os

import numpy as np
import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bd():
    from paper_1509_07925_gb300 import buildlib
    buildlib.build()
    from paper_1509_07925_gb300 import binding
    return binding


CASES = [  # (dim, n, L, r, tree, kernel)
    (2, 16, 2, 8, "uniform", "dft"),
    (2, 16, 4, 8, "polar", "fio_iso"),
    (3, 8, 2, 8, "uniform", "dft"),
]


def _build(bd, case):
    dim, n, L, r, tree, kern = case
    t = {"uniform": bd.MBF_TREE_UNIFORM, "polar": bd.MBF_TREE_POLAR}[tree]
    return bd.HostFactors.build(dim, n, L, r, tree=t, kernel=kern, seed=11)


def _same(a, b):
    for k in ("d", "L", "n_out", "n_in", "nnz"):
        assert a[k] == b[k], k
    for k in ("x_perm", "x_off", "w_perm", "w_off", "RU", "RV", "UL", "VL", "S"):
        assert a[k].dtype == b[k].dtype and np.array_equal(a[k], b[k]), k
    assert len(a["G"]) == len(b["G"]) and len(a["H"]) == len(b["H"])
    for x, y in zip(a["G"] + a["H"], b["G"] + b["H"]):
        assert x.shape == y.shape and np.array_equal(x.view(np.float64), y.view(np.float64))


@pytest.mark.parametrize("case", CASES)
def test_round_trip_is_bit_identical(bd, case, tmp_path):
    hf = _build(bd, case)
    p = tmp_path / "f.mbf"
    hf.save(p)
    assert p.exists() and not (tmp_path / "f.mbf.tmp").exists()
    back = bd.HostFactors.load(p)
    _same(hf.arrays(), back.arrays())
    # a reloaded set saves to the same bytes
    p2 = tmp_path / "g.mbf"
    back.save(p2)
    assert p.read_bytes() == p2.read_bytes()
    back.close()
    hf.close()


def _io_error(bd, fn):
    with pytest.raises(bd.MbfError) as e:
        fn()
    assert e.value.code == bd.MBF_ERR_IO, str(e.value)
    return str(e.value)


@pytest.fixture(scope="module")
def saved(bd, tmp_path_factory):
    hf = _build(bd, CASES[1])
    p = tmp_path_factory.mktemp("ff") / "polar.mbf"
    hf.save(p)
    hf.close()
    return p.read_bytes()


def test_every_single_byte_flip_in_the_payload_is_caught(bd, saved, tmp_path):
    rng = np.random.default_rng(3)
    p = tmp_path / "bad.mbf"
    for off in sorted(set(rng.integers(64, len(saved) - 8, size=12).tolist())):
        b = bytearray(saved)
        b[off] ^= 0x10
        p.write_bytes(bytes(b))
        msg = _io_error(bd, lambda: bd.HostFactors.load(p))
        assert "checksum" in msg or "corrupt" in msg or "does not match" in msg


def test_flipped_checksum_is_caught(bd, saved, tmp_path):
    b = bytearray(saved)
    b[-1] ^= 1
    p = tmp_path / "bad.mbf"
    p.write_bytes(bytes(b))
    assert "checksum" in _io_error(bd, lambda: bd.HostFactors.load(p))


@pytest.mark.parametrize("keep", [0, 10, 64, 200, -8, -1])
def test_truncated_file(bd, saved, tmp_path, keep):
    p = tmp_path / "short.mbf"
    p.write_bytes(saved[:keep] if keep >= 0 else saved[:len(saved) + keep])
    _io_error(bd, lambda: bd.HostFactors.load(p))


def test_trailing_bytes(bd, saved, tmp_path):
    p = tmp_path / "long.mbf"
    p.write_bytes(saved + b"\0" * 16)
    assert "does not match" in _io_error(bd, lambda: bd.HostFactors.load(p))


def test_header_fields(bd, saved, tmp_path):
    p = tmp_path / "h.mbf"
    for off, val, word in [(0, b"XBFFACT1", "not a factor file"), (8, (2).to_bytes(4, "little"), "version"),
                           (12, (0x04030201).to_bytes(4, "little"), "byte order"),
                           (16, (5).to_bytes(4, "little"), "header")]:
        b = bytearray(saved)
        b[off:off + len(val)] = val
        p.write_bytes(bytes(b))
        assert word in _io_error(bd, lambda: bd.HostFactors.load(p))


def test_missing_file_and_unwritable_path(bd, tmp_path):
    _io_error(bd, lambda: bd.HostFactors.load(tmp_path / "none.mbf"))
    hf = _build(bd, CASES[0])
    _io_error(bd, lambda: hf.save(tmp_path / "no_such_dir" / "f.mbf"))
    hf.close()


def test_inconsistent_factor_set_is_not_written(bd, tmp_path):
    hf = _build(bd, CASES[0])
    a = hf.arrays()
    x_perm = a["x_perm"].copy()
    x_perm[0] = x_perm[1]   # not a permutation
    bad = bd.HostFactors.from_arrays(a["d"], a["L"], a["n_out"], a["n_in"], x_perm, a["x_off"], a["w_perm"],
                                     a["w_off"], a["RU"], a["RV"], a["UL"], a["VL"], a["G"], a["H"], a["S"])
    with pytest.raises(bd.MbfError) as e:
        bad.save(tmp_path / "x.mbf")
    assert e.value.code == bd.MBF_ERR_INVALID
    assert not os.path.exists(tmp_path / "x.mbf") and not os.path.exists(tmp_path / "x.mbf.tmp")
    hf.close()


def test_build_option_writes_then_loads_the_checkpoint(bd, tmp_path):
    """opts.factor_file: the first build writes the file, the second loads it (a damaged
    file makes the second build fail, so it was read rather than rebuilt)."""
    p = tmp_path / "ck.mbf"
    kw = dict(tree=bd.MBF_TREE_POLAR, kernel="fio_iso", seed=5)
    a = bd.HostFactors.build(2, 16, 4, 8, factor_file=p, **kw)
    assert p.exists()
    b = bd.HostFactors.build(2, 16, 4, 8, factor_file=p, **kw)
    _same(a.arrays(), b.arrays())
    raw = bytearray(p.read_bytes())
    raw[len(raw) // 2] ^= 0x01
    p.write_bytes(bytes(raw))
    _io_error(bd, lambda: bd.HostFactors.build(2, 16, 4, 8, factor_file=p, **kw))
    a.close()
    b.close()


def test_build_option_rejects_a_checkpoint_of_another_problem(bd, tmp_path):
    p = tmp_path / "ck.mbf"
    bd.HostFactors.build(2, 16, 2, 8, factor_file=p).close()
    for args, kw in [((2, 32, 2, 8), {}), ((2, 16, 4, 8), {}), ((2, 16, 2, 4), {}),
                     ((2, 16, 2, 8), dict(tree=bd.MBF_TREE_POLAR))]:
        with pytest.raises(bd.MbfError) as e:
            bd.HostFactors.build(*args, factor_file=p, **kw)
        assert e.value.code == bd.MBF_ERR_INVALID and "another problem" in str(e.value)
    # a square Omega tree over a point subset: the subset is part of the problem
    idx = np.arange(0, 256, 2)
    q = tmp_path / "sq.mbf"
    kw = dict(tree=bd.MBF_TREE_SQUARE, kernel="fio_iso", w_lo=-8.0, w_side=16.0)
    bd.HostFactors.build(2, 16, 2, 8, factor_file=q, w_index=idx, **kw).close()
    bd.HostFactors.build(2, 16, 2, 8, factor_file=q, w_index=idx, **kw).close()
    with pytest.raises(bd.MbfError) as e:
        bd.HostFactors.build(2, 16, 2, 8, factor_file=q, w_index=idx + 1, **kw)
    assert e.value.code == bd.MBF_ERR_INVALID and "point set" in str(e.value)


def test_build_option_rejects_a_checkpoint_of_another_kernel(bd, tmp_path):
    """A 2-D DFT and a 2-D FIO without polar transform share n, L, trees and ranks; the
    kernel record written beside the file tells them apart, and a file without one
    (written by mbf_factors_save, not by a build) is not taken for a build."""
    p = tmp_path / "k.mbf"
    bd.HostFactors.build(2, 16, 2, 8, kernel="dft", factor_file=p).close()
    assert (tmp_path / "k.mbf.kernel").exists()
    bd.HostFactors.build(2, 16, 2, 8, kernel="dft", factor_file=p).close()   # same kernel: loads
    with pytest.raises(bd.MbfError) as e:
        bd.HostFactors.build(2, 16, 2, 8, kernel="fio_iso", factor_file=p)
    assert e.value.code == bd.MBF_ERR_INVALID and "kernel" in str(e.value)
    (tmp_path / "k.mbf.kernel").unlink()
    with pytest.raises(bd.MbfError) as e:
        bd.HostFactors.build(2, 16, 2, 8, kernel="dft", factor_file=p)
    assert e.value.code == bd.MBF_ERR_INVALID and "no kernel record" in str(e.value)


def test_array_views_equal_the_copies(bd):
    """HostFactors.arrays(copy=False) gives views of the library's arrays (no second copy
    of a large factor set) with the same contents as the copies."""
    hf = bd.HostFactors.build(2, 32, 4, 8, tree=bd.MBF_TREE_POLAR, kernel="fio_iso", seed=3)
    a, v = hf.arrays(), hf.arrays(copy=False)
    for key in ("UL", "VL", "S", "x_perm", "w_off"):
        assert np.array_equal(a[key], v[key]), key
    for q in range(len(a["G"])):
        assert np.array_equal(a["G"][q], v["G"][q]) and np.array_equal(a["H"][q], v["H"][q])
    assert not v["G"][0].flags["OWNDATA"] and a["G"][0].flags["OWNDATA"]
    hf.close()
