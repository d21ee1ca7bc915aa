"""The C boundary from plain C: tests/c_abi_client.c includes include/mbf.h as C99
(-Wall -Wextra -pedantic -Werror), links libmbf.so and runs the host-side calls --
a build with a caller-written entry function, its factor-file checkpoint, operator
creation (MBF_ERR_CUDA without a GPU: no CPU apply) and the error codes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    pytest.importorskip("torch")
    from paper_1509_07925_gb300 import buildlib
    lib = buildlib.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path / "client"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                         "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_client.c"),
                         "-o", str(exe), f"-L{libdir}", "-lmbf", "-lm", f"-Wl,-rpath,{libdir}"],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe), str(tmp_path / "dft16.mbf")], capture_output=True, text=True, timeout=600)
    print(run.stdout)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "0 failed" in run.stdout
    assert (tmp_path / "dft16.mbf").exists()
