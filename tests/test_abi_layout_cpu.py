"""The ctypes binding mirrors the C structs of include/mbf.h field for field: a C99
program compiled against the header prints every struct's size and every field's
offset, and each must equal the binding's (a field added to one side and not the
other would shift everything after it)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> binding class name
PAIRS = {
    "mbf_problem_t": "Problem",
    "mbf_build_opts_t": "BuildOpts",
    "mbf_factors_t": "Factors",
    "mbf_op_info_t": "OpInfo",
    "mbf_profile_t": "Profile",
    "mbf_msbf_info_t": "MsbfInfo",
    "mbf_tune_result_t": "TuneResult",
    "mbf_server_opts_t": "ServerOpts",
    "mbf_request_status_t": "RequestStatus",
    "mbf_server_stats_t": "ServerStats",
}


def test_binding_structs_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1509_07925_gb300 import binding as bd
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mbf.h"', "int main(void) {"]
    for cname, pyname in PAIRS.items():
        cls = getattr(bd, pyname)
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                         "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            cname, key, val = ln.split()
            got[(cname, key)] = int(val)
    for cname, pyname in PAIRS.items():
        cls = getattr(bd, pyname)
        assert got[(cname, "size")] == C.sizeof(cls), (cname, got[(cname, "size")], C.sizeof(cls))
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
