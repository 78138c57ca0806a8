"""CPU-side checks of the C ABI library: it builds for sm_103a, loads without a
GPU, and exports every function that include/dmrg.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dmrg.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:dmrg_status|void|int|long long|const char \*)\s*\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_03960_gb300.build import build
    return build()


def test_header_declares_hot_path_calls():
    names = header_functions()
    for n in ["dmrg_build_mpo", "dmrg_sweep", "bond_update", "svd_truncate", "entropy_pid_step"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    for n in header_functions():
        assert hasattr(L, n)
    L.dmrg_mpo_dim.restype = ctypes.c_int
    assert [L.dmrg_mpo_dim(m) for m in (0, 1, 2, 7)] == [5, 8, 3, -1]


def test_binding_lists_header_symbols():
    import paper_2604_03960_gb300 as G
    assert sorted(G.exported_symbols()) == header_functions()


def test_library_targets_sm103a(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_ctypes_structs_match_header(tmp_path):
    """The binding's ctypes mirrors have the header's sizes and field offsets
    (a mismatch would silently misread every record after the first)."""
    import paper_2604_03960_gb300 as G
    pairs = [("dmrg_params", G.Params), ("dmrg_model_params", G.ModelParams), ("dmrg_ctrl_state", G.CtrlState),
             ("dmrg_sweep_record", G.SweepRecord), ("dmrg_visit_record", G.VisitRecord)]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "dmrg.h"', 'int main(void){']
    for cname, py in pairs:
        src.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            src.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
