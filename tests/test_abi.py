"""The C-ABI library loads and exports every entry point include/helm.h declares (CPU only)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2112_00087_gb300", "lib", "libhelm.so")


def declared_functions():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_0-9]+)\s*\(", src)))


def ensure_built():
    if not os.path.exists(LIB):
        from paper_2112_00087_gb300 import build
        build.build()


def test_library_exports_every_declared_symbol():
    ensure_built()
    lib = ctypes.CDLL(LIB)
    names = declared_functions()
    assert "helm_solve" in names and "helm_spmv" in names and len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    ensure_built()
    from paper_2112_00087_gb300 import helm
    assert sorted(helm.EXPORTED) == declared_functions()
    for n in declared_functions():
        if n in ("helm_destroy", "helm_matrix_free", "helm_last_error", "helm_sizes", "helm_matrix_csr",
                 "helm_matrix_dia27", "helm_shared_free"):
            continue
        assert hasattr(helm, n), n


def test_argument_errors_need_no_gpu():
    # argument validation happens before any CUDA call
    ensure_built()
    from paper_2112_00087_gb300 import helm
    h = ctypes.c_void_p()
    bad = helm.MeshDesc(0, 4, 4, 1.0, 1.0, 1.0)
    st = helm.LIB.helm_create(ctypes.byref(h), ctypes.byref(bad), ctypes.byref(helm.Phys(340.0, 1.2)), None)
    assert st == helm.HELM_ERR_ARG
    assert b"nx" in helm.LIB.helm_last_error()
    out = (ctypes.c_double * 2)()
    assert helm.LIB.helm_reduce(7, 10, None, None, out, None) == helm.HELM_ERR_ARG


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of the ABI structs have the C sizes and field offsets (plain C, gcc)
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2112_00087_gb300 import helm
    structs = {"helm_solve_opts": helm.SolveOpts, "helm_solve_stats": helm.SolveStats,
               "helm_mesh_desc": helm.MeshDesc, "helm_phys": helm.Phys}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "helm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
