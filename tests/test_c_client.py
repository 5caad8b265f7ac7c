"""The C ABI from C: tests/c/abi_check.c, a C99 client of include/chhs.h,
compiled with gcc (-std=c99 -Wall -Wextra -pedantic -Werror, so the header
must be valid C), linked against the in-tree library and run.  It makes only
calls that need no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c99_client_builds_and_runs(tmp_path):
    from paper_1611_02967_gb300 import build, chhs
    build.build()
    libdir = os.path.dirname(chhs.LIB_PATH)
    exe = str(tmp_path / "abi_check")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-o", exe, "-L", libdir, "-lchhs",
           "-Wl,-rpath," + libdir, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi_check: ok" in r.stdout


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes through the ABI has the size and the
    field offsets that a C compiler gives the header's declaration."""
    import ctypes

    from paper_1611_02967_gb300 import chhs
    structs = {"chhs_opts": chhs.chhs_opts, "chhs_tuning": chhs.Tuning, "chhs_request": chhs.chhs_request,
               "chhs_run_desc": chhs.chhs_run_desc}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "chhs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = dict(line.split() for line in subprocess.run([exe], capture_output=True, text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out["%s.%s" % (cname, fname)]) == getattr(py, fname).offset, (cname, fname)


def test_binding_structs_have_every_header_field():
    """The binding's structs declare the header's fields, all of them, in order."""
    import re

    from paper_1611_02967_gb300 import chhs
    src = open(os.path.join(ROOT, "include", "chhs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    structs = {"chhs_opts": chhs.chhs_opts, "chhs_tuning": chhs.Tuning, "chhs_request": chhs.chhs_request,
               "chhs_run_desc": chhs.chhs_run_desc}
    for cname, py in structs.items():
        m = re.search(r"typedef struct \{([^{}]*)\}\s*%s;" % cname, src)
        assert m, cname
        names = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "int tile_w, tile_h", "int n[3]", "const double* phi0"
            head, *rest = decl.split(",")
            names.append(re.findall(r"(\w+)\s*(?:\[\d+\])?\s*$", head)[0])
            names += [re.findall(r"(\w+)", r)[0] for r in rest]
        assert names == [f for f, _ in py._fields_], (cname, names)
