"""The C ABI library loads and exports every function include/*.h declares
(CPU-only: no compute call is made)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "defined"):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1112_1805_gb300 import build

    if not build.up_to_date():
        try:
            build.build()
        except RuntimeError as e:  # pragma: no cover - toolkit missing
            pytest.skip(str(e))
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("shfilters_build", "shfilters_destroy", "shfilters_info", "shearlet_analyze", "shearlet_synthesize",
              "seg_admm_init", "seg_admm_step", "seg_admm_solve", "seg_admm_get", "seg_admm_save", "seg_admm_load",
              "seg_admm_destroy"):
        assert n in names, n


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_the_header():
    from paper_1112_1805_gb300 import binding

    for n in declared_functions():
        assert n in binding._SIG, f"{n} has no binding"


def test_argument_errors_without_gpu():
    from paper_1112_1805_gb300 import binding as B

    assert B.shf_version() >= 100
    for H, W, J in [(7, 8, 1), (8, 9, 1), (14, 16, 1), (64, 44, 2), (4096, 64, 2)]:
        with pytest.raises(B.ShearsegError) as ei:
            B.shfilters_build(H, W, J)
        assert ei.value.code == B.SHF_ERR_SIZE
    with pytest.raises(B.ShearsegError) as ei:
        B.shfilters_build(64, 64, 0)
    assert ei.value.code == B.SHF_ERR_ARG
    with pytest.raises(B.ShearsegError) as ei:
        B.seg_admm_step(None, 1)
    assert ei.value.code == B.SHF_ERR_ARG
    assert B.seg_admm_kernel_name(0) == "row_ustep" and B.seg_admm_kernel_name(99) == ""


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors of the header's parameter and plan structs: same size
    # and same offset for every field (a C program compiled against the header
    # prints them)
    import shutil
    import subprocess

    from paper_1112_1805_gb300 import binding as B

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = [B.seg_params, B.seg_plan, B.tv_params, B.nl_params]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "shearseg.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            cname = name.rstrip("_")
            lines.append(f'  printf("{st.__name__} {name} %zu\\n", offsetof({st.__name__}, {cname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert got[(st.__name__, name)] == getattr(st, name).offset, (st.__name__, name)
