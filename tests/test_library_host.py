"""Host-side checks of the C-ABI library (no GPU needed).

The library builds for sm_103a, loads, and exports every function that
include/pt2.h declares; without a GPU, pt2_create fails with a status code
and a message instead of crashing.
"""

import ctypes
import os
import re

import pytest

from paper_1808_02049_gb300 import build, pt2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return pt2.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pt2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pt2_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(pt2.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_library_is_built_for_sm103a(lib):
    out = os.popen(f"cuobjdump --list-elf {pt2.LIB_PATH} 2>/dev/null").read()
    if not out:
        pytest.skip("cuobjdump not available")
    assert "sm_103a" in out


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES", None) not in ("", None) or
                    os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_create_without_gpu_reports_an_error(lib):
    with pytest.raises(pt2.Pt2Error) as e:
        pt2.pt2_create(0)
    assert e.value.code in (pt2.PT2_ERR_CUDA, pt2.PT2_ERR_INVALID)
    assert pt2.pt2_last_error(None)


@pytest.mark.parametrize("struct", [pt2.pt2_opts, pt2.pt2_result])
def test_binding_structs_match_the_header_layout(struct, tmp_path):
    # the C compiler's size and field offsets of each struct the binding
    # mirrors, against ctypes' (a field added on one side only fails here)
    name = struct.__name__
    fields = [f for f, _ in struct._fields_]
    src = tmp_path / "layout.c"
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pt2.h"', "int main(void) {",
             f'    printf("size %zu\\n", sizeof({name}));']
    lines += [f'    printf("{f} %zu\\n", offsetof({name}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess

    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                     check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(struct)
    for f in fields:
        assert int(out[f]) == getattr(struct, f).offset, f
