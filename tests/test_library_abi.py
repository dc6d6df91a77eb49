"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports
every function include/fgr.h declares, and the ctypes structures of the
binding have the C layout."""

import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fgr.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fgr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_21785_gb300 import _build, fgr
    _build.build()
    return fgr.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fgr_create", "fgr_destroy", "fgr_propagate", "fgr_reconstruct_direct",
                     "fgr_reconstruct_fggc", "fgr_submit", "fgr_poll", "fgr_last_error"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    from paper_2504_21785_gb300 import fgr
    names = _declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fgr.SIGNATURES), set(names) ^ set(fgr.SIGNATURES)


def test_ctypes_layout_matches_c(tmp_path):
    # compile a C program against include/fgr.h printing sizeof/offsetof
    import ctypes
    from paper_2504_21785_gb300 import fgr
    structs = {"fgr_grid": fgr.fgr_grid, "fgr_options": fgr.fgr_options,
               "fgr_packets": fgr.fgr_packets, "fgr_potential": fgr.fgr_potential,
               "fgr_info": fgr.fgr_info, "fgr_stats": fgr.fgr_stats,
               "fgr_request": fgr.fgr_request, "fgr_result": fgr.fgr_result, "fgr_axis": fgr.fgr_axis}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fgr.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out["%s.%s" % (name, fname)]) == getattr(cls, fname).offset, (name, fname)


def test_default_options_without_gpu(lib):
    from paper_2504_21785_gb300 import fgr
    o = fgr.fgr_default_options()
    assert (o.nq, o.np, o.precision) == (4, 2, fgr.FGR_FP64)
    assert abs(o.cq - 0.5) < 1e-15 and abs(o.cp - 0.39269908169872414) < 1e-15


def test_missing_library_fails_loudly(tmp_path):
    from paper_2504_21785_gb300 import fgr
    saved = fgr._lib
    fgr._lib = None
    try:
        with pytest.raises(RuntimeError):
            fgr.load(str(tmp_path / "nope.so"))
    finally:
        fgr._lib = saved
