"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/ffm.h declares (no GPU needed: nothing here calls into the device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ffm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ffm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_05600_gb300 import build, ffm
    build.build()
    return ffm.lib()


def test_header_declares_plan_apply_destroy():
    names = _declared()
    for n in ("ffm_plan", "ffm_apply", "ffm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1909_05600_gb300 import ffm
    names = _declared()
    assert set(names) == set(ffm.ABI_SYMBOLS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_without_a_device(lib):
    assert lib.ffm_status_str(0) == b"FFM_OK"
    assert lib.ffm_status_str(2) == b"FFM_ENOMEM"
    assert lib.ffm_launch_count() == 0


def test_null_arguments_are_rejected_on_the_host(lib):
    import ctypes as C
    from paper_1909_05600_gb300 import ffm
    h = C.c_void_p()
    rc = lib.ffm_plan(None, 1, 10, None, 1, 10, 0, 0.0, 1e-3, None, None, C.byref(h))
    assert rc == 1 and not h.value
    assert lib.ffm_apply(None, None, 0, 1, None, None) == 1
    lib.ffm_destroy(None)
    info = ffm.Info()
    assert lib.ffm_plan_info(None, C.byref(info)) == 1


def test_python_structs_match_the_header_layout(tmp_path):
    """ffm_opts and ffm_info as the C compiler lays them out (size and the offset of every
    field) equal the ctypes mirrors of the binding."""
    import ctypes
    import subprocess

    from paper_1909_05600_gb300 import ffm

    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ffm.h"', 'int main(void) {']
    for cname, py in (("ffm_opts", ffm.Opts), ("ffm_info", ffm.Info)):
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().split("\n") if l)
    for cname, py in (("ffm_opts", ffm.Opts), ("ffm_info", ffm.Info)):
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)
