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
