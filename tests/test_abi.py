"""The C-ABI library builds, loads and exports every symbol ``include/sfm.h``
declares (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_6923_gb300 import _build, sfm
    if not os.path.exists(sfm.LIB_PATH):
        _build.build()
    return sfm.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "sfm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sfm_[a-z_]+)\s*\(", txt)))


def test_header_declares_what_the_binding_lists():
    from paper_1406_6923_gb300 import sfm
    assert _declared() == sorted(sfm.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_last_error_without_handle_is_callable(lib):
    assert isinstance(lib.sfm_last_error(None), bytes)


def test_binding_fails_loudly_without_the_library():
    from paper_1406_6923_gb300 import sfm
    saved = sfm._lib
    try:
        sfm._lib = None
        with pytest.raises(ImportError):
            sfm.load(os.path.join(ROOT, "no_such_directory", "libsfm.so"))
    finally:
        sfm._lib = saved


def test_checkpoint_calls_reject_a_null_handle(lib):
    import ctypes as C
    from paper_1406_6923_gb300 import sfm
    n = C.c_size_t(0)
    assert lib.sfm_checkpoint(None, None, C.byref(n)) == sfm.SFM_ERR_ARG
    assert lib.sfm_restore(None, None, 0) == sfm.SFM_ERR_ARG


def test_read_probe_rejects_bad_arguments_before_any_device_call(lib):
    import ctypes as C
    from paper_1406_6923_gb300 import sfm
    v = C.c_double(0.0)
    assert lib.sfm_probe_read_gbs(0, 8, 4, C.byref(v)) == sfm.SFM_ERR_ARG       # fewer than 16 bytes
    assert lib.sfm_probe_read_gbs(0, 1 << 20, 0, C.byref(v)) == sfm.SFM_ERR_ARG  # no repeat
    assert lib.sfm_probe_read_gbs(0, 1 << 20, 4, None) == sfm.SFM_ERR_ARG        # no output
    assert b"bad arguments" in lib.sfm_last_error(None)
