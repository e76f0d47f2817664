"""CPU checks of the boundary: libsf builds for sm_103a, loads, and exports every
function that the headers under include/ declare.  No GPU calls."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sf.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions(header=None):
    names = set()
    for path in [header] if header else HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(sf_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_six_calls_and_exports():
    assert HEADER in HEADERS and len(HEADERS) >= 2
    names = declared_functions(HEADER)
    for must in ["sf_create", "sf_apply_clifford", "sf_apply_nonclifford", "sf_coalesce", "sf_measure",
                 "sf_amplitude", "sf_destroy", "sf_get_tableau", "sf_get_frame"]:
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_1712_03554_gb300 import _build
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_marshals_every_declared_call():
    from paper_1712_03554_gb300 import sf
    lib = sf.load()
    for name in declared_functions():
        assert getattr(lib, name).argtypes is not None or name == "sf_last_error", name


@pytest.mark.parametrize("header", HEADERS, ids=os.path.basename)
def test_each_declaration_is_documented(header):
    text = open(header).read()
    for name in declared_functions(header):
        m = re.search(r"\n(?:const )?[a-z_0-9]+\*? ?\*?" + name + r"\(", text)
        assert m, name
        idx = m.start()
        before = text[max(0, idx - 600):idx]
        assert "/*" in before or "*/" in before, name


def test_invalid_args_without_gpu_are_rejected_on_the_host():
    from paper_1712_03554_gb300 import sf
    lib = sf.load()
    h = ctypes.c_void_p()
    assert lib.sf_create(0, 16, None, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_create(2000, 16, None, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_create(4, 0, None, ctypes.byref(h)) == sf.SF_EINVAL
    assert lib.sf_destroy(None) == sf.SF_EINVAL
    assert lib.sf_apply_program(None, None, 0, 0.0, 0, None, None) == sf.SF_EINVAL
    assert lib.sf_apply_program_grid(None, None, 0, 0.0, None) == sf.SF_EINVAL
    assert lib.sf_last_error(None)


def test_multiframe_invalid_args_without_gpu():
    from paper_1712_03554_gb300 import sf
    lib = sf.load()
    m = ctypes.c_void_p()
    assert lib.sf_mf_create(0, 16, 4, None, ctypes.byref(m)) == sf.SF_EINVAL
    assert lib.sf_mf_create(64, 16, 4, None, ctypes.byref(m)) == sf.SF_EINVAL
    assert lib.sf_mf_create(8, 16, 0, None, ctypes.byref(m)) == sf.SF_EINVAL
    assert lib.sf_mf_destroy(None) == sf.SF_EINVAL
    assert lib.sf_mf_apply_clifford(None, None, 0) == sf.SF_EINVAL
    assert lib.sf_mf_apply_toffoli(None, 0, 1, 2, 0.0) == sf.SF_EINVAL
    assert lib.sf_mf_apply_cr(None, 0, 1, 0.5, 0.0) == sf.SF_EINVAL
    assert lib.sf_mf_apply_nonclifford(None, 0, 0, 0, 0.0, 0.0) == sf.SF_EINVAL
    assert lib.sf_mf_coalesce(None, 0.0, None, None) == sf.SF_EINVAL
    assert lib.sf_mf_count(None, None, None) == sf.SF_EINVAL
    assert lib.sf_mf_amplitude(None, None, None, None) == sf.SF_EINVAL
    assert lib.sf_mf_frame(None, 0, None) == sf.SF_EINVAL
    assert lib.sf_mf_launches(None) == 0
    assert lib.sf_mf_last_error(None)

