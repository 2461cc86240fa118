"""Host-side checks of the C-ABI library (no GPU needed)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_07094_gb300 import build
    return C.CDLL(build.build())


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(df_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "df_chem_integrate" in names and "df_mech_load" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2210_07094_gb300 import _lib
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(_declared()) <= bound


def test_error_strings_and_defaults(lib):
    lib.df_strerror.restype = C.c_char_p
    assert lib.df_strerror(0) == b"success"
    assert lib.df_strerror(-4) == b"invalid mechanism"
    from paper_2210_07094_gb300 import _lib
    o = _lib.default_opts()
    assert o.rtol > 0 and o.max_substeps > 0 and o.method == 0


def test_mech_load_rejects_bad_files(lib, tmp_path):
    """Parsing errors are reported before any device work."""
    from paper_2210_07094_gb300 import _lib
    L = _lib.load()
    h = C.c_void_p()
    assert L.df_mech_load(b"/nonexistent/mech.json", C.byref(h)) == -4
    bad = tmp_path / "bad.json"
    bad.write_text('{"species": [1, 2], "reactions": []')
    assert L.df_mech_load(str(bad).encode(), C.byref(h)) == -4
    bad.write_text('{"species": [{"name": "A", "W": 1.0, "nasa7": [1,2,3]}], "reactions": []}')
    assert L.df_mech_load(str(bad).encode(), C.byref(h)) == -4
    buf = C.create_string_buffer(256)
    L.df_get_last_error_detail(buf, 256)
    assert b"nasa7" in buf.value
    assert L.df_mech_load(None, C.byref(h)) == -1
