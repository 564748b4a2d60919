"""The C-ABI library loads and exports every symbol include/qrkit.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qrkit.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qrkit_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1802_03773_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared()
    for must in ("qrkit_create", "qrkit_destroy", "qrkit_plan", "qrkit_factor_solve",
                 "qrkit_last_error", "qrkit_sync_status"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1802_03773_gb300 import qrkit
    assert sorted(qrkit.declared_symbols()) == declared()


def test_status_strings(lib):
    f = lib.qrkit_status_string
    f.restype = ctypes.c_char_p
    assert f(0) == b"QRKIT_OK"
    assert f(8) == b"QRKIT_EUNSUPPORTED"


def test_create_rejects_bad_arguments(lib):
    """Argument checks run on the host before any CUDA call."""
    f = lib.qrkit_create
    f.restype = ctypes.c_int
    assert f(None, 0, None, 1) == 1
    h = ctypes.c_void_p()
    assert f(ctypes.byref(h), 0, None, 7) == 1


def test_every_entry_point_cites_its_passage():
    """Each declaration's comment names the paper passage it implements, or says it has none."""
    src = open(HEADER).read()
    decls = [(m.start(), m.group(1)) for m in
             re.finditer(r"\n(?:qrkit_status|int64_t|const char\*|void)\s+(qrkit_[a-z0-9_]+)\(", src)]
    missing = []
    prev = 0
    for pos, name in decls:
        seg = src[prev:pos]
        comment = seg[seg.rfind("/*"):] if "/*" in seg else ""
        comment = re.sub(r"\s*\n\s*\*\s*", " ", comment)     # join the comment's lines
        if not re.search(r"Sec\.|Eq\.|not in the paper|no paper counterpart|paper has no counterpart",
                         comment, flags=re.I):
            missing.append(name)
        prev = pos
    assert not missing, missing
