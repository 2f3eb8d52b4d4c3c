"""The C-ABI library builds here (no GPU needed), loads, and exports every
function that include/ebr.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ebr.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    names = set(re.findall(r"\b(ebr_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ebr_build_index", "ebr_score_topk", "ebr_submit", "ebr_poll",
                 "ebr_server_create", "ebr_server_destroy", "ebr_expand_query",
                 "ebr_index_export", "ebr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2511_22460_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.ebr_version.restype = ctypes.c_int
    assert lib.ebr_version() > 0
