"""The binding's ctypes structs have the layout of the C structs in
include/ebr.h: every field at the same offset with the same size, and the
same total size (compiled with the host C compiler, no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("IndexDesc", "ebr_index_desc"), ("IndexInfo", "ebr_index_info"),
         ("CrossDesc", "ebr_cross_desc"), ("QueryC", "ebr_query"),
         ("ServerCfg", "ebr_server_cfg"), ("ServerStats", "ebr_server_stats"),
         ("Profile", "ebr_profile")]


def _c_layouts(tmp_path, ebr):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ebr.h"', "int main(void) {"]
    for py, c in PAIRS:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (c, c))
        for name, _ in getattr(ebr, py)._fields_:
            lines.append('  printf("%s %s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s *)0)->%s));'
                         % (c, name, c, name, c, name))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        parts = line.split()
        if parts[1] == "size":
            res[(parts[0], None)] = int(parts[2])
        else:
            res[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return res


def test_ctypes_structs_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    from paper_2511_22460_gb300 import ebr
    lay = _c_layouts(tmp_path, ebr)
    for py, c in PAIRS:
        cls = getattr(ebr, py)
        assert lay[(c, None)] == ctypes.sizeof(cls), (py, c)
        for name, _ in cls._fields_:
            f = getattr(cls, name)
            assert lay[(c, name)] == (f.offset, f.size), (py, name, lay[(c, name)],
                                                          (f.offset, f.size))
