"""The Python binding's mirror of fsi_exec_desc (include/ibfsi.h) has the C layout: a host program built against
the header prints the struct's size and every field's offset, which must equal the ctypes structure's (no GPU;
needs a C compiler)."""

import shutil
import subprocess

import pytest

from paper_2103_06415_gb300 import _lib

FIELDS = ["precision", "stream", "max_iters", "tol", "history_cap", "use_graph", "b0_method", "dst_method",
          "coupling", "krylov_tol", "krylov_max_iters", "fsi_solver", "dev_alloc", "dev_free", "dev_alloc_user"]


def test_exec_desc_layout_matches_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    import os
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"ibfsi.h\"\nint main(void) {\n"
                   "  printf(\"size %zu\\n\", sizeof(fsi_exec_desc));\n" +
                   "".join("  printf(\"%s %%zu\\n\", offsetof(fsi_exec_desc, %s));\n" % (f, f) for f in FIELDS) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    assert int(out["size"]) == __import__("ctypes").sizeof(_lib.ExecDesc)
    for f in FIELDS:
        assert int(out[f]) == getattr(_lib.ExecDesc, f).offset, f
