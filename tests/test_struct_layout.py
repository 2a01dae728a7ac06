"""The ctypes mirrors of the C ABI structs have the field order and offsets of include/tm.h."""
import ctypes
import os
import re
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def c_offsets(struct, fields):
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"tm.h\"\nint main(){\n"
    src += f'printf("%zu\\n", sizeof({struct}));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof({struct}, {f}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return [int(v) for v in out]


def test_ctypes_structs_match_the_header():
    from paper_1311_4462_gb300 import _lib as L
    for cls, name in ((L.tm_params, "tm_params"), (L.tm_field, "tm_field"), (L.tm_solver_params, "tm_solver_params"),
                      (L.tm_solver_stats, "tm_solver_stats")):
        names = [f[0] for f in cls._fields_]
        got = c_offsets(name, names)
        assert got[0] == ctypes.sizeof(cls), name
        assert got[1:] == [getattr(cls, n).offset for n in names], name
