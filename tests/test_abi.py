"""The C-ABI library loads and exports every symbol include/ovl.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ovl.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const char \*|ovl_status )\s*(ovl_\w+)\s*\(", text, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    assert "ovl_step" in names and "ovl_scene_upload" in names and len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_2403_17261_gb300 import build as B
    from paper_2403_17261_gb300 import ovl
    B.build()
    lib = ctypes.CDLL(B.LIB)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(ovl.EXPORTED) == _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2403_17261_gb300 import ovl
    with pytest.raises(ovl.OvlError):
        ovl.load_library(str(tmp_path / "missing.so"))


def test_oracle_builds():
    from oracle import oracle as O
    assert os.path.exists(O.build())


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the header's size and field
    offsets (a field added on one side only would shift every later one)."""
    import subprocess
    from paper_2403_17261_gb300 import ovl
    structs = {"ovl_params": ovl.ovl_params, "ovl_scene_desc": ovl.ovl_scene_desc,
               "ovl_stats": ovl.ovl_stats, "ovl_train_desc": ovl.ovl_train_desc}
    lines = []
    for name, py in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in py._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ovl.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, py in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(py), name
        for f in py._fields_:
            assert got[(name, f[0])] == getattr(py, f[0]).offset, (name, f[0])
