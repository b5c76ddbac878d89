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
