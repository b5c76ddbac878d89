"""Every Python module of the repository compiles, including the helpers and
test modules that only GPU runs import."""
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "tests", "*.py")) + glob.glob(os.path.join(ROOT, "oracle", "*.py"))
               + glob.glob(os.path.join(ROOT, "paper_2403_17261_gb300", "*.py"))
               + [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")])


@pytest.mark.parametrize("path", FILES, ids=[os.path.relpath(f, ROOT) for f in FILES])
def test_compiles(path):
    with open(path) as f:
        compile(f.read(), path, "exec")
