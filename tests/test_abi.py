"""Host-only checks of the C ABI: the library builds and loads without a GPU,
exports every entry point include/om.h declares, the binding covers each of
them, and the CUDA path and the oracle share no code."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "om.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(om_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libom():
    from paper_1410_1921_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libom):
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(libom, n), n


def test_binding_covers_every_declared_symbol():
    import paper_1410_1921_gb300 as P
    assert sorted(P.exported_symbols()) == _declared()


def test_version_string(libom):
    libom.om_version.restype = ctypes.c_char_p
    assert libom.om_version().startswith(b"om-gb300")


def test_cuda_path_and_oracle_share_no_code():
    pkg = os.path.join(ROOT, "paper_1410_1921_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", re.sub(r"#.*|//.*", "", text)), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1410_1921_gb300" not in text and "om.h" not in text, f


def test_synthetic_inputs_hold_no_method_arithmetic():
    text = open(os.path.join(ROOT, "synthetic.py")).read()
    for word in ("import oracle", "paper_1410_1921_gb300", "collide", "knudsen"):
        assert word not in text
