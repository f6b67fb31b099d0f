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


# The binding's ctypes structures against the C compiler's view of
# include/om.h: size and every field's offset (a field added on one side
# only, or in another order, shifts the ones after it).
STRUCTS = ("om_domain", "om_recon_params", "om_flow_params", "om_diff_params", "om_run_info",
           "om_slip_corrections", "om_structure_results")


def test_abi_structures_match_the_header(tmp_path):
    import shutil
    import subprocess

    import paper_1410_1921_gb300 as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "om.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(P, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for s in STRUCTS:
        cls = getattr(P, s)
        assert got[(s, "size")] == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert got[(s, f)] == getattr(cls, f).offset, (s, f)
