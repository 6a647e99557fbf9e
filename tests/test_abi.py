"""The C-ABI library builds, loads and exports every function include/prnu.h
declares, and the ctypes structures match the header's layout.  CPU only: no
compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "prnu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|uint64_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2207_14507_gb300 as p
    return p.build()


def test_every_declared_symbol_is_exported(libpath):
    names = _declared()
    assert "eis_grid_search" in names and "query_poll" in names and len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_the_header(libpath):
    import paper_2207_14507_gb300 as p
    assert sorted(p.EXPORTED) == _declared()
    L = p.lib()
    for n in _declared():
        assert getattr(L, n) is not None


def test_struct_layouts():
    import paper_2207_14507_gb300 as p
    assert ctypes.sizeof(p.prnu_result) == 32 and p.prnu_result.pce.offset == 16
    assert ctypes.sizeof(p.prnu_grid) == 24
    assert ctypes.sizeof(p.prnu_window) == 16


def test_no_oracle_on_the_product_path():
    """The package neither imports nor names the oracle."""
    pkg = os.path.join(ROOT, "paper_2207_14507_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2207_14507_gb300 as p
    monkeypatch.setattr(p, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(p, "_lib", None)
    with pytest.raises(RuntimeError):
        p.lib()
