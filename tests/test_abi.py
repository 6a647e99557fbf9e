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


def test_similarity_from_homography_matches_the_oracle(libpath):
    """Host-only entry point (no CUDA call): the start estimate the library
    derives from a co-registration equals the oracle's polar-decomposition fit,
    and malformed homographies are rejected with PRNU_EINVAL."""
    import numpy as np
    import paper_2207_14507_gb300 as p
    from oracle import prnu_oracle as oracle
    rng = np.random.default_rng(11)
    for _ in range(50):
        lam, th = rng.uniform(0.8, 1.2), rng.uniform(-20, 20)
        t = np.deg2rad(th)
        Hm = np.array([[lam * np.cos(t), -lam * np.sin(t), rng.uniform(-50, 50)],
                       [lam * np.sin(t), lam * np.cos(t), rng.uniform(-50, 50)], [0, 0, 1.0]])
        Hm[:2, :2] += rng.normal(0, 0.02, (2, 2))
        Hm[2, :2] = rng.normal(0, 1e-4, 2)
        Hm *= rng.uniform(0.5, 2.0)
        l_c, t_c = p.similarity_from_homography(Hm)
        l_o, t_o = oracle.similarity_from_homography(Hm)
        # both round a double to float32; the doubles differ in the last bits
        assert abs(l_c - np.float32(l_o)) <= abs(np.spacing(np.float32(l_o)))
        assert abs(t_c - np.float32(t_o)) <= abs(np.spacing(np.float32(t_o)))
    for bad in (np.zeros((3, 3)), np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1.0]]),
                np.array([[np.nan, 0, 0], [0, 1, 0], [0, 0, 1.0]])):
        with pytest.raises(p.PrnuError, match="PRNU_EINVAL"):
            p.similarity_from_homography(bad)
