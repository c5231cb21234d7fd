"""The C ABI library loads without a GPU and exports every symbol declared in include/."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|const char\*)\s+(ibfem_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("ibfem_create", "ibfem_crit_dt", "ibfem_step", "ibfem_sample", "ibfem_destroy"):
        assert must in names


def test_library_exports_all_declared_symbols():
    import ctypes
    from paper_2501_19013_gb300 import ibfem
    if not os.path.exists(ibfem.LIB_PATH):
        from paper_2501_19013_gb300 import build
        build.build()
    L = ctypes.CDLL(ibfem.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert isinstance(ibfem.lib().ibfem_last_error(), bytes)   # "" until a call fails


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2501_19013_gb300 import ibfem
    monkeypatch.setattr(ibfem, "_lib", None)
    monkeypatch.setattr(ibfem, "LIB_PATH", str(tmp_path / "libibfem.so"))
    with pytest.raises(ImportError):
        ibfem.lib()


# declarations documented by the comment of the declaration right above them
GROUPED = {"ibfem_autotune": "ibfem_set_tile_variant"}


def test_every_entry_point_is_documented():
    """Each declaration in include/ is preceded by its comment (GROUPED: shares the comment
    of the declaration right above it)."""
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", f)).read().splitlines()
        decl = re.compile(r"^\s*(?:int|const char\*)\s+(ibfem_\w+)\s*\(")
        for i, line in enumerate(lines):
            m = decl.match(line)
            if not m:
                continue
            j = i - 1
            while j >= 0 and not lines[j].strip():
                j -= 1
            prev = lines[j].strip()
            pm = decl.match(lines[j])
            grouped = pm is not None and GROUPED.get(m.group(1)) == pm.group(1)
            assert prev.endswith("*/") or grouped, m.group(1)
