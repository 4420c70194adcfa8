"""The C-ABI library builds and exports every function include/fe.h declares
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"^\s*(?:int|const char\*|double)\s+(\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fe_mesh_create", "fe_assemble_residual", "fe_assemble_tangent", "nl_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2203_05610_gb300 import build as B
    so = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    ctypes.CDLL(so)  # loads without a GPU


def test_binding_signatures_cover_the_header():
    import paper_2203_05610_gb300 as fe
    assert set(_declared()) == set(fe.SIGNATURES)
