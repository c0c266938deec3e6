"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports
every function that include/infft.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "infft.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(infft_[a-zA-Z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2302_00414_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("infft_plan", "infft_weights", "infft_optimize_B", "infft_adjoint", "infft_forward", "infft_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (infft_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_header(libpath):
    import paper_2302_00414_gb300 as L
    lib = L.load()
    for n in declared_functions():
        assert hasattr(lib, n)
    assert set(declared_functions()) <= set(L.EXPORTED) | {"infft_plan_N"}
    assert isinstance(L.last_error(), str)
