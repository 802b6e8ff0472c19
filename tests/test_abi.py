"""The C-ABI library loads and exports every entry point that include/bie.h declares (CPU only:
no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bie_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1706_07919_gb300 import build
    build.build()
    from paper_1706_07919_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("bie_create", "bie_destroy", "bie_set_geometry", "bie_solve_frequencies", "bie_eval_field",
                 "bie_synthesize", "bie_pulse_spectrum", "bie_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(bie_\w+)", out))
    assert _declared() <= exported


def test_binding_names_match_header(lib):
    from paper_1706_07919_gb300 import binding
    for name in _declared():
        assert callable(getattr(binding, name)), name
    assert set(binding.EXPORTED) == _declared()


def test_version_string_without_gpu(lib):
    from paper_1706_07919_gb300 import binding
    assert "sm_103a" in binding.bie_version()
