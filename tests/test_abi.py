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


def test_binding_rejects_mismatched_synthesis_buffers_before_launch():
    """The synthesis writes P*M*Nt values of out_dtype: a short or mistyped output buffer is
    rejected by the binding before any call into the library (CPU tensors, no GPU needed)."""
    import numpy as np
    import torch
    from paper_1706_07919_gb300 import binding as B
    Nk, M, P, Nt = 3, 5, 2, 16
    T = torch.zeros((Nk, M), dtype=torch.complex128)
    S = torch.zeros((P, Nt // 2 + 1), dtype=torch.complex128)
    midx = np.arange(1, Nk + 1)
    for fn in (lambda o, d: B.bie_synthesize(0, T, midx, S, Nt, o, d),
               lambda o, d: B.bie_synthesize_noalloc(T, midx, S, Nt, o, d)):
        with pytest.raises(ValueError, match="dtype"):
            fn(torch.zeros((P, M, Nt), dtype=torch.float32), 0)
        with pytest.raises(ValueError, match="elements"):
            fn(torch.zeros((P, M, Nt - 1), dtype=torch.float64), 0)
        with pytest.raises(ValueError, match="out_dtype"):
            fn(torch.zeros((P, M, Nt), dtype=torch.float64), 2)
    with pytest.raises(ValueError, match="Nt/2"):
        B.bie_synthesize(0, T, midx, torch.zeros((P, Nt // 2), dtype=torch.complex128), Nt,
                         torch.zeros((P, M, Nt), dtype=torch.float64), 0)
    with pytest.raises(ValueError, match="T_out"):
        B.bie_eval_field(0, torch.zeros((M, 3), dtype=torch.float64), np.ones(Nk), None, 0,
                         torch.zeros((Nk, M - 1), dtype=torch.complex128))


def test_binding_constants_match_header():
    """Every integer constant of include/bie.h (return codes, modes, report flags, the network's
    parameter count) has the same value in the binding; report flags are distinct bits."""
    from paper_1706_07919_gb300 import binding as B
    txt = open(os.path.join(ROOT, "include", "bie.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in
              re.finditer(r"^#define (BIE_\w+)\s+\(?(-?\d+)u?\)?", txt, flags=re.M)}
    assert {"BIE_OK", "BIE_ERR_TIMEOUT", "BIE_MODE_MIXED", "BIE_FLAG_FP32_REFACTOR"} <= set(consts)
    for name, value in consts.items():
        assert getattr(B, name) == value, name
    flags = [v for n, v in consts.items() if n.startswith("BIE_FLAG_")]
    assert all(v & (v - 1) == 0 for v in flags) and len(set(flags)) == len(flags)


def test_every_option_is_documented():
    """Every name bie_set_option accepts is documented in include/bie.h and vice versa (the option
    table of the header against the names compared in the implementation; CPU only)."""
    src = open(os.path.join(ROOT, "paper_1706_07919_gb300", "csrc", "capi.cu")).read()
    accepted = set(re.findall(r'n == "([a-z0-9_.]+)"', src))
    hdr = open(os.path.join(ROOT, "include", "bie.h")).read()
    documented = set(re.findall(r'^ \*   "([a-z0-9_.]+)"', hdr, flags=re.M))
    documented |= set(re.findall(r'^ \*   "[a-z0-9_.]+", "([a-z0-9_.]+)"', hdr, flags=re.M))
    assert accepted and accepted == documented, (accepted - documented, documented - accepted)
