"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/grprec.h declares (no GPU needed, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grp_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2602_21911_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = declared("grprec.h")
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_without_a_gpu():
    from paper_2602_21911_gb300 import grprec
    assert grprec.grp_status_string(0) == "ok"
    assert "invalid" in grprec.grp_status_string(-1)


def test_invalid_problem_is_rejected_on_the_host():
    from paper_2602_21911_gb300 import grprec, inputs
    prob, *_ = inputs.advection_sine(8)
    for bad in (dict(M=5), dict(M=0), dict(cfl=1.5), dict(cfl=0.0), dict(lam=0.0)):
        with pytest.raises(grprec.GrpError, match="invalid"):
            grprec.Solver(dict(prob, **bad))
    with pytest.raises(grprec.GrpError, match="invalid"):
        grprec.Solver(dict(prob, n_cells=[0]))
