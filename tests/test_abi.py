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


def test_source_combinations_are_rejected_on_the_host():
    """A source term needs its system (S = k q: advection; the acceleration:
    Euler), the Toro-Titarev solver, linear GRPrec and a finite coefficient."""
    from paper_2602_21911_gb300 import grprec, inputs
    prob, *_ = inputs.sod(20, M=2)
    for bad in (dict(source=inputs.SOURCE_LINEAR, source_coef=1.0),
                dict(source=inputs.SOURCE_GRAVITY, source_coef=1.0, solver=1),
                dict(source=inputs.SOURCE_GRAVITY, source_coef=1.0, recon=1),
                dict(source=inputs.SOURCE_GRAVITY, source_coef=float("nan")),
                dict(source=7, source_coef=1.0)):
        with pytest.raises(grprec.GrpError, match="invalid"):
            grprec.Solver(dict(prob, **bad))
    adv, *_ = inputs.advection_sine(8)
    with pytest.raises(grprec.GrpError, match="invalid"):
        grprec.Solver(dict(adv, source=inputs.SOURCE_GRAVITY, source_coef=1.0))


class _FakeCuda:
    """Stands in for a torch CUDA tensor: only the attributes the buffer
    checks of the allocation-free step read (no GPU, no library call)."""

    def __init__(self, n, dtype="torch.float64", contiguous=True, device=0, addr=1 << 20, cuda=True):
        self.n, self.dtype, self.contiguous, self.addr, self.is_cuda = n, dtype, contiguous, addr, cuda
        self.device = type("Dev", (), {"index": device})()

    def data_ptr(self):
        return self.addr

    def is_contiguous(self):
        return self.contiguous

    def numel(self):
        return self.n


def test_noalloc_buffers_are_checked_before_any_launch():
    from paper_2602_21911_gb300 import grprec, inputs
    prob, *_ = inputs.sod(100, M=2)                      # transmissive: 101 interfaces
    N, nif = 100, 101

    def bufs(**over):
        b = dict(avg_in=_FakeCuda(3 * N, addr=1 << 20), iface_in=_FakeCuda(3 * nif, addr=2 << 20),
                 avg_out=_FakeCuda(3 * N, addr=3 << 20), iface_out=_FakeCuda(3 * nif, addr=4 << 20))
        b.update(over)
        return [b[k] for k in ("avg_in", "iface_in", "avg_out", "iface_out")]

    assert grprec.noalloc_check_buffers(prob, *bufs(), current_device=0) == [1 << 20, 2 << 20, 3 << 20, 4 << 20]
    bad = {
        "CUDA tensor": dict(avg_in=_FakeCuda(3 * N, cuda=False)),
        "float64": dict(iface_in=_FakeCuda(3 * nif, dtype="torch.float32", addr=2 << 20)),
        "contiguous": dict(avg_out=_FakeCuda(3 * N, contiguous=False, addr=3 << 20)),
        "expected": dict(iface_out=_FakeCuda(3 * N, addr=4 << 20)),          # 3 N instead of 3 (N + 1)
        "current device": dict(avg_out=_FakeCuda(3 * N, device=1, addr=3 << 20)),
        "overlap": dict(avg_out=_FakeCuda(3 * N, addr=(1 << 20) + 8)),
    }
    for what, over in bad.items():
        with pytest.raises(grprec.GrpError, match=what):
            grprec.noalloc_check_buffers(prob, *bufs(**over), current_device=0)
    with pytest.raises(grprec.GrpError, match="one domain"):
        two = dict(prob, n_cells=[50, 50])
        grprec.noalloc_check_buffers(two, *bufs(), current_device=0)
    # a numpy array is host memory: rejected
    import numpy as np
    with pytest.raises(grprec.GrpError, match="CUDA tensor"):
        grprec.noalloc_check_buffers(prob, np.zeros(3 * N), *bufs()[1:], current_device=0)
