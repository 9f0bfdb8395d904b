"""The C ABI library builds for sm_103a, loads, and exports every function include/kafmm.h
declares; argument validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kafmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kafmm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_15155_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "kafmm_plan" in names and "kafmm_eval" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_are_rejected_on_the_host(lib):
    lib.kafmm_plan.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_void_p)]
    lib.kafmm_last_error.restype = ctypes.c_char_p
    lib.kafmm_last_error.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p(1)
    # kernel or boundary out of range, p or q out of range, charges + dipoles and quadrupoles
    # with the triply periodic boundary, the wall (alone or with PX / PXY) with a derivative
    # form or Laplace, and the StokesPVel-table kernels (double layer, StokesPVel, their
    # derivative forms) with the singly or doubly periodic boundary
    for args in [(14, 0, 8, 64), (-1, 0, 8, 64), (1, 7, 8, 64), (1, -1, 8, 64), (1, 0, 1, 64), (1, 0, 8, 0),
                 (1, 0, 17, 64), (5, 3, 8, 64), (13, 3, 8, 64), (9, 4, 8, 64), (0, 4, 8, 64), (0, 5, 8, 64),
                 (4, 6, 8, 64), (3, 1, 8, 64), (6, 2, 8, 64), (9, 2, 8, 64), (12, 1, 8, 64)]:
        assert lib.kafmm_plan(*args, ctypes.byref(out)) == -1
        assert out.value is None
        assert len(lib.kafmm_last_error(None)) > 0
    lib.kafmm_eval.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    assert lib.kafmm_eval(None, None, None, 0) == -1


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2010_15155_gb300 import kafmm
    monkeypatch.setattr(kafmm, "_lib", None)
    monkeypatch.setattr(kafmm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        kafmm.lib()


def test_python_constants_match_the_header():
    """Every KAFMM_* enum value the header declares equals the binding's constant."""
    from paper_2010_15155_gb300 import kafmm
    src = open(os.path.join(ROOT, "include", "kafmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(KAFMM_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    assert len(values) > 30
    errors = {v: k for k, v in kafmm.ERRORS.items()}
    for name, v in values.items():
        short = name[len("KAFMM_"):]
        if short.startswith("ERR_"):
            assert errors[name] == v, name
        elif short == "OK":
            assert v == 0
        elif short in ("LAPLACE", "STOKESLET", "RPY", "STOKES_DL", "STOKES_REG", "LAPLACE_QD",
                       "STOKES_PVEL", "STOKES_PVEL_GRAD", "STOKES_PVEL_LAPL", "STOKES_PVEL_TRACTION",
                       "STOKES_DL_GRAD", "STOKES_DL_LAPL", "STOKES_DL_TRACTION", "LAPLACE_QUAD"):
            assert getattr(kafmm, short) == v, name
            assert v in kafmm.KDIM, name
        else:
            assert getattr(kafmm, short) == v, name
