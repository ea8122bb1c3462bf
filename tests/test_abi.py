"""Host-side checks that need no GPU: the C-ABI library builds, loads, and exports every
entry point include/rbws.h declares; the product package never touches the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"RBWS_API[^;{]*?\b(rbws_\w+)\s*\(", text, flags=re.S))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2311_13862_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for must in ("rbws_problem_create", "rbws_problem_destroy", "rbws_apply_operator",
                 "rbws_offline_greedy", "rbws_solve_batch", "rbws_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(rbws_\w+)\b", out))
    assert set(declared_symbols()) <= exported


def test_errors_without_gpu_are_reported_not_hidden(lib_path):
    from paper_2311_13862_gb300 import rbws
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(rbws.RbwsError):
        rbws.rbws_problem_create((8, 8, 8), (2, 1, 1))


def test_invalid_arguments_are_rejected(lib_path):
    from paper_2311_13862_gb300 import rbws
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_problem_create((1, 8, 8), (2, 1, 1))
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_problem_create((8, 8, 8), (2, 1, 1), Q=3)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_13862_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f
                assert "rbws_oracle" not in text and "liborc" not in text, f


def test_options_default_sets_every_field(lib_path):
    """rbws_options_default must overwrite every field (internal callers rely on it)."""
    import ctypes as C
    from paper_2311_13862_gb300 import rbws
    o = rbws.rbws_options()
    C.memset(C.byref(o), 0xAB, C.sizeof(o))
    rbws._lib().rbws_options_default(C.byref(o))
    assert o.max_iters == 20000 and o.precond == rbws.PREC_JACOBI and o.precision == rbws.FP64
    assert o.max_restarts == 3 and o.inner_tol == 1e-2 and o.max_outer == 10 and o.check_every == 0
    assert o.stream is None and not o.profile
