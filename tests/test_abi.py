"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/coarse.h declares.

No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "coarse.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(coarse_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2205_09104_gb300 import build
    return build()


def test_header_lists_the_boundary():
    names = _declared()
    for n in ["coarse_op_create", "coarse_op_update", "coarse_op_destroy", "coarse_apply", "coarse_solve",
              "coarse_solve_batched", "coarse_solve_adjoint", "coarse_block_grad", "coarse_residual"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(L, n), n
    from paper_2205_09104_gb300 import _abi
    assert sorted(_abi.EXPORTS) == _declared()
    L.coarse_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.coarse_version()


def test_null_arguments_are_rejected_without_gpu(libpath):
    """Argument validation happens before any CUDA call."""
    from paper_2205_09104_gb300 import _abi
    L = _abi.lib()
    assert L.coarse_op_create(None, None, None, None, None) == -1
    assert b"NULL" in L.coarse_last_error()
    assert L.coarse_apply(None, None, None, 1, 0, None) == -1
    assert L.coarse_solve(None, None, None, 1, None, None, None) == -1
    assert L.coarse_solve_batched(None, -1, None, None, None, None, None, None) == -1


def test_autotune_set_and_forget_without_gpu(libpath):
    """coarse_autotune_set fixes a decision (plain key: every device) and a < 0 forgets it again;
    both are host-side table operations, visible in coarse_autotune_report."""
    L = ctypes.CDLL(libpath)
    L.coarse_autotune_set.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.coarse_autotune_report.argtypes = [ctypes.c_char_p, ctypes.c_longlong]

    def report():
        buf = ctypes.create_string_buffer(1 << 14)
        assert L.coarse_autotune_report(buf, len(buf)) == 0
        return buf.value.decode()
    assert L.coarse_autotune_set(b"eo/p1/n48/v16", 3, 0, 0) == 0
    assert "eo/p1/n48/v16 -> 3 0 0" in report()
    assert L.coarse_autotune_set(b"eo/p1/n48/v16", -1, 0, 0) == 0
    assert "eo/p1/n48/v16 ->" not in report()
    assert L.coarse_autotune_set(b"", 1, 0, 0) == -1
