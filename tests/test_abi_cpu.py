"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/qbvh.h, and rejects bad arguments before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_08088_gb300 import build_lib
    from paper_1901_08088_gb300 import _lib

    build_lib.build()
    return _lib.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "qbvh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:qbvh|nlist)_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("qbvh_build", "qbvh_query", "nlist_get", "qbvh_create", "qbvh_destroy",
                 "qbvh_lj_forward", "qbvh_lj_backward", "qbvh_build_batched"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_entry_point():
    from paper_1901_08088_gb300 import _lib

    assert set(_declared()) == set(_lib.SIGNATURES)


def test_strerror_names_every_code(lib):
    from paper_1901_08088_gb300 import _lib

    codes = [v for k, v in vars(_lib).items() if k.startswith("QBVH_ERR_") or k == "QBVH_OK"]
    msgs = {lib.qbvh_strerror(c).decode() for c in codes}
    assert len(msgs) == len(codes)
    assert lib.qbvh_strerror(12345).decode() == "unknown status"


def test_null_and_invalid_arguments_are_rejected_on_host(lib):
    from paper_1901_08088_gb300 import _lib

    E = _lib.QBVH_ERR_INVALID_ARG
    assert lib.qbvh_create(None, 0) == E
    assert lib.qbvh_destroy(None) == E
    assert lib.qbvh_build(None, None, 0, 1.0, 1, None) == E
    assert lib.qbvh_query(None, None, 8, 0, None) == E
    assert lib.qbvh_query_status(None, None) == E
    assert lib.qbvh_query_lj_async(None, None, None, 8, None, None, None, None, None, None, None, None, None) == E
    assert lib.nlist_get(None, None, None, None, None) == E
    assert lib.qbvh_set_option(None, 1, 4) == E
    assert lib.qbvh_pack_positions(None, None, -1, None, None) == E
    # misaligned device pointer is refused before any launch
    assert lib.qbvh_pack_positions(C.c_void_p(8), None, 4, C.c_void_p(8), None) == E


def test_create_without_a_device_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1901_08088_gb300 import _lib

    h = C.c_void_p()
    assert lib.qbvh_create(C.byref(h), 0) == _lib.QBVH_ERR_CUDA
    assert h.value is None


def test_package_has_no_cpu_fallback():
    # the product imports nothing from the oracle
    pkg = os.path.join(ROOT, "paper_1901_08088_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "_oracle.so" not in text, f

