"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol include/labfm.h declares, and rejects bad arguments before any kernel runs.
No compute call is made here (no GPU is needed)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "labfm.h")) as fh:
        src = fh.read()
    return sorted(set(re.findall(r"^\s*(?:labfm_status|void|const char \*)\s*\**\s*(labfm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_06441_gb300.build import build_library

    return ct.CDLL(build_library())


def test_header_declarations_match_binding():
    import paper_1912_06441_gb300 as P

    assert _declared() == sorted(P.C_FUNCTIONS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_null_context_and_arguments_rejected(lib):
    lib.labfm_build_neighbours.restype = ct.c_int
    lib.labfm_build_weights.restype = ct.c_int
    lib.labfm_apply.restype = ct.c_int
    lib.labfm_step.restype = ct.c_int
    lib.labfm_create.restype = ct.c_int
    lib.labfm_last_error.restype = ct.c_char_p
    # null context -> LABFM_ERR_ARG, without touching the GPU
    assert lib.labfm_build_neighbours(None, ct.c_int64(10), None, None, 0, None, None, None) == 1
    assert lib.labfm_build_weights(None, None, 4, 0, 1, None, 0, 0, None, None) == 1
    assert lib.labfm_apply(None, ct.c_uint32(1), None, 0, None) == 1
    assert lib.labfm_step(None, None, None, 0, ct.c_double(0.1), ct.c_int64(1), None) == 1
    assert lib.labfm_create(None, 0, None) == 1
    assert lib.labfm_last_error(None) == b"null context"
    lib.labfm_destroy(None)


def test_no_device_reports_cuda_error(lib):
    """Without a usable device labfm_create fails with LABFM_ERR_CUDA (no CPU fallback)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = ct.c_void_p()
    lib.labfm_create.restype = ct.c_int
    assert lib.labfm_create(ct.byref(ctx), 0, None) == 2
    import paper_1912_06441_gb300 as P

    with pytest.raises(RuntimeError):
        P.Labfm(0)


def test_rpoly_table_independent_of_oracle():
    """Nothing under the package imports the oracle, and the oracle imports nothing from the
    package (the two sides share only the seeded input generators)."""
    pkg = os.path.join(ROOT, "paper_1912_06441_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    txt = fh.read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, re.M), f
                assert "labfm_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            with open(os.path.join(ROOT, "oracle", f)) as fh:
                txt = fh.read()
            assert not re.search(r"^\s*(from|import)\s+paper_1912_06441_gb300", txt, re.M), f
            assert not re.search(r"#include\s+[\"<](labfm\.h|.*\.cuh)", txt), f
