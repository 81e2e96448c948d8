"""The C-ABI library builds for sm_103a, loads, and exports what include/ivf.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2002_09094_gb300 import ivf

    return ivf.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ivf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ivfb?_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_2002_09094_gb300 import ivf

    assert sorted(ivf.EXPORTS) == names


def test_null_safe_calls(lib):
    lib.ivf_destroy(None)
    assert lib.ivf_last_error(None) == b"null context"
    assert b"sm_103a" in lib.ivf_version()
    assert lib.ivf_launch_count() >= 0


def test_library_is_sm103a_only():
    from paper_2002_09094_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_null_out_pointer_is_invalid(lib):
    from paper_2002_09094_gb300 import ivf

    cfg = ivf.Config(n_docs=1, n_terms=1, nnz=1, k=1)
    # out == NULL is rejected before any CUDA call
    assert lib.ivf_create(ctypes.byref(cfg), None, None, None, None, None) == ivf.IVF_E_INVALID
