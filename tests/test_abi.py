"""The C-ABI library loads and exports every symbol include/kdtree.h declares
(CPU only: no compute calls), and the Python binding mirrors those names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kdtree.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kd_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_5420_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kd_create", "kd_presort", "kd_build", "kd_build_batch", "kd_submit", "kd_wait",
                     "kd_destroy", "kd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_the_abi(lib):
    from paper_1410_5420_gb300 import _lib, api
    assert set(_lib.EXPORTS) == set(declared_functions())
    for name in declared_functions():
        if name in ("kd_last_error", "kd_handle_info"):
            continue
        assert hasattr(api, name), name


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1410_5420_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="must be built"):
        _lib.load()


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # status codes for null contexts / handles need no device
    assert lib.kd_presort(None, None, None) == -1
    assert lib.kd_build(None, None, None) == -1
    assert lib.kd_destroy(None) == -1
    assert lib.kd_launch_count(None) == 0


def test_noalloc_binding_refuses_unsafe_output_buffers():
    """The allocation-free entry point writes through raw pointers; the
    binding refuses a buffer of the wrong type, size, layout or device
    before any call (a tensor on another device needs no second GPU to
    check: a CPU tensor stands for it)."""
    import torch
    from paper_1410_5420_gb300 import api
    with pytest.raises(ValueError):  # a buffer on another device than the context's
        api._check_out_buffer("arrays_out", torch.empty((3, 10), dtype=torch.int32), torch.device("cuda", 1), 30)
    here = torch.device("cpu")
    api._check_out_buffer("arrays_out", torch.empty((3, 10), dtype=torch.int32), here, 30)
    for t in (torch.empty((3, 9), dtype=torch.int32),                     # too small
              torch.empty((3, 10), dtype=torch.int64),                    # wrong type
              torch.empty((10, 3), dtype=torch.int32).t()):               # not contiguous
        with pytest.raises(ValueError):
            api._check_out_buffer("arrays_out", t, here, 30)
