"""The C-ABI library builds, loads and exports every symbol the header
declares (no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

from paper_2605_16182_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "tempest.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tempest_[a-z_0-9]+)\s*\(", txt)))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    L = _lib.load()
    assert _lib.tempest_version().startswith("tempest-gb300")
    assert L is _lib.load()


def test_every_declared_symbol_is_exported():
    L = _lib.load()
    decl = header_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(_lib.EXPORTED) == decl


def test_library_is_built_for_sm_103a_only():
    # the build passes exactly one -gencode for sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(_lib.TempestError) as e:
        _lib.tempest_create(0, True)
    assert e.value.code == _lib.TEMPEST_ECUDA
    assert "CUDA" in _lib.tempest_last_error(None) or "device" in _lib.tempest_last_error(None)


def test_null_handle_is_rejected():
    L = _lib.load()
    assert L.tempest_set_scheduler(None, 0) == _lib.TEMPEST_EINVAL
    assert L.tempest_destroy(None) == _lib.TEMPEST_OK
