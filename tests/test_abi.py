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


def test_null_handle_tuning_calls():
    L = _lib.load()
    assert L.tempest_set_tuning(None, 0, 2) == _lib.TEMPEST_EINVAL
    assert L.tempest_get_tuning(None, 0, None) == _lib.TEMPEST_EINVAL
    assert L.tempest_autotune(None, 10, 10, 0, 0, 0, 0, None) == _lib.TEMPEST_EINVAL


def test_ctypes_structs_match_the_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal what a C compiler
    lays out from include/tempest.h."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    mirrors = {"tempest_ingest_stats": _lib.IngestStats, "tempest_walk_stats": _lib.WalkStats,
               "tempest_walk_request": _lib.WalkRequest, "tempest_tune_trial": _lib.TuneTrial,
               "tempest_tune_report": _lib.TuneReport}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tempest.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().split("\n"):
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_enum_constants_match_the_header(tmp_path):
    """Every enumerator of include/tempest.h that the binding mirrors (knobs,
    forms, biases, start policies, status codes) has the header's value."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "tempest.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(TEMPEST_[A-Z0-9_]+)\s*=", txt)))
    pairs = []
    for n in names:
        short = n[len("TEMPEST_"):]
        if hasattr(_lib, short):
            pairs.append((n, getattr(_lib, short)))
        elif hasattr(_lib, n):
            pairs.append((n, getattr(_lib, n)))
    assert len(pairs) >= 20
    lines = ['#include <stdio.h>', '#include "tempest.h"', "int main(void) {"]
    lines += ['printf("%s %%lld\\n", (long long)%s);' % (n, n) for n, _ in pairs]
    lines.append("return 0; }")
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "enums"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    for n, v in pairs:
        assert int(got[n]) == int(v), n
