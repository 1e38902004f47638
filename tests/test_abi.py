"""The C-ABI library loads and exports every entry point include/rpforest.h
declares; argument checks that need no GPU reject bad input."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1812_11689_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rpforest.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rpf_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert "rpf_build" in syms and "rpf_all_knn" in syms and "rpf_query" in syms
    for s in syms:
        assert hasattr(L, s), s
    from paper_1812_11689_gb300 import _lib
    assert set(_lib.EXPORTED) <= set(syms) | set(_lib.EXPORTED)
    for s in _lib.EXPORTED:
        assert s in syms, s


def test_error_strings_and_defaults(L):
    from paper_1812_11689_gb300 import _lib
    assert _lib.error_string(0) == "success"
    assert _lib.error_string(-1) == "invalid argument"
    assert _lib.error_string(-2) == "out of memory"
    p = _lib.rpf_params()
    L.rpf_default_params(ctypes.byref(p))
    assert (p.n_trees, p.leaf_max, p.n_try, p.form, p.growth) == (10, 50, 5, 0, 0)


def test_build_rejects_bad_arguments_before_touching_the_gpu(L):
    from paper_1812_11689_gb300 import _lib
    p = _lib.rpf_params(10, 50, 5, 0, 0, 0, 0)
    out = ctypes.c_void_p()
    buf = (ctypes.c_float * 20)()
    assert L.rpf_build(None, 10, 2, ctypes.byref(p), None, ctypes.byref(out)) == -1
    assert L.rpf_build(buf, 0, 2, ctypes.byref(p), None, ctypes.byref(out)) == -1
    assert L.rpf_build(buf, 10, 0, ctypes.byref(p), None, ctypes.byref(out)) == -1
    assert L.rpf_build(buf, 10, 2, ctypes.byref(p), None, None) == -1
    for bad in (dict(n_trees=0), dict(leaf_max=0), dict(leaf_max=1025), dict(n_try=0), dict(n_try=65),
                dict(form=2), dict(growth=3), dict(split_rule=2), dict(split_rule=-1)):
        q = _lib.rpf_params(10, 50, 5, 0, 0, 0, 0)
        for k, v in bad.items():
            setattr(q, k, v)
        assert L.rpf_build(buf, 10, 2, ctypes.byref(q), None, ctypes.byref(out)) == -1, bad
    # n * T must stay below 2^31
    q = _lib.rpf_params(3, 50, 5, 0, 0, 0, 0)
    assert L.rpf_build(buf, 1 << 30, 2, ctypes.byref(q), None, ctypes.byref(out)) == -1
    assert L.rpf_all_knn(None, 5, None, None, None, 0, None) == -1
    assert L.rpf_all_knn_async(None, 5, None, None, None, 0, None) == -1
    assert L.rpf_query(None, None, 1, 5, None, None, None, 0, None) == -1
    assert L.rpf_workspace_bytes(None, 10, 5, 1) == 0
    assert L.rpf_set_query_scan(None, 0) == -1
    assert L.rpf_gather_probe(None, 10, 4, 1, 0, None, None) == -1
    L.rpf_free(None)


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: include/rpforest.h compiles as C99 with no
    C++ or CUDA types, and every declaration has C linkage."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "rpforest.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "h.o")],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
