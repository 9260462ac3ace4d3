"""The C-ABI library builds, loads and exports every function that
include/bitsort.h declares (no GPU: nothing is called that computes)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bitsort.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(bitsort\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1312_0138_gb300 import builder as b
    return b.build()


def test_header_declares_the_expected_api():
    names = declared_functions()
    import paper_1312_0138_gb300 as p
    assert set(p.EXPORTS) == set(names), set(p.EXPORTS) ^ set(names)


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_signatures(lib_path):
    import paper_1312_0138_gb300 as p
    lib = p.load(lib_path)
    for n in p.EXPORTS:
        assert getattr(lib, n).argtypes is not None, n


def test_status_strings(lib_path):
    import paper_1312_0138_gb300 as p
    lib = p.load(lib_path)
    assert lib.bitsort_status_string(0) == b"ok"
    assert lib.bitsort_status_string(3) == b"duplicate keys"


def test_no_fallback_when_library_missing(tmp_path):
    import importlib
    import paper_1312_0138_gb300 as p
    saved = p._lib
    try:
        p._lib = None
        with pytest.raises(ImportError):
            p.load(str(tmp_path / "missing.so"))
    finally:
        p._lib = saved


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1312_0138_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", src).lower() or f == "__init__.py" and \
                    "import oracle" not in src, f
                assert "import oracle" not in src and "from oracle" not in src, f


def test_binding_refuses_host_tensors_and_missing_gpu(lib_path):
    # the device entry points take device memory only: a CPU tensor is an
    # error before anything is called, never a silent host computation
    import torch
    import paper_1312_0138_gb300 as p
    p.load(lib_path)
    keys = torch.arange(8, dtype=torch.int32)
    with pytest.raises(ValueError):
        p.bitsort(keys, 7)
    with pytest.raises(TypeError):
        p._ptr(keys.to(torch.float32).cuda() if torch.cuda.is_available() else 3.0)
    assert p._host_ptr(keys) == keys.data_ptr()
    with pytest.raises(TypeError):
        p._host_ptr(keys.to(torch.float32))
    if not torch.cuda.is_available():
        # without a GPU a context cannot be made: the call fails loudly
        with pytest.raises(p.BitsortError):
            p.Context(0)
