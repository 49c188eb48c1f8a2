"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point include/musr.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(musr_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1604_02334_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = declared_functions(os.path.join(ROOT, "include", "musr.h"))
    for n in ("musr_create_run", "musr_chi2", "musr_chi2_batch", "musr_chi2_grad", "musr_fit"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for header in os.listdir(os.path.join(ROOT, "include")):
        for name in declared_functions(os.path.join(ROOT, "include", header)):
            assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1604_02334_gb300 import _lib
    _lib.load()
    for header in os.listdir(os.path.join(ROOT, "include")):
        for name in declared_functions(os.path.join(ROOT, "include", header)):
            assert name in _lib.SIGNATURES, name


def test_status_strings_without_gpu(lib_path):
    from paper_1604_02334_gb300 import _lib
    lib = _lib.load()
    assert lib.musr_strerror(_lib.MUSR_EDOMAIN).startswith(b"Poisson")
    assert b"sm_103a" in lib.musr_version()


def test_create_run_without_gpu_fails_cleanly(lib_path):
    """With no CUDA device the boundary returns an error code instead of aborting."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import workloads as W
    from paper_1604_02334_gb300 import MusrError, Run
    lay, theta, _ = W.config_single()
    with pytest.raises(MusrError):
        Run(lay, None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the compiled library the binding raises
    from paper_1604_02334_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libmusr.so"))
    with pytest.raises(ImportError):
        _lib.load()
