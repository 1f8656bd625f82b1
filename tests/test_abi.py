"""Host-only checks of the C ABI: the library loads, exports every function that
include/fa.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1608_04431_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:[\w\s\*]+?)\b(fa_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_builds_for_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "fa_accumulate" in names and "fa_workspace_size" in names
    for n in names:
        assert hasattr(lib, n), f"libfa.so does not export {n}"
    # and the binding knows the signature of each
    for n in names:
        assert n in _lib.SIGNATURES, f"binding lacks a signature for {n}"


def test_version(lib):
    assert lib.fa_version() >= 100


def test_workspace_size_host_logic(lib):
    o = _lib.fa_options()
    assert lib.fa_workspace_size(0, 0, ctypes.byref(o)) > 0
    small = lib.fa_workspace_size(100, 100, ctypes.byref(o))
    big = lib.fa_workspace_size(4096, 4096, ctypes.byref(o))
    assert 0 < small < big
    bad = _lib.fa_options(0, 20000, 0, 0)  # tile too large
    assert lib.fa_workspace_size(100, 100, ctypes.byref(bad)) == 0
    neg = _lib.fa_options(-1, 4, 0, 0)
    assert lib.fa_workspace_size(100, 100, ctypes.byref(neg)) == 0


def test_accumulate_rejects_bad_args_without_gpu(lib):
    o = _lib.fa_options()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: validation fails first
    st = lib.fa_accumulate(None, 10, 10, 10, None, 0, None, 0, fake, _lib.FA_OUT_U32, 10,
                           fake, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG  # NULL codes
    st = lib.fa_accumulate(fake, 10, 10, 5, None, 0, None, 0, fake, _lib.FA_OUT_U32, 10,
                           fake, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG  # pitch < cols
    st = lib.fa_accumulate(fake, 10, 10, 10, fake, 10, None, 0, fake, _lib.FA_OUT_U32, 10,
                           fake, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG  # weights with uint32 output
    st = lib.fa_accumulate(fake, 10, 10, 10, None, 0, None, 0, fake, _lib.FA_OUT_U32, 10,
                           None, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_WORKSPACE  # no workspace
    st = lib.fa_accumulate(fake, 10, 10, 10, None, 0, None, 0, fake, _lib.FA_OUT_U32, 10,
                           fake, 16, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_WORKSPACE  # too small
    st = lib.fa_accumulate(fake, 10, 10, 10, None, 0, None, 0, fake, 7, 10,
                           fake, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG  # unknown dtype
