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


def _raster(rows, cols, n_fields, fake, pitch=None):
    r = _lib.fa_raster()
    r.codes = fake
    r.rows, r.cols = rows, cols
    r.pitch_codes = r.pitch_w = r.pitch_out = cols if pitch is None else pitch
    for f in range(max(n_fields, 1)):
        r.out[f] = fake
        if n_fields:
            r.weights[f] = fake
    return r


def test_batched_host_logic_without_gpu(lib):
    o = _lib.fa_options()
    fake = 1 << 20  # never dereferenced: validation and sizing only
    arr = (_lib.fa_raster * 3)(_raster(100, 100, 0, fake), _raster(0, 7, 0, fake),
                               _raster(300, 500, 0, fake))
    one = lib.fa_batched_workspace_size(arr, 1, 0, ctypes.byref(o))
    three = lib.fa_batched_workspace_size(arr, 3, 0, ctypes.byref(o))
    assert 0 < one < three
    # an empty raster adds no tiles and no table entry
    assert lib.fa_batched_workspace_size(arr, 2, 0, ctypes.byref(o)) == one
    w3 = (_lib.fa_raster * 1)(_raster(100, 100, 3, fake))
    w1 = (_lib.fa_raster * 1)(_raster(100, 100, 1, fake))
    assert lib.fa_batched_workspace_size(w3, 1, 3, ctypes.byref(o)) > \
        lib.fa_batched_workspace_size(w1, 1, 1, ctypes.byref(o)) > 0
    # rejected: negative count, too many fields, pitch < cols, missing output
    assert lib.fa_batched_workspace_size(arr, -1, 0, ctypes.byref(o)) == 0
    assert lib.fa_batched_workspace_size(w3, 1, _lib.FA_MAX_FIELDS + 1, ctypes.byref(o)) == 0
    bad = (_lib.fa_raster * 1)(_raster(100, 100, 0, fake, pitch=50))
    assert lib.fa_batched_workspace_size(bad, 1, 0, ctypes.byref(o)) == 0
    nout = (_lib.fa_raster * 1)(_raster(100, 100, 0, fake))
    nout[0].out[0] = None
    assert lib.fa_batched_workspace_size(nout, 1, 0, ctypes.byref(o)) == 0
    nw = (_lib.fa_raster * 1)(_raster(100, 100, 2, fake))
    nw[0].weights[1] = None
    assert lib.fa_batched_workspace_size(nw, 1, 2, ctypes.byref(o)) == 0
    # workspace missing, misaligned or too small: refused before any CUDA call
    st = lib.fa_accumulate_batched(arr, 3, 0, None, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_WORKSPACE
    st = lib.fa_accumulate_batched(arr, 3, 0, fake + 8, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_WORKSPACE
    st = lib.fa_accumulate_batched(arr, 3, 0, fake, three - 1, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_WORKSPACE
    st = lib.fa_accumulate_batched(bad, 1, 0, fake, 1 << 30, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG
    plan = ctypes.c_void_p(123)
    st = lib.fa_batched_plan_create(arr, 3, 0, fake, three - 1, ctypes.byref(o), None, None,
                                    ctypes.byref(plan))
    assert st == _lib.FA_ERR_WORKSPACE and not plan.value
    st = lib.fa_batched_plan_create(arr, 3, 0, fake, three, ctypes.byref(o), None, None, None)
    assert st == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_plan_launch(None, None) == _lib.FA_ERR_INVALID_ARG
    lib.fa_plan_destroy(None)


def test_autotune_host_logic_without_gpu(lib):
    o = _lib.fa_options()
    fake = 1 << 20  # never dereferenced: every path below returns before a CUDA call
    need = lib.fa_autotune_workspace_size(1000, 1200, ctypes.byref(o))
    assert need >= lib.fa_workspace_size(1000, 1200, ctypes.byref(o)) > 0
    best = _lib.fa_options()
    # no candidate fits a tiny workspace
    st = lib.fa_autotune(fake, 1000, 1200, 1200, None, 0, None, 0, fake, _lib.FA_OUT_U32, 1200,
                         fake, 64, ctypes.byref(o), None, ctypes.byref(best))
    assert st == _lib.FA_ERR_WORKSPACE
    # NULL result
    st = lib.fa_autotune(fake, 1000, 1200, 1200, None, 0, None, 0, fake, _lib.FA_OUT_U32, 1200,
                         fake, need, ctypes.byref(o), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG
    arr = (_lib.fa_raster * 1)(_raster(100, 100, 0, fake))
    assert lib.fa_autotune_batched_workspace_size(arr, 1, 0, ctypes.byref(o)) >= \
        lib.fa_batched_workspace_size(arr, 1, 0, ctypes.byref(o)) > 0
    st = lib.fa_autotune_batched(arr, 1, 0, fake, 64, ctypes.byref(o), None, ctypes.byref(best))
    assert st == _lib.FA_ERR_WORKSPACE


def test_d8_rejects_bad_args_without_gpu(lib):
    fake = 1 << 20  # never dereferenced
    assert lib.fa_d8_codes(fake, -1, 5, 5, None, 0, fake, 5, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_d8_codes(fake, 5, 5, 4, None, 0, fake, 5, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_d8_codes(fake, 5, 5, 5, None, 0, fake, 4, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_d8_codes(fake, 5, 5, 5, fake, 2, fake, 5, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_d8_codes(fake + 2, 5, 5, 5, None, 0, fake, 5, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_d8_codes(None, 0, 5, 5, None, 0, None, 5, None) == _lib.FA_OK  # empty
    # more rows than the launch grid covers (65535 x 4 threads of 8 rows)
    assert lib.fa_d8_codes(fake, 2097121, 5, 5, None, 0, fake, 5, None) == _lib.FA_ERR_INVALID_ARG


def test_packed_codes_host_logic_without_gpu(lib):
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: validation fails first
    nib = _lib.fa_options(0, 0, 0, _lib.FA_CODES_NIBBLE)
    bad = _lib.fa_options(0, 0, 0, 2)  # unknown code format
    assert lib.fa_workspace_size(100, 100, ctypes.byref(bad)) == 0
    assert lib.fa_workspace_size(100, 100, ctypes.byref(nib)) == \
        lib.fa_workspace_size(100, 100, ctypes.byref(_lib.fa_options()))
    st = lib.fa_accumulate(fake, 10, 11, 11, None, 0, None, 0, fake, _lib.FA_OUT_U32, 11,
                           fake, 1 << 30, ctypes.byref(bad), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG
    # packed rows of 11 cells need 6 bytes: pitch 5 is short, 6 passes on to
    # the workspace check
    st = lib.fa_accumulate(fake, 10, 11, 5, None, 0, None, 0, fake, _lib.FA_OUT_U32, 11,
                           fake, 16, ctypes.byref(nib), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG
    st = lib.fa_accumulate(fake, 10, 11, 6, None, 0, None, 0, fake, _lib.FA_OUT_U32, 11,
                           fake, 16, ctypes.byref(nib), None, None)
    assert st == _lib.FA_ERR_WORKSPACE
    st = lib.fa_accumulate_adjoint(fake, 10, 11, 5, None, 0, fake, 11, fake, 11, fake, 16,
                                   ctypes.byref(nib), None, None)
    assert st == _lib.FA_ERR_INVALID_ARG
    st = lib.fa_accumulate_adjoint(fake, 10, 11, 6, None, 0, fake, 11, fake, 11, fake, 16,
                                   ctypes.byref(nib), None, None)
    assert st == _lib.FA_ERR_WORKSPACE
    r = _raster(10, 11, 0, 1 << 20, pitch=11)
    r.pitch_codes = 5
    arr = (_lib.fa_raster * 1)(r)
    assert lib.fa_batched_workspace_size(arr, 1, 0, ctypes.byref(nib)) == 0
    arr[0].pitch_codes = 6
    assert lib.fa_batched_workspace_size(arr, 1, 0, ctypes.byref(nib)) > 0
    assert lib.fa_batched_workspace_size(arr, 1, 0, ctypes.byref(_lib.fa_options())) == 0


def test_recode_rejects_bad_args_without_gpu(lib):
    fake = 1 << 20  # never dereferenced
    B, N = _lib.FA_CODES_BYTE, _lib.FA_CODES_NIBBLE
    assert lib.fa_recode(fake, -1, 5, 5, None, fake, 5, B, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_recode(fake, 5, 5, 5, None, fake, 5, 2, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_recode(None, 5, 5, 5, None, fake, 5, B, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_recode(fake, 5, 5, 4, None, fake, 5, B, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_recode(fake, 5, 5, 5, None, fake, 4, B, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_recode(fake, 5, 5, 5, None, fake, 2, N, None) == _lib.FA_ERR_INVALID_ARG
    assert lib.fa_recode(None, 0, 5, 5, None, None, 0, N, None) == _lib.FA_OK  # empty


def test_power_of_two_table():
    # typed from the scheme: E 1, SE 2, S 4, SW 8, W 16, NW 32, N 64, NE 128
    import paper_1608_04431_gb300 as fa
    t = fa.power_of_two_table()
    want = {0: 0, 1: 1, 2: 8, 4: 7, 8: 6, 16: 5, 32: 4, 64: 3, 128: 2}
    assert len(t) == 256
    for v in range(256):
        assert t[v] == want.get(v, 10)


def test_absorb_host_logic_without_gpu(lib):
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: validation fails first
    o = _lib.fa_options()
    assert lib.fa_absorb_workspace_size(100, 100, ctypes.byref(o)) > 0
    big = _lib.fa_options(128, 64, 0, 0)  # 8192 cells: above the 4096-cell tile limit
    assert lib.fa_absorb_workspace_size(100, 100, ctypes.byref(big)) == 0

    def call(codes=fake, pc=10, factors=fake, pf=10, out=fake, po=10, ws=fake, nbytes=1 << 30,
             opts=o):
        return lib.fa_accumulate_absorb(codes, 10, 10, pc, None, 0, factors, pf, None, 0, out, po,
                                        ws, nbytes, ctypes.byref(opts), None, None)

    assert call(codes=None) == _lib.FA_ERR_INVALID_ARG
    assert call(factors=None) == _lib.FA_ERR_INVALID_ARG
    assert call(out=None) == _lib.FA_ERR_INVALID_ARG
    assert call(pf=9) == _lib.FA_ERR_INVALID_ARG
    assert call(po=9) == _lib.FA_ERR_INVALID_ARG
    assert call(factors=ctypes.c_void_p((1 << 20) + 2)) == _lib.FA_ERR_INVALID_ARG
    assert call(opts=big) == _lib.FA_ERR_INVALID_ARG
    assert call(ws=None) == _lib.FA_ERR_WORKSPACE
    assert call(nbytes=64) == _lib.FA_ERR_WORKSPACE


def test_ooc_host_logic_without_gpu(lib):
    """Out-of-core entry: workspace sizing follows the block plan, and bad
    arguments return before any stream or copy is made."""
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: validation fails first
    o = _lib.fa_options()
    size = lib.fa_ooc_workspace_size
    a = size(1000, 1000, 100, 100, ctypes.byref(o))
    b = size(1000, 1000, 200, 200, ctypes.byref(o))
    assert 0 < a < b  # bigger blocks: bigger buffers, fewer perimeter slots do not win
    assert size(1000, 1000, 0, 0, ctypes.byref(o)) == size(1000, 1000, 1000, 1000, ctypes.byref(o))
    assert size(40000, 40000, 16384, 16384, ctypes.byref(o)) > 0     # 65532 perimeter slots
    assert size(40000, 40000, 16384, 16385, ctypes.byref(o)) > 0     # 65534: the last that fits
    assert size(40000, 40000, 16385, 16385, ctypes.byref(o)) == 0    # 65536 slots
    assert size(100, 100, -1, 10, ctypes.byref(o)) == 0
    nib = _lib.fa_options(0, 0, 0, 1)
    assert size(100, 100, 10, 10, ctypes.byref(nib)) == 0
    badtile = _lib.fa_options(128, 128, 0, 0)
    assert size(100, 100, 10, 10, ctypes.byref(badtile)) == 0

    def call(codes=fake, pc=10, out=fake, po=10, ws=fake, nbytes=1 << 30, bh=5, bw=5, opts=o):
        return lib.fa_accumulate_ooc(codes, 10, 10, pc, out, po, bh, bw, ws, nbytes,
                                     ctypes.byref(opts), None, None)

    assert call(codes=None) == _lib.FA_ERR_INVALID_ARG
    assert call(out=None) == _lib.FA_ERR_INVALID_ARG
    assert call(pc=9) == _lib.FA_ERR_INVALID_ARG
    assert call(po=9) == _lib.FA_ERR_INVALID_ARG
    assert call(bh=-2) == _lib.FA_ERR_INVALID_ARG
    assert call(opts=nib) == _lib.FA_ERR_INVALID_ARG
    assert call(ws=None) == _lib.FA_ERR_WORKSPACE
    assert call(ws=ctypes.c_void_p((1 << 20) + 16)) == _lib.FA_ERR_WORKSPACE
    assert call(nbytes=64) == _lib.FA_ERR_WORKSPACE


def test_header_is_plain_c(tmp_path):
    """include/*.h is a C ABI: it must compile as C99 with warnings as errors."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use_header.c"
    src.write_text("".join(f'#include "{os.path.basename(h)}"\n' for h in HEADERS) +
                   "int main(void) { fa_options o = {0, 0, FA_OPT_NO_TMA, FA_CODES_NIBBLE};\n"
                   "  (void)o; return fa_version() > 0 ? 0 : 1; }\n")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)])
