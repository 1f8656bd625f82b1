"""fa_accumulate_noalloc against fa_accumulate.

fa_accumulate_noalloc is for callers that can pass their own input and output
rasters but cannot allocate scratch memory on the device (a plugin host that
hands over only the caller's buffers, a pipeline whose device memory is all
reserved at start-up, a program whose memory belongs to another framework's
allocator).  It takes its scratch from one fixed buffer inside the library, so
it must give exactly what fa_accumulate gives with a caller-supplied workspace.
It is called twice in a row, on different rasters, because every call reuses
the same buffer, which still holds the previous call's data.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

fa = pytest.importorskip("paper_1608_04431_gb300")
RTOL = 2e-5  # the float32 tolerance used by the other parity tests


def _u32(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


@pytest.mark.gpu
def test_noalloc_matches_fa_accumulate_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    opts = fa.options()
    status = torch.zeros(fa.FA_STATUS_WORDS, dtype=torch.int32, device=dev)

    # first call: unit weights, uint32 counts, with a NoData mask
    codes_a = synth.dem_codes(1500, 1700, 5)
    mask_a = (synth.rng(6).random(codes_a.shape) < 0.01).astype(np.uint8)
    ca = torch.from_numpy(codes_a).to(dev)
    ma = torch.from_numpy(mask_a).to(dev)
    ref_a = _u32(fa.accumulate(ca, None, ma))
    out_a = torch.full(codes_a.shape, 0xFFFF, dtype=torch.uint32, device=dev)
    st = fa.fa_accumulate_noalloc(ca, None, ma, out_a, fa.FA_OUT_U32, opts, status, stream)
    assert st == fa.FA_OK
    assert fa.fa_status_read(status, None, stream)[0] == fa.FA_OK
    np.testing.assert_array_equal(_u32(out_a), ref_a)

    # second call, straight after, on another raster and shape with float32
    # weights: nothing left in the shared buffer may leak into the result
    codes_b = synth.dem_codes(2300, 1100, 7)
    w_b = synth.lognormal_weights(codes_b.shape, 8)
    cb = torch.from_numpy(codes_b).to(dev)
    wb = torch.from_numpy(w_b).to(dev)
    ref_b = fa.accumulate(cb, wb).cpu().numpy().astype(np.float64)
    out_b = torch.full(codes_b.shape, -1.0, dtype=torch.float32, device=dev)
    st = fa.fa_accumulate_noalloc(cb, wb, None, out_b, fa.FA_OUT_F32, opts, status, stream)
    assert st == fa.FA_OK
    assert fa.fa_status_read(status, None, stream)[0] == fa.FA_OK
    got_b = out_b.cpu().numpy().astype(np.float64)
    assert (np.abs(got_b - ref_b) <= RTOL * np.abs(ref_b)).all()

    # and the first raster once more, after the second call used the buffer
    out_c = torch.zeros(codes_a.shape, dtype=torch.uint32, device=dev)
    st = fa.fa_accumulate_noalloc(ca, None, ma, out_c, fa.FA_OUT_U32, opts, status, stream)
    assert st == fa.FA_OK
    np.testing.assert_array_equal(_u32(out_c), ref_a)


@pytest.mark.gpu
def test_noalloc_staged_code_tiles_match_and_oracle(oracle_mod):
    """An unmasked raster whose width is a multiple of 16, so that pass 1
    stages its code tiles by TMA (with the bounded barrier wait) inside the
    no-allocation entry point too: bit for bit against fa_accumulate, and the
    counts against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    status = torch.zeros(fa.FA_STATUS_WORDS, dtype=torch.int32, device=dev)
    codes = synth.dem_codes(1536, 2048, 11)
    c = torch.from_numpy(codes).to(dev)
    assert c.data_ptr() % 16 == 0
    ref = _u32(fa.accumulate(c))
    for _ in range(2):  # two calls in a row on the shared buffer
        out = torch.full(codes.shape, 7, dtype=torch.uint32, device=dev)
        st = fa.fa_accumulate_noalloc(c, None, None, out, fa.FA_OUT_U32, fa.options(), status,
                                      stream)
        assert st == fa.FA_OK
        assert fa.fa_status_read(status, None, stream)[0] == fa.FA_OK
        np.testing.assert_array_equal(_u32(out), ref)
    np.testing.assert_array_equal(ref, oracle_mod.counts(codes).values.astype(np.uint32))


def test_noalloc_rejects_rasters_beyond_its_buffer():
    """Host-side check: a raster whose scratch would not fit the fixed buffer
    is refused with FA_ERR_TOO_LARGE before anything reaches a GPU."""
    lib = fa._lib.load()
    o = fa.fa_options()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the size check comes first
    n = 20000
    need = lib.fa_workspace_size(n, n, ctypes.byref(o))
    assert need > fa.FA_NOALLOC_SCRATCH_BYTES
    st = lib.fa_accumulate_noalloc(fake, n, n, n, None, 0, None, 0, fake, fa.FA_OUT_U32, n,
                                   ctypes.byref(o), None, None)
    assert st == fa.FA_ERR_TOO_LARGE


@pytest.mark.parametrize("n,fits", [(4700, True), (4800, True), (4801, False)])
def test_noalloc_size_boundary(n, fits):
    """The limit stated in include/fa.h for the default 64 x 64 tiles: square
    rasters up to 4800 x 4800 pass the size check, 4801 x 4801 does not.  NULL
    buffers make an accepted size fail the later pointer check, so nothing is
    ever enqueued."""
    lib = fa._lib.load()
    o = fa.fa_options()
    st = lib.fa_accumulate_noalloc(None, n, n, n, None, 0, None, 0, None, fa.FA_OUT_U32, n,
                                   ctypes.byref(o), None, None)
    assert st == (fa.FA_ERR_INVALID_ARG if fits else fa.FA_ERR_TOO_LARGE)
