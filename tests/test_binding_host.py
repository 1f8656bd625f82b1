"""Host-side logic of the Python binding: argument checks and option
marshalling that run before any kernel (no GPU needed)."""
import pytest
import torch

import paper_1608_04431_gb300 as fa


def test_packed_codes_checks_its_shape():
    data = torch.zeros((4, 5), dtype=torch.uint8)
    pk = fa.PackedCodes(data, 9)  # 9 cells need 5 bytes per row
    assert pk.shape == (4, 9) and pk.dtype == torch.uint8 and not pk.is_cuda
    assert pk.data_ptr() == data.data_ptr()
    with pytest.raises(ValueError):
        fa.PackedCodes(data, 11)  # 11 cells need 6 bytes
    with pytest.raises(TypeError):
        fa.PackedCodes(torch.zeros((4, 5), dtype=torch.int32), 9)
    with pytest.raises(TypeError):
        fa.PackedCodes(torch.zeros(20, dtype=torch.uint8), 9)


def test_code_format_follows_the_codes():
    o = fa.options((32, 64), fa.FA_OPT_NO_TMA)
    assert (o.tile_h, o.tile_w, o.flags, o.code_format) == (32, 64, fa.FA_OPT_NO_TMA, fa.FA_CODES_BYTE)
    pk = fa.PackedCodes(torch.zeros((2, 2), dtype=torch.uint8), 3)
    p = fa._with_format(pk, o)
    assert (p.tile_h, p.tile_w, p.flags, p.code_format) == (32, 64, fa.FA_OPT_NO_TMA, fa.FA_CODES_NIBBLE)
    assert o.code_format == fa.FA_CODES_BYTE  # the caller's options are not changed
    b = fa._with_format(torch.zeros((2, 3), dtype=torch.uint8), None)
    assert b.code_format == fa.FA_CODES_BYTE and (b.tile_h, b.tile_w) == (0, 0)
    assert fa._pitch(pk) == 2


def test_batches_hold_one_code_format():
    byte = {"codes": torch.zeros((2, 3), dtype=torch.uint8)}
    packed = {"codes": fa.PackedCodes(torch.zeros((2, 2), dtype=torch.uint8), 3)}
    assert fa._batch_format([byte, byte]) == fa.FA_CODES_BYTE
    assert fa._batch_format([packed, packed]) == fa.FA_CODES_NIBBLE
    assert fa._batch_format([]) == fa.FA_CODES_BYTE
    with pytest.raises(ValueError):
        fa._batch_format([byte, packed])


def test_host_tensors_are_refused_before_any_launch():
    codes = torch.ones((3, 3), dtype=torch.uint8)
    with pytest.raises(TypeError):
        fa.accumulate(codes)
    with pytest.raises(TypeError):
        fa.recode(codes)
    with pytest.raises(TypeError):
        fa.d8_codes(torch.zeros((3, 3), dtype=torch.float32))
    with pytest.raises(TypeError):
        fa.absorb(codes, torch.ones((3, 3), dtype=torch.float64))
    with pytest.raises(ValueError):
        fa.fa_recode(codes, b"\x00" * 255, codes, fa.FA_CODES_BYTE)  # a table has 256 entries
