"""The bounded device wait running out, on purpose and without a fault.

Pass 1 stages code tiles by TMA and waits for each copy on an mbarrier with a
time limit; a wait that runs out sets FA_FLAG_TIMEOUT and the kernel returns.
fa_selftest_wait_timeout runs that same wait against a barrier phase that can
never complete (no copy is in flight), so the timed-out path is exercised: the
status must read FA_ERR_TIMEOUT, the wait must have lasted about its limit,
and the context must stay usable for the next call.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

fa = pytest.importorskip("paper_1608_04431_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_wait_times_out_and_context_survives(oracle_mod):
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    status = torch.zeros(fa.FA_STATUS_WORDS, dtype=torch.int32, device=dev)
    limit_ns = 20_000_000  # 20 ms
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    assert fa.fa_selftest_wait_timeout(limit_ns, status, stream) == fa.FA_OK
    e1.record(stream)
    st, count, first = fa.fa_status_read(status, None, stream)
    assert st == fa.FA_ERR_TIMEOUT
    assert count == 1 and first == -1
    ms = e0.elapsed_time(e1)
    assert 0.9 * limit_ns / 1e6 <= ms < 5000.0, ms
    # the context is still usable: an accumulation right after is exact
    codes = synth.dem_codes(200, 320, 3)
    got = fa.accumulate(torch.from_numpy(codes).to(dev), check=True)
    ref = oracle_mod.counts(codes).values.astype(np.uint32)
    np.testing.assert_array_equal(got.view(torch.int32).cpu().numpy().view(np.uint32), ref)


def test_selftest_rejects_bad_arguments():
    dev = torch.device("cuda:0")
    status = torch.zeros(fa.FA_STATUS_WORDS, dtype=torch.int32, device=dev)
    assert fa.fa_selftest_wait_timeout(-1, status) == fa.FA_ERR_INVALID_ARG
    assert fa.fa_selftest_wait_timeout(10**11, status) == fa.FA_ERR_INVALID_ARG
    assert fa.fa_selftest_wait_timeout(1000, None) == fa.FA_ERR_INVALID_ARG
