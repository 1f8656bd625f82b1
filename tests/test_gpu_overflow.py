"""Counts at and beyond 2^32: the overflow flag of the uint32 form and the exact
uint64 counts of the out-of-core form.

The raster is 65537 x 65536 (4,295,032,832 cells, just over 2^32), every cell
flowing east except the last column, which flows south, and the bottom-right
cell, which drains off the grid.  Closed form (Eq. 1 on this raster): cell
(r, c) with c < C - 1 counts c + 1; the last column collects whole rows, so
cell (r, C - 1) counts (r + 1) * C.  The bottom cells of the last column pass
2^32: the uint32 form must return them modulo 2^32 and report
FA_WARN_OVERFLOW (Section 4 of the paper stores FP64 because such values
occur); the out-of-core form must return them exactly.
"""
import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

fa = pytest.importorskip("paper_1608_04431_gb300")

R, C = 65537, 65536


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 48 << 30:
        pytest.skip("needs about 40 GB of device memory")


def east_then_south():
    codes = torch.full((R, C), 1, dtype=torch.uint8, device="cuda")  # E
    codes[:, C - 1] = 7                                              # S
    codes[R - 1, C - 1] = 1                                          # off the grid (E)
    return codes


def last_column_exact():
    return (torch.arange(1, R + 1, dtype=torch.int64, device="cuda") * C)


def test_uint32_counts_wrap_and_are_flagged():
    codes = east_then_south()
    out = fa.accumulate(codes)
    st, _, _ = fa.fa_status_read(None, fa.workspace(0, "cuda"))
    assert st == fa.FA_WARN_OVERFLOW
    o32 = out.view(torch.int32)
    as_u32 = lambda t: t.to(torch.int64) & 0xFFFFFFFF  # noqa: E731
    assert torch.equal(as_u32(o32[:, C - 1]), last_column_exact() & 0xFFFFFFFF)
    cols = torch.arange(1, C, dtype=torch.int64, device="cuda")
    for r in (0, 1, 4097, R // 2, R - 1):
        assert torch.equal(as_u32(o32[r, :C - 1]), cols)
    del out, codes
    fa._ws_cache.clear()
    torch.cuda.empty_cache()


_OOC_CHECK = r"""
import sys
import torch
import paper_1608_04431_gb300 as fa
R, C = int(sys.argv[1]), int(sys.argv[2])
codes = torch.full((R, C), 1, dtype=torch.uint8)
codes[:, C - 1] = 7
codes[R - 1, C - 1] = 1
out = fa.accumulate_ooc(codes)  # default 16384 x 16384 blocks, uint64 in an int64 tensor
want = torch.arange(1, R + 1, dtype=torch.int64) * C
assert int(want[-1]) == R * C and R * C > 1 << 32
assert torch.equal(out[:, C - 1], want), "last column"
cols = torch.arange(1, C, dtype=torch.int64)
for r in (0, 16383, 16384, R // 2, R - 1):
    assert torch.equal(out[r, :C - 1], cols), r
print("ok")
"""


def _host_bytes_available():
    """MemAvailable of the host, capped by the cgroup's memory limit."""
    avail = None
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    try:
        with open("/sys/fs/cgroup/memory.max") as f:
            lim = f.read().strip()
        with open("/sys/fs/cgroup/memory.current") as f:
            cur = int(f.read().strip())
        if lim != "max":
            avail = min(avail, int(lim) - cur) if avail is not None else int(lim) - cur
    except OSError:
        pass
    return avail


def test_out_of_core_counts_are_exact_beyond_2_32():
    """Run in a process of its own, with the device memory of this one given
    back first: the raster (4.3 GB) and its uint64 counts (34 GB) live in
    host memory, which must have room for both."""
    import gc
    import os
    import subprocess
    import sys

    fa._ws_cache.clear()
    gc.collect()
    torch.cuda.empty_cache()
    need = R * C * 9 + (8 << 30)
    avail = _host_bytes_available()
    if avail is not None and avail < need:
        pytest.skip(f"needs {need >> 30} GiB of host memory, {avail >> 30} GiB available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-X", "faulthandler", "-c", _OOC_CHECK, str(R), str(C)], cwd=root,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stderr[-2000:])
