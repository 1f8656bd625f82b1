"""Planted mistakes in the oracle: each must make at least one pin fail.

The pins in tests/test_oracle.py hold the oracle to facts fixed by the paper
and by mathematics.  To show they would notice a plausible mistake, each
mistake below is planted in a copy of the oracle (a one-line change to the C
source, built with gcc into a temporary library, or a replaced Python
decoder) and the pins are run against the copy until one fails.  Every
planted change keeps memory accesses in bounds.  The real oracle is restored
after each case.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests import test_oracle as pins


def _cases(fn):
    """Keyword sets of a pin's parametrize marks (their cartesian product)."""
    combos = [{}]
    for m in getattr(fn, "pytestmark", []):
        if m.name != "parametrize":
            continue
        names = m.args[0]
        names = [n.strip() for n in names.split(",")] if isinstance(names, str) else list(names)
        grown = []
        for c in combos:
            for v in m.args[1]:
                v = getattr(v, "values", v)
                v = (v,) if len(names) == 1 else tuple(v)
                grown.append({**c, **dict(zip(names, v))})
        combos = grown
    return combos


PINS = [(getattr(pins, n), kw) for n in dir(pins) if n.startswith("test_")
        for kw in _cases(getattr(pins, n))]


def first_failing_pin(mod):
    """Name of the first pin that fails against `mod`, or None."""
    for fn, kw in PINS:
        try:
            fn(mod, **kw)
        except Exception:  # an assertion, or a crash of the planted copy's logic
            return f"{fn.__name__}{kw}"
    return None


# (unique text in fa_oracle.c, its replacement)
C_MUTANTS = {
    "conservation: every valid cell counted as a terminal": (
        "            if (downstream(&R, r, c) < 0) s += A[r * apitch + c];",
        "            s += A[r * apitch + c];"),
    "band residual: the last row of a band skipped": (
        "    for (int64_t r = r_begin; r < r_end; ++r)\n        for (int64_t c = 0; c < cols; ++c) {\n            uint32_t expect;",
        "    for (int64_t r = r_begin; r < r_end - 1; ++r)\n        for (int64_t c = 0; c < cols; ++c) {\n            uint32_t expect;"),
    "direction table: NE steps south": (
        "static const int ODR[10] = {0, 0, -1, -1, -1, 0, 1, 1, 1, 0};",
        "static const int ODR[10] = {0, 0, 1, -1, -1, 0, 1, 1, 1, 0};"),
    "sign: the downstream step reversed": (
        "    int64_t rr = r + ODR[k], cc = c + ODC[k];\n    if (!valid_cell(R, rr, cc)) return -1;",
        "    int64_t rr = r - ODR[k], cc = c - ODC[k];\n    if (!valid_cell(R, rr, cc)) return -1;"),
    "dropped term: a cell's own unit": (
        "        out[c] += 1;\n", "        out[c] += 0;\n"),
    "dropped term: upstream flow not passed on (weights)": (
        "        out[c] += (double)w[r * wpitch + cc];\n        if (next[c] >= 0) out[next[c]] += out[c];",
        "        out[c] += (double)w[r * wpitch + cc];\n        if (next[c] >= 0) out[next[c]] += 0.0;"),
    "doubled weight": (
        "        out[c] += (double)w[r * wpitch + cc];",
        "        out[c] += 2.0 * (double)w[r * wpitch + cc];"),
    "transposed weight index": (
        "        int64_t r = c / cols, cc = c % cols;\n        out[c] += (double)w[r * wpitch + cc];",
        "        int64_t r = c % rows, cc = c / rows;\n        out[c] += (double)w[r * wpitch + cc];"),
    "mask ignored": (
        "    if (R->mask && R->mask[r * R->mpitch + c]) return 0;",
        "    if (0 && R->mask && R->mask[r * R->mpitch + c]) return 0;"),
    "NoFlow flows (onto itself)": (
        "    if (k == 0 || k >= 9) return -1;", "    if (k == 0 || k > 9) return -1;"),
    "invalid codes taken as valid cells": (
        "    if (k == 0 || k > 9) return 0;", "    if (k == 0) return 0;"),
    "adjoint: the downstream chain dropped": (
        "            if (ok[next[c]]) v += lam[next[c]];",
        "            if (ok[next[c]]) v += 0.0 * lam[next[c]];"),
    "brute force: unit weight doubled": (
        "        double wy = w ? (double)w[r * wpitch + c] : 1.0;",
        "        double wy = w ? (double)w[r * wpitch + c] : 2.0;"),
    "residual check: the cell's own unit left out": (
        "                expect = 1u;", "                expect = 0u;"),
    "absorption: the receiving cell's factor": (
        "out[next[c]] += (double)a[r * apitch + cc] * out[c];",
        "out[next[c]] += (double)a[next[c]] * out[c];"),
    "absorption: factor ignored": (
        "out[next[c]] += (double)a[r * apitch + cc] * out[c];",
        "out[next[c]] += out[c];"),
    "absorption: own weight absorbed too": (
        "        out[c] += w ? (double)w[r * wpitch + cc] : 1.0;",
        "        out[c] += (w ? (double)w[r * wpitch + cc] : 1.0) * (double)a[r * apitch + cc];"),
    "uint64 residual: the expected count kept in 32 bits": (
        "            uint64_t expect;", "            uint32_t expect;"),
    "uint64 residual: the cell's own unit left out": (
        "                expect = 1;", "                expect = 0;"),
    "uint64 conservation: every valid cell counted as a terminal": (
        "            if (downstream(&R, r, c) < 0) s += A64[r * apitch + c];",
        "            s += A64[r * apitch + c];"),
    "upstream sums: the query cell's own weight skipped": (
        "            sum += w ? (double)w[r * wpitch + c] : 1.0;",
        "            sum += u == p ? 0.0 : (w ? (double)w[r * wpitch + c] : 1.0);"),
    "upstream sums: every valid neighbour taken as upstream": (
        "                if (!valid_cell(&R, rr, cc) || downstream(&R, rr, cc) != u) continue;",
        "                if (!valid_cell(&R, rr, cc)) continue;"),
    "D8: ties go to the later direction": (
        "                if (slope > best) {", "                if (slope >= best) {"),
    "D8: no distance factor on diagonals": (
        "? drop : drop * inv_sqrt2;", "? drop : drop;"),
    "D8: wrong corner direction": (
        "                if (top && left) *out = 4;", "                if (top && left) *out = 3;"),
    "D8: the last NoData neighbour instead of the first": (
        "                    if (!into_nodata) into_nodata = (uint8_t)k;",
        "                    into_nodata = (uint8_t)k;"),
}


@pytest.fixture(scope="module")
def gcc():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    return "gcc"


def test_every_pin_passes_on_the_oracle(oracle_mod):
    assert first_failing_pin(oracle_mod) is None


@pytest.mark.parametrize("name", sorted(C_MUTANTS))
def test_planted_c_mistake_is_caught(oracle_mod, gcc, tmp_path, name):
    old, new = C_MUTANTS[name]
    src = open(oracle_mod._SRC).read()
    assert src.count(old) == 1, "the planted text must name one place in the oracle"
    c_file, so = tmp_path / "oracle_mutant.c", tmp_path / "liboracle_mutant.so"
    c_file.write_text(src.replace(old, new))
    subprocess.check_call([gcc, "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(c_file)])
    saved = oracle_mod._load()
    oracle_mod._lib = oracle_mod._configure(ctypes.CDLL(os.fspath(so)))
    try:
        caught = first_failing_pin(oracle_mod)
    finally:
        oracle_mod._lib = saved
    assert caught is not None, f"no pin notices: {name}"


class _Replaced:
    """The oracle module with some of its functions replaced."""

    def __init__(self, mod, **repl):
        self._mod, self._repl = mod, repl

    def __getattr__(self, k):
        return self._repl[k] if k in self._repl else getattr(self._mod, k)


def _unpack_swapped(packed, cols):
    p = np.asarray(packed, dtype=np.uint8)
    out = np.zeros((p.shape[0], cols), np.uint8)
    for c in range(cols):
        out[:, c] = (p[:, c // 2] >> 4) if c % 2 == 0 else (p[:, c // 2] & 15)
    return out


def _unpack_spare_nibble_read(packed, cols):
    p = np.asarray(packed, dtype=np.uint8)
    out = np.zeros((p.shape[0], cols), np.uint8)
    for c in range(cols):
        byte = p[:, c // 2]
        out[:, c] = (byte & 15) if c % 2 == 0 else (byte >> 4)
    if cols % 2:  # reads the row's spare nibble as the last cell
        out[:, -1] = p[:, cols // 2] >> 4
    return out


PY_MUTANTS = {
    "packed: nibble order swapped": {"unpack_nibbles": _unpack_swapped},
    "packed: spare nibble read": {"unpack_nibbles": _unpack_spare_nibble_read},
    "code table ignored": {"recode": lambda codes, table: np.asarray(codes, np.uint8).copy()},
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_decoder_mistake_is_caught(oracle_mod, name):
    assert first_failing_pin(_Replaced(oracle_mod, **PY_MUTANTS[name])) is not None
