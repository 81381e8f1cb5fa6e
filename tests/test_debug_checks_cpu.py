"""The debug build's range check on the CPU.

The debug library's kernels test every checked access with dbg_in_ranges
(csrc/gfk_debug.h) against the table of registered device buffers.  The same
function compiles as plain C++; here it is built with g++ and given accesses
that fall outside the ranges (below, past the end, straddling an end, in the
gap between two buffers, into a buffer after it is unregistered), which must
all be refused, and accesses inside them, which must pass.  The release
library reports that it is not the debug build without touching CUDA."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1703_08977_gb300 import gfk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1703_08977_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "gfk_debug.h"
int main() {
    // two buffers: [0x1000, 0x1100) and [0x2000, 0x2040)
    unsigned long long lo[2] = {0x1000ull, 0x2000ull}, hi[2] = {0x1100ull, 0x2040ull};
    struct Case { unsigned long long p, bytes; int n; int want; } cases[] = {
        {0x1000, 16, 2, 1},   // first element
        {0x10f0, 16, 2, 1},   // last element
        {0x2030, 16, 2, 1},   // last element of the second buffer
        {0x1100, 0, 2, 0},    // empty access at the end: starts outside
        {0x0ff0, 16, 2, 0},   // below the first buffer
        {0x10f8, 16, 2, 0},   // straddles its end
        {0x1100, 16, 2, 0},   // just past its end
        {0x1800, 4, 2, 0},    // in the gap
        {0x2040, 8, 2, 0},    // past the second buffer
        {0x2000, 0x41, 2, 0}, // longer than the buffer
        {0x2000, 16, 1, 0},   // the second buffer unregistered (table of one)
        {0x1000, 16, 0, 0},   // empty table
    };
    int bad = 0;
    for (const Case& c : cases) {
        const int got = gfk::dbg_in_ranges(lo, hi, c.n, c.p, c.bytes) ? 1 : 0;
        if (got != c.want) {
            std::printf("case p=%llx bytes=%llu n=%d: got %d want %d\n", c.p, c.bytes, c.n, got,
                        c.want);
            ++bad;
        }
    }
    std::printf("%d\n", bad);
    return bad != 0;
}
"""


def test_range_check_refuses_out_of_range_accesses(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "dbg_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "dbg_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().splitlines()[-1] == "0"


def test_release_library_reports_no_debug_checks():
    if os.environ.get("GFK_DEBUG", "0") not in ("", "0"):
        pytest.skip("the debug library is loaded")
    b, f, a = gfk.gfk_debug_status(clear=False)
    assert (b, f, a) == (0, 0, 0)
