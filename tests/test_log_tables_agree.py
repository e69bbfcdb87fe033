"""The library's compile-time log tables (csrc/ssa_logtab.h: 128-bit
fixed-point series, evaluated by the C++ compiler) and the oracle's (Python
big-integer series) are produced independently; both must be the correctly
rounded values, so they must be identical."""
import os
import subprocess
import tempfile

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
#include <cstdio>
#include "ssa_logtab.h"
int main() {
  constexpr const ssa_logtab::Tables& T = ssa_logtab::kTables;
  printf("%llu %d %d\n", (unsigned long long)T.ln2, T.k3, T.k5);
  for (int i = 0; i < ssa_logtab::kCells; ++i)
    printf("%llu %llu\n", (unsigned long long)T.inv[i], (unsigned long long)T.lnf[i]);
  return 0;
}
"""


def test_library_and_oracle_log_tables_are_identical():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "tab.cpp")
        exe = os.path.join(d, "tab")
        open(src, "w").write(PROBE)
        subprocess.run(["g++", "-std=c++17", "-fconstexpr-ops-limit=1000000000", "-I",
                        os.path.join(ROOT, "paper_1007_1768_gb300", "csrc"), "-o", exe, src], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    inv, lnf, ln2, k3, k5 = oracle.log_constants()
    head = [int(v) for v in lines[0].split()]
    assert head == [ln2, k3, k5]
    for i in range(512):
        a, b = (int(v) for v in lines[1 + i].split())
        assert (a, b) == (inv[i], lnf[i]), i
