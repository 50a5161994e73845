"""The multi-solve engine's graph-cache key without a GPU.  A C++ program compiled with the host
compiler includes the engine's host-only signature header and replays the sequence that once
replayed a dead solve's graph: a solve finishes in slot 0, its handle is destroyed, and a new
solve is admitted into slot 0 (its handle may sit at the same address).  The tick signatures of
the two solves must differ, and a signature must name the slots it includes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_12522_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "engine_sig.h"
using cmcg::detail::TickSignature;
int main() {
    int fails = 0;
    auto check = [&](bool ok, const char* what) { if (!ok) { std::printf("FAIL %s\n", what); ++fails; } };
    const int OUTER = 2, INNER = 3;
    // tick configuration of the first solve (submission 1) in slot 0 beside a solve in slot 1
    TickSignature a; a.add(0, INNER, 1); a.add(1, INNER, 2);
    // the same slots and units after slot 0 was released and refilled (submission 3)
    TickSignature b; b.add(0, INNER, 3); b.add(1, INNER, 2);
    check(a != b, "a refilled slot gives a new signature");
    TickSignature a2; a2.add(0, INNER, 1); a2.add(1, INNER, 2);
    check(a == a2, "the same solves in the same units give the same signature");
    TickSignature c; c.add(0, OUTER, 1); c.add(1, INNER, 2);
    check(a != c, "a unit change gives a new signature");
    check(a.names_slot(0) && a.names_slot(1) && !a.names_slot(2), "names_slot");
    TickSignature d; d.add(4, INNER, 7);
    check(d.names_slot(4) && !d.names_slot(0) && !d.names_slot(7) && !d.names_slot(3), "names_slot by slot only");
    TickSignature e;
    check(e.empty() && !e.names_slot(0), "empty signature");
    a.clear();
    check(a.empty() && a != a2, "clear");
    std::printf(fails ? "FAILED\n" : "OK\n");
    return fails;
}
"""


def test_refilled_slot_never_matches_the_old_signature(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "sig.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "sig"
    r = subprocess.run([cxx, "-std=c++17", "-Wall", "-Werror", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout
