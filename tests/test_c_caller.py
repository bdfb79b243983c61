"""The C ABI from plain C: tests/c/count_paths.c compiles against include/dm.h with gcc and links
libdmotif.so (checked here on any machine); on a GPU it runs and its counts, checksums and rows
equal the oracle's (6x6 grid: P5 = 1712, C4 = 200, closed forms pinned in the oracle tests)."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2508_21287_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "count_paths.c")


def _compile(tmp_path):
    from paper_2508_21287_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "count_paths")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
                           "-o", exe, "-L", os.path.dirname(lib), "-ldmotif",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    return exe


def test_c_caller_compiles_and_links(tmp_path):
    exe = _compile(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_caller_matches_oracle(tmp_path):
    exe = _compile(tmp_path)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    g = I.grid(6, 6)
    p5, c4 = oracle.enumerate(g, I.path(5)), oracle.enumerate(g, I.cycle(4))
    assert out[0] == f"{p5.count} {p5.checksum}" and p5.count == 1712
    assert out[1] == f"{c4.count} {c4.checksum}" and c4.count == 200
    rows = np.array([[int(x) for x in line.split()] for line in out[2:] if line.strip()], dtype=np.int32)
    assert np.array_equal(rows, c4.rows)
