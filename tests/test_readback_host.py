"""CPU check of the host text readback: the parallel renderer must give the
same text (canonical names included), reached-agent count and numeral as
the sequential walk, on random forests of terms scattered over an arena.
Compiles tests/readback_check.cpp against the library's host sources."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1404_0076_gb300", "csrc")


def test_parallel_text_readback_matches_the_sequential_walk():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "readback_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        os.path.join(ROOT, "tests", "readback_check.cpp"), os.path.join(CSRC, "inet_text.cpp"),
                        "-o", exe], check=True)
        p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.startswith("ok 62 cases")
