"""Host-side logic of the library checked on the CPU (no GPU)."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_01495_gb300", "csrc")


def test_invariant_division_is_exact():
    """Multiply-high division used to delinearise keys equals n / d."""
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "udiv_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "udiv_check.cpp")], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad=0" in r.stdout
