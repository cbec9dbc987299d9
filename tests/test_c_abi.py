"""The C boundary used from plain C (no Python in the loop, no GPU): a small
C program links the library, checks pattern validation and host-only plans,
and checks the morph transform against closed-form counts on the complete
graph (tests/c_abi_check.c)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_2012_04553_b300")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_program_against_closed_forms(tmp_path):
    exe = str(tmp_path / "c_abi_check")
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", LIBDIR, "-lpm_b300",
                           f"-Wl,-rpath,{LIBDIR}", "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "ok"
