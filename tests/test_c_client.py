"""The C ABI from a C99 program (tests/c/plan_from_c.c): the header compiles as C with every struct
at its documented size, and planning, inspection, OpenQASM parse / export and the error path work
through the shared library. Host entry points only: no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2404_09213_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_2404_09213_gb300")


def test_c99_client(lib_dir):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    out_dir = os.path.join(lib_dir, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "plan_from_c")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "plan_from_c.c"), "-L", lib_dir, "-lqsim",
                    "-Wl,-rpath," + lib_dir, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.splitlines()
    assert lines[0] == "info 2 4 1 1 1"                      # 2 qubits, 4 gates, 1 param, 1 input, 1 pass
    assert lines[1] == "qasm 3 1 2 0.78539816339744828"      # pi/4 parsed to the nearest double
    assert lines[2].startswith("error -2 gate 0:")
