"""The C ABI from a C program (no Python in the caller): tests/c_abi_ghz.c includes qs.h as
plain C99, links libqs.so, and checks GHZ states through compiled plans (every mode, both
dtypes), the per-gate calls and the serving calls against the closed form.  On the CPU the
program is only compiled and linked (qs.h is valid C); on the GPU it runs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

qs = pytest.importorskip("paper_2010_09746_gb300")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    qs._lib.load()   # builds the library if needed
    libdir = os.path.dirname(qs.lib_path())
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_ghz")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", os.path.join(ROOT, "tests", "c_abi_ghz.c"),
                        "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lqs", f"-Wl,-rpath,{libdir}", "-lm",
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_c_and_program_links(program):
    assert os.path.exists(program)


@pytest.mark.gpu
def test_c_program_runs(program):
    r = subprocess.run([program], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.strip() == "ok"
