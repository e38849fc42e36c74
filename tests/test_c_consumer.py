"""The C ABI from a C compiler (no GPU needed).

`tests/c_consumer.c` is a plain C99 program that includes the public headers
and links the library: the headers must compile as strict C, the library must
link and load from C, and the host calls (parameters, mesh, export, tile plan,
partition, error codes and messages) must behave as the headers say.
"""
import os
import shutil
import subprocess

import pytest

from paper_2307_16758_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("compiler,lang", [("gcc", ["-std=c99"]), ("g++", ["-x", "c++", "-std=c++17"])])
def test_plain_c_program_uses_the_abi(tmp_path, compiler, lang):
    """The same program as strict C99 and as C++17 (the headers' extern "C" guards)."""
    if shutil.which(compiler) is None:
        pytest.skip(f"needs {compiler}")
    lib = B.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_consumer")
    cmd = [compiler, *lang, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_consumer.c"), "-o", exe, "-L", libdir, "-l:libswe.so",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
