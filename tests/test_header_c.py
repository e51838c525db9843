"""The C ABI is usable from plain C and C++: include/ff.h compiles as C11 and
C++17 with warnings as errors (the CUDA runtime headers it includes are
treated as system headers), and a C program linked against libff.so calls it
(host-side paths only, no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "ff.h"

int main(void)
{
    ff2 x = {1.0f, 0.0f};
    int err = -1;
    if (strcmp(ff_status_string(FF_ERR_WORKSPACE), "FF_ERR_WORKSPACE") != 0) return 1;
    /* argument checks run on the host before anything touches the device */
    if (ff_add(NULL, &x, &x, 10, 0) != FF_ERR_INVALID_ARG) return 2;
    if (ff_add(NULL, NULL, NULL, 0, 0) != FF_OK) return 3;
    if (ff_gemm(2, 0, 4, 4, 4, &x, 4, &x, 4, &x, 4, 0) != FF_ERR_INVALID_ARG) return 4;
    if (ff_last_cuda_error(&err) != FF_OK || err != 0) return 5;
    if (ff_last_cuda_error(NULL) != FF_ERR_INVALID_ARG) return 6;
    printf("%s\n", ff_build_id());
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    from paper_cs_0603115_gb300 import build, _lib
    build.build()
    return _lib.load()


def _compiler(name):
    path = shutil.which(name)
    if path is None:
        pytest.skip(f"{name} not available")
    return path


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles_cleanly(tmp_path, lang):
    cc = _compiler("gcc" if lang == "c" else "g++")
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "ff.h"\nint ff_header_check(void) { return (int)sizeof(ff2) + (int)FF_OK; }\n')
    std = "-std=c11" if lang == "c" else "-std=c++17"
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        "-isystem", CUDA_INC, "-c", str(src), "-o", str(tmp_path / "h.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_the_library(tmp_path, lib):
    cc = _compiler("gcc")
    libdir = os.path.dirname(lib._name)
    src = tmp_path / "use.c"
    src.write_text(C_SRC)
    exe = tmp_path / "use"
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-isystem", CUDA_INC,
                        str(src), "-o", str(exe), "-L", libdir, "-lff", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == lib.ff_build_id().decode()
