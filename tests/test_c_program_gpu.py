"""A plain C program drives the reductions through the C ABI the way the
header documents it: device buffers from cudaMalloc, the reduction workspace
zeroed once with cudaMemset, then several ff_dot / ff_sum / ff_sum2 calls on
that one workspace (each call leaves its arrival ticket zero for the next),
and results read back with cudaMemcpy.  The results must equal, bit for
bit, the same calls made through the Python wrappers."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"

C_SRC = r"""
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "ff.h"

#define CHECK(x) do { if ((x) != 0) { fprintf(stderr, "failed: %s\n", #x); return 1; } } while (0)

int main(int argc, char** argv)
{
    if (argc != 4) return 2;
    size_t n = (size_t)atol(argv[1]);
    FILE* f = fopen(argv[2], "rb");
    if (!f) return 3;
    ff2* hx = (ff2*)malloc(n * sizeof(ff2));
    ff2* hy = (ff2*)malloc(n * sizeof(ff2));
    float* hz = (float*)malloc(n * sizeof(float));
    if (fread(hx, sizeof(ff2), n, f) != n || fread(hy, sizeof(ff2), n, f) != n || fread(hz, sizeof(float), n, f) != n)
        return 4;
    fclose(f);
    ff2 *x, *y, *out;
    float* z;
    void* ws;
    size_t wsb = ff_reduce_workspace_bytes(n);
    CHECK(cudaMalloc((void**)&x, n * sizeof(ff2)));
    CHECK(cudaMalloc((void**)&y, n * sizeof(ff2)));
    CHECK(cudaMalloc((void**)&z, n * sizeof(float)));
    CHECK(cudaMalloc((void**)&out, 4 * sizeof(ff2)));
    CHECK(cudaMalloc(&ws, wsb));
    CHECK(cudaMemset(ws, 0, wsb));      /* once, when the workspace is made */
    CHECK(cudaMemcpy(x, hx, n * sizeof(ff2), cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(y, hy, n * sizeof(ff2), cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(z, hz, n * sizeof(float), cudaMemcpyHostToDevice));
    CHECK(ff_dot(x, y, n, out + 0, ws, wsb, 0));
    CHECK(ff_sum(x, n, out + 1, ws, wsb, 0));
    CHECK(ff_sum2(z, n, out + 2, ws, wsb, 0));
    CHECK(ff_dot(x, y, n, out + 3, ws, wsb, 0));   /* the same workspace again */
    ff2 res[4];
    CHECK(cudaMemcpy(res, out, sizeof(res), cudaMemcpyDeviceToHost));
    f = fopen(argv[3], "wb");
    if (!f || fwrite(res, sizeof(ff2), 4, f) != 4) return 5;
    fclose(f);
    return 0;
}
"""


def test_c_program_reductions_match_the_wrappers(tmp_path):
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    libdir = os.path.dirname(lib._name)
    src = tmp_path / "red.c"
    src.write_text(C_SRC)
    exe = tmp_path / "red"
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-isystem", os.path.join(CUDA, "include"), str(src), "-o", str(exe), "-L", libdir, "-lff",
                        "-L", os.path.join(CUDA, "lib64"), "-lcudart", f"-Wl,-rpath,{libdir}",
                        f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    n = 1_000_003
    g = inputs.ill_dot(n, 1e9, inputs.seed_for(2, 80))
    z = g.x[:, 0].contiguous()
    data = tmp_path / "in.bin"
    with open(data, "wb") as fh:
        fh.write(g.x.numpy().tobytes())
        fh.write(g.y.numpy().tobytes())
        fh.write(z.numpy().tobytes())
    res = tmp_path / "out.bin"
    r = subprocess.run([str(exe), str(n), str(data), str(res)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    got = np.fromfile(res, dtype=np.float32).reshape(4, 2)
    x, y, zd = g.x.cuda(), g.y.cuda(), z.cuda()
    want = np.stack([ff.dot(x, y).cpu().numpy(), ff.sum(x).cpu().numpy(), ff.sum2(zd).cpu().numpy(),
                     ff.dot(x, y).cpu().numpy()])
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
