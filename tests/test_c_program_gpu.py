"""Plain C programs drive the library through the C ABI the way the header
documents it, and their results must equal, bit for bit, the same calls made
through the Python wrappers.  The first runs the reductions: device buffers
from cudaMalloc, the reduction workspace zeroed once with cudaMemset, then
several ff_dot / ff_sum / ff_sum2 calls on that one workspace (each call
leaves its arrival ticket zero for the next), results read back with
cudaMemcpy.  The second runs the GEMV family, a GEMM and a batched plan of a
dot, an AXPY and a GEMV instance."""
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


def _compile(tmp_path, name, source):
    """Compile and link a C11 program against libff.so and the CUDA runtime."""
    from paper_cs_0603115_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    libdir = os.path.dirname(lib._name)
    src = tmp_path / f"{name}.c"
    src.write_text(source)
    exe = tmp_path / name
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-isystem", os.path.join(CUDA, "include"), str(src), "-o", str(exe), "-L", libdir, "-lff",
                        "-L", os.path.join(CUDA, "lib64"), "-lcudart", f"-Wl,-rpath,{libdir}",
                        f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_reductions_match_the_wrappers(tmp_path):
    import paper_cs_0603115_gb300 as ff
    exe = _compile(tmp_path, "red", C_SRC)
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


C_SRC_MAT = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime.h>
#include "ff.h"

#define CHECK(x) do { if ((x) != 0) { fprintf(stderr, "failed: %s\n", #x); return 1; } } while (0)

static ff2* upload(const ff2* h, size_t count)
{
    ff2* d = NULL;
    if (cudaMalloc((void**)&d, count * sizeof(ff2)) != cudaSuccess) return NULL;
    if (h && cudaMemcpy(d, h, count * sizeof(ff2), cudaMemcpyHostToDevice) != cudaSuccess) return NULL;
    return d;
}

static int download(FILE* f, const ff2* d, size_t count)
{
    ff2* h = (ff2*)malloc(count * sizeof(ff2));
    if (!h || cudaMemcpy(h, d, count * sizeof(ff2), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    int bad = fwrite(h, sizeof(ff2), count, f) != count;
    free(h);
    return bad;
}

int main(int argc, char** argv)
{
    if (argc != 6) return 2;
    const int64_t m = atol(argv[1]), n = atol(argv[2]), k = atol(argv[3]);
    FILE* f = fopen(argv[4], "rb");
    if (!f) return 3;
    ff2* hA = (ff2*)malloc((size_t)(m * n) * sizeof(ff2));
    ff2* hX = (ff2*)malloc((size_t)(k * n) * sizeof(ff2));
    ff2* hdY = (ff2*)malloc((size_t)(k * m) * sizeof(ff2));
    if (fread(hA, sizeof(ff2), (size_t)(m * n), f) != (size_t)(m * n) ||
        fread(hX, sizeof(ff2), (size_t)(k * n), f) != (size_t)(k * n) ||
        fread(hdY, sizeof(ff2), (size_t)(k * m), f) != (size_t)(k * m))
        return 4;
    fclose(f);
    ff2* A = upload(hA, (size_t)(m * n));
    ff2* X = upload(hX, (size_t)(k * n));
    ff2* dY = upload(hdY, (size_t)(k * m));
    ff2* Y = upload(NULL, (size_t)(k * m));
    ff2* dX = upload(NULL, (size_t)(k * n));
    ff2* dA = upload(NULL, (size_t)(m * n));
    ff2* C = upload(NULL, (size_t)(m * k));
    ff2* bdot = upload(NULL, 1);
    ff2* baxpy = upload(NULL, (size_t)n);
    ff2* bgemv = upload(NULL, (size_t)m);
    if (!A || !X || !dY || !Y || !dX || !dA || !C || !bdot || !baxpy || !bgemv) return 6;

    CHECK(ff_gemv(A, m, n, n, X, n, k, Y, m, 0));
    size_t wsb = ff_gemv_t_workspace_bytes(m, n, k);
    void* ws = NULL;
    CHECK(cudaMalloc(&ws, wsb));
    CHECK(ff_gemv_t(A, m, n, n, dY, m, k, dX, n, ws, wsb, 0));
    CHECK(ff_gemv_dA(dY, m, m, X, n, n, k, dA, n, 0));
    CHECK(ff_gemm(0, 1, m, k, n, A, n, X, n, C, k, 0));   /* C = A X^T, m x k */

    ff_batch_instance inst[3];
    memset(inst, 0, sizeof(inst));
    inst[0].kind = FF_BATCH_DOT;  inst[0].n = n; inst[0].x = A; inst[0].y = X; inst[0].out = bdot;
    inst[1].kind = FF_BATCH_AXPY; inst[1].n = n; inst[1].x = X; inst[1].y = X + n; inst[1].out = baxpy;
    inst[1].alpha.hi = 1.5f; inst[1].alpha.lo = 3.0e-9f;
    inst[2].kind = FF_BATCH_GEMV; inst[2].n = n; inst[2].x = A; inst[2].y = X; inst[2].out = bgemv;
    inst[2].m = m; inst[2].lda = n;
    ff_batch_plan* plan = NULL;
    CHECK(ff_batch_plan_create(inst, 3, NULL, &plan));
    size_t bwsb = ff_batch_workspace_bytes(plan);
    void* bws = NULL;
    CHECK(cudaMalloc(&bws, bwsb));
    CHECK(ff_batch_run(plan, bws, bwsb, 0));
    CHECK(cudaDeviceSynchronize());
    ff_batch_plan_destroy(plan);

    f = fopen(argv[5], "wb");
    if (!f) return 5;
    if (download(f, Y, (size_t)(k * m)) || download(f, dX, (size_t)(k * n)) || download(f, dA, (size_t)(m * n)) ||
        download(f, C, (size_t)(m * k)) || download(f, bdot, 1) || download(f, baxpy, (size_t)n) ||
        download(f, bgemv, (size_t)m))
        return 7;
    fclose(f);
    return 0;
}
"""


def test_c_program_gemv_gemm_and_batch_match_the_wrappers(tmp_path):
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import batch
    exe = _compile(tmp_path, "mat", C_SRC_MAT)
    m, n, k = 301, 258, 3
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 160))
    data = tmp_path / "in.bin"
    with open(data, "wb") as fh:
        for t in (gi.A, gi.X, gi.dY):
            fh.write(t.contiguous().numpy().tobytes())
    res = tmp_path / "out.bin"
    r = subprocess.run([str(exe), str(m), str(n), str(k), str(data), str(res)], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    got = np.fromfile(res, dtype=np.float32).reshape(-1, 2)
    A, X, dY = gi.A.cuda(), gi.X.cuda(), gi.dY.cuda()
    alpha = (1.5, 3.0e-9)
    dot = torch.empty(1, 2, dtype=torch.float32, device="cuda")
    axpy = torch.empty(n, 2, dtype=torch.float32, device="cuda")
    gemv = torch.empty(m, 2, dtype=torch.float32, device="cuda")
    plan = batch.BatchPlan(batch.make_instances([(batch.DOT, A[0], X[0], dot, None),
                                                 (batch.AXPY, X[0], X[1], axpy, alpha),
                                                 (batch.GEMV, A, X[0], gemv, None)]))
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(axpy.view(torch.int32), ff.axpy(alpha, X[0], X[1]).view(torch.int32))
    want = [ff.gemv(A, X), ff.gemv_t(A, dY), ff.gemv_dA(dY, X), ff.gemm(A, X, transb=True), dot, axpy, gemv]
    want = np.concatenate([w.reshape(-1, 2).cpu().numpy() for w in want])
    plan.close()
    assert got.shape == want.shape
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
