"""The hand-written adjoints against FP64 central finite differences and an
FP64 reference gradient.

Dot: L = dout * sum_i x_i y_i, so dL/dx_i = dout * y_i.  The finite
difference perturbs one float-float input x_i by a power of two h (about
2^-10 |x_i|), evaluates L(x +- h) exactly (the oracle's superaccumulator,
rounded to binary128), and divides by the exact perturbation in binary64.
The kernel's gradient must agree with it, and with the binary64 product
dout * y_i, to the Mul22 bound 2^-44 (plus the binary64 rounding of the
references).  Sweeps the condition numbers of the ill-conditioned dot.

GEMV: L = sum_c <dY_c, (A X)_c>, dL/dX = A^T dY, checked against binary64
finite differences of L (evaluated in binary64) on sampled coordinates.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _val(p):
    return float(p[0]) + float(p[1])


@pytest.mark.parametrize("cond", [1e3, 1e6, 1e9, 1e12])
def test_dot_gradient_vs_fd_and_f64(cond):
    import paper_cs_0603115_gb300 as ff
    n = 1 << 10
    g = inputs.ill_dot(n, cond, inputs.seed_for(2, 20 + int(math.log10(cond))))
    xn, yn = g.x.numpy(), g.y.numpy()
    dout = inputs.scalar_ff(321).numpy()
    x = g.x.to(DEV).requires_grad_(True)
    y = g.y.to(DEV).requires_grad_(True)
    d = ff.ffdot(x, y)
    d.backward(torch.from_numpy(dout.copy()).to(DEV))
    dx = x.grad.cpu().numpy()
    dy = y.grad.cpu().numpy()
    dval = _val(dout)
    rng = np.random.default_rng(int(cond) % 1000)
    worst_fd = worst_ref = 0.0
    for i in rng.choice(n, size=64, replace=False):
        hi = float(xn[i, 0])
        h = 2.0 ** (math.floor(math.log2(abs(hi))) - 10)
        xp, xm = xn.copy(), xn.copy()
        xp[i, 0] = np.float32(hi + h)
        xm[i, 0] = np.float32(hi - h)
        sp = oracle.exact_dot(xp, yn)
        sm = oracle.exact_dot(xm, yn)
        df = (sp[0] - sm[0]) + (sp[1] - sm[1])          # exact difference to ~2^-106 |L|
        dxi = (float(xp[i, 0]) - float(xm[i, 0]))        # exact in binary64
        fd = dval * df / dxi
        ref = dval * _val(yn[i])                         # binary64 reference gradient
        got = _val(dx[i])
        worst_fd = max(worst_fd, abs(got - fd) / abs(fd))
        worst_ref = max(worst_ref, abs(got - ref) / abs(ref))
    assert worst_fd <= 2.0 ** -44 + 2.0 ** -50
    assert worst_ref <= 2.0 ** -44 + 2.0 ** -51
    # dy: exact binary128 products against the kernel
    D = np.tile(dout, (n, 1))
    assert oracle.relerr("mul", D, xn, dy).max() <= 2.0 ** -44


def test_gemv_adjoint_vs_fd():
    import paper_cs_0603115_gb300 as ff
    m, n, k = 96, 80, 3
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 30))
    A, X, dY = gi.A.to(DEV), gi.X.to(DEV).requires_grad_(True), gi.dY.to(DEV)
    Y = ff.ffgemv(A, X)
    Y.backward(dY)
    g = X.grad.cpu().numpy()
    A64 = inputs.ff_to_f64(gi.A).numpy()
    X64 = inputs.ff_to_f64(gi.X).numpy()
    dY64 = inputs.ff_to_f64(gi.dY).numpy()

    def L(Xv):
        return float(np.sum(dY64 * (Xv @ A64.T)))

    # binary64 evaluation of L carries about (n + 4) 2^-53 of sum |dY| |X| |A|
    l_abs = float(np.sum(np.abs(dY64) * (np.abs(X64) @ np.abs(A64).T)))
    rng = np.random.default_rng(3)
    for _ in range(24):
        c, j = int(rng.integers(k)), int(rng.integers(n))
        h = 2.0 ** (math.floor(math.log2(abs(X64[c, j]))) - 10)
        Xp, Xm = X64.copy(), X64.copy()
        Xp[c, j] += h
        Xm[c, j] -= h
        fd = (L(Xp) - L(Xm)) / (2 * h)
        exact = float(np.dot(A64[:, j], dY64[c]))
        got = _val(g[c, j])
        scale = float(np.sum(np.abs(A64[:, j] * dY64[c])))
        assert abs(got - exact) <= m * 2.0 ** -44 * scale
        assert abs(got - fd) <= m * 2.0 ** -44 * scale + 2 * (n + 4) * 2.0 ** -53 * l_abs / h
