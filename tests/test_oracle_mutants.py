"""The oracle's pins have teeth: each test below plants one plausible mistake
in a copy of the oracle's C source (a dropped term, a wrong sign, a
transposed operand or index, a wrong constant), builds it on the CPU, binds
the oracle's wrappers to it, and checks that at least one pin of
test_oracle_pins.py fails on it.  The shipped oracle is never modified.
"""
import os
import shutil

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(oracle.HERE, "ff_oracle.c")

# (name, exact source text, planted replacement)
MUTANTS = [
    ("add12: dropped (b - v) term", "float r = (a - (s - v)) + (b - v);", "float r = (a - (s - v));"),
    ("add12: operands transposed", "float r = (a - (s - v)) + (b - v);", "float r = (b - (s - v)) + (a - v);"),
    ("split: constant 2^12", "const float two_s_plus_1 = 4097.0f;", "const float two_s_plus_1 = 4096.0f;"),
    ("mul12 (Dekker): sign of a_hi*b_lo", "float err3 = err2 - (a_hi * b_lo);", "float err3 = err2 + (a_hi * b_lo);"),
    ("mul12 (fused): error sign", "float y = fmaf(a, b, -x);", "float y = -fmaf(a, b, -x);"),
    ("add22: dropped al", "s = (((ah - r) + bh) + bl) + al;", "s = (((ah - r) + bh) + bl);"),
    ("add22: branch test inverted", "if (fabsf(ah) >= fabsf(bh))", "if (fabsf(ah) <= fabsf(bh))"),
    ("add22: second branch uses al twice", "s = (((bh - r) + ah) + al) + bl;", "s = (((bh - r) + ah) + al) + al;"),
    ("add22: low parts swapped (first branch)", "s = (((ah - r) + bh) + bl) + al;", "s = (((ah - r) + bh) + al) + bl;"),
    ("add22: low parts swapped (second branch)", "s = (((bh - r) + ah) + al) + bl;", "s = (((bh - r) + ah) + bl) + al;"),
    ("mul22: printed Add12(t1, t2)",
     "    float t3 = ((ah * bl) + (al * bh)) + t2;\n    add12(t1, t3, rh, rl);\n}\n\n/* Mul22 with the paper's own",
     "    float t3 = ((ah * bl) + (al * bh)) + t2;\n    (void)t3;\n    add12(t1, t2, rh, rl);\n}\n\n/* Mul22 with the paper's own"),
    ("mul22: index al*bl for al*bh",
     "    mul12_fma(ah, bh, &t1, &t2);\n    float t3 = ((ah * bl) + (al * bh)) + t2;",
     "    mul12_fma(ah, bh, &t1, &t2);\n    float t3 = ((ah * bl) + (al * bl)) + t2;"),
    ("div22: dropped al", "float cl = ((((ah - uh) - ul) + al) - (ch * bl)) / bh;",
     "float cl = ((((ah - uh) - ul)) - (ch * bl)) / bh;"),
    ("div22: sign of ch*bl", "float cl = ((((ah - uh) - ul) + al) - (ch * bl)) / bh;",
     "float cl = ((((ah - uh) - ul) + al) + (ch * bl)) / bh;"),
    ("sqrt22: no halving", "float cc = ((((ah - u) - uu) + al) * 0.5f) / c;", "float cc = ((((ah - u) - uu) + al) * 1.0f) / c;"),
    ("sqrt22: dropped uu", "float cc = ((((ah - u) - uu) + al) * 0.5f) / c;", "float cc = ((((ah - u)) + al) * 0.5f) / c;"),
    ("dot: low part of the product dropped",
     "        mul22(x[2 * i], x[2 * i + 1], y[2 * i], y[2 * i + 1], &ph, &pl);\n        add22(h, l, ph, pl, &h, &l);",
     "        mul22(x[2 * i], x[2 * i + 1], y[2 * i], y[2 * i + 1], &ph, &pl);\n        add22(h, l, ph, 0.0f, &h, &l);"),
    ("dot backward: dx from x", "mul22(dout[0], dout[1], y[2 * i], y[2 * i + 1], &dx[2 * i], &dx[2 * i + 1]);",
     "mul22(dout[0], dout[1], x[2 * i], x[2 * i + 1], &dx[2 * i], &dx[2 * i + 1]);"),
    ("axpy: alpha on y", "mul22(alpha[0], alpha[1], x[2 * i], x[2 * i + 1], &ph, &pl);\n        add22(ph, pl, y[2 * i], y[2 * i + 1]",
     "mul22(alpha[0], alpha[1], y[2 * i], y[2 * i + 1], &ph, &pl);\n        add22(ph, pl, x[2 * i], x[2 * i + 1]"),
    ("gemv: A transposed", "const float *a = &A[2 * (r * lda + j)];\n                const float *xv",
     "const float *a = &A[2 * (j * lda + r)];\n                const float *xv"),
    ("gemv_t: dY column index", "const float *dy = &dY[2 * (c * lddy + r)];\n                float ph, pl;\n                mul22(a[0], a[1], dy[0], dy[1], &ph, &pl);",
     "const float *dy = &dY[2 * (c * lddy + j % lddy)];\n                float ph, pl;\n                mul22(a[0], a[1], dy[0], dy[1], &ph, &pl);"),
    ("accurate add: dropped tl", "    float w = tl + vl;", "    float w = vl;"),
    ("fast2sum: sign", "    float t = b - z;", "    float t = z - b;"),
    ("sum2: error term dropped", "        add12(p, x[i], &p, &q);\n        s = s + q;", "        add12(p, x[i], &p, &q);\n        s = s + 0.0f * q;"),
    ("dot2: product error r dropped", "        s = s + (q + r);", "        s = s + q;"),
    ("gemv_dA: X of the first right-hand side for every term",
     "const float *dy = &dY[2 * (c * lddy + r)];\n                const float *xv = &X[2 * (c * ldx + j)];",
     "const float *dy = &dY[2 * (c * lddy + r)];\n                const float *xv = &X[2 * j];"),
    ("gemv_dA: dY of row 0 for every row",
     "const float *dy = &dY[2 * (c * lddy + r)];\n                const float *xv = &X[2 * (c * ldx + j)];",
     "const float *dy = &dY[2 * (c * lddy)];\n                const float *xv = &X[2 * (c * ldx + j)];"),
    ("gemm: op(A) index not transposed", "transa ? &A[2 * (p * lda + i)]", "transa ? &A[2 * (i * lda + p)]"),
    ("gemm: B read by column", ": &B[2 * (p * ldb + j)];", ": &B[2 * (j * ldb + p)];"),
]

# quick pins first; each mutant stops at the first pin that fails
PINS = [
    (pins.test_add22_closed_forms, ()), (pins.test_add22_low_part_order, ()),
    (pins.test_add22_geometric_series_sum, ()),
    (pins.test_mul22_closed_forms, ()), (pins.test_div22_special_cases, ()),
    (pins.test_sqrt22_special_cases, ()), (pins.test_add22_accurate_special_cases, ()),
    (pins.test_sum_of_ones, ()), (pins.test_dot_with_ones_is_sum_and_n1_is_mul22, ()),
    (pins.test_axpy_special_cases, ()), (pins.test_dot_backward_accuracy, ()),
    (pins.test_gemv_identity_and_transpose, ()), (pins.test_gemv_rows_within_bound, ()),
    (pins.test_gemv_dA_outer_product_and_bound, ()), (pins.test_add12_paper_anomaly_is_exact_under_rn, ()),
    (pins.test_split_matches_fractions, ()), (pins.test_split_nonoverlap_and_exact, ()),
    (pins.test_add12_random_wide_exponents_exact, ()), (pins.test_mul12_random_domain, ()),
    (pins.test_add22_bound_random, ()), (pins.test_mul22_bound_random, ()), (pins.test_div22_accuracy, ()),
    (pins.test_sqrt22_accuracy_and_square_roundtrip, ()),
    (pins.test_add22_accurate_bound_random_with_cancellation, ()),
    (pins.test_dot2_within_oro_bound_small_n, (1e8,)), (pins.test_sum2_within_oro_bound_and_exact_cases, ()),
    (pins.test_dot2_reduces_to_sum2_and_twoproduct, ()), (pins.test_add22_reduces_to_add12, ()),
    (pins.test_mul22_reduces_to_mul12, ()), (pins.test_mul12_bruteforce_exact_and_forms_agree, ()),
    (pins.test_dot_ill_conditioned_within_bound, (1e12,)),
    (pins.test_gemm_small_integers_exact, ()), (pins.test_gemm_within_bound_and_transpose_identity, ()),
]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_mutants")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,orig,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(mutant_dir, name, orig, repl):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site not unique or missing: {name}"
    tag = "m%02d" % [m[0] for m in MUTANTS].index(name)
    csrc = os.path.join(mutant_dir, f"ff_oracle_{tag}.c")
    with open(csrc, "w") as fh:
        fh.write(src.replace(orig, repl))
    so = os.path.join(mutant_dir, f"liboracle_{tag}.so")
    oracle.compile_sources([csrc, os.path.join(oracle.HERE, "ff_exact.c")], so)
    prev = oracle.swap_library(so)
    caught = None
    try:
        for fn, args in PINS:
            try:
                fn(oracle, *args)
            except Exception as exc:  # a failing pin: the mistake is caught
                caught = f"{fn.__name__}: {type(exc).__name__}"
                break
    finally:
        oracle.swap_library(prev)
    assert caught is not None, f"no pin caught the planted mistake: {name}"
