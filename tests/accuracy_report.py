"""Accuracy report of the GPU results (the paper's Section 6.1 experiment,
Table 5, regenerated): run on a machine with a GPU,

    python tests/accuracy_report.py > accuracy.md

For each elementwise operator, 2^24 values of the elementwise workload are
computed on the GPU and compared with the exact result (binary128 /
superaccumulator references of the oracle): maximum relative error in log2
and a histogram of floor(-log2 rel err).  Add22 is split into inputs that
cancel (|a + b| < 2^-20 (|a| + |b|)) and inputs that do not.  The dot
product is measured on 2^26 values for each condition number, in units of
2^-44 sum |x_i y_i|.  The paper's own figures (7800GTX, faithful rounding,
denormals excluded) are printed beside ours for context.
"""
import json
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_cs_0603115_gb300 as ff  # noqa: E402
from paper_cs_0603115_gb300 import build as ffbuild  # noqa: E402
from paper_cs_0603115_gb300 import inputs  # noqa: E402


def hist(rel):
    rel = np.asarray(rel)
    bits = np.where(rel > 0, np.floor(-np.log2(np.where(rel > 0, rel, 1.0))), 999).astype(int)
    vals, counts = np.unique(bits, return_counts=True)
    return ", ".join(f"{'exact' if v == 999 else v}: {c}" for v, c in zip(vals, counts))


def mx(rel):
    m = float(np.max(rel)) if len(rel) else 0.0
    return "exact" if m == 0 else f"{math.log2(m):.2f}"


def main():
    ffbuild.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_accuracy.json")))["max_error_log2"]
    n = 1 << 24
    e = inputs.elementwise(n, inputs.seed_for(1, 0), device=dev)
    a, b, ab, asq = (t.cpu().numpy() for t in (e.a, e.b, e.ab, e.a_sqrt))
    print("# Accuracy of the GB300 float-float operators\n")
    print(f"2^24 values of the elementwise workload (seed {inputs.seed_for(1, 0)}), GPU results against exact "
          "references (binary128 / superaccumulator).  `max` is log2 of the largest relative error.\n")
    print("| operator | max (ours, GB300, IEEE RN) | paper (7800GTX, Table 5) | histogram of floor(-log2 rel err) |")
    print("|---|---|---|---|")
    se = ff.add12(e.ab).cpu().numpy()
    bad = oracle.count_sum2_mismatch(ab, se)
    print(f"| Add12 | {'exact' if bad == 0 else f'{bad} inexact'} | {gold['Add12']} | all {n} exact |")
    pe = ff.mul12(e.ab).cpu().numpy()
    bad = oracle.count_prod_mismatch(ab, pe)
    print(f"| Mul12 | {'exact' if bad == 0 else f'{bad} inexact'} | {gold['Mul12']} | all {n} exact |")
    r = ff.add(e.a, e.b).cpu().numpy()
    rel = oracle.relerr("add", a, b, r)
    av = np.abs(a[:, 0].astype(np.float64) + a[:, 1]) + np.abs(b[:, 0].astype(np.float64) + b[:, 1])
    sv = np.abs((a[:, 0].astype(np.float64) + a[:, 1]) + (b[:, 0].astype(np.float64) + b[:, 1]))
    canc = sv < 2.0 ** -20 * av
    print(f"| Add22 (all) | {mx(rel)} | {gold['Add22']} | {hist(rel)} |")
    print(f"| Add22 (no cancellation, {int((~canc).sum())}) | {mx(rel[~canc])} | | {hist(rel[~canc])} |")
    print(f"| Add22 (cancellation, {int(canc.sum())}) | {mx(rel[canc])} | | {hist(rel[canc])} |")
    bd = oracle.add22_bound(a, b, r)
    viol = int(np.sum(bd[:, 0] > np.maximum(bd[:, 1], bd[:, 2])))
    print(f"| Add22 bound of Section 4.1 | {viol} violations | | |")
    r = ff.add_accurate(e.a, e.b).cpu().numpy()
    rel = oracle.relerr("add", a, b, r)
    print(f"| accurate add (JMP Alg. 6) | {mx(rel)} | | {hist(rel)} |")
    r = ff.mul(e.a, e.b).cpu().numpy()
    rel = oracle.relerr("mul", a, b, r)
    print(f"| Mul22 | {mx(rel)} | {gold['Mul22']} | {hist(rel)} |")
    r = ff.div(e.a, e.b).cpu().numpy()
    rel = oracle.relerr("div", a, b, r)
    print(f"| Div22 | {mx(rel)} | (not in paper) | {hist(rel)} |")
    r = ff.sqrt(e.a_sqrt).cpu().numpy()
    rel = oracle.relerr("sqrt", asq, None, r)
    print(f"| Sqrt22 | {mx(rel)} | (not in paper) | {hist(rel)} |")
    del e
    torch.cuda.empty_cache()

    nd = 1 << 26
    print("\n## Dot products, n = 2^26\n")
    print("Error |r - x.y| in units of 2^-44 sum|x_i y_i|; the stated bound is n 2^-46 sum|x_i y_i| "
          f"= {nd / 4:.3g} units.\n")
    print("| cond (target) | cond (achieved, exact) | ff_dot (float-float inputs) | Dot2 (binary32 inputs) |")
    print("|---|---|---|---|")
    for cond in (1e3, 1e6, 1e9, 1e12):
        g = inputs.ill_dot(nd, cond, inputs.seed_for(2, int(math.log10(cond))), device=dev)
        res = ff.dot(g.x, g.y).cpu().numpy()
        xs, ys = g.x.cpu().numpy(), g.y.cpu().numpy()
        s_hi, _, A, E = oracle.exact_dot(xs, ys, res)
        g2 = inputs.ill_dot_f32(nd, cond, inputs.seed_for(5, int(math.log10(cond))), device=dev)
        r2 = ff.dot2(g2.x, g2.y).cpu().numpy()
        _, _, A2, E2 = oracle.exact_dot_f32(g2.x.cpu().numpy(), g2.y.cpu().numpy(), r2)
        print(f"| {cond:.0e} | {2 * A / abs(s_hi):.4g} | {abs(E) / (A * 2.0 ** -44):.3g} | "
              f"{abs(E2) / (A2 * 2.0 ** -44):.3g} |")
        del g, g2
        torch.cuda.empty_cache()


if __name__ == "__main__":
    main()
