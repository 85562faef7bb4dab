"""Host-side checks of the multiply-add chains the code generator emits (no GPU).

The generator writes every maximal sum of three or more terms, whose inner
nodes have one user each, as a chain acc = t_1, acc = acc +- t_j (a term that
is not a product first).  These tests run the emitted statements in Python
and compare them with the expression graph's own interpreter:

* on small graphs: every term of a chained sum appears exactly once with its
  sign, a non-product term leads, a shared subsum is not merged into its
  users, and a sum of two terms is left as written;
* on the committed vacuum right-hand side (about 1800 statements): every output
  of the emitted code equals the graph's value on seeded inputs, up to the
  rounding of the reordered sums.
"""
import math
import pathlib
import re

import numpy as np

from paper_2606_02053_gb300 import inputs
from paper_2606_02053_gb300.codegen import bssn
from paper_2606_02053_gb300.codegen.expr import Graph, emit_function, evaluate

STMT = re.compile(r"const double (\w+) = (.+);")
OUT = re.compile(r"(\w+)\[(\d+)\] = (\w+);")


def run_emitted(body, in_values, params, in_array="in", out_array="out", param_struct="p"):
    """Execute the statements of an emitted function body; returns {k: out[k]}."""
    env = {"IN": list(in_values), "P": dict(params), "sqrt": math.sqrt, "fabs": abs, "fmax": max, "fmin": min}
    outs = {}

    def py(expr):
        expr = re.sub(rf"\b{in_array}\[(\d+)\]", r"IN[\1]", expr)
        return re.sub(rf"\b{param_struct}\.(\w+)", r"P['\1']", expr)

    for line in body.split("\n"):
        line = line.strip()
        m = STMT.fullmatch(line)
        if m:
            env[m.group(1)] = eval(py(m.group(2)), env)
            continue
        m = OUT.fullmatch(line)
        if m and m.group(1) == out_array:
            outs[int(m.group(2))] = env[m.group(3)]
    return outs


def body_of(src):
    return src[src.index("{") + 1:src.rindex("}")]


def small_graph():
    g = Graph()
    a, b, c, d, e, f = (g.input(x) for x in "abcdef")
    shared = a * b + c * d  # two users: its own sum, not merged into them
    s4 = a * b + c * e + d * f + a  # four terms, a non-product among them
    s_neg = -(a * c) - (b * d + e) - f * f  # signs through sub and neg
    products = a * b + b * c + c * d  # products only: one lone multiply is unavoidable
    pair = a * e + b * f  # two terms: left as written
    outs = [s4, s_neg, products, pair, shared * e, shared + f * f + c]
    return g, "abcdef", outs


def test_chained_sums_evaluate_like_the_graph():
    g, names, outs = small_graph()
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.standard_normal(len(names))
        want = evaluate(g, outs, dict(zip(names, x)), {})
        for chains in (True, False):
            src = emit_function(g, "f", list(names), outs, [], chains=chains)
            got = run_emitted(body_of(src), x, {})
            for k, w in enumerate(want):
                assert abs(got[k] - w) <= 1e-14 * (1 + abs(w)), (chains, k, got[k], w)


def test_chains_take_each_term_once_with_a_non_product_first():
    g, names, outs = small_graph()
    src = emit_function(g, "f", list(names), outs, [], chains=True)
    lines = [STMT.fullmatch(l.strip()) for l in body_of(src).split("\n")]
    defs = {m.group(1): m.group(2) for m in lines if m}
    order = [m.group(1) for m in lines if m]
    # the chain of s4 (output 0): its steps are the temporaries t<root>_j and t<root>
    root = OUT.search(src[src.index("out[0]"):]).group(3)
    steps = [t for t in order if t == root or t.startswith(root + "_")]
    assert len(steps) == 4  # four terms, one per step
    assert defs[steps[0]] == "in[0]"  # the non-product term a leads
    for prev, t in zip(steps, steps[1:]):  # each step adds one term to the previous one
        assert re.fullmatch(rf"{prev} \+ t\d+", defs[t]), (prev, defs[t])
    # every product of s4 appears once among the chain's operands
    prods = [defs[defs[t].split(" ")[-1]] for t in steps[1:]]
    assert sorted(prods) == sorted(["in[0] * in[1]", "in[2] * in[4]", "in[3] * in[5]"])
    # the two-term sum keeps its single add
    root_pair = OUT.search(src[src.index("out[3]"):]).group(3)
    assert not any(t.startswith(root_pair + "_") for t in order)
    assert re.fullmatch(r"t\d+ \+ t\d+", defs[root_pair])
    # the shared subsum a*b + c*d stays one statement, a single term of the chain of output 5
    root5 = OUT.search(src[src.index("out[5]"):]).group(3)
    steps5 = [t for t in order if t == root5 or t.startswith(root5 + "_")]
    assert len(steps5) == 3
    terms = [defs[steps5[0]]] + [defs[t].split(" ")[-1] for t in steps5[1:]]
    assert "in[2]" in terms  # the term c, a plain input, leads
    assert sum(1 for x in terms if x in defs and re.fullmatch(r"t\d+ \+ t\d+", defs[x])) == 1


def vac_rhs_body():
    import os

    path = os.path.join(os.path.dirname(__file__), "..", "paper_2606_02053_gb300", "csrc", "generated",
                        "bssn_algebra.cuh")
    src = pathlib.Path(path).read_text()
    ns = src[src.index("namespace alg_vac {"):src.index("}  // namespace alg_vac")]
    start = ns.index("void rhs(const In& in, Out&& out, const AlgebraParams& p) {")
    end = ns.index("\n}\n", start)
    return ns[start:end]


def test_emitted_vacuum_rhs_equals_the_graph():
    """The committed header's vacuum right-hand side, run statement by statement."""
    g, L, out = bssn.algebra(False, False)
    body = vac_rhs_body()
    assert "_0 = " in body  # the header carries multiply-add chains
    n = 8
    s = inputs.smooth_state(n, seed=41, scale=0.5)
    rng = np.random.default_rng(42)
    params = dict(eta=1.5, Kref=-0.3, lapse_c1=2.0, lapse_c2=0.0, shift_on=1.0, w=1.0 / 3.0)
    for p in [(1, 2, 3), (5, 0, 7), (7, 7, 7)]:
        vals = {f"u{f}": float(s[f, p[2], p[1], p[0]]) for f in range(L["nf"])}
        for nm in L["names"]:
            if nm not in vals:
                vals[nm] = float(rng.standard_normal())
        want = np.array(evaluate(g, out, vals, params), dtype=float)
        got_d = run_emitted(body, [vals[nm] for nm in L["names"]], params)
        got = np.array([got_d[k] for k in range(len(out))])
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-12 * scale, (p, np.abs(got - want).max(), scale)
