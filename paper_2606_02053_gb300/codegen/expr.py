"""Straight-line FP64 expression graphs -> CUDA device code.

A small tracer: arithmetic on ``Ex`` objects builds a hash-consed DAG (every
distinct (op, operands) pair exists once, so common subexpressions are shared
automatically), with constant folding and the trivial identities x+0, x*1,
x*0, -(-x).  ``emit_function`` writes the reachable part of the graph as one
``__device__`` function of ``const double`` temporaries in topological order;
nvcc then contracts multiply-add pairs into DFMA.  ``vjp`` builds, in the same
graph, the reverse-mode adjoint of chosen outputs with respect to chosen
inputs (one adjoint expression per input), which is how the adjoint kernels
are generated from the forward definition.

Ops: in, param, const, add, sub, mul, neg, rcp (1/x), sqrt, abs, max, min,
minmod.  Piecewise ops (abs, max, min, minmod) use one-sided derivatives at
their kinks (the branch taken), which is what a hand-written adjoint does.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence


class Graph:
    def __init__(self):
        self.ops: List[str] = []
        self.args: List[tuple] = []
        self.data: List[object] = []  # const value / input or param name
        self._cache: Dict[tuple, int] = {}
        self.inputs: Dict[str, int] = {}
        self.params: Dict[str, int] = {}

    def _node(self, op, args=(), data=None):
        key = (op, args, data)
        nid = self._cache.get(key)
        if nid is None:
            nid = len(self.ops)
            self.ops.append(op)
            self.args.append(args)
            self.data.append(data)
            self._cache[key] = nid
        return nid

    # public constructors
    def input(self, name: str) -> "Ex":
        nid = self._node("in", (), name)
        self.inputs[name] = nid
        return Ex(self, nid)

    def param(self, name: str) -> "Ex":
        nid = self._node("param", (), name)
        self.params[name] = nid
        return Ex(self, nid)

    def const(self, v: float) -> "Ex":
        return Ex(self, self._node("const", (), float(v)))

    def is_const(self, nid, v=None):
        if self.ops[nid] != "const":
            return False
        return v is None or self.data[nid] == v


def _c(g: Graph, x) -> "Ex":
    if isinstance(x, Ex):
        return x
    return g.const(float(x))


class Ex:
    __slots__ = ("g", "id")

    def __init__(self, g: Graph, nid: int):
        self.g = g
        self.id = nid

    # ---- folding helpers ----
    def _cv(self):
        return self.g.data[self.id] if self.g.ops[self.id] == "const" else None

    def __add__(self, o):
        g = self.g
        o = _c(g, o)
        a, b = self._cv(), o._cv()
        if a is not None and b is not None:
            return g.const(a + b)
        if a == 0.0:
            return o
        if b == 0.0:
            return self
        if g.ops[o.id] == "neg":
            return self - Ex(g, g.args[o.id][0])
        x, y = sorted((self.id, o.id))
        return Ex(g, g._node("add", (x, y)))

    __radd__ = __add__

    def __sub__(self, o):
        g = self.g
        o = _c(g, o)
        a, b = self._cv(), o._cv()
        if a is not None and b is not None:
            return g.const(a - b)
        if b == 0.0:
            return self
        if a == 0.0:
            return -o
        if self.id == o.id:
            return g.const(0.0)
        if g.ops[o.id] == "neg":
            return self + Ex(g, g.args[o.id][0])
        return Ex(g, g._node("sub", (self.id, o.id)))

    def __rsub__(self, o):
        return _c(self.g, o) - self

    def __mul__(self, o):
        g = self.g
        o = _c(g, o)
        a, b = self._cv(), o._cv()
        if a is not None and b is not None:
            return g.const(a * b)
        if a == 0.0 or b == 0.0:
            return g.const(0.0)
        if a == 1.0:
            return o
        if b == 1.0:
            return self
        if a == -1.0:
            return -o
        if b == -1.0:
            return -self
        x, y = sorted((self.id, o.id))
        return Ex(g, g._node("mul", (x, y)))

    __rmul__ = __mul__

    def __truediv__(self, o):
        g = self.g
        o = _c(g, o)
        b = o._cv()
        if b is not None:
            return self * (1.0 / b)
        return self * o.rcp()

    def __rtruediv__(self, o):
        return _c(self.g, o) * self.rcp()

    def __neg__(self):
        g = self.g
        a = self._cv()
        if a is not None:
            return g.const(-a)
        if g.ops[self.id] == "neg":
            return Ex(g, g.args[self.id][0])
        return Ex(g, g._node("neg", (self.id,)))

    def rcp(self):
        g = self.g
        a = self._cv()
        if a is not None:
            return g.const(1.0 / a)
        return Ex(g, g._node("rcp", (self.id,)))


def _unary(op, x: Ex) -> Ex:
    g = x.g
    a = x._cv()
    if a is not None:
        return g.const({"sqrt": math.sqrt, "abs": abs}[op](a))
    return Ex(g, g._node(op, (x.id,)))


def sqrt(x: Ex) -> Ex:
    return _unary("sqrt", x)


def fabs(x: Ex) -> Ex:
    return _unary("abs", x)


def fmax(a: Ex, b: Ex) -> Ex:
    x, y = sorted((a.id, b.id))
    return Ex(a.g, a.g._node("max", (x, y)))


def fmin(a: Ex, b: Ex) -> Ex:
    x, y = sorted((a.id, b.id))
    return Ex(a.g, a.g._node("min", (x, y)))


def minmod(a: Ex, b: Ex) -> Ex:
    """0 if a, b differ in sign (or one is 0), else the one of smaller modulus."""
    return Ex(a.g, a.g._node("minmod", (a.id, b.id)))


# ---------------------------------------------------------------------------
# Reverse mode
# ---------------------------------------------------------------------------
def _reachable(g: Graph, roots: Sequence[int]) -> List[int]:
    seen = set()
    stack = list(roots)
    while stack:
        n = stack.pop()
        if n in seen:
            continue
        seen.add(n)
        stack.extend(g.args[n])
    return sorted(seen)  # node ids are created in topological order


def vjp(g: Graph, outputs: Sequence[Ex], cotangents: Sequence[Ex], wrt: Sequence[Ex]) -> List[Ex]:
    """Adjoint sum_k cot_k d out_k / d w for each w in wrt (as graph expressions)."""
    order = _reachable(g, [o.id for o in outputs])
    adj: Dict[int, List[Ex]] = {}
    for o, c in zip(outputs, cotangents):
        adj.setdefault(o.id, []).append(c)
    zero = g.const(0.0)

    def total(n):
        terms = adj.get(n)
        if not terms:
            return None
        s = terms[0]
        for t in terms[1:]:
            s = s + t
        return s

    def push(n, e):
        adj.setdefault(n, []).append(e)

    for n in reversed(order):
        op = g.ops[n]
        if op in ("in", "param", "const"):
            continue
        A = total(n)
        if A is None or A.id == zero.id:
            continue
        args = g.args[n]
        X = [Ex(g, a) for a in args]
        me = Ex(g, n)
        if op == "add":
            push(args[0], A)
            push(args[1], A)
        elif op == "sub":
            push(args[0], A)
            push(args[1], -A)
        elif op == "mul":
            push(args[0], A * X[1])
            push(args[1], A * X[0])
        elif op == "neg":
            push(args[0], -A)
        elif op == "rcp":
            push(args[0], -(A * me * me))
        elif op == "sqrt":
            push(args[0], A * 0.5 * me.rcp())
        elif op == "abs":
            push(args[0], A * Ex(g, g._node("sgn", (args[0],))))
        elif op in ("max", "min", "minmod"):
            # derivative selects the branch: emitted as a selector node
            sa = Ex(g, g._node(op + "_da", (args[0], args[1])))
            sb = Ex(g, g._node(op + "_db", (args[0], args[1])))
            push(args[0], A * sa)
            push(args[1], A * sb)
        else:
            raise NotImplementedError(op)
    out = []
    for w in wrt:
        t = total(w.id)
        out.append(t if t is not None else zero)
    return out


# ---------------------------------------------------------------------------
# CUDA emission
# ---------------------------------------------------------------------------
def _fmt(v: float) -> str:
    if v == 0.0:
        return "0.0"
    r = repr(float(v))
    if "e" not in r and "." not in r and "inf" not in r and "nan" not in r:
        r += ".0"
    return r


def _expr(g: Graph, n: int, name) -> str:
    op = g.ops[n]
    a = g.args[n]
    if op == "add":
        return f"{name(a[0])} + {name(a[1])}"
    if op == "sub":
        return f"{name(a[0])} - {name(a[1])}"
    if op == "mul":
        return f"{name(a[0])} * {name(a[1])}"
    if op == "neg":
        return f"-{name(a[0])}"
    if op == "rcp":
        return f"1.0 / {name(a[0])}"
    if op == "sqrt":
        return f"sqrt({name(a[0])})"
    if op == "abs":
        return f"fabs({name(a[0])})"
    if op == "sgn":
        return f"({name(a[0])} < 0.0 ? -1.0 : 1.0)"
    if op == "max":
        return f"fmax({name(a[0])}, {name(a[1])})"
    if op == "min":
        return f"fmin({name(a[0])}, {name(a[1])})"
    if op == "minmod":
        x, y = name(a[0]), name(a[1])
        return (f"(({x} > 0.0 && {y} > 0.0) ? fmin({x}, {y}) : "
                f"(({x} < 0.0 && {y} < 0.0) ? fmax({x}, {y}) : 0.0))")
    if op == "max_da":
        return f"({name(a[0])} >= {name(a[1])} ? 1.0 : 0.0)"
    if op == "max_db":
        return f"({name(a[0])} >= {name(a[1])} ? 0.0 : 1.0)"
    if op == "min_da":
        return f"({name(a[0])} <= {name(a[1])} ? 1.0 : 0.0)"
    if op == "min_db":
        return f"({name(a[0])} <= {name(a[1])} ? 0.0 : 1.0)"
    if op == "minmod_da":
        x, y = name(a[0]), name(a[1])
        return (f"((({x} > 0.0 && {y} > 0.0) && {x} <= {y}) || (({x} < 0.0 && {y} < 0.0) && {x} >= {y}) ? 1.0 : 0.0)")
    if op == "minmod_db":
        x, y = name(a[0]), name(a[1])
        return (f"((({x} > 0.0 && {y} > 0.0) && {x} > {y}) || (({x} < 0.0 && {y} < 0.0) && {x} < {y}) ? 1.0 : 0.0)")
    raise NotImplementedError(op)


FLOP_OPS = {"add", "sub", "mul", "neg", "rcp", "sqrt"}


def op_counts(g: Graph, outputs: Sequence[Ex]) -> Dict[str, int]:
    order = _reachable(g, [o.id for o in outputs])
    c: Dict[str, int] = {}
    for n in order:
        op = g.ops[n]
        if op in ("in", "param", "const"):
            continue
        c[op] = c.get(op, 0) + 1
    return c


_SUM_OPS = ("add", "sub", "neg")


def sum_chains(g: Graph, order: Sequence[int], out_ids: Sequence[int]):
    """The sums of the emitted code that are rebuilt as multiply-add chains.

    A sum tree is a maximal set of add / sub / neg nodes in which every node but
    the root has exactly one user, another node of the tree (and is no output).
    Its terms are the operands below it with their signs.  The real value is
    the same in any order of the terms; the rounding is that of a sequential
    sum.  A tree of k >= 3 terms becomes the chain acc = t_1, acc = acc +- t_j,
    whose every step can absorb a product term into one DFMA; the chain starts
    with a term that is not a product when there is one (so that no product is
    left as a lone multiply), the others follow in the order they become
    available, which keeps the products short-lived.

    Returns ({root: [(sign, term), ...]}, the set of interior nodes)."""
    uses: Dict[int, List[int]] = {}
    for n in order:
        for a in g.args[n]:
            uses.setdefault(a, []).append(n)
    outs = set(out_ids)

    def interior(n):
        u = uses.get(n, [])
        return g.ops[n] in _SUM_OPS and len(u) == 1 and n not in outs and g.ops[u[0]] in _SUM_OPS

    pos = {n: i for i, n in enumerate(order)}
    chains: Dict[int, List[tuple]] = {}
    inner = set()
    for n in order:
        if g.ops[n] not in _SUM_OPS or interior(n):
            continue
        terms: List[tuple] = []
        seen_inner: List[int] = []

        def collect(x, s, top):
            if top or interior(x):
                if not top:
                    seen_inner.append(x)
                op, a = g.ops[x], g.args[x]
                if op == "add":
                    collect(a[0], s, False)
                    collect(a[1], s, False)
                elif op == "sub":
                    collect(a[0], s, False)
                    collect(a[1], -s, False)
                else:  # neg
                    collect(a[0], -s, False)
            else:
                terms.append((s, x))

        collect(n, 1, True)
        if len(terms) < 3:
            continue
        by_pos = sorted(terms, key=lambda st: pos[st[1]])
        lead = [st for st in by_pos if g.ops[st[1]] != "mul"]
        if lead:
            pos_lead = [st for st in lead if st[0] > 0]
            first = (pos_lead or lead)[0]
        else:
            first = by_pos[0]
        rest = list(by_pos)
        rest.remove(first)
        chains[n] = [first] + rest
        inner.update(seen_inner)
    return chains, inner


def emit_function(g: Graph, fname: str, in_names: Sequence[str], out_exprs: Sequence[Ex], params: Sequence[str],
                  in_array="in", out_array="out", param_struct="p", qualifiers="__device__ __forceinline__",
                  extra_args="", accessors=False, order=None, chains=True) -> str:
    """Emit `void fname(const double* in, double* out, const ParamT& p)`.

    in_names[i] is the input name stored at in[i]; outputs go to out[k].
    With ``accessors`` the function is a template over the input and output
    types (anything with ``in[i]`` and ``out[k] = v``, e.g. loads straight from
    global memory and a store functor), and each output is written as soon as
    its value exists.  ``order`` (a list of the reachable non-leaf nodes) fixes
    the statement order; the default is creation (topological) order.  With
    ``chains`` every sum of three or more terms is written as a multiply-add
    chain (``sum_chains``): each step is emitted as soon as its term exists."""
    in_index = {nm: i for i, nm in enumerate(in_names)}
    reach = _reachable(g, [o.id for o in out_exprs])
    if order is None:
        order = reach
    else:
        leaves = [n for n in reach if g.ops[n] in ("in", "param", "const")]
        assert sorted(order) == sorted(n for n in reach if g.ops[n] not in ("in", "param", "const"))
        order = leaves + list(order)
    outs_of: Dict[int, List[int]] = {}
    for k, o in enumerate(out_exprs):
        outs_of.setdefault(o.id, []).append(k)
    cmap, inner = sum_chains(g, order, [o.id for o in out_exprs]) if chains else ({}, set())
    pos = {n: i for i, n in enumerate(order)}
    steps_at: Dict[int, List[tuple]] = {}  # position -> [(root, step index)]
    for r, terms in cmap.items():
        p = -1
        for j, (_, x) in enumerate(terms):
            p = max(p, pos[x])
            steps_at.setdefault(p, []).append((r, j))
    names: Dict[int, str] = {}
    lines = []
    written = set()

    def write_outputs(n, t):
        if accessors:
            for k in outs_of.get(n, []):
                lines.append(f"  {out_array}[{k}] = {t};")
                written.add(k)

    for i, n in enumerate(order):
        op = g.ops[n]
        if op == "in":
            nm = g.data[n]
            if nm not in in_index:
                raise KeyError(f"input {nm} not in the input list")
            names[n] = f"{in_array}[{in_index[nm]}]"
        elif op == "param":
            names[n] = f"{param_struct}.{g.data[n]}"
        elif op == "const":
            names[n] = _fmt(g.data[n])
        elif n not in inner and n not in cmap:
            t = f"t{n}"
            lines.append(f"  const double {t} = {_expr(g, n, lambda a: names[a])};")
            names[n] = t
            write_outputs(n, t)
        for r, j in steps_at.get(i, []):
            terms = cmap[r]
            s, x = terms[j]
            last = j == len(terms) - 1
            t = f"t{r}" if last else f"t{r}_{j}"
            if j == 0:
                rhs = names[x] if s > 0 else f"-{names[x]}"
            else:
                rhs = f"t{r}_{j - 1} {'+' if s > 0 else '-'} {names[x]}"
            lines.append(f"  const double {t} = {rhs};")
            if last:
                names[r] = t
                write_outputs(r, t)
    for k, o in enumerate(out_exprs):
        if k not in written:
            lines.append(f"  {out_array}[{k}] = {names[o.id]};")
    if accessors:
        sig = (f"template <class In, class Out>\n{qualifiers} void {fname}(const In& {in_array}, Out&& {out_array}")
    else:
        sig = f"{qualifiers} void {fname}(const double* __restrict__ {in_array}, double* __restrict__ {out_array}"
    if params:
        sig += f", const {params[0]}& {param_struct}"
    sig += extra_args + ")"
    return sig + " {\n" + "\n".join(lines) + "\n}\n"


# ---------------------------------------------------------------------------
# Host-side interpreter (numpy), for checking generated algebra on the CPU
# ---------------------------------------------------------------------------
def evaluate(g: Graph, outputs: Sequence[Ex], inputs: Dict[str, float], params: Dict[str, float]):
    import numpy as np

    order = _reachable(g, [o.id for o in outputs])
    val: Dict[int, float] = {}
    for n in order:
        op = g.ops[n]
        a = [val[x] for x in g.args[n]]
        if op == "in":
            v = inputs[g.data[n]]
        elif op == "param":
            v = params[g.data[n]]
        elif op == "const":
            v = g.data[n]
        elif op == "add":
            v = a[0] + a[1]
        elif op == "sub":
            v = a[0] - a[1]
        elif op == "mul":
            v = a[0] * a[1]
        elif op == "neg":
            v = -a[0]
        elif op == "rcp":
            v = 1.0 / a[0]
        elif op == "sqrt":
            v = np.sqrt(a[0])
        elif op == "abs":
            v = np.abs(a[0])
        elif op == "sgn":
            v = np.where(a[0] < 0.0, -1.0, 1.0)
        elif op == "max":
            v = np.maximum(a[0], a[1])
        elif op == "min":
            v = np.minimum(a[0], a[1])
        elif op == "minmod":
            x, y = a
            v = np.where((x > 0) & (y > 0), np.minimum(x, y), np.where((x < 0) & (y < 0), np.maximum(x, y), 0.0))
        else:
            raise NotImplementedError(op)
        val[n] = v
    return [val[o.id] for o in outputs]
