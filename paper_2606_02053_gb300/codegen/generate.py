"""Write the generated CUDA headers of the pointwise algebra.

Usage: python -m paper_2606_02053_gb300.codegen.generate [--check]
"""
from __future__ import annotations

import argparse
import os
import pathlib
import sys

from . import bssn
from . import fluid as fluid_dsl
from .expr import Ex, emit_function, op_counts, vjp

ADJOINT_VARIANTS = ("vac", "fluid", "scalar", "fluid_scalar")

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(os.path.dirname(HERE), "csrc", "generated")

VARIANTS = [("vac", False, False), ("fluid", True, False), ("scalar", False, True), ("fluid_scalar", True, True)]

HEADER = """// GENERATED by paper_2606_02053_gb300/codegen/generate.py -- do not edit.
// Pointwise BSSN + matter right-hand side (without Kreiss-Oliger dissipation
// and without the fluid flux divergence), one grid point per call.
// Input layout and parameters: see paper_2606_02053_gb300/codegen/bssn.py.
#pragma once

struct AlgebraParams {
  double eta;       // Gamma-driver damping
  double Kref;      // background trace K_ref at the stage time
  double lapse_c1;  // d_t alpha = beta.d alpha - alpha (c1 + c2 alpha)(K - Kref)
  double lapse_c2;
  double shift_on;  // 1: Gamma-driver shift, 0: frozen shift
  double w;         // fluid equation of state P = w rho
};
"""


def render() -> dict:
    files = {}
    body = [HEADER]
    stats = []
    for name, fluid, scalar in VARIANTS:
        g, L, out = bssn.algebra(fluid, scalar)
        c = op_counts(g, out)
        stats.append((name, c))
        body.append(f"// variant {name}: fluid={int(fluid)} scalar={int(scalar)}; ops {dict(sorted(c.items()))}")
        body.append(f"namespace alg_{name} {{")
        body.append(f"constexpr int NF = {L['nf']};")
        body.append(f"constexpr int ND1 = {len(L['d1'])};")
        body.append(f"constexpr int ND2 = {len(L['d2'])};")
        body.append(f"constexpr int NIN = {L['nin']};")
        body.append(_table_fn("d1_field", L["d1"]))
        body.append(_table_fn("d2_field", L["d2"]))
        body.append(_slot_fn("d1_slot", L["d1"]))
        body.append(_slot_fn("d2_slot", L["d2"]))
        body.append(emit_function(g, "rhs", L["names"], out, ["AlgebraParams"], accessors=True))
        body.append(emit_function(g, "constraints", L["names"], g.constraints, ["AlgebraParams"]))
        if name in ADJOINT_VARIANTS:
            # reverse mode: in[0 .. NIN) as for rhs, in[NIN + f] = cotangent of out[f];
            # out[k] = sum_f cot_f d out_f / d in[k]
            w = [g.input(f"w{f}") for f in range(L["nf"])]
            wrt = [Ex(g, g.inputs[nm]) for nm in L["names"]]
            adj = vjp(g, out, w, wrt)
            stats.append((name + "_vjp", op_counts(g, adj)))
            body.append(f"// reverse mode of rhs: ops {dict(sorted(op_counts(g, adj).items()))}")
            body.append(emit_function(g, "rhs_vjp", L["names"] + [f"w{f}" for f in range(L["nf"])], adj,
                                      ["AlgebraParams"], accessors=True))
        if name == "vac":
            # reverse mode of H (first constraint) w.r.t. chi, d chi, dd chi: initial-data adjoint
            hb = g.input("hb")
            chi_in = ["u0"] + [f"d0_{k}" for k in range(3)] + [f"dd0_{m}" for m in range(6)]
            adjh = vjp(g, g.constraints[:1], [hb], [Ex(g, g.inputs[nm]) for nm in chi_in])
            body.append(emit_function(g, "ham_vjp_chi", L["names"] + ["hb"], adjh, ["AlgebraParams"]))
        body.append(f"}}  // namespace alg_{name}\n")
    files["bssn_algebra.cuh"] = "\n".join(body)
    fb = [FLUID_HEADER]
    g, names, out = fluid_dsl.prim()
    stats.append(("prim", op_counts(g, out)))
    fb.append("// inputs: " + ", ".join(names))
    # The fluid header keeps the sums as the formulas group them (no multiply-add chains): a
    # face flux is symmetric under the exchange of its left and right states (with the odd
    # components negated), and its paired sums (F_L + F_R, U_R - U_L) keep that symmetry bitwise,
    # so mirror-symmetric data keep their velocities exactly zero on the symmetry planes.
    fb.append(emit_function(g, "fluid_prim", names, out, ["FluidParams"], chains=False))
    qb = [g.input(f"qb{m}") for m in range(4)]
    adj = vjp(g, out, qb, [Ex(g, g.inputs[nm]) for nm in names])
    fb.append("// reverse mode: in[11 + m] = cotangent of (rho, v0, v1, v2)[m]; out = cotangents of the inputs")
    fb.append(emit_function(g, "fluid_prim_vjp", names + [f"qb{m}" for m in range(4)], adj, ["FluidParams"],
                            chains=False))
    for d in range(3):
        g, names, out = fluid_dsl.face_flux(d)
        stats.append((f"face{d}", op_counts(g, out)))
        if d == 0:
            fb.append("// face-flux inputs: " + ", ".join(names))
        fb.append(emit_function(g, f"fluid_face_flux_{d}", names, out, ["FluidParams"], chains=False))
        hb = [g.input(f"hb{m}") for m in range(4)]
        adj = vjp(g, out, hb, [Ex(g, g.inputs[nm]) for nm in names])
        fb.append(emit_function(g, f"fluid_face_flux_{d}_vjp", names + [f"hb{m}" for m in range(4)], adj,
                                ["FluidParams"], chains=False))
    files["fluid_algebra.cuh"] = "\n".join(fb)
    return files, stats


def _table_fn(name, values):
    expr = "-1"
    for m in reversed(range(len(values))):
        expr = f"(m == {m} ? {values[m]} : {expr})"
    return f"__host__ __device__ __forceinline__ constexpr int {name}(int m) {{ return {expr}; }}"


def _slot_fn(name, values):
    """Inverse table: field -> position in `values`, or -1."""
    expr = "-1"
    for m in reversed(range(len(values))):
        expr = f"(f == {values[m]} ? {m} : {expr})"
    return f"__host__ __device__ __forceinline__ constexpr int {name}(int f) {{ return {expr}; }}"


FLUID_HEADER = """// GENERATED by paper_2606_02053_gb300/codegen/generate.py -- do not edit.
// Fluid primitive recovery and Kurganov-Tadmor face fluxes (see
// paper_2606_02053_gb300/codegen/fluid.py for the formulas and the inputs).
#pragma once

struct FluidParams {
  double w;       // P = w rho
  double sqrt_w;  // sound speed
};
"""


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--check", action="store_true", help="fail if the committed files differ")
    a = ap.parse_args(argv)
    files, stats = render()
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = []
    for fn, text in files.items():
        path = os.path.join(OUT_DIR, fn)
        old = pathlib.Path(path).read_text() if os.path.exists(path) else None
        if old != text:
            stale.append(fn)
            if not a.check:
                with open(path, "w") as f:
                    f.write(text)
    for name, c in stats:
        print(name, sum(v for k, v in c.items()), dict(sorted(c.items())))
    if a.check and stale:
        print("stale:", stale)
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
