"""The C-ABI library builds, loads and exports every symbol include/*.h
declares, and its struct layouts agree between C and the ctypes binding.
No compute calls (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cosmos_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_02053_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cosmos_init_grid", "cosmos_rhs", "cosmos_rk4_step", "cosmos_constraints"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_symbols(libpath):
    from paper_2606_02053_gb300 import cosmos

    L = cosmos.lib()
    for n in declared_functions():
        assert hasattr(L, n)
        assert n in cosmos._SIGS, f"binding lacks {n}"
    assert L.cosmos_strerror(cosmos.COSMOS_EINVAL) == b"invalid argument"


def test_struct_layout_matches_c(tmp_path):
    from paper_2606_02053_gb300 import cosmos

    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "cosmos.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(cosmos_grid), sizeof(cosmos_params),"
        " sizeof(cosmos_id), offsetof(cosmos_grid, h), offsetof(cosmos_params, eta), offsetof(cosmos_id, q));"
        "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    assert vals == [ctypes.sizeof(cosmos.cosmos_grid), ctypes.sizeof(cosmos.cosmos_params),
                    ctypes.sizeof(cosmos.cosmos_id), cosmos.cosmos_grid.h.offset, cosmos.cosmos_params.eta.offset,
                    cosmos.cosmos_id.q.offset]


def test_host_side_validation_without_gpu(libpath):
    """Size queries and argument checks run on the host only."""
    from paper_2606_02053_gb300 import cosmos as C

    g = C.make_grid((20, 12, 9), 0.05, pitch=24)
    p = C.make_params(fluid=1)
    assert C.cosmos_nfields(p) == 28
    assert C.cosmos_field_stride(g) == 24 * 12 * 9
    fs = 24 * 12 * 9
    rk4 = C.cosmos_workspace_bytes(g, p, C.COSMOS_OP_RK4)
    assert rk4 >= (3 * 28 + 16) * fs * 8
    bad = C.make_grid((20, 12, 9), 0.05, pitch=10)  # pitch < nx
    assert C.cosmos_workspace_bytes(bad, p, C.COSMOS_OP_RK4) == 0
    assert C.lib().cosmos_rhs(ctypes.byref(bad), ctypes.byref(p), None, None, 0.0, None, 0, None) == C.COSMOS_EINVAL
    pw = C.make_params(fluid=1, w=0.0)
    assert C.lib().cosmos_rhs(ctypes.byref(g), ctypes.byref(pw), None, None, 0.0, None, 0, None) == C.COSMOS_EINVAL
