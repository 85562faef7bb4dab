"""The C-ABI library builds, loads and exports every symbol include/*.h
declares, and its struct layouts agree between C and the ctypes binding.
No compute calls (no GPU needed)."""
import ctypes
import glob
import os
import pathlib
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = pathlib.Path(h).read_text()
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
    # one field's offsets must fit in 32 bits: 2^31 elements per field is refused, one row less is sized
    huge = C.make_grid((1024, 2048, 1024), 0.05)
    assert C.cosmos_workspace_bytes(huge, p, C.COSMOS_OP_RK4) == 0
    assert C.cosmos_workspace_bytes(C.make_grid((1024, 2047, 1024), 0.05), p, C.COSMOS_OP_RK4) > 0
    pw = C.make_params(fluid=1, w=0.0)
    assert C.lib().cosmos_rhs(ctypes.byref(g), ctypes.byref(pw), None, None, 0.0, None, 0, None) == C.COSMOS_EINVAL


def test_both_constraint_entry_points_check_arguments_alike(libpath):
    """cosmos_constraints and its static-scratch variant refuse the same grids and
    parameters before any launch: here a small grid whose row pitch makes one field
    2^31 elements or more, a non-finite spacing and a negative KO strength."""
    from paper_2606_02053_gb300 import cosmos as C

    norms = (ctypes.c_double * 8)()
    fake_state = ctypes.c_void_p(1 << 12)  # never dereferenced: refused first
    p = C.make_params()
    cases = [(C.make_grid((32, 16, 16), 0.05, pitch=1 << 23), p),
             (C.make_grid((32, 16, 16), float("inf")), p),
             (C.make_grid((32, 16, 16), 0.05), C.make_params(ko_sigma=-0.1))]
    for g, pp in cases:
        assert C.lib().cosmos_constraints(ctypes.byref(g), ctypes.byref(pp), fake_state, None, norms, None, 0,
                                          None) == C.COSMOS_EINVAL
        assert C.lib().cosmos_constraints_noalloc(ctypes.byref(g), ctypes.byref(pp), fake_state, None, norms,
                                                  None) == C.COSMOS_EINVAL


def test_state_scan_host_checks_without_gpu(libpath):
    """The failure-detection scan sizes its workspace (one count per field) and
    refuses bad arguments before touching the device."""
    from paper_2606_02053_gb300 import cosmos as C

    g = C.make_grid((20, 12, 9), 0.05, pitch=24)
    for p, nf in ((C.make_params(), 24), (C.make_params(fluid=1, scalar=1), 30)):
        assert C.cosmos_workspace_bytes(g, p, C.COSMOS_OP_SCAN) == 256 * ((4 * nf + 255) // 256)
    p = C.make_params(fluid=1)
    counts = (ctypes.c_int * 28)()
    assert C.lib().cosmos_scan_state(ctypes.byref(g), ctypes.byref(p), None, counts, None, 0, None) == C.COSMOS_EINVAL
    assert C.lib().cosmos_scan_state(ctypes.byref(g), ctypes.byref(p), 8, counts, None, 0, None) == C.COSMOS_EALIGN
    assert C.lib().cosmos_scan_state(ctypes.byref(g), ctypes.byref(p), 256, counts, None, 0, None) == C.COSMOS_EINVAL


def test_autotuner_candidates_without_gpu(libpath):
    """The library's built-in candidate list (host only) is the one the Python side names."""
    from paper_2606_02053_gb300 import batch
    from paper_2606_02053_gb300 import cosmos as C

    assert [batch.as_tuple(t) for t in C.cosmos_batch_default_candidates()] == batch.CANDIDATES
    assert C.lib().cosmos_batch_autotune(None, None, 0, 1, None, None, None, None, None) == C.COSMOS_EINVAL
    assert C.lib().cosmos_strerror(C.COSMOS_EIO) == b"file could not be opened, read or written"


def test_fmr_struct_layout_matches_c(tmp_path):
    from paper_2606_02053_gb300 import cosmos

    src = tmp_path / "fsz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "cosmos.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(cosmos_fmr), offsetof(cosmos_fmr, grid),"
        " offsetof(cosmos_fmr, origin), offsetof(cosmos_fmr, lo), offsetof(cosmos_fmr, hi));return 0;}\n")
    exe = tmp_path / "fsz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    F = cosmos.cosmos_fmr
    assert vals == [ctypes.sizeof(F), F.grid.offset, F.origin.offset, F.lo.offset, F.hi.offset]


def test_fmr_hierarchy_validation_without_gpu(libpath):
    """Hierarchy checks (spacing ratio, alignment, ghost width, nesting) run on
    the host before anything is launched."""
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.inputs import nested_boxes

    p = C.make_params(fluid=1, H0=40.0)
    lv = nested_boxes(32, 1.0 / 32, (-0.5,) * 3, 3, [32, 32])
    good = C.make_fmr(lv, 32)
    nb = C.cosmos_fmr_workspace_bytes(good, p)
    fs = [C.cosmos_field_stride(good.grid[l]) for l in range(3)]
    assert nb >= 4 * 28 * (fs[0] + fs[1]) * 8  # saved states of levels 0 and 1
    assert C.cosmos_fmr_workspace_bytes(C.make_fmr(lv[:1], 32), p) > 0  # a single level is a plain grid

    def bad(edit):
        m = C.make_fmr(lv, 32)
        edit(m)
        return m

    cases = [
        lambda m: setattr(m, "levels", 0),
        lambda m: setattr(m, "levels", C.COSMOS_FMR_MAX_LEVELS + 1),
        lambda m: m.lo[1].__setitem__(0, 2),                      # fewer than 3 ghost layers
        lambda m: m.hi[2].__setitem__(1, 30),                     # 2 ghost layers above
        lambda m: m.origin[1].__setitem__(2, 16),                 # x0 no longer matches the origin
        lambda m: m.grid[2].h.__setitem__(0, 1.0 / 100),          # ratio not 2
    ]
    for edit in cases:
        m = bad(edit)
        assert C.cosmos_fmr_workspace_bytes(m, p) == 0
        assert C.lib().cosmos_fmr_step(ctypes.byref(m), ctypes.byref(p), None, 0.0, 0.1, None, 0,
                                       None) == C.COSMOS_EINVAL
    # a level 2 whose interpolation would read level 1's ghost points
    big = nested_boxes(32, 1.0 / 32, (-0.5,) * 3, 3, [32, 48])
    assert C.cosmos_fmr_workspace_bytes(C.make_fmr(big, 32), p) == 0
    # NULL states, short workspace
    assert C.lib().cosmos_fmr_step(ctypes.byref(good), ctypes.byref(p), None, 0.0, 0.1, None, 0,
                                   None) == C.COSMOS_EINVAL
    states = (ctypes.c_void_p * 3)(256, 512, 768)
    assert C.lib().cosmos_fmr_step(ctypes.byref(good), ctypes.byref(p), states, 0.0, 0.1, ctypes.c_void_p(256),
                                   nb - 8, None) == C.COSMOS_EWORKSPACE


def test_pipelined_host_evolution_refuses_bad_arguments_before_any_copy(libpath):
    """cosmos_evolve_host_many checks its buffers before it creates a stream or
    copies anything: a negative count or step count, nbuf outside 1..16, a NULL
    buffer, two device buffers that overlap, and a result buffer that overlaps an
    input buffer are refused; count = 0 does nothing.  The addresses are never
    dereferenced."""
    from paper_2606_02053_gb300 import cosmos as C

    g = C.make_grid((16, 8, 8), 0.05)
    p = C.make_params()
    bytes_ = C.cosmos_field_stride(g) * C.cosmos_nfields(p) * 8
    base = 1 << 20

    def arr(*xs):
        return (ctypes.c_void_p * max(len(xs), 1))(*xs)

    def call(count, ins, outs, devs, nbuf, steps=1, ws=None):
        return C.lib().cosmos_evolve_host_many(ctypes.byref(g), ctypes.byref(p), count, ins, outs, devs, nbuf, steps,
                                               0.0, 0.01, ws, 0, None)

    ins, outs = arr(base), arr(base + 4 * bytes_)
    devs = arr(base + 8 * bytes_, base + 10 * bytes_)
    assert call(0, None, None, None, 1) == C.COSMOS_OK
    assert call(-1, ins, outs, devs, 2) == C.COSMOS_EINVAL
    assert call(1, ins, outs, devs, 2, steps=-1) == C.COSMOS_EINVAL
    for nbuf in (0, 17):
        assert call(1, ins, outs, devs, nbuf) == C.COSMOS_EINVAL
    assert call(1, ins, arr(None), devs, 2) == C.COSMOS_EINVAL
    assert call(1, ins, outs, arr(base + 8 * bytes_, base + 8 * bytes_ + 256), 2) == C.COSMOS_EINVAL
    assert call(1, ins, arr(base + bytes_ // 2), devs, 2) == C.COSMOS_EINVAL  # result over the input
    assert call(2, arr(base, base + 2 * bytes_), arr(base + 4 * bytes_, base + 2 * bytes_ + 8), devs,
                2) == C.COSMOS_EINVAL  # a result over a later input
    assert call(1, ins, outs, arr(base + 8 * bytes_ + 8), 1) == C.COSMOS_EALIGN
    # with valid buffers the workspace check comes next, still before any copy
    assert call(1, ins, outs, devs, 2, ws=ctypes.c_void_p(base + 16 * bytes_)) == C.COSMOS_EWORKSPACE
