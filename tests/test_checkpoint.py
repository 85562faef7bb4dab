"""Checkpoint / resume (cosmos_checkpoint_save / _load) on host buffers: no
GPU needed, the same file code as for device buffers (tests/test_gpu_checkpoint.py).

* a round trip is bitwise, padding columns are neither stored nor written;
* the header is one JSON object that names the grid, the parameters, the
  field order, t and the step counter;
* a checkpoint of another grid or other parameters, a flipped payload byte,
  a truncated or an extended file are refused (COSMOS_ECHECKPOINT) and leave
  the target untouched; a missing file is COSMOS_EIO.
"""
import json
import os
import pathlib

import numpy as np
import pytest

from paper_2606_02053_gb300 import build
from paper_2606_02053_gb300 import cosmos as C


@pytest.fixture(scope="module")
def lib():
    build.build()
    return C.lib()


def state_for(g, p, seed):
    nf = C.cosmos_nfields(p)
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((nf, g.nz, g.ny, g.pitch))
    s[..., g.nx:] = np.nan  # padding columns: must not be stored
    return np.ascontiguousarray(s)


def test_round_trip_is_bitwise_and_skips_padding(lib, tmp_path):
    g = C.make_grid((13, 7, 5), (0.1, 0.125, 0.2), x0=(-0.5, 0.25, 1.0), pitch=16)
    p = C.make_params(slicing=1, shift=0, fluid=1, scalar=1, eta=1.7, ko_sigma=0.05, w=0.3, H0=3.5, t0=0.25)
    a = state_for(g, p, 1)
    path = str(tmp_path / "ck.bin")
    assert C.cosmos_checkpoint_save(path, g, p, a, t=1.0 / 3.0, step=123456789012) == C.COSMOS_OK
    nf = C.cosmos_nfields(p)
    assert os.path.getsize(path) == 4096 + nf * 13 * 7 * 5 * 8
    assert not os.path.exists(path + ".partial")
    b = np.full_like(a, 7.0)
    code, t, step = C.cosmos_checkpoint_load(path, g, p, b)
    assert code == C.COSMOS_OK and t == 1.0 / 3.0 and step == 123456789012
    assert np.array_equal(a[..., :13].view(np.int64), b[..., :13].view(np.int64))
    assert np.all(b[..., 13:] == 7.0)


def test_header_is_json_naming_the_run(lib, tmp_path):
    g = C.make_grid((9, 8, 6), 0.1, pitch=9)
    p = C.make_params(fluid=1, H0=2.0)
    path = str(tmp_path / "ck.bin")
    C.check(C.cosmos_checkpoint_save(path, g, p, state_for(g, p, 2), t=0.75, step=3))
    with open(path, "rb") as f:
        head = f.read(4096)
    assert head.endswith(b"\n")
    h = json.loads(head.decode())
    assert h["format"] == "cosmos-checkpoint" and h["n"] == [9, 8, 6] and h["h"] == [0.1, 0.1, 0.1]
    assert h["nfields"] == 28 and h["fields"][0] == "chi" and h["fields"][17] == "alpha"
    assert h["fields"][24:] == ["tau", "S_x", "S_y", "S_z"]
    assert h["params"]["fluid"] == 1 and h["params"]["H0"] == 2.0 and h["t"] == 0.75 and h["step"] == 3
    assert h["payload_bytes"] == 28 * 9 * 8 * 6 * 8
    ps = C.make_params(scalar=1)
    C.check(C.cosmos_checkpoint_save(path, g, ps, state_for(g, ps, 3), t=0.0, step=0))
    with open(path, "rb") as f:
        assert json.loads(f.read(4096).decode())["fields"][24:] == ["phi", "Pi"]


def test_mismatch_and_corruption_are_refused(lib, tmp_path):
    g = C.make_grid((10, 6, 5), 0.1, pitch=12)
    p = C.make_params(fluid=1, H0=2.0)
    a = state_for(g, p, 4)
    path = str(tmp_path / "ck.bin")
    C.check(C.cosmos_checkpoint_save(path, g, p, a, t=0.5, step=7))

    def refused(gg, pp, pth=path, code=C.COSMOS_ECHECKPOINT):
        t = np.full((C.cosmos_nfields(pp), gg.nz, gg.ny, gg.pitch), 3.0)
        assert C.cosmos_checkpoint_load(pth, gg, pp, t)[0] == code
        assert np.all(t == 3.0)

    refused(C.make_grid((10, 6, 6), 0.1, pitch=12), p)                  # other size
    refused(C.make_grid((10, 6, 5), 0.1 + 1e-16, pitch=12), p)          # other spacing (one ulp off)
    refused(C.make_grid((10, 6, 5), 0.1, x0=(0.0, 0.0, 1e-300), pitch=12), p)  # other origin
    refused(g, C.make_params(fluid=1, H0=2.0, w=0.3))                   # other parameters
    refused(g, C.make_params(fluid=1, scalar=1, H0=2.0))                # other field set
    refused(g, p, str(tmp_path / "missing.bin"), C.COSMOS_EIO)
    assert C.cosmos_checkpoint_load(path, C.make_grid((10, 6, 5), 0.1, pitch=16), p,
                                    np.zeros((28, 5, 6, 16)))[0] == C.COSMOS_OK  # another pitch is fine
    raw = pathlib.Path(path).read_bytes()
    for name, data in (("flip", raw[:5000] + bytes([raw[5000] ^ 1]) + raw[5001:]),
                       ("short", raw[:-8]), ("long", raw + b"\0" * 8), ("header", raw[:100])):
        bad = str(tmp_path / f"{name}.bin")
        pathlib.Path(bad).write_bytes(data)
        refused(g, p, bad)


def test_bad_arguments(lib, tmp_path):
    g = C.make_grid((10, 6, 5), 0.1)
    p = C.make_params()
    a = state_for(g, p, 5)
    assert C.lib().cosmos_checkpoint_save(None, g, p, a.ctypes.data, 0, 0.0, 0, None) == C.COSMOS_EINVAL
    assert C.lib().cosmos_checkpoint_save(str(tmp_path / "x").encode(), g, p, None, 0, 0.0, 0, None) == C.COSMOS_EINVAL
    assert C.cosmos_checkpoint_save(str(tmp_path / "no_dir" / "x.bin"), g, p, a, 0.0, 0) == C.COSMOS_EIO
    assert C.lib().cosmos_strerror(C.COSMOS_ECHECKPOINT).startswith(b"checkpoint")
