"""Batched scan (uneven grids, one persistent launch per stage, CUDA graph)
against the per-instance loop and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2606_02053_gb300 import build, cosmos

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cosmos.lib()
    return cosmos


def scan_setup(C, ns, mus, fluid=1):
    grids, dts, ids = [], [], []
    for n, mu in zip(ns, mus):
        h = 1.0 / n
        grids.append(C.make_grid(n, h, x0=(-(n // 2) * h,) * 3))
        dts.append(0.25 * h)
        ids.append(C.make_id(1, mu=mu, sigma=0.14, q=(1.0, 0.9, 1.1)))
    p = C.make_params(fluid=fluid, w=1.0 / 3.0, H0=20.0)
    return grids, dts, ids, p


def per_instance(C, grids, dts, ids, p, steps):
    from paper_2606_02053_gb300.evolve import Evolution

    out = []
    for g, dt, ident in zip(grids, dts, ids):
        ev = Evolution(g, p)
        ev.init(ident)
        ev.step(0.0, dt, steps)
        out.append(ev.state.clone())
    return out


def test_batch_equals_per_instance_loop_bitwise_all_tunings(C):
    from paper_2606_02053_gb300.batch import CANDIDATES, BatchScan

    ns = [18, 21, 24]
    grids, dts, ids, p = scan_setup(C, ns, [0.4, 0.6, 0.8])
    steps = 3
    ref = per_instance(C, grids, dts, ids, p, steps)
    for use_graph in (False, True):
        for cand in CANDIDATES:
            b = BatchScan(grids, p, dts, max_steps=steps, tune=cand)
            b.init(ids)
            b.run(0, steps, use_graph=use_graph, stream=torch.cuda.Stream())
            torch.cuda.synchronize()
            for i in range(len(ns)):
                assert torch.equal(b.states[i], ref[i]), (cand, use_graph, i)
            b.close()


def test_batch_graph_replays_in_segments(C):
    """Steps 0-1 then 2-3 (two graphs) equal four unsegmented steps."""
    from paper_2606_02053_gb300.batch import BatchScan

    grids, dts, ids, p = scan_setup(C, [16, 19], [0.5, 0.7])
    s = torch.cuda.Stream()
    a = BatchScan(grids, p, dts, max_steps=4)
    a.init(ids)
    a.run(0, 2, stream=s)
    a.run(2, 2, stream=s)
    b = BatchScan(grids, p, dts, max_steps=4)
    b.init(ids)
    b.run(0, 4, stream=s)
    torch.cuda.synchronize()
    for x, y in zip(a.states, b.states):
        assert torch.equal(x, y)


def test_batch_instance_matches_oracle(C, O):
    from paper_2606_02053_gb300.batch import BatchScan

    ns = [20, 17]
    grids, dts, ids, p = scan_setup(C, ns, [0.5, 0.3])
    steps = 3
    b = BatchScan(grids, p, dts, max_steps=steps, tune=(1, 32, 4, 2))
    b.init(ids)
    b.run(0, steps, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    op = O.params_array(fluid=1, w=1.0 / 3.0, H0=20.0)
    for i, n in enumerate(ns):
        h = 1.0 / n
        og = O.OGrid((n, n, n), h, x0=(-(n // 2) * h,) * 3)
        ref = O.init(og, op, O.id_array(1, mu=[0.5, 0.3][i], sigma=0.14, q=(1.0, 0.9, 1.1)))
        O.evolve(og, op, ref, 0.0, dts[i], steps)
        got = b.states[i].view(-1, n, n, n).cpu().numpy()
        den = np.maximum(np.abs(ref).reshape(28, -1).max(axis=1), 1e-300)
        err = (np.abs(got - ref).reshape(28, -1).max(axis=1) / den).max()
        assert err <= 1e-10, (i, err)


def test_autotune_picks_a_candidate_and_caches(C, tmp_path):
    from paper_2606_02053_gb300.batch import CANDIDATES, BatchScan, tuning

    grids, dts, ids, p = scan_setup(C, [16, 20, 18], [0.4, 0.5, 0.6])
    b = BatchScan(grids, p, dts, max_steps=1)
    b.init(ids)
    before = [s.clone() for s in b.states]
    cache = tmp_path / "tune.txt"
    cache.write_text("some other device|fluid=0|scalar=0|8x8x8\t0 32 4 3\t1.5\n")
    r = b.autotune(reps=2, cache_path=str(cache))
    assert tuple(r["best"]) in CANDIDATES and not r["cache_hit"]
    assert len(r["ms"]) == len(CANDIDATES) and all(v > 0 for v in r["ms"].values())
    assert min(r["ms"], key=r["ms"].get) == str(r["best"])
    for x, y in zip(before, b.states):  # timing passes leave the states untouched
        assert torch.equal(x, y)
    lines = cache.read_text().splitlines()
    assert len(lines) == 2 and lines[0].startswith("some other device")  # other keys are kept
    assert lines[1].split("\t")[0].endswith("|fluid=1|scalar=0|16x16x16,20x20x20,18x18x18")
    r2 = b.autotune(reps=2, cache_path=str(cache))
    assert r2["cache_hit"] and r2["best"] == r["best"] and r2["ms"] == {}
    assert len(cache.read_text().splitlines()) == 2
    # an explicit candidate list; an invalid candidate is refused before anything is timed
    r3 = b.autotune(candidates=[(1, 32, 4, 2), (0, 16, 8, 3)], reps=1)
    assert tuple(r3["best"]) in [(1, 32, 4, 2), (0, 16, 8, 3)] and len(r3["ms"]) == 2
    code, *_ = C.cosmos_batch_autotune(b.plan, [tuning(t) for t in [(0, 32, 4, 3), (0, 32, 8, 3)]], 1)
    assert code == C.COSMOS_EINVAL


def test_batch_rejects_bad_arguments(C):
    from paper_2606_02053_gb300.batch import BatchScan, tuning

    grids, dts, ids, p = scan_setup(C, [16], [0.5])
    b = BatchScan(grids, p, dts, max_steps=2)
    assert C.cosmos_batch_run(b.plan, 1, 2, 0) == C.COSMOS_EINVAL  # beyond max_steps
    assert C.cosmos_batch_run(b.plan, 0, 1, 1, None) == C.COSMOS_EINVAL  # graph needs a non-default stream
    assert C.cosmos_batch_set_tuning(b.plan, tuning((0, 32, 8, 3))) == C.COSMOS_EINVAL  # 256 threads
    assert C.cosmos_batch_set_tuning(b.plan, tuning((2, 32, 4, 3))) == C.COSMOS_EINVAL
