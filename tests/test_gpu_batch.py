"""Batching form: many independent instances in one context and one persistent launch per system, compared
with one context per instance and with the oracle (needs a B300)."""
import numpy as np
import pytest

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2409_13036_b300 import build
    build.build()
    yield


def _instances():
    """Five uneven instances (sizes, electrode voltage and depth, sigma0 differ; none a multiple of 32 nodes)."""
    draws = [(6, 12.0, 12.0, 0.27, 11), (9, 35.0, 25.0, 0.41, 12), (11, 20.0, 18.0, 0.33, 13), (13, 15.0, 29.0, 0.30, 14),
             (8, 40.0, 10.0, 0.45, 15)]
    return [mg.batch_mesh(d) for d in draws]


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-9), (1, 1e-11, 1e-8)])
def test_batch_matches_single_instance_contexts(precision, tol, bound):
    """Every instance of the batch (rafem_batch_run) against a single-instance context of its own and against the
    oracle's direct solves."""
    from paper_2409_13036_b300 import rafem
    meshes = _instances()
    steps = 3
    with rafem.Context.batch(meshes, precision=precision, tol=tol, dt=5.0) as b:
        s, per = b.batch_run(steps)
        assert s == rafem.RAFEM_OK, per
        assert per == b.batch_stats()
        T = b.get_field(rafem.RAFEM_SYS_T)
        V = b.get_field(rafem.RAFEM_SYS_V)
        off = b.offsets
    assert len(per) == len(meshes) and all(p["status"] == 0 and p["step"] == steps for p in per)
    assert len({p["iters_V"] for p in per}) > 1  # instances converge on their own schedules
    for i, m in enumerate(meshes):
        Ti, Vi = T[off[i]:off[i] + m.n_nodes], V[off[i]:off[i] + m.n_nodes]
        with rafem.Context(m, precision=0, tol=1e-12, dt=5.0) as c:
            c.run(steps)
            assert O.rel_err(Ti, c.get_field(rafem.RAFEM_SYS_T)) <= bound
            assert O.rel_err(Vi, c.get_field(rafem.RAFEM_SYS_V)) <= bound
        # the padding nodes between instances keep their boundary values
        pad = slice(off[i] + m.n_nodes, off[i + 1])
        assert np.all(V[pad] == 0.0)
        # each instance against the oracle's direct solves
        T_ref, V_ref = O.Model(m, O.Params(dt=5.0)).run(steps)
        assert O.rel_err(Ti, T_ref[-1]) <= bound, i
        assert O.rel_err(Vi, V_ref[-1]) <= bound, i


def test_batch_limits():
    from paper_2409_13036_b300 import rafem
    m = mg.cube_mesh(2)
    with pytest.raises(rafem.RafemError) as e:
        rafem.Context.batch([m] * 97)
    assert e.value.status == rafem.RAFEM_ERR_BAD_INPUT
    with rafem.Context.batch([m]) as b:
        s, st = b.run(1)
        assert s == rafem.RAFEM_OK and b.n_inst == 1


def test_autotuner_caches_its_choice_and_keeps_the_fields(tmp_path, monkeypatch):
    """The schedule autotuner times the candidate tile sizes on a live batch, keeps the fastest and stores it in
    its cache file; a second context of the same shape takes the cached choice without timing. The tile size only
    changes the work split: a batch run with the tuned schedule gives the same fields as the default schedule up to
    the solver tolerance (both solved to 1e-12; cond(A) ~1e2 on these instances, bound 1e-9)."""
    from paper_2409_13036_b300 import rafem
    from paper_2409_13036_b300.autotune import autotune_schedule, cache_path
    monkeypatch.setenv("RAFEM_CACHE_DIR", str(tmp_path))
    meshes = _instances()
    with rafem.Context.batch(meshes, tol=1e-12, dt=5.0) as b:
        rep = autotune_schedule(b, candidates=(0, 1024, 4096), steps=1)
        assert not rep["cached"] and len(rep["trials"]) == 3
        assert rep["rows_per_tile"] == min(rep["trials"], key=lambda t: t["ms_per_iteration"])["rows_per_tile"]
        assert b.get_schedule()["rows_per_tile"] == rep["rows_per_tile"]
    import json
    with open(cache_path()) as f:
        assert len(json.load(f)) == 1
    with rafem.Context.batch(meshes, tol=1e-12, dt=5.0) as tuned, rafem.Context.batch(meshes, tol=1e-12, dt=5.0) as ref:
        rep2 = autotune_schedule(tuned, candidates=(0, 1024, 4096), steps=1)
        assert rep2["cached"] and rep2["rows_per_tile"] == rep["rows_per_tile"]
        assert tuned.get_schedule()["rows_per_tile"] == rep["rows_per_tile"]
        s1, _ = tuned.run(3)
        s2, _ = ref.run(3)
        assert s1 == 0 and s2 == 0
        for which in (rafem.RAFEM_SYS_T, rafem.RAFEM_SYS_V):
            a, c = tuned.get_field(which), ref.get_field(which)
            assert np.linalg.norm(a - c) <= 1e-9 * np.linalg.norm(c)
