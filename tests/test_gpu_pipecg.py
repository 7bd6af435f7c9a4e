"""Pipelined Jacobi-PCG (one grid barrier per iteration) against the oracle's direct solves, against CG, in the
batching form, and with residual replacement (needs a B300)."""
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
    torch.cuda.init()
    yield


def R():
    from paper_2409_13036_b300 import rafem
    return rafem


@pytest.mark.parametrize("n,lanes", [(12, 0), (15, 8)])
def test_pipecg_steps_match_oracle(n, lanes):
    """Backward-Euler steps solved by the pipelined solver (SELL-32 and CSR layouts) vs the oracle's LU path:
    relative error <= 1e-9 per field per step at tolerance 1e-12."""
    rafem = R()
    m = mg.cube_mesh(n, jitter=0.1, seed=40 + n, sigma0="lognormal")
    steps = 4
    Ts, Vs = [], []
    with rafem.Context(m, tol=1e-12, dt=5.0, solver=rafem.RAFEM_SOLVER_PIPECG, lanes_per_row=lanes) as ctx:
        for _ in range(steps):
            s, st = ctx.solve_step()
            assert s == rafem.RAFEM_OK, st.as_dict()
            assert st.relres_V <= 1e-12 and st.relres_T <= 1e-12
            Ts.append(ctx.get_field(rafem.RAFEM_SYS_T))
            Vs.append(ctx.get_field(rafem.RAFEM_SYS_V))
    T_ref, V_ref = O.Model(m, O.Params(dt=5.0)).run(steps)
    for k in range(steps):
        assert O.rel_err(Vs[k], V_ref[k]) <= 1e-9
        assert O.rel_err(Ts[k], T_ref[k]) <= 1e-9


def test_pipecg_iterates_like_cg():
    """Same Krylov iterates in exact arithmetic: the iteration counts per solve match CG's within a few and the
    fields agree within the solver tolerance."""
    rafem = R()
    m = mg.cube_mesh(20, jitter=0.1, seed=7, sigma0="lognormal")
    res = {}
    for solver in (rafem.RAFEM_SOLVER_PCG, rafem.RAFEM_SOLVER_PIPECG):
        iters = []
        with rafem.Context(m, tol=1e-10, dt=5.0, solver=solver, predictor=0) as ctx:
            for _ in range(3):
                s, st = ctx.solve_step()
                assert s == rafem.RAFEM_OK
                iters.append((st.iters_V, st.iters_T))
            res[solver] = (iters, ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V))
    (ic, Tc, Vc), (ip, Tp, Vp) = res[rafem.RAFEM_SOLVER_PCG], res[rafem.RAFEM_SOLVER_PIPECG]
    for (a, b), (c, d) in zip(ic, ip):
        assert abs(a - c) <= max(3, a // 20) and abs(b - d) <= 2, (ic, ip)
    assert O.rel_err(Tp, Tc) <= 1e-9 and O.rel_err(Vp, Vc) <= 1e-7


def test_pipecg_batch_matches_single_contexts():
    rafem = R()
    draws = [(6, 12.0, 12.0, 0.27, 11), (9, 35.0, 25.0, 0.41, 12), (11, 20.0, 18.0, 0.33, 13)]
    meshes = [mg.batch_mesh(d) for d in draws]
    with rafem.Context.batch(meshes, tol=1e-12, dt=5.0, solver=rafem.RAFEM_SOLVER_PIPECG) as b:
        s, st = b.run(3)
        assert s == rafem.RAFEM_OK
        T, V, off = b.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_V), b.offsets
        per = b.batch_stats()
    assert all(p["status"] == 0 for p in per) and len({p["iters_V"] for p in per}) > 1
    for i, m in enumerate(meshes):
        with rafem.Context(m, tol=1e-12, dt=5.0) as c:
            c.run(3)
            assert O.rel_err(T[off[i]:off[i] + m.n_nodes], c.get_field(rafem.RAFEM_SYS_T)) <= 1e-9
            assert O.rel_err(V[off[i]:off[i] + m.n_nodes], c.get_field(rafem.RAFEM_SYS_V)) <= 1e-9


def test_pipecg_tight_tolerance_reaches_true_residual():
    """At 1e-13 the pipelined recurrences drift from the true residual; residual replacement restarts bring the
    true residual under the target (or the solve says it did not converge)."""
    rafem = R()
    m = mg.cube_mesh(24, jitter=0.1, seed=8, sigma0="lognormal")
    with rafem.Context(m, tol=1e-13, dt=5.0, solver=rafem.RAFEM_SOLVER_PIPECG, predictor=0) as ctx:
        s, st = ctx.solve_step()
        assert s in (rafem.RAFEM_OK, rafem.RAFEM_NOT_CONVERGED)
        if s == rafem.RAFEM_OK:
            assert st.relres_V <= 1e-13 and st.relres_T <= 1e-13


def test_pipecg_rejected_configurations():
    rafem = R()
    m = mg.cube_mesh(5)
    for kw in ({"precision": rafem.RAFEM_PRECISION_MIXED}, {"precond": rafem.RAFEM_PRECOND_ILU0},
               {"lift": rafem.RAFEM_LIFT_ROW}, {"coupling": rafem.RAFEM_COUPLING_MONOLITHIC}):
        with pytest.raises(rafem.RafemError):
            rafem.Context(m, solver=rafem.RAFEM_SOLVER_PIPECG, **kw)
