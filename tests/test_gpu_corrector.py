"""Corrector passes on the device (CUDA graph with a conditional loop) and dynamic step size, vs the oracle
(needs a B300)."""
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


def _strong(n=6, V=40.0):
    return mg.cube_mesh(n, jitter=0.1, seed=71, sigma0="lognormal", V_electrode=V)


def test_corrector_steps_match_oracle():
    """Two steps of dt = 30 s with up to 50 corrector passes (tol 1e-8 degC): the GPU's device-side loop takes the
    same number of passes as the oracle and its fields agree to 1e-9."""
    rafem = R()
    m = _strong(8)
    model = O.Model(m, O.Params(dt=30.0, n_corrector=50, corrector_tol=1e-8))
    T = np.full(m.n_nodes, 37.0)
    with rafem.Context(m, dt=30.0, n_corrector=50, corrector_tol=1e-8, tol=1e-13) as ctx:
        for k in range(2):
            T, V, passes, ok = model.step_detail(T)
            s, st = ctx.solve_step()
            assert s == 0 and ok and st.correctors == passes and st.step == k + 1
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), T) <= 1e-9
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), V) <= 1e-9


def test_corrector_graph_equals_host_loop_and_reports_nonconvergence():
    """The conditional graph (rafem_run) and the host loop (tracing on) give bitwise the same fields; with too few
    passes the step reports NOT_CONVERGED and uses all of them."""
    rafem = R()
    m = _strong(8)
    kw = dict(dt=30.0, n_corrector=6, corrector_tol=1e-8, tol=1e-12)
    with rafem.Context(m, **kw) as a, rafem.Context(m, **kw) as b:
        sa, st = a.run(2)
        assert sa == rafem.RAFEM_NOT_CONVERGED and st.correctors == 6 and st.step == 2
        assert a.graph_info()["corrector_graph"] == 1
        b.set_tracing(True)
        sb, _ = b.run(2)
        assert sb == rafem.RAFEM_NOT_CONVERGED
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_T))
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_V), b.get_field(rafem.RAFEM_SYS_V))


def test_advance_matches_oracle_rejections_and_fields():
    """Dynamic step size over 100 s from dt = 60 s with at most 8 passes: the GPU rejects and halves exactly where
    the oracle does (2 rejections, 7 accepted steps, final dt 15 s) and ends at the same fields (1e-9)."""
    rafem = R()
    m = _strong(6)
    model = O.Model(m, O.Params(dt=60.0, n_corrector=8, corrector_tol=1e-6))
    T, V, log = O.advance(model, 100.0, dt_min=1.0)
    acc = [e for e in log if e[3]]
    with rafem.Context(m, dt=60.0, n_corrector=8, corrector_tol=1e-6, tol=1e-13) as ctx:
        s, st = ctx.advance(100.0, 1.0)
        assert s == 0
        assert st["accepted"] == len(acc) and st["rejected"] == len(log) - len(acc)
        assert st["passes"] == sum(e[1] for e in acc)
        assert abs(st["time"] - 100.0) < 1e-9 and st["dt"] == 15.0
        assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), T) <= 1e-9
        assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), V) <= 1e-9


def test_set_dt_equals_fresh_context_and_lagged_advance():
    """rafem_set_dt then stepping equals a context created with that dt (bitwise); lagged steps (one pass) are
    always accepted, the last one shortened to end at the requested time."""
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=72, sigma0="lognormal")
    with rafem.Context(m, dt=1.0) as a, rafem.Context(m, dt=2.5) as b:
        a.set_dt(2.5)
        a.run(3)
        b.run(3)
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_T))
    model = O.Model(m, O.Params(dt=2.0))
    T, V, log = O.advance(model, 7.0, dt_min=0.1)
    assert [e[0] for e in log] == [2.0, 2.0, 2.0, 1.0]
    with rafem.Context(m, dt=2.0, tol=1e-13) as ctx:
        s, st = ctx.advance(7.0, 0.1)
        assert s == 0 and st["accepted"] == 4 and st["rejected"] == 0 and st["dt"] == 2.0
        assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), T) <= 1e-9
