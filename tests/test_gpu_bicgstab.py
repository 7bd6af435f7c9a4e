"""BiCGSTAB (the solver option for nonsymmetric systems) on the GPU vs the oracle, on the symmetric systems and on
the nonsymmetric row-lifted systems (needs a B300)."""
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


@pytest.mark.parametrize("lift", [0, 1], ids=["symmetric", "row"])
@pytest.mark.parametrize("assembly", [0, 1], ids=["gather", "colour"])
def test_bicgstab_time_steps_match_oracle(lift, assembly):
    """Four time steps with BiCGSTAB (tol 1e-12) on a jittered lognormal 12^3 mesh agree with the oracle's direct
    solves (relative error <= 1e-9 for V and T at every step), with the symmetric and the row-only lift."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=51, sigma0="lognormal")
    Ts, Vs = O.Model(m).run(4)
    with rafem.Context(m, solver=1, lift=lift, assembly=assembly, tol=1e-12) as ctx:
        for k in range(4):
            s, st = ctx.solve_step()
            assert s == 0 and st.iters_V > 0
            assert st.relres_V <= 1e-12 and st.relres_T <= 1e-12
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), Ts[k]) <= 1e-9
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), Vs[k]) <= 1e-9


@pytest.mark.parametrize("assembly", [0, 1], ids=["gather", "colour"])
def test_row_lifted_systems_match_oracle(assembly):
    """The row-lifted (nonsymmetric) potential and thermal systems, slot by slot against the oracle's."""
    rafem = R()
    m = mg.cube_mesh(9, jitter=0.1, seed=52, sigma0="lognormal")
    rng = np.random.default_rng(4)
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 20.0 * rng.random(m.n_nodes))
    V = np.where(m.bc_V.astype(bool), m.g_V, 20.0 * rng.random(m.n_nodes))
    model = O.Model(m, O.Params(lift="row"))
    with rafem.Context(m, solver=1, lift=1, assembly=assembly) as ctx:
        ctx.set_state(T=T, V=V)
        ctx.assemble(rafem.RAFEM_SYS_V)
        ctx.assemble(rafem.RAFEM_SYS_T)
        sysV = ctx.get_system(rafem.RAFEM_SYS_V)
        sysT = ctx.get_system(rafem.RAFEM_SYS_T)
    AV, bV = model.system_V(T)
    AT, bT = model.system_T(T, O.joule(model.sigma(T), V, model.tets, model.grad))
    for (rp, col, vals, rhs), (A, b) in ((sysV, (AV, bV)), (sysT, (AT, bT))):
        np.testing.assert_array_equal(rp, A.indptr)
        np.testing.assert_array_equal(col, A.indices)
        np.testing.assert_allclose(vals, A.data, rtol=1e-13, atol=1e-14 * np.abs(A.data).max())
        np.testing.assert_allclose(rhs, b, rtol=1e-13, atol=1e-14 * np.abs(b).max())


def test_bicgstab_solve_rhs_full_size_residual():
    """On the 48^3 workload, rafem_solve_rhs with BiCGSTAB on the assembled potential system and a random
    right-hand side returns x with ||b - A x|| / ||b|| <= 1e-10 measured independently through rafem_spmv."""
    import torch
    rafem = R()
    m = mg.workload_48()
    with rafem.Context(m, solver=1) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        g = torch.Generator(device="cuda").manual_seed(7)
        b = torch.randn(m.n_nodes, dtype=torch.float64, device="cuda", generator=g)
        b[torch.tensor(m.bc_V.astype(bool), device="cuda")] = 0.0
        x = torch.zeros_like(b)
        y = torch.empty_like(b)
        torch.cuda.synchronize()
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
        assert s == 0
        ctx.spmv(rafem.RAFEM_SYS_V, x, y)
        rel = float(torch.linalg.norm(b - y) / torch.linalg.norm(b))
    assert rel <= 1.0001e-10 and abs(rel - st.relres_V) <= 1e-3 * rel + 1e-15


def test_bicgstab_limits_and_rejections():
    """Iteration cap gives NOT_CONVERGED; the row lift needs BiCGSTAB; BiCGSTAB is FP64/Jacobi/SELL-32/single
    instance; the adjoint refuses the row lift."""
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=53)
    with rafem.Context(m, solver=1, max_iter=2) as ctx:
        s, st = ctx.solve_step()
        assert s == rafem.RAFEM_NOT_CONVERGED and st.iters_V == 2
    for kw in (dict(lift=1), dict(solver=1, precision=1), dict(solver=1, lanes_per_row=8), dict(solver=1, precond=1),
               dict(lift=2, solver=1)):
        with pytest.raises(rafem.RafemError):
            rafem.Context(m, **kw)
    with pytest.raises(rafem.RafemError):
        rafem.Context.batch([m, m], solver=1)
    with rafem.Context(m, solver=1, lift=1) as ctx:
        with pytest.raises(rafem.RafemError):
            ctx.tape_begin(2)
