"""Restarted GMRES(m) (the paper's iterative method) on the GPU vs the oracle, on the symmetric and the row-lifted
nonsymmetric systems (needs a B300)."""
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
@pytest.mark.parametrize("restart", [30, 5])
def test_gmres_time_steps_match_oracle(lift, restart):
    """Four time steps with GMRES(m) (tol 1e-13, m = 30 and m = 5) on a jittered lognormal 12^3 mesh agree with the
    oracle's direct solves (relative error <= 1e-9 at every step); the short restart needs several cycles."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=54, sigma0="lognormal")
    Ts, Vs = O.Model(m).run(4)
    with rafem.Context(m, solver=2, lift=lift, gmres_restart=restart, tol=1e-13) as ctx:
        for k in range(4):
            s, st = ctx.solve_step()
            assert s == 0 and st.iters_V > 0 and st.relres_V <= 1e-13
            if restart == 5:
                assert st.refine_V >= 2
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), Ts[k]) <= 1e-9
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), Vs[k]) <= 1e-9


def test_gmres_solve_rhs_full_size_residual():
    """On the 48^3 workload, rafem_solve_rhs with GMRES(30) on the assembled potential system and a random
    right-hand side gives ||b - A x|| / ||b|| <= 1e-10, measured independently through rafem_spmv."""
    import torch
    rafem = R()
    m = mg.workload_48()
    with rafem.Context(m, solver=2) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        g = torch.Generator(device="cuda").manual_seed(8)
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


def test_gmres_limits_and_rejections():
    """Iteration cap gives NOT_CONVERGED; restart outside 1..64, mixed precision, ILU(0), CSR lanes or a batch give
    BAD_INPUT."""
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=55)
    with rafem.Context(m, solver=2, max_iter=3) as ctx:
        s, st = ctx.solve_step()
        assert s == rafem.RAFEM_NOT_CONVERGED and st.iters_V == 3
    for kw in (dict(solver=2, gmres_restart=65), dict(solver=2, precision=1), dict(solver=2, precond=1),
               dict(solver=2, lanes_per_row=8)):
        with pytest.raises(rafem.RafemError):
            rafem.Context(m, **kw)
    with pytest.raises(rafem.RafemError):
        rafem.Context.batch([m, m], solver=2)


@pytest.mark.parametrize("lift", [0, 1], ids=["symmetric", "row"])
def test_adaptive_gmres_time_steps_match_oracle(lift):
    """GMRES with the cycle length adapting between 4 and 30 (Sec. III-B's adaptive m) gives the oracle's fields
    (relative error <= 1e-9 at every step of four)."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=56, sigma0="lognormal")
    Ts, Vs = O.Model(m).run(4)
    with rafem.Context(m, solver=2, lift=lift, gmres_restart=30, gmres_min_restart=4, tol=1e-13) as ctx:
        for k in range(4):
            s, st = ctx.solve_step()
            assert s == 0 and st.relres_V <= 1e-13
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), Ts[k]) <= 1e-9
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), Vs[k]) <= 1e-9


def _solve_potential(m, **kw):
    import torch
    rafem = R()
    with rafem.Context(m, solver=2, lift=1, tol=1e-10, max_iter=20000, **kw) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        _, _, _, rhs = ctx.get_system(rafem.RAFEM_SYS_V)
        b = torch.tensor(rhs, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
        return s, st, x.cpu().numpy()


def test_adaptive_length_beats_a_slow_short_restart():
    """On the 24^3 potential system (row lift, from zero to 1e-10) the short restart GMRES(4) converges slowly;
    the adaptive length (4..30) reaches the tolerance in fewer Arnoldi steps, and its solution is the direct
    solve's."""
    rafem = R()
    m = mg.cube_mesh(24, jitter=0.1, seed=57, sigma0="lognormal")
    s4, st4, x4 = _solve_potential(m, gmres_restart=4)
    sa, sta, xa = _solve_potential(m, gmres_restart=30, gmres_min_restart=4)
    assert s4 == rafem.RAFEM_OK and sa == rafem.RAFEM_OK
    assert sta.iters_V < st4.iters_V, (sta.iters_V, st4.iters_V)
    A, b = O.Model(m, O.Params(lift="row")).system_V(np.full(m.n_nodes, 37.0))
    x_ref = O.solve(A, b)
    assert O.rel_err(xa, x_ref) <= 1e-6  # cond(A) x 1e-10
    assert O.rel_err(x4, x_ref) <= 1e-6


@pytest.mark.parametrize("min_restart", [0, 4])
def test_stagnation_ends_the_solve(min_restart):
    """No Dirichlet node and a right-hand side with a component along the constants (the null space): no residual
    below that component exists. GMRES stops after two full-length cycles that each keep more than 99.9% of the
    residual, long before the iteration cap, with NOT_CONVERGED."""
    import dataclasses
    import torch
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=58)
    m = dataclasses.replace(m, bc_V=np.zeros_like(m.bc_V), g_V=np.zeros_like(m.g_V))
    with rafem.Context(m, solver=2, lift=1, gmres_restart=20, gmres_min_restart=min_restart, tol=1e-10,
                       max_iter=20000) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        b = torch.tensor(1.0 + m.coords[:, 0] / 0.04, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
    assert s == rafem.RAFEM_NOT_CONVERGED
    assert st.iters_V < 2000 and st.refine_V < 100, st.as_dict()
