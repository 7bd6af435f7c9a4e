"""Failure paths of the persistent solvers on the GPU, exercised without a fault (needs a B300).

- Bounded waits: rafem_set_wait_limit(limit, missing_arrivals = 1) starts the solver's grid-barrier counter one
  arrival short, so its first barrier can never complete. Every block's wait must run out after the limit, the
  solve must return RAFEM_ERR_TIMEOUT in bounded time, and the context must give correct steps again once the
  limit is restored and the state reset (the same fields as a fresh context, bit for bit). Every solver kernel
  family is covered: Chronopoulos-Gear CG (FP64 and mixed, with the bulk-copy ring), pipelined CG, BiCGSTAB,
  GMRES(m) and ILU(0)-PCG.
- A singular potential system (no Dirichlet node) with an inconsistent right-hand side: CG cannot converge and
  must stop at max_iter with RAFEM_NOT_CONVERGED.
- A NaN reaching a running solve (through a device right-hand side, which is not checked on the host): the solver
  must stop with RAFEM_ERR_NONFINITE.
The main loop's own failure handling (a step whose corrector does not converge is halved, Sec. IV) is covered in
test_gpu_corrector.py.
"""
import dataclasses
import time

import numpy as np
import pytest

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


def R():
    from paper_2409_13036_b300 import rafem
    return rafem


SOLVERS = {
    "cg64": dict(),
    "cg_mixed": dict(precision=1),
    "pipecg": dict(solver=3),
    "bicgstab": dict(solver=1, lift=1),
    "gmres": dict(solver=2, lift=1, gmres_restart=10),
    "ilu": dict(precond=1),
}

LIMIT_NS = 50_000_000  # 50 ms: far above any copy or barrier latency, short enough for a quick test


@pytest.mark.parametrize("name", list(SOLVERS))
def test_wait_runs_out_and_context_recovers(name):
    rafem = R()
    kw = SOLVERS[name]
    m = mg.cube_mesh(16, jitter=0.1, seed=21, sigma0="lognormal")
    with rafem.Context(m, tol=1e-11, **kw) as ctx, rafem.Context(m, tol=1e-11, **kw) as fresh:
        s, _ = ctx.run(1)
        assert s == rafem.RAFEM_OK
        ctx.set_wait_limit(LIMIT_NS, 1)
        t0 = time.monotonic()
        with pytest.raises(rafem.RafemError) as e:
            ctx.solve_step()
        elapsed = time.monotonic() - t0
        assert e.value.status == rafem.RAFEM_ERR_TIMEOUT, str(e.value)
        # every block gives up after the limit: the step ends long before the default 5 s limit would
        assert elapsed < 2.0, elapsed
        # the context is still usable: default limit, defined state, the same steps as a fresh context
        ctx.set_wait_limit(0, 0)
        ctx.reset()
        s1, _ = ctx.run(3)
        s2, _ = fresh.run(3)
        assert s1 == rafem.RAFEM_OK and s2 == rafem.RAFEM_OK
        for which in (rafem.RAFEM_SYS_V, rafem.RAFEM_SYS_T):
            np.testing.assert_array_equal(ctx.get_field(which), fresh.get_field(which))


def test_wait_limit_arguments():
    rafem = R()
    m = mg.cube_mesh(4)
    with rafem.Context(m) as ctx:
        for bad in (-1, 5000):
            with pytest.raises(rafem.RafemError) as e:
                ctx.set_wait_limit(0, bad)
            assert e.value.status == rafem.RAFEM_ERR_BAD_INPUT


def test_singular_potential_system_not_converged():
    """No Dirichlet node in the potential system: A_V has the constants as null space. A right-hand side with a
    component along the constants has no solution, and the residual cannot drop below that component: CG stops at
    max_iter with RAFEM_NOT_CONVERGED. A consistent right-hand side (b = A y) on the same matrix converges."""
    import torch
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=22)
    m = dataclasses.replace(m, bc_V=np.zeros_like(m.bc_V), g_V=np.zeros_like(m.g_V))
    N = m.n_nodes
    max_iter = 40
    bh = 1.0 + m.coords[:, 0] / 0.04  # mean 1 plus a ramp
    floor = abs(bh.mean()) * np.sqrt(N) / np.linalg.norm(bh)  # ||P b|| / ||b||, P onto the constants
    with rafem.Context(m, max_iter=max_iter) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        b = torch.tensor(bh, dtype=torch.float64, device="cuda")
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
        assert s == rafem.RAFEM_NOT_CONVERGED, (rafem.status_string(s), st.as_dict())
        assert st.iters_V == max_iter
        assert st.relres_V >= floor * (1 - 1e-9)
    with rafem.Context(m, max_iter=2000, tol=1e-10) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        y = torch.tensor(np.sin(40.0 * m.coords[:, 1]), dtype=torch.float64, device="cuda")
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        ctx.spmv(rafem.RAFEM_SYS_V, y, b)
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
        assert s == rafem.RAFEM_OK and st.relres_V <= 1e-10, st.as_dict()


@pytest.mark.parametrize("name", ["cg64", "cg_mixed", "bicgstab", "gmres", "ilu"])
def test_nan_in_running_solve(name):
    """A NaN in a device right-hand side (device inputs are not checked on the host) reaches the solver's first
    residual: the solve stops with RAFEM_ERR_NONFINITE instead of iterating on NaNs."""
    import torch
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=23)
    with rafem.Context(m, max_iter=500, **SOLVERS[name]) as ctx:
        ctx.assemble(rafem.RAFEM_SYS_V)
        b = torch.ones(m.n_nodes, dtype=torch.float64, device="cuda")
        b[m.n_nodes // 2] = float("nan")
        x = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        with pytest.raises(rafem.RafemError) as e:
            ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
        assert e.value.status == rafem.RAFEM_ERR_NONFINITE, str(e.value)
