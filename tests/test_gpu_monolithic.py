"""Monolithic coupled step (the paper's 2N x 2N system, Newton's method) on the GPU vs the oracle (needs a B300)."""
import numpy as np
import pytest
import scipy.sparse as sp

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


@pytest.mark.parametrize("assembly", [0, 1], ids=["gather", "colour"])
def test_coupled_jacobian_and_residual_match_oracle(assembly):
    """The 2 x 2 Jacobian blocks on the node pattern and the interleaved residual of the monolithic step at a
    non-trivial (V, T), entry by entry against the oracle's coupled_jacobian / coupled_residual (T_old = T)."""
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=81, sigma0="lognormal", V_electrode=40.0)
    rng = np.random.default_rng(1)
    V = np.where(m.bc_V.astype(bool), m.g_V, 20.0 * rng.random(m.n_nodes))
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 20.0 * rng.random(m.n_nodes))
    model = O.Model(m, O.Params(dt=30.0))
    with rafem.Context(m, dt=30.0, coupling=1, assembly=assembly) as ctx:
        ctx.set_state(T=T, V=V)
        blocks, res = ctx.get_coupled_system()
        rp, col, _, _ = ctx.get_system(rafem.RAFEM_SYS_V)
    J = O.coupled_jacobian(model, V, T).tocsr()
    Rref = O.coupled_residual(model, V, T, T)
    rows = np.repeat(np.arange(m.n_nodes), np.diff(rp))
    for a in range(2):
        for b in range(2):
            ref = np.asarray(J[2 * rows + a, 2 * col + b]).ravel()
            np.testing.assert_allclose(blocks[:, a, b], ref, rtol=1e-12, atol=1e-13 * np.abs(J.data).max())
    np.testing.assert_allclose(res.ravel(), Rref, rtol=1e-11, atol=1e-12 * np.abs(Rref).max())


@pytest.mark.parametrize("assembly", [0, 1], ids=["gather", "colour"])
def test_coupled_system_after_k_and_dt_change(assembly):
    """The coupled Jacobian and residual after rafem_set_params (new thermal conductivities) and rafem_set_dt: the
    constant thermal block (k G + (rho_c/dt + perf) M) follows both changes, entry by entry against the oracle."""
    import dataclasses
    rafem = R()
    m = mg.cube_mesh(7, jitter=0.1, seed=85, sigma0="lognormal", V_electrode=30.0)
    rng = np.random.default_rng(2)
    V = np.where(m.bc_V.astype(bool), m.g_V, 15.0 * rng.random(m.n_nodes))
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 10.0 * rng.random(m.n_nodes))
    k2 = m.k * (0.5 + rng.random(m.n_tets))
    m2 = dataclasses.replace(m, k=k2)
    model = O.Model(m2, O.Params(dt=12.0))
    with rafem.Context(m, dt=30.0, coupling=1, assembly=assembly) as ctx:
        ctx.set_params(k=k2)
        ctx.set_dt(12.0)
        ctx.set_state(T=T, V=V)
        blocks, res = ctx.get_coupled_system()
        rp, col, _, _ = ctx.get_system(rafem.RAFEM_SYS_V)
    J = O.coupled_jacobian(model, V, T).tocsr()
    Rref = O.coupled_residual(model, V, T, T)
    rows = np.repeat(np.arange(m.n_nodes), np.diff(rp))
    for a in range(2):
        for b in range(2):
            ref = np.asarray(J[2 * rows + a, 2 * col + b]).ravel()
            np.testing.assert_allclose(blocks[:, a, b], ref, rtol=1e-12, atol=1e-13 * np.abs(J.data).max())
    np.testing.assert_allclose(res.ravel(), Rref, rtol=1e-11, atol=1e-12 * np.abs(Rref).max())


def test_coupled_system_full_size_sampled_rows():
    """At the 127^3 bench workload (2,097,152 nodes, launch configuration of the bench's monolithic leg), the
    coupled Jacobian and residual of the row-owner assembly on sampled rows (2,000 random rows, 200 Dirichlet rows
    of each field and the last row) against the oracle applied to the elements around them."""
    from tests.sampled_rows import coupled_rows
    rafem = R()
    m = mg.workload_127()
    rng = np.random.default_rng(3)
    V = np.where(m.bc_V.astype(bool), m.g_V, 30.0 * rng.random(m.n_nodes))
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 15.0 * rng.random(m.n_nodes))
    with rafem.Context(m, coupling=1, n_corrector=20, corrector_tol=1e-6) as ctx:
        ctx.set_state(T=T, V=V)
        blocks, res = ctx.get_coupled_system()
        rp, col, _, _ = ctx.get_system(rafem.RAFEM_SYS_V)
    sample = np.concatenate([rng.choice(m.n_nodes, 2000, replace=False),
                             rng.choice(np.flatnonzero(m.bc_V), 200, replace=False),
                             rng.choice(np.flatnonzero(m.bc_T), 200, replace=False), [m.n_nodes - 1]])
    rows, ref, ref_res = coupled_rows(m, sample, V, T)
    scale = max(abs(v) for e in ref.values() for v in e.values())
    rscale = max(max(abs(a), abs(b)) for a, b in ref_res.values())
    for i in rows:
        got = {}
        for q in range(rp[i], rp[i + 1]):
            for a in range(2):
                for b in range(2):
                    got[(a, int(col[q]), b)] = blocks[q, a, b]
        want = ref[int(i)]
        for key in set(got) | set(want):
            g, w = got.get(key, 0.0), want.get(key, 0.0)
            assert abs(g - w) <= 1e-12 * abs(w) + 1e-13 * scale, (int(i), key, g, w)
        for a in range(2):
            assert abs(res[i, a] - ref_res[int(i)][a]) <= 1e-11 * abs(ref_res[int(i)][a]) + 1e-12 * rscale


@pytest.mark.parametrize("solver", [0, 1], ids=["fgmres", "bicgstab"])
def test_monolithic_steps_match_oracle_fixed_point(solver):
    """Two monolithic steps (dt = 30 s, 40 V, Newton to max |dT| < 1e-9) agree with the oracle's Newton step and
    with the corrector's fixed point (1e-9), in a few Newton iterations, through the device-side loop; with either
    linear solver (flexible GMRES with the split-system preconditioner: at most 8 outer iterations per Newton
    iteration, reported as refine_V; block-Jacobi BiCGSTAB)."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=82, sigma0="lognormal", V_electrode=40.0)
    model = O.Model(m, O.Params(dt=30.0, n_corrector=50, corrector_tol=1e-11))
    T = np.full(m.n_nodes, 37.0)
    with rafem.Context(m, dt=30.0, coupling=1, n_corrector=20, corrector_tol=1e-9, tol=1e-13,
                       coupled_solver=solver) as ctx:
        for k in range(2):
            Tn, Vn, it, _ = O.step_newton(model, T, tol=1e-11)
            Tp, Vp, _ = model.step(T)
            s, st = ctx.solve_step()
            assert s == 0 and 2 <= st.correctors <= 8
            if solver == 0:
                assert 1 <= st.refine_V <= 8 * st.correctors and st.iters_V > 0 and st.iters_T > 0
            Tg, Vg = ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V)
            for ref_T, ref_V in ((Tn, Vn), (Tp, Vp)):
                assert O.rel_err(Tg, ref_T) <= 1e-9
                assert O.rel_err(Vg, ref_V) <= 1e-9
            T = Tn
        assert ctx.graph_info()["corrector_graph"] == 1


def test_monolithic_rejections():
    """Monolithic coupling needs FP64, the SELL-32 layout and a single instance; it has no adjoint."""
    rafem = R()
    m = mg.cube_mesh(6, jitter=0.1, seed=83)
    for kw in (dict(coupling=1, precision=1), dict(coupling=1, lanes_per_row=8), dict(coupling=2),
               dict(coupling=1, coupled_solver=2)):
        with pytest.raises(rafem.RafemError):
            rafem.Context(m, **kw)
    with pytest.raises(rafem.RafemError):
        rafem.Context.batch([m, m], coupling=1)
    with rafem.Context(m, coupling=1) as ctx:
        with pytest.raises(rafem.RafemError):
            ctx.tape_begin(2)


def test_monolithic_fresh_process():
    """A monolithic context with the flexible-GMRES solver in a process where no other context ever ran: its inner
    mixed-precision solves must find their kernel prepared by the context itself (not by an earlier mixed context
    of the same process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2409_13036_b300 import meshgen as mg, rafem\n"
            "m = mg.cube_mesh(12, jitter=0.1, seed=84, V_electrode=40.0)\n"
            "with rafem.Context(m, dt=30.0, coupling=1, n_corrector=20, corrector_tol=1e-9) as ctx:\n"
            "    s, st = ctx.run(2)\n"
            "    print(s, st.correctors, st.refine_V)\n" % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    s, corr, outer = (int(x) for x in r.stdout.split()[-3:])
    assert s == 0 and corr >= 1 and outer >= 1
