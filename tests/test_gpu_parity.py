"""CUDA path vs the FP64 CPU oracle, element by element, through the C-ABI (needs a B300)."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg
from tests.sampled_rows import lifted_rows, rows_adjacent_to

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


def _csr(rp, col, vals, n):
    return sp.csr_matrix((vals, col, rp), shape=(n, n))


def _nonuniform_T(mesh, seed=0):
    rng = np.random.default_rng(seed)
    T = 37.0 + 25.0 * rng.random(mesh.n_nodes)
    return np.where(mesh.bc_T.astype(bool), mesh.g_T, T)


@pytest.mark.parametrize("assembly", [0, 1])
def test_assembled_potential_system_matches_oracle(assembly):
    """A_V(sigma(T)) and its lifted rhs, slot by slot, on a jittered lognormal mesh with a non-uniform T, for the
    row-owner gather (0) and the colour-partitioned scatter (1)."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=21, sigma0="lognormal")
    T = _nonuniform_T(m)
    with rafem.Context(m, assembly=assembly) as ctx:
        ctx.set_state(T=T)
        ctx.assemble(rafem.RAFEM_SYS_V)
        rp, col, vals, rhs = ctx.get_system(rafem.RAFEM_SYS_V)
    A, b = O.Model(m).system_V(T)
    np.testing.assert_array_equal(rp, A.indptr)
    np.testing.assert_array_equal(col, A.indices)
    scale = np.abs(A.data).max()
    np.testing.assert_allclose(vals, A.data, rtol=1e-13, atol=1e-14 * scale)
    np.testing.assert_allclose(rhs, b, rtol=1e-13, atol=1e-14 * np.abs(b).max())


@pytest.mark.parametrize("assembly", [0, 1])
def test_assembled_thermal_system_matches_oracle(assembly):
    """Constant thermal matrix and the rhs (Joule from V, mass term from T), slot by slot, both assemblies."""
    rafem = R()
    m = mg.cube_mesh(9, jitter=0.1, seed=22, sigma0="lognormal")
    T = _nonuniform_T(m, 1)
    rng = np.random.default_rng(2)
    V = np.where(m.bc_V.astype(bool), m.g_V, 20.0 * rng.random(m.n_nodes))
    model = O.Model(m)
    with rafem.Context(m, assembly=assembly) as ctx:
        ctx.set_state(T=T, V=V)
        ctx.assemble(rafem.RAFEM_SYS_T)
        rp, col, vals, rhs = ctx.get_system(rafem.RAFEM_SYS_T)
    Q = O.joule(model.sigma(T), V, model.tets, model.grad)
    A, b = model.system_T(T, Q)
    np.testing.assert_array_equal(rp, A.indptr)
    np.testing.assert_array_equal(col, A.indices)
    np.testing.assert_allclose(vals, A.data, rtol=1e-13, atol=1e-14 * np.abs(A.data).max())
    np.testing.assert_allclose(rhs, b, rtol=1e-13, atol=1e-14 * np.abs(b).max())


def test_potential_solve_matches_direct_solve():
    """One PCG solve to a 1e-13 relative residual agrees with the oracle's LU solution to 1e-10."""
    rafem = R()
    m = mg.cube_mesh(14, jitter=0.1, seed=23, sigma0="lognormal")
    T = _nonuniform_T(m, 3)
    with rafem.Context(m, tol=1e-13) as ctx:
        ctx.set_state(T=T)
        ctx.assemble(rafem.RAFEM_SYS_V)
        s, st = ctx.solve(rafem.RAFEM_SYS_V)
        V = ctx.get_field(rafem.RAFEM_SYS_V)
    assert s == rafem.RAFEM_OK and st.relres_V <= 1e-13 and st.iters_V > 10
    A, b = O.Model(m).system_V(T)
    V_ref = O.solve(A, b)
    assert O.rel_err(V, V_ref) <= 1e-10


@pytest.mark.parametrize("n,steps,assembly", [(12, 6, 0), (20, 4, 0), (12, 3, 1)])
def test_time_steps_match_oracle(n, steps, assembly):
    """Full backward-Euler steps (assemble V, solve, Joule + thermal rhs, solve) vs the oracle's LU path:
    relative error <= 1e-9 per field per step (solver tolerance 1e-12), temperature PSNR >= 80 dB."""
    rafem = R()
    m = mg.cube_mesh(n, jitter=0.1, seed=24 + n, sigma0="lognormal")
    Ts, Vs = [], []
    with rafem.Context(m, tol=1e-12, dt=5.0, assembly=assembly) as ctx:
        for _ in range(steps):
            s, st = ctx.solve_step()
            assert s == rafem.RAFEM_OK, st.as_dict()
            Ts.append(ctx.get_field(rafem.RAFEM_SYS_T))
            Vs.append(ctx.get_field(rafem.RAFEM_SYS_V))
    model = O.Model(m, O.Params(dt=5.0))
    T_ref, V_ref = model.run(steps)
    for k in range(steps):
        assert O.rel_err(Vs[k], V_ref[k]) <= 1e-9
        assert O.rel_err(Ts[k], T_ref[k]) <= 1e-9
    assert np.all(O.psnr(T_ref, np.array(Ts)) >= 80.0)
    assert T_ref[-1].max() > 37.5  # the run actually heats


@pytest.mark.parametrize("lanes", [1, 4, 8, 16, 32])
def test_lanes_and_ragged_tiles_agree(lanes):
    """SELL-32 (lanes 1) and every CSR lane width, with a ragged tile size (37 rows, rounded up to 64 for
    SELL), give the same two steps as the default schedule to 1e-11."""
    rafem = R()
    m = mg.cube_mesh(11, jitter=0.1, seed=31, sigma0="lognormal")
    with rafem.Context(m, tol=1e-12) as ref:
        ref.run(2)
        T0 = ref.get_field(rafem.RAFEM_SYS_T)
        V0 = ref.get_field(rafem.RAFEM_SYS_V)
    with rafem.Context(m, tol=1e-12, lanes_per_row=lanes, rows_per_tile=37) as ctx:
        ctx.run(2)
        assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), T0) <= 1e-11
        assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), V0) <= 1e-11


@pytest.mark.parametrize("n,steps", [(14, 3)])
def test_mixed_precision_matches_oracle(n, steps):
    """FP32 inner iterations + FP64 refinement: relative error vs the oracle <= 1e-8 per field per step,
    temperature PSNR >= 80 dB, at least one refinement per potential solve. The error is bounded by
    cond(A) x relative residual and cond(A_V) ~ 1e2 here, so the refinement runs to an FP64 residual of 1e-11
    (at 1e-10 the measured error was 1.0e-8, on the bound)."""
    rafem = R()
    m = mg.cube_mesh(n, jitter=0.1, seed=41, sigma0="lognormal")
    Ts, Vs = [], []
    with rafem.Context(m, precision=rafem.RAFEM_PRECISION_MIXED, dt=5.0, tol=1e-11) as ctx:
        for _ in range(steps):
            s, st = ctx.solve_step()
            assert s == rafem.RAFEM_OK, st.as_dict()
            assert st.refine_V >= 1 and st.relres_V <= 1e-11 and st.relres_T <= 1e-11
            Ts.append(ctx.get_field(rafem.RAFEM_SYS_T))
            Vs.append(ctx.get_field(rafem.RAFEM_SYS_V))
    T_ref, V_ref = O.Model(m, O.Params(dt=5.0)).run(steps)
    for k in range(steps):
        assert O.rel_err(Vs[k], V_ref[k]) <= 1e-8
        assert O.rel_err(Ts[k], T_ref[k]) <= 1e-8
    assert np.all(O.psnr(T_ref, np.array(Ts)) >= 80.0)


@pytest.mark.parametrize("lanes", [1, 8])
def test_mixed_matches_fp64_gpu_at_48(lanes):
    """At 48^3 (117,649 nodes) over 5 steps, mixed and FP64 GPU fields agree to 1e-8 relative. The field
    error is bounded by cond(A) x residual and cond(A_V) is ~1e3 at this size (a 1e-11 residual left a 2.4e-8
    difference), so both run to a 1e-12 FP64 residual."""
    rafem = R()
    m = mg.workload_48()
    out = {}
    for prec in (rafem.RAFEM_PRECISION_FP64, rafem.RAFEM_PRECISION_MIXED):
        with rafem.Context(m, precision=prec, lanes_per_row=lanes, tol=1e-12) as ctx:
            s, st = ctx.run(5)
            assert s == rafem.RAFEM_OK, st.as_dict()
            out[prec] = (ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V))
    assert O.rel_err(out[1][0], out[0][0]) <= 1e-8
    assert O.rel_err(out[1][1], out[0][1]) <= 1e-8


def test_graph_run_equals_step_loop_bitwise():
    """rafem_run (one CUDA graph per step) and repeated rafem_solve_step give bit-identical fields; two runs
    are bit-identical (fixed reduction order)."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=32)
    out = []
    for mode in ("run", "step", "run"):
        with rafem.Context(m) as ctx:
            if mode == "run":
                s, st = ctx.run(4)
            else:
                for _ in range(4):
                    s, st = ctx.solve_step()
            assert s == rafem.RAFEM_OK and st.step == 4
            out.append((ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V)))
    for T, V in out[1:]:
        np.testing.assert_array_equal(T, out[0][0])
        np.testing.assert_array_equal(V, out[0][1])


def test_state_roundtrip_continues_run_bitwise():
    """Reading the fields back and setting them again at the same step index continues the run exactly (the
    predictor history is kept); setting them at another index restarts the history but stays within the
    solver tolerance of the uninterrupted run."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=34)
    with rafem.Context(m, tol=1e-12) as a:
        a.run(4)
        T4, V4 = a.get_field(rafem.RAFEM_SYS_T), a.get_field(rafem.RAFEM_SYS_V)
    with rafem.Context(m, tol=1e-12) as b:
        b.run(2)
        T2, V2 = b.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_V)
        b.set_state(T=T2, V=V2, step=2)
        b.run(2)
        np.testing.assert_array_equal(b.get_field(rafem.RAFEM_SYS_T), T4)
        np.testing.assert_array_equal(b.get_field(rafem.RAFEM_SYS_V), V4)
    with rafem.Context(m, tol=1e-12) as c:
        c.set_state(T=T2, V=V2, step=2)
        c.run(2)
        assert O.rel_err(c.get_field(rafem.RAFEM_SYS_V), V4) <= 1e-9
        assert O.rel_err(c.get_field(rafem.RAFEM_SYS_T), T4) <= 1e-9


def test_iteration_cap_reports_not_converged():
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=33)
    with rafem.Context(m, max_iter=3) as ctx:
        s, st = ctx.solve_step()
    assert s == rafem.RAFEM_NOT_CONVERGED
    assert st.iters_V == 3 and st.relres_V > 1e-10


def test_bad_inputs_rejected():
    rafem = R()
    m = mg.cube_mesh(3)
    bad = dataclasses.replace(m, sigma0=np.where(np.arange(m.n_tets) == 5, np.nan, m.sigma0))
    with pytest.raises(rafem.RafemError) as e:
        rafem.Context(bad)
    assert e.value.status == rafem.RAFEM_ERR_NONFINITE
    t = m.tets.copy()
    t[7] = [0, 1, 2, 3]  # coplanar nodes on the bottom face
    with pytest.raises(rafem.RafemError) as e:
        rafem.Context(dataclasses.replace(m, tets=t))
    assert e.value.status == rafem.RAFEM_ERR_BAD_MESH
    t = m.tets.copy()
    t[2, 1] = m.n_nodes + 5
    with pytest.raises(rafem.RafemError) as e:
        rafem.Context(dataclasses.replace(m, tets=t))
    assert e.value.status == rafem.RAFEM_ERR_BAD_INPUT


@pytest.mark.parametrize("n", [1, 2])
def test_degenerate_tiny_meshes(n):
    """n=1: every node is Dirichlet (the solution is the boundary data). n=2: one interior node."""
    rafem = R()
    m = mg.cube_mesh(n)
    with rafem.Context(m) as ctx:
        s, st = ctx.run(2)
        assert s == rafem.RAFEM_OK
        T = ctx.get_field(rafem.RAFEM_SYS_T)
        V = ctx.get_field(rafem.RAFEM_SYS_V)
    T_ref, V_ref = O.Model(m).run(2)
    np.testing.assert_allclose(V, V_ref[-1], rtol=0, atol=1e-9 * 20)
    np.testing.assert_allclose(T, T_ref[-1], rtol=0, atol=1e-9 * 37)


def _sampled_check(m, ctx, rafem, T_before, rng, n_rand=3000):
    """Sampled-row parity of both lifted systems and of the solutions after one step at full size."""
    V = ctx.get_field(rafem.RAFEM_SYS_V)
    T = ctx.get_field(rafem.RAFEM_SYS_T)
    # rows carrying the potential's right-hand side, plus random rows
    hot = rows_adjacent_to(m, np.nonzero(m.electrode)[0])
    rows = np.unique(np.concatenate([hot, rng.integers(0, m.n_nodes, n_rand)]))
    rp, col, vals, rhs = ctx.get_system(rafem.RAFEM_SYS_V)
    r_ids, ref, b_ref = lifted_rows(m, rows, T_before, which="V")
    bnorm = np.sqrt(np.sum(b_ref[np.isin(r_ids, hot)] ** 2))  # all nonzero rhs rows are in `hot`
    worst_val = worst_res = 0.0
    for k, i in enumerate(r_ids):
        cols = col[rp[i]:rp[i + 1]]
        got = vals[rp[i]:rp[i + 1]]
        exp = np.array([ref[i].get(int(c), np.nan) for c in cols])
        assert set(cols.tolist()) == set(ref[i].keys())
        worst_val = max(worst_val, np.abs(got - exp).max() / np.abs(exp).max())
        assert abs(rhs[i] - b_ref[k]) <= 1e-13 * max(abs(b_ref[k]), 1.0)
        worst_res = max(worst_res, abs(np.dot(exp, V[cols]) - b_ref[k]))
    assert worst_val <= 1e-13
    assert worst_res <= 2e-10 * bnorm, (worst_res, bnorm)
    # thermal system rows with the GPU's V and the pre-step T (sigma and mass term)
    rp, col, vals, rhs = ctx.get_system(rafem.RAFEM_SYS_T)
    r_ids, ref, b_ref = lifted_rows(m, rows, T_before, which="T", V=V, T_old=T_before)
    for k, i in enumerate(r_ids):
        cols = col[rp[i]:rp[i + 1]]
        exp = np.array([ref[i][int(c)] for c in cols])
        np.testing.assert_allclose(vals[rp[i]:rp[i + 1]], exp, rtol=1e-13, atol=1e-14 * np.abs(exp).max())
        np.testing.assert_allclose(rhs[i], b_ref[k], rtol=1e-12)
        # ||r|| <= tol ||b|| with ||b|| >= ||b_sampled||: per-row bound on the sampled rows
        assert abs(np.dot(exp, T[cols]) - b_ref[k]) <= 1e-10 * np.sqrt(m.n_nodes) * np.abs(b_ref).max()


@pytest.mark.parametrize("n", [48, 127])
def test_full_size_sampled_rows(n):
    """At the full workload sizes (48^3 and 127^3 cells, bench launch configuration): after one step the
    assembled rows agree with the oracle slot by slot and the solutions satisfy the oracle's equations on
    sampled rows (all rows carrying the potential's rhs plus 3000 random rows)."""
    rafem = R()
    m = mg.workload_48() if n == 48 else mg.workload_127()
    rng = np.random.default_rng(n)
    with rafem.Context(m) as ctx:
        T_before = ctx.get_field(rafem.RAFEM_SYS_T)
        s, st = ctx.run(1)
        assert s == rafem.RAFEM_OK, st.as_dict()
        assert st.relres_V <= 1e-10 and st.relres_T <= 1e-10
        _sampled_check(m, ctx, rafem, T_before, rng)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_predictor_reproduces_steady_fields(order):
    """With alpha_sigma = 0 the potential does not change from step to step, and every extrapolation order
    reproduces a constant sequence exactly (its coefficients sum to one), so from the second step on the potential
    solve starts at its converged solution and takes no iteration."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=61, sigma0="lognormal")
    with rafem.Context(m, alpha_sigma=0.0, predictor=order) as ctx:
        s, st = ctx.solve_step()
        assert s == 0 and st.iters_V > 0
        for _ in range(4):
            s, st = ctx.solve_step()
            assert s == 0 and st.iters_V == 0


def test_renumbered_meshes_give_the_same_fields():
    """A seeded random renumbering of the nodes (scattered gathers) and its reverse Cuthill-McKee renumbering give,
    mapped back to the lattice numbering, the fields of the lattice-numbered mesh after 3 steps (to 1e-9 at a
    1e-12 residual)."""
    rafem = R()
    m = mg.cube_mesh(14, jitter=0.1, seed=62, sigma0="lognormal")
    shuffled, p1 = mg.shuffled_nodes(m, 7)
    p2 = rafem.reorder_rcm(shuffled)
    rcm = mg.permute_nodes(shuffled, p2)
    out = {}
    for name, mesh, to_lattice in (("lattice", m, np.arange(m.n_nodes)), ("random", shuffled, p1),
                                   ("rcm", rcm, p1[p2])):
        with rafem.Context(mesh, tol=1e-12) as ctx:
            ctx.run(3)
            T = np.empty(m.n_nodes)
            V = np.empty(m.n_nodes)
            T[to_lattice] = ctx.get_field(rafem.RAFEM_SYS_T)
            V[to_lattice] = ctx.get_field(rafem.RAFEM_SYS_V)
            out[name] = (T, V, ctx.layout_info()["column_bytes"])
    for name in ("random", "rcm"):
        assert O.rel_err(out[name][0], out["lattice"][0]) <= 1e-9
        assert O.rel_err(out[name][1], out["lattice"][1]) <= 1e-9


def test_set_tol_and_graph_kernels():
    """rafem_set_tol changes the residual target of a live context (graphs rebuilt, state kept); the step graph
    reports its kernel count."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=12, sigma0="lognormal")
    with rafem.Context(m, precision=rafem.RAFEM_PRECISION_MIXED, tol=1e-6) as ctx:
        s, st = ctx.run(3)
        assert s == 0 and st.relres_V <= 1e-6 and st.relres_T <= 1e-6
        g = ctx.graph_info()
        assert g["step_graph"] == 1 and g["step_kernels"] >= 8
        ctx.set_tol(1e-12, 1e-5)
        s, st = ctx.run(1)
        assert s == 0 and st.relres_V <= 1e-12 and st.relres_T <= 1e-12 and st.step == 4
        with pytest.raises(rafem.RafemError):
            ctx.set_tol(0.0)
        with pytest.raises(rafem.RafemError):
            ctx.set_tol(1e-8, 1.5)


@pytest.mark.parametrize("basis", [1, 2, 3, 6, 8])
def test_projection_basis_sizes(basis):
    """The projection predictor with 1..8 past solutions (the basis rebuilt each step from the previous one):
    steady potential reproduced exactly from the second step (no iteration), and a heating run that matches the
    oracle's direct solves at 1e-9 after 12 steps, in both arithmetics of the predictor's passes."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=61, sigma0="lognormal")
    with rafem.Context(m, alpha_sigma=0.0, proj_basis=basis) as ctx:
        s, st = ctx.solve_step()
        assert s == 0 and st.iters_V > 0
        for _ in range(3):
            s, st = ctx.solve_step()
            assert s == 0 and st.iters_V == 0
    steps = 12
    T_ref, V_ref = O.Model(m, O.Params(dt=5.0)).run(steps)
    for arith in (rafem.RAFEM_ARITH_DW, rafem.RAFEM_ARITH_FP64):
        with rafem.Context(m, tol=1e-12, dt=5.0, proj_basis=basis, arith=arith) as ctx:
            s, st = ctx.run(steps)
            assert s == 0
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), V_ref[-1]) <= 1e-9
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), T_ref[-1]) <= 1e-9


def test_larger_projection_basis_saves_iterations():
    """Over a heating run the 8-solution basis needs fewer potential iterations than the 4-solution basis."""
    rafem = R()
    m = mg.cube_mesh(20, jitter=0.1, seed=62, sigma0="lognormal")
    iters = {}
    for basis in (4, 8):
        with rafem.Context(m, proj_basis=basis) as ctx:
            ctx.run(5)
            ctx.set_tracing(True)
            ctx.run(25)
            iters[basis] = ctx.get_trace()["iters_V"]
    assert iters[8] < iters[4], iters


@pytest.mark.parametrize("basis", [2, 4])
def test_projection_guess_matches_oracle(basis):
    """The potential's initial guess equals the oracle's A-norm projection of the same system onto the same past
    solutions (the oracle's own, from its direct solves) to 1e-8: a solve whose tolerance accepts any residual
    returns the guess unchanged. Guesses from neighbouring basis sizes differ by 2e-6 (3 vs 4) to 4e-5 (2 vs 4) on
    this run, so the bound also checks which solutions the basis holds: after six steps the last min(basis, 5)
    (the first solve never enters the basis)."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=64, sigma0="lognormal")
    model = O.Model(m, O.Params(dt=5.0))
    T_ref, V_ref = model.run(6)
    with rafem.Context(m, tol=1e-13, dt=5.0, proj_basis=basis, precision=rafem.RAFEM_PRECISION_FP64) as ctx:
        s, _ = ctx.run(6)
        assert s == 0
        assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), T_ref[5]) <= 1e-9
        ctx.set_tol(1e100)
        s, st = ctx.solve_step()
        assert s == 0 and st.iters_V == 0
        guess = ctx.get_field(rafem.RAFEM_SYS_V)
    k = min(basis, 5)
    X = np.stack([V_ref[5 - j] for j in range(k)], axis=1)
    A, b = model.system_V(T_ref[5])
    x0 = O.projection_guess(A, b, X, ~m.bc_V.astype(bool))
    assert O.rel_err(guess, x0) <= 1e-8
    assert O.rel_err(guess, O.solve(A, b)) > 1e-8  # a guess, not the solution


@pytest.mark.parametrize("pinned", [False, True])
def test_step_host_equals_device_steps(pinned):
    """rafem_step_host (state in and out of host buffers, copies overlapped with the step on a second stream)
    gives bitwise the fields and statistics of the same steps run on device-resident state."""
    import torch
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=63, sigma0="lognormal")
    with rafem.Context(m, precision=rafem.RAFEM_PRECISION_MIXED) as a, \
            rafem.Context(m, precision=rafem.RAFEM_PRECISION_MIXED) as b:
        a.run(2)
        b.run(2)
        if pinned:
            T = torch.from_numpy(b.get_field(rafem.RAFEM_SYS_T)).pin_memory()
            V = torch.from_numpy(b.get_field(rafem.RAFEM_SYS_V)).pin_memory()
            ptr = lambda x: x.data_ptr()
            tonp = lambda x: x.numpy()
        else:
            T, V = b.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_V)
            ptr = lambda x: x.ctypes.data
            tonp = lambda x: x
        for _ in range(4):
            sa, sta = a.solve_step()
            # V stays on the device (b's equals a's): the launches of a device step
            sb, stb = b.step_host_ptr(ptr(T), None, ptr(T), ptr(V))
            assert sa == sb == 0
            assert sta.as_dict() == stb.as_dict()
            np.testing.assert_array_equal(tonp(T), a.get_field(rafem.RAFEM_SYS_T))
            np.testing.assert_array_equal(tonp(V), a.get_field(rafem.RAFEM_SYS_V))
        # V read from the host too: the predictor then forms A D in a pass of its own (the assembly, which would
        # otherwise form it, runs while V is copied in), rounded differently, so the solves agree to their tolerance
        for _ in range(3):
            sa, sta = a.solve_step()
            sb, stb = b.step_host_ptr(ptr(T), ptr(V), ptr(T), ptr(V))
            assert sa == sb == 0
            assert stb.relres_V <= 1e-10 and stb.relres_T <= 1e-10
            assert abs(sta.iters_V - stb.iters_V) <= 1 and abs(sta.iters_T - stb.iters_T) <= 1
            assert O.rel_err(tonp(T), a.get_field(rafem.RAFEM_SYS_T)) <= 1e-9
            assert O.rel_err(tonp(V), a.get_field(rafem.RAFEM_SYS_V)) <= 1e-8
        if pinned:
            assert b.graph_info()["step_graph"] in (-1, 0, 1)
