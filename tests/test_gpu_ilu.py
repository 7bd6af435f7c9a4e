"""ILU(0) preconditioner on the GPU vs the oracle: level order (bit-exact), factors on the pattern, the
preconditioner application, and whole time steps solved with ILU(0)-PCG (needs a B300)."""

import numpy as np
import pytest

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

ORDERS = {"multicolor": 0, "natural": 1}


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


def _nonuniform_T(mesh, seed=0):
    rng = np.random.default_rng(seed)
    return np.where(mesh.bc_T.astype(bool), mesh.g_T, 37.0 + 25.0 * rng.random(mesh.n_nodes))


def _oracle_factors_on_original_pattern(A, order):
    perm, _ = O.ilu_permutation(A, order)
    F = O.ilu0(O.permute_symmetric(A, perm))
    back = O.permute_symmetric(F, np.argsort(perm))
    return perm, F, back


@pytest.mark.parametrize("order", ["multicolor", "natural"])
@pytest.mark.parametrize("layout", [dict(), dict(lanes_per_row=8, assembly=1)], ids=["sell-gather", "csr8-colour"])
def test_ilu_order_and_factors_match_oracle(order, layout):
    """The level order equals the oracle's (bit-exact), and the ILU(0) factors of the assembled potential system at
    a non-uniform temperature and of the thermal system agree entry by entry (rtol 1e-12)."""
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=41, sigma0="lognormal")
    T = _nonuniform_T(m)
    model = O.Model(m)
    with rafem.Context(m, precond=1, ilu_order=ORDERS[order], **layout) as ctx:
        info = ctx.precond_info()
        ctx.set_state(T=T)
        ctx.assemble(rafem.RAFEM_SYS_V)
        FV = ctx.get_precond(rafem.RAFEM_SYS_V)
        FT = ctx.get_precond(rafem.RAFEM_SYS_T)
    AV, _ = model.system_V(T)
    AT, _ = model.system_T(T, np.zeros(m.n_tets))
    perm, _, FV_ref = _oracle_factors_on_original_pattern(AV, order)
    np.testing.assert_array_equal(info["order"], perm)
    assert info["n_levels"] == (4 if order == "multicolor" else 3 * 8 + 1)
    np.testing.assert_allclose(FV, FV_ref.data, rtol=1e-12, atol=1e-13 * np.abs(FV_ref.data).max())
    _, _, FT_ref = _oracle_factors_on_original_pattern(AT, order)
    np.testing.assert_allclose(FT, FT_ref.data, rtol=1e-12, atol=1e-13 * np.abs(FT_ref.data).max())


@pytest.mark.parametrize("order", ["multicolor", "natural"])
def test_ilu_apply_matches_oracle(order):
    """z = M^-1 r through rafem_precond_apply equals the oracle's forward/backward substitution with its own
    factors (rtol 1e-11), for the potential system."""
    import torch
    rafem = R()
    m = mg.cube_mesh(9, jitter=0.1, seed=42, sigma0="lognormal")
    T = _nonuniform_T(m, 1)
    r = np.random.default_rng(3).normal(size=m.n_nodes)
    with rafem.Context(m, precond=1, ilu_order=ORDERS[order]) as ctx:
        ctx.set_state(T=T)
        ctx.assemble(rafem.RAFEM_SYS_V)
        rd = torch.tensor(r, dtype=torch.float64, device="cuda")
        zd = torch.empty_like(rd)
        torch.cuda.synchronize()
        ctx.precond_apply(rafem.RAFEM_SYS_V, rd, zd)
        z = zd.cpu().numpy()
    AV, _ = O.Model(m).system_V(T)
    perm, F, _ = _oracle_factors_on_original_pattern(AV, order)
    zp = O.ilu0_apply(F, r[perm])
    z_ref = np.empty_like(zp)
    z_ref[perm] = zp
    np.testing.assert_allclose(z, z_ref, rtol=1e-11, atol=1e-11 * np.abs(z_ref).max())


@pytest.mark.parametrize("order", ["multicolor", "natural"])
def test_ilu_time_steps_match_oracle(order):
    """Four time steps with ILU(0)-PCG (tol 1e-12) on a jittered lognormal 12^3 mesh agree with the oracle's direct
    solves: relative error of V and T <= 1e-9 at every step."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=43, sigma0="lognormal")
    Ts, Vs = O.Model(m).run(4)
    with rafem.Context(m, precond=1, ilu_order=ORDERS[order], tol=1e-12) as ctx:
        for k in range(4):
            s, st = ctx.solve_step()
            assert s == 0 and st.iters_V > 0
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), Ts[k]) <= 1e-9
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), Vs[k]) <= 1e-9


def test_ilu_needs_fewer_iterations_than_jacobi_and_agrees():
    """On the 48^3 jittered workload the ILU(0) (multicolour) solves take fewer Krylov iterations than Jacobi, and
    after 3 steps both give the same fields to 2e-8 (both at the 1e-12 residual; the potential system's condition
    number turns a 1e-10 residual into differences near 5e-7)."""
    rafem = R()
    m = mg.workload_48()
    out = {}
    for name, kw in (("jacobi", dict(tol=1e-12)), ("ilu", dict(precond=1, tol=1e-12))):
        with rafem.Context(m, **kw) as ctx:
            s, st = ctx.run(3)
            assert s == 0
            out[name] = (st.iters_V, st.iters_T, ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V))
    assert out["ilu"][0] < out["jacobi"][0] and out["ilu"][1] <= out["jacobi"][1]
    assert O.rel_err(out["ilu"][2], out["jacobi"][2]) < 2e-8
    assert O.rel_err(out["ilu"][3], out["jacobi"][3]) < 2e-8


def test_ilu_graph_run_equals_step_loop_and_adjoint_works():
    """rafem_run (CUDA graph) gives bitwise the fields of the step-by-step loop with ILU(0), and the adjoint runs
    on ILU(0) contexts (gradients equal to the Jacobi context's to 1e-8)."""
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=44, sigma0="lognormal")
    with rafem.Context(m, precond=1, tol=1e-13) as a, rafem.Context(m, precond=1, tol=1e-13) as b:
        a.run(3)
        for _ in range(3):
            b.solve_step()
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_T))
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_V), b.get_field(rafem.RAFEM_SYS_V))
    grads = []
    for kw in (dict(precond=1), dict()):
        with rafem.Context(m, tol=1e-13, dt=5.0, **kw) as ctx:
            ctx.tape_begin(2)
            ctx.run(3)
            T = ctx.get_field(rafem.RAFEM_SYS_T)
            grads.append(ctx.adjoint(2.0 * (T - 37.2)))
    for q in range(3):
        ref = grads[1][q]
        assert np.abs(grads[0][q] - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("order", ["multicolor", "natural"])
def test_ilu_mixed_time_steps_match_oracle(order):
    """Mixed-precision ILU(0)-PCG (FP32 factors, values and vectors in the inner iterations, FP64 residual
    refinement, tol 1e-11): four time steps on a jittered lognormal 12^3 mesh agree with the oracle's direct solves
    to 1e-8 (the mixed-precision parity bound), and the potential solves refine at least once."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=45, sigma0="lognormal")
    Ts, Vs = O.Model(m).run(4)
    with rafem.Context(m, precond=1, precision=1, ilu_order=ORDERS[order], tol=1e-11) as ctx:
        for k in range(4):
            s, st = ctx.solve_step()
            assert s == 0 and st.iters_V > 0 and st.refine_V >= 1 and st.relres_V <= 1e-11
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_T), Ts[k]) <= 1e-8
            assert O.rel_err(ctx.get_field(rafem.RAFEM_SYS_V), Vs[k]) <= 1e-8


@pytest.mark.parametrize("order", ["multicolor", "natural"])
def test_ilu_iterations_match_oracle_pcg(order):
    """The GPU's FP64 ILU(0)-PCG from x = 0 on the assembled potential system takes the iterations of the oracle's
    textbook PCG with the oracle's ILU(0) factors of the same permuted system (within one: rounding), and reaches
    its solution: a weaker or different preconditioner would converge too, but in a different number of steps."""
    import torch
    rafem = R()
    m = mg.cube_mesh(10, jitter=0.1, seed=46, sigma0="lognormal")
    T = _nonuniform_T(m, 3)
    AV, bV = O.Model(m).system_V(T)
    perm, _ = O.ilu_permutation(AV, order)
    Ap = O.permute_symmetric(AV, perm)
    F = O.ilu0(Ap)
    xo, it_o = O.pcg(Ap, bV[perm], np.zeros(m.n_nodes), lambda r: O.ilu0_apply(F, r), 1e-10)
    with rafem.Context(m, precond=1, ilu_order=ORDERS[order], tol=1e-10) as ctx:
        ctx.set_state(T=T)
        ctx.assemble(rafem.RAFEM_SYS_V)
        b = torch.tensor(bV, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x)
    assert s == 0
    assert abs(st.iters_V - it_o) <= 1, (st.iters_V, it_o)
    x_o = np.empty(m.n_nodes)
    x_o[perm] = xo
    assert O.rel_err(x.cpu().numpy(), x_o) <= 1e-7


def test_ilu_rejected_combinations():
    """ILU(0) is single-instance: a batch or an unknown ordering give BAD_INPUT; inspection calls on a Jacobi
    context give BAD_INPUT."""
    rafem = R()
    m = mg.cube_mesh(4, jitter=0.1, seed=5)
    with pytest.raises(rafem.RafemError):
        rafem.Context(m, precond=1, ilu_order=7)
    with pytest.raises(rafem.RafemError):
        rafem.Context.batch([m, m], precond=1)
    with rafem.Context(m) as ctx:
        with pytest.raises(rafem.RafemError):
            ctx.precond_info()
