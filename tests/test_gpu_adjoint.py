"""Differentiation form on the GPU: rafem_adjoint vs the oracle's dense adjoint and vs central differences,
checkpoint invariance, state restoration, batching and the torch.autograd bridge (needs a B300)."""
import numpy as np
import pytest

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-13, dt=5.0)


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


def _relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def _tiny():
    return mg.cube_mesh(4, jitter=0.1, seed=5, sigma0="lognormal")


def _gpu_grad(mesh, n_steps, every, lam_of_T, **kw):
    rafem = R()
    with rafem.Context(mesh, **kw) as ctx:
        ctx.tape_begin(every)
        ctx.run(n_steps)
        T = ctx.get_field(rafem.RAFEM_SYS_T)
        gs, gk, g0, st = ctx.adjoint(lam_of_T(T))
    return gs, gk, g0, st, T


@pytest.mark.parametrize("kw", [dict(), dict(precision=1), dict(lanes_per_row=8, assembly=1)],
                         ids=["fp64-gather", "mixed-gather", "csr8-colour"])
def test_adjoint_matches_oracle_dense_adjoint(kw):
    """dL/dsigma0, dL/dk and dL/dT0 of L = |T^N - target|^2 on a 125-node jittered lognormal mesh after 3 steps
    (checkpoint every 2): GPU adjoint vs the oracle's dense adjoint (explicit Jacobians), max-norm relative error
    <= 1e-8 (both solve to 1e-13 residual; the oracle directly)."""
    m = _tiny()
    model = O.Model(m, O.Params(dt=5.0))
    Tref, _ = model.run(3)
    target = Tref[-1] + np.random.default_rng(0).normal(0.0, 0.5, model.N)
    lam = 2.0 * (Tref[-1] - target)
    o_s, o_k, o_0 = O.gradient_dense_adjoint(model, 3, lam)
    gs, gk, g0, st, T = _gpu_grad(m, 3, 2, lambda T: 2.0 * (T - target), **TIGHT, **kw)
    assert st["status"] == 0 and st["forward_status"] == 0 and st["steps"] == 3 and st["segments"] == 2
    assert _relmax(T, Tref[-1]) < 1e-12
    assert _relmax(gs, o_s) <= 1e-8
    assert _relmax(gk, o_k) <= 1e-8
    assert _relmax(g0, o_0) <= 1e-8


def test_checkpoint_spacing_gives_bitwise_identical_gradients():
    """The recomputed forward states are bitwise those of the recorded run, so every checkpoint spacing gives the
    same gradients bit for bit."""
    m = mg.cube_mesh(8, jitter=0.1, seed=3, sigma0="lognormal")
    target = np.full(m.n_nodes, 37.5)
    out = [_gpu_grad(m, 7, every, lambda T: 2.0 * (T - target), dt=5.0) for every in (1, 3, 7, 50)]
    for gs, gk, g0, st, _ in out[1:]:
        np.testing.assert_array_equal(gs, out[0][0])
        np.testing.assert_array_equal(gk, out[0][1])
        np.testing.assert_array_equal(g0, out[0][2])
    assert [o[3]["segments"] for o in out] == [7, 3, 1, 1]


def test_adjoint_leaves_forward_state_unchanged():
    """After rafem_adjoint the fields are bitwise those before it, and continuing the run gives bitwise the same
    fields as a run that never called the adjoint (predictor history and statistics restored too)."""
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=4, sigma0="lognormal")
    with rafem.Context(m, dt=5.0) as a, rafem.Context(m, dt=5.0) as b:
        a.tape_begin(2)
        a.run(5)
        b.run(5)
        T5 = a.get_field(rafem.RAFEM_SYS_T)
        V5 = a.get_field(rafem.RAFEM_SYS_V)
        a.adjoint(np.ones(m.n_nodes))
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_T), T5)
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_V), V5)
        _, sa = a.run(3)
        _, sb = b.run(3)
        assert sa.step == sb.step == 8
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_T))
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_V), b.get_field(rafem.RAFEM_SYS_V))


def test_adjoint_matches_central_differences_on_gpu():
    """12^3 mesh, 10 steps, checkpoint every 4: adjoint gradients for 6 elements next to the electrode (sigma0 and
    k) and 3 free nodes of T0 agree with central differences of the GPU forward (relative step 1e-3, solves to
    1e-13) within 1e-5 relative."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.1, seed=8, sigma0="lognormal")
    n, every = 10, 4
    target = np.where(m.bc_T.astype(bool), m.g_T, 38.0)

    def loss(ctx, s0=None, kk=None, T0=None):
        ctx.set_params(m.sigma0 if s0 is None else s0, m.k if kk is None else kk)
        ctx.reset()
        if T0 is not None:
            ctx.set_state(T=T0, step=0)
        ctx.run(n)
        return float(np.sum((ctx.get_field(rafem.RAFEM_SYS_T) - target) ** 2))

    with rafem.Context(m, **TIGHT) as ctx:
        ctx.tape_begin(every)
        ctx.run(n)
        T = ctx.get_field(rafem.RAFEM_SYS_T)
        gs, gk, g0, st = ctx.adjoint(2.0 * (T - target))
        assert st["status"] == 0
        cent = m.coords[m.tets].mean(axis=1)
        tip = np.array([0.0, 0.0, 0.02])
        elems = np.argsort(np.sum((cent - tip) ** 2, axis=1))[[0, 3, 10, 40, 200, 1000]]
        for which, g in (("sigma0", gs), ("k", gk)):
            base = m.sigma0 if which == "sigma0" else m.k
            fd = []
            for e in elems:
                h = 1e-3 * base[e]
                vals = []
                for sgn in (1.0, -1.0):
                    q = base.copy()
                    q[e] += sgn * h
                    vals.append(loss(ctx, **({"s0": q} if which == "sigma0" else {"kk": q})))
                fd.append((vals[0] - vals[1]) / (2 * h))
            fd = np.array(fd)
            assert np.abs(g[elems] - fd).max() <= 1e-5 * np.abs(fd).max(), (which, g[elems], fd)
        free = np.flatnonzero(~m.bc_T.astype(bool))
        T0 = np.where(m.bc_T.astype(bool), m.g_T, 37.0)
        for i in free[[0, len(free) // 2, -1]]:
            vals = []
            for sgn in (1.0, -1.0):
                t = T0.copy()
                t[i] += sgn * 1e-3
                vals.append(loss(ctx, T0=t))
            fd = (vals[0] - vals[1]) / 2e-3
            assert abs(g0[i] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g0).max())


def test_batch_adjoint_equals_single_instance_adjoints():
    """A batch of two instances back-propagates each instance independently: the gradients equal those of
    separate contexts (to solver tolerance)."""
    rafem = R()
    ms = [mg.cube_mesh(6, jitter=0.1, seed=31, sigma0="lognormal"),
          mg.cube_mesh(7, jitter=0.1, seed=32, sigma0="lognormal", V_electrode=30.0)]
    singles = [_gpu_grad(mm, 4, 3, lambda T: 2.0 * (T - 38.0), **TIGHT) for mm in ms]
    with rafem.Context.batch(ms, **TIGHT) as ctx:
        ctx.tape_begin(3)
        ctx.run(4)
        T = ctx.get_field(rafem.RAFEM_SYS_T)
        gs, gk, g0, st = ctx.adjoint(2.0 * (T - 38.0))
    off = ctx.offsets
    e0 = 0
    for i, mm in enumerate(ms):
        e1 = e0 + mm.n_tets
        assert _relmax(gs[e0:e1], singles[i][0]) < 1e-9
        assert _relmax(gk[e0:e1], singles[i][1]) < 1e-9
        assert _relmax(g0[off[i]:off[i] + mm.n_nodes], singles[i][2]) < 1e-9
        e0 = e1


def test_autograd_bridge_fp32_parameters():
    """torch.autograd through final_temperature with FP32 parameter tensors: gradients equal rafem_adjoint's
    (cast to FP32), and loss.backward() leaves the context usable for another forward."""
    import torch

    from paper_2409_13036_b300.adjoint import final_temperature
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=6, sigma0="lognormal")
    dev = torch.device("cuda:0")
    target = torch.full((m.n_nodes,), 37.4, dtype=torch.float64, device=dev)
    with rafem.Context(m, dt=5.0) as ctx:
        s0 = torch.tensor(m.sigma0, dtype=torch.float32, device=dev, requires_grad=True)
        kk = torch.tensor(m.k, dtype=torch.float32, device=dev, requires_grad=True)
        T = final_temperature(ctx, s0, kk, 6, checkpoint_every=2)
        loss = ((T - target) ** 2).sum()
        loss.backward()
        assert s0.grad.dtype == torch.float32 and kk.grad.dtype == torch.float32
        # the same through the host API with the FP32-rounded parameters
        ctx.set_params(s0.detach().double().cpu().numpy(), kk.detach().double().cpu().numpy())
        ctx.reset()
        ctx.tape_begin(3)
        ctx.run(6)
        Th = ctx.get_field(rafem.RAFEM_SYS_T)
        np.testing.assert_array_equal(Th, T.detach().cpu().numpy())
        gs, gk, _, _ = ctx.adjoint(2.0 * (Th - 37.4))
        np.testing.assert_allclose(s0.grad.cpu().numpy(), gs.astype(np.float32), rtol=1e-6,
                                   atol=1e-6 * np.abs(gs).max())
        np.testing.assert_allclose(kk.grad.cpu().numpy(), gk.astype(np.float32), rtol=1e-6,
                                   atol=1e-6 * np.abs(gk).max())


def test_set_params_equals_fresh_context():
    """rafem_set_params(sigma0', k') followed by a run gives bitwise the fields of a context created with them."""
    import dataclasses
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=7, sigma0="lognormal")
    rng = np.random.default_rng(3)
    s1 = m.sigma0 * (1.0 + 0.2 * rng.random(m.n_tets))
    k1 = m.k * (1.0 + 0.2 * rng.random(m.n_tets))
    m1 = dataclasses.replace(m, sigma0=s1, k=k1)
    with rafem.Context(m, dt=5.0) as a, rafem.Context(m1, dt=5.0) as b:
        a.run(2)
        a.set_params(s1, k1)
        a.reset()
        a.run(4)
        b.run(4)
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_T), b.get_field(rafem.RAFEM_SYS_T))
        np.testing.assert_array_equal(a.get_field(rafem.RAFEM_SYS_V), b.get_field(rafem.RAFEM_SYS_V))


def test_set_params_device_fp32_equals_fp64_of_rounded_values():
    """rafem_set_params_device (FP32 device arrays, widened in the library) gives bitwise the fields of
    rafem_set_params with the same FP32-rounded values as FP64 host arrays."""
    import torch
    rafem = R()
    m = mg.cube_mesh(8, jitter=0.1, seed=8, sigma0="lognormal")
    rng = np.random.default_rng(4)
    s32 = (m.sigma0 * (1.0 + 0.3 * rng.random(m.n_tets))).astype(np.float32)
    k32 = (m.k * (1.0 + 0.3 * rng.random(m.n_tets))).astype(np.float32)
    with rafem.Context(m, dt=5.0) as a, rafem.Context(m, dt=5.0) as b:
        ds = torch.tensor(s32, device="cuda")
        dk = torch.tensor(k32, device="cuda")
        torch.cuda.synchronize()
        a.set_params_device(ds, dk)
        b.set_params(s32.astype(np.float64), k32.astype(np.float64))
        a.run(3)
        b.run(3)
        for which in (rafem.RAFEM_SYS_V, rafem.RAFEM_SYS_T):
            np.testing.assert_array_equal(a.get_field(which), b.get_field(which))


def test_adjoint_input_errors():
    """No tape, tape with corrector passes, bad spacing: BAD_INPUT; an empty tape returns dL/dT as dL/dT0."""
    rafem = R()
    m = mg.cube_mesh(4, jitter=0.1, seed=5)
    with rafem.Context(m) as ctx:
        with pytest.raises(rafem.RafemError):
            ctx.adjoint(np.ones(m.n_nodes))
        with pytest.raises(rafem.RafemError):
            ctx.tape_begin(0)
        ctx.tape_begin(2)
        lam = np.arange(m.n_nodes, dtype=np.float64)
        gs, gk, g0, st = ctx.adjoint(lam)
        assert st["steps"] == 0 and np.all(gs == 0) and np.all(gk == 0)
        np.testing.assert_array_equal(g0, lam)
        ctx.run(1)
        ctx.set_state(T=ctx.get_field(rafem.RAFEM_SYS_T), step=0)  # ends the tape
        with pytest.raises(rafem.RafemError):
            ctx.adjoint(lam)
    with rafem.Context(m, n_corrector=3) as ctx:
        with pytest.raises(rafem.RafemError):
            ctx.tape_begin(2)
