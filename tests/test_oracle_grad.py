"""Pins of the oracle's gradients (differentiation of the time loop) against what does not depend on them.

The dense adjoint (explicit step Jacobians from the tangent-linear step, accumulated with their transposes) is
checked against central finite differences of the oracle's forward model, which is itself pinned by the
physics tests, and against an exact homogeneity identity. No GPU.
"""
import dataclasses

import numpy as np

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg

N_STEPS = 3


def _tiny():
    """5x5x5 nodes with an interior electrode node, jittered, lognormal sigma0; dt = 5 s for visible heating."""
    m = mg.cube_mesh(4, jitter=0.1, seed=5, sigma0="lognormal")
    assert ((m.g_V > 0) & m.bc_V.astype(bool)).sum() >= 2
    return m, O.Model(m, O.Params(dt=5.0))


def test_dense_adjoint_matches_central_differences():
    """dL/dsigma0_e, dL/dk_e and dL/dT0_i of L = |T^N - target|^2 from the dense adjoint agree with central
    differences (relative step 1e-3 for the conductivities, 1e-3 degC for T0; truncation error ~1e-7)."""
    m, model = _tiny()
    T, _ = model.run(N_STEPS)
    target = T[-1] + np.random.default_rng(0).normal(0.0, 0.5, model.N)
    g_s, g_k, g_0 = O.gradient_dense_adjoint(model, N_STEPS, 2.0 * (T[-1] - target))
    elems = [0, 5, 17, 100, 200, 383]
    fd_s = O.gradient_fd(model, N_STEPS, target, "sigma0", elems, eps=1e-3)
    fd_k = O.gradient_fd(model, N_STEPS, target, "k", elems, eps=1e-3)
    assert np.abs(g_s[elems] - fd_s).max() <= 1e-6 * np.abs(fd_s).max()
    assert np.abs(g_k[elems] - fd_k).max() <= 1e-6 * np.abs(fd_k).max()
    # initial state: a free node, and boundary nodes that do / do not reach a free row
    T0 = np.full(model.N, 37.0)
    for i in [0, 12, 62, 70]:
        h = 1e-3
        lp = O.loss_final_T(model, N_STEPS, target, np.where(np.arange(model.N) == i, 37.0 + h, T0))
        lm = O.loss_final_T(model, N_STEPS, target, np.where(np.arange(model.N) == i, 37.0 - h, T0))
        fd = (lp - lm) / (2 * h)
        assert abs(g_0[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g_0).max())


def test_sigma0_gradient_homogeneity_identity():
    """With alpha = 0, T_a = T0 = Dirichlet T = 37, scaling every sigma0 by c leaves V unchanged and scales the
    Joule source by c; the thermal update is linear and homogeneous in (T - 37, source), so T^N - 37 scales by c
    exactly. Hence sum_e sigma0_e dL/dsigma0_e = dL/dc at c = 1 = lam^T (T^N - 37) with lam = dL/dT^N."""
    m = mg.cube_mesh(4, jitter=0.1, seed=9, sigma0="lognormal")
    model = O.Model(m, O.Params(dt=5.0, alpha_sigma=0.0))
    T, _ = model.run(N_STEPS)
    lam = np.random.default_rng(1).normal(size=model.N)
    g_s, _, _ = O.gradient_dense_adjoint(model, N_STEPS, lam)
    lhs = float(np.dot(model.sigma0, g_s))
    rhs = float(np.dot(lam, T[-1] - 37.0))
    assert abs(rhs) > 0
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_tangent_step_linear_in_direction_and_matches_step():
    """The tangent step returns the forward step's T^{n+1}, and its derivative is linear in the direction
    (the sum of two directions gives the sum of the derivatives)."""
    m, model = _tiny()
    rng = np.random.default_rng(2)
    T1, _, _ = model.step(np.full(model.N, 37.0))
    Tn = T1 + rng.normal(0.0, 0.1, model.N) * (~model.bc_T)
    E = len(model.tets)
    d1 = [rng.normal(size=(model.N, 1)), rng.normal(size=(E, 1)), rng.normal(size=(E, 1))]
    d2 = [rng.normal(size=(model.N, 1)), rng.normal(size=(E, 1)), rng.normal(size=(E, 1))]
    Tnew, _, a = O.step_tangent(model, Tn, *d1)
    _, _, b = O.step_tangent(model, Tn, *d2)
    _, _, c = O.step_tangent(model, Tn, *[x + y for x, y in zip(d1, d2)])
    ref, _, _ = model.step(Tn)
    np.testing.assert_allclose(Tnew, ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(c, a + b, rtol=0, atol=1e-10 * np.abs(c).max())


def test_gradient_zero_without_electrode_source_for_sigma():
    """With V = 0 everywhere (electrode voltage 0) the Joule source vanishes for every sigma0, so dL/dsigma0 = 0
    exactly, while dL/dk does not vanish when T^N differs from the target."""
    m = mg.cube_mesh(4, jitter=0.1, seed=5, sigma0="lognormal", V_electrode=0.0)
    model = O.Model(m, O.Params(dt=5.0))
    T, _ = model.run(2)
    target = T[-1] + 0.3 * (~model.bc_T)
    g_s, g_k, _ = O.gradient_dense_adjoint(model, 2, 2.0 * (T[-1] - target))
    assert np.abs(g_s).max() == 0.0
    # T stays at 37 everywhere, so K_k T = 0 and dL/dk = 0 too; perturb the initial state to make it nonzero
    T0 = 37.0 + 0.5 * (~model.bc_T)
    g_s2, g_k2, _ = O.gradient_dense_adjoint(model, 2, 2.0 * (model.run(2, T0)[0][-1] - target), T0=T0)
    assert np.abs(g_s2).max() == 0.0 and np.abs(g_k2).max() > 0.0
