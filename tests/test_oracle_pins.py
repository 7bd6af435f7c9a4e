"""Pins of the FP64 CPU oracle against what the mathematics and physics fix (no GPU).

Each test states the invariant it checks. Together they are chosen so that a dropped term, a wrong sign, a
wrong index or a transposed operand anywhere in the oracle breaks at least one of them.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg

L = 0.04  # half side of the cube, metres


def _slab_mesh(n, V0=10.0, T_D=37.0, jitter=0.0):
    """Cube with Dirichlet data on the two x faces only (Neumann elsewhere), for 1-D reductions."""
    m = mg.cube_mesh(n, jitter=jitter, seed=7)
    fx = (m.lattice[:, 0] == 0) | (m.lattice[:, 0] == n)
    return dataclasses.replace(m, bc_V=fx.astype(np.uint8), g_V=np.where(m.lattice[:, 0] == n, V0, 0.0),
                               bc_T=fx.astype(np.uint8), g_T=np.where(fx, T_D, 0.0))


def test_patch_test_linear_potential_reproduced():
    """P1 patch test: with Dirichlet data from a linear field on all faces, the FE solution equals the field
    at every node, on a jittered mesh with uniform conductivity."""
    m = mg.cube_mesh(6, jitter=0.1, seed=11)
    x, y, z = m.coords.T
    lin = 3.0 + 200.0 * x - 500.0 * y + 700.0 * z
    vol, grad = O.element_geometry(m.coords, m.tets)
    K = O.assemble(O.element_stiffness(np.full(m.n_tets, 0.4), vol, grad), m.tets, m.n_nodes)
    face = m.bc_T.astype(bool)
    A, b = O.dirichlet_lift(K, np.zeros(m.n_nodes), face, np.where(face, lin, 0.0))
    u = O.solve(A, b)
    assert (~face).sum() > 50
    np.testing.assert_allclose(u, lin, rtol=0, atol=1e-12 * np.abs(lin).max())


def test_stiffness_rows_sum_to_zero_and_symmetric():
    """K 1 = 0 (constants are in the kernel of the Laplacian) and K = K^T, with per-element conductivity."""
    m = mg.cube_mesh(5, jitter=0.1, seed=3, sigma0="lognormal")
    vol, grad = O.element_geometry(m.coords, m.tets)
    K = O.assemble(O.element_stiffness(m.sigma0, vol, grad), m.tets, m.n_nodes)
    scale = np.abs(K).max()
    assert np.abs(K @ np.ones(m.n_nodes)).max() < 1e-13 * scale
    assert abs(K - K.T).max() < 1e-15 * scale


def test_element_stiffness_psd_rank3():
    """Each element stiffness is symmetric positive semidefinite with a one-dimensional kernel (constants)."""
    m = mg.cube_mesh(3, jitter=0.1, seed=5)
    vol, grad = O.element_geometry(m.coords, m.tets)
    Ke = O.element_stiffness(np.ones(m.n_tets), vol, grad)
    w = np.linalg.eigvalsh(Ke)
    assert np.all(np.abs(w[:, 0]) < 1e-12 * w[:, -1])
    assert np.all(w[:, 1] > 1e-6 * w[:, -1])


def test_element_matrices_brute_force():
    """Independent route: shape functions from the 4x4 system [1 x y z] c = e_a, stiffness from their
    gradients, mass by the 4-point degree-2 tetrahedral quadrature (exact for products of linears)."""
    m = mg.cube_mesh(2, jitter=0.15, seed=9)
    vol, grad = O.element_geometry(m.coords, m.tets)
    Ke = O.element_stiffness(np.full(m.n_tets, 2.0), vol, grad)
    Me = O.element_mass(vol)
    a_, b_ = 0.5854101966249685, 0.1381966011250105
    bary = np.full((4, 4), b_) + np.eye(4) * (a_ - b_)          # quadrature points in barycentric coords
    for e in range(m.n_tets):
        X = m.coords[m.tets[e]]
        P = np.hstack([np.ones((4, 1)), X])
        C = np.linalg.solve(P, np.eye(4))                        # column a: coefficients of phi_a
        g = C[1:, :].T                                            # [4, 3]
        v = abs(np.linalg.det(X[1:] - X[0])) / 6.0
        np.testing.assert_allclose(vol[e], v, rtol=1e-13)
        np.testing.assert_allclose(Ke[e], 2.0 * v * g @ g.T, rtol=1e-11, atol=1e-12 * np.abs(Ke[e]).max())
        pts = bary @ X                                            # physical quadrature points
        phi = np.hstack([np.ones((4, 1)), pts]) @ C               # phi[q, a]
        Mq = v / 4.0 * phi.T @ phi
        np.testing.assert_allclose(Me[e], Mq, rtol=1e-12)


def test_mass_matrix_totals():
    """sum(M) equals the cube volume (80 mm)^3 and M 1 equals each node's share sum_e vol_e / 4."""
    m = mg.cube_mesh(5, jitter=0.1, seed=2)
    vol, _ = O.element_geometry(m.coords, m.tets)
    M = O.assemble(O.element_mass(vol), m.tets, m.n_nodes)
    np.testing.assert_allclose(M.sum(), 0.08 ** 3, rtol=1e-13)
    share = np.zeros(m.n_nodes)
    np.add.at(share, m.tets.ravel(), np.repeat(vol / 4.0, 4))
    np.testing.assert_allclose(M @ np.ones(m.n_nodes), share, rtol=1e-13)


def test_sigma_uses_element_mean_temperature():
    """For a linear temperature field the element mean equals the field at the centroid, so
    sigma_e = sigma0_e (1 + alpha (T(centroid) - 37)) exactly; a uniform +10 degC raises K by 15%."""
    m = mg.cube_mesh(4, jitter=0.1, seed=4, sigma0="lognormal")
    x, y, z = m.coords.T
    T = 37.0 + 100.0 * x + 50.0 * y - 80.0 * z
    cen = m.coords[m.tets].mean(axis=1)
    Tc = 37.0 + 100.0 * cen[:, 0] + 50.0 * cen[:, 1] - 80.0 * cen[:, 2]
    np.testing.assert_allclose(O.sigma_of_T(m.sigma0, T, m.tets, 0.015), m.sigma0 * (1 + 0.015 * (Tc - 37.0)),
                               rtol=1e-14)
    model = O.Model(m)
    A37, _ = model.system_V(np.full(m.n_nodes, 37.0))
    A47, _ = model.system_V(np.full(m.n_nodes, 47.0))
    free = ~m.bc_V.astype(bool)
    rows = np.repeat(np.arange(m.n_nodes), np.diff(A37.indptr))
    sel = free[rows] & free[A37.indices]
    np.testing.assert_allclose(A47.data[sel], 1.15 * A37.data[sel], rtol=1e-13)


def test_joule_uniform_field():
    """A potential linear in x (E = V0 / 2L) gives Q_e = sigma E^2 on every element, exactly."""
    m = mg.cube_mesh(4, jitter=0.12, seed=6)
    V0 = 10.0
    V = V0 * (m.coords[:, 0] + L) / (2 * L)
    _, grad = O.element_geometry(m.coords, m.tets)
    Q = O.joule(np.full(m.n_tets, 0.333), V, m.tets, grad)
    np.testing.assert_allclose(Q, 0.333 * (V0 / (2 * L)) ** 2, rtol=1e-12)


def test_joule_power_balance():
    """Total Joule power sum_e Q_e vol_e equals V^T K V, and for the discrete solution it equals the
    electrode voltage times the net current sum_{i in electrode} (K V)_i (outer faces are at 0 V)."""
    m = mg.cube_mesh(6, jitter=0.1, seed=8, sigma0="lognormal")
    model = O.Model(m)
    T0 = np.full(m.n_nodes, 37.0)
    A, b = model.system_V(T0)
    V = O.solve(A, b)
    sig = model.sigma(T0)
    Q = O.joule(sig, V, model.tets, model.grad)
    P = np.sum(Q * model.vol)
    K = O.assemble(O.element_stiffness(sig, model.vol, model.grad), m.tets, m.n_nodes)
    np.testing.assert_allclose(P, V @ (K @ V), rtol=1e-12)
    el = m.electrode.astype(bool) & ~m.bc_T.astype(bool)
    I_el = (K @ V)[m.electrode.astype(bool)]
    np.testing.assert_allclose(P, m.V_electrode * I_el.sum(), rtol=1e-9)
    assert el.sum() > 0
    F = O.load_vector(Q, model.vol, m.tets, m.n_nodes)
    np.testing.assert_allclose(F.sum(), P, rtol=1e-13)


def test_uniform_temperature_decay_closed_form():
    """All-Neumann thermal problem, no source, uniform T^n: the step gives
    T^{n+1} = ((rho_c/dt) T^n + perf T_a) / (rho_c/dt + perf) at every node (K 1 = 0; M preserves constants)."""
    m = mg.cube_mesh(4, jitter=0.1, seed=12)
    m = dataclasses.replace(m, bc_T=np.zeros(m.n_nodes, np.uint8))
    for dt in (1.0, 30.0):
        p = O.Params(dt=dt)
        model = O.Model(m, p)
        A, b = model.system_T(np.full(m.n_nodes, 50.0), np.zeros(m.n_tets))
        T1 = O.solve(A, b)
        expect = (p.rho_c / dt * 50.0 + p.perf * p.T_a) / (p.rho_c / dt + p.perf)
        np.testing.assert_allclose(T1, expect, rtol=1e-12)


def test_body_temperature_is_a_fixed_point():
    """With the electrode at 0 V there is no heating; T = 37 everywhere stays 37 through full steps
    (checks the sign of the perfusion term against T_a = 37 and the lifted outer faces)."""
    m = dataclasses.replace(mg.cube_mesh(5, jitter=0.1, seed=13), V_electrode=0.0)
    m = dataclasses.replace(m, g_V=np.zeros(m.n_nodes))
    model = O.Model(m)
    T = np.full(m.n_nodes, 37.0)
    for _ in range(2):
        T, V, _ = model.step(T)
    np.testing.assert_allclose(T, 37.0, rtol=0, atol=1e-11)
    assert np.abs(V).max() == 0.0


def test_slab_steady_joule_quadratic_exact():
    """1-D reduction through the full step: plates at 0 and V0 on the x faces give uniform Q = sigma E^2;
    with perfusion off and dt -> infinity the temperature solves -k T'' = Q, T(+-L) = 37, whose P1 nodal
    values on the unjittered Kuhn slab are exactly 37 + Q/(2k) (L^2 - x^2)."""
    n, V0 = 8, 10.0
    m = _slab_mesh(n, V0=V0)
    model = O.Model(m, O.Params(dt=1e18, perf=0.0))
    T, V, _ = model.step(np.full(m.n_nodes, 37.0))
    x = m.coords[:, 0]
    np.testing.assert_allclose(V, V0 * (x + L) / (2 * L), rtol=0, atol=1e-12 * V0)
    Q = 0.333 * (V0 / (2 * L)) ** 2
    Tex = 37.0 + Q / (2 * 0.512) * (L * L - x * x)
    np.testing.assert_allclose(T, Tex, rtol=0, atol=1e-11 * (Tex.max() - 37.0) + 1e-12)


def test_slab_bioheat_perfusion_converges_second_order():
    """Steady -k T'' + perf (T - T_a) = 0 on the slab, T(+-L) = 47: the exact solution is
    T_a + 10 cosh(m x) / cosh(m L), m = sqrt(perf / k); P1 nodal errors fall by ~4x per halving of h."""
    k, perf = 0.512, 2.4e4 / 64.0
    mm = np.sqrt(perf / k)
    errs = []
    for n in (6, 12, 24):
        m = _slab_mesh(n, V0=0.0, T_D=47.0)
        model = O.Model(m, O.Params(dt=1e18, perf=perf))
        T, _, _ = model.step(np.full(m.n_nodes, 37.0))
        x = m.coords[:, 0]
        Tex = 37.0 + 10.0 * np.cosh(mm * x) / np.cosh(mm * L)
        errs.append(np.abs(T - Tex).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.8 < r2 < 4.3, (errs, r1, r2)


def test_lift_equals_reduced_system():
    """The symmetrically lifted full system has the same solution as the reduced free-node system
    A_ff x_f = -A_fD g_D, and stays symmetric."""
    m = mg.cube_mesh(5, jitter=0.1, seed=14, sigma0="lognormal")
    model = O.Model(m)
    T = 37.0 + np.linspace(0, 5, m.n_nodes)
    A, b = model.system_V(T)
    x = O.solve(A, b)
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()
    K = O.assemble(O.element_stiffness(model.sigma(T), model.vol, model.grad), m.tets, m.n_nodes).toarray()
    D = m.bc_V.astype(bool)
    f = ~D
    xf = np.linalg.solve(K[np.ix_(f, f)], -K[np.ix_(f, D)] @ m.g_V[D])
    np.testing.assert_allclose(x[f], xf, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(x[D], m.g_V[D])


def test_sparse_lu_matches_dense_lu():
    """Above the dense limit the oracle uses SuperLU; on a 16^3 system it agrees with dense LU and leaves a
    residual below 1e-13 ||b||."""
    m = mg.cube_mesh(16, jitter=0.1, seed=15)
    assert m.n_nodes > O.DENSE_LIMIT
    model = O.Model(m)
    A, b = model.system_V(np.full(m.n_nodes, 37.0))
    xs = O.solve(A, b)
    xd = np.linalg.solve(A.toarray(), b)
    np.testing.assert_allclose(xs, xd, rtol=0, atol=1e-12 * np.abs(xd).max())
    assert np.linalg.norm(A @ xs - b) <= 1e-13 * np.linalg.norm(b)


def test_psnr_noise_calibration():
    """Sec. IV control lines: adding noise of magnitude d (random sign) at every node gives MSE = d^2, so
    PSNR = 20 log10(MAX / d) exactly; identical fields give +inf."""
    rng = np.random.default_rng(0)
    A = 37.0 + 60.0 * rng.random((5, 1000))
    # adding 1e-12 to values near 100 is exact only to half an ulp (7e-15), i.e. within 0.07 dB
    for d, tol_db in ((1e-5, 1e-6), (1e-12, 0.07)):
        B = A + d * rng.choice([-1.0, 1.0], size=A.shape)
        np.testing.assert_allclose(O.psnr(A, B), 20 * np.log10(A.max() / d), rtol=0, atol=tol_db)
    assert np.all(np.isinf(O.psnr(A, A)))


def test_corrector_converges_to_fixed_point():
    """With fixed-point passes on, the returned pair satisfies the step equations with sigma evaluated at
    the returned temperature (to the corrector tolerance), unlike the lagged single pass."""
    m = mg.cube_mesh(6, jitter=0.1, seed=16)
    p = O.Params(dt=60.0, n_corrector=50, corrector_tol=1e-10)
    model = O.Model(m, p)
    T0 = np.full(m.n_nodes, 37.0)
    T1, V1, passes = model.step(T0)
    assert 1 < passes < 50
    A, b = model.system_V(T1)
    np.testing.assert_allclose(A @ V1, b, rtol=0, atol=1e-8 * np.abs(b).max())
    lag = O.Model(m, dataclasses.replace(p, n_corrector=1))
    T1l, _, _ = lag.step(T0)
    assert np.abs(T1l - T1).max() > 1e-6


# ---- ILU(0) ------------------------------------------------------------------------------------------------

def _potential_system(n=5, seed=3):
    m = mg.cube_mesh(n, jitter=0.1, seed=seed, sigma0="lognormal")
    A, _ = O.Model(m).system_V(np.full(m.n_nodes, 45.0))
    return A


def test_ilu0_product_matches_matrix_on_pattern():
    """Defining property of ILU(0): with L unit lower and U upper on the pattern of A, (L U)_ij = a_ij for every
    stored (i, j); the product differs from A only outside the pattern (the dropped fill), and that fill is not
    zero for a 3-D stencil (so the test would notice a factorisation that silently kept it)."""
    A = _potential_system()
    L, U = O.ilu0_split(O.ilu0(A))
    P = (L @ U).toarray()
    Ad = A.toarray()
    patt = sp.csr_matrix((np.ones_like(A.data), A.indices, A.indptr), shape=A.shape).toarray() > 0
    assert np.abs(P - Ad)[patt].max() <= 1e-14 * np.abs(Ad).max()
    assert np.abs(P[~patt]).max() > 1e-6 * np.abs(Ad).max()


def test_ilu0_is_exact_lu_without_fill():
    """A tridiagonal matrix has no fill, so ILU(0) is its exact LU: L U = A everywhere, and L, U equal the
    Doolittle factors of the dense matrix (no pivoting for a diagonally dominant matrix)."""
    import scipy.linalg as sla
    rng = np.random.default_rng(4)
    n = 40
    off = rng.uniform(-1.0, 1.0, n - 1)
    A = sp.diags([off, 4.0 + rng.random(n), rng.uniform(-1.0, 1.0, n - 1)], [-1, 0, 1], format="csr")
    L, U = O.ilu0_split(O.ilu0(A))
    Pm, Ld, Ud = sla.lu(A.toarray())
    assert np.array_equal(Pm, np.eye(n))
    np.testing.assert_allclose(L.toarray(), Ld, rtol=0, atol=1e-14)
    np.testing.assert_allclose(U.toarray(), Ud, rtol=0, atol=1e-13)


def test_ilu0_apply_inverts_the_factors():
    """z = ilu0_apply(F, r) solves (L U) z = r."""
    A = _potential_system(4, 8)
    F = O.ilu0(A)
    L, U = O.ilu0_split(F)
    r = np.random.default_rng(5).normal(size=A.shape[0])
    z = O.ilu0_apply(F, r)
    np.testing.assert_allclose((L @ (U @ z)), r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_ilu_orderings_are_valid_level_orders():
    """Greedy colours and level-modulo colours are proper colourings (no two neighbours share one): 8 greedy
    colours and 4 = 1 + the largest level gap (offsets of the Kuhn stencil sum to 1, 2 or 3) on the Kuhn
    lattice, the fewest possible since every tetrahedron is a 4-clique. Dependency levels: every stored lower
    neighbour of a row lies on an earlier level (3 n + 1 levels on an (n+1)^3 lattice). After the permutation
    the levels are contiguous and non-decreasing."""
    n = 5
    A = _potential_system(n)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    offd = rows != A.indices
    for col, count in ((O.greedy_node_colors(A), 8), (O.level_modulo_colors(A), 4)):
        assert np.all(col[rows[offd]] != col[A.indices[offd]])
        assert col.max() + 1 == count
    _, lv = O.ilu_permutation(A, "multicolor")
    assert lv.max() + 1 == 4
    lev = O.dependency_levels(A)
    low = A.indices < rows
    assert np.all(lev[A.indices[low]] < lev[rows[low]])
    assert lev.max() + 1 == 3 * n + 1
    for order in ("multicolor", "natural"):
        perm, lv = O.ilu_permutation(A, order)
        assert np.array_equal(np.sort(perm), np.arange(A.shape[0]))
        assert np.all(np.diff(lv) >= 0)


def test_ilu0_natural_level_sort_is_a_relabelling():
    """Sorting rows by dependency level keeps the relative order of every pair of neighbours, so the ILU(0) of the
    level-sorted matrix is the level-sorted ILU(0) of the original: P F(A) P^T = F(P A P^T) (to rounding)."""
    A = _potential_system(4, 9)
    perm, _ = O.ilu_permutation(A, "natural")
    F1 = O.permute_symmetric(O.ilu0(A), perm)
    F2 = O.ilu0(O.permute_symmetric(A, perm))
    np.testing.assert_array_equal(F1.indices, F2.indices)
    np.testing.assert_allclose(F1.data, F2.data, rtol=1e-13, atol=1e-14 * np.abs(F1.data).max())


def test_row_lift_same_solution_nonsymmetric_system():
    """The row-only lift keeps the Dirichlet columns: the matrix is nonsymmetric (Dirichlet nodes have free
    neighbours), its Dirichlet rows are identity rows, its free rows equal the unlifted rows, and its solution
    equals the symmetric lift's (to 1e-12), for the potential and the thermal system."""
    m = mg.cube_mesh(6, jitter=0.1, seed=12, sigma0="lognormal")
    T = 37.0 + 10.0 * np.random.default_rng(2).random(m.n_nodes)
    T = np.where(m.bc_T.astype(bool), m.g_T, T)
    sym = O.Model(m)
    row = O.Model(m, O.Params(lift="row"))
    for which in ("V", "T"):
        if which == "V":
            (As, bs), (Ar, br) = sym.system_V(T), row.system_V(T)
            bc = m.bc_V.astype(bool)
            K = O.assemble(O.element_stiffness(sym.sigma(T), sym.vol, sym.grad), m.tets, m.n_nodes)
        else:
            Q = np.full(m.n_tets, 1e5)
            (As, bs), (Ar, br) = sym.system_T(T, Q), row.system_T(T, Q)
            bc = m.bc_T.astype(bool)
            K = sym.A_T
        assert abs(Ar - Ar.T).max() > 1e-6 * abs(Ar).max()
        Ad = Ar.toarray()
        np.testing.assert_array_equal(Ad[bc], np.eye(m.n_nodes)[bc])
        np.testing.assert_allclose(Ad[~bc], K.toarray()[~bc], rtol=0, atol=1e-15 * abs(K).max())
        xs, xr = O.solve(As, bs), O.solve(Ar, br)
        np.testing.assert_allclose(xr, xs, rtol=0, atol=1e-12 * np.abs(xs).max())


def test_adaptive_time_stepping_rules():
    """Dynamic step size (Sec. II-A, Sec. IV): with enough corrector passes and a duration that is a whole number
    of steps, advance() equals the fixed-step loop exactly; with too few passes it rejects steps and halves the
    size (every rejection halves, accepted sizes never grow, the last step is shortened), the accepted sizes add
    up to the duration, and every accepted step converged."""
    m = mg.cube_mesh(6, jitter=0.1, seed=71, sigma0="lognormal", V_electrode=40.0)
    full = O.Model(m, O.Params(dt=30.0, n_corrector=50, corrector_tol=1e-6))
    T, _, log = O.advance(full, 90.0, dt_min=1.0)
    Tf = np.full(m.n_nodes, 37.0)
    for _ in range(3):
        Tf, _, _ = full.step(Tf)
    np.testing.assert_array_equal(T, Tf)
    assert [e[3] for e in log] == [True] * 3
    few = O.Model(m, O.Params(dt=60.0, n_corrector=8, corrector_tol=1e-6))
    T, _, log = O.advance(few, 100.0, dt_min=1.0)
    acc = [e for e in log if e[3]]
    rej = [e for e in log if not e[3]]
    assert rej and all(not e[2] for e in rej) and all(e[2] for e in acc)
    assert abs(sum(e[0] for e in acc) - 100.0) <= 1e-9
    for a, b in zip(log, log[1:]):
        if not a[3]:
            assert b[0] == min(a[0] * 0.5, b[0]) or b[0] == a[0] * 0.5
    sizes = [e[0] for e in acc]
    assert all(x >= y for x, y in zip(sizes[:-2], sizes[1:-1]))


def test_rcm_order_is_a_bandwidth_reducing_permutation():
    """The oracle's reverse Cuthill-McKee order is a permutation; on a shuffled lattice mesh it brings the
    bandwidth from ~N back below the lattice numbering's, equal to within 10% of scipy's reverse_cuthill_mckee."""
    import scipy.sparse.csgraph as cg
    m = mg.cube_mesh(7, jitter=0.1, seed=3)
    ms, _ = mg.shuffled_nodes(m, 5)
    A = O.Model(ms).system_V(np.full(ms.n_nodes, 37.0))[0]
    p = O.rcm_order(A)
    assert np.array_equal(np.sort(p), np.arange(ms.n_nodes))
    bw = O.bandwidth(O.permute_symmetric(A, p))
    ref = O.bandwidth(O.permute_symmetric(A, cg.reverse_cuthill_mckee(A.tocsr(), symmetric_mode=True)))
    nat = O.bandwidth(O.Model(m).system_V(np.full(m.n_nodes, 37.0))[0])
    assert O.bandwidth(A) > 4 * nat and bw <= nat and bw <= 1.1 * ref


def test_coupled_jacobian_matches_central_differences_and_newton_reaches_the_fixed_point():
    """The monolithic step's Jacobian (element derivatives of K(sigma(T)) V and of the Joule source) equals central
    differences of its residual (relative 1e-6, 250 columns); Newton's method converges quadratically (each
    correction at most ~(previous)^2 x const once close) to the corrector's fixed point (to 1e-12 degC)."""
    m = mg.cube_mesh(4, jitter=0.1, seed=5, sigma0="lognormal", V_electrode=40.0)
    model = O.Model(m, O.Params(dt=30.0, n_corrector=50, corrector_tol=1e-12))
    N = model.N
    rng = np.random.default_rng(0)
    T_old = np.where(m.bc_T.astype(bool), m.g_T, 37 + 5 * rng.random(N))
    V = np.where(m.bc_V.astype(bool), m.g_V, 20 * rng.random(N))
    T = np.where(m.bc_T.astype(bool), m.g_T, 40 + 10 * rng.random(N))
    J = O.coupled_jacobian(model, V, T).toarray()
    x = np.empty(2 * N)
    x[0::2], x[1::2] = V, T
    h = 1e-6
    for k in range(2 * N):
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        col = (O.coupled_residual(model, xp[0::2], xp[1::2], T_old) -
               O.coupled_residual(model, xm[0::2], xm[1::2], T_old)) / (2 * h)
        assert np.abs(J[:, k] - col).max() <= 1e-6 * np.abs(J).max()
    Tn, Vn, it, hist = O.step_newton(model, T_old)
    Tp, Vp, _ = model.step(T_old)
    assert it <= 8
    np.testing.assert_allclose(Tn, Tp, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Vn, Vp, rtol=0, atol=1e-12 * np.abs(Vp).max())
    for a, b in zip(hist[1:-1], hist[2:]):
        if a < 1e-2:
            assert b <= 10.0 * a * a


def _projection_case(seed=0):
    m = mg.cube_mesh(6, jitter=0.1, seed=5, sigma0="lognormal")
    model = O.Model(m)
    rng = np.random.default_rng(seed)
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 10.0 * rng.random(m.n_nodes))
    A, b = model.system_V(T)
    free = ~m.bc_V.astype(bool)
    xs = O.solve(A, b)
    return m, A, b, free, xs, rng


def _a_err(A, free, x, xs):
    e = (x - xs)[free]
    return float(e @ (sp.csr_matrix(A)[free][:, free] @ e))


def test_projection_guess_exact_when_the_solution_is_in_the_span():
    """With the exact solution among the columns, the projection returns it (the other columns get no weight)."""
    m, A, b, free, xs, rng = _projection_case()
    other = np.where(free, rng.standard_normal(m.n_nodes), xs)
    for X in (np.stack([xs, other], axis=1), np.stack([xs, 0.5 * xs + other, other - xs], axis=1)):
        np.testing.assert_allclose(O.projection_guess(A, b, X, free), xs, rtol=0, atol=1e-12 * np.abs(xs).max())


def test_projection_guess_minimises_the_energy_error():
    """Brute force: no other combination of the columns is closer to the solution in the A-norm, and a single
    column gives the closed form x = (x1^T b / x1^T A x1) x1 on the free rows."""
    m, A, b, free, xs, rng = _projection_case(1)
    X = np.stack([np.where(free, xs + 0.05 * rng.standard_normal(m.n_nodes) * np.abs(xs).max(), xs)
                  for _ in range(3)], axis=1)
    x0 = O.projection_guess(A, b, X, free)
    e0 = _a_err(A, free, x0, xs)
    c0 = np.linalg.lstsq(X[free], x0[free], rcond=None)[0]
    for _ in range(300):
        c = c0 + 1e-3 * rng.standard_normal(3) * np.abs(c0).max()
        assert _a_err(A, free, np.where(free, X @ c, xs), xs) >= e0
    x1 = X[:, :1]
    Aff = sp.csr_matrix(A)[free][:, free]
    alpha = (x1[free, 0] @ b[free]) / (x1[free, 0] @ (Aff @ x1[free, 0]))
    np.testing.assert_allclose(O.projection_guess(A, b, x1, free)[free], alpha * x1[free, 0], rtol=1e-12)


def test_projection_guess_depends_only_on_the_span():
    """Raw past solutions and their backward differences (the same span) give the same guess on the free rows."""
    m, A, b, free, xs, rng = _projection_case(2)
    X = np.stack([np.where(free, xs * (1.0 + 0.02 * j) + 0.01 * rng.standard_normal(m.n_nodes), xs)
                  for j in range(4)], axis=1)
    D = np.stack([X[:, 0], X[:, 0] - X[:, 1], X[:, 0] - 2 * X[:, 1] + X[:, 2],
                  X[:, 0] - 3 * X[:, 1] + 3 * X[:, 2] - X[:, 3]], axis=1)
    np.testing.assert_allclose(O.projection_guess(A, b, D, free)[free], O.projection_guess(A, b, X, free)[free],
                               rtol=0, atol=1e-11 * np.abs(xs).max())


def test_pcg_finite_termination_and_preconditioning():
    """The oracle's PCG: on an SPD matrix with k distinct eigenvalues CG ends in at most k iterations (the Krylov
    space then holds the solution exactly); the exact inverse as preconditioner ends in one; Jacobi on a diagonal
    matrix ends in one; and on a Poisson-like system the ILU(0) preconditioner needs fewer iterations than Jacobi,
    each reaching the direct solve."""
    import scipy.sparse as sp
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.repeat([1.0, 3.0, 7.0], 4)
    A = sp.csr_matrix(Q @ np.diag(lam) @ Q.T)
    b = rng.standard_normal(12)
    x, it = O.pcg(A, b, np.zeros(12), lambda r: r, 1e-10)
    assert it <= 3 and np.allclose(A @ x, b, atol=1e-9)
    Ainv = np.linalg.inv(A.toarray())
    _, it1 = O.pcg(A, b, np.zeros(12), lambda r: Ainv @ r, 1e-10)
    assert it1 == 1
    D = sp.diags(rng.uniform(1, 5, 20)).tocsr()
    bd = rng.standard_normal(20)
    xd, itd = O.pcg(D, bd, np.zeros(20), lambda r: r / D.diagonal(), 1e-12)
    assert itd == 1 and np.allclose(xd, bd / D.diagonal())
    m = mg.cube_mesh(8, jitter=0.1, seed=12, sigma0="lognormal")
    AV, bV = O.Model(m).system_V(np.full(m.n_nodes, 37.0))
    x_ref = O.solve(AV, bV)
    perm, _ = O.ilu_permutation(AV, "multicolor")
    Ap = O.permute_symmetric(AV, perm)
    F = O.ilu0(Ap)
    _, it_j = O.pcg(Ap, bV[perm], np.zeros(m.n_nodes), lambda r: r / Ap.diagonal(), 1e-10)
    xi, it_i = O.pcg(Ap, bV[perm], np.zeros(m.n_nodes), lambda r: O.ilu0_apply(F, r), 1e-10)
    assert it_i < it_j
    assert np.linalg.norm(xi - x_ref[perm]) <= 1e-7 * np.linalg.norm(x_ref)
