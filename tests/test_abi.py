"""Host-side checks (no GPU): the C-ABI library loads and exports every entry point of include/rafem.h, and
the sampled-row oracle helper agrees with the full oracle."""
import ctypes
import os

import numpy as np
import pytest

from oracle import rafem_oracle as O
from paper_2409_13036_b300 import meshgen as mg
from tests.sampled_rows import lifted_rows


@pytest.fixture(scope="module")
def built():
    from paper_2409_13036_b300 import build
    return build.build()


def test_library_exports_every_header_symbol(built):
    from paper_2409_13036_b300 import rafem
    names = rafem.header_symbols()
    assert "rafem_create" in names and "rafem_run" in names and len(names) >= 14
    L = ctypes.CDLL(built)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert rafem.lib() is not None


# The calls of the boundary named for the hot path (mesh, tissue properties, boundary conditions, time stepping,
# assemble and solve: the problem statement of Sec. II-A), each exported under its own name.
BOUNDARY_CALLS = ["rafem_create", "rafem_assemble", "rafem_solve_step", "rafem_run", "rafem_get_field",
                  "rafem_set_state", "rafem_set_params_device", "rafem_adjoint", "rafem_batch_create",
                  "rafem_batch_run", "rafem_destroy", "rafem_status_string"]


def test_boundary_calls_exported_and_bound(built):
    from paper_2409_13036_b300 import rafem
    names = rafem.header_symbols()
    L = rafem.lib()
    for n in BOUNDARY_CALLS:
        assert n in names, n
        assert hasattr(L, n), n
    # every declared entry point has a ctypes signature in the binding (marshalling is typed, not guessed)
    unbound = [n for n in names if getattr(L, n).argtypes is None and n != "rafem_status_string"]
    assert not unbound, unbound


def test_status_strings(built):
    from paper_2409_13036_b300 import rafem
    assert rafem.status_string(0) == "OK"
    assert rafem.status_string(-5) == "ERR_TIMEOUT"
    p = rafem.default_params()
    assert p.tol == 1e-10 and p.alpha_sigma == 0.015 and p.n_corrector == 1


def test_sampled_rows_helper_matches_full_oracle():
    m = mg.cube_mesh(6, jitter=0.1, seed=3, sigma0="lognormal")
    rng = np.random.default_rng(0)
    T = 37 + 10 * rng.random(m.n_nodes)
    V = 20 * rng.random(m.n_nodes)
    model = O.Model(m)
    rows = rng.choice(m.n_nodes, 60, replace=False)
    for which in ("V", "T"):
        if which == "V":
            A, b = model.system_V(T)
            r, ref, bs = lifted_rows(m, rows, T, which="V")
        else:
            A, b = model.system_T(T, O.joule(model.sigma(T), V, model.tets, model.grad))
            r, ref, bs = lifted_rows(m, rows, T, which="T", V=V, T_old=T)
        np.testing.assert_allclose(bs, b[r], rtol=1e-12, atol=1e-14 * np.abs(b).max())
        for i in r:
            lo, hi = A.indptr[i], A.indptr[i + 1]
            got = np.array([ref[i][c] for c in A.indices[lo:hi]])
            np.testing.assert_allclose(got, A.data[lo:hi], rtol=1e-12, atol=1e-14 * np.abs(A.data).max())


def test_coupled_rows_helper_matches_full_oracle():
    """The sub-mesh rows of the monolithic system (tests/sampled_rows.coupled_rows) equal the rows of the oracle's
    coupled_jacobian and coupled_residual on the whole mesh, Dirichlet rows of both fields included."""
    from tests.sampled_rows import coupled_rows
    m = mg.cube_mesh(7, jitter=0.1, seed=85, sigma0="lognormal", V_electrode=30.0)
    rng = np.random.default_rng(2)
    V = np.where(m.bc_V.astype(bool), m.g_V, 15.0 * rng.random(m.n_nodes))
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 10.0 * rng.random(m.n_nodes))
    model = O.Model(m)
    J = O.coupled_jacobian(model, V, T).tocsr()
    R = O.coupled_residual(model, V, T, T)
    rows = np.concatenate([rng.choice(m.n_nodes, 40, replace=False), np.flatnonzero(m.bc_V)[:3],
                           np.flatnonzero(m.bc_T)[:3], [m.n_nodes - 1]])
    r, ref, res = coupled_rows(m, rows, V, T)
    for i in r:
        full = {}
        for a in range(2):
            lo, hi = J.indptr[2 * i + a], J.indptr[2 * i + a + 1]
            full.update({(a, int(c // 2), int(c % 2)): v for c, v in zip(J.indices[lo:hi], J.data[lo:hi])})
        assert set(full) == set(ref[int(i)])
        for k, v in full.items():
            assert abs(ref[int(i)][k] - v) <= 1e-13 * abs(v) + 1e-15
        assert res[int(i)] == pytest.approx((R[2 * i], R[2 * i + 1]), rel=1e-13, abs=1e-12 * np.abs(R).max())


def test_mesh_generator_counts():
    for n, N, E, el in ((8, 729, 3072, 3), (48, 117649, 663552, 13)):
        m = mg.cube_mesh(n, jitter=0.1, seed=1)
        assert (m.n_nodes, m.n_tets, int(m.electrode.sum())) == (N, E, el)
    m = mg.cube_mesh(127, jitter=0.0)
    assert int(m.electrode.sum()) == 16 * 32


def test_reorder_rcm_matches_oracle():
    """rafem_reorder_rcm (host-only entry point) returns the oracle's reverse Cuthill-McKee order bit for bit, on
    a shuffled jittered cube and on a mesh of two disconnected cubes."""
    import dataclasses
    import numpy as np
    from oracle import rafem_oracle as O
    from paper_2409_13036_b300 import meshgen as mg, rafem
    a, _ = mg.shuffled_nodes(mg.cube_mesh(6, jitter=0.1, seed=3), 9)
    b, _ = mg.shuffled_nodes(mg.cube_mesh(4, jitter=0.1, seed=4), 10)
    two = dataclasses.replace(
        a, coords=np.vstack([a.coords, b.coords + 1.0]), tets=np.vstack([a.tets, b.tets + a.n_nodes]).astype(np.int32),
        lattice=np.vstack([a.lattice, b.lattice]), bc_V=np.concatenate([a.bc_V, b.bc_V]),
        g_V=np.concatenate([a.g_V, b.g_V]), bc_T=np.concatenate([a.bc_T, b.bc_T]), g_T=np.concatenate([a.g_T, b.g_T]),
        sigma0=np.concatenate([a.sigma0, b.sigma0]), k=np.concatenate([a.k, b.k]),
        electrode=np.concatenate([a.electrode, b.electrode]))
    for m in (a, two):
        A = O.Model(m).system_V(np.full(m.n_nodes, 37.0))[0]
        np.testing.assert_array_equal(rafem.reorder_rcm(m), O.rcm_order(A))
