"""Double-word (float pair) element and node passes of the gather assembly against the FP64 passes, and how
RAFEM_ARITH_AUTO resolves (needs a B300)."""
import dataclasses

import numpy as np
import pytest

from paper_2409_13036_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

# A double-word value carries 48 significant bits (unit roundoff 2^-48 = 3.6e-15); an assembled entry is a sum
# of a few products (six to eight elements per edge, each sigma0 G f), every operation adding at most a few units
# of 2^-48 of the magnitudes involved, and the FP64 passes add their own 2^-53 roundings. 64 units of 2^-48
# relative to the row's largest magnitude bounds the difference with margin (2.3e-13).
DW_REL = 64 * 2.0 ** -48


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


def _state(mesh, seed):
    rng = np.random.default_rng(seed)
    T = np.where(mesh.bc_T.astype(bool), mesh.g_T, 37.0 + 40.0 * rng.random(mesh.n_nodes))
    V = np.where(mesh.bc_V.astype(bool), mesh.g_V, 20.0 * rng.random(mesh.n_nodes))
    return T, V


def test_arith_resolution():
    rafem = R()
    m = mg.cube_mesh(6, jitter=0.1, seed=3)
    with rafem.Context(m) as ctx:
        assert ctx.layout_info()["arith"] == rafem.RAFEM_ARITH_DW
    with rafem.Context(m, arith=rafem.RAFEM_ARITH_FP64) as ctx:
        assert ctx.layout_info()["arith"] == rafem.RAFEM_ARITH_FP64
    with rafem.Context(m, assembly=rafem.RAFEM_ASSEMBLY_COLOR) as ctx:
        assert ctx.layout_info()["arith"] == rafem.RAFEM_ARITH_FP64
    with pytest.raises(rafem.RafemError):
        rafem.Context(m, assembly=rafem.RAFEM_ASSEMBLY_COLOR, arith=rafem.RAFEM_ARITH_DW)
    with pytest.raises(rafem.RafemError):
        rafem.Context(m, arith=7)
    # element volumes far below 2^-90 m^3: AUTO keeps FP64, an explicit request is refused
    tiny = dataclasses.replace(m, coords=m.coords * 1e-12)
    with rafem.Context(tiny) as ctx:
        assert ctx.layout_info()["arith"] == rafem.RAFEM_ARITH_FP64
    with pytest.raises(rafem.RafemError):
        rafem.Context(tiny, arith=rafem.RAFEM_ARITH_DW)


@pytest.mark.parametrize("precision", [0, 1])
def test_dw_systems_match_fp64(precision):
    """Both assembled systems, entry by entry, on a jittered lognormal mesh spanning many tiles, with
    non-uniform T and V (Joule heating everywhere)."""
    rafem = R()
    m = mg.cube_mesh(24, jitter=0.1, seed=5, sigma0="lognormal")
    T, V = _state(m, 1)
    out = {}
    for arith in (rafem.RAFEM_ARITH_FP64, rafem.RAFEM_ARITH_DW):
        with rafem.Context(m, arith=arith, precision=precision) as ctx:
            assert ctx.layout_info()["arith"] == arith
            ctx.set_state(T=T, V=V)
            ctx.assemble(rafem.RAFEM_SYS_V)
            ctx.assemble(rafem.RAFEM_SYS_T)
            out[arith] = (ctx.get_system(rafem.RAFEM_SYS_V), ctx.get_system(rafem.RAFEM_SYS_T))
    for k in (0, 1):
        rp, col, v64, b64 = out[rafem.RAFEM_ARITH_FP64][k]
        _, _, vdw, bdw = out[rafem.RAFEM_ARITH_DW][k]
        rows = np.repeat(np.arange(m.n_nodes), np.diff(rp))
        rowmax = np.maximum.reduceat(np.abs(v64), rp[:-1])
        err = np.abs(vdw - v64) / rowmax[rows]
        assert err.max() <= DW_REL, (k, err.max())
        assert np.abs(bdw - b64).max() <= DW_REL * np.abs(b64).max(), k


def test_dw_joule_term_alone():
    """With the mass term made negligible by a huge time step and no perfusion, the thermal rhs away from the
    Dirichlet faces is the Joule heat alone; the double-word quadratic form (edge differences) agrees with the
    FP64 one (full quadratic form)."""
    rafem = R()
    m = mg.cube_mesh(12, jitter=0.15, seed=9, sigma0="lognormal")
    T, V = _state(m, 2)
    res = {}
    for arith in (rafem.RAFEM_ARITH_FP64, rafem.RAFEM_ARITH_DW):
        with rafem.Context(m, arith=arith, dt=1e9, perf=0.0) as ctx:
            ctx.set_state(T=T, V=V)
            ctx.assemble(rafem.RAFEM_SYS_T)
            res[arith] = ctx.get_system(rafem.RAFEM_SYS_T)
    rp, col, _, b64 = res[rafem.RAFEM_ARITH_FP64]
    bdw = res[rafem.RAFEM_ARITH_DW][3]
    assert np.abs(bdw - b64).max() <= DW_REL * np.abs(b64).max()
    # rows away from the Dirichlet faces hold only element sums of nonnegative Joule heat (plus a vanishing mass
    # term): entry-wise relative agreement there
    bc = m.bc_T.astype(bool)
    interior = np.array([not bc[i] and not bc[col[rp[i]:rp[i + 1]]].any() for i in range(m.n_nodes)])
    assert interior.sum() > 100 and (b64[interior] > 0).all()
    np.testing.assert_allclose(bdw[interior], b64[interior], rtol=DW_REL)


def test_dw_run_matches_fp64_run():
    """Twenty default steps (mixed precision, projection predictor) with each arithmetic, solved tightly: the
    fields agree far inside the solver tolerance."""
    rafem = R()
    m = mg.cube_mesh(16, jitter=0.1, seed=4, sigma0="lognormal")
    fields = {}
    for arith in (rafem.RAFEM_ARITH_FP64, rafem.RAFEM_ARITH_DW):
        with rafem.Context(m, arith=arith, precision=rafem.RAFEM_PRECISION_MIXED, tol=1e-13) as ctx:
            status, _ = ctx.run(20)
            assert status == 0
            fields[arith] = (ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V))
    for k in (0, 1):
        a, b = fields[rafem.RAFEM_ARITH_FP64][k], fields[rafem.RAFEM_ARITH_DW][k]
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a), k


def test_dw_matches_fp64_on_the_48_cube_after_ten_steps():
    """The 48^3 workload (117,649 nodes, jitter 10%): ten FP64 steps with double-word element passes against ten
    with FP64 element passes, both solved to a relative residual of 1e-13. The entries differ by at most
    DW_REL (2.3e-13) of their row's magnitude and each solve leaves a residual of at most 1e-13, so the fields may
    differ by about cond(A) x (2.3e-13 + 2e-13); cond(A_V) is ~1e3 at this size (the potential system's condition
    number grows like the square of the cells per side: ~1e2 at 14^3, ~1e5 at 127^3), giving ~4e-10. The bound
    1e-9 keeps a factor 2 for the ten steps' accumulation."""
    rafem = R()
    m = mg.workload_48()
    fields = {}
    for arith in (rafem.RAFEM_ARITH_FP64, rafem.RAFEM_ARITH_DW):
        with rafem.Context(m, arith=arith, tol=1e-13) as ctx:
            assert ctx.layout_info()["arith"] == arith
            status, _ = ctx.run(10)
            assert status == 0
            fields[arith] = (ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V))
    for k in (0, 1):
        a, b = fields[rafem.RAFEM_ARITH_FP64][k], fields[rafem.RAFEM_ARITH_DW][k]
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a), (k, np.linalg.norm(a - b) / np.linalg.norm(a))
