"""The allocation-free solve (rafem_pcg_csr_noalloc) against the context-based solve (rafem_solve_rhs).

rafem_pcg_csr_noalloc is for callers that cannot call cudaMalloc when they need a solve, for example code inside a
framework whose caching allocator already owns the device memory, or a loop that cannot absorb the device-wide
synchronisation of cudaMalloc/cudaFree. It works out of one fixed scratch array inside the library. This test
builds a potential system with a context, passes a device copy of its CSR matrix to the allocation-free entry
point twice in a row (the second call starts from whatever the first left in the shared scratch array) and checks
both solutions against the context's own solve, within the 1e-9 relative tolerance the FP64 parity tests use. It
also checks that a system larger than the scratch array holds is refused, that malformed CSR input (a row without
its diagonal, a column index out of range) is refused with x left untouched, and that a solve on a stream other
than the default one gives the same solution.
"""
import numpy as np
import pytest

from paper_2409_13036_b300 import meshgen as mg

pytestmark = pytest.mark.gpu


def test_noalloc_pcg_matches_context_solve_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2409_13036_b300 import build
    build.build()
    from paper_2409_13036_b300 import rafem

    m = mg.cube_mesh(40, jitter=0.1, seed=51, sigma0="lognormal")   # 68,921 rows
    N = m.n_nodes
    assert N <= 131072  # RAFEM_NOALLOC_MAX_ROWS
    rng = np.random.default_rng(5)
    T = np.where(m.bc_T.astype(bool), m.g_T, 37.0 + 20.0 * rng.random(N))
    with rafem.Context(m, tol=1e-12) as ctx:
        ctx.set_state(T=T)
        ctx.assemble(rafem.RAFEM_SYS_V)
        rp, col, vals, rhs = ctx.get_system(rafem.RAFEM_SYS_V)
        b = torch.tensor(rhs, dtype=torch.float64, device="cuda")
        x_ref = torch.zeros(N, dtype=torch.float64, device="cuda")
        s, st = ctx.solve_rhs(rafem.RAFEM_SYS_V, b, x_ref)
        assert s == rafem.RAFEM_OK and st.relres_V <= 1e-12
    x_ref = x_ref.cpu().numpy()

    d_rp = torch.tensor(rp, dtype=torch.int32, device="cuda")
    d_col = torch.tensor(col, dtype=torch.int32, device="cuda")
    d_vals = torch.tensor(vals, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    results = []
    for _ in range(2):
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s, st = rafem.pcg_csr_noalloc(N, d_rp, d_col, d_vals, b, x, tol=1e-12, max_iter=20000)
        assert s == rafem.RAFEM_OK, rafem.status_string(s)
        assert st.relres_V <= 1e-12 and st.iters_V > 10
        xs = x.cpu().numpy()
        assert np.linalg.norm(xs - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
        results.append(xs)
    # same inputs, same fixed schedule: the second call reproduces the first exactly
    np.testing.assert_array_equal(results[0], results[1])

    too_big = 131072 + 1
    s, _ = rafem.pcg_csr_noalloc(too_big, d_rp, d_col, d_vals, b, x, tol=1e-12, max_iter=10)
    assert s == rafem.RAFEM_ERR_BAD_INPUT

    # malformed CSR input, about 100 rows: refused before any solver work, x untouched
    n = 100
    rp_s = np.arange(n + 1, dtype=np.int32) * 3
    col_s = np.stack([np.maximum(np.arange(n) - 1, 0), np.arange(n), np.minimum(np.arange(n) + 1, n - 1)],
                     axis=1).astype(np.int32).reshape(-1)
    vals_s = np.tile(np.array([-1.0, 4.0, -1.0]), n)
    b_s = torch.ones(n, dtype=torch.float64, device="cuda")
    for name, fix in (("missing diagonal", lambda c: c.__setitem__(3 * 17 + 1, 18)),
                      ("column out of range", lambda c: c.__setitem__(3 * 42 + 2, n))):
        bad_col = col_s.copy()
        fix(bad_col)
        d_rp_s = torch.tensor(rp_s, device="cuda")
        d_col_s = torch.tensor(bad_col, device="cuda")
        d_vals_s = torch.tensor(vals_s, device="cuda")
        x_s = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s, _ = rafem.pcg_csr_noalloc(n, d_rp_s, d_col_s, d_vals_s, b_s, x_s, tol=1e-12, max_iter=100)
        assert s == rafem.RAFEM_ERR_BAD_INPUT, name
        assert torch.all(x_s == 7.0).item(), name

    # a solve issued on a non-default stream gives the default stream's solution
    side = torch.cuda.Stream()
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s, st = rafem.pcg_csr_noalloc(N, d_rp, d_col, d_vals, b, x, tol=1e-12, max_iter=20000, stream=side.cuda_stream)
    assert s == rafem.RAFEM_OK, rafem.status_string(s)
    np.testing.assert_array_equal(x.cpu().numpy(), results[0])
