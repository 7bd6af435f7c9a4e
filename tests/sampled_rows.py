"""Oracle values for a subset of rows of the lifted systems, for checks at sizes where a full oracle solve is
out of reach. Uses only oracle functions, applied to the elements that touch the sampled rows (which is all
that the rows' entries depend on)."""
import numpy as np

from oracle import rafem_oracle as O


def elements_touching(tets, rows):
    mask = np.zeros(int(tets.max()) + 1, dtype=bool)
    mask[rows] = True
    return np.nonzero(mask[tets].any(axis=1))[0]


def lifted_rows(mesh, rows, T, *, which, V=None, T_old=None, params=None):
    """Dense {row: {col: value}} of the lifted matrix and the lifted rhs entries for the sampled rows.

    which = "V": A_V(sigma(T)) with its lifted rhs; which = "T": the thermal matrix and rhs built from V, T
    (sigma) and T_old (mass term)."""
    p = params or O.Params()
    rows = np.unique(np.asarray(rows, dtype=np.int64))
    N = mesh.coords.shape[0]
    els = elements_touching(mesh.tets, rows)
    tets = np.asarray(mesh.tets, dtype=np.int64)[els]
    vol, grad = O.element_geometry(mesh.coords, tets)
    if which == "V":
        sig = O.sigma_of_T(mesh.sigma0[els], T, tets, p.alpha_sigma)
        Ke = O.element_stiffness(sig, vol, grad)
        bc, g = mesh.bc_V.astype(bool), np.asarray(mesh.g_V, dtype=np.float64)
        src = np.zeros(N)
    else:
        Ke = (O.element_stiffness(mesh.k[els], vol, grad) + (p.rho_c / p.dt + p.perf) * O.element_mass(vol))
        bc, g = mesh.bc_T.astype(bool), np.asarray(mesh.g_T, dtype=np.float64)
        sig = O.sigma_of_T(mesh.sigma0[els], T, tets, p.alpha_sigma)
        Q = O.joule(sig, V, tets, grad)
        Me = O.element_mass(vol)
        src = np.zeros(N)
        # (rho_c/dt) M T_old + perf T_a M 1 + F, restricted to the sampled elements (complete for sampled rows)
        contrib = (p.rho_c / p.dt) * np.einsum("eab,eb->ea", Me, T_old[tets]) + p.perf * p.T_a * Me.sum(axis=2) \
            + (Q * vol / 4.0)[:, None]
        np.add.at(src, tets.ravel(), contrib.ravel())
    A = O.assemble(Ke, tets, N)
    A = A[rows]
    gD = np.where(bc, g, 0.0)
    b = src[rows] - A @ gD
    A = A.tocsr()
    out_rows = {}
    for k, i in enumerate(rows):
        lo, hi = A.indptr[k], A.indptr[k + 1]
        cols = A.indices[lo:hi]
        vals = A.data[lo:hi].copy()
        if bc[i]:
            vals[:] = 0.0
            vals[cols == i] = 1.0
            b[k] = g[i]
        else:
            vals[bc[cols]] = 0.0
        out_rows[int(i)] = dict(zip(cols.tolist(), vals.tolist()))
    return rows, out_rows, b


def rows_adjacent_to(mesh, nodes):
    """All nodes sharing an element with any of `nodes` (including them)."""
    els = elements_touching(mesh.tets, nodes)
    return np.unique(np.asarray(mesh.tets)[els].ravel())


def coupled_rows(mesh, rows, V, T, params=None):
    """Rows of the monolithic Newton system (the oracle's coupled_jacobian and coupled_residual with T_old = T)
    for the sampled nodes, from the oracle applied to the sub-mesh of the elements that touch them: a node's rows
    depend only on its incident elements, its own boundary flags and the fields at their vertices.
    Returns (rows, {row: {(a, col, b): value}}, {row: (R_V, R_T)}) with a, b in {0: V, 1: T}."""
    import types
    rows = np.unique(np.asarray(rows, dtype=np.int64))
    els = elements_touching(mesh.tets, rows)
    tets = np.asarray(mesh.tets, dtype=np.int64)[els]
    nodes = np.unique(tets.ravel())
    local = {int(n): k for k, n in enumerate(nodes)}
    sub = types.SimpleNamespace(
        coords=np.asarray(mesh.coords)[nodes], tets=np.searchsorted(nodes, tets),
        bc_V=np.asarray(mesh.bc_V)[nodes], g_V=np.asarray(mesh.g_V)[nodes],
        bc_T=np.asarray(mesh.bc_T)[nodes], g_T=np.asarray(mesh.g_T)[nodes],
        sigma0=np.asarray(mesh.sigma0)[els], k=np.asarray(mesh.k)[els])
    model = O.Model(sub, params or O.Params())
    Vs, Ts = np.asarray(V, dtype=np.float64)[nodes], np.asarray(T, dtype=np.float64)[nodes]
    J = O.coupled_jacobian(model, Vs, Ts).tocsr()
    R = O.coupled_residual(model, Vs, Ts, Ts)
    out, res = {}, {}
    for i in rows:
        li = local[int(i)]
        ent = {}
        for a in range(2):
            lo, hi = J.indptr[2 * li + a], J.indptr[2 * li + a + 1]
            for c, v in zip(J.indices[lo:hi], J.data[lo:hi]):
                ent[(a, int(nodes[c // 2]), int(c % 2))] = float(v)
        out[int(i)] = ent
        res[int(i)] = (float(R[2 * li]), float(R[2 * li + 1]))
    return rows, out, res
