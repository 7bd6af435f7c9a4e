"""FP64 CPU oracle of the RAFEM time step (assembly + Dirichlet lift + sparse direct solve).

TEST INFRASTRUCTURE ONLY. This module is imported by the tests, by the package's smoke check and by the
benchmark's CPU-baseline leg; the product path never calls it. It shares no code with the CUDA library: it has
its own element geometry, its own assembly (COO triplets summed into CSR by scipy), its own boundary handling
and a direct solve (numpy dense LU for small systems, SuperLU otherwise).

What it computes (Sec. II-A, main application loop): per time step, the element equations are recomputed
from updated values and assembled into a global sparse matrix that is then solved. The paper defers the PDE
to its cited formulation; the reading implemented here is the staggered electric-potential / Pennes-bioheat
pair on P1 tetrahedra, advanced by backward Euler:

    div(sigma(T) grad V) = 0,               sigma_e = sigma0_e * (1 + alpha * (mean_e(T) - 37))
    rho_c dT/dt = div(k grad T) + sigma |grad V|^2 - perf * (T - T_a)

discretised as
    K_sigma(T^n) V^{n+1} = 0                 (Dirichlet-lifted: electrode V_e, outer faces 0)
    Q_e = sigma_e |grad V^{n+1}_e|^2,         F_i = sum_e Q_e vol_e / 4
    [(rho_c/dt + perf) M + K_k] T^{n+1} = (rho_c/dt) M T^n + perf T_a M 1 + F   (lifted: outer faces 37)

with the consistent P1 mass matrix M. An optional fixed-point corrector re-evaluates sigma at the newest
temperature iterate (the corrector passes of the main loop, Sec. II-A; at most 50 passes, Sec. IV).

The PSNR quality metric follows Sec. IV, Eq. 1 and Eq. 2, read as 20*log10(MAX(A)/sqrt(MSE_i)).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DENSE_LIMIT = 3000


@dataclasses.dataclass
class Params:
    alpha_sigma: float = 0.015   # 1/degC
    rho_c: float = 3.6e6         # J/m^3/K
    perf: float = 2.4e4          # W/m^3/K
    T_a: float = 37.0            # degC
    dt: float = 1.0              # s
    n_corrector: int = 1         # fixed-point passes per step (1 = lagged coefficients)
    corrector_tol: float = 1e-6  # degC, infinity norm of the temperature change between passes


# ----------------------------------------------------------------------------------------------------------
# Element level
# ----------------------------------------------------------------------------------------------------------

def element_geometry(coords, tets):
    """Volume and gradients of the four P1 shape functions of every tetrahedron.

    With E = [x1-x0 | x2-x0 | x3-x0] (edge vectors as columns), the barycentric coordinates are
    xi = E^{-1} (x - x0), so grad(phi_a) is row a-1 of E^{-1} for a = 1..3 and grad(phi_0) = -sum of them.
    Returns vol [E] (must be > 0) and grad [E, 4, 3].
    """
    X = np.asarray(coords, dtype=np.float64)[np.asarray(tets)]
    Emat = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))      # columns are edges
    det = np.linalg.det(Emat)
    vol = det / 6.0
    if not np.all(vol > 0):
        raise ValueError("non-positive element volume")
    Einv = np.linalg.inv(Emat)                                      # rows are grad(xi_a)
    grad = np.empty((X.shape[0], 4, 3))
    grad[:, 1:, :] = Einv
    grad[:, 0, :] = -Einv.sum(axis=1)
    return vol, grad


def element_stiffness(coef, vol, grad):
    """K_e[a, b] = coef_e * vol_e * grad(phi_a) . grad(phi_b)."""
    return (np.asarray(coef, dtype=np.float64) * vol)[:, None, None] * np.einsum("eai,ebi->eab", grad, grad)


def element_mass(vol):
    """Consistent P1 mass: M_e[a, b] = vol_e / 20 * (1 + delta_ab)."""
    base = np.ones((4, 4)) + np.eye(4)
    return (vol / 20.0)[:, None, None] * base[None, :, :]


def element_mean(u, tets):
    return np.asarray(u, dtype=np.float64)[np.asarray(tets)].mean(axis=1)


def sigma_of_T(sigma0, T, tets, alpha):
    """sigma_e = sigma0_e * (1 + alpha * (Tbar_e - 37)), Tbar_e the mean of the element's 4 nodal temperatures."""
    return np.asarray(sigma0, dtype=np.float64) * (1.0 + alpha * (element_mean(T, tets) - 37.0))


def joule(sigma_e, V, tets, grad):
    """Q_e = sigma_e * |sum_a V_a grad(phi_a)|^2 (constant on each element)."""
    gV = np.einsum("ea,eai->ei", np.asarray(V, dtype=np.float64)[np.asarray(tets)], grad)
    return sigma_e * np.sum(gV * gV, axis=1)


# ----------------------------------------------------------------------------------------------------------
# Global level
# ----------------------------------------------------------------------------------------------------------

def assemble(Ke, tets, N):
    """Sum element matrices into a global CSR matrix (triplets, duplicates summed)."""
    tets = np.asarray(tets, dtype=np.int64)
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    A = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(N, N)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def load_vector(q_e, vol, tets, N):
    """F_i = sum over elements containing i of q_e * integral(phi_i) = q_e * vol_e / 4."""
    F = np.zeros(N)
    np.add.at(F, np.asarray(tets).ravel(), np.repeat(q_e * vol / 4.0, 4))
    return F


def dirichlet_lift(A, b, bc, g):
    """Symmetric Dirichlet lift: b -= A[:, D] g_D; zero rows and columns of D; unit diagonal; b_D = g_D.

    The pattern of A is kept (zeroed entries stay stored), so the result is comparable slot by slot with a
    lifted matrix stored on the fixed CSR pattern.
    """
    bc = np.asarray(bc).astype(bool)
    g = np.where(bc, np.asarray(g, dtype=np.float64), 0.0)
    b = np.asarray(b, dtype=np.float64) - A @ g
    A = A.tocsr(copy=True)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    cols = A.indices
    kill = bc[rows] | bc[cols]
    A.data[kill] = 0.0
    A.data[kill & (rows == cols)] = 1.0
    b[bc] = g[bc]
    return A, b


def solve(A, b):
    """Direct solve: dense LU with partial pivoting for N <= 3000, SuperLU (symmetric ordering) otherwise."""
    N = A.shape[0]
    if N <= DENSE_LIMIT:
        return np.linalg.solve(A.toarray(), b)
    lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
    return lu.solve(b)


class Model:
    """Mesh-constant quantities of one instance (geometry, mass and thermal stiffness)."""

    def __init__(self, mesh, params: Params | None = None):
        self.p = params or Params()
        self.coords = np.asarray(mesh.coords, dtype=np.float64)
        self.tets = np.asarray(mesh.tets, dtype=np.int64)
        self.N = self.coords.shape[0]
        self.bc_V = np.asarray(mesh.bc_V).astype(bool)
        self.g_V = np.asarray(mesh.g_V, dtype=np.float64)
        self.bc_T = np.asarray(mesh.bc_T).astype(bool)
        self.g_T = np.asarray(mesh.g_T, dtype=np.float64)
        self.sigma0 = np.asarray(mesh.sigma0, dtype=np.float64)
        self.k = np.asarray(mesh.k, dtype=np.float64)
        self.vol, self.grad = element_geometry(self.coords, self.tets)
        self.M = assemble(element_mass(self.vol), self.tets, self.N)
        self.Kk = assemble(element_stiffness(self.k, self.vol, self.grad), self.tets, self.N)
        p = self.p
        self.A_T = ((p.rho_c / p.dt + p.perf) * self.M + self.Kk).tocsr()
        self.A_T.sort_indices()

    # -- the potential system -------------------------------------------------------------------------
    def sigma(self, T):
        return sigma_of_T(self.sigma0, T, self.tets, self.p.alpha_sigma)

    def system_V(self, T):
        """Lifted (A_V, b_V) for sigma evaluated at temperature T."""
        K = assemble(element_stiffness(self.sigma(T), self.vol, self.grad), self.tets, self.N)
        return dirichlet_lift(K, np.zeros(self.N), self.bc_V, self.g_V)

    # -- the thermal system ---------------------------------------------------------------------------
    def rhs_T_unlifted(self, T_old, Q_e):
        p = self.p
        return ((p.rho_c / p.dt) * (self.M @ T_old) + p.perf * p.T_a * (self.M @ np.ones(self.N))
                + load_vector(Q_e, self.vol, self.tets, self.N))

    def system_T(self, T_old, Q_e):
        return dirichlet_lift(self.A_T, self.rhs_T_unlifted(T_old, Q_e), self.bc_T, self.g_T)

    def solve_T(self, T_old, Q_e):
        """Solve the lifted thermal system; its matrix is constant, so its factorisation is kept."""
        A, b = self.system_T(T_old, Q_e)
        if self.N <= DENSE_LIMIT:
            return np.linalg.solve(A.toarray(), b)
        if getattr(self, "_lu_T", None) is None:
            self._lu_T = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
        return self._lu_T.solve(b)

    # -- one backward-Euler step with optional fixed-point corrector -------------------------------------
    def step(self, T_old):
        p = self.p
        T_it = T_old
        passes = 0
        for passes in range(1, max(1, p.n_corrector) + 1):
            sig = self.sigma(T_it)
            A_V, b_V = self.system_V(T_it)
            V_new = solve(A_V, b_V)
            Q = joule(sig, V_new, self.tets, self.grad)
            T_new = self.solve_T(T_old, Q)
            change = float(np.max(np.abs(T_new - T_it)))
            T_it = T_new
            if p.n_corrector > 1 and change < p.corrector_tol:
                break
        return T_it, V_new, passes

    def run(self, n_steps, T0=None):
        """Returns arrays T [n_steps, N] and V [n_steps, N] after each step."""
        T = np.full(self.N, 37.0) if T0 is None else np.asarray(T0, dtype=np.float64).copy()
        Ts, Vs = [], []
        for _ in range(n_steps):
            T, V, _ = self.step(T)
            Ts.append(T)
            Vs.append(V)
        return np.array(Ts), np.array(Vs)


# ----------------------------------------------------------------------------------------------------------
# Quality metrics (Sec. IV)
# ----------------------------------------------------------------------------------------------------------

def psnr(A_steps, B_steps):
    """PSNR per step (Eq. 1 with the MSE of Eq. 2): 20*log10(MAX(A) / sqrt(MSE_i)).

    A_steps is the reference field [steps, n], B_steps the field under test. MAX(A) is the largest value of
    the reference over all steps and nodes. A step with MSE = 0 gives +inf.
    """
    A = np.atleast_2d(np.asarray(A_steps, dtype=np.float64))
    B = np.atleast_2d(np.asarray(B_steps, dtype=np.float64))
    mse = np.mean((A - B) ** 2, axis=1)
    peak = float(A.max())
    with np.errstate(divide="ignore"):
        return 20.0 * np.log10(peak / np.sqrt(mse))


def rel_err(x, x_ref):
    """||x - x_ref||_2 / ||x_ref||_2."""
    x_ref = np.asarray(x_ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(x, dtype=np.float64) - x_ref) / np.linalg.norm(x_ref))
