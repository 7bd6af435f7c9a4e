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

Beyond the paper's loop it also provides what the library's extensions are checked against: the A-norm
projection that serves as the potential's initial guess (projection_guess), the tangent-linear step and a dense
adjoint for the gradients, ILU(0), reverse Cuthill-McKee, the adaptive step rules and the coupled Newton step.
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
    lift: str = "symmetric"      # Dirichlet lift: "symmetric" (SPD systems) or "row" (nonsymmetric, same solution)
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


def dirichlet_lift_row(A, b, bc, g):
    """Row-only Dirichlet lift: rows of D become identity rows with b_D = g_D; columns are kept, so the system is
    nonsymmetric but has the same solution as the symmetric lift. The pattern of A is kept."""
    bc = np.asarray(bc).astype(bool)
    g = np.where(bc, np.asarray(g, dtype=np.float64), 0.0)
    b = np.asarray(b, dtype=np.float64).copy()
    A = A.tocsr(copy=True)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    kill = bc[rows]
    A.data[kill] = 0.0
    A.data[kill & (rows == A.indices)] = 1.0
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
        return self._lift(K, np.zeros(self.N), self.bc_V, self.g_V)

    def _lift(self, A, b, bc, g):
        return (dirichlet_lift_row if self.p.lift == "row" else dirichlet_lift)(A, b, bc, g)

    # -- the thermal system ---------------------------------------------------------------------------
    def rhs_T_unlifted(self, T_old, Q_e):
        p = self.p
        return ((p.rho_c / p.dt) * (self.M @ T_old) + p.perf * p.T_a * (self.M @ np.ones(self.N))
                + load_vector(Q_e, self.vol, self.tets, self.N))

    def system_T(self, T_old, Q_e):
        return self._lift(self.A_T, self.rhs_T_unlifted(T_old, Q_e), self.bc_T, self.g_T)

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
        T, V, passes, _ = self.step_detail(T_old)
        return T, V, passes

    def step_detail(self, T_old):
        """One step; returns (T, V, passes, converged). With n_corrector > 1 the corrector passes (sigma at the
        newest temperature iterate, mass term at T^n) stop once max |T^{k+1} - T^k| < corrector_tol; converged
        tells whether that happened within n_corrector passes (always True for the lagged single pass)."""
        p = self.p
        T_it = T_old
        passes = 0
        converged = p.n_corrector <= 1
        for passes in range(1, max(1, p.n_corrector) + 1):
            sig = self.sigma(T_it)
            A_V, b_V = self.system_V(T_it)
            V_new = solve(A_V, b_V)
            Q = joule(sig, V_new, self.tets, self.grad)
            T_new = self.solve_T(T_old, Q)
            change = float(np.max(np.abs(T_new - T_it)))
            T_it = T_new
            if p.n_corrector > 1 and change < p.corrector_tol:
                converged = True
                break
        return T_it, V_new, passes, converged

    def run(self, n_steps, T0=None):
        """Returns arrays T [n_steps, N] and V [n_steps, N] after each step."""
        T = np.full(self.N, 37.0) if T0 is None else np.asarray(T0, dtype=np.float64).copy()
        Ts, Vs = [], []
        for _ in range(n_steps):
            T, V, _ = self.step(T)
            Ts.append(T)
            Vs.append(V)
        return np.array(Ts), np.array(Vs)


def model_with_dt(model: "Model", dt) -> "Model":
    """A copy of `model` with time step dt (the thermal matrix depends on it)."""
    m = Model.__new__(Model)
    m.__dict__.update({key: val for key, val in model.__dict__.items() if key != "_lu_T"})
    m.p = dataclasses.replace(model.p, dt=float(dt))
    m.A_T = ((m.p.rho_c / m.p.dt + m.p.perf) * m.M + m.Kk).tocsr()
    m.A_T.sort_indices()
    return m


def advance(model: "Model", duration, dt_min, T0=None):
    """Dynamic time stepping of the main loop (Sec. II-A: dynamically sized steps; Sec. IV: a step whose corrector
    does not converge within the maximum number of passes is not accepted and the step size is halved, so the
    run still ends at the same final time). From T0 (default 37 everywhere), steps of the current size
    dt = model.p.dt, the last one shortened to end exactly at `duration`; a step that does not converge is
    rejected and retried from the same state with half the size, which is kept afterwards; when half the size would
    fall below dt_min the step is accepted unconverged. Returns (T, V, log) with log = [(dt, passes, converged,
    accepted), ...] for every attempted step."""
    T = np.full(model.N, 37.0) if T0 is None else np.asarray(T0, dtype=np.float64).copy()
    V = None
    t, dt, log = 0.0, float(model.p.dt), []
    while t < duration * (1.0 - 1e-12):
        dt_step = min(dt, duration - t)
        T_new, V_new, passes, ok = model_with_dt(model, dt_step).step_detail(T)
        if ok or dt_step * 0.5 < dt_min:
            T, V, t = T_new, V_new, t + dt_step
            log.append((dt_step, passes, ok, True))
        else:
            dt = dt_step * 0.5
            log.append((dt_step, passes, ok, False))
    return T, V, log


# ----------------------------------------------------------------------------------------------------------
# Initial guess by projection (an extension of the predictor step of the main loop, Sec. II-A)
# ----------------------------------------------------------------------------------------------------------

def projection_guess(A, b, X, free):
    """The element of span(X) closest to the solution of the SPD system A x = b in the A-norm, on the free rows.

    Minimising (x - x*)^T A (x - x*) over x = X c gives the Galerkin condition X^T (b - A X c) = 0, solved here
    with an orthonormal basis Q of span(X) from numpy's QR (the span, not the basis, defines the result):
    (Q^T A Q) y = Q^T b, x = Q y. Rows outside `free` (the identity rows of the lifted system) keep the values
    of the newest column X[:, 0]. A and b are the lifted system, X holds the past solutions as columns.
    """
    X = np.asarray(X, dtype=np.float64)
    free = np.asarray(free, dtype=bool)
    Q, _ = np.linalg.qr(X[free])
    Aff = sp.csr_matrix(A)[free][:, free]
    y = np.linalg.solve(Q.T @ (Aff @ Q), Q.T @ np.asarray(b, dtype=np.float64)[free])
    x0 = X[:, 0].copy()
    x0[free] = Q @ y
    return x0


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


# ----------------------------------------------------------------------------------------------------------
# Differentiation of the time loop (gradient of a loss on the final temperature with respect to the
# per-element conductivities sigma0_e and k_e, and to the initial temperature).
#
# Two independent routes, both on the lagged step (n_corrector = 1):
#   * forward mode: the tangent-linear step, obtained by differentiating every line of Model.step, propagates
#     directional derivatives (dT^n, dsigma0, dk) -> dT^{n+1};
#   * central finite differences of the forward model.
# gradient_dense_adjoint builds, for tiny meshes, the full step Jacobians column by column with the tangent step
# and accumulates the gradient backwards with their explicit transposes (no symmetry of any matrix is used).
# ----------------------------------------------------------------------------------------------------------

def _scatter(vals_e4, tets, N):
    """Sum per-(element, vertex) values [E, 4, m] into nodes [N, m]."""
    out = np.zeros((N, vals_e4.shape[2]))
    np.add.at(out, np.asarray(tets).ravel(), vals_e4.reshape(-1, vals_e4.shape[2]))
    return out


def _solve_many(A, B):
    """Solve A X = B for a block of right-hand sides with a direct method."""
    if A.shape[0] <= DENSE_LIMIT:
        return np.linalg.solve(A.toarray(), B)
    return spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A").solve(B)


def model_with_params(model: "Model", sigma0=None, k=None) -> "Model":
    """A copy of `model` with new per-element sigma0 and/or k (the thermal matrix is rebuilt)."""
    m = Model.__new__(Model)
    m.__dict__.update({key: val for key, val in model.__dict__.items() if key != "_lu_T"})
    if sigma0 is not None:
        m.sigma0 = np.asarray(sigma0, dtype=np.float64).copy()
    if k is not None:
        m.k = np.asarray(k, dtype=np.float64).copy()
        m.Kk = assemble(element_stiffness(m.k, m.vol, m.grad), m.tets, m.N)
        p = m.p
        m.A_T = ((p.rho_c / p.dt + p.perf) * m.M + m.Kk).tocsr()
        m.A_T.sort_indices()
    return m


def step_tangent(model: "Model", T_old, dT_old, dsig0, dk):
    """One lagged step and its forward-mode derivative.

    dT_old [N, m], dsig0 [E, m], dk [E, m] are m directions; returns (T_new, V_new, dT_new [N, m]). Every term
    differentiates the corresponding line of the step:
      sigma_e = sigma0_e f_e, f_e = 1 + alpha (Tbar_e - 37)
          d sigma_e = dsigma0_e f_e + sigma0_e alpha dTbar_e
      K(sigma) V = 0 (lifted)      ->  K_ff dV_f = -(dK V)_f,  dK V = sum_e dsigma_e G_e V_e
      F_a = sum_e sigma_e V_e^T G_e V_e / 4
          dF_a = sum_e (dsigma_e V_e^T G_e V_e + 2 sigma_e V_e^T G_e dV_e) / 4
      A_T T^{n+1} = (rho_c/dt) M T^n + perf T_a M 1 + F (lifted)
          A_T,ff dT_f = ((rho_c/dt) M dT^n + dF - (dA_T T^{n+1}))_f,  dA_T T = sum_e dk_e G_e T_e
    with G_e = vol_e grad(phi) grad(phi)^T and zero derivatives on Dirichlet rows.
    """
    p = model.p
    tets = model.tets
    N = model.N
    dT_old = np.asarray(dT_old, dtype=np.float64)
    dsig0 = np.asarray(dsig0, dtype=np.float64)
    dk = np.asarray(dk, dtype=np.float64)
    f = 1.0 + p.alpha_sigma * (element_mean(T_old, tets) - 37.0)
    sig = model.sigma0 * f
    A_V, b_V = model.system_V(T_old)
    V = solve(A_V, b_V)
    Q = joule(sig, V, tets, model.grad)
    A_T, b_T = model.system_T(T_old, Q)
    T_new = solve(A_T, b_T)

    G = element_stiffness(np.ones(len(tets)), model.vol, model.grad)       # [E, 4, 4]
    GV = np.einsum("eab,eb->ea", G, V[tets])                                 # [E, 4]
    dTbar = dT_old[tets].mean(axis=1)                                        # [E, m]
    dsig = dsig0 * f[:, None] + model.sigma0[:, None] * p.alpha_sigma * dTbar
    rhs_V = -_scatter(GV[:, :, None] * dsig[:, None, :], tets, N)
    rhs_V[model.bc_V] = 0.0
    dV = _solve_many(A_V, rhs_V)
    VGV = np.einsum("ea,ea->e", V[tets], GV)
    VGdV = np.einsum("ea,eam->em", GV, dV[tets])
    dq = 0.25 * (dsig * VGV[:, None] + 2.0 * sig[:, None] * VGdV)          # [E, m]
    dF = _scatter(np.repeat(dq[:, None, :], 4, axis=1), tets, N)
    GT = np.einsum("eab,eb->ea", G, T_new[tets])
    rhs_T = (p.rho_c / p.dt) * (model.M @ dT_old) + dF - _scatter(GT[:, :, None] * dk[:, None, :], tets, N)
    rhs_T[model.bc_T] = 0.0
    dT_new = _solve_many(A_T, rhs_T)
    return T_new, V, dT_new


def gradient_dense_adjoint(model: "Model", n_steps, dL_dT_final, T0=None):
    """Reverse accumulation with dense step Jacobians (tiny meshes only).

    For each step n the Jacobians J_T = dT^{n+1}/dT^n [N, N], J_s = dT^{n+1}/dsigma0 [N, E] and
    J_k = dT^{n+1}/dk [N, E] are built column by column with step_tangent; then, from lam = dL/dT^N backwards,
    g_sigma0 += J_s^T lam, g_k += J_k^T lam, lam <- J_T^T lam. Returns (g_sigma0, g_k, dL/dT^0); the last one is
    the derivative with respect to every entry of the initial state vector (Dirichlet entries included: they
    enter the first step through sigma(Tbar) and the mass term).
    """
    if model.p.n_corrector != 1:
        raise ValueError("the gradient is defined for the lagged step (n_corrector = 1)")
    N, E = model.N, len(model.tets)
    T = np.full(N, 37.0) if T0 is None else np.asarray(T0, dtype=np.float64).copy()
    states = [T]
    for _ in range(n_steps):
        T, _, _ = model.step(T)
        states.append(T)
    lam = np.asarray(dL_dT_final, dtype=np.float64).copy()
    g_s = np.zeros(E)
    g_k = np.zeros(E)
    for n in reversed(range(n_steps)):
        Tn = states[n]
        _, _, J_T = step_tangent(model, Tn, np.eye(N), np.zeros((E, N)), np.zeros((E, N)))
        _, _, J_s = step_tangent(model, Tn, np.zeros((N, E)), np.eye(E), np.zeros((E, E)))
        _, _, J_k = step_tangent(model, Tn, np.zeros((N, E)), np.zeros((E, E)), np.eye(E))
        g_s += J_s.T @ lam
        g_k += J_k.T @ lam
        lam = J_T.T @ lam
    return g_s, g_k, lam


def loss_final_T(model: "Model", n_steps, target, T0=None):
    """L = sum_i (T^N_i - target_i)^2 after n_steps lagged steps."""
    T, _ = model.run(n_steps, T0)
    return float(np.sum((T[-1] - np.asarray(target, dtype=np.float64)) ** 2))


def gradient_fd(model: "Model", n_steps, target, which, elems, eps=1e-6, T0=None):
    """Central finite differences of loss_final_T with respect to sigma0_e or k_e (which = "sigma0" | "k") for the
    listed elements; the step is h = eps * |p_e| (relative perturbation)."""
    base = model.sigma0 if which == "sigma0" else model.k
    out = np.empty(len(elems))
    for i, e in enumerate(elems):
        h = eps * abs(base[e])
        vals = []
        for sgn in (1.0, -1.0):
            q = base.copy()
            q[e] += sgn * h
            m = model_with_params(model, **{which: q})
            vals.append(loss_final_T(m, n_steps, target, T0))
        out[i] = (vals[0] - vals[1]) / (2.0 * h)
    return out


# ----------------------------------------------------------------------------------------------------------
# ILU(0) preconditioner (Sec. II-B: preconditioning accelerates the Krylov solvers). The factorisation is taken
# on a symmetric permutation P A P^T of the system in which rows of one level never depend on each other:
#   "natural":    nodes sorted (stably) by dependency level in the given numbering,
#                 lev(i) = 1 + max{lev(j) : j < i, a_ij != 0} (0 if none); levels = these sets;
#   "multicolor": nodes sorted (stably) by a colour. With g the largest |lev(i) - lev(j)| over the edges, the
#                 colouring lev mod (g + 1) is proper (neighbours are 1..g levels apart); it is used unless the
#                 greedy colouring (each node takes the smallest colour not used by an already-coloured
#                 neighbour, nodes visited in index order) needs fewer colours. Levels = colours.
# ----------------------------------------------------------------------------------------------------------

def greedy_node_colors(A):
    A = sp.csr_matrix(A)
    N = A.shape[0]
    color = np.full(N, -1, dtype=np.int64)
    for i in range(N):
        used = {int(color[j]) for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i and color[j] >= 0}
        c = 0
        while c in used:
            c += 1
        color[i] = c
    return color


def dependency_levels(A):
    A = sp.csr_matrix(A)
    N = A.shape[0]
    lev = np.zeros(N, dtype=np.int64)
    for i in range(N):
        lower = [j for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j < i]
        lev[i] = 1 + max(lev[j] for j in lower) if lower else 0
    return lev


def level_modulo_colors(A):
    """lev mod (g + 1), g = the largest dependency-level gap along an edge (capped at the number of levels)."""
    A = sp.csr_matrix(A)
    lev = dependency_levels(A)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    gap = int(np.abs(lev[rows] - lev[A.indices]).max()) if A.nnz else 0
    m = min(gap + 1, int(lev.max()) + 1)
    return lev % m


def ilu_permutation(A, order="multicolor"):
    """(perm, level_of_new_row): perm[new] = old row; rows sorted stably by colour or dependency level."""
    if order == "multicolor":
        mod = level_modulo_colors(A)
        greedy = greedy_node_colors(A)
        key = mod if mod.max() <= greedy.max() else greedy
    else:
        key = dependency_levels(A)
    perm = np.argsort(key, kind="stable")
    return perm, key[perm]


def permute_symmetric(A, perm):
    """P A P^T with (P A P^T)[a, b] = A[perm[a], perm[b]], indices sorted."""
    B = sp.csr_matrix(A)[perm][:, perm].tocsr()
    B.sort_indices()
    return B


def ilu0(A):
    """ILU(0) on the stored pattern of A (CSR, sorted indices, every diagonal stored), row by row (IKJ form):
    for row i, for each stored k < i in increasing order: w_k <- w_k / u_kk, then w_j <- w_j - w_k u_kj for every
    stored j > k of row k that is also stored in row i; no fill outside the pattern. Returns F on A's pattern with
    the strictly lower part = L (unit diagonal implied) and the diagonal + upper part = U."""
    A = sp.csr_matrix(A, dtype=np.float64, copy=True)
    A.sort_indices()
    ip, ix, F = A.indptr, A.indices, A.data
    N = A.shape[0]
    diag = np.empty(N, dtype=np.int64)
    for i in range(N):
        d = np.flatnonzero(ix[ip[i]:ip[i + 1]] == i)
        if d.size != 1:
            raise ValueError("every diagonal entry must be stored")
        diag[i] = ip[i] + d[0]
    for i in range(N):
        pos = {int(ix[q]): q for q in range(ip[i], ip[i + 1])}
        for q in range(ip[i], diag[i]):
            k = int(ix[q])
            F[q] = F[q] / F[diag[k]]
            for t in range(diag[k] + 1, ip[k + 1]):
                j = int(ix[t])
                if j in pos:
                    F[pos[j]] -= F[q] * F[t]
    return sp.csr_matrix((F, ix.copy(), ip.copy()), shape=A.shape)


def ilu0_split(F):
    """(L, U) dense-free: L = I + strictly lower part of F, U = diagonal + upper part of F."""
    F = sp.csr_matrix(F)
    L = sp.tril(F, k=-1, format="csr") + sp.identity(F.shape[0], format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L.tocsr(), U.tocsr()


def ilu0_apply(F, r):
    """z = U^{-1} L^{-1} r (forward then backward substitution)."""
    L, U = ilu0_split(F)
    y = spla.spsolve_triangular(L, np.asarray(r, dtype=np.float64), lower=True, unit_diagonal=True)
    return spla.spsolve_triangular(U, y, lower=False)


def pcg(A, b, x0, apply_Minv, tol, max_iter=100000):
    """Preconditioned conjugate gradients (Sec. II-B: CG for symmetric positive-definite systems, preconditioned to
    speed up convergence), textbook Hestenes-Stiefel form: r = b - A x, z = M^-1 r, p = z; then alpha =
    (r, z) / (p, A p), x += alpha p, r -= alpha A p, z = M^-1 r, beta = (r, z)_new / (r, z)_old, p = z + beta p,
    until ||r|| <= tol ||b||. Returns (x, iterations). For iteration counts of a preconditioner, not for speed."""
    A = sp.csr_matrix(A)
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    r = b - A @ x
    bn = np.linalg.norm(b)
    bn = bn if bn > 0 else 1.0
    if np.linalg.norm(r) <= tol * bn:
        return x, 0
    z = apply_Minv(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, max_iter + 1):
        Ap = A @ p
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= tol * bn:
            return x, it
        z = apply_Minv(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter


# ----------------------------------------------------------------------------------------------------------
# Node renumbering (locality of unstructured-like numberings): reverse Cuthill-McKee
# ----------------------------------------------------------------------------------------------------------

def rcm_order(A):
    """Reverse Cuthill-McKee order of the graph of A (perm[new] = old). For each connected component, taken in
    order of its lowest node: start at the smallest-degree node (lowest index on ties); while the smallest-degree
    node of the last breadth-first level (lowest index on ties) has a larger eccentricity, move there; then number
    breadth first, appending each node's unnumbered neighbours in increasing (degree, index). Reverse at the end."""
    A = sp.csr_matrix(A)
    N = A.shape[0]
    nbrs = [[int(j) for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i] for i in range(N)]
    deg = [len(x) for x in nbrs]
    done = [False] * N
    order = []

    def levels(s):
        depth = {s: 0}
        frontier = [s]
        while True:
            nxt = []
            for u in frontier:
                for v in nbrs[u]:
                    if not done[v] and v not in depth:
                        depth[v] = depth[u] + 1
                        nxt.append(v)
            if not nxt:
                return depth[frontier[0]], frontier
            frontier = nxt

    def smallest(nodes):
        return min(nodes, key=lambda v: (deg[v], v))

    for first in range(N):
        if done[first]:
            continue
        comp, seen = [first], {first}
        for u in comp:
            for v in nbrs[u]:
                if not done[v] and v not in seen:
                    seen.add(v)
                    comp.append(v)
        s = smallest(comp)
        ecc, last = levels(s)
        while True:
            c = smallest(last)
            e2, last2 = levels(c)
            if e2 <= ecc:
                break
            s, ecc, last = c, e2, last2
        start = len(order)
        order.append(s)
        done[s] = True
        h = start
        while h < len(order):
            u = order[h]
            for v in sorted((v for v in nbrs[u] if not done[v]), key=lambda v: (deg[v], v)):
                done[v] = True
                order.append(v)
            h += 1
    return np.array(order[::-1], dtype=np.int64)


def bandwidth(A):
    """max |i - j| over the stored entries."""
    A = sp.coo_matrix(A)
    return int(np.abs(A.row - A.col).max()) if A.nnz else 0


# ----------------------------------------------------------------------------------------------------------
# Monolithic coupled step (the paper's 2N x 2N system shape, Table II): V and T of a step solved together by
# Newton's method on
#   R_V = K(sigma(T)) V                                            (free potential rows)
#   R_T = A_T T - (rho_c/dt) M T^n - perf T_a M 1 - F(V, sigma(T))  (free thermal rows)
# with sigma at the element mean of the new T (no lagging). Its solution is the fixed point the corrector passes
# converge to. Unknowns are interleaved per node: x[2i] = V_i, x[2i+1] = T_i.
# ----------------------------------------------------------------------------------------------------------

def coupled_residual(model: "Model", V, T, T_old):
    """R (length 2N, interleaved) of the coupled step at (V, T); Dirichlet rows hold x - g."""
    p = model.p
    tets = model.tets
    sig = model.sigma(T)
    K = assemble(element_stiffness(sig, model.vol, model.grad), tets, model.N)
    RV = K @ V
    Q = joule(sig, V, tets, model.grad)
    RT = model.A_T @ T - model.rhs_T_unlifted(T_old, Q)
    RV = np.where(model.bc_V, V - model.g_V, RV)
    RT = np.where(model.bc_T, T - model.g_T, RT)
    R = np.empty(2 * model.N)
    R[0::2] = RV
    R[1::2] = RT
    return R


def coupled_jacobian(model: "Model", V, T):
    """dR/dx of coupled_residual (2N x 2N CSR, interleaved), from the element derivatives:
      d(K V)_i/dT_a   = sum_e (sigma0_e alpha / 4) (G_e V_e)_i
      dF_i/dV_j       = sum_e (sigma_e / 4) 2 (G_e V_e)_j
      dF_i/dT_a       = sum_e (sigma0_e alpha / 4) (V_e^T G_e V_e) / 4
    (sums over the elements containing both nodes), G_e = vol_e grad(phi) grad(phi)^T; Dirichlet rows are
    identity rows of their own unknown."""
    p = model.p
    tets = model.tets
    N, E = model.N, len(tets)
    sig = model.sigma(T)
    G = element_stiffness(np.ones(E), model.vol, model.grad)          # [E, 4, 4]
    Ve = np.asarray(V)[tets]
    GV = np.einsum("eab,eb->ea", G, Ve)                                  # [E, 4]
    quad = np.einsum("ea,ea->e", Ve, GV)
    ds = model.sigma0 * p.alpha_sigma / 4.0                              # d sigma_e / d T_a, a in e
    KVV = sig[:, None, None] * G                                         # d R_V / d V
    KVT = ds[:, None, None] * np.repeat(GV[:, :, None], 4, axis=2)      # [e, i, a] = ds_e (G V)_i
    KTV = -(sig / 4.0)[:, None, None] * 2.0 * np.repeat(GV[:, None, :], 4, axis=1)   # [e, i, j] = -(s/4) 2 (G V)_j
    KTT = -(ds * quad / 4.0)[:, None, None] * np.ones((1, 4, 4))        # - dF_i / dT_a
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    blocks = []
    for (bi, bj, Ke) in ((0, 0, KVV), (0, 1, KVT), (1, 0, KTV), (1, 1, KTT)):
        blocks.append((2 * rows + bi, 2 * cols + bj, Ke.ravel()))
    AT = sp.coo_matrix(model.A_T)
    blocks.append((2 * AT.row + 1, 2 * AT.col + 1, AT.data))
    r = np.concatenate([b[0] for b in blocks])
    c = np.concatenate([b[1] for b in blocks])
    v = np.concatenate([b[2] for b in blocks])
    J = sp.coo_matrix((v, (r, c)), shape=(2 * N, 2 * N)).tocsr()
    J.sum_duplicates()
    dir_rows = np.concatenate([2 * np.flatnonzero(model.bc_V), 2 * np.flatnonzero(model.bc_T) + 1])
    J = J.tolil()
    for rr in dir_rows:
        J.rows[rr] = [int(rr)]
        J.data[rr] = [1.0]
    J = J.tocsr()
    J.sort_indices()
    return J


def step_newton(model: "Model", T_old, V0=None, tol=1e-10, max_iter=50):
    """One coupled step by Newton's method from (V0, T_old) (Dirichlet values imposed first); stops when
    max |dT| < tol. Returns (T, V, iterations, [max |dT| per iteration])."""
    N = model.N
    V = np.where(model.bc_V, model.g_V, np.zeros(N) if V0 is None else np.asarray(V0, dtype=np.float64))
    T = np.where(model.bc_T, model.g_T, np.asarray(T_old, dtype=np.float64))
    hist = []
    for it in range(1, max_iter + 1):
        R = coupled_residual(model, V, T, T_old)
        J = coupled_jacobian(model, V, T)
        d = spla.spsolve(J.tocsc(), -R)
        V = V + d[0::2]
        T = T + d[1::2]
        hist.append(float(np.max(np.abs(d[1::2]))))
        if hist[-1] < tol:
            break
    return T, V, it, hist
