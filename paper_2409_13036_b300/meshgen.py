"""Seeded synthetic inputs for the RAFEM hot path: tetrahedral cube meshes and their boundary data.

This module only produces problem inputs (coordinates, connectivity, boundary masks and values, per-element
tissue properties). It holds none of the method's arithmetic: no element matrices, no assembly, no solves.
Both the CUDA path's tests/bench and the CPU oracle draw their inputs from here.

Workload shape. The paper's meshes (a liver with two electrodes; Table II: 3,548 and 8,364 nodes) are not
available, so seeded cubes of side 80 mm stand in for them: n x n x n hexahedral cells, each split into six
P1 tetrahedra along the v0-v7 diagonal (Kuhn/Freudenthal split, conforming because every cell uses the same
diagonal direction). A needle electrode occupies the nodes within 1.5 mm of the central z-axis down to a given
depth below the top face (Sec. II-A describes the electrode-driven Joule heating the mesh must carry).

Node numbering is lexicographic: node(i, j, k) = i + (n+1) * (j + (n+1) * k).
Coordinates are in metres (generated in millimetres, converted once at the end).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

SEED_BASE = 2409_13036

# Physical defaults of the liver workload (metres, seconds, Kelvin-degrees Celsius, SI units).
LIVER_SIGMA0 = 0.333      # S/m electrical conductivity at 37 degC
LIVER_K = 0.512           # W/m/K thermal conductivity
LIVER_RHO_C = 3.6e6       # J/m^3/K volumetric heat capacity
LIVER_PERF = 2.4e4        # W/m^3/K perfusion coefficient (omega_b * c_b)
ALPHA_SIGMA = 0.015       # 1/degC temperature coefficient of sigma
T_BODY = 37.0             # degC arterial / initial / outer-face temperature


@dataclasses.dataclass
class Mesh:
    """One problem instance. Arrays are C-contiguous with the dtypes listed."""
    n_cells: int
    coords: np.ndarray      # float64 [N, 3], metres
    tets: np.ndarray        # int32   [E, 4], positively oriented
    lattice: np.ndarray     # int32   [N, 3], (i, j, k) lattice index of each node
    bc_V: np.ndarray        # uint8   [N], 1 = Dirichlet for the potential
    g_V: np.ndarray         # float64 [N], prescribed potential (V) where bc_V == 1, else 0
    bc_T: np.ndarray        # uint8   [N], 1 = Dirichlet for the temperature
    g_T: np.ndarray         # float64 [N], prescribed temperature (degC) where bc_T == 1, else 0
    sigma0: np.ndarray      # float64 [E], electrical conductivity at 37 degC (S/m)
    k: np.ndarray           # float64 [E], thermal conductivity (W/m/K)
    electrode: np.ndarray   # uint8   [N], 1 = electrode node
    V_electrode: float = 20.0

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def kuhn_tets(n: int) -> np.ndarray:
    """Connectivity of the 6-tet split of an n^3-cell lattice; tets ordered cell-major (cell id, then tet)."""
    n1 = n + 1
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # cell-major order with i fastest, matching the node numbering
    i = i.transpose(2, 1, 0).ravel()
    j = j.transpose(2, 1, 0).ravel()
    k = k.transpose(2, 1, 0).ravel()
    corner = np.empty((i.size, 8), dtype=np.int64)
    for b in range(8):
        di, dj, dk = b & 1, (b >> 1) & 1, (b >> 2) & 1
        corner[:, b] = (i + di) + n1 * ((j + dj) + n1 * (k + dk))
    local = []
    for perm in itertools.permutations(range(3)):
        a0, a1, _ = perm
        b1 = 1 << a0
        b2 = b1 | (1 << a1)
        # orientation of the path v0 -> v_b1 -> v_b2 -> v7 on the unit cube
        P = np.array([[(b >> s) & 1 for s in range(3)] for b in (0, b1, b2, 7)], dtype=np.float64)
        det = np.linalg.det(P[1:] - P[0])
        local.append((0, b1, b2, 7) if det > 0 else (0, b2, b1, 7))
    tets = np.empty((i.size, 6, 4), dtype=np.int64)
    for t, loc in enumerate(local):
        for a in range(4):
            tets[:, t, a] = corner[:, loc[a]]
    return np.ascontiguousarray(tets.reshape(-1, 4).astype(np.int32))


def _signed_volumes(coords: np.ndarray, tets: np.ndarray) -> np.ndarray:
    x = coords[tets]
    return np.linalg.det(x[:, 1:, :] - x[:, :1, :]) / 6.0


def cube_mesh(n: int, *, jitter: float = 0.0, seed: int | None = None, side_mm: float = 80.0,
              electrode_radius_mm: float = 1.5, electrode_depth_mm: float = 20.0, V_electrode: float = 20.0,
              sigma0: float | str = LIVER_SIGMA0, sigma0_cv: float = 0.10, k: float = LIVER_K,
              T_face: float = T_BODY) -> Mesh:
    """Build one seeded cube instance.

    jitter: interior nodes move by uniform(-jitter*h, +jitter*h) per coordinate (faces stay planar).
    sigma0: a scalar, or "lognormal" for a per-element lognormal draw with mean 0.333 S/m and CV sigma0_cv.
    Electrode nodes are selected on the unjittered lattice: x^2 + y^2 <= r^2 and z >= z_top - depth. When the
    axis falls between lattice lines so far that no node lies within r, the nodes nearest the axis are used.
    Boundary data: every outer-face node has V = 0 and T = T_face; electrode nodes have V = V_electrode
    (the electrode wins over the face value for V; T stays prescribed on the faces only).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    n1 = n + 1
    h = side_mm / n
    half = side_mm / 2.0
    idx = np.arange(n1 ** 3, dtype=np.int64)
    li = idx % n1
    lj = (idx // n1) % n1
    lk = idx // (n1 * n1)
    lattice = np.stack([li, lj, lk], axis=1).astype(np.int32)
    x0 = -half + lattice.astype(np.float64) * h          # unjittered, mm
    on_face = ((li == 0) | (li == n) | (lj == 0) | (lj == n) | (lk == 0) | (lk == n))

    rng = np.random.default_rng(seed if seed is not None else SEED_BASE)
    x = x0.copy()
    if jitter > 0.0:
        d = rng.uniform(-jitter * h, jitter * h, size=x.shape)
        d[on_face] = 0.0
        x += d

    r2 = x0[:, 0] ** 2 + x0[:, 1] ** 2
    r_min2 = float(r2.min())
    r_sel2 = max(electrode_radius_mm ** 2, r_min2) + 1e-9
    electrode = (r2 <= r_sel2) & (x0[:, 2] >= half - electrode_depth_mm - 1e-9)

    tets = kuhn_tets(n)
    coords = np.ascontiguousarray(x * 1e-3)
    vol = _signed_volumes(coords, tets)
    if not np.all(vol > 0):
        raise ValueError("jitter produced an inverted tetrahedron")

    E = tets.shape[0]
    if isinstance(sigma0, str):
        if sigma0 != "lognormal":
            raise ValueError(sigma0)
        s = np.sqrt(np.log1p(sigma0_cv ** 2))
        mu = np.log(LIVER_SIGMA0) - 0.5 * s * s
        sig = rng.lognormal(mu, s, size=E)
    else:
        sig = np.full(E, float(sigma0))

    bc_V = (on_face | electrode).astype(np.uint8)
    g_V = np.where(electrode, V_electrode, 0.0).astype(np.float64)
    bc_T = on_face.astype(np.uint8)
    g_T = np.where(on_face, T_face, 0.0).astype(np.float64)
    return Mesh(n_cells=n, coords=coords, tets=tets, lattice=lattice, bc_V=bc_V, g_V=g_V, bc_T=bc_T, g_T=g_T,
                sigma0=np.ascontiguousarray(sig, dtype=np.float64), k=np.full(E, float(k)),
                electrode=electrode.astype(np.uint8), V_electrode=float(V_electrode))


def permute_nodes(mesh: Mesh, perm) -> Mesh:
    """The same mesh with its nodes renumbered: new node k is old node perm[k] (element order unchanged)."""
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.shape[0])
    return dataclasses.replace(
        mesh, coords=np.ascontiguousarray(mesh.coords[perm]), tets=np.ascontiguousarray(inv[mesh.tets], dtype=np.int32),
        lattice=np.ascontiguousarray(mesh.lattice[perm]), bc_V=np.ascontiguousarray(mesh.bc_V[perm]),
        g_V=np.ascontiguousarray(mesh.g_V[perm]), bc_T=np.ascontiguousarray(mesh.bc_T[perm]),
        g_T=np.ascontiguousarray(mesh.g_T[perm]), electrode=np.ascontiguousarray(mesh.electrode[perm]))


def shuffled_nodes(mesh: Mesh, seed: int) -> tuple[Mesh, np.ndarray]:
    """A seeded random renumbering of the nodes (an unstructured-like numbering without locality); returns the
    renumbered mesh and perm (new node k = old node perm[k])."""
    perm = np.random.default_rng(seed).permutation(mesh.n_nodes)
    return permute_nodes(mesh, perm), perm


# ---------------------------------------------------------------------------------------------------------
# Named workloads (sizes and draws of the liver-cube workloads)
# ---------------------------------------------------------------------------------------------------------

def workload_single_step_8() -> Mesh:
    """8^3 cells (729 nodes, 3,072 tets), no jitter, uniform sigma0: one backward-Euler step."""
    return cube_mesh(8, jitter=0.0, seed=SEED_BASE + 0)


def workload_48() -> Mesh:
    """48^3 cells (117,649 nodes, 663,552 tets), interior jitter +-10% of h, uniform sigma0."""
    return cube_mesh(48, jitter=0.10, seed=SEED_BASE + 1)


def workload_127() -> Mesh:
    """127^3 cells (2,097,152 nodes, 12,290,298 tets), jitter +-10%, lognormal sigma0 (10% CV)."""
    return cube_mesh(127, jitter=0.10, seed=SEED_BASE + 2, sigma0="lognormal")


def batch_draws(count: int = 96, seed: int = SEED_BASE + 3, n_lo: int = 12, n_hi: int = 64):
    """Per-instance parameters of the batching workload: (n, V_electrode, depth_mm, sigma0, seed)."""
    rng = np.random.default_rng(seed)
    n = rng.integers(n_lo, n_hi + 1, size=count)
    V = rng.uniform(10.0, 40.0, size=count)
    depth = rng.uniform(10.0, 30.0, size=count)
    sig = rng.uniform(0.25, 0.45, size=count)
    return [(int(n[i]), float(V[i]), float(depth[i]), float(sig[i]), int(seed * 1000 + i)) for i in range(count)]


def batch_mesh(draw) -> Mesh:
    n, V, depth, sig, s = draw
    return cube_mesh(n, jitter=0.10, seed=s, V_electrode=V, electrode_depth_mm=depth, sigma0=sig)


def tumour_sigma0(mesh: Mesh, *, seed: int = SEED_BASE + 4, radius_mm: float = 15.0, inside: float = 0.5,
                  outside: float = LIVER_SIGMA0) -> np.ndarray:
    """Two-region sigma0: a sphere of radius 15 mm (element centroids on the unjittered lattice) centred at the
    electrode tip (0, 0, z_top - 20 mm) plus a seeded uniform offset in [-5, 5] mm per axis."""
    rng = np.random.default_rng(seed)
    n = mesh.n_cells
    half = 40.0
    centre = np.array([0.0, 0.0, half - 20.0]) + rng.uniform(-5.0, 5.0, size=3)
    x0 = -half + mesh.lattice.astype(np.float64) * (80.0 / n)
    cent = x0[mesh.tets].mean(axis=1)
    inside_mask = np.sum((cent - centre) ** 2, axis=1) <= radius_mm ** 2
    return np.where(inside_mask, inside, outside).astype(np.float64)
