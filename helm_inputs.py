"""Seeded synthetic inputs for the cavity Helmholtz workloads.

This module is shared by the CPU oracle (``oracle/``), the tests and ``bench.py``.
It holds no arithmetic of the method (no assembly, no solver step): only the
description of each workload (box, lattice, frequencies, solver settings) and the
seeded draws of its boundary data, laid out in the node / face numbering that
``include/helm.h`` defines:

* node id ``= i + (nx+1) * (j + (ny+1) * l)`` for lattice indices (i, j, l);
* boundary quads numbered side by side in the order x-, x+, y-, y+, z-, z+;
  inside a side, the quad at in-plane element indices (u, v) has index
  ``u + nu * v`` where u runs over the first remaining axis (x before y before z).

The paper's compartment mesh and its CFD pressure spectra are not available, so
these draws stand in for them (paper Sec. 3.2: sun-roof pressure used as Dirichlet
data on the opening, compartment walls otherwise).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

C_SOUND = 340.0  # m/s
RHO_AIR = 1.2    # kg/m^3


@dataclasses.dataclass(frozen=True)
class Mesh:
    """Box [0,Lx]x[0,Ly]x[0,Lz] cut into nx*ny*nz equal bricks (z is vertical)."""
    nx: int
    ny: int
    nz: int
    Lx: float
    Ly: float
    Lz: float

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_bfaces(self) -> int:
        nx, ny, nz = self.nx, self.ny, self.nz
        return 2 * (ny * nz + nx * nz + nx * ny)

    @property
    def nnz27(self) -> int:
        """Entries of the full 27-point pattern (explicit zeros included)."""
        return (3 * self.nx + 1) * (3 * self.ny + 1) * (3 * self.nz + 1)

    def side_offsets(self) -> List[int]:
        nx, ny, nz = self.nx, self.ny, self.nz
        sizes = [ny * nz, ny * nz, nx * nz, nx * nz, nx * ny, nx * ny]
        return [int(v) for v in np.concatenate([[0], np.cumsum(sizes)])]


@dataclasses.dataclass
class Problem:
    """One mesh with its boundary data (frequency-independent)."""
    mesh: Mesh
    beta: np.ndarray        # complex128 [n_bfaces], admittance per boundary quad (0 = rigid)
    dir_nodes: np.ndarray   # int32 [n_dir], ascending node ids with prescribed pressure
    p_dir: np.ndarray       # complex128 [n_dir], prescribed pressure (Pa)
    c: float = C_SOUND
    rho: float = RHO_AIR


# ---------------------------------------------------------------------------
# Boundary-data draws
# ---------------------------------------------------------------------------

def floor_face_index(mesh: Mesh, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Index of the floor quad (z- side) with element indices (i, j)."""
    return mesh.side_offsets()[4] + i + mesh.nx * j


def top_patch_nodes(mesh: Mesh, x0: float, x1: float, y0: float, y1: float) -> np.ndarray:
    """Ascending ids of top-face nodes (z = Lz) inside the closed patch [x0,x1]x[y0,y1]."""
    hx, hy = mesh.Lx / mesh.nx, mesh.Ly / mesh.ny
    eps = 1e-9
    i = np.arange(mesh.nx + 1)
    j = np.arange(mesh.ny + 1)
    I, J = np.meshgrid(i, j, indexing="xy")
    x, y = I * hx, J * hy
    m = (x >= x0 - eps) & (x <= x1 + eps) & (y >= y0 - eps) & (y <= y1 + eps)
    ids = I[m] + (mesh.nx + 1) * (J[m] + (mesh.ny + 1) * mesh.nz)
    return np.sort(ids).astype(np.int32)


def fourier_patch_pressure(mesh: Mesh, nodes: np.ndarray, patch: Tuple[float, float, float, float],
                           seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """Synthetic sun-roof pressure: 8 seeded cosine modes over the patch.

    p_s = scale * sum_{m<8} a_m e^{i theta_m} cos(pi m_x xi) cos(pi m_y eta),
    (m_x, m_y) = (m // 2, m % 2), xi, eta in [0,1] patch-local; a ~ N(0,1) drawn
    first, then theta ~ U[0, 2 pi).
    """
    x0, x1, y0, y1 = patch
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(8)
    theta = rng.uniform(0.0, 2.0 * np.pi, 8)
    nodes = np.asarray(nodes, dtype=np.int64)
    i = nodes % (mesh.nx + 1)
    j = (nodes // (mesh.nx + 1)) % (mesh.ny + 1)
    x = i * (mesh.Lx / mesh.nx)
    y = j * (mesh.Ly / mesh.ny)
    xi = (x - x0) / (x1 - x0)
    eta = (y - y0) / (y1 - y0)
    p = np.zeros(len(nodes), dtype=np.complex128)
    for m in range(8):
        mx, my = m // 2, m % 2
        p += a[m] * np.exp(1j * theta[m]) * np.cos(np.pi * mx * xi) * np.cos(np.pi * my * eta)
    return scale * p


def seat_floor_faces(mesh: Mesh, xa: float = 0.8, xb: float = 2.0) -> np.ndarray:
    """Floor quads whose centre has x in [xa, xb] (all y): the seat footprint."""
    hx = mesh.Lx / mesh.nx
    eps = 1e-9
    i = np.arange(mesh.nx)
    j = np.arange(mesh.ny)
    I, J = np.meshgrid(i, j, indexing="xy")  # J outer, I inner -> ascending face index
    xc = (I + 0.5) * hx
    m = (xc >= xa - eps) & (xc <= xb + eps)
    return np.sort(floor_face_index(mesh, I[m], J[m])).astype(np.int64)


def random_seat_beta(mesh: Mesh, seed: int = 1) -> np.ndarray:
    """beta_e = U[0.01,0.2] + i U[-0.05,0.05] on the seat floor quads (re drawn first)."""
    faces = seat_floor_faces(mesh)
    rng = np.random.default_rng(seed)
    re = rng.uniform(0.01, 0.2, len(faces))
    im = rng.uniform(-0.05, 0.05, len(faces))
    beta = np.zeros(mesh.n_bfaces, dtype=np.complex128)
    beta[faces] = re + 1j * im
    return beta


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

CABIN = (2.5, 1.4, 1.2)
SUNROOF = (1.0, 1.6, 0.45, 0.95)
SMALL_BOX = (1.0, 0.8, 0.6)
SMALL_PATCH = (0.3, 0.7, 0.25, 0.55)
LISTENER_CENTRE = (1.6, 0.4, 0.9)
LISTENER_RADIUS = 0.15


def small_box_problem(nx: int = 20, ny: int = 16, nz: int = 12) -> Problem:
    """1.0x0.8x0.6 m box, top patch Fourier pressure, whole floor beta = 0.05+0.01i."""
    mesh = Mesh(nx, ny, nz, *SMALL_BOX)
    nodes = top_patch_nodes(mesh, *SMALL_PATCH)
    p = fourier_patch_pressure(mesh, nodes, SMALL_PATCH, seed=0, scale=1.0)
    beta = np.zeros(mesh.n_bfaces, dtype=np.complex128)
    off = mesh.side_offsets()
    beta[off[4]:off[5]] = 0.05 + 0.01j
    return Problem(mesh, beta, nodes, p)


def cabin_problem(nx: int, ny: int, nz: int, beta_seed: int = 1, p_scale: float = 0.1) -> Problem:
    """2.5x1.4x1.2 m cabin, 0.6x0.5 m sun-roof Dirichlet patch, random seat admittance."""
    mesh = Mesh(nx, ny, nz, *CABIN)
    nodes = top_patch_nodes(mesh, *SUNROOF)
    p = fourier_patch_pressure(mesh, nodes, SUNROOF, seed=0, scale=p_scale)
    beta = random_seat_beta(mesh, seed=beta_seed)
    return Problem(mesh, beta, nodes, p)


def sweep_mesh_dims(f: float, c: float = C_SOUND) -> Tuple[int, int, int]:
    """Elements per axis for the multi-mesh sweep: max(min, ceil(40 L f / c))."""
    mins = (24, 14, 12)
    return tuple(max(mn, int(math.ceil(40.0 * L * f / c - 1e-9))) for mn, L in zip(mins, CABIN))


def sweep_freqs(n: int = 256) -> np.ndarray:
    return np.geomspace(20.0, 500.0, n)


def resonance_freqs(n: int = 64) -> np.ndarray:
    """Frequencies of the resonance sweep: bins 4 .. 4+n-1 of a 512-point FFT sampled at 256 Hz
    (0.5 Hz spacing, 2.0 .. 33.5 Hz for n = 64), around the compartment's 13 Hz response
    (paper Sec. 3.1: the sun-roof spectrum peaks near 13 Hz, with a half harmonic near 6 Hz)."""
    return 0.5 * (4 + np.arange(n))


def resonance_spectrum(freqs: np.ndarray, seed: int = 2) -> np.ndarray:
    """Complex amplitude of the sun-roof pressure per frequency: sqrt of a PSD shape with a
    Lorentzian peak at 13 Hz (half width 1.5 Hz), a weaker one at 6.5 Hz (half width 1 Hz) and a
    floor, times a seeded random phase (a PSD carries no phase)."""
    f = np.asarray(freqs, dtype=np.float64)
    psd = 1.0 / (1.0 + ((f - 13.0) / 1.5) ** 2) + 0.3 / (1.0 + ((f - 6.5) / 1.0) ** 2) + 0.02
    phase = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, f.size)
    return np.sqrt(psd) * np.exp(1j * phase)


def listener_weights(mesh: Mesh, centre=LISTENER_CENTRE, radius=LISTENER_RADIUS) -> np.ndarray:
    """w_i = 1/|S| for nodes within the listener sphere S, else 0 (real64 [n])."""
    n = mesh.n_nodes
    ids = np.arange(n)
    i = ids % (mesh.nx + 1)
    j = (ids // (mesh.nx + 1)) % (mesh.ny + 1)
    l = ids // ((mesh.nx + 1) * (mesh.ny + 1))
    x = i * (mesh.Lx / mesh.nx) - centre[0]
    y = j * (mesh.Ly / mesh.ny) - centre[1]
    z = l * (mesh.Lz / mesh.nz) - centre[2]
    inside = x * x + y * y + z * z <= radius * radius + 1e-12
    w = np.zeros(n)
    if inside.any():
        w[inside] = 1.0 / inside.sum()
    return w


@dataclasses.dataclass
class Workload:
    name: str
    problems: List[Problem]       # one per system (len 1 when all freqs share a mesh)
    freqs: np.ndarray             # one per system when len(problems) > 1
    solver: str                   # "gmres" | "cocg"
    restart: int = 50
    tol: float = 1e-10
    precond: Optional[str] = None  # None | "ras"
    ras_parts: Tuple[int, int, int] = (8, 4, 4)
    ras_overlap: int = 2
    mixed: bool = False


def workload(name: str) -> Workload:
    """The workloads: box100 (n=4641), cabin282k, sweep256, cabin2m, adjoint64, resonance64."""
    if name == "box100":
        return Workload(name, [small_box_problem()], np.array([100.0]), "gmres", restart=30)
    if name == "cabin282k":
        return Workload(name, [cabin_problem(100, 56, 48)], np.array([20.0, 100.0, 200.0]),
                        "gmres", restart=50, precond="ras")
    if name == "sweep256":
        f = sweep_freqs(256)
        probs = [cabin_problem(*sweep_mesh_dims(fi)) for fi in f]
        return Workload(name, probs, f, "cocg")
    if name == "cabin2m":
        return Workload(name, [cabin_problem(200, 112, 96)], np.geomspace(100.0, 400.0, 32),
                        "cocg", mixed=True)
    if name == "adjoint64":
        return Workload(name, [cabin_problem(100, 56, 48)], np.geomspace(20.0, 300.0, 64), "cocg")
    if name == "resonance64":
        # the sun-roof pattern of cabin_problem scaled per frequency by resonance_spectrum(f)
        return Workload(name, [cabin_problem(100, 56, 48)], resonance_freqs(64), "cocg")
    raise KeyError(name)


def random_complex(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded standard complex normal vector (test vectors for SpMV / reductions)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(dtype)
