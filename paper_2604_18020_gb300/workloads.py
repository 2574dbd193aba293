"""Seeded synthetic inputs: meshes, boundary conditions, loads, density and
vector fields.

This module holds no arithmetic of the method (no stiffness, filter, solver
or update): it only builds the data a caller hands to the library -- the load
vector ``f``, the per-node fixed-DOF mask and random fields drawn from a
seed.  Both the CUDA path and the CPU oracle consume what it returns, and it
imports neither of them.

Conventions (the paper fixes none of them; they are the library's):
  * elements (i, j, k), i fastest: e = i + nelx*(j + nely*k); element edge h = 1;
  * nodes n = i + (nelx+1)*(j + (nely+1)*k); DOF = 3*n + c, c in {x, y, z};
  * x is the beam length, y its height ("downward" is -y), z its depth, the
    2 x 1 x 0.5 cantilever domain of Sec. 4.1 of the paper;
  * the fixed set is a per-node uint8 mask, bit c set when DOF c is fixed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FIX_X, FIX_Y, FIX_Z = 1, 2, 4
FIX_ALL = FIX_X | FIX_Y | FIX_Z


@dataclass(frozen=True)
class Mesh:
    nelx: int
    nely: int
    nelz: int

    @property
    def n_elem(self) -> int:
        return self.nelx * self.nely * self.nelz

    @property
    def node_dims(self):
        return (self.nelx + 1, self.nely + 1, self.nelz + 1)

    @property
    def n_node(self) -> int:
        return (self.nelx + 1) * (self.nely + 1) * (self.nelz + 1)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_node

    def node(self, i, j, k):
        return i + (self.nelx + 1) * (j + (self.nely + 1) * k)


@dataclass
class Problem:
    """A load case: mesh, load vector(s) and fixed-DOF mask."""
    name: str
    mesh: Mesh
    f: np.ndarray            # float64 [n_dof] or [nrhs, n_dof]
    fixed: np.ndarray        # uint8 [n_node]
    volfrac: float
    rmin: float
    meta: dict


def _node_grid(mesh: Mesh):
    """Integer node coordinates as arrays shaped [nz+1, ny+1, nx+1]."""
    k, j, i = np.meshgrid(np.arange(mesh.nelz + 1), np.arange(mesh.nely + 1),
                          np.arange(mesh.nelx + 1), indexing="ij")
    return i, j, k


def fixed_face(mesh: Mesh, face: str) -> np.ndarray:
    """Per-node mask with every DOF of one box face clamped.

    face is one of 'x0', 'x1', 'y0', 'y1', 'z0', 'z1'."""
    i, j, k = _node_grid(mesh)
    axis, side = face[0], face[1]
    coord = {"x": i, "y": j, "z": k}[axis]
    top = {"x": mesh.nelx, "y": mesh.nely, "z": mesh.nelz}[axis]
    sel = coord == (0 if side == "0" else top)
    m = np.zeros(mesh.node_dims[::-1], dtype=np.uint8)
    m[sel] = FIX_ALL
    return m.reshape(-1)


def cantilever(nelx: int, nely: int, nelz: int, volfrac: float = 0.3,
               rmin: float = 1.5) -> Problem:
    """Cantilever with the x=0 face clamped and a unit total -y load shared
    equally by the nelz+1 nodes of the bottom edge of the x=end face
    (i = nelx, j = 0, k = 0..nelz)."""
    mesh = Mesh(nelx, nely, nelz)
    f = np.zeros(mesh.n_dof)
    share = 1.0 / (nelz + 1)
    for k in range(nelz + 1):
        f[3 * mesh.node(nelx, 0, k) + 1] = -share
    return Problem("cantilever", mesh, f, fixed_face(mesh, "x0"), volfrac,
                   rmin, {"load": "bottom edge of x=end face, equal shares"})


def cantilever_point(nelx: int, nely: int, nelz: int, volfrac: float = 0.3,
                     rmin: float = 1.5) -> Problem:
    """Cantilever of Sec. 4.1: x=0 face clamped, unit -y point load at the
    node (nelx, nely//2, nelz//2), the midpoint of the right face."""
    mesh = Mesh(nelx, nely, nelz)
    f = np.zeros(mesh.n_dof)
    f[3 * mesh.node(nelx, nely // 2, nelz // 2) + 1] = -1.0
    return Problem("cantilever_point", mesh, f, fixed_face(mesh, "x0"),
                   volfrac, rmin, {"load": "unit point load, right-face midpoint"})


def torsion(nelx: int = 55, nely: int = 55, nelz: int = 165,
            volfrac: float = 0.2, rmin: float = 2.0) -> Problem:
    """Torsion bar along z: z=0 face clamped; every node of the z=end face
    carries a tangential force proportional to its distance from the bar
    axis (x_c, y_c) = (nelx/2, nely/2), scaled to a unit total torque."""
    mesh = Mesh(nelx, nely, nelz)
    xc, yc = nelx / 2.0, nely / 2.0
    f = np.zeros(mesh.n_dof)
    jj, ii = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    dx = ii.astype(np.float64) - xc
    dy = jj.astype(np.float64) - yc
    r2 = dx * dx + dy * dy
    scale = 1.0 / r2.sum()
    nodes = mesh.node(ii, jj, nelz)
    f[3 * nodes + 0] = -dy * scale
    f[3 * nodes + 1] = dx * scale
    return Problem("torsion", mesh, f, fixed_face(mesh, "z0"), volfrac, rmin,
                   {"load": "tangential, proportional to radius, unit torque"})


def multi_rhs_cantilever(nelx: int, nely: int, nelz: int, nrhs: int = 8,
                         seed: int = 3, volfrac: float = 0.3,
                         rmin: float = 1.5) -> Problem:
    """nrhs load cases on one cantilever: unit -y point loads at distinct
    free-end nodes (i = nelx) drawn with numpy's default_rng(seed)."""
    mesh = Mesh(nelx, nely, nelz)
    rng = np.random.default_rng(seed)
    face = [(j, k) for k in range(nelz + 1) for j in range(nely + 1)]
    pick = rng.choice(len(face), size=nrhs, replace=False)
    f = np.zeros((nrhs, mesh.n_dof))
    nodes = []
    for r, p in enumerate(pick):
        j, k = face[int(p)]
        n = mesh.node(nelx, j, k)
        f[r, 3 * n + 1] = -1.0
        nodes.append((nelx, j, k))
    return Problem("multi_rhs_cantilever", mesh, f, fixed_face(mesh, "x0"),
                   volfrac, rmin, {"load_nodes": nodes, "seed": seed})


def uneven_instances(count: int = 64, seed: int = 5, kmin: int = 8,
                     kmax: int = 24) -> list[Problem]:
    """count independent cantilevers of seeded uneven size 2k x k x k with
    k ~ U{kmin..kmax} (16x8x8 ... 48x24x24), each with the edge load of
    :func:`cantilever`."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(kmin, kmax + 1, size=count)
    return [cantilever(2 * int(k), int(k), int(k)) for k in ks]


# ---------------------------------------------------------------- fields

def rho_uniform(mesh: Mesh, value: float) -> np.ndarray:
    return np.full(mesh.n_elem, float(value))


def rho_random(mesh: Mesh, seed: int, lo: float = 0.01, hi: float = 1.0) -> np.ndarray:
    """Element field ~ U(lo, hi), float64, element order."""
    return np.random.default_rng(seed).uniform(lo, hi, mesh.n_elem)


def rho_binary(mesh: Mesh, seed: int, volfrac: float = 0.3) -> np.ndarray:
    """Late-SIMP-like field: each element 1 with probability volfrac, else
    1e-3 (solid/void contrast of a nearly converged design)."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(mesh.n_elem) < volfrac, 1.0, 1e-3)


def vec_random(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Vector ~ U(lo, hi), float64."""
    return np.random.default_rng(seed).uniform(lo, hi, n)


def zero_fixed(v: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """Copy of a DOF vector with the fixed DOFs set to zero (a legal initial
    guess or load for the masked operator)."""
    out = np.array(v, dtype=np.float64, copy=True)
    bits = np.stack([(fixed >> c) & 1 for c in range(3)], axis=1).reshape(-1)
    out[..., bits.astype(bool)] = 0.0
    return out


def fixed_dofs(fixed: np.ndarray) -> np.ndarray:
    """Boolean [n_dof] mask expanded from the per-node bit mask."""
    return np.stack([(fixed >> c) & 1 for c in range(3)], axis=1).reshape(-1).astype(bool)


def edof_random(mesh: Mesh, seed: int = 42) -> np.ndarray:
    """Random element connectivity of the synthetic hot-path microbenchmark
    (Sec. 5, Tab. profiling): the tensor shapes of the mesh's operator (its
    element and node counts) with each element's 8 node ids drawn uniformly
    from all nodes, then expanded to DOFs 3 n + c in the local order of the
    structured table.  int32 [n_elem, 24]."""
    rng = np.random.default_rng(seed)
    nodes = rng.integers(0, mesh.n_node, size=(mesh.n_elem, 8), dtype=np.int64)
    edof = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(mesh.n_elem, 24)
    return np.ascontiguousarray(edof.astype(np.int32))


def mbb(nelx: int = 150, nely: int = 50, nelz: int = 25, volfrac: float = 0.5,
        rmin: float = 1.5) -> Problem:
    """MBB hard problem of Sec. 4.1 (domain 3 x 1 x 0.5): u_x = 0 on the
    left face x = 0, u_y = 0 at the bottom-right node of the middle depth
    (nelx, 0, nelz // 2), a unit -y point load at the top-left node of the
    middle depth (0, nely, nelz // 2).  The z translation and the rotation
    about the x axis through the support stay free (the near-rigid-body
    modes the paper names as what makes it hard); the load is orthogonal to
    both, so the masked system is consistent."""
    mesh = Mesh(nelx, nely, nelz)
    i, j, k = _node_grid(mesh)
    m = np.zeros(mesh.node_dims[::-1], dtype=np.uint8)
    m[i == 0] |= FIX_X
    fixed = m.reshape(-1)
    fixed[mesh.node(nelx, 0, nelz // 2)] |= FIX_Y
    f = np.zeros(mesh.n_dof)
    f[3 * mesh.node(0, nely, nelz // 2) + 1] = -1.0
    return Problem("mbb", mesh, f, fixed, volfrac, rmin,
                   {"load": "unit point load, top-left node of the middle depth"})


def bridge(nelx: int = 150, nely: int = 50, nelz: int = 25, volfrac: float = 0.3,
           rmin: float = 1.5) -> Problem:
    """Bridge hard problem of Sec. 4.1 (domain 3 x 1 x 0.5): every DOF fixed
    on the left lower edge (0, 0, k), rollers along x on the right lower edge
    (nelx, 0, k: u_y = u_z = 0), a unit total -y load shared equally by the
    nodes of the top face (j = nely)."""
    mesh = Mesh(nelx, nely, nelz)
    fixed = np.zeros(mesh.n_node, dtype=np.uint8)
    for k in range(nelz + 1):
        fixed[mesh.node(0, 0, k)] = FIX_ALL
        fixed[mesh.node(nelx, 0, k)] = FIX_Y | FIX_Z
    f = np.zeros(mesh.n_dof)
    top = [mesh.node(i, nely, k) for k in range(nelz + 1) for i in range(nelx + 1)]
    for n in top:
        f[3 * n + 1] = -1.0 / len(top)
    return Problem("bridge", mesh, f, fixed, volfrac, rmin,
                   {"load": "unit total load, equal shares on the top face"})


# Named workloads: sizes of the paper's benchmarks and the configurations
# the library is measured on.
WORKLOADS = {
    "cantilever_24x12x12": lambda: cantilever(24, 12, 12, 0.3, 1.5),
    "cantilever_120x60x30": lambda: cantilever(120, 60, 30, 0.3, 1.5),
    "torsion_55x55x165": lambda: torsion(55, 55, 165, 0.2, 2.0),
    "cantilever_100x50x50_8rhs": lambda: multi_rhs_cantilever(100, 50, 50, 8, 3),
    "cantilever_256x128x150": lambda: cantilever(256, 128, 150, 0.12, 1.5),
    "cantilever_160x80x40": lambda: cantilever(160, 80, 40, 0.3, 1.5),
    "cantilever_200x100x50": lambda: cantilever(200, 100, 50, 0.3, 1.5),
    "cantilever_252x126x63": lambda: cantilever(252, 126, 63, 0.3, 1.5),
    "cantilever_340x170x85": lambda: cantilever(340, 170, 85, 0.3, 1.5),
    "cantilever_600x300x150": lambda: cantilever(600, 300, 150, 0.3, 1.5),
    "mbb_150x50x25": lambda: mbb(150, 50, 25),
    "bridge_150x50x25": lambda: bridge(150, 50, 25),
}
