"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module builds only *inputs*: nuclear geometries, a graded structured mesh of
P2 tetrahedra, the Dirichlet mask and the seeded random starting block V.  It
holds none of the method's arithmetic (no basis functions, no quadrature, no
assembly, no potentials): both sides of every parity test receive these arrays
and compute everything else on their own.

The paper's molecules (CCCBDB geometries) and its Gmsh radial meshes (Sec. 4.1,
Sec. 4.2) are not available, so synthetic systems of the same shape stand in:

* ``lih``        Z=3 at the origin and Z=1 at (3.015, 0, 0) bohr, box [-10, 10]^3,
                 24^3 cells, p=2 doubly occupied orbitals.
* ``chain``      a C10H22-like zigzag (C-C 2.9 bohr, 111 deg backbone angle,
                 C-H 2.06 bohr, H-C-H 109.5 deg), p=41, box = nuclei bounding box
                 padded by 10 bohr, 80x44x43 cells.
* ``lattice60``  4x4x4 sites at 2.9 bohr spacing minus four corners, Z alternating
                 6/1, p=210 singly occupied orbitals, 80^3 cells.
* ``hydrogenic`` one nucleus of charge Z at the origin (fixed-potential tests).
* ``random_nuclei`` 4-12 nuclei, Z in {1,6,7,8}, uniform in a 6 bohr box.

Mesh recipe (the reading used throughout): per axis, anchors are the two box walls
and the distinct nuclear coordinates on that axis (anchors closer than 0.3 bohr are
merged to their mean).  Cells are shared among the segments between anchors in
proportion to their length, at least 2 per segment.  A segment ending at a nucleus
is graded toward it with a tanh map of strength g=3.  Each hexahedron is split into
the 6 Kuhn tetrahedra around its (0,0,0)-(1,1,1) diagonal, so the mesh is
conforming; P2 nodes are the vertices plus the physical midpoints of the straight
edges, i.e. the full (2N+1)-lattice of the tensor-product coordinates.

Second grading (``make_mesh(system, grading="msf")``): the paper's mesh-size function
(Eq. meshsizefunction, Sec. 4.2), h(r) = min(gamma1 Z_1^{-2/5} r_1^{6/5}, ..., gamma1 Z_M^{-2/5}
r_M^{6/5}, gamma2), restricted to each axis (r_j = |x - X_j| along the axis, the finest size any
point of that coordinate plane asks for).  The paper meshes with Gmsh (unstructured); here the
same size function grades the tensor-product grid (``axis_vertices_msf``): the spacing follows
h's shape (held at its value 0.05 bohr from the largest charge nearer than that), scaled to the
cell budget; per axis the anchors are as above and the vertices equidistribute 1/spacing.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

GRADING = 3.0
MERGE_TOL = 0.3


@dataclass
class System:
    """Nuclei, box, cell counts, number of orbitals p and occupation f."""
    name: str
    Z: np.ndarray            # (M,) nuclear charges
    R: np.ndarray            # (M, 3) positions, bohr
    box_lo: np.ndarray       # (3,)
    box_hi: np.ndarray       # (3,)
    cells: tuple             # (Nx, Ny, Nz) hexahedra per axis
    p: int                   # number of orbitals
    occ: float               # electrons per orbital (f)

    def with_cells(self, cells, name=None) -> "System":
        return System(name or f"{self.name}@{'x'.join(map(str, cells))}", self.Z.copy(), self.R.copy(),
                      self.box_lo.copy(), self.box_hi.copy(), tuple(int(c) for c in cells), self.p, self.occ)

    def with_p(self, p, occ=None) -> "System":
        return System(self.name, self.Z.copy(), self.R.copy(), self.box_lo.copy(), self.box_hi.copy(),
                      self.cells, int(p), self.occ if occ is None else float(occ))


@dataclass
class Mesh:
    """Conforming P2 tetrahedral mesh.

    xyz       (n_nodes, 3) float64 node coordinates
    tet10     (n_tets, 10) int64 node ids; order: vertices 0..3, then the midpoints of
              edges 01, 02, 03, 12, 13, 23
    dirichlet (n_nodes,) uint8, 1 on the boundary of the box
    lattice   (Lx, Ly, Lz) lattice extents, node id = (a*Ly + b)*Lz + c
    """
    xyz: np.ndarray
    tet10: np.ndarray
    dirichlet: np.ndarray
    lattice: tuple
    axes: tuple = field(default=())   # per-axis lattice coordinates (length 2N+1 each)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tet10.shape[0])

    @property
    def n_free(self) -> int:
        return int(self.n_nodes - int(self.dirichlet.sum()))

    def free_ids(self) -> np.ndarray:
        """Global ids of the free (non-Dirichlet) nodes in increasing order."""
        return np.nonzero(self.dirichlet == 0)[0]


# ----------------------------------------------------------------------------- geometry

def lih() -> System:
    return System("lih", np.array([3.0, 1.0]), np.array([[0.0, 0.0, 0.0], [3.015, 0.0, 0.0]]),
                  np.full(3, -10.0), np.full(3, 10.0), (24, 24, 24), 2, 2.0)


def chain(n_carbon: int = 10, cells=(80, 44, 43), pad: float = 10.0) -> System:
    """Zigzag CkH(2k+2) chain in the z=0 plane.

    Carbon j sits at (j*d*sin(a/2), (j mod 2)*d*cos(a/2), 0) with d=2.9 bohr and a=111 deg.
    Each carbon carries two H in the plane x = x_Cj, placed symmetrically in +-z and tilted
    away from the backbone in y so that H-C-H = 109.5 deg.  Each terminal carbon gets one more
    H along the direction to the (absent) next backbone site, continuing the zigzag.
    """
    d, half = 2.9, np.deg2rad(111.0) / 2.0
    dh, hh = 2.06, np.deg2rad(109.5) / 2.0
    dx, dy = d * np.sin(half), d * np.cos(half)
    C = np.array([[j * dx, (j % 2) * dy, 0.0] for j in range(n_carbon)])
    H = []
    for j in range(n_carbon):
        s = -1.0 if j % 2 == 0 else 1.0            # away from the neighbours in y
        for sz in (1.0, -1.0):
            H.append(C[j] + dh * np.array([0.0, s * np.cos(hh), sz * np.sin(hh)]))
    for j, jv in ((0, -1), (n_carbon - 1, n_carbon)):
        virt = np.array([jv * dx, (jv % 2) * dy, 0.0])
        u = virt - C[j]
        H.append(C[j] + dh * u / np.linalg.norm(u))
    R = np.vstack([C, np.array(H)])
    Z = np.concatenate([np.full(n_carbon, 6.0), np.ones(len(H))])
    n_el = int(Z.sum())
    lo, hi = R.min(axis=0) - pad, R.max(axis=0) + pad
    return System(f"chain_c{n_carbon}", Z, R, lo, hi, tuple(cells), n_el // 2, 2.0)


def lattice60(cells=(80, 80, 80), pad: float = 10.0) -> System:
    """4x4x4 sites (2.9 bohr) minus the corners (0,0,0), (3,3,0), (3,0,3), (0,3,3).

    Z alternates 6, 1 over the remaining 60 sites in lexicographic order (30 C + 30 H =
    210 electrons); p = 210 singly occupied orbitals (f = 1) keep the system neutral.
    """
    drop = {(0, 0, 0), (3, 3, 0), (3, 0, 3), (0, 3, 3)}
    sites = [s for s in itertools.product(range(4), repeat=3) if s not in drop]
    R = 2.9 * np.array(sites, dtype=np.float64)
    Z = np.array([6.0 if i % 2 == 0 else 1.0 for i in range(len(sites))])
    lo, hi = R.min(axis=0) - pad, R.max(axis=0) + pad
    return System("lattice60", Z, R, lo, hi, tuple(cells), int(Z.sum()), 1.0)


def hydrogenic(Z: float = 1.0, half: float = 10.0, cells=(16, 16, 16), p: int = 1) -> System:
    """One nucleus of charge Z at the origin of the box [-half, half]^3."""
    return System(f"hyd_z{Z:g}", np.array([float(Z)]), np.zeros((1, 3)), np.full(3, -half),
                  np.full(3, half), tuple(cells), int(p), 2.0)


def random_nuclei(seed: int, cells=(16, 16, 16), pad: float = 8.0) -> System:
    """4-12 nuclei, Z drawn from {1,6,7,8}, positions uniform in a 6 bohr cube.

    p = ceil(sum Z / 2) doubly occupied orbitals (odd electron counts round up).
    """
    rng = np.random.default_rng(seed)
    m = int(rng.integers(4, 13))
    Z = rng.choice(np.array([1.0, 6.0, 7.0, 8.0]), size=m)
    R = rng.uniform(-3.0, 3.0, size=(m, 3))
    lo, hi = R.min(axis=0) - pad, R.max(axis=0) + pad
    return System(f"rand{seed}", Z, R, lo, hi, tuple(cells), int(np.ceil(Z.sum() / 2)), 2.0)


SYSTEMS = {"lih": lih, "chain": chain, "lattice60": lattice60}


# ----------------------------------------------------------------------------- mesh

def _merge(values, lo, hi, tol):
    vals = sorted(v for v in values if lo + tol < v < hi - tol)
    out = []
    group = []
    for v in vals:
        if group and v - group[-1] >= tol:
            out.append(float(np.mean(group)))
            group = []
        group.append(v)
    if group:
        out.append(float(np.mean(group)))
    return out


def _split_cells(lengths, n_total, n_min=2):
    lengths = np.asarray(lengths, dtype=np.float64)
    k = len(lengths)
    if n_total < n_min * k:
        raise ValueError(f"{n_total} cells cannot give {k} segments at least {n_min} each")
    ideal = n_total * lengths / lengths.sum()
    n = np.maximum(n_min, np.floor(ideal)).astype(np.int64)
    while n.sum() < n_total:
        n[int(np.argmax(ideal - n))] += 1
    while n.sum() > n_total:
        cand = np.where(n > n_min, n - ideal, -np.inf)
        n[int(np.argmax(cand))] -= 1
    return n


def axis_vertices(lo: float, hi: float, n_cells: int, nuclei_coords, g: float = GRADING,
                  tol: float = MERGE_TOL) -> np.ndarray:
    """Graded vertex coordinates (n_cells + 1 values) of one axis."""
    inner = _merge(list(nuclei_coords), lo, hi, tol)
    anchors = [lo] + inner + [hi]
    kinds = ["wall"] + ["nucleus"] * len(inner) + ["wall"]
    nseg = _split_cells(np.diff(anchors), n_cells)
    th = np.tanh(g)
    pts = [np.array([lo])]
    for s in range(len(anchors) - 1):
        a, b = anchors[s], anchors[s + 1]
        xi = np.arange(1, nseg[s] + 1) / nseg[s]
        ka, kb = kinds[s], kinds[s + 1]
        if ka == "wall" and kb == "nucleus":
            x = a + (b - a) * np.tanh(g * xi) / th
        elif ka == "nucleus" and kb == "wall":
            x = b + (a - b) * np.tanh(g * (1.0 - xi)) / th
        elif ka == "nucleus" and kb == "nucleus":
            x = a + (b - a) * 0.5 * (1.0 + np.tanh(g * (2.0 * xi - 1.0)) / th)
        else:
            x = a + (b - a) * xi
        x[-1] = b
        pts.append(x)
    return np.concatenate(pts)


GAMMA1, GAMMA2 = 0.125, 8.0      # Sec. 5.1: gamma_1 = 0.125, gamma_2 = 8 (the smaller molecules)


def mesh_size_1d(x, coords, Z, gamma1=GAMMA1, gamma2=GAMMA2):
    """Eq. (meshsizefunction) along one axis: min_j gamma1 Z_j^(-2/5) |x - X_j|^(6/5), capped at gamma2."""
    x = np.asarray(x, dtype=np.float64)
    h = np.full(x.shape, float(gamma2))
    for X, z in zip(coords, Z):
        h = np.minimum(h, gamma1 * float(z) ** -0.4 * np.abs(x - float(X)) ** 1.2)
    return h


MSF_R0 = 0.05                    # bohr: the size function is held at its value there nearer a nucleus


def axis_vertices_msf(lo: float, hi: float, n_cells: int, nuclei_coords, Z, gamma1: float = GAMMA1,
                      gamma2: float = GAMMA2, r0: float = MSF_R0, tol: float = MERGE_TOL,
                      samples: int = 200001) -> np.ndarray:
    """Vertex coordinates (n_cells + 1 values) of one axis graded by the mesh-size function.

    The spacing is C max(h(x), h(r0)) with h the size function of Eq. (meshsizefunction) along the
    axis (largest charge for h(r0)) and C the one scale that spends exactly the cell budget (the
    paper's sizes are those of an unstructured mesh; a tensor-product grid of the same local sizes
    would need far more cells, so the shape is kept and the scale fitted).  Cells go to the
    segments between anchors in proportion to the integral of 1/spacing and equidistribute it
    inside each segment.
    """
    xs = np.linspace(lo, hi, samples)
    zmax = float(np.max(Z)) if len(Z) else 1.0
    shape = np.maximum(mesh_size_1d(xs, nuclei_coords, Z, gamma1, gamma2), gamma1 * zmax ** -0.4 * r0 ** 1.2)
    dens = 1.0 / shape
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(xs))])
    # the scale C only stretches the cumulative count, so equidistribution does not depend on it
    inner = _merge(list(nuclei_coords), lo, hi, tol)
    anchors = [lo] + inner + [hi]
    ca = np.interp(anchors, xs, cum)
    nseg = _split_cells(np.diff(ca), n_cells)
    pts = [np.array([lo])]
    for sgm in range(len(anchors) - 1):
        targets = ca[sgm] + (ca[sgm + 1] - ca[sgm]) * np.arange(1, nseg[sgm] + 1) / nseg[sgm]
        x = np.interp(targets, cum, xs)
        x[-1] = anchors[sgm + 1]
        pts.append(x)
    return np.concatenate(pts)


# Kuhn split: one tetrahedron per ordering of the three axes.
KUHN_PERMS = tuple(itertools.permutations((0, 1, 2)))
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def make_mesh(system: System, g: float = GRADING, grading: str = "tanh") -> Mesh:
    """The P2 mesh of a system: tanh grading (default) or the mesh-size function ("msf")."""
    axes = []
    for d in range(3):
        if grading == "msf":
            v = axis_vertices_msf(float(system.box_lo[d]), float(system.box_hi[d]), int(system.cells[d]),
                                  system.R[:, d], system.Z)
        elif grading == "tanh":
            v = axis_vertices(float(system.box_lo[d]), float(system.box_hi[d]), int(system.cells[d]),
                              system.R[:, d], g)
        else:
            raise ValueError(f"unknown grading {grading}")
        lat = np.empty(2 * len(v) - 1)
        lat[0::2] = v
        lat[1::2] = 0.5 * (v[:-1] + v[1:])
        axes.append(lat)
    Lx, Ly, Lz = (len(a) for a in axes)
    A, Bc, C = np.meshgrid(axes[0], axes[1], axes[2], indexing="ij")
    xyz = np.stack([A.ravel(), Bc.ravel(), C.ravel()], axis=1)

    Nx, Ny, Nz = system.cells
    hi_, hj, hk = np.meshgrid(np.arange(Nx), np.arange(Ny), np.arange(Nz), indexing="ij")
    base = np.stack([2 * hi_.ravel(), 2 * hj.ravel(), 2 * hk.ravel()], axis=1)  # (nhex, 3) lattice coords
    nhex = base.shape[0]

    def gid(lc):
        return (lc[..., 0] * Ly + lc[..., 1]) * Lz + lc[..., 2]

    tets = np.empty((nhex, 6, 10), dtype=np.int64)
    eye2 = 2 * np.eye(3, dtype=np.int64)
    for t, perm in enumerate(KUHN_PERMS):
        v0 = base
        v1 = v0 + eye2[perm[0]]
        v2 = v1 + eye2[perm[1]]
        v3 = v0 + 2
        verts = [v0, v1, v2, v3]
        for a in range(4):
            tets[:, t, a] = gid(verts[a])
        for e, (a, b) in enumerate(EDGES):
            tets[:, t, 4 + e] = gid((verts[a] + verts[b]) // 2)
    tet10 = tets.reshape(-1, 10)

    la, lb, lc = np.meshgrid(np.arange(Lx), np.arange(Ly), np.arange(Lz), indexing="ij")
    bnd = ((la == 0) | (la == Lx - 1) | (lb == 0) | (lb == Ly - 1) | (lc == 0) | (lc == Lz - 1))
    return Mesh(xyz, tet10, bnd.ravel().astype(np.uint8), (Lx, Ly, Lz), tuple(axes))


def initial_block(n_free: int, p: int, seed: int = 0) -> np.ndarray:
    """Seeded Gaussian starting block V (n_free x p, row-major float64)."""
    return np.random.default_rng(seed).standard_normal((n_free, p))


def sizes(system: System) -> dict:
    """Closed-form sizes of the mesh a system produces (no mesh is built)."""
    Nx, Ny, Nz = system.cells
    return {"n": (2 * Nx - 1) * (2 * Ny - 1) * (2 * Nz - 1),
            "n_nodes": (2 * Nx + 1) * (2 * Ny + 1) * (2 * Nz + 1),
            "n_tets": 6 * Nx * Ny * Nz, "n_q": 24 * Nx * Ny * Nz}
