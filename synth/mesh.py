"""Seeded perturbed lattice meshes of [0,1]^3 with random numbering and orientation.

Recipe (the mesh family the solver is exercised on):
  * an (E+1)^3 lattice of vertices on [0,1]^3, spacing h = 1/E;
  * every coordinate moved by U(-a*h, a*h); on the boundary only the
    coordinates tangent to the boundary move, so corners stay fixed, edge
    vertices slide along their edge and the domain stays exactly [0,1]^3;
  * vertices and hexes renumbered by random permutations;
  * every hex's 8-vertex list re-expressed in one of the 24 proper rotations
    of the reference cube (orientation preserving, so the Jacobian sign is kept).
Hex vertex order is the VTK/gmsh one: corner c has reference signs
VTK_CORNER_BITS[c] in (xi, eta, zeta), 0 = -1 and 1 = +1.
"""
from dataclasses import dataclass
import itertools
import numpy as np

# reference-cube bits (xi, eta, zeta) of each VTK hex corner
VTK_CORNER_BITS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                            [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)


def _corner_index_of_bits():
    lut = np.zeros((2, 2, 2), dtype=np.int64)
    for c, (a, b, d) in enumerate(VTK_CORNER_BITS):
        lut[a, b, d] = c
    return lut


_CORNER_OF_BITS = _corner_index_of_bits()


def _proper_rotations():
    """The 24 signed permutation matrices with determinant +1."""
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                mats.append(R)
    return np.array(mats)


PROPER_ROTATIONS = _proper_rotations()


def _rotation_corner_maps():
    """For each proper rotation R, the map new-corner -> old-corner.

    A new local corner with sign vector s is the old corner with sign vector R s.
    """
    maps = np.zeros((len(PROPER_ROTATIONS), 8), dtype=np.int64)
    signs = 2 * VTK_CORNER_BITS - 1
    for r, R in enumerate(PROPER_ROTATIONS):
        for c in range(8):
            s_old = R @ signs[c]
            b = (s_old + 1) // 2
            maps[r, c] = _CORNER_OF_BITS[b[0], b[1], b[2]]
    return maps


_ROT_MAPS = _rotation_corner_maps()


@dataclass
class HexMesh:
    """An all-hex mesh: vertex coordinates (n_vert x 3, float64) and hex
    connectivity (n_hex x 8, int64, VTK corner order)."""
    xyz: np.ndarray
    hex2vert: np.ndarray
    E: int = 0
    a: float = 0.0
    seed: int = 0

    @property
    def n_vert(self):
        return self.xyz.shape[0]

    @property
    def n_hex(self):
        return self.hex2vert.shape[0]


def lattice_hex_mesh(E, a=0.0, seed=0, renumber=True, rotate=True, box=(1.0, 1.0, 1.0)):
    """Perturbed Ex x Ey x Ez hex lattice of the box [0,bx]x[0,by]x[0,bz].

    Parameters: E hexes per direction (an int, or (Ex, Ey, Ez) for a rod or slab), a the
    perturbation amplitude as a fraction of the spacing, seed for numpy.random.default_rng.
    Returns a HexMesh.
    """
    Es = np.array([int(E)] * 3 if np.ndim(E) == 0 else [int(v) for v in E], dtype=np.int64)
    if Es.shape != (3,) or Es.min() < 1:
        raise ValueError("E must be >= 1 (or three counts >= 1)")
    rng = np.random.default_rng(seed)
    nx, ny, nz = (Es + 1).tolist()
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)   # lattice index of vertex
    vid_of = lambda i, j, k: i + nx * (j + ny * k)
    order = np.argsort(vid_of(lat[:, 0], lat[:, 1], lat[:, 2]))
    lat = lat[order]                                             # vertex id = i + nx*(j + ny*k)
    h = np.array(box, dtype=np.float64) / Es
    xyz = lat.astype(np.float64) * h
    d = rng.uniform(-a, a, size=xyz.shape) * h
    on_bnd = (lat == 0) | (lat == Es)
    d[on_bnd] = 0.0                                              # tangential-only on the boundary
    xyz = xyz + d

    ci, cj, ck = np.meshgrid(np.arange(Es[0]), np.arange(Es[1]), np.arange(Es[2]), indexing="ij")
    cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    hexes = np.empty((cells.shape[0], 8), dtype=np.int64)
    for c, (ba, bb, bc) in enumerate(VTK_CORNER_BITS):
        hexes[:, c] = vid_of(cells[:, 0] + ba, cells[:, 1] + bb, cells[:, 2] + bc)

    if rotate:
        rot = rng.integers(0, len(PROPER_ROTATIONS), size=hexes.shape[0])
        hexes = np.take_along_axis(hexes, _ROT_MAPS[rot], axis=1)
    if renumber:
        vperm = rng.permutation(xyz.shape[0])          # new id of old vertex
        new_xyz = np.empty_like(xyz)
        new_xyz[vperm] = xyz
        xyz = new_xyz
        hexes = vperm[hexes]
        eperm = rng.permutation(hexes.shape[0])
        hexes = hexes[eperm]
    return HexMesh(xyz=np.ascontiguousarray(xyz), hex2vert=np.ascontiguousarray(hexes),
                   E=int(Es[0]) if np.ndim(E) == 0 else tuple(Es.tolist()), a=float(a), seed=int(seed))


def split_triangle_hex_mesh(N, layers, a=0.0, seed=0, height=1.0, rotate=True, renumber=True):
    """All-hex mesh with irregular edge valences on [0,1]^2 x [0,height].

    The unit square is cut into N x N cells, each cell into two triangles (diagonal direction
    drawn at random), and each triangle into three quads through its centroid and edge
    midpoints; the quads are extruded through `layers` layers. Interior vertical edges then
    have valence 3 (centroids), 4 (edge midpoints) or 6 to 8 (cell corners). Interior vertices
    move by U(-a h, a h) in x and y (h = 1/N, along-boundary only on the boundary) and by
    U(-a dz, a dz) in z off the top and bottom. Random proper rotations of the corner lists
    and random renumbering as in lattice_hex_mesh. The split quads have small corners: up to
    a = 0.1 every element keeps a positive Jacobian (smallest GLL-corner |J| about a fifth of
    the median over seeds 1..11); at a = 0.2 some invert. Returns a HexMesh.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / N
    pts = {}
    def pid(key, xy):
        if key not in pts:
            pts[key] = (len(pts), xy)
        return pts[key][0]
    quads = []
    for i in range(N):
        for j in range(N):
            c = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            corner = [pid(("v", a_, b_), (a_ * h, b_ * h)) for a_, b_ in c]
            tris = [(0, 1, 2), (0, 2, 3)] if rng.random() < 0.5 else [(0, 1, 3), (1, 2, 3)]
            for t in tris:
                tv = [c[k] for k in t]
                ids = [corner[k] for k in t]
                xy = np.array([[a_ * h, b_ * h] for a_, b_ in tv])
                cen = pid(("c", i, j, t), tuple(xy.mean(axis=0)))
                mids = []
                for k in range(3):
                    e = tuple(sorted((tv[k], tv[(k + 1) % 3])))
                    mids.append(pid(("m",) + e, tuple((xy[k] + xy[(k + 1) % 3]) / 2)))
                for k in range(3):      # quad: vertex k, midpoint k, centroid, midpoint k-1
                    q = [ids[k], mids[k], cen, mids[k - 1]]
                    quads.append(q)
    n2 = len(pts)
    xy = np.zeros((n2, 2))
    for key, (k, v) in pts.items():
        xy[k] = v
    # counter-clockwise orientation for every quad
    for qi, q in enumerate(quads):
        p0, p1, p2, p3 = xy[q]
        area = 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1])
                      + (p2[0] - p0[0]) * (p3[1] - p0[1]) - (p3[0] - p0[0]) * (p2[1] - p0[1]))
        if area < 0:
            quads[qi] = [q[0], q[3], q[2], q[1]]
    on_x = (np.abs(xy[:, 0]) < 1e-12) | (np.abs(xy[:, 0] - 1) < 1e-12)
    on_y = (np.abs(xy[:, 1]) < 1e-12) | (np.abs(xy[:, 1] - 1) < 1e-12)
    d = rng.uniform(-a, a, size=xy.shape) * h * 0.5
    d[on_x, 0] = 0.0
    d[on_y, 1] = 0.0
    xy = xy + d
    dz = height / layers
    zs = np.arange(layers + 1) * dz
    zpert = rng.uniform(-a, a, size=(layers + 1, n2)) * dz
    zpert[0] = zpert[-1] = 0.0
    xyz = np.zeros(((layers + 1) * n2, 3))
    for L in range(layers + 1):
        xyz[L * n2:(L + 1) * n2, :2] = xy
        xyz[L * n2:(L + 1) * n2, 2] = zs[L] + zpert[L]
    hexes = []
    for L in range(layers):
        for q in quads:
            lo = [L * n2 + v for v in q]
            hi = [(L + 1) * n2 + v for v in q]
            hexes.append(lo + hi)        # VTK order: bottom quad counter-clockwise, then top
    hexes = np.array(hexes, dtype=np.int64)
    if rotate:
        rot = rng.integers(0, len(PROPER_ROTATIONS), size=hexes.shape[0])
        hexes = np.take_along_axis(hexes, _ROT_MAPS[rot], axis=1)
    if renumber:
        vperm = rng.permutation(xyz.shape[0])
        new_xyz = np.empty_like(xyz)
        new_xyz[vperm] = xyz
        xyz = new_xyz
        hexes = vperm[hexes]
        hexes = hexes[rng.permutation(hexes.shape[0])]
    return HexMesh(xyz=np.ascontiguousarray(xyz), hex2vert=np.ascontiguousarray(hexes), E=N, a=float(a),
                   seed=int(seed))


def manufactured_u(xyz):
    """u*(x,y,z) = sin(pi x) sin(pi y) sin(pi z); zero on the boundary of [0,1]^3."""
    x = np.asarray(xyz, dtype=np.float64)
    return np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])


def manufactured_s(xyz, lam):
    """Source s = lam*u* - laplacian(u*) = (3 pi^2 + lam) u* for the manufactured u*."""
    return (3.0 * np.pi ** 2 + lam) * manufactured_u(xyz)


def moving_source(xyz, t, q0=1000.0, width=0.25, start=(0.5, 0.5, 1.0), velocity=(0.0, 0.0, 2.0)):
    """Volume heat source Q(x, t) = q0 exp(-|x - c(t)|^2 / (2 width^2)), c(t) = start + velocity t."""
    x = np.asarray(xyz, dtype=np.float64)
    c = np.asarray(start, dtype=np.float64) + np.asarray(velocity, dtype=np.float64) * t
    return q0 * np.exp(-np.sum((x - c) ** 2, axis=1) / (2.0 * width ** 2))


def gaussian_load(n, seed):
    """Seeded N(0,1) load vector of length n."""
    return np.random.default_rng(seed).standard_normal(n)
