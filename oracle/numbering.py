"""Global numbering of GLL nodes, scatter and gather (Sec. 2.2, Eq. scatter, Eq. gather).

The oracle numbers nodes by *position*: two local GLL nodes are the same global
node exactly when the trilinear maps of their elements send them to the same
physical point (conforming meshes). Coincident points are found with a k-d tree
(scipy) and merged with connected components. This is independent of any
topological (vertex/edge/face) construction.
Boundary nodes are those lying on a hex face that belongs to one hex only.
Pinned by: count of global nodes = (nE+1)^3 on lattice meshes, scatter/gather
adjointness, boundary nodes lie on the faces of the unit cube.
"""
import numpy as np
from scipy.spatial import cKDTree
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from synth import VTK_CORNER_BITS


def trilinear_points(xyz_e, t):
    """Physical coordinates x^e(t_i, t_j, t_k) of all GLL nodes: [E, p, p, p, 3] (i<->xi, j<->eta, k<->zeta)."""
    s = 2 * VTK_CORNER_BITS - 1                     # corner signs in (xi, eta, zeta)
    p = len(t)
    out = np.zeros((xyz_e.shape[0], p, p, p, 3))
    for c in range(8):
        Nx = (1 + s[c, 0] * t) / 2
        Ny = (1 + s[c, 1] * t) / 2
        Nz = (1 + s[c, 2] * t) / 2
        N = Nx[:, None, None] * Ny[None, :, None] * Nz[None, None, :]
        out += N[None, :, :, :, None] * xyz_e[:, c, None, None, None, :]
    return out


def number_by_position(points, tol):
    """Label points (L x 3) so that points closer than tol share a label; labels 0..G-1."""
    tree = cKDTree(points)
    pairs = tree.query_pairs(tol, output_type="ndarray")
    L = points.shape[0]
    graph = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(L, L))
    n_comp, labels = connected_components(graph, directed=False)
    return n_comp, labels


def local_to_global(mesh, t):
    """l2g[e, i, j, k] (int64) and the coordinates of every global node (G x 3)."""
    xyz_e = mesh.xyz[mesh.hex2vert]
    pts = trilinear_points(xyz_e, t)
    L = pts.shape[0] * len(t) ** 3
    flat = pts.reshape(L, 3)
    span = np.ptp(mesh.xyz, axis=0).max()
    G, labels = number_by_position(flat, 1e-9 * span)
    l2g = labels.reshape(pts.shape[:4])
    coords = np.zeros((G, 3))
    coords[labels] = flat
    return l2g, coords


HEX_FACES = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]   # (normal axis, side 0=low/1=high)


def face_corners(axis, side):
    """VTK corner indices of a hex face given by normal axis and side."""
    return [c for c in range(8) if VTK_CORNER_BITS[c, axis] == side]


def face_neighbours(mesh):
    """For every (element, face) the neighbouring element and its face index, or -1.

    Faces are matched by their set of 4 vertex ids. Returns nb_elem[E, 6], nb_face[E, 6].
    """
    E = mesh.n_hex
    keys = {}
    nb_elem = -np.ones((E, 6), dtype=np.int64)
    nb_face = -np.ones((E, 6), dtype=np.int64)
    for f, (ax, sd) in enumerate(HEX_FACES):
        corners = face_corners(ax, sd)
        fv = np.sort(mesh.hex2vert[:, corners], axis=1)
        for e in range(E):
            key = tuple(fv[e])
            keys.setdefault(key, []).append((e, f))
    for key, lst in keys.items():
        if len(lst) > 2:
            raise ValueError("non-manifold face shared by more than two hexes")
        if len(lst) == 2:
            (e1, f1), (e2, f2) = lst
            nb_elem[e1, f1], nb_face[e1, f1] = e2, f2
            nb_elem[e2, f2], nb_face[e2, f2] = e1, f1
    return nb_elem, nb_face


def boundary_mask(l2g, nb_elem, G):
    """1 for every global node that lies on a face owned by a single hex."""
    n = l2g.shape[1] - 1
    mask = np.zeros(G, dtype=np.uint8)
    for f, (ax, sd) in enumerate(HEX_FACES):
        idx = 0 if sd == 0 else n
        sl = [slice(None)] * 4
        sl[1 + ax] = idx
        on_face = l2g[tuple(sl)]                      # [E, p, p]
        bnd = nb_elem[:, f] < 0
        mask[on_face[bnd].ravel()] = 1
    return mask


def scatter(x, l2g):
    """u_{ijk;e} = u_{I(ijk;e)} (Eq. scatter)."""
    return x[l2g]


def gather(r_local, l2g, G):
    """r_N = sum of the local copies of node N (Eq. gather)."""
    return np.bincount(l2g.ravel(), weights=r_local.ravel(), minlength=G)
