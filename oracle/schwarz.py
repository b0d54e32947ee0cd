"""Fine-scale overlapping additive Schwarz preconditioner P^f.

Paper: Sec. 4.2 (local preconditioner), Eq. subd, the extended 1D pencil matrix,
Eq. z and the additive update of P^f.
Readings:
  * Extended 1D pencil: the element plus one node on each side; the matrices are
    the rows/columns -1..n+1 of the three-element 1D assembly (stiffness
    d_ij = sum_m rho_m phi_i'(t_m) phi_j'(t_m), mass diag(rho)), i.e. homogeneous
    Dirichlet beyond -1 and n+1. The neighbours are assumed to have the same h.
  * "Suitable boundary conditions" (Sec. 4.2) at a side with no neighbour that is not
    Dirichlet (a natural-boundary face): that side's neighbour is left out of the
    assembly, so the end node keeps its own element's share alone, and the row beyond it
    is decoupled (pencil_variant; Problem(pencils="boundary"), the default). Dirichlet
    faces keep the extended pencil (their nodes are masked).
  * The eigen-form is the generalised problem K S = M S Lambda with S^T M S = I, so
    z = 8/(hx hy hz) (S x S x S) diag[1/(4(l_a/hx^2 + l_b/hy^2 + l_c/hz^2) + c)]
        (S^T x S^T x S^T) r,
    which is Eq. z with M^{-1} cancelled (the printed V/V^{-1} indices are inconsistent).
  * A patch node with exactly one index in {-1, n+1} is the face-neighbour's node one
    layer inside it, next to the shared face node; nodes with two or more indices
    outside 0..n, and layers beyond a boundary face, are absent (r = 0, z dropped).
    With patch = "full" (fill_edges_corners) the edge and corner layers are filled too,
    giving the (n+3)^3 nodes per subdomain that Sec. 4.2 counts.
  * h_x, h_y, h_z: mean length of the element's 4 edges along xi, eta, zeta.
  * No overlap weights: the corrections are summed (the paper's P^f, the default). Option:
    weights w_N = c_N^(-1/2), c_N the number of patches containing node N, applied to the
    residual before the patch solves and to the sum after them, W P^f W (symmetric).
Pinned by: the pencil matrices equal the printed extended matrix pattern, the
fast-diagonalisation solve equals a dense solve of the Kronecker-sum box matrix,
S^T M S = I and K S = M S Lambda (scipy eigh), symmetry and positivity of P^f; on an
unperturbed lattice the filled box nodes sit where the element's (affine) map, extended
one GLL step beyond each face, puts them; the variant pencil without free sides is the
extended one, and on one undistorted, insulated hex P^f = A^-1.
"""
import numpy as np
import scipy.linalg

from .numbering import HEX_FACES


def pencil_matrices(Dh, rho):
    """Extended 1D stiffness K and mass M (size n+3, rows -1..n+1) by three-element assembly."""
    n = len(rho) - 1
    d = Dh.T @ np.diag(rho) @ Dh                 # d_ij = sum_m rho_m phi_i'(t_m) phi_j'(t_m)
    N = 3 * n + 1                                # nodes -n .. 2n
    Kf = np.zeros((N, N))
    Mf = np.zeros(N)
    for el in range(3):
        o = el * n
        Kf[o:o + n + 1, o:o + n + 1] += d
        Mf[o:o + n + 1] += rho
    keep = np.arange(n - 1, 2 * n + 2)           # global nodes -1 .. n+1
    return Kf[np.ix_(keep, keep)], np.diag(Mf[keep])


def pencil_variant(Dh, rho, low_free, high_free):
    """Extended 1D pencil of an element with no neighbour on its low and/or high side (a
    free, natural-boundary side): only the present elements are assembled, so the end node
    on a free side keeps its own element's share alone; the row beyond a free side has no
    node and is decoupled (K = M = 1 there, and its data is always zero)."""
    n = len(rho) - 1
    d = Dh.T @ np.diag(rho) @ Dh
    N = 3 * n + 1
    Kf = np.zeros((N, N))
    Mf = np.zeros(N)
    for el, present in ((0, not low_free), (1, True), (2, not high_free)):
        if present:
            o = el * n
            Kf[o:o + n + 1, o:o + n + 1] += d
            Mf[o:o + n + 1] += rho
    keep = np.arange(n - 1, 2 * n + 2)
    K, m = Kf[np.ix_(keep, keep)], Mf[keep].copy()
    for row, free in ((0, low_free), (n + 2, high_free)):
        if free:
            K[row, :] = 0.0
            K[:, row] = 0.0
            K[row, row] = 1.0
            m[row] = 1.0
    return K, np.diag(m)


def free_sides(nb_elem, l2g, mask):
    """free[e, axis, side]: the element has no neighbour there and the face is not wholly
    masked (a natural-boundary face)."""
    E, p = l2g.shape[0], l2g.shape[1]
    n = p - 1
    free = np.zeros((E, 3, 2), dtype=bool)
    for f, (ax, sd) in enumerate(HEX_FACES):
        sl = [slice(None)] * 3
        sl[ax] = 0 if sd == 0 else n
        face = l2g[(slice(None),) + tuple(sl)].reshape(E, -1)
        free[:, ax, sd] = (nb_elem[:, f] < 0) & ~np.all(mask[face] > 0, axis=1)
    return free


def pencil_eig(K, M):
    """Generalised eigenpairs K S = M S diag(ev), S^T M S = I (scipy.linalg.eigh)."""
    ev, S = scipy.linalg.eigh(K, M)
    return ev, S


def patch_table(l2g, nb_elem, nb_face):
    """ip[e, I, J, K] = global node of extended-box node (I-1, J-1, K-1), or -1 if absent."""
    E, p = l2g.shape[0], l2g.shape[1]
    n = p - 1
    P = n + 3
    Gn = int(l2g.max()) + 1
    ip = -np.ones((E, P, P, P), dtype=np.int64)
    ip[:, 1:n + 2, 1:n + 2, 1:n + 2] = l2g
    # lookup (element, global node) -> local (i, j, k)
    keys = (np.arange(E)[:, None] * Gn + l2g.reshape(E, -1)).ravel()
    order = np.argsort(keys)
    skeys = keys[order]
    loc = np.stack(np.unravel_index(np.arange(p ** 3), (p, p, p)), axis=1)
    for f, (ax, sd) in enumerate(HEX_FACES):
        has = nb_elem[:, f] >= 0
        es = np.where(has)[0]
        if len(es) == 0:
            continue
        e2 = nb_elem[es, f]
        ax2 = np.array([HEX_FACES[g][0] for g in nb_face[es, f]])
        sd2 = np.array([HEX_FACES[g][1] for g in nb_face[es, f]])
        sl = [slice(None)] * 3
        sl[ax] = 0 if sd == 0 else n
        face_g = l2g[es][(slice(None),) + tuple(sl)]          # [m, p, p] global ids on the face
        q = (e2[:, None, None] * Gn + face_g)
        pos = np.searchsorted(skeys, q.ravel())
        assert np.all(skeys[pos] == q.ravel()), "face node not found in neighbour"
        lidx = order[pos] % (p ** 3)
        ijk2 = loc[lidx].reshape(face_g.shape + (3,))          # local coords in the neighbour
        step = np.where(sd2 == 0, 1, -1)
        ijk2 = ijk2.copy()
        rows = np.arange(len(es))
        ijk2[rows, :, :, ax2] += step[:, None, None]
        inner = l2g[e2[:, None, None], ijk2[..., 0], ijk2[..., 1], ijk2[..., 2]]
        dst = [slice(1, n + 2)] * 3
        dst[ax] = 0 if sd == 0 else P - 1
        ip[(es,) + tuple(dst)] = inner
    return ip


def fill_edges_corners(ip, l2g):
    """Full-box patches: the box nodes with two or three indices in {-1, n+1} (edge and corner
    layers), which `patch_table` leaves absent, taken from the GLL grid graph.

    The graph joins the global nodes that are adjacent along a local axis of some element.
    A box node with out-of-range axes S has, for each axis in S, a box neighbour one step
    back inside along that axis; the node is the one common graph neighbour of those that is
    not already in the element's box (edges first, then corners). Absent when a needed
    neighbour is absent or the common neighbour is not unique.
    """
    E, p = l2g.shape[0], l2g.shape[1]
    n = p - 1
    P = n + 3
    adj = {}
    for ax in range(3):
        a = np.moveaxis(l2g, ax + 1, 1)
        for x, y in zip(a[:, :-1].ravel().tolist(), a[:, 1:].ravel().tolist()):
            adj.setdefault(x, set()).add(y)
            adj.setdefault(y, set()).add(x)
    out = ip.copy()
    rng = range(-1, n + 2)
    out_of = lambda c: [d for d in range(3) if c[d] < 0 or c[d] > n]
    for level in (2, 3):
        for e in range(E):
            box = set(out[e][out[e] >= 0].tolist())
            for c in [(I, J, K) for K in rng for J in rng for I in rng]:
                S = out_of(c)
                if len(S) != level:
                    continue
                nbrs = []
                for d in S:
                    c2 = list(c)
                    c2[d] = 0 if c[d] < 0 else n
                    nbrs.append(int(out[e, c2[0] + 1, c2[1] + 1, c2[2] + 1]))
                if min(nbrs) < 0:
                    continue
                cand = set.intersection(*[adj.get(g, set()) for g in nbrs]) - box
                if len(cand) == 1:
                    g = cand.pop()
                    out[e, c[0] + 1, c[1] + 1, c[2] + 1] = g
                    box.add(g)
    return out


def fast_diag_solve(rp, S, ev, h, lam):
    """Eq. z: z = 8/(hx hy hz) S^{x3} diag^{-1} S^{T x3} r for patch arrays rp[e, P, P, P]."""
    scale = 8.0 / (h[:, 0] * h[:, 1] * h[:, 2])
    t = np.einsum("ia,eijk->eajk", S, rp)
    t = np.einsum("jb,eajk->eabk", S, t)
    t = np.einsum("kc,eabk->eabc", S, t)
    den = 4.0 * (ev[None, :, None, None] / h[:, 0, None, None, None] ** 2
                 + ev[None, None, :, None] / h[:, 1, None, None, None] ** 2
                 + ev[None, None, None, :] / h[:, 2, None, None, None] ** 2) + lam
    t = t / den * scale[:, None, None, None]
    t = np.einsum("kc,eabc->eabk", S, t)
    t = np.einsum("jb,eabk->eajk", S, t)
    return np.einsum("ia,eajk->eijk", S, t)


def box_matrix(K, M, h, lam):
    """Dense Kronecker-sum operator of one box, C order over (I, J, K)."""
    hx, hy, hz = h
    return 4.0 * (np.kron(K, np.kron(M, M)) / hx ** 2 + np.kron(M, np.kron(K, M)) / hy ** 2
                  + np.kron(M, np.kron(M, K)) / hz ** 2) + lam * np.kron(M, np.kron(M, M))


def fast_diag_solve_axes(rp, S3, ev3, h, lam):
    """Eq. z with its own pencil per axis: S3 = (Sx, Sy, Sz), ev3 = (evx, evy, evz)."""
    (Sx, Sy, Sz), (ex, ey, ez) = S3, ev3
    scale = 8.0 / (h[:, 0] * h[:, 1] * h[:, 2])
    t = np.einsum("ia,eijk->eajk", Sx, rp)
    t = np.einsum("jb,eajk->eabk", Sy, t)
    t = np.einsum("kc,eabk->eabc", Sz, t)
    den = 4.0 * (ex[None, :, None, None] / h[:, 0, None, None, None] ** 2
                 + ey[None, None, :, None] / h[:, 1, None, None, None] ** 2
                 + ez[None, None, None, :] / h[:, 2, None, None, None] ** 2) + lam
    t = t / den * scale[:, None, None, None]
    t = np.einsum("kc,eabc->eabk", Sz, t)
    t = np.einsum("jb,eabk->eajk", Sy, t)
    return np.einsum("ia,eajk->eijk", Sx, t)


def cover_weights(ip, G):
    """w_N = c_N^(-1/2), c_N the number of patches that contain node N (1 where none)."""
    present = ip >= 0
    cover = np.bincount(ip[present], minlength=G).astype(np.float64)
    return 1.0 / np.sqrt(np.where(cover > 0, cover, 1.0))


def apply_fine(r, ip, S, ev, h, lam, mask=None, variants=None, weights=None):
    """P^f r: restrict to every patch, solve each box, add the present nodes back. With
    variants = (var[E, 3] in 0..3 = low_free + 2 high_free, [(S, ev)] per variant), each
    element uses the pencil of its sides along each axis. With weights w (per node), the
    overlap-weighted sum W (sum_s R_s^T A_s^-1 R_s) W, W = diag(w), still symmetric."""
    Gn = r.shape[0]
    rm = r if mask is None else np.where(mask > 0, 0.0, r)
    if weights is not None:
        rm = rm * weights
    present = ip >= 0
    rp = np.where(present, rm[np.where(present, ip, 0)], 0.0)
    if variants is None:
        zp = fast_diag_solve(rp, S, ev, h, lam)
    else:
        var, table = variants
        zp = np.zeros_like(rp)
        for combo in {tuple(v) for v in var.tolist()}:
            sel = np.all(var == np.array(combo), axis=1)
            zp[sel] = fast_diag_solve_axes(rp[sel], [table[c][0] for c in combo], [table[c][1] for c in combo],
                                           h[sel], lam)
    z = np.bincount(ip[present], weights=zp[present], minlength=Gn)
    if weights is not None:
        z = z * weights
    if mask is not None:
        z = np.where(mask > 0, 0.0, z)
    return z


def apply_fine_abs(r, ip, S, ev, h, lam, mask=None):
    """Magnitude of every term of Eq. z (|S|, |r| and positive eigen-sums), summed over
    the patches: the reference magnitude for rounding bounds of a reduced-precision P^f."""
    Gn = r.shape[0]
    rm = np.abs(r) if mask is None else np.where(mask > 0, 0.0, np.abs(r))
    present = ip >= 0
    rp = np.where(present, rm[np.where(present, ip, 0)], 0.0)
    zp = fast_diag_solve(rp, np.abs(S), ev, h, lam)
    z = np.bincount(ip[present], weights=zp[present], minlength=Gn)
    if mask is not None:
        z = np.where(mask > 0, 0.0, z)
    return z
