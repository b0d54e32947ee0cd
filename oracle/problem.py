"""One screened-Poisson problem on a hex mesh, assembled from the oracle pieces.

Problem(mesh, n, lam, dirichlet=True) builds the numbering, geometry, the
Schwarz patches and eigen-tables, the coarse matrix and its AMG hierarchy, and
offers apply_A, apply_Pf, apply_Pc, apply_P (= P^c + P^f, Sec. 4), solve (Algorithm 1),
mass (m_N) and dense/sparse assembled matrices for small cases.
"""
import numpy as np
from scipy.sparse import csr_matrix

from . import gll, numbering, geometry, operator, schwarz, coarse, amg, pcg


class Problem:
    def __init__(self, mesh, n, lam, dirichlet=True, coarse_solver="amg", with_schwarz=True, patch="face",
                 pencils="boundary", weights="none"):
        self.mesh = mesh
        self.n = n
        self.lam = float(lam)
        self.t, self.rho = gll.gll_nodes_weights(n)
        self.Dh = gll.derivative_matrix(n)
        self.l2g, self.coords = numbering.local_to_global(mesh, self.t)
        self.G = self.coords.shape[0]
        self.xyz_e = mesh.xyz[mesh.hex2vert]
        self.Gf, self.m_loc, self.detJ = geometry.geometric_factors(self.xyz_e, self.t, self.rho)
        if self.detJ.min() <= 0:
            raise ValueError("non-positive Jacobian")
        self.m_N = np.bincount(self.l2g.ravel(), weights=self.m_loc.ravel(), minlength=self.G)
        self.nb_elem, self.nb_face = numbering.face_neighbours(mesh)
        if dirichlet:
            self.mask = numbering.boundary_mask(self.l2g, self.nb_elem, self.G)
        else:
            self.mask = np.zeros(self.G, dtype=np.uint8)
        self.coarse_solver = coarse_solver
        self.patch = patch
        self.pencils = pencils
        self.weights = weights
        if with_schwarz:
            self._setup_schwarz()
        if coarse_solver is not None:
            self._setup_coarse()

    # --- fine scale ---------------------------------------------------------
    def _setup_schwarz(self):
        K, M = schwarz.pencil_matrices(self.Dh, self.rho)
        self.K1, self.M1 = K, M
        self.ev, self.S = schwarz.pencil_eig(K, M)
        self.h = geometry.element_box_sizes(self.xyz_e)
        self.ip = schwarz.patch_table(self.l2g, self.nb_elem, self.nb_face)
        if self.patch == "full":
            self.ip = schwarz.fill_edges_corners(self.ip, self.l2g)
        self.variants = None
        if self.pencils == "boundary":
            free = schwarz.free_sides(self.nb_elem, self.l2g, self.mask)
            var = free[:, :, 0].astype(np.int64) + 2 * free[:, :, 1].astype(np.int64)
            table = []
            for v in range(4):
                Kv, Mv = schwarz.pencil_variant(self.Dh, self.rho, bool(v & 1), bool(v & 2))
                ev, S = schwarz.pencil_eig(Kv, Mv)
                table.append((S, ev))
            self.variants = (var, table)
        self.w = schwarz.cover_weights(self.ip, self.G) if self.weights == "cover" else None

    # --- coarse scale -------------------------------------------------------
    def _setup_coarse(self):
        self.B = coarse.vandermonde(self.t)
        nv = self.mesh.n_vert
        cl2g = coarse.coarse_l2g(self.mesh.hex2vert)
        t1, rho1 = gll.gll_nodes_weights(1)
        J1 = geometry.jacobians(self.xyz_e, t1)
        Ae = operator.element_matrices(t1, rho1, J1, self.lam)
        A0full = operator.assemble(Ae, cl2g, nv)
        # vertex -> its global GLL node, to read the Dirichlet mask on vertices
        corner_node = np.zeros((self.mesh.n_hex, 8), dtype=np.int64)
        n = self.n
        from synth import VTK_CORNER_BITS
        for c, (a, b, d) in enumerate(VTK_CORNER_BITS):
            corner_node[:, c] = self.l2g[:, a * n, b * n, d * n]
        vdof = np.zeros(nv, dtype=np.int64)
        vdof[self.mesh.hex2vert.ravel()] = corner_node.ravel()
        self.vert_dof = vdof
        self.free_vert = np.where(self.mask[vdof] == 0)[0]        # ascending vertex id
        fv = self.free_vert
        self.A0 = csr_matrix(A0full[fv][:, fv])
        if self.coarse_solver in ("amg", "kcycle"):
            self.amg = amg.AMG(self.A0, kind="vcycle" if self.coarse_solver == "amg" else "kcycle")
            self.P0 = self.amg.apply
        elif self.coarse_solver == "exact":
            A0d = self.A0.toarray()
            self.P0 = lambda R: np.linalg.solve(A0d, R)
        else:
            raise ValueError(self.coarse_solver)

    # --- operators ----------------------------------------------------------
    def apply_A(self, x):
        return operator.matfree_apply(x, self.l2g, self.Dh, self.Gf, self.m_loc, self.lam, self.mask)

    def apply_Pf(self, r):
        return schwarz.apply_fine(r, self.ip, self.S, self.ev, self.h, self.lam, self.mask, self.variants, self.w)

    def apply_Pc(self, r):
        rm = np.where(self.mask > 0, 0.0, r)
        R = coarse.restrict(rm, self.l2g, self.m_loc, self.m_N, self.B, self.mesh.hex2vert,
                            self.mesh.n_vert)
        Zf = self.P0(R[self.free_vert])
        Z = np.zeros(self.mesh.n_vert)
        Z[self.free_vert] = Zf
        z = coarse.prolong(Z, self.l2g, self.m_loc, self.m_N, self.B, self.mesh.hex2vert)
        return np.where(self.mask > 0, 0.0, z)

    def apply_P(self, r):
        return self.apply_Pc(r) + self.apply_Pf(r)

    def load(self, s):
        """b = m_N s (lumped GLL load), masked."""
        return np.where(self.mask > 0, 0.0, self.m_N * s)

    def solve(self, b, rtol=1e-8, maxit=1000, precond="two-scale"):
        bm = np.where(self.mask > 0, 0.0, b)
        P = {"two-scale": self.apply_P, "fine": self.apply_Pf, "none": lambda r: r.copy()}[precond]
        flexible = self.coarse_solver == "kcycle" and precond == "two-scale"   # the K-cycle is nonlinear
        return (pcg.fpcg if flexible else pcg.pcg)(self.apply_A, P, bm, rtol, maxit)

    def assembled(self):
        """Sparse A_D by explicit element-matrix assembly (small meshes only)."""
        J = geometry.jacobians(self.xyz_e, self.t)
        Ae = operator.element_matrices(self.t, self.rho, J, self.lam)
        A = operator.assemble(Ae, self.l2g, self.G)
        return operator.apply_dirichlet(A, self.mask)
