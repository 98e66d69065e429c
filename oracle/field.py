"""IFE field solve (oracle; test infrastructure only).

Follows arXiv:2011.10214 Sec. 2.1 (Eqs. 2.1-2.5: the elliptic interface
problem, Dirichlet / Neumann boundaries, [phi] = 0, [eps d_n phi] = q) and
Sec. 2.5 (a PCG matrix solve is the innermost iteration level; stopping on the
relative residual, Sec. 3.2, Sec. 4, Sec. 5.2.2).

Weak form (derived from Eqs. 2.1, 2.4, 2.5 by integrating by parts on each
side of the interface): a(phi, v) = (rho, v) - int_Gamma q v.  The
non-homogeneous IFE solution is phi_h = u_h + phi_J with phi_J the element-wise
jump function (zero at every node, flux jump q on interface tets) and u_h in
the IFE space solving a_h(u_h, psi_i) = F_i - int_Gamma q psi_i - a_h(phi_J, psi_i).

Readings where the paper is silent:
  * load vector F_i = sum_p q_p S_i(x_p), S_i the trilinear (Q1) weight of the
    PIC cell -- the scatter result itself, which conserves charge exactly;
  * surface charge: each cut PIC cell c collects the charge Q_c of the
    particles that hit the object there; sigma_c = Q_c / A_c (A_c the Gamma_h
    area in the cell) and q_T = -sigma_c on every interface tet of the cell
    (Gauss: [eps E . n] = sigma, E = -grad phi);
  * preconditioner: Jacobi; stopping test ||r||_2 <= tol ||b||_2 with b the
    right-hand side after the Dirichlet lift; warm start from the previous phi;
  * node field: E_i = -(sum |P| grad phi_h|_P) / (sum |P|) over the element
    pieces P around node i that lie in Omega^+ if their volume is positive,
    otherwise over all pieces;
  * layered object (geometry.set_bedrock): regular tets take the permittivity
    of their region (plasma, regolith, bedrock); a tet inside the object cut by
    the bedrock plane is an interface tet of that plane (bedrock on its minus
    side, homogeneous flux jump, no surface charge, no Gamma_h area for the
    surface bookkeeping); a tet cut by the object's surface stays an interface
    tet of the surface alone even if the bedrock plane also crosses it (its
    object side takes the regolith's permittivity);
  * Dirichlet value of a node on several Dirichlet faces: the first such face
    in the order x-, x+, y-, y+, z-, z+.
"""
import numpy as np
import scipy.sparse as sp

from .geometry import TETS, VERT_OFF, ife_local, regular_grad_table, tri_area

# neighbour scan order for the surface-charge fallback: offsets sorted by
# L1 distance, then lexicographically by (dz, dy, dx)
_SCAN = sorted([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dx, dy, dz) != (0, 0, 0)], key=lambda o: (abs(o[0]) + abs(o[1]) + abs(o[2]), o[2], o[1], o[0]))
FACE_NAMES = ("x-", "x+", "y-", "y+", "z-", "z+")


class FieldSystem:
    """Mesh + object + field boundary conditions -> IFE system (Sec. 2.1).

    face_bc: sequence of 6 entries for x-, x+, y-, y+, z-, z+; each is either
    ("D", value) (Dirichlet, Eq. 2.2) or ("N",) (zero Neumann, Eq. 2.3 with p = 0).
    """

    def __init__(self, mesh, obj, face_bc):
        self.mesh = mesh
        self.obj = obj
        h = mesh.h
        ni, nj, nk = mesh.node_ijk()
        self.Lnode = obj.L(ni.astype(np.float64), nj.astype(np.float64), nk.astype(np.float64))
        self.minus = self.Lnode < 0
        # layered object: bedrock (L_b = z - z_b < 0, inside the object) under the regolith
        bed = getattr(obj, "bed", None)
        if bed is not None:
            zb, eb = bed
            self.Lbed = nk.astype(np.float64) - zb
            self.bmask = self.Lbed < 0
            if np.any(self.bmask & ~self.minus):
                raise ValueError("the bedrock must lie inside the object")
        else:
            eb = None
            self.Lbed = None
            self.bmask = np.zeros(mesh.nnodes, dtype=bool)
        cv = mesh.cube_vertex_nodes()
        par = mesh.cell_parity()
        G, V = regular_grad_table(h)
        em, ep = obj.eps_minus, obj.eps_plus
        rows, cols, vals = [], [], []
        # per-tet piece data for the node field: regular tets by shape
        self.reg = []          # list of (cells, tet nodes (m,4), grads (4,3), vol, region_plus (m,))
        it_cell, it_t, it_nodes, it_data, it_kind = [], [], [], [], []
        for p in range(2):
            cells_p = np.nonzero(par == p)[0]
            for t, tv in enumerate(TETS[p]):
                nodes = cv[cells_p][:, list(tv)]
                nm = self.minus[nodes].sum(axis=1)
                nb = self.bmask[nodes].sum(axis=1)
                regions = [("+", ep, nm == 0), ("-", em, (nm == 4) & (nb == 0))]
                if bed is not None:
                    regions.append(("b", eb, nb == 4))
                for region, eps, mask in regions:
                    sel = nodes[mask]
                    Kt = eps * V[t] * (G[p][t] @ G[p][t].T)
                    for a in range(4):
                        for b in range(4):
                            rows.append(sel[:, a]); cols.append(sel[:, b])
                            vals.append(np.full(len(sel), Kt[a, b]))
                    self.reg.append((sel, G[p][t], V[t], region == "+"))
                # interface tets: cut by the object's surface (kind 0; also when the
                # bedrock plane crosses the same tet: that tet keeps the surface
                # only, its object side with the regolith's permittivity), or lying
                # inside the object and cut by the bedrock plane only (kind 1:
                # homogeneous flux jump, no surface charge)
                for kind, icells in ((0, cells_p[(nm > 0) & (nm < 4)]),
                                     (1, cells_p[(nm == 4) & (nb > 0) & (nb < 4)])):
                    for c in icells:
                        nd = cv[c][list(tv)]
                        verts = VERT_OFF[list(tv)].astype(np.float64) * h
                        if kind == 0:
                            d = ife_local(verts, self.Lnode[nd], em, ep)
                        else:
                            d = ife_local(verts, self.Lbed[nd], eb, em)
                        it_cell.append(c); it_t.append(t); it_nodes.append(nd); it_data.append(d)
                        it_kind.append(kind)
        order = np.lexsort((np.array(it_t, dtype=np.int64), np.array(it_cell, dtype=np.int64))) \
            if it_cell else np.zeros(0, dtype=np.int64)
        self.it_cell = np.array(it_cell, dtype=np.int64)[order]
        self.it_t = np.array(it_t, dtype=np.int64)[order]
        self.it_nodes = np.array(it_nodes, dtype=np.int64).reshape(-1, 4)[order]
        self.it_kind = np.array(it_kind, dtype=np.int64)[order]
        data = [it_data[i] for i in order]
        self.it = data
        nit = len(data)
        self.it_K = np.array([d["K"] for d in data]).reshape(nit, 4, 4)
        self.it_c = np.array([d["c"] for d in data]).reshape(nit, 4)
        # Gamma_h area of the charged surface only (bedrock-plane tets carry none)
        self.it_area = np.array([d["area"] if k == 0 else 0.0 for d, k in zip(data, self.it_kind)])
        self.it_volp = np.array([d["vol_plus"] for d in data])
        self.it_volm = np.array([d["vol_minus"] for d in data])
        self.it_gp = np.array([d["gp"] for d in data]).reshape(nit, 5, 3)
        self.it_gm = np.array([d["gm"] for d in data]).reshape(nit, 5, 3)
        for a in range(4):
            for b in range(4):
                rows.append(self.it_nodes[:, a]); cols.append(self.it_nodes[:, b])
                vals.append(self.it_K[:, a, b])
        N = mesh.nnodes
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(N, N))
        self._setup_cut_cells()
        self._setup_dirichlet(face_bc)

    # -- surface charge bookkeeping (reading; see module docstring) ----------
    def _setup_cut_cells(self):
        m = self.mesh
        area = np.zeros(m.ncells)
        np.add.at(area, self.it_cell, self.it_area)
        self.cut_cells = np.nonzero(area > 0)[0]
        self.cut_area = area[self.cut_cells]
        acc = np.full(m.ncells, -1, dtype=np.int64)
        acc[self.cut_cells] = np.arange(len(self.cut_cells))
        ci, cj, ck = m.cell_ijk()
        target = acc.copy()
        for dx, dy, dz in _SCAN:
            ii, jj, kk = ci + dx, cj + dy, ck + dz
            ok = (ii >= 0) & (ii < m.nx) & (jj >= 0) & (jj < m.ny) & (kk >= 0) & (kk < m.nz)
            nb = np.where(ok, m.cell(np.clip(ii, 0, m.nx - 1), np.clip(jj, 0, m.ny - 1),
                                     np.clip(kk, 0, m.nz - 1)), 0)
            cand = np.where(ok, acc[nb], -1)
            fill = (target < 0) & (cand >= 0)
            target[fill] = cand[fill]
        self.cell_to_acc = target
        # cut-cell index of each interface tet (-1 if its cell has no Gamma_h area,
        # and for the bedrock-plane tets)
        self.it_acc = np.where(self.it_kind == 0, acc[self.it_cell], -1) if len(self.it_cell) \
            else np.zeros(0, dtype=np.int64)

    def _setup_dirichlet(self, face_bc):
        m = self.mesh
        ni, nj, nk = m.node_ijk()
        on_face = [ni == 0, ni == m.nx, nj == 0, nj == m.ny, nk == 0, nk == m.nz]
        self.is_dir = np.zeros(m.nnodes, dtype=bool)
        self.g = np.zeros(m.nnodes)
        for f in range(6):
            bc = face_bc[f]
            if bc[0] == "D":
                new = on_face[f] & ~self.is_dir
                self.g[new] = float(bc[1])
                self.is_dir |= on_face[f]
        self.free = np.nonzero(~self.is_dir)[0]
        self.dirn = np.nonzero(self.is_dir)[0]
        A = self.A
        self.A_ff = A[self.free][:, self.free].tocsr()
        self.A_fd = A[self.free][:, self.dirn].tocsr()

    # -- right-hand side ------------------------------------------------------
    def q_tets(self, Q_cut):
        """q_T = -Q_c / A_c for the interface tets of cut cell c, 0 elsewhere."""
        q = np.zeros(len(self.it_cell))
        has = self.it_acc >= 0
        sigma = Q_cut / self.cut_area
        q[has] = -sigma[self.it_acc[has]]
        return q

    def load(self, F, qT):
        """Nodal load F_i plus the flux-jump term sum_T q_T c_{T,i}."""
        b = np.array(F, dtype=np.float64, copy=True)
        if len(qT):
            np.add.at(b, self.it_nodes, qT[:, None] * self.it_c)
        return b

    # -- Jacobi PCG (Sec. 2.5, PCG level) --------------------------------------
    def solve(self, F, qT, phi0=None, tol=1e-6, maxit=150):
        """Solve the IFE system; returns (phi, iterations, relative residual).

        Textbook preconditioned conjugate gradients on the free nodes with a
        Jacobi (diagonal) preconditioner.  The Dirichlet values are lifted into
        the right-hand side.  Stops when ||r|| <= tol ||b|| (r the recursively
        updated residual) or after maxit iterations.
        """
        b_all = self.load(F, qT)
        b = b_all[self.free] - self.A_fd @ self.g[self.dirn]
        phi = self.g.copy()
        x = np.zeros(len(self.free)) if phi0 is None else np.array(phi0[self.free], dtype=np.float64)
        bnorm = np.sqrt(b @ b)
        if bnorm == 0.0:
            return phi, 0, 0.0
        A = self.A_ff
        dinv = 1.0 / A.diagonal()
        r = b - A @ x
        z = dinv * r
        p = z.copy()
        rz = r @ z
        rnorm = np.sqrt(r @ r)
        it = 0
        while rnorm > tol * bnorm and it < maxit:
            q = A @ p
            alpha = rz / (p @ q)
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            rnorm = np.sqrt(r @ r)
            z = dinv * r
            rz_new = r @ z
            beta = rz_new / rz
            rz = rz_new
            p = z + beta * p
        phi[self.free] = x
        return phi, it, rnorm / bnorm

    # -- node electric field (reading; see module docstring) -------------------
    def node_E(self, phi, qT):
        m = self.mesh
        N = m.nnodes
        acc_all = np.zeros((N, 3)); vol_all = np.zeros(N)
        acc_pl = np.zeros((N, 3)); vol_pl = np.zeros(N)

        def scatter(nodes, g, vol, plus):
            for a in range(4):
                np.add.at(acc_all, nodes[:, a], vol[:, None] * g)
                np.add.at(vol_all, nodes[:, a], vol)
                sel = plus & (vol > 0)
                np.add.at(acc_pl, nodes[sel, a], vol[sel, None] * g[sel])
                np.add.at(vol_pl, nodes[sel, a], vol[sel])

        for nodes, Gt, Vt, plus in self.reg:
            if len(nodes) == 0:
                continue
            g = phi[nodes] @ Gt                                 # (m,3)
            scatter(nodes, g, np.full(len(nodes), Vt), np.full(len(nodes), plus))
        if len(self.it_cell):
            ph = phi[self.it_nodes]                             # (nit,4)
            gpl = np.einsum("ta,tak->tk", ph, self.it_gp[:, :4]) + qT[:, None] * self.it_gp[:, 4]
            gmi = np.einsum("ta,tak->tk", ph, self.it_gm[:, :4]) + qT[:, None] * self.it_gm[:, 4]
            nit = len(self.it_cell)
            # the + piece is plasma only on the object's surface, not on the bedrock plane
            scatter(self.it_nodes, gpl, self.it_volp, self.it_kind == 0)
            scatter(self.it_nodes, gmi, self.it_volm, np.zeros(nit, dtype=bool))
        use_pl = vol_pl > 0
        E = np.empty((N, 3))
        E[use_pl] = -acc_pl[use_pl] / vol_pl[use_pl, None]
        E[~use_pl] = -acc_all[~use_pl] / vol_all[~use_pl, None]
        return E

    def surface_potential(self, phi, qT):
        """Area-weighted mean of phi_h over Gamma_h (diagnostic, Sec. 5.4)."""
        if len(self.it_cell) == 0 or self.it_area.sum() == 0:
            return 0.0
        tot = 0.0
        for n, d in enumerate(self.it):
            if self.it_kind[n] != 0:
                continue
            coef = d["coef"]
            for tri in d["tris"]:
                cen = tri.mean(axis=0)
                val = (coef[0, :4] + cen @ coef[1:, :4]) @ phi[self.it_nodes[n]] \
                    + qT[n] * (coef[0, 4] + cen @ coef[1:, 4])
                tot += tri_area(*tri) * val
        return tot / self.it_area.sum()
