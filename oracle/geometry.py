"""Mesh, level sets and linear IFE local spaces (oracle; test infrastructure only).

Follows arXiv:2011.10214:
  * Sec. 3.1.1: a globally uniform Cartesian PIC mesh whose cubic cells are each
    cut into 5 tetrahedra; the IFE mesh equals the PIC mesh.
  * Sec. 2.1, Eqs. 2.1-2.5: -div(eps grad phi) = rho on both sides of the
    interface, [phi] = 0 and [eps d phi / d n] = q across it, n pointing from
    Omega^- to Omega^+, jump = (+ side) - (- side), eps piecewise constant.
  * Sec. 1 / Sec. 2.1: IFE functions are ordinary FE functions adjusted locally
    on interface elements to satisfy the interface conditions, with the same
    degrees of freedom (nodal values) as the standard linear FE space.

Readings where the paper is silent:
  * 5-tet split: one central tet on the cube's four globally even vertices
    ((i+j+k) even), four corner tets, each an odd vertex with its three axis
    neighbours.  Face diagonals then match between neighbouring cubes.
  * The object is given by an analytic level set L, L >= 0 in the plasma
    (Omega^+), L < 0 in the object (Omega^-).  A node with L == 0 is in Omega^+.
  * A layered object (set_bedrock) has a second, planar level set L_b = z - z_b
    inside it: bedrock where L_b < 0.
  * Gamma_h on a tet is the zero set of the linear interpolant of the nodal L
    values (a plane piece: a triangle for a 1-3 sign split, a planar quad for a
    2-2 split).
  * Linear IFE on an interface tet T: psi+ = a + b.x on T, psi- = psi+ + beta d(x)
    with d the signed distance to the plane of Gamma_h (d > 0 on the + side).
    The flux-jump condition eps+ n.b - eps-(n.b + beta) = q gives
    beta = ((eps+ - eps-) n.b - q) / eps-.  Nodal values psi(v) = u_v, using the
    piece that contains v, fix (a, b) through a 4x4 system linear in (u, q).
    Basis functions: u = e_j, q = 0.  Jump function phi_J: u = 0, q given.

Positions are in cell units (xi = (x - origin)/h); level sets are evaluated in
cell units.  Geometry passed to the IFE local solve is physical (lengths x h).
"""
import numpy as np

# local vertex l = a + 2b + 4c  <->  offset (a, b, c); this is also the node
# order of the trilinear weights (000, 100, 010, 110, 001, 101, 011, 111)
VERT_OFF = np.array([[l & 1, (l >> 1) & 1, (l >> 2) & 1] for l in range(8)], dtype=np.int64)


def cube_tets(parity):
    """The 5 tets of a cube whose corner (i,j,k) has (i+j+k) % 2 == parity.

    Returns a list of 5 tuples of local vertex indices: tet 0 is the central
    tet on the 4 globally even vertices (ascending local index); tets 1..4 are
    the corner tets (o, o^1, o^2, o^4) for the odd vertices o in ascending
    order.  Reading of Sec. 3.1.1 (5 tets per cube; split unstated).
    """
    even = [l for l in range(8) if (VERT_OFF[l].sum() % 2) == parity]
    odd = [l for l in range(8) if (VERT_OFF[l].sum() % 2) != parity]
    return [tuple(even)] + [(o, o ^ 1, o ^ 2, o ^ 4) for o in odd]


TETS = [cube_tets(0), cube_tets(1)]


class Mesh:
    """Uniform Cartesian mesh of nx*ny*nz cubic cells of size h (Sec. 3.1.1)."""

    def __init__(self, nx, ny, nz, h, origin=(0.0, 0.0, 0.0)):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.h = float(h)
        self.origin = np.asarray(origin, dtype=np.float64)
        self.NX, self.NY, self.NZ = self.nx + 1, self.ny + 1, self.nz + 1
        self.nnodes = self.NX * self.NY * self.NZ
        self.ncells = self.nx * self.ny * self.nz

    def node(self, i, j, k):
        return i + self.NX * (j + self.NY * k)

    def cell(self, i, j, k):
        return i + self.nx * (j + self.ny * k)

    def node_ijk(self):
        n = np.arange(self.nnodes)
        return n % self.NX, (n // self.NX) % self.NY, n // (self.NX * self.NY)

    def cell_ijk(self):
        c = np.arange(self.ncells)
        return c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)

    def cube_vertex_nodes(self):
        """(ncells, 8) global node ids of each cube's vertices, local order."""
        i, j, k = self.cell_ijk()
        out = np.empty((self.ncells, 8), dtype=np.int64)
        for l in range(8):
            a, b, c = VERT_OFF[l]
            out[:, l] = self.node(i + a, j + b, k + c)
        return out

    def cell_parity(self):
        i, j, k = self.cell_ijk()
        return (i + j + k) % 2


# ---------------------------------------------------------------------------
# Analytic level sets in cell units.  L >= 0: plasma (Omega^+); L < 0: object.
# The operation order is part of the definition (hit decisions are compared
# bit-exactly), so each is written out as a fixed sequence of IEEE operations.
# ---------------------------------------------------------------------------

class Sphere:
    """Dielectric sphere of Sec. 3.1 (centre c, radius R, physical units)."""

    kind = "sphere"

    def __init__(self, mesh, center, radius, eps_in, eps_out):
        self.c = (np.asarray(center, dtype=np.float64) - mesh.origin) / mesh.h
        r = float(radius) / mesh.h
        self.r2 = r * r
        self.eps_minus = float(eps_in)
        self.eps_plus = float(eps_out)

    def L(self, x, y, z):
        dx = x - self.c[0]
        dy = y - self.c[1]
        dz = z - self.c[2]
        return ((dx * dx + dy * dy) + dz * dz) - self.r2


class CapCrater:
    """Planar ground at height z_g with a spherical-cap crater (Sec. 5.2.1).

    The paper builds its crater from rim radii and rim height (Sec. 5.2.1);
    this reading uses a spherical cap of rim radius a and depth D centred at
    (xc, yc): cap sphere radius Rs = (a^2 + D^2)/(2D), centre height
    z_g - D + Rs.  All arguments physical; L = z - z_s(x, y) in cell units.
    """

    kind = "cap_crater"

    def __init__(self, mesh, z_ground, xc, yc, rim_radius, depth, eps_in, eps_out):
        h = mesh.h
        self.zg = (float(z_ground) - mesh.origin[2]) / h
        self.xc = (float(xc) - mesh.origin[0]) / h
        self.yc = (float(yc) - mesh.origin[1]) / h
        a = float(rim_radius) / h
        D = float(depth) / h
        Rs = (a * a + D * D) / (2.0 * D)
        self.a2 = a * a
        self.Rs2 = Rs * Rs
        self.zc = (self.zg - D) + Rs
        self.eps_minus = float(eps_in)
        self.eps_plus = float(eps_out)

    def L(self, x, y, z):
        dx = x - self.xc
        dy = y - self.yc
        r2 = dx * dx + dy * dy
        inside = r2 < self.a2
        zs = np.where(inside, self.zc - np.sqrt(np.where(inside, self.Rs2 - r2, 0.0)), self.zg)
        return z - zs


class RimCrater:
    """Planar ground at height z_g with a raised-rim crater centred at (xc, yc).

    Sec. 5.2.1 describes the lunar crater by an algebraic surface z = z(x, y)
    set by its inner-rim, top-rim and outer-rim radii and its top height; the
    profile between them is not printed.  This reading: a flat floor at depth D
    below the ground inside the inner-rim radius Ri; an inner wall rising from
    the floor to the rim top, H above the ground, at the top-rim radius Rt; an
    outer flank falling back to the ground at the outer-rim radius Ro.  Both
    ramps are the cubic smoothstep s(t) = t^2 (3 - 2t) of the radial
    coordinate, so the surface is continuous with a continuous slope.  All
    arguments physical; L = z - z_s(x, y) in cell units.
    """

    kind = "rim_crater"

    def __init__(self, mesh, z_ground, xc, yc, r_inner, r_top, r_outer, height, depth, eps_in, eps_out):
        h = mesh.h
        self.zg = (float(z_ground) - mesh.origin[2]) / h
        self.xc = (float(xc) - mesh.origin[0]) / h
        self.yc = (float(yc) - mesh.origin[1]) / h
        self.ri = float(r_inner) / h
        self.rt = float(r_top) / h
        self.ro = float(r_outer) / h
        H = float(height) / h
        D = float(depth) / h
        if not (0.0 <= self.ri < self.rt < self.ro) or H < 0.0 or D < 0.0:
            raise ValueError("rim crater needs 0 <= r_inner < r_top < r_outer, height >= 0, depth >= 0")
        self.H = H
        self.zfloor = self.zg - D
        self.ztop = self.zg + H
        self.rise = D + H
        self.w_in = self.rt - self.ri
        self.w_out = self.ro - self.rt
        self.eps_minus = float(eps_in)
        self.eps_plus = float(eps_out)

    def surface(self, x, y):
        dx = x - self.xc
        dy = y - self.yc
        r = np.sqrt(dx * dx + dy * dy)
        t1 = (r - self.ri) / self.w_in
        s1 = (t1 * t1) * (3.0 - 2.0 * t1)
        t2 = (r - self.rt) / self.w_out
        s2 = (t2 * t2) * (3.0 - 2.0 * t2)
        z_in = self.zfloor + self.rise * s1
        z_out = self.ztop - self.H * s2
        return np.where(r <= self.ri, self.zfloor,
                        np.where(r <= self.rt, z_in, np.where(r < self.ro, z_out, self.zg)))

    def L(self, x, y, z):
        return z - self.surface(x, y)


class Refined:
    """An object seen from a mesh r times finer than the one it was built on
    (the IFE mesh of a hybrid grid, Sec. 2.2: the PIC and IFE meshes may have
    different resolutions): L_fine(xi) = L(xi / r) in the fine mesh's cell
    units.  r is a power of two, so xi / r is exact and the fine level set is
    the coarse one scaled by an exact power of two: same signs, same
    interpolation ratios.  A bedrock plane moves to fine units (z_b r)."""

    def __init__(self, obj, r):
        self.obj = obj
        self.r = float(r)
        self.kind = obj.kind
        self.eps_minus = obj.eps_minus
        self.eps_plus = obj.eps_plus
        bed = getattr(obj, "bed", None)
        if bed is not None:
            self.bed = (bed[0] * self.r, bed[1])

    def L(self, x, y, z):
        return self.obj.L(x / self.r, y / self.r, z / self.r)


def set_bedrock(obj, mesh, z_bed, eps_bed):
    """A second dielectric layer of the object (Sec. 5.2.1: lunar regolith over
    bedrock).  Below the plane z = z_bed (physical) the object has permittivity
    eps_bed; its level set is L_b = z - z_bed in cell units, L_b < 0 in the
    bedrock, which must lie inside the object (checked by the field set-up).
    Returns obj with the attribute bed = (z_bed in cell units, eps_bed)."""
    if not (float(eps_bed) > 0.0):
        raise ValueError("eps_bed must be positive")
    obj.bed = ((float(z_bed) - mesh.origin[2]) / mesh.h, float(eps_bed))
    return obj


class Plane:
    """Planar interface n.xi = d0 (cell units), used by pins; L = n.xi - d0."""

    kind = "plane"

    def __init__(self, normal, d0, eps_minus, eps_plus):
        self.n = np.asarray(normal, dtype=np.float64)
        self.d0 = float(d0)
        self.eps_minus = float(eps_minus)
        self.eps_plus = float(eps_plus)

    def L(self, x, y, z):
        return ((self.n[0] * x + self.n[1] * y) + self.n[2] * z) - self.d0


class NoObject:
    """Empty domain (every node in Omega^+)."""

    kind = "none"

    def __init__(self, eps=1.0):
        self.eps_minus = self.eps_plus = float(eps)

    def L(self, x, y, z):
        return np.ones(np.broadcast(x, y, z).shape)


# ---------------------------------------------------------------------------
# Linear IFE local space on one interface tetrahedron.
# ---------------------------------------------------------------------------

def tet_volume(p0, p1, p2, p3):
    return abs(np.linalg.det(np.array([p1 - p0, p2 - p0, p3 - p0]))) / 6.0


def tri_area(p0, p1, p2):
    return 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0))


def interface_pieces(verts, Lv):
    """Split of a tet by the plane piece Gamma_h (zero set of the linear interpolant).

    verts: (4,3) physical vertex coordinates; Lv: (4,) nodal level-set values
    with mixed signs (L < 0 is Omega^-).  Returns (vol_minus, vol_plus,
    triangles) where triangles is a list of (3,3) arrays that tile Gamma_h on
    the tet (one for a 1-3 split, two for a 2-2 split).
    """
    minus = Lv < 0
    V = tet_volume(*verts)
    mi = [v for v in range(4) if minus[v]]
    pl = [v for v in range(4) if not minus[v]]

    def cut(u, w):  # u in Omega^-, w in Omega^+: zero of the interpolant on edge uw
        t = Lv[u] / (Lv[u] - Lv[w])
        return verts[u] + t * (verts[w] - verts[u]), t

    if len(mi) == 1 or len(mi) == 3:
        lone_minus = len(mi) == 1
        u = mi[0] if lone_minus else pl[0]
        others = pl if lone_minus else mi
        pts, fr = [], []
        for w in others:
            if lone_minus:
                p, t = cut(u, w)
                fr.append(t)
            else:
                p, t = cut(w, u)      # edge (minus w, plus u); fraction from u is 1-t
                fr.append(1.0 - t)
            pts.append(p)
        vcut = V * fr[0] * fr[1] * fr[2]          # piece that holds the lone vertex
        tris = [np.array(pts)]
        if lone_minus:
            return vcut, V - vcut, tris
        return V - vcut, vcut, tris
    # 2-2 split: minus vertices a, b; plus vertices c, d
    a, b = mi
    c, d = pl
    pac, _ = cut(a, c)
    pad, _ = cut(a, d)
    pbc, _ = cut(b, c)
    pbd, _ = cut(b, d)
    A1, A2, A3 = verts[a], pac, pad          # prism: A_k <-> B_k along planar quads
    B1, B2, B3 = verts[b], pbc, pbd
    vminus = tet_volume(A1, A2, A3, B3) + tet_volume(A1, A2, B2, B3) + tet_volume(A1, B1, B2, B3)
    tris = [np.array([pac, pad, pbd]), np.array([pac, pbd, pbc])]
    return vminus, V - vminus, tris


def ife_local(verts, Lv, eps_minus, eps_plus):
    """Linear IFE space on an interface tet (Sec. 2.1, Eqs. 2.4-2.5).

    Returns a dict with
      n          unit normal of Gamma_h, from Omega^- to Omega^+
      coef       (4, 5) rows (a, b_x, b_y, b_z) ... columns: basis 0..3, jump fn
      gp, gm     (5, 3) gradients on the + and - pieces (basis 0..3, jump fn
                 for unit q)
      vol_plus, vol_minus, area, tris
      K          (4, 4) element stiffness eps+|T+| gp gp^T + eps-|T-| gm gm^T
      S          (4,) integrals of psi_i over Gamma_h on the tet
      c          (4,) unit-jump load: c_i = -S_i - a_T(phi_J, psi_i) for q = 1;
                 the flux jump q on this tet adds q * c_i to the load of vertex i
    """
    verts = np.asarray(verts, dtype=np.float64)
    Lv = np.asarray(Lv, dtype=np.float64)
    minus = Lv < 0
    M = verts[1:] - verts[0]
    gL = np.linalg.solve(M, Lv[1:] - Lv[0])       # gradient of the linear interpolant of L
    gnorm = np.linalg.norm(gL)
    n = gL / gnorm
    dist = Lv / gnorm                              # signed distance of each vertex to Gamma_h
    kappa = (eps_plus - eps_minus) / eps_minus
    A = np.zeros((4, 4))
    R = np.zeros((4, 5))
    for v in range(4):
        A[v, 0] = 1.0
        A[v, 1:] = verts[v] + (dist[v] * kappa * n if minus[v] else 0.0)
        R[v, v] = 1.0
        R[v, 4] = dist[v] / eps_minus if minus[v] else 0.0
    coef = np.linalg.solve(A, R)                   # (4, 5)
    b = coef[1:, :].T                              # (5, 3)
    q = np.array([0.0, 0.0, 0.0, 0.0, 1.0])
    beta = kappa * (b @ n) - q / eps_minus
    gp = b
    gm = b + beta[:, None] * n[None, :]
    vol_minus, vol_plus, tris = interface_pieces(verts, Lv)
    K = eps_plus * vol_plus * (gp[:4] @ gp[:4].T) + eps_minus * vol_minus * (gm[:4] @ gm[:4].T)
    aJ = eps_plus * vol_plus * (gp[:4] @ gp[4]) + eps_minus * vol_minus * (gm[:4] @ gm[4])
    S = np.zeros(4)
    area = 0.0
    for tri in tris:
        ar = tri_area(*tri)
        area += ar
        cen = tri.mean(axis=0)
        S += ar * (coef[0, :4] + cen @ coef[1:, :4])   # psi_i linear on Gamma_h
    return dict(n=n, dist=dist, coef=coef, gp=gp, gm=gm, beta=beta, vol_plus=vol_plus,
                vol_minus=vol_minus, area=area, tris=tris, K=K, S=S, c=-S - aJ)


def regular_grad_table(h):
    """Gradients of the 4 P1 basis functions of each of the 10 tet shapes.

    Returns G[parity][t] as a (4, 3) array (rows: tet vertices in tet order)
    and the tet volume V[t] (central h^3/3, corner h^3/6).
    """
    G = [[None] * 5 for _ in range(2)]
    V = np.zeros(5)
    for p in range(2):
        for t, tv in enumerate(TETS[p]):
            X = VERT_OFF[list(tv)].astype(np.float64) * h
            M = np.hstack([np.ones((4, 1)), X])
            inv = np.linalg.inv(M)          # column j: coefficients of basis j
            G[p][t] = inv[1:, :].T
            V[t] = tet_volume(*X)
    return G, V
