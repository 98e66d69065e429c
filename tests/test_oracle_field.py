"""Pins of oracle.field: the IFE solve against a manufactured interface solution,
brute force on 4^3, a library sparse solver, and the node field.

P3 (manufactured sphere, Sec. 2.1 Eqs. 2.1-2.5 with q != 0): on [-1,1]^3 with
R = 0.6183, eps- = 4, eps+ = 1, u- = r^2/eps-,
u+ = r^2/eps+ + gamma (1/R - 1/r) + R^2 (1/eps- - 1/eps+): rho = -6 on both
sides, [u] = 0, [eps du/dr] = eps+ gamma / R^2 (constant).  A dropped or
sign-flipped flux-jump term leaves an O(1) error; the correct one converges at
second order in L2.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.geometry import TETS, VERT_OFF, Mesh, NoObject, Sphere, ife_local, regular_grad_table
from oracle.field import FieldSystem


def manufactured(n, gamma=1.0, em=4.0, ep=1.0, flip=1.0):
    R = 0.6183
    h = 2.0 / n
    m = Mesh(n, n, n, h, origin=(-1, -1, -1))
    fs = FieldSystem(m, Sphere(m, (0, 0, 0), R, em, ep), [("D", 0.0)] * 6)
    i, j, k = m.node_ijk()
    X, Y, Z = -1 + i * h, -1 + j * h, -1 + k * h
    r = np.sqrt(X * X + Y * Y + Z * Z)
    up = r * r / ep + gamma * (1 / R - 1 / np.maximum(r, 1e-300)) + R * R * (1 / em - 1 / ep)
    u = np.where(fs.minus, r * r / em, up)
    fs.g[:] = np.where(fs.is_dir, u, 0.0)
    F = np.full(m.nnodes, -6.0 * h ** 3)      # int rho S_i dx for the Q1 weight S_i
    qT = np.full(len(fs.it_cell), flip * ep * gamma / R ** 2)
    phi, it, rr = fs.solve(F, qT, tol=1e-12, maxit=5000)
    e = phi - u
    return np.sqrt((e * e).mean()), it, rr


def test_manufactured_sphere_second_order():
    e = [manufactured(n)[0] for n in (8, 16, 32)]
    assert e[2] < 2.0e-3
    assert e[0] / e[1] > 3.3 and e[1] / e[2] > 3.4


@pytest.mark.parametrize("flip", [0.0, -1.0])
def test_manufactured_sphere_detects_wrong_jump(flip):
    e = [manufactured(n, flip=flip)[0] for n in (8, 16)]
    assert min(e) > 0.2


def test_pcg_matches_library_direct_solve():
    m = Mesh(10, 9, 8, 0.5)
    fs = FieldSystem(m, Sphere(m, (2.4, 2.3, 2.1), 1.3, 6.0, 1.0), [("D", 0.1)] * 3 + [("N",)] * 3)
    g = np.random.default_rng(5)
    F = g.normal(size=m.nnodes) * 0.01
    qT = g.normal(size=len(fs.it_cell))
    phi, it, rr = fs.solve(F, qT, tol=1e-13, maxit=4000)
    b = fs.load(F, qT)[fs.free] - fs.A_fd @ fs.g[fs.dirn]
    x = spla.spsolve(fs.A_ff.tocsc(), b)
    assert np.abs(phi[fs.free] - x).max() < 1e-10 * np.abs(x).max()
    assert np.all(phi[fs.dirn] == 0.1)


def _brute_force_system(m, obj, face_bc):
    """Independent dense assembly: loop over every cube and tet, classify, take
    the regular P1 or IFE element matrix and jump vector, add into dense arrays."""
    N = m.nnodes
    A = np.zeros((N, N))
    C = []          # (nodes, c) per interface tet, in loop order
    G, V = regular_grad_table(m.h)
    for k in range(m.nz):
        for j in range(m.ny):
            for i in range(m.nx):
                p = (i + j + k) % 2
                for t in TETS[p]:
                    nodes = [m.node(i + VERT_OFF[l][0], j + VERT_OFF[l][1], k + VERT_OFF[l][2]) for l in t]
                    pos = [np.array([i + VERT_OFF[l][0], j + VERT_OFF[l][1], k + VERT_OFF[l][2]], float) for l in t]
                    Lv = np.array([obj.L(*q) for q in pos])
                    nm = int((Lv < 0).sum())
                    if 0 < nm < 4:
                        d = ife_local(VERT_OFF[list(t)].astype(float) * m.h, Lv, obj.eps_minus, obj.eps_plus)
                        Ke = d["K"]
                        C.append((nodes, d["c"]))
                    else:
                        X = np.array(pos) * m.h
                        M = np.hstack([np.ones((4, 1)), X])
                        grads = np.linalg.inv(M)[1:, :].T
                        vol = abs(np.linalg.det(X[1:] - X[0])) / 6
                        eps = obj.eps_plus if nm == 0 else obj.eps_minus
                        Ke = eps * vol * grads @ grads.T
                    for a in range(4):
                        for b in range(4):
                            A[nodes[a], nodes[b]] += Ke[a, b]
    return A, C


def _gauss_pp(A, b):
    """Dense Gaussian elimination with partial pivoting (textbook)."""
    A = A.copy(); b = b.copy(); n = len(b)
    for c in range(n):
        p = c + int(np.argmax(np.abs(A[c:, c])))
        A[[c, p]] = A[[p, c]]; b[[c, p]] = b[[p, c]]
        for r in range(c + 1, n):
            f = A[r, c] / A[c, c]
            A[r, c:] -= f * A[c, c:]
            b[r] -= f * b[c]
    x = np.zeros(n)
    for r in range(n - 1, -1, -1):
        x[r] = (b[r] - A[r, r + 1:] @ x[r + 1:]) / A[r, r]
    return x


def test_brute_force_4cubed():
    """P4: dense element-loop assembly + Gaussian elimination == oracle PCG to 1e-12."""
    m = Mesh(4, 4, 4, 0.5)
    obj = Sphere(m, (1.03, 0.97, 1.01), 0.62, 4.0, 1.0)
    bc = [("D", 0.0), ("D", 0.3), ("N",), ("D", -0.2), ("N",), ("N",)]
    fs = FieldSystem(m, obj, bc)
    A, C = _brute_force_system(m, obj, bc)
    assert np.abs(A - fs.A.toarray()).max() < 1e-13
    g = np.random.default_rng(2)
    F = g.normal(size=m.nnodes) * 0.05
    q = 0.7
    b = F.copy()
    for nodes, c in C:
        for a in range(4):
            b[nodes[a]] += q * c[a]
    free, dirn = fs.free, fs.dirn
    rhs = b[free] - A[np.ix_(free, dirn)] @ fs.g[dirn]
    x = _gauss_pp(A[np.ix_(free, free)], rhs)
    phi, it, rr = fs.solve(F, np.full(len(fs.it_cell), q), tol=1e-14, maxit=2000)
    assert np.abs(phi[free] - x).max() < 1e-12 * max(1.0, np.abs(x).max())


def test_node_field_linear_and_plasma_side():
    """Node field reproduces -grad of a linear phi (no interface), and for the
    sphere takes only Omega^+ pieces at nodes that touch the plasma."""
    m = Mesh(6, 6, 6, 0.4)
    fs = FieldSystem(m, NoObject(2.0), [("D", 0.0)] * 6)
    i, j, k = m.node_ijk()
    phi = 0.5 - 0.3 * i * m.h + 1.1 * j * m.h + 0.2 * k * m.h
    E = fs.node_E(phi, np.zeros(0))
    assert np.abs(E - np.array([0.3, -1.1, -0.2])).max() < 1e-12
    # piecewise-linear phi with a kink on a sphere: plasma-side nodes see +side gradient
    obj = Sphere(m, (1.2, 1.2, 1.2), 0.5, 4.0, 1.0)
    fs2 = FieldSystem(m, obj, [("D", 0.0)] * 6)
    phi2 = 0.7 * k * m.h            # linear everywhere: every piece has the same gradient
    E2 = fs2.node_E(phi2, np.zeros(len(fs2.it_cell)))
    # not exactly -0.7 near the interface (IFE functions bend), exact away from it
    far = np.ones(m.nnodes, dtype=bool)
    far[fs2.it_nodes.ravel()] = False
    assert np.abs(E2[far] - np.array([0.0, 0.0, -0.7])).max() < 1e-12


def test_gauss_law_sphere_charge():
    """P8 (loose): a charged sphere with no plasma; phi outside ~ Q/(4 pi r) plus
    the grounded-box correction, checked along an axis to O(h) accuracy."""
    n, h = 32, 0.25
    m = Mesh(n, n, n, h)
    R = 1.0
    c = (4.0, 4.0, 4.0)
    fs = FieldSystem(m, Sphere(m, c, R, 4.0, 1.0), [("D", 0.0)] * 6)
    sigma = 0.1
    qT = np.full(len(fs.it_cell), -sigma)
    phi, it, rr = fs.solve(np.zeros(m.nnodes), qT, tol=1e-12, maxit=5000)
    Q = sigma * fs.it_area.sum()
    # images are ignored: compare the field-free potential difference between two radii
    i0 = m.node(16, 16, 16)
    r1, r2 = 1.5, 2.0
    p1 = phi[m.node(16 + int(r1 / h), 16, 16)]
    p2 = phi[m.node(16 + int(r2 / h), 16, 16)]
    expect = Q / (4 * np.pi) * (1 / r1 - 1 / r2)
    assert abs((p1 - p2) - expect) < 0.1 * expect
    assert phi[i0] > p1 > p2 > 0
