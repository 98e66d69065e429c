"""Pins of the oracle pieces that the GPU parity tests compare against but that
no closed form had fixed yet:

  * the leapfrog start (Simulation.leapfrog_init -> particles.half_kick_back):
    in a uniform field, the half kick back followed by n pushes is the exact
    constant-acceleration motion x0 + v0 t + a t^2 / 2 at t = n dt;
  * the node field at interface nodes (FieldSystem.node_E): a planar interface
    (Eqs. 2.4-2.5) with a piecewise-linear u that satisfies [u] = 0 and
    [eps du/dn] = q lies in the local IFE space of every cut tet, so the field
    must be -grad u+ at every node that touches the plasma and -grad u- at
    nodes surrounded by the object;
  * the area-mean surface potential (FieldSystem.surface_potential): for the
    same u, the mean of u+ over the plane inside the box, a closed form;
  * the cut-cell fallback of the surface charge (FieldSystem._setup_cut_cells):
    hand-built neighbourhoods whose answer follows the stated order (L1
    distance, then dz, dy, dx ascending).

Each pin is also run against a planted mistake (a sign error, a dropped term,
a wrong scan order), put into the oracle on the CPU, and must fail on it."""
import numpy as np
import pytest

import oracle.field as ofield
from oracle import particles as pt
from oracle.field import FieldSystem
from oracle.geometry import TETS, Mesh, NoObject, Plane
from oracle.pic import Simulation


# ---------------------------------------------------------------------------
# leapfrog start
# ---------------------------------------------------------------------------

E0 = np.array([0.37, -0.21, 0.13])
Q, M, DT, H = -1.0, 1.0, 0.2, 0.5


def _leapfrog_error(nsteps=25):
    """Largest deviation (cell units) of positions, and of velocities, from the
    constant-acceleration closed form after leapfrog_init and nsteps steps."""
    m = Mesh(60, 60, 60, H)
    sim = Simulation(m, NoObject(), [("D", 0.0)] * 6, DT)
    sim.add_species(Q, M, 1.0)
    g = np.random.default_rng(31)
    n = 64
    x0 = g.uniform(25.0, 35.0, (3, n))
    v0 = g.normal(0.0, 0.3, (3, n))
    sim.load_particles(0, *x0, *v0)
    sim.set_external_E(np.tile(E0, (m.nnodes, 1)))
    sim.leapfrog_init()
    for _ in range(nsteps):
        sim.step()
    P = sim.P[0]
    order = np.argsort(P["id"])
    got_x = np.stack([P[k][order] for k in ("x", "y", "z")])
    got_v = np.stack([P[k][order] for k in ("vx", "vy", "vz")])
    a = (Q / M) * E0[:, None]
    t = nsteps * DT
    want_x = x0 + (v0 * t + 0.5 * a * t * t) / H          # cell units
    want_v = v0 + a * (t - 0.5 * DT)                      # v at t - dt/2
    return np.abs(got_x - want_x).max(), np.abs(got_v - want_v).max()


def test_leapfrog_start_gives_constant_acceleration_motion():
    ex, ev = _leapfrog_error()
    assert ex < 1e-11 and ev < 1e-12


@pytest.mark.parametrize("mistake", ["sign", "none"])
def test_leapfrog_pin_fails_on_planted_mistake(monkeypatch, mistake):
    def wrong(mesh, E, P, k):
        ex, ey, ez = pt.gather(mesh, E, P["x"], P["y"], P["z"])
        hk = 0.5 * k if mistake == "sign" else 0.0
        P["vx"] = P["vx"] + hk * ex
        P["vy"] = P["vy"] + hk * ey
        P["vz"] = P["vz"] + hk * ez
    monkeypatch.setattr(pt, "half_kick_back", wrong)
    ex, ev = _leapfrog_error()
    assert ex > 1e-3 and ev > 1e-3


# ---------------------------------------------------------------------------
# planar interface: node field and surface potential
# ---------------------------------------------------------------------------

NCELL = (6, 5, 7)
HP = 0.4
NORMAL = np.array([0.3, -0.2, 1.0])       # cell units; the plane z = D0 - 0.3 x + 0.2 y
D0 = 3.3137
EM, EP = 4.0, 1.0
QJ = 0.8                                  # flux jump [eps du/dn] on the plane
A0 = 0.25
GPLUS = np.array([0.6, -1.1, 0.45])       # grad u+ (physical units)


def _planar_case():
    """Mesh, field system and the exact u.  u+ = A0 + GPLUS . x on the plasma
    side, u- = u+ + beta d(x) in the object, d the signed distance to the plane
    (positive in the plasma): [u] = 0 on the plane and
    eps+ n.grad u+ - eps- n.grad u- = QJ fix beta."""
    m = Mesh(*NCELL, HP)
    obj = Plane(NORMAL, D0, EM, EP)
    fs = FieldSystem(m, obj, [("D", 0.0)] * 6)
    nhat = NORMAL / np.linalg.norm(NORMAL)
    beta = ((EP - EM) * (nhat @ GPLUS) - QJ) / EM
    gminus = GPLUS + beta * nhat
    i, j, k = m.node_ijk()
    X = np.stack([i, j, k], axis=1).astype(np.float64) * HP
    L = obj.L(i.astype(np.float64), j.astype(np.float64), k.astype(np.float64))
    d = L * HP / np.linalg.norm(NORMAL)
    uplus = A0 + X @ GPLUS
    u = np.where(L >= 0.0, uplus, uplus + beta * d)
    qT = np.full(len(fs.it_cell), QJ)
    return m, fs, u, qT, gminus


def _plasma_touching_nodes(m, fs):
    """Nodes that are a vertex of at least one tet with a vertex in the plasma
    (brute force over every cube and tet)."""
    touch = np.zeros(m.nnodes, dtype=bool)
    cv = m.cube_vertex_nodes()
    par = m.cell_parity()
    plus = ~fs.minus
    for c in range(m.ncells):
        for tv in TETS[par[c]]:
            nd = cv[c][list(tv)]
            if plus[nd].any():
                touch[nd] = True
    return touch


def _node_field_error(fs, u, qT, gminus, m):
    E = fs.node_E(u, qT)
    touch = _plasma_touching_nodes(m, fs)
    want = np.where(touch[:, None], -GPLUS[None, :], -gminus[None, :])
    return np.abs(E - want).max(), touch


def test_planar_case_is_nontrivial():
    m, fs, u, qT, gminus = _planar_case()
    touch = _plasma_touching_nodes(m, fs)
    assert len(fs.it_cell) > 100
    assert (touch & fs.minus).sum() > 20          # object nodes next to the plasma
    assert (~touch).sum() > 20                    # nodes surrounded by the object
    assert np.abs(gminus - GPLUS).max() > 0.1


def test_node_field_at_interface_nodes_is_exact_for_planar_ife_function():
    m, fs, u, qT, gminus = _planar_case()
    err, _ = _node_field_error(fs, u, qT, gminus, m)
    assert err < 1e-12


@pytest.mark.parametrize("mistake", ["dropped_jump_term", "flipped_jump_term", "all_pieces"])
def test_node_field_pin_fails_on_planted_mistake(mistake):
    m, fs, u, qT, gminus = _planar_case()
    if mistake == "dropped_jump_term":
        qT = np.zeros_like(qT)                    # the q_T gp[4] term contributes nothing
    elif mistake == "flipped_jump_term":
        qT = -qT
    else:                                         # average over every piece, not the plasma ones
        fs.reg = [(n, g, v, False) for (n, g, v, _) in fs.reg]
        fs.it_kind = np.ones_like(fs.it_kind)
    err, _ = _node_field_error(fs, u, qT, gminus, m)
    assert err > 1e-3


def _surface_mean_exact(m):
    """Mean of u+ over the plane inside the box.  The plane
    z = (D0 - 0.3 x + 0.2 y) stays inside [0, nz] over the whole (x, y)
    rectangle, so its area is a fixed multiple of the rectangle's: the
    area-weighted mean of a linear function is its value above the
    rectangle's centre."""
    xc, yc = m.nx / 2.0, m.ny / 2.0
    zc = (D0 - NORMAL[0] * xc - NORMAL[1] * yc) / NORMAL[2]
    return A0 + np.array([xc, yc, zc]) * HP @ GPLUS


def test_surface_potential_is_the_mean_over_the_plane():
    m, fs, u, qT, _ = _planar_case()
    zs = (D0 - NORMAL[0] * np.array([0, m.nx]) - NORMAL[1] * np.array([0, m.ny])[:, None]) / NORMAL[2]
    assert zs.min() > 0 and zs.max() < m.nz
    assert fs.surface_potential(u, qT) == pytest.approx(_surface_mean_exact(m), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("qscale", [0.0, -1.0])
def test_surface_potential_pin_fails_on_planted_mistake(qscale):
    m, fs, u, qT, _ = _planar_case()
    got = fs.surface_potential(u, qscale * qT)
    assert abs(got - _surface_mean_exact(m)) > 1e-3


# ---------------------------------------------------------------------------
# cut-cell fallback scan
# ---------------------------------------------------------------------------

# (cut cells as offsets from the centre cell (1, 1, 1) of a 3^3 mesh, expected
# offset of the cell that takes a hit in the centre cell, why)
FALLBACK_CASES = [
    ([(1, 0, 0), (0, 0, 1)], (1, 0, 0), "same L1: the smaller dz comes first"),
    ([(1, 1, 0), (0, 0, 1)], (0, 0, 1), "the smaller L1 distance wins over a smaller dz"),
    ([(-1, 1, 0), (1, -1, 0)], (1, -1, 0), "same L1 and dz: the smaller dy comes first"),
    ([(1, 0, 1), (-1, 0, 1)], (-1, 0, 1), "same L1, dz and dy: the smaller dx comes first"),
    ([(1, 1, 1)], (1, 1, 1), "a corner neighbour is within reach"),
    ([(0, -1, -1), (-1, 0, -1), (0, 0, 1)], (0, 0, 1), "L1 1 before the L1-2 cells"),
    ([(-1, -1, 1), (1, 1, -1)], (1, 1, -1), "same L1: dz -1 before dz +1"),
]


def _fallback_target(cut_offsets, mesh_n=3, centre=(1, 1, 1)):
    m = Mesh(mesh_n, mesh_n, mesh_n, 1.0)
    fs = FieldSystem(m, NoObject(), [("D", 0.0)] * 6)
    cells = [m.cell(centre[0] + dx, centre[1] + dy, centre[2] + dz) for dx, dy, dz in cut_offsets]
    fs.it_cell = np.array(cells, dtype=np.int64)
    fs.it_area = np.full(len(cells), 0.5)
    fs.it_kind = np.zeros(len(cells), dtype=np.int64)
    fs._setup_cut_cells()
    t = fs.cell_to_acc[m.cell(*centre)]
    if t < 0:
        return None
    c = int(fs.cut_cells[t])
    ci, cj, ck = c % m.nx, (c // m.nx) % m.ny, c // (m.nx * m.ny)
    return (ci - centre[0], cj - centre[1], ck - centre[2])


@pytest.mark.parametrize("cut,want,why", FALLBACK_CASES)
def test_cut_cell_fallback_order(cut, want, why):
    assert _fallback_target(cut) == want, why


def test_cut_cell_fallback_reach_and_self():
    # a cut cell two cells away is out of reach: the charge is lost
    assert _fallback_target([(3, 3, 3)], mesh_n=5) is None
    # a cut cell takes its own hits whatever its neighbours
    assert _fallback_target([(0, 0, 0), (1, 0, 0)]) == (0, 0, 0)


@pytest.mark.parametrize("order", ["dx_dy_dz", "no_l1"])
def test_cut_cell_fallback_pin_fails_on_planted_mistake(monkeypatch, order):
    offs = [o for o in ofield._SCAN]
    if order == "dx_dy_dz":
        wrong = sorted(offs, key=lambda o: (abs(o[0]) + abs(o[1]) + abs(o[2]), o[0], o[1], o[2]))
    else:
        wrong = sorted(offs, key=lambda o: (o[2], o[1], o[0]))
    monkeypatch.setattr(ofield, "_SCAN", wrong)
    failures = sum(_fallback_target(cut) != want for cut, want, _ in FALLBACK_CASES)
    assert failures > 0
