"""Pins of the oracle's hybrid grid (Sec. 2.2: the IFE mesh may have a different
resolution from the PIC mesh; oracle/pic.py refine, geometry.Refined): the IFE
mesh is the PIC mesh refined r times, particles deposit on it and gather at the
PIC nodes, which are IFE nodes."""
import numpy as np
import pytest

from oracle import particles as pt
from oracle.field import FieldSystem
from oracle.geometry import Mesh, Plane, Sphere, set_bedrock
from oracle.pic import Simulation
from paper_2011_10214_gb300 import workloads as wl

BC = [("D", 0.0)] * 6


def _fine(mesh, r):
    return Mesh(r * mesh.nx, r * mesh.ny, r * mesh.nz, mesh.h / r, mesh.origin)


@pytest.mark.parametrize("r", [2, 4])
def test_refined_system_is_the_fine_mesh_system(r):
    """The hybrid grid's field system is, entry for entry, the system of the
    same physical object built directly on the fine mesh."""
    m = Mesh(6, 5, 4, 0.5, (0.1, -0.2, 0.3))
    sim = Simulation(m, Sphere(m, (1.6, 1.1, 1.2), 0.83, 4.0, 1.0), BC, 0.05, refine=r)
    fm = _fine(m, r)
    fs = FieldSystem(fm, Sphere(fm, (1.6, 1.1, 1.2), 0.83, 4.0, 1.0), BC)
    assert sim.fmesh.nnodes == fm.nnodes
    assert np.array_equal(sim.fs.it_cell, fs.it_cell) and np.array_equal(sim.fs.it_t, fs.it_t)
    assert abs(sim.fs.A - fs.A).max() == 0.0
    assert np.array_equal(sim.fs.cut_cells, fs.cut_cells)
    assert np.array_equal(sim.fs.cut_area, fs.cut_area)


def test_refined_bedrock_moves_to_fine_units():
    m = Mesh(4, 4, 8, 1.0)
    sim = Simulation(m, set_bedrock(Plane((0.0, 0.0, 1.0), 5.3, 4.0, 1.0), m, 2.6, 10.0),
                     [("N",)] * 5 + [("D", 0.0)], 0.05, refine=2)
    fm = _fine(m, 2)
    fs = FieldSystem(fm, set_bedrock(Plane((0.0, 0.0, 1.0), 10.6, 4.0, 1.0), fm, 2.6, 10.0),
                     [("N",)] * 5 + [("D", 0.0)])
    assert np.array_equal(sim.fs.it_kind, fs.it_kind) and (fs.it_kind == 1).any()
    assert abs(sim.fs.A - fs.A).max() == 0.0


def test_refined_deposit_restricts_to_the_pic_deposit():
    """The PIC nodes' trilinear hat functions are trilinear on every IFE cell,
    so restricting the IFE charge with the hat values at the IFE nodes gives
    the PIC charge; each particle's integer rounding moves it by at most 11
    units per node.  Totals are exact."""
    m = Mesh(6, 5, 7, 0.5)
    r = 2
    sim = Simulation(m, Sphere(m, (10.0, 10.0, 10.0), 0.1, 4.0, 1.0), BC, 0.05, refine=r)
    sim.add_species(-1.0, 1.0, 0.01)
    x, y, z, vx, vy, vz = wl.random_particles((6, 5, 7), 3000, 4, vth=1.0)
    sim.load_particles(0, x, y, z, vx, vy, vz, np.arange(len(x)))
    W = sim.deposit_all()[0]
    assert W.sum() == 2 ** 32 * len(x)
    Wp = pt.deposit(m, x, y, z)
    # restriction: sum over IFE nodes j of hat_i(x_j) W_j
    fm = sim.fmesh
    fi, fj, fk = fm.node_ijk()
    R = np.zeros(m.nnodes)
    xj, yj, zj = fi / r, fj / r, fk / r
    ci = np.minimum(np.floor(xj), m.nx - 1).astype(np.int64)
    cj = np.minimum(np.floor(yj), m.ny - 1).astype(np.int64)
    ck = np.minimum(np.floor(zj), m.nz - 1).astype(np.int64)
    fx, fy, fz = xj - ci, yj - cj, zj - ck
    for l in range(8):
        a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
        w = (fx if a else 1 - fx) * (fy if b else 1 - fy) * (fz if c else 1 - fz)
        np.add.at(R, m.node(ci + a, cj + b, ck + c), w * W)
    cnt = np.zeros(m.nnodes)
    i0, j0, k0, _ = pt.cell_and_weights(x, y, z)
    for nid in pt.node_ids(m, i0, j0, k0):
        np.add.at(cnt, nid, 1)
    assert np.all(np.abs(R - Wp) <= 11.0 * np.maximum(cnt, 1))


def test_pic_nodes_read_the_ife_field():
    m = Mesh(5, 4, 3, 1.0)
    sim = Simulation(m, Plane((0.0, 0.0, 1.0), 1.7, 4.0, 1.0), BC, 0.05, refine=2)
    E = np.random.default_rng(3).normal(size=(sim.fmesh.nnodes, 3))
    sim.set_external_E(E)
    i, j, k = m.node_ijk()
    assert np.array_equal(sim.E_pic(), E[sim.fmesh.node(2 * i, 2 * j, 2 * k)])


def test_hit_cell_is_the_ife_cell_of_the_crossing_point():
    """A particle crossing the plane z = 1.7 (PIC units) between x = 2.3 and 2.45
    is accumulated in the IFE cell (4, ., 3) of the crossing point."""
    m = Mesh(5, 4, 4, 1.0)
    sim = Simulation(m, Plane((0.0, 0.0, 1.0), 1.7, 4.0, 1.0), [("N",)] * 5 + [("D", 0.0)], 0.5, refine=2)
    sim.add_species(-1.0, 1.0, 0.01)
    sim.load_particles(0, np.array([2.3]), np.array([1.6]), np.array([1.8]), np.array([0.3]),
                       np.array([0.0]), np.array([-0.4]), np.array([0]))
    sim.set_external_E(np.zeros((sim.fmesh.nnodes, 3)))
    st = sim.step()
    assert st["collected"][0] == 1
    fm, fs = sim.fmesh, sim.fs
    xc = 2.3 + 0.1 / 0.2 * 0.15           # crossing point: t = (1.8 - 1.7) / 0.2 along the move
    cell = fm.cell(int(np.floor(2 * xc)), int(np.floor(2 * 1.6)), int(np.floor(2 * 1.7)))
    acc = fs.cell_to_acc[cell]
    assert acc >= 0 and sim.surf[acc, 0] == 1 and sim.surf[:, 0].sum() == 1


def test_refined_pic_loop_bookkeeping():
    """Counts, ids and surface charge stay consistent on a hybrid grid."""
    m = Mesh(8, 8, 8, 0.5)
    sim = Simulation(m, Sphere(m, (2.0, 2.0, 2.0), 0.8, 4.0, 1.0), BC, 0.1, refine=2)
    sim.add_species(-1.0, 1.0, 0.01)
    sim.load_maxwellian(0, 4, 1.0, (0.0, 0.0, 0.0), 5)
    sim.set_injection(0, 0b111111, 1.0, 1.0, (0.0, 0.0, 0.0), 5)
    n0 = len(sim.P[0]["x"])
    sim.solve()
    sim.leapfrog_init()
    inj = ab = co = 0
    for _ in range(5):
        st = sim.step()
        inj += st["injected"][0]; ab += st["absorbed"][0]; co += st["collected"][0]
        assert st["lost"][0] == 0
    assert len(sim.P[0]["x"]) == n0 + inj - ab - co
    assert sim.surf[:, 0].sum() == co
    assert sim.W[0].sum() == 2 ** 32 * len(sim.P[0]["x"])
    assert len(np.unique(sim.P[0]["id"])) == len(sim.P[0]["id"])
