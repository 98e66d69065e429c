"""Pins of the oracle's reflecting particle faces (pt.reflect; the paper
reflects particles at its symmetry plane, Sec. 5.2.2)."""
import numpy as np
import pytest

from oracle import particles as pt
from oracle.geometry import Mesh, NoObject
from oracle.pic import Simulation


def _triangle(u, n):
    """Position of an unfolded coordinate u in a box [0, n] with mirror walls."""
    w = np.mod(u, 2.0 * n)
    return np.where(w <= n, w, 2.0 * n - w)


def test_bounce_follows_the_unfolded_line():
    m = Mesh(6, 5, 4, 1.0)
    sim = Simulation(m, NoObject(), [("D", 0.0)] * 6, 0.1)
    sim.add_species(-1.0, 1.0, 0.01)
    sim.set_particle_bc(0, ["reflect"] * 6)
    x0 = np.array([0.3, 2.5, 5.7]); y0 = np.array([1.1, 4.9, 0.2]); z0 = np.array([3.3, 0.4, 2.0])
    vx = np.array([-5.3, 3.7, 4.1]); vy = np.array([2.9, -6.1, 1.3]); vz = np.array([-1.7, 2.3, -3.9])
    sim.load_particles(0, x0, y0, z0, vx, vy, vz)
    sim.set_external_E(np.zeros((m.nnodes, 3)))
    sim.solve()
    K = 60
    for _ in range(K):
        sim.step()
    P = sim.P[0]
    o = np.argsort(P["id"])
    t = K * sim.dth
    for key, p0, v, n in (("x", x0, vx, m.nx), ("y", y0, vy, m.ny), ("z", z0, vz, m.nz)):
        assert np.allclose(P[key][o], _triangle(p0 + v * t, n), atol=1e-11), key
    # speeds unchanged, directions per the number of wall hits
    assert np.allclose(np.abs(P["vx"][o]), np.abs(vx)) and np.allclose(np.abs(P["vy"][o]), np.abs(vy))


def test_reflecting_box_keeps_every_particle():
    m = Mesh(8, 8, 8, 0.5)
    sim = Simulation(m, NoObject(), [("D", 0.0)] * 6, 0.2)
    sim.add_species(-1.0, 1.0, 0.01)
    sim.set_particle_bc(0, ["reflect"] * 6)
    g = np.random.default_rng(3)
    n = 4000
    sim.load_particles(0, g.uniform(0, 8, n), g.uniform(0, 8, n), g.uniform(0, 8, n), *g.normal(0, 3.0, (3, n)))
    sim.set_external_E(g.normal(0, 0.5, (m.nnodes, 3)))
    sim.solve()
    for _ in range(20):
        st = sim.step()
        assert st["absorbed"][0] == 0
    P = sim.P[0]
    assert len(P["x"]) == n
    for k, nn in (("x", m.nx), ("y", m.ny), ("z", m.nz)):
        assert P[k].min() >= 0.0 and P[k].max() < nn


def test_mirror_onto_the_plus_face_stays_inside():
    m = Mesh(4, 4, 4, 1.0)
    P = dict(x=np.array([4.0, 5.0, 4.25]), y=np.zeros(3) + 1.0, z=np.zeros(3) + 1.0,
             vx=np.array([1.0, 2.0, 3.0]), vy=np.zeros(3), vz=np.zeros(3))
    pt.reflect(m, P, 0b000010)
    assert P["x"][0] == np.nextafter(4.0, 0.0) and P["x"][1] == 3.0 and P["x"][2] == 3.75
    assert list(P["vx"]) == [-1.0, -2.0, -3.0]


def test_reflecting_face_cannot_inject():
    m = Mesh(4, 4, 4, 1.0)
    sim = Simulation(m, NoObject(), [("D", 0.0)] * 6, 0.1)
    sim.add_species(-1.0, 1.0, 0.01)
    sim.set_particle_bc(0, ["reflect", "absorb", "absorb", "absorb", "absorb", "absorb"])
    with pytest.raises(ValueError):
        sim.set_injection(0, 0b000001, 1.0, 1.0, (0, 0, 0), 1)
