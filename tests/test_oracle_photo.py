"""Pins of the oracle's photoemission (oracle/photo.py; Sec. 5.2.2: emission from
the sunlit surface by the local sunlight index) against closed forms,
distributions and exact integer identities."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle.field import FieldSystem
from oracle.geometry import CapCrater, Mesh, Plane
from oracle.photo import RATE_ONE, Photoemission
from oracle.pic import Simulation

DT = 0.05
W = 0.01


def _plane_case(theta_deg=30.0):
    m = Mesh(8, 8, 8, 0.5)
    obj = Plane((0.0, 0.0, 1.0), 3.3, 4.0, 1.0)
    fs = FieldSystem(m, obj, [("N",)] * 5 + [("D", 0.0)])
    th = math.radians(theta_deg)
    sun = (-math.cos(th), 0.0, math.sin(th))
    return m, obj, fs, sun, th


def test_flat_ground_normals_rate_and_no_shadow():
    m, obj, fs, sun, th = _plane_case()
    ph = Photoemission(fs, 0, sun, 1.0, 1.0, W, DT, 7)
    assert len(ph.tets) > 0
    for d in ph.tets:
        assert np.allclose(d["n"], (0.0, 0.0, 1.0), atol=1e-14)
        assert abs(d["S"] - math.sin(th)) < 1e-14
    # every cube of the cut layer emits (no shadow on a plane): the Gamma_h
    # pieces tile the plane, area nx * ny cells
    assert abs(sum(d["A"] for d in ph.tets) - m.nx * m.ny) < 1e-10
    J = 1.0 * 1.0 / math.sqrt(2.0 * math.pi)
    expect = J * math.sin(th) * (m.nx * m.ny * m.h * m.h) * DT / W
    assert abs(ph.rate_per_step() - expect) <= len(ph.tets) * 0.5 / RATE_ONE + 1e-12 * expect


def test_counts_are_exact_integer_floors():
    m, obj, fs, sun, th = _plane_case()
    ph = Photoemission(fs, 0, sun, 3.0, 1.0, W, DT, 7)
    K = 23
    total = 0
    for k in range(K):
        total += ph.emit(k)["count"]
    assert total == int(sum((K * q) // RATE_ONE for q in ph.Q))


def test_overhead_sun_lights_the_whole_crater():
    m = Mesh(24, 24, 12, 1.0)
    obj = CapCrater(m, 6.3, 12.0, 12.0, 8.0, 3.0, 4.0, 1.0)
    fs = FieldSystem(m, obj, [("N",)] * 5 + [("D", 0.0)])
    ph = Photoemission(fs, 0, (0.0, 0.0, 1.0), 1.0, 1.0, W, DT, 7)
    # every interface tet faces up, so every one emits
    assert len(ph.tets) == len(fs.it_cell)


def test_low_sun_shadows_match_the_analytic_bowl():
    """For a spherical-cap bowl the ray from a wall point towards the sun leaves
    the sphere at t* = -2 (c - C).s; it is blocked iff that exit lies below the
    rim plane.  Compare on tets whose exit is more than half a cell from it."""
    m = Mesh(24, 24, 12, 1.0)
    zg, a, D, xc, yc = 6.3, 8.0, 3.0, 12.0, 12.0
    obj = CapCrater(m, zg, xc, yc, a, D, 4.0, 1.0)
    fs = FieldSystem(m, obj, [("N",)] * 5 + [("D", 0.0)])
    th = math.radians(20.0)
    sun = np.array([-math.cos(th), 0.0, math.sin(th)])
    ph = Photoemission(fs, 0, sun, 1.0, 1.0, W, DT, 7)
    lit = {d["T"] for d in ph.tets}
    Rs = (a * a + D * D) / (2 * D)
    C = np.array([xc, yc, zg - D + Rs])
    from oracle.photo import gamma_triangles, tri_area_cells
    from oracle.geometry import TETS, regular_grad_table
    G, _ = regular_grad_table(1.0)
    checked = shadowed_n = 0
    for T in range(len(fs.it_cell)):
        c = int(fs.it_cell[T])
        ci, cj, ck = c % m.nx, (c // m.nx) % m.ny, c // (m.nx * m.ny)
        p = (ci + cj + ck) & 1
        Lv = fs.Lnode[fs.it_nodes[T]]
        g = sum(Lv[v] * G[p][int(fs.it_t[T])][v] for v in range(4))
        if g @ sun <= 0:
            continue                      # faces away: never emits
        tris = [P + np.array([ci, cj, ck], float) for P in gamma_triangles(Lv, TETS[p][int(fs.it_t[T])])]
        ar = [tri_area_cells(P) for P in tris]
        if sum(ar) <= 0:
            continue
        cen = sum(a_ * P.mean(axis=0) for a_, P in zip(ar, tris)) / sum(ar)
        if (cen[0] - xc) ** 2 + (cen[1] - yc) ** 2 >= (a - 1.0) ** 2:
            continue                      # flat ground or the rim: never shadowed by the bowl
        tstar = -2.0 * (cen - C) @ sun
        ez = cen[2] + tstar * sun[2]
        if abs(ez - zg) < 0.5:
            continue
        checked += 1
        blocked = ez < zg
        shadowed_n += blocked
        assert (T not in lit) == blocked, (T, ez)
    assert checked > 50 and 0 < shadowed_n < checked


def test_emitted_speeds_and_positions():
    m, obj, fs, sun, th = _plane_case()
    vth = 1.3
    ph = Photoemission(fs, 0, sun, 40.0, vth, W, DT, 11)
    P0, V = [], []
    for k in range(12):
        out = ph.emit(k)
        P0.append(out["p0"][out["ok"]])
        V.append(np.stack([out["vx"], out["vy"], out["vz"]], axis=1)[out["ok"]])
    P0, V = np.concatenate(P0), np.concatenate(V)
    assert len(V) > 5000
    # start points on the plane, uniform over it
    assert np.abs(P0[:, 2] - 3.3).max() < 1e-12
    assert stats.kstest(P0[:, 0] / m.nx, "uniform").pvalue > 1e-3
    assert stats.kstest(P0[:, 1] / m.ny, "uniform").pvalue > 1e-3
    # normal speed: flux-weighted half-Maxwellian (Rayleigh); tangential: Gaussian
    assert stats.kstest(V[:, 2] / vth, lambda v: 1.0 - np.exp(-0.5 * v * v)).pvalue > 1e-3
    assert stats.kstest(V[:, 0] / vth, "norm").pvalue > 1e-3
    assert stats.kstest(V[:, 1] / vth, "norm").pvalue > 1e-3


def test_pic_loop_charge_and_count_bookkeeping():
    m, obj, fs, sun, th = _plane_case()
    sim = Simulation(m, obj, [("N",)] * 5 + [("D", 0.0)], DT)
    sim.add_species(-1.0, 1.0, W)
    sim.set_photoemission(0, sun, 5.0, 1.0, 3)
    sim.set_external_E(np.zeros((m.nnodes, 3)))
    sim.solve()
    n_emit = n_abs = n_col = 0
    for _ in range(15):
        st = sim.step()
        n_emit += st["injected"][0]
        n_abs += st["absorbed"][0]
        n_col += st["collected"][0]
    assert n_emit > 0
    assert len(sim.P[0]["x"]) == n_emit - n_abs - n_col
    # every emitted electron left one count behind; every collected one returned one
    assert sim.surf[:, 0].sum() == n_col - n_emit
    assert len(np.unique(sim.P[0]["id"])) == len(sim.P[0]["id"])
