"""Pins of the oracle's layered ground (geometry.set_bedrock, field.FieldSystem;
Sec. 5.2.1: regolith over bedrock under the lunar surface) and of the
rim-crater surface (geometry.RimCrater), against closed forms."""
import numpy as np
import pytest

from oracle.field import FieldSystem
from oracle.geometry import Mesh, Plane, RimCrater, set_bedrock
from oracle.photo import Photoemission

# three layers on a 4 x 4-cell column of height 12: bedrock below z_b, regolith
# up to z_g, vacuum above; phi fixed at the bottom and the top, zero Neumann on
# the sides (all lengths physical)
HEIGHT, ZB, ZG = 12.0, 3.6, 7.3
EB, ER, EV = 10.0, 4.0, 1.0
V_BOT, V_TOP = 0.0, 1.0
BC = [("N",)] * 4 + [("D", V_BOT), ("D", V_TOP)]


def _column(nz, bed=True):
    h = HEIGHT / nz
    m = Mesh(4, 4, nz, h)
    obj = Plane((0.0, 0.0, 1.0), ZG / h, ER, EV)
    if bed:
        set_bedrock(obj, m, ZB, EB)
    return m, FieldSystem(m, obj, BC)


def _exact_column(z, sigma=0.0):
    """1-D series capacitor: flux D = -eps phi' constant inside the object and
    D + sigma above the surface (Gauss); phi piecewise linear, continuous."""
    a = ZB / EB + (ZG - ZB) / ER + (HEIGHT - ZG) / EV
    D = -((V_TOP - V_BOT) + sigma * (HEIGHT - ZG) / EV) / a
    phi_b = V_BOT - D * ZB / EB
    phi_g = phi_b - D * (ZG - ZB) / ER
    return np.where(z <= ZB, V_BOT - D * z / EB,
                    np.where(z <= ZG, phi_b - D * (z - ZB) / ER, phi_g - (D + sigma) * (z - ZG) / EV))


def _column_error(nz, sigma=0.0, bed=True):
    m, fs = _column(nz, bed)
    qT = fs.q_tets(sigma * fs.cut_area) if sigma else np.zeros(len(fs.it_cell))
    phi, _, _ = fs.solve(np.zeros(m.nnodes), qT, tol=1e-14, maxit=20000)
    _, _, nk = m.node_ijk()
    return np.abs(phi - _exact_column(nk * m.h, sigma)).max(), fs


def test_bedrock_plane_is_a_plane_interface():
    """Inside an object that fills the box, the bedrock plane is the only
    interface: the system must be the one of a plane object with the bedrock on
    its minus side and the regolith on its plus side, entry for entry."""
    m = Mesh(4, 4, 12, 1.0)
    fs1 = FieldSystem(m, set_bedrock(Plane((0.0, 0.0, 1.0), 30.0, ER, EV), m, ZB, EB), BC)
    fs2 = FieldSystem(m, Plane((0.0, 0.0, 1.0), ZB, EB, ER), BC)
    assert np.all(fs1.it_kind == 1) and len(fs1.it_kind) == len(fs2.it_kind) > 0
    assert abs(fs1.A - fs2.A).max() == 0.0
    assert len(fs1.cut_cells) == 0 and np.all(fs1.it_acc == -1)
    p1, _, _ = fs1.solve(np.zeros(m.nnodes), np.zeros(len(fs1.it_cell)), tol=1e-14, maxit=5000)
    p2, _, _ = fs2.solve(np.zeros(m.nnodes), np.zeros(len(fs2.it_cell)), tol=1e-14, maxit=5000)
    assert np.abs(p1 - p2).max() == 0.0


def test_three_layer_column_converges_to_the_series_capacitor():
    """The layered column approaches the exact piecewise-linear potential as the
    mesh is refined (the linear IFE space is not conforming across interface
    elements, so it is not exact on a coarse mesh).  Reading the bedrock as
    regolith leaves an O(1) error on every mesh."""
    e12, fs = _column_error(12)
    e48, _ = _column_error(48)
    assert np.bincount(fs.it_kind, minlength=2).min() > 0
    assert e12 < 6e-3 and e48 < 1.5e-3
    assert _column_error(48, bed=False)[0] > 5e-2


def test_surface_charge_sits_on_the_surface_only():
    """A surface charge sigma on the ground: the flux jumps by sigma at z_g and
    nowhere else; the bedrock-plane tets carry no charge and no area."""
    e48, fs = _column_error(48, sigma=0.37)
    assert e48 < 1.5e-3
    qT = fs.q_tets(0.37 * fs.cut_area)
    assert np.all(qT[fs.it_kind == 1] == 0.0) and np.all(qT[fs.it_kind == 0] != 0.0)
    assert np.all(fs.it_acc[fs.it_kind == 1] == -1)
    assert len(fs.cut_cells) == 16                    # one layer of the 4 x 4 column
    assert abs(fs.cut_area.sum() - 16.0 * fs.mesh.h ** 2) < 1e-12


def test_node_field_in_each_layer():
    """Away from the interfaces E = -phi' of the layer, D / eps."""
    m, fs = _column(48)
    phi, _, _ = fs.solve(np.zeros(m.nnodes), np.zeros(len(fs.it_cell)), tol=1e-14, maxit=20000)
    E = fs.node_E(phi, np.zeros(len(fs.it_cell)))
    _, _, nk = m.node_ijk()
    a = ZB / EB + (ZG - ZB) / ER + (HEIGHT - ZG) / EV
    D = -(V_TOP - V_BOT) / a
    for z, eps in ((1.5, EB), (5.5, ER), (10.0, EV)):
        sel = nk == int(round(z / m.h))
        assert np.allclose(E[sel, 2], D / eps, rtol=2e-2)
        assert np.allclose(E[sel, :2], 0.0, atol=1e-3 * abs(D))


def test_bedrock_must_lie_inside_the_object():
    m = Mesh(4, 4, 12, 1.0)
    obj = set_bedrock(Plane((0.0, 0.0, 1.0), ZG, ER, EV), m, ZG + 1.0, EB)
    with pytest.raises(ValueError):
        FieldSystem(m, obj, BC)


def test_rim_crater_profile():
    m = Mesh(64, 64, 32, 1.0)
    zg, xc, yc, ri, rt, ro, H, D = 10.0, 32.0, 30.0, 6.0, 11.0, 17.0, 2.5, 3.5
    c = RimCrater(m, zg, xc, yc, ri, rt, ro, H, D, 4.0, 1.0)

    def zs(r):
        return float(c.surface(np.array(xc + r), np.array(yc)))

    assert zs(0.0) == zg - D and zs(ri) == zg - D           # flat floor
    assert zs(rt) == zg + H                                 # rim top
    assert zs(ro) == zg and zs(ro + 5.0) == zg              # ground
    assert abs(zs(0.5 * (ri + rt)) - (zg - D + 0.5 * (D + H))) < 1e-13   # smoothstep midpoints
    assert abs(zs(0.5 * (rt + ro)) - (zg + 0.5 * H)) < 1e-13
    # continuous with a continuous slope at the three radii
    for r0 in (ri, rt, ro):
        e = 1e-6
        assert abs(zs(r0 + e) - zs(r0 - e)) < 1e-5
        s_in = (zs(r0) - zs(r0 - e)) / e
        s_out = (zs(r0 + e) - zs(r0)) / e
        assert abs(s_in - s_out) < 1e-4
    # the level set is z - z_s, radially symmetric
    assert float(c.L(np.array(xc), np.array(yc + 7.0), np.array(5.0))) == 5.0 - zs(7.0)


def test_photoemission_ignores_the_bedrock_plane():
    """Bedrock under a sunlit ground changes no emitting tet and no rate."""
    m = Mesh(8, 8, 10, 1.0)
    sun = (-0.5, 0.0, 0.8)
    rates = []
    for bed in (False, True):
        obj = Plane((0.0, 0.0, 1.0), 6.3, 4.0, 1.0)
        if bed:
            set_bedrock(obj, m, 2.5, 10.0)
        fs = FieldSystem(m, obj, [("N",)] * 5 + [("D", 0.0)])
        ph = Photoemission(fs, 0, sun, 1.0, 1.0, 0.01, 0.05, 3)
        assert all(int(fs.it_kind[d["T"]]) == 0 for d in ph.tets)
        rates.append((len(ph.tets), int(ph.Q.sum())))
    assert rates[0] == rates[1]
