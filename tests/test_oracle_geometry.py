"""Pins of oracle.geometry: the 5-tet split, the P1 stencil and the IFE local spaces.

Each check is fixed by mathematics independent of the oracle's own formulas
(volumes, conformity, closed-form P1 element integrals, a divided-difference
volume formula, the interface conditions of Sec. 2.1 Eqs. 2.4-2.5).
"""
import itertools

import numpy as np
import pytest

from oracle.geometry import (TETS, VERT_OFF, CapCrater, Mesh, NoObject, Plane, Sphere, ife_local,
                             interface_pieces, regular_grad_table, tet_volume)
from oracle.field import FieldSystem


def test_five_tets_tile_the_cube():
    for p in range(2):
        vols = [tet_volume(*(VERT_OFF[list(t)].astype(float))) for t in TETS[p]]
        assert abs(sum(vols) - 1.0) < 1e-15
        assert abs(vols[0] - 1.0 / 3.0) < 1e-15 and all(abs(v - 1.0 / 6.0) < 1e-15 for v in vols[1:])
        # central tet: the 4 vertices of one global parity; corners: odd vertex + 3 axis neighbours
        assert len(set(TETS[p][0])) == 4


def test_split_is_conforming_across_faces():
    """Every cube face is cut along the same diagonal from both sides."""
    def face_diagonals(i, j, k):
        par = (i + j + k) % 2
        edges = set()
        for t in TETS[par]:
            for a, b in itertools.combinations(t, 2):
                pa = tuple(np.array((i, j, k)) + VERT_OFF[a])
                pb = tuple(np.array((i, j, k)) + VERT_OFF[b])
                edges.add(frozenset((pa, pb)))
        return edges
    e0 = face_diagonals(0, 0, 0)
    for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        e1 = face_diagonals(*d)
        shared = [e for e in e0 | e1 if all(np.dot(np.array(v) - 0, d) == 1 for v in e)]
        for e in shared:     # an edge on the common face is in both cubes' split
            assert e in e0 and e in e1


def test_regular_stencil_closed_form():
    """P1 patch: eps constant, no interface -> assembled rows equal the closed-form
    stencil (odd: 4 eps h, -2 eps h/3 on 6 axis neighbours; even: 6 eps h,
    -2 eps h/3 axis, -eps h/6 on 12 face diagonals); row sums vanish."""
    h, eps = 0.37, 2.5
    m = Mesh(4, 4, 4, h)
    fs = FieldSystem(m, NoObject(eps), [("N",)] * 6)
    A = fs.A.toarray()
    assert np.abs(A.sum(axis=1)).max() < 1e-13
    for (i, j, k) in [(2, 2, 2), (1, 2, 2), (2, 1, 1), (1, 1, 1)]:
        r = A[m.node(i, j, k)]
        even = (i + j + k) % 2 == 0
        assert r[m.node(i, j, k)] == pytest.approx((6.0 if even else 4.0) * eps * h, rel=1e-14)
        for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            for s in (1, -1):
                assert r[m.node(i + s * d[0], j + s * d[1], k + s * d[2])] == pytest.approx(-2 * eps * h / 3, rel=1e-14)
        fd = [(a, b, 0) for a in (1, -1) for b in (1, -1)] + [(a, 0, b) for a in (1, -1) for b in (1, -1)] \
            + [(0, a, b) for a in (1, -1) for b in (1, -1)]
        for d in fd:
            v = r[m.node(i + d[0], j + d[1], k + d[2])]
            assert v == pytest.approx(-eps * h / 6, rel=1e-14) if even else v == 0.0
        assert np.count_nonzero(np.abs(r) > 1e-15) == (19 if even else 7)


def test_patch_linear_reproduced():
    """Any globally linear phi lies in the FE space: the discrete solution with
    linear Dirichlet data and no source is that linear function to round-off."""
    m = Mesh(5, 4, 6, 0.3)
    fs = FieldSystem(m, NoObject(3.0), [("D", 0.0)] * 6)
    i, j, k = m.node_ijk()
    u = 0.3 + 1.7 * i * m.h - 0.4 * j * m.h + 2.2 * k * m.h
    fs.g[:] = np.where(fs.is_dir, u, 0.0)
    phi, it, _ = fs.solve(np.zeros(m.nnodes), np.zeros(0), tol=1e-14, maxit=500)
    assert np.abs(phi - u).max() < 1e-12
    E = fs.node_E(phi, np.zeros(0))
    assert np.abs(E - np.array([-1.7, 0.4, -2.2])).max() < 1e-11


def _random_interface_tets(nt, seed):
    g = np.random.default_rng(seed)
    out = []
    h = 0.5
    while len(out) < nt:
        p = g.integers(0, 2)
        t = g.integers(0, 5)
        verts = VERT_OFF[list(TETS[p][t])].astype(float) * h
        Lv = g.normal(size=4)
        if (Lv < 0).any() and (Lv >= 0).any():
            out.append((verts, Lv))
    return out


@pytest.mark.parametrize("ratio", [(4.0, 1.0), (1.0, 10.0), (2.0, 2.0)])
def test_ife_local_interface_conditions(ratio):
    """P7: psi_i(v_j) = delta_ij (piece of v_j), continuity on Gamma_h, flux jump
    0 for the basis and q for the jump function, partition of unity."""
    em, ep = ratio
    for verts, Lv in _random_interface_tets(50, 7):
        d = ife_local(verts, Lv, em, ep)
        coef, n, gp, gm = d["coef"], d["n"], d["gp"], d["gm"]
        minus = Lv < 0
        for f in range(5):
            for v in range(4):
                val = coef[0, f] + verts[v] @ coef[1:, f]
                if minus[v]:
                    val += d["beta"][f] * d["dist"][v]
                expect = (1.0 if f == v else 0.0) if f < 4 else 0.0
                assert abs(val - expect) < 1e-10
            jump = ep * (n @ gp[f]) - em * (n @ gm[f])
            assert abs(jump - (1.0 if f == 4 else 0.0)) < 1e-10
            # tangential gradient continuous across Gamma_h
            tg = (gp[f] - gm[f]) - ((gp[f] - gm[f]) @ n) * n
            assert np.abs(tg).max() < 1e-10
        assert np.abs(gp[:4].sum(axis=0)).max() < 1e-9 and np.abs(gm[:4].sum(axis=0)).max() < 1e-9
        assert abs(coef[0, :4].sum() - 1.0) < 1e-12
        # the interface plane passes through the cut points: psi+ == psi- there
        for tri in d["tris"]:
            for pnt in tri:          # signed distance of every cut point to Gamma_h's plane
                assert abs((pnt - verts[0]) @ n + d["dist"][0]) < 1e-12
        assert np.allclose(d["K"], d["K"].T, atol=1e-14)
        w = np.linalg.eigvalsh(d["K"])
        assert w.min() > -1e-12 and abs(d["K"].sum()) < 1e-10


def _frac_negative(Lv):
    """Independent closed form: vol{L < 0}/V = sum_i (-l_i)_+^3 / prod_{j!=i}(l_j - l_i)
    (third divided difference of x_+^3 / 3! times 3!) for distinct values."""
    l = -np.asarray(Lv, dtype=float)
    s = 0.0
    for i in range(4):
        if l[i] > 0:
            den = 1.0
            for j in range(4):
                if j != i:
                    den *= l[i] - l[j]
            s += l[i] ** 3 / den
    return s


def test_subvolumes_match_divided_difference_formula():
    for verts, Lv in _random_interface_tets(200, 3):
        vm, vp, tris = interface_pieces(verts, Lv)
        V = tet_volume(*verts)
        assert abs(vm / V - _frac_negative(Lv)) < 1e-9
        assert abs(vm + vp - V) < 1e-15


def test_ife_equals_p1_when_no_jump():
    """eps- == eps+, q = 0: the IFE basis is the standard P1 basis."""
    G, V = regular_grad_table(0.5)
    g = np.random.default_rng(11)
    for p in range(2):
        for t in range(5):
            verts = VERT_OFF[list(TETS[p][t])].astype(float) * 0.5
            Lv = np.array([-1.0, 0.4, 0.7, -0.3]) + 0.1 * g.normal(size=4)
            d = ife_local(verts, Lv, 3.0, 3.0)
            assert np.allclose(d["gp"][:4], G[p][t], atol=1e-12)
            assert np.allclose(d["K"], 3.0 * V[t] * G[p][t] @ G[p][t].T, atol=1e-12)


def test_sphere_area_and_volume_converge():
    """Gamma_h area -> 4 pi R^2 and |Omega^-| -> 4/3 pi R^3 at second order."""
    errs_a, errs_v = [], []
    for n in (8, 16, 32):
        h = 2.0 / n
        m = Mesh(n, n, n, h, origin=(-1, -1, -1))
        R = 0.6183
        fs = FieldSystem(m, Sphere(m, (0, 0, 0), R, 4.0, 1.0), [("D", 0.0)] * 6)
        vol = sum(len(nodes) * Vt for nodes, Gt, Vt, plus in fs.reg if not plus) + fs.it_volm.sum()
        errs_a.append(abs(fs.it_area.sum() - 4 * np.pi * R ** 2))
        errs_v.append(abs(vol - 4 / 3 * np.pi * R ** 3))
    assert errs_a[1] / errs_a[2] > 3.0 and errs_v[1] / errs_v[2] > 3.0


def test_flat_ground_on_node_plane():
    """Ground plane through a node layer (the crater case's flat part): L == 0 nodes
    are in Omega^+, interface tets under the plane carry Gamma_h of area h^2 per cell."""
    m = Mesh(6, 6, 6, 1.0)
    obj = CapCrater(m, 3.0, 3.0, 3.0, 0.5, 0.25, 4.0, 1.0)     # tiny crater in the middle
    fs = FieldSystem(m, obj, [("N",)] * 5 + [("D", 0.0)])
    ground = [c for c in fs.cut_cells if m.cell_ijk()[2][c] == 2]
    i, j, k = m.cell_ijk()
    a = dict(zip(fs.cut_cells, fs.cut_area))
    far = [c for c in ground if (abs(i[c] + 0.5 - 3.0) > 1.2 or abs(j[c] + 0.5 - 3.0) > 1.2)]
    assert far and all(abs(a[c] - 1.0) < 1e-12 for c in far)
