"""Photoelectron emission from the sunlit, unshadowed object surface (oracle;
test infrastructure only -- only tests/, the smoke check and the bench's CPU
baseline import this package).

Sec. 5.2.2 states that photoelectrons are generated at the sunlit regions
according to the local sunlight index, the inner product of the sun vector and
the local surface normal (Fig. 12a).  Everything else is silent; the readings
below are this oracle's (and the CUDA path's) definition:

  * emitting element: every interface tet T, through its Gamma_h piece (the
    triangles of the zero set of the linear interpolant of the nodal level set,
    computed here in cell units);
  * normal n_T = grad L_h / |grad L_h| (from the object into the plasma) with
    grad L_h = sum_v L_v G_v, G the P1 basis gradients of the tet shape (h = 1),
    summed in vertex order;
  * sunlight index S_T = max(0, n_T . s), s the unit vector towards the sun;
  * shadow: T does not emit if a ray from its Gamma_h centroid towards the sun
    enters the object: the analytic level set is sampled at steps of 1/4 cell
    until the ray leaves the box, and any negative sample shadows T;
  * emitted flux at normal incidence J = n vth / sqrt(2 pi) (the one-sided flux
    of a Maxwellian of density n); rate per step R_T = J S_T A_T dt / w with A_T
    the physical Gamma_h area; R_T is held in fixed point, Q_T = rint(R_T 2^20),
    and the count per step is the integer part of carry + Q_T (exact integers,
    so every implementation emits the same counts);
  * particle m of a step (m counts all emissions of the step in tet order) uses
    the Philox streams of purpose PHOTO with counter (m, block, 0, 0): block 0
    picks the triangle (u A_T < A_tri0), the point on it (sqrt(r1), r2) and the
    fraction U of the first step; block 1 the tangential normals; blocks 2.. the
    flux-weighted normal speed (the injection sampler with zero drift);
  * velocity vth (v_n n + g1 t1 + g2 t2), t1 = n x e / |n x e| with e the axis
    least aligned with n (first of x, y, z on ties), t2 = n x t1;
  * position p + v U dt/h (cell units); a particle whose partial step ends
    inside the object is not emitted (it would be re-collected at once, no net
    charge); one that ends outside the box is emitted and absorbed;
  * each emitted particle takes its charge away from the surface: the cut-cell
    accumulator of its tet's cell loses one count of the emitting species.
"""
import math

import numpy as np

from . import rng
from .geometry import TETS, VERT_OFF, regular_grad_table
from .particles import MAX_TRIES, flux_normal_speed

RATE_BITS = 20
RATE_ONE = 1 << RATE_BITS
RAY_STEP = 0.25


def gamma_triangles(Lv, tv):
    """Triangles of Gamma_h on one tet in cube-local cell units: same cut and
    triangulation as geometry.interface_pieces (1-3 split: one triangle over the
    three cut edges in tet order; 2-2 split: two triangles of the quad)."""
    V = VERT_OFF[list(tv)].astype(np.float64)
    minus = Lv < 0
    mi = [v for v in range(4) if minus[v]]
    pl = [v for v in range(4) if not minus[v]]

    def cut(u, w):                       # u in Omega^-, w in Omega^+
        t = Lv[u] / (Lv[u] - Lv[w])
        return V[u] + t * (V[w] - V[u])

    if len(mi) == 1:
        return [np.array([cut(mi[0], w) for w in pl])]
    if len(mi) == 3:
        return [np.array([cut(w, pl[0]) for w in mi])]
    a, b = mi
    c, d = pl
    pac, pad, pbc, pbd = cut(a, c), cut(a, d), cut(b, c), cut(b, d)
    return [np.array([pac, pad, pbd]), np.array([pac, pbd, pbc])]


def tri_area_cells(P):
    e1 = P[1] - P[0]
    e2 = P[2] - P[0]
    c = np.array([e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]])
    return 0.5 * math.sqrt((c[0] * c[0] + c[1] * c[1]) + c[2] * c[2])


def tangent_basis(n):
    a = int(np.argmin(np.abs(n)))
    e = np.zeros(3)
    e[a] = 1.0
    c = np.array([n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]])
    t1 = c / math.sqrt((c[0] * c[0] + c[1] * c[1]) + c[2] * c[2])
    t2 = np.array([n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]])
    return t1, t2


def shadowed(obj, mesh, c, s):
    """Ray c + t s, t = RAY_STEP, 2 RAY_STEP, ... inside the box: True if the
    analytic level set is negative at any sample."""
    k = 1
    while True:
        t = RAY_STEP * k
        q = (c[0] + t * s[0], c[1] + t * s[1], c[2] + t * s[2])
        if q[0] < 0.0 or q[0] > mesh.nx or q[1] < 0.0 or q[1] > mesh.ny or q[2] < 0.0 or q[2] > mesh.nz:
            return False
        if float(obj.L(np.float64(q[0]), np.float64(q[1]), np.float64(q[2]))) < 0.0:
            return True
        k += 1


class Photoemission:
    """Emission set-up of one species (per-tet fixed-point rates) and the
    particles of each step."""

    def __init__(self, fs, species, sun_dir, density, vth, w, dt, seed):
        mesh, obj = fs.mesh, fs.obj
        s = np.asarray(sun_dir, dtype=np.float64)
        s = s / math.sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2])
        G, _ = regular_grad_table(1.0)
        J = density * vth / math.sqrt(2.0 * math.pi)
        h2 = mesh.h * mesh.h
        self.species, self.vth, self.seed = species, float(vth), int(seed)
        self.dth = dt / mesh.h
        rows = []
        for T in range(len(fs.it_cell)):
            if int(fs.it_kind[T]) != 0:
                continue                      # bedrock plane: not a surface
            c = int(fs.it_cell[T])
            ci, cj, ck = c % mesh.nx, (c // mesh.nx) % mesh.ny, c // (mesh.nx * mesh.ny)
            p = (ci + cj + ck) & 1
            t = int(fs.it_t[T])
            tv = TETS[p][t]
            Lv = fs.Lnode[fs.it_nodes[T]]
            g = Lv[0] * G[p][t][0]
            for v in range(1, 4):
                g = g + Lv[v] * G[p][t][v]
            n = g / math.sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2])
            S = max(0.0, (n[0] * s[0] + n[1] * s[1]) + n[2] * s[2])
            if S <= 0.0 or int(fs.it_acc[T]) < 0:
                continue
            base = np.array([ci, cj, ck], dtype=np.float64)
            tris = [P + base for P in gamma_triangles(Lv, tv)]
            areas = [tri_area_cells(P) for P in tris]
            A = areas[0] + (areas[1] if len(areas) > 1 else 0.0)
            if A <= 0.0:
                continue
            cen = (areas[0] / 3.0) * ((tris[0][0] + tris[0][1]) + tris[0][2])
            if len(tris) > 1:
                cen = cen + (areas[1] / 3.0) * ((tris[1][0] + tris[1][1]) + tris[1][2])
            cen = cen / A
            if shadowed(obj, mesh, cen, s):
                continue
            R = J * S * (A * h2) * dt / w
            Q = int(np.rint(R * RATE_ONE))
            if Q <= 0:
                continue
            t1, t2 = tangent_basis(n)
            rows.append(dict(T=T, acc=int(fs.it_acc[T]), Q=Q, n=n, t1=t1, t2=t2, tris=tris, areas=areas, A=A,
                             S=S, cen=cen))
        self.tets = rows
        self.Q = np.array([r["Q"] for r in rows], dtype=np.int64)
        self.carry = np.zeros(len(rows), dtype=np.int64)

    def rate_per_step(self):
        """Mean emitted particles per step (before the inside-object test)."""
        return float(self.Q.sum()) / RATE_ONE

    def emit(self, step):
        """Counts per emitting tet, then every particle of this step: dict of
        positions (cell units), velocities, the emitting tet's accumulator,
        the step index m and flags."""
        tot = self.carry + self.Q
        counts = tot >> RATE_BITS
        self.carry = tot & (RATE_ONE - 1)
        ntot = int(counts.sum())
        out = dict(x=np.zeros(ntot), y=np.zeros(ntot), z=np.zeros(ntot), vx=np.zeros(ntot), vy=np.zeros(ntot),
                   vz=np.zeros(ntot), p0=np.zeros((ntot, 3)), tet=np.zeros(ntot, dtype=np.int64),
                   acc=np.zeros(ntot, dtype=np.int64), ok=np.zeros(ntot, dtype=bool),
                   index=np.arange(ntot, dtype=np.int64), count=ntot)
        if ntot == 0:
            return out
        m = np.arange(ntot, dtype=np.uint64)
        key1 = rng.stream_key(rng.PURPOSE_PHOTO, self.species, 0, step)
        b0 = rng.philox4x64(m, 0, 0, 0, self.seed, key1)
        b1 = rng.philox4x64(m, 1, 0, 0, self.seed, key1)
        tries = []
        for t in range(MAX_TRIES):
            bt = rng.philox4x64(m, 2 + t, 0, 0, self.seed, key1)
            tries.append((rng.uniform(bt[0]), rng.uniform(bt[1]), rng.uniform(bt[2])))
        vn, ok = flux_normal_speed(tries, 0.0)
        g1, g2 = rng.box_muller(rng.uniform(b1[0]), rng.uniform(b1[1]))
        u_tri, r1, r2, U = (rng.uniform(b0[0]), rng.uniform(b0[1]), rng.uniform(b0[2]), rng.uniform(b0[3]))
        tet_of = np.repeat(np.arange(len(self.tets)), counts)
        for i in range(ntot):
            d = self.tets[tet_of[i]]
            k = 1 if (len(d["tris"]) > 1 and u_tri[i] * d["A"] >= d["areas"][0]) else 0
            P = d["tris"][k]
            sq = math.sqrt(r1[i])
            a0, a1, a2 = 1.0 - sq, sq * (1.0 - r2[i]), sq * r2[i]
            pt = (a0 * P[0] + a1 * P[1]) + a2 * P[2]
            vv = (((self.vth * vn[i]) * d["n"] + (self.vth * g1[i]) * d["t1"]) + (self.vth * g2[i]) * d["t2"])
            sl = U[i] * self.dth
            x = pt + vv * sl
            out["x"][i], out["y"][i], out["z"][i] = x
            out["vx"][i], out["vy"][i], out["vz"][i] = vv
            out["acc"][i] = d["acc"]
            out["p0"][i] = pt
            out["tet"][i] = tet_of[i]
        out["ok"] = ok
        return out
