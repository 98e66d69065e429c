"""The IFE-PIC loop (oracle; test infrastructure only).

Follows arXiv:2011.10214 Sec. 2.1 (Fig. 1: scatter -> field-solve -> gather ->
particle-push, repeated), Sec. 3.1.3 (pre-load before the initial field solve,
injection at open faces each step, absorption at open faces) and Sec. 5.2.2
(collection at the object surface with accumulated charge; the floating
potential follows from the non-homogeneous flux jump, Sec. 3.1.2).

One step (a reading of the loop's order):
  1. gather + push every particle with the current node field;
  2. mirror particles back at reflecting faces; remove particles outside the
     domain, then collect particles inside the object (their charge goes to the
     surface accumulator of the crossing cell);
  3. inject new particles at open faces (partial first step; same two tests),
     then emit photoelectrons from the sunlit surface (photo.py);
  4. scatter (fixed-point deposit) of all particles;
  5. field solve: right-hand side with the flux jump from the accumulated
     surface charge, Jacobi PCG warm-started from the previous potential;
  6. node field from the new potential.
"""
import math

import numpy as np

from .field import FieldSystem
from .geometry import Mesh, Refined
from . import particles as pt
from .photo import Photoemission

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "id")


class Species:
    def __init__(self, q, m, w, dt):
        self.q, self.m, self.w = float(q), float(m), float(w)
        self.k = (self.q / self.m) * dt      # (q/m) dt
        self.inj = None                      # (face_mask, density, vth, drift, seed)
        self.photo = None                    # photo.Photoemission of this species
        self.reflect = 0                     # reflecting particle faces (bit f = face f)
        self.carry = np.zeros(6)
        self.next_id = 0


def _empty():
    return {k: np.zeros(0, dtype=np.int64 if k == "id" else np.float64) for k in FIELDS}


class Simulation:
    """Plain FP64 IFE-PIC (Sec. 2.1, Fig. 1).

    mesh: geometry.Mesh (the PIC mesh); obj: a level-set object built on it;
    face_bc: 6 field BCs; dt: time step (1/omega_pe units); absorbing particle
    faces on all six sides.  refine: the IFE mesh is the PIC mesh with each
    cell split r x r x r (Sec. 2.2: PIC and IFE meshes may differ in
    resolution; r a power of two, 1 = the same mesh).  Particles move, gather
    and are binned on the PIC mesh; they deposit their charge on the IFE mesh
    (trilinear weights of the IFE cell); the node field is solved on the IFE
    mesh and read at the PIC nodes, which are IFE nodes.
    """

    def __init__(self, mesh, obj, face_bc, dt, tol=1e-6, maxit=150, refine=1):
        self.mesh, self.obj, self.dt = mesh, obj, float(dt)
        self.dth = self.dt / mesh.h
        self.r = int(refine)
        if self.r < 1 or (self.r & (self.r - 1)):
            raise ValueError("refine must be a power of two")
        if self.r == 1:
            self.fmesh, fobj = mesh, obj
        else:
            r = self.r
            self.fmesh = Mesh(r * mesh.nx, r * mesh.ny, r * mesh.nz, mesh.h / r, mesh.origin)
            fobj = Refined(obj, r)
        self.fs = FieldSystem(self.fmesh, fobj, face_bc)
        self.tol, self.maxit = tol, maxit
        self.species = []
        self.P = []
        self.surf = np.zeros((len(self.fs.cut_cells), 0), dtype=np.int64)
        self.phi = self.fs.g.copy()
        self.E = np.zeros((self.fmesh.nnodes, 3))
        self.W = None
        self.qT = np.zeros(len(self.fs.it_cell))
        self.external_E = False
        self.step_no = 0
        self.last = {}

    # -- set-up ----------------------------------------------------------------
    def add_species(self, q, m, w):
        self.species.append(Species(q, m, w, self.dt))
        self.P.append(_empty())
        self.surf = np.zeros((len(self.fs.cut_cells), len(self.species)), dtype=np.int64)
        return len(self.species) - 1

    def pic_nodes(self):
        """IFE node index of every PIC node (they coincide on a hybrid grid)."""
        m, r = self.mesh, self.r
        i, j, k = m.node_ijk()
        return self.fmesh.node(r * i, r * j, r * k)

    def E_pic(self):
        """The node field at the PIC nodes (what the gather reads)."""
        return self.E if self.r == 1 else self.E[self.pic_nodes()]

    def load_maxwellian(self, s, ppc, vth, drift, seed):
        P = pt.load_maxwellian(self.mesh, self.obj, seed, s, ppc, vth, drift)
        self.P[s] = {k: np.concatenate([self.P[s][k], P[k]]) for k in FIELDS}
        sp = self.species[s]
        sp.next_id = max(sp.next_id, self.mesh.ncells * ppc)

    def load_particles(self, s, x, y, z, vx, vy, vz, ids=None):
        n = len(x)
        if ids is None:
            ids = np.arange(self.species[s].next_id, self.species[s].next_id + n, dtype=np.int64)
        P = dict(x=x, y=y, z=z, vx=vx, vy=vy, vz=vz, id=np.asarray(ids, dtype=np.int64))
        self.P[s] = {k: np.concatenate([self.P[s][k], np.asarray(P[k])]) for k in FIELDS}
        self.species[s].next_id = max(self.species[s].next_id, int(np.max(ids)) + 1 if n else 0)

    def set_injection(self, s, face_mask, density, vth, drift, seed):
        if int(face_mask) & self.species[s].reflect:
            raise ValueError("a reflecting face cannot inject")
        self.species[s].inj = (int(face_mask), float(density), float(vth),
                               tuple(float(d) for d in drift), int(seed))

    def set_particle_bc(self, s, face_kinds):
        """Per face: "absorb" (default), "inject" (absorbing; injection is set by
        set_injection) or "reflect" (particles mirrored back, pt.reflect)."""
        mask = 0
        for f, kind in enumerate(face_kinds):
            if kind == "reflect":
                mask |= 1 << f
            elif kind not in ("absorb", "inject"):
                raise ValueError(kind)
        sp = self.species[s]
        if sp.inj is not None and (sp.inj[0] & mask):
            raise ValueError("a reflecting face cannot inject")
        sp.reflect = mask

    def set_photoemission(self, s, sun_dir, density, vth, seed):
        """Species s is emitted from the sunlit, unshadowed object surface (Sec. 5.2.2; photo.py)."""
        sp = self.species[s]
        sp.photo = Photoemission(self.fs, s, sun_dir, density, vth, sp.w, self.dt, seed)

    def injection_rate(self, s, f):
        """Expected macro-particles per step through face f (one-way flux x A dt / w)."""
        mask, dens, vth, drift, _ = self.species[s].inj
        m = self.mesh
        ax = pt.FACE_AXIS[f]
        t1, t2 = pt.face_tangents(f)
        n_axes = (m.nx, m.ny, m.nz)
        area = (n_axes[t1] * m.h) * (n_axes[t2] * m.h)
        vdn = pt.FACE_SIGN[f] * drift[ax]
        return pt.flux_density(dens, vth, vdn) * area * self.dt / self.species[s].w

    def set_external_E(self, E):
        """Freeze the node field (given at the IFE nodes)."""
        self.E = np.array(E, dtype=np.float64).reshape(-1, 3)
        self.external_E = True

    # -- scatter / field-solve ---------------------------------------------------
    def deposit_all(self):
        """Fixed-point charge of every particle on the IFE nodes (positions
        scaled to IFE cell units: exact, r a power of two)."""
        r = float(self.r)
        self.W = np.stack([pt.deposit(self.fmesh, r * P["x"], r * P["y"], r * P["z"]) for P in self.P]) \
            if self.P else np.zeros((0, self.fmesh.nnodes), dtype=np.int64)
        return self.W

    def node_load(self):
        F = np.zeros(self.fmesh.nnodes)
        for s, sp in enumerate(self.species):
            F = F + ((sp.q * sp.w) / 4294967296.0) * self.W[s].astype(np.float64)
        return F

    def cut_charge(self):
        Q = np.zeros(len(self.fs.cut_cells))
        for s, sp in enumerate(self.species):
            Q = Q + (sp.q * sp.w) * self.surf[:, s].astype(np.float64)
        return Q

    def solve(self):
        """Scatter, then the IFE field solve and the node field (Sec. 2.1)."""
        self.deposit_all()
        if self.external_E:
            return
        F = self.node_load()
        self.qT = self.fs.q_tets(self.cut_charge())
        self.phi, it, rr = self.fs.solve(F, self.qT, phi0=self.phi, tol=self.tol, maxit=self.maxit)
        self.E = self.fs.node_E(self.phi, self.qT)
        self.last.update(pcg_iters=it, pcg_relres=rr)

    def leapfrog_init(self):
        E = self.E_pic()
        for s, sp in enumerate(self.species):
            pt.half_kick_back(self.mesh, E, self.P[s], sp.k)

    # -- one PIC step --------------------------------------------------------------
    def _collect(self, s, keep_mask, xo, yo, zo, P):
        """Remove outside / collect object hits; returns kept mask and counts."""
        m, obj = self.mesh, self.obj
        out = pt.outside(m, P["x"], P["y"], P["z"])
        Ln = obj.L(P["x"], P["y"], P["z"])
        hit = keep_mask & ~out & (Ln < 0.0)
        lost = 0
        if hit.any():
            cells = pt.hit_cells(self.fmesh, obj, xo[hit], yo[hit], zo[hit], P["x"][hit], P["y"][hit],
                                 P["z"][hit], self.r)
            acc = self.fs.cell_to_acc[cells]
            np.add.at(self.surf[:, s], acc[acc >= 0], 1)
            lost = int((acc < 0).sum())
        keep = keep_mask & ~out & ~hit
        return keep, int((keep_mask & out).sum()), int(hit.sum()), lost

    def step(self):
        st = dict(pushed=[], absorbed=[], collected=[], injected=[], lost=[], inj_rejected=[])
        m = self.mesh
        E = self.E_pic()
        for s, sp in enumerate(self.species):
            P = self.P[s]
            st["pushed"].append(len(P["x"]))
            xo, yo, zo = P["x"].copy(), P["y"].copy(), P["z"].copy()
            pt.push(m, E, P, sp.k, self.dth)
            pt.reflect(m, P, sp.reflect)
            keep, nab, nco, lost = self._collect(s, np.ones(len(xo), dtype=bool), xo, yo, zo, P)
            P = {k: v[keep] for k, v in P.items()}
            ninj = nrej = 0
            if sp.inj is not None:
                mask, dens, vth, drift, seed = sp.inj
                offset = 0
                new = []
                for f in range(6):
                    if not (mask >> f) & 1:
                        continue
                    sp.carry[f] = sp.carry[f] + self.injection_rate(s, f)
                    cnt = int(math.floor(sp.carry[f]))
                    sp.carry[f] = sp.carry[f] - cnt
                    I = pt.inject_face(m, self.obj, seed, s, f, self.step_no, cnt, vth, drift, self.dth)
                    pt.reflect(m, I, sp.reflect)
                    valid = I["accepted"] & (self.obj.L(I["x0"], I["y0"], I["z0"]) >= 0.0)
                    nrej += int((~valid).sum())
                    k2, a2, c2, l2 = self._collect(s, valid, I["x0"], I["y0"], I["z0"], I)
                    nab += a2; nco += c2; lost += l2
                    I["id"] = sp.next_id + offset + I["index"]
                    new.append({k: I[k][k2] for k in FIELDS})
                    ninj += int(valid.sum())
                    offset += cnt
                sp.next_id += offset
                for N in new:
                    P = {k: np.concatenate([P[k], N[k]]) for k in FIELDS}
            if sp.photo is not None:
                I = sp.photo.emit(self.step_no)
                if self.r > 1:   # emitted in IFE cell units: to PIC units (exact)
                    for k in ("x", "y", "z"):
                        I[k] = I[k] / float(self.r)
                    I["p0"] = I["p0"] / float(self.r)
                pt.reflect(m, I, sp.reflect)
                inside = self.obj.L(I["x"], I["y"], I["z"]) < 0.0
                emitted = I["ok"] & ~inside
                out = pt.outside(m, I["x"], I["y"], I["z"])
                np.add.at(self.surf[:, s], I["acc"][emitted], -1)
                keep = emitted & ~out
                nab += int((emitted & out).sum())
                nrej += int((~emitted).sum())
                ninj += int(emitted.sum())
                I["id"] = sp.next_id + I["index"]
                sp.next_id += I["count"]
                P = {k: np.concatenate([P[k], I[k][keep]]) for k in FIELDS}
            self.P[s] = P
            st["absorbed"].append(nab); st["collected"].append(nco)
            st["injected"].append(ninj); st["lost"].append(lost); st["inj_rejected"].append(nrej)
        self.solve()
        self.step_no += 1
        self.last.update(st)
        return st

    # -- diagnostics -----------------------------------------------------------------
    def counts(self):
        return [len(P["x"]) for P in self.P]

    def surface_potential(self):
        return self.fs.surface_potential(self.phi, self.qT)
