"""Particle load, injection, gather/push, boundaries, object hits, deposit.

Oracle; test infrastructure only.  Follows arXiv:2011.10214:
  * Sec. 2.1 (PIC loop): charge weighted to nodes ("scatter"), field
    interpolated at particle positions ("gather"), velocity and position
    update ("particle-push");
  * Sec. 3.1.3: particles pre-loaded before the initial field solve, injected
    at open faces every step, absorbed (removed) at open faces;
  * Sec. 5.2.2: particles injected at an angle (drifting plasma); particles
    hitting the object surface are collected and their charge accumulated.

Readings where the paper is silent:
  * positions in cell units xi = (x - origin)/h; velocities physical;
  * gather: trilinear weights of the PIC cell, node order 000,100,...,111,
    w = (wx*wy)*wz, E_p accumulated left to right; leapfrog
    v += k E_p with k = (q/m) dt, then xi += v (dt/h); no FMA anywhere;
  * the leapfrog starts with a half kick back, v <- v - (k/2) E(x0);
  * an absorbing face removes any particle with xi outside [0, n);
    the face test precedes the object test; a particle whose new position has
    L < 0 is collected by the object, at the PIC cell that holds the
    crossing point x_old + t (x_new - x_old), t = L_old / (L_old - L_new);
  * deposit: W_l = rint(w_l 2^32) for l < 7, W_7 = 2^32 - sum; int64 sums per
    node and species, so every particle deposits exactly 2^32 units;
  * injection: per species and open face, count = floor(rate + carry) with
    rate = Gamma A dt / w (Gamma the drifting-Maxwellian one-way flux);
    uniform position on the face, flux-weighted normal speed (rejection
    sampler, proposal N(mu, 1), mu the mode), Gaussian tangential speeds plus
    drift, then a random fraction U of one step of motion; a start point
    inside the object is rejected;
  * load: ppc particles per cell, uniform in the cell, Maxwellian plus drift;
    particles inside the object are rejected without replacement.
"""
import math

import numpy as np

from . import rng

TWO32 = 4294967296.0
MAX_TRIES = 32            # rejection tries for the flux-weighted normal speed


# ---------------------------------------------------------------------------
# trilinear weights and gather/push (Sec. 2.1 gather + particle-push)
# ---------------------------------------------------------------------------

def cell_and_weights(x, y, z):
    """Cell (i,j,k) = floor(xi) and the 8 trilinear weights, fixed op order."""
    cx = np.floor(x); cy = np.floor(y); cz = np.floor(z)
    fx = x - cx; fy = y - cy; fz = z - cz
    wx = (1.0 - fx, fx); wy = (1.0 - fy, fy); wz = (1.0 - fz, fz)
    w = []
    for l in range(8):
        a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
        w.append((wx[a] * wy[b]) * wz[c])
    return cx.astype(np.int64), cy.astype(np.int64), cz.astype(np.int64), w


def node_ids(mesh, i, j, k):
    out = []
    for l in range(8):
        a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
        out.append(mesh.node(i + a, j + b, k + c))
    return out


def gather(mesh, E, x, y, z):
    """E at particle positions: sum_l w_l E_l accumulated in node order."""
    i, j, k, w = cell_and_weights(x, y, z)
    nid = node_ids(mesh, i, j, k)
    out = []
    for comp in range(3):
        acc = w[0] * E[nid[0], comp]
        for l in range(1, 8):
            acc = acc + w[l] * E[nid[l], comp]
        out.append(acc)
    return out


def push(mesh, E, P, k, dth):
    """Leapfrog kick and drift of the particle dict P in place."""
    ex, ey, ez = gather(mesh, E, P["x"], P["y"], P["z"])
    P["vx"] = P["vx"] + k * ex
    P["vy"] = P["vy"] + k * ey
    P["vz"] = P["vz"] + k * ez
    P["x"] = P["x"] + P["vx"] * dth
    P["y"] = P["y"] + P["vy"] * dth
    P["z"] = P["z"] + P["vz"] * dth


def half_kick_back(mesh, E, P, k):
    """v^{-1/2} = v^0 - (k/2) E(x^0) (leapfrog start)."""
    ex, ey, ez = gather(mesh, E, P["x"], P["y"], P["z"])
    hk = 0.5 * k
    P["vx"] = P["vx"] - hk * ex
    P["vy"] = P["vy"] - hk * ey
    P["vz"] = P["vz"] - hk * ez


# ---------------------------------------------------------------------------
# boundaries and object collection
# ---------------------------------------------------------------------------

def outside(mesh, x, y, z):
    return (x < 0.0) | (x >= mesh.nx) | (y < 0.0) | (y >= mesh.ny) | (z < 0.0) | (z >= mesh.nz)


def reflect(mesh, P, mask):
    """Reflecting particle faces (bit f of mask for face f = x-, x+, y-, y+, z-,
    z+; the paper reflects particles at its symmetry plane, Sec. 5.2.2): a
    particle beyond a reflecting face is mirrored back, xi -> -xi at the minus
    face and xi -> 2 n - xi at the plus face, and its normal velocity reversed.
    A mirrored coordinate landing exactly on the plus face (the box is [0, n))
    takes the largest double below n.  Applied in place after a move and before
    the boundary and object tests."""
    if not mask:
        return
    n_axes = (mesh.nx, mesh.ny, mesh.nz)
    for ax, (kx, kv) in enumerate((("x", "vx"), ("y", "vy"), ("z", "vz"))):
        n = float(n_axes[ax])
        if (mask >> (2 * ax)) & 1:
            lo = P[kx] < 0.0
            P[kx] = np.where(lo, -P[kx], P[kx])
            P[kv] = np.where(lo, -P[kv], P[kv])
        if (mask >> (2 * ax + 1)) & 1:
            hi = P[kx] >= n
            x2 = np.where(hi, (2.0 * n) - P[kx], P[kx])
            P[kx] = np.where(hi & (x2 >= n), np.nextafter(n, 0.0), x2)
            P[kv] = np.where(hi, -P[kv], P[kv])


def hit_cells(mesh, obj, xo, yo, zo, xn, yn, zn, r=1):
    """Cell index of the crossing point for particles that entered the object.

    Positions are in the particle mesh's cell units; mesh is the field (IFE)
    mesh, r times finer (r a power of two, 1 when the meshes coincide): the
    crossing point's IFE cell is floor(r xi_c)."""
    Lo = obj.L(xo, yo, zo)
    Ln = obj.L(xn, yn, zn)
    t = Lo / (Lo - Ln)
    xc = xo + t * (xn - xo)
    yc = yo + t * (yn - yo)
    zc = zo + t * (zn - zo)
    i = np.clip(np.floor(r * xc), 0, mesh.nx - 1).astype(np.int64)
    j = np.clip(np.floor(r * yc), 0, mesh.ny - 1).astype(np.int64)
    kk = np.clip(np.floor(r * zc), 0, mesh.nz - 1).astype(np.int64)
    return mesh.cell(i, j, kk)


# ---------------------------------------------------------------------------
# fixed-point deposit (Sec. 2.1 scatter)
# ---------------------------------------------------------------------------

def deposit(mesh, x, y, z):
    """int64 node sums of the fixed-point weights (2^32 units per particle)."""
    W = np.zeros(mesh.nnodes, dtype=np.int64)
    if len(x) == 0:
        return W
    i, j, k, w = cell_and_weights(x, y, z)
    nid = node_ids(mesh, i, j, k)
    rest = np.full(len(x), 1 << 32, dtype=np.int64)
    for l in range(7):
        Wl = np.rint(w[l] * TWO32).astype(np.int64)
        rest -= Wl
        np.add.at(W, nid[l], Wl)
    np.add.at(W, nid[7], rest)
    return W


# ---------------------------------------------------------------------------
# sampling (readings; see module docstring)
# ---------------------------------------------------------------------------

def flux_density(n, vth, vdn):
    """One-way flux of a drifting Maxwellian through a face, per unit area.

    n vth [exp(-s^2/2)/sqrt(2 pi) + (s/2)(1 + erf(s/sqrt 2))], s = vdn/vth,
    vdn the drift component along the inward normal.
    """
    s = vdn / vth
    return n * vth * (math.exp(-0.5 * s * s) / math.sqrt(2.0 * math.pi)
                      + 0.5 * s * (1.0 + math.erf(s / math.sqrt(2.0))))


def flux_normal_speed(U, s):
    """Sample v > 0 with density ~ v exp(-(v - s)^2 / 2) (units of vth).

    U: list of (u0, u1, u2) uniform triples per try.  Proposal N(mu, 1) with
    mu = (s + sqrt(s^2 + 4))/2 the mode of the target; accept with
    probability (v/mu) exp(1 - v/mu) (the ratio target/proposal, maximal 1 at
    v = mu).  Returns (v, accepted).
    """
    mu = 0.5 * (s + math.sqrt(s * s + 4.0))
    m = len(U[0][0])
    v_out = np.zeros(m)
    done = np.zeros(m, dtype=bool)
    for u0, u1, u2 in U:
        z, _ = rng.box_muller(u0, u1)
        v = mu + z
        ratio = v / mu
        acc = (~done) & (v > 0.0) & (u2 < ratio * np.exp(1.0 - ratio))
        v_out[acc] = v[acc]
        done |= acc
    return v_out, done


FACE_AXIS = (0, 0, 1, 1, 2, 2)
FACE_SIGN = (1.0, -1.0, 1.0, -1.0, 1.0, -1.0)        # inward normal sign


def face_tangents(f):
    ax = FACE_AXIS[f]
    return [a for a in range(3) if a != ax]


def inject_face(mesh, obj, seed, species, face, step, count, vth, drift, dth):
    """Particles injected through one face in one step (before any removal).

    Returns a dict with positions after the partial step, velocities, the
    start point, the index within the face batch and flags.
    """
    n_axes = (mesh.nx, mesh.ny, mesh.nz)
    ax = FACE_AXIS[face]
    t1, t2 = face_tangents(face)
    sgn = FACE_SIGN[face]
    m = np.arange(count, dtype=np.uint64)
    key1 = rng.stream_key(rng.PURPOSE_INJECT, species, face, step)
    b0 = rng.philox4x64(m, 0, 0, 0, seed, key1)
    b1 = rng.philox4x64(m, 1, 0, 0, seed, key1)
    tries = []
    for t in range(MAX_TRIES):
        bt = rng.philox4x64(m, 2 + t, 0, 0, seed, key1)
        tries.append((rng.uniform(bt[0]), rng.uniform(bt[1]), rng.uniform(bt[2])))
    s = sgn * drift[ax] / vth
    vn, ok = flux_normal_speed(tries, s)
    g1, g2 = rng.box_muller(rng.uniform(b1[0]), rng.uniform(b1[1]))
    pos0 = [None, None, None]
    pos0[ax] = np.full(count, 0.0 if sgn > 0 else float(n_axes[ax]))
    pos0[t1] = rng.uniform(b0[0]) * float(n_axes[t1])
    pos0[t2] = rng.uniform(b0[1]) * float(n_axes[t2])
    frac = rng.uniform(b0[2])
    vel = [None, None, None]
    vel[ax] = sgn * (vth * vn)
    vel[t1] = drift[t1] + vth * g1
    vel[t2] = drift[t2] + vth * g2
    step_len = frac * dth
    pos = [pos0[a] + vel[a] * step_len for a in range(3)]
    return dict(x0=pos0[0], y0=pos0[1], z0=pos0[2], x=pos[0], y=pos[1], z=pos[2],
                vx=vel[0], vy=vel[1], vz=vel[2], accepted=ok, index=np.arange(count, dtype=np.int64))


def load_maxwellian(mesh, obj, seed, species, ppc, vth, drift):
    """ppc particles per cell, uniform in the cell, Maxwellian velocities.

    Counter (cell, particle-in-cell, block); block 0 gives the position,
    block 1 the three normals.  Particles with L < 0 are dropped.  Returns
    the particle dict with ids cell*ppc + p.
    """
    ci, cj, ck = mesh.cell_ijk()
    cells = np.repeat(np.arange(mesh.ncells, dtype=np.uint64), ppc)
    pic = np.tile(np.arange(ppc, dtype=np.uint64), mesh.ncells)
    key1 = rng.stream_key(rng.PURPOSE_LOAD, species, 0, 0)
    b0 = rng.philox4x64(cells, pic, 0, 0, seed, key1)
    b1 = rng.philox4x64(cells, pic, 1, 0, seed, key1)
    ii = np.repeat(ci, ppc).astype(np.float64)
    jj = np.repeat(cj, ppc).astype(np.float64)
    kk = np.repeat(ck, ppc).astype(np.float64)
    x = ii + rng.uniform(b0[0])
    y = jj + rng.uniform(b0[1])
    z = kk + rng.uniform(b0[2])
    g0, g1 = rng.box_muller(rng.uniform(b1[0]), rng.uniform(b1[1]))
    g2, _ = rng.box_muller(rng.uniform(b1[2]), rng.uniform(b1[3]))
    P = dict(x=x, y=y, z=z, vx=drift[0] + vth * g0, vy=drift[1] + vth * g1, vz=drift[2] + vth * g2,
             id=(cells * np.uint64(ppc) + pic).astype(np.int64))
    keep = obj.L(x, y, z) >= 0.0
    return {k: v[keep] for k, v in P.items()}
