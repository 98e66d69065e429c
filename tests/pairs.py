"""Paired CUDA-library / oracle instances on identical seeded inputs (test helper)."""
import numpy as np

from oracle.geometry import CapCrater, Mesh, NoObject, Plane, RimCrater, Sphere, set_bedrock
from oracle.field import FieldSystem
from oracle.pic import Simulation as OracleSim
from paper_2011_10214_gb300 import workloads as wl

# geometry cases: ragged sizes (not multiples of the 4-cell bin), mixed boundaries
CASES = {
    "sphere16": dict(n=(16, 16, 16), h=0.5, obj=("sphere", (4.0, 4.0, 4.0), 2.0, 4.0, 1.0),
                     bc=[("D", 0.0)] * 6),
    "ragged": dict(n=(18, 13, 11), h=0.3, obj=("sphere", (2.71, 1.93, 1.64), 0.83, 6.0, 1.0),
                   bc=[("D", 0.0), ("D", 0.25), ("N",), ("D", -0.1), ("N",), ("N",)]),
    "crater": dict(n=(24, 22, 16), h=1.0, obj=("cap_crater", 6.0, 12.0, 11.0, 6.0, 3.0, 4.0, 1.0),
                   bc=[("N",)] * 5 + [("D", 0.0)]),
    "plane": dict(n=(12, 12, 12), h=0.5, obj=("plane", (0.3, -0.5, 1.0), 4.37, 10.0, 1.0),
                  bc=[("D", 0.0)] * 6),
    # off-node ground with a bowl, for photoemission under a low sun (shadows)
    "crater_sun": dict(n=(24, 24, 12), h=1.0, obj=("cap_crater", 6.3, 12.0, 12.0, 8.0, 3.0, 4.0, 1.0),
                       bc=[("N",)] * 5 + [("D", 0.0)]),
    # layered lunar ground: raised-rim crater in regolith (eps 4) over bedrock
    # (eps 10) below z = 2.45, the crater centred on the y = 0 face (a half crater)
    "lunar": dict(n=(30, 16, 16), h=1.0,
                  obj=("rim_crater", 7.37, 15.0, 0.0, 4.1, 7.9, 11.6, 2.6, 2.2, 4.0, 1.0),
                  bed=(2.45, 10.0), bc=[("N",)] * 5 + [("D", 0.0)]),
    # hybrid grids: the IFE mesh twice (four times) as fine as the PIC mesh
    "sphere_h2": dict(n=(12, 10, 9), h=0.5, obj=("sphere", (2.71, 2.43, 2.12), 1.13, 6.0, 1.0),
                      bc=[("D", 0.0), ("D", 0.25), ("N",), ("D", -0.1), ("N",), ("N",)], refine=2),
    "crater_h4": dict(n=(8, 8, 6), h=1.0, obj=("cap_crater", 3.3, 4.0, 4.0, 3.0, 1.5, 4.0, 1.0),
                      bed=(1.3, 10.0), bc=[("N",)] * 5 + [("D", 0.0)], refine=4),
    # the same with a floor below the top of the bedrock's cells: tets cut twice
    "lunar_deep": dict(n=(30, 16, 16), h=1.0,
                       obj=("rim_crater", 7.37, 15.0, 0.0, 4.1, 7.9, 11.6, 2.6, 4.6, 4.0, 1.0),
                       bed=(2.45, 10.0), bc=[("N",)] * 5 + [("D", 0.0)]),
}


# edge cases, outside the parametrised sweeps over CASES: a box with no object
# (no interface tets, no cut cells) and a mesh smaller than one particle bin
EDGE_CASES = {
    "empty_box": dict(n=(10, 9, 7), h=0.5, obj=("none",),
                      bc=[("D", 0.0), ("D", 0.3), ("N",), ("N",), ("D", -0.2), ("N",)]),
    "tiny": dict(n=(4, 3, 2), h=0.5, obj=("none",), bc=[("D", 0.1), ("D", -0.1), ("N",), ("D", 0.0), ("N",), ("N",)]),
}


def oracle_object(m, o, bed=None):
    if o[0] == "sphere":
        obj = Sphere(m, o[1], o[2], o[3], o[4])
    elif o[0] == "cap_crater":
        obj = CapCrater(m, *o[1:])
    elif o[0] == "rim_crater":
        obj = RimCrater(m, *o[1:])
    elif o[0] == "plane":
        obj = Plane(o[1], o[2], o[3], o[4])
    else:
        obj = NoObject()
    if bed is not None:
        set_bedrock(obj, m, *bed)
    return obj


def gpu_object(sim, o, bed=None):
    from paper_2011_10214_gb300 import capi
    if bed is not None:
        sim.set_bedrock(*bed)
    if o[0] == "sphere":
        sim.set_object(capi.OBJ_SPHERE, list(o[1]) + [o[2]], o[3], o[4])
    elif o[0] == "cap_crater":
        sim.set_object(capi.OBJ_CAP_CRATER, list(o[1:6]), o[6], o[7])
    elif o[0] == "rim_crater":
        sim.set_object(capi.OBJ_RIM_CRATER, list(o[1:9]), o[9], o[10])
    elif o[0] == "plane":
        sim.set_object(capi.OBJ_PLANE, list(o[1]) + [o[2]], o[3], o[4])
    else:
        sim.set_object(capi.OBJ_NONE, [], 1.0, 1.0)


def make_pair(case, dt=0.05, tol=1e-12, maxit=2000, track=True, precision=0, refine=None):
    from paper_2011_10214_gb300 import capi
    c = CASES[case] if case in CASES else EDGE_CASES[case]
    r = c.get("refine", 1) if refine is None else refine
    m = Mesh(*c["n"], c["h"])
    obj = oracle_object(m, c["obj"], c.get("bed"))
    orc = OracleSim(m, obj, c["bc"], dt, tol=tol, maxit=maxit, refine=r)
    gpu = capi.Simulation(c["n"], c["h"], dt, precision=precision, pcg_tol=tol, pcg_max_iter=maxit,
                          track_ids=track, ife_refine=r)
    gpu.set_field_bc(c["bc"])
    gpu_object(gpu, c["obj"], c.get("bed"))
    return gpu, orc


def add_species_both(gpu, orc, q, m, w):
    a = gpu.add_species(q, m, w)
    b = orc.add_species(q, m, w)
    assert a == b
    return a


def by_id(P):
    o = np.argsort(P["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in P.items()}


def explicit_particles(gpu, orc, s, n, seed, vth, margin=0.0):
    x, y, z, vx, vy, vz = wl.random_particles(gpu.n, n, seed, vth=vth, margin=margin)
    keep = orc.obj.L(x, y, z) >= 0
    arr = [a[keep] for a in (x, y, z, vx, vy, vz)]
    ids = np.arange(len(arr[0]), dtype=np.int64) * 3 + 5
    gpu.load_particles(s, *arr, ids)
    orc.load_particles(s, *arr, ids)
    return len(ids)
