"""GPU reflecting particle faces (pifepic_set_particle_bc; the symmetry planes
of Sec. 3 and Sec. 5.2.2) vs the oracle (oracle/particles.py reflect).

Bars: FP64 bit-exact (particle set, states, fixed-point node charges, surface
counts, event counts) with a frozen field; MIXED within the FP32 bar of
test_gpu_mixed; a closed reflecting box conserves every particle exactly in
both precisions, also at the full 50^3 eighth-sphere size."""
import math

import numpy as np
import pytest

from paper_2011_10214_gb300 import capi
from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import add_species_both, by_id, explicit_particles, make_pair

pytestmark = pytest.mark.gpu

MIXED = 1
TOL32 = 1e-4


def _compare_exact(gpu, orc, s):
    g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
    assert np.array_equal(g["id"], o["id"]), f"particle sets differ: {len(g['id'])} vs {len(o['id'])}"
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], o[k]), k
    assert np.array_equal(gpu.node_charge(s), orc.W[s])
    assert np.array_equal(gpu.surface_counts(s), orc.surf[:, s])


@pytest.mark.parametrize("case,kinds", [
    ("sphere16", ["reflect", "absorb"] * 3),
    ("ragged", ["reflect", "reflect", "absorb", "reflect", "absorb", "reflect"]),
    ("crater", ["reflect"] * 4 + ["absorb", "absorb"]),
])
def test_reflect_frozen_field_bit_exact(case, kinds):
    gpu, orc = make_pair(case, dt=0.2)
    E = wl.random_node_field(orc.mesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        gpu.set_particle_bc(s, kinds)
        orc.set_particle_bc(s, kinds)
        explicit_particles(gpu, orc, s, 20000, 300 + s, 3.0 / (1 + 4 * s))
    gpu.set_external_E(E)
    orc.set_external_E(E)
    for step in range(10):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            for key in ("pushed", "absorbed", "collected", "injected"):
                assert sg[key][s] == so[key][s], (step, s, key)
    for s in range(2):
        _compare_exact(gpu, orc, s)
        # nothing is ever found beyond a reflecting face
        P = gpu.particles(s)
        n = gpu.n
        for ax, key in enumerate(("x", "y", "z")):
            assert P[key].min() >= 0.0 and P[key].max() < n[ax]
    gpu.close()


@pytest.mark.parametrize("case,kinds,inject", [
    ("ragged", ["reflect", "reflect", "absorb", "reflect", "inject", "reflect"], 0b010000),
    ("crater", ["reflect"] * 4 + ["absorb", "inject"], 0b100000),
])
def test_reflect_with_injection(case, kinds, inject):
    """Injection next to reflecting faces: exact counts and ids; injected states
    to 1e-12 (the Box-Muller normals of CUDA and libm differ in the last ulp, so
    the injected particles are not bit-identical)."""
    gpu, orc = make_pair(case, dt=0.2)
    E = wl.random_node_field(orc.mesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        gpu.set_particle_bc(s, kinds)
        orc.set_particle_bc(s, kinds)
        explicit_particles(gpu, orc, s, 5000, 310 + s, 3.0 / (1 + 4 * s))
        gpu.set_injection(s, inject, 1.0, 2.0 / (1 + 4 * s), (0.3, -0.2, 0.1), 41)
        orc.set_injection(s, inject, 1.0, 2.0 / (1 + 4 * s), (0.3, -0.2, 0.1), 41)
    gpu.set_external_E(E)
    orc.set_external_E(E)
    for step in range(8):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            for key in ("pushed", "absorbed", "collected", "injected"):
                assert sg[key][s] == so[key][s], (step, s, key)
    for s in range(2):
        g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
        assert np.array_equal(g["id"], o["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.allclose(g[k], o[k], rtol=1e-12, atol=1e-12), k
        for ax, key in enumerate(("x", "y", "z")):
            assert g[key].min() >= 0.0 and g[key].max() < gpu.n[ax]
    gpu.close()


def test_reflect_exact_face_landings():
    """Moves that end exactly on a face: on the plus face the mirror is n again
    and the particle takes the largest double below n; on the minus face +0.0
    is inside and nothing happens.  Zero field, dt/h = 1/2."""
    gpu, orc = make_pair("sphere16", dt=0.25)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    for sim in (gpu, orc):
        sim.set_particle_bc(0, ["reflect"] * 6)
    n = 16.0
    x = np.array([n - 0.25, 0.25, 0.125, n - 0.125, 12.0, 13.0])
    y = np.array([14.0, 14.0, 14.0, 14.0, n - 0.25, 0.25])
    z = np.array([13.0, 13.0, 13.0, 13.0, 13.0, 13.0])
    vx = np.array([0.5, -0.5, -0.5, 0.75, 0.0, 0.0])
    vy = np.array([0.0, 0.0, 0.0, 0.0, 0.5, -0.5])
    vz = np.zeros(6)
    ids = np.arange(6, dtype=np.int64)
    gpu.load_particles(0, x, y, z, vx, vy, vz, ids)
    orc.load_particles(0, x, y, z, vx, vy, vz, ids)
    E = np.zeros((orc.mesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    gpu.step(1); orc.step()
    _compare_exact(gpu, orc, 0)
    g = by_id(gpu.particles(0))
    below = np.nextafter(n, 0.0)
    assert g["x"][0] == below and g["vx"][0] == -0.5          # landed on n: largest double below
    assert g["x"][1] == 0.0 and g["vx"][1] == -0.5            # landed on +0.0: inside, not mirrored
    assert g["x"][2] == 0.125 and g["vx"][2] == 0.5           # mirrored at the minus face
    assert g["x"][3] == n - 0.25 and g["vx"][3] == -0.75      # mirrored at the plus face
    assert g["y"][4] == below and g["y"][5] == 0.0
    gpu.close()


def test_reflect_mixed_frozen_field():
    kinds = ["reflect", "reflect", "absorb", "reflect", "inject", "reflect"]
    gpu, orc = make_pair("ragged", dt=0.2, precision=MIXED)
    E = wl.random_node_field(orc.mesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        gpu.set_particle_bc(s, kinds)
        orc.set_particle_bc(s, kinds)
        explicit_particles(gpu, orc, s, 20000, 300 + s, 3.0 / (1 + 4 * s))
        gpu.set_injection(s, 0b010000, 1.0, 2.0 / (1 + 4 * s), (0.3, -0.2, 0.1), 41)
        orc.set_injection(s, 0b010000, 1.0, 2.0 / (1 + 4 * s), (0.3, -0.2, 0.1), 41)
    gpu.set_external_E(E); orc.set_external_E(E)
    for _ in range(10):
        gpu.step(1)
        orc.step()
    for s in range(2):
        g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
        common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
        n = len(o["id"])
        mismatch = (len(g["id"]) - len(common)) + (n - len(common))
        assert mismatch <= max(2, 1e-3 * n), f"absorb/collect mismatch {mismatch} of {n}"
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            d = np.abs(g[k][gi] - o[k][oi]) / np.maximum(np.abs(o[k][oi]), 1.0)
            assert d.max() <= TOL32, (k, d.max())
        W = gpu.node_charge(s)
        assert W.sum() == 2 ** 32 * len(g["id"])
        assert np.abs(W - orc.W[s]).max() <= TOL32 * 2 ** 32 * 8
        P = gpu.particles(s)
        for ax, key in enumerate(("x", "y", "z")):
            assert P[key].min() >= 0.0 and P[key].max() < gpu.n[ax]
    gpu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_reflect_photoemission(precision):
    """Photoelectrons emitted towards a reflecting face are mirrored before the
    inside-object and boundary tests (low sun from X_min)."""
    gpu, orc = make_pair("crater_sun", dt=0.2, precision=precision)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    kinds = ["reflect", "absorb", "reflect", "reflect", "absorb", "absorb"]
    sun = (-math.cos(math.radians(20.0)), 0.0, math.sin(math.radians(20.0)))
    for sim in (gpu, orc):
        sim.set_particle_bc(0, kinds)
        sim.set_photoemission(0, sun, 6.0, 2.0, 13)
    E = np.zeros((orc.mesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    for step in range(8):
        sg, so = gpu.step(1), orc.step()
        for key in ("injected", "inj_rejected", "absorbed", "collected"):
            assert sg[key][0] == so[key][0], (step, key)
    assert np.array_equal(gpu.surface_counts(0), orc.surf[:, 0])
    g, o = by_id(gpu.particles(0)), by_id(orc.P[0])
    assert np.array_equal(g["id"], o["id"])
    tol = 1e-12 if precision == 0 else 2e-6
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.allclose(g[k], o[k], rtol=tol, atol=tol), k
    gpu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_closed_reflecting_box_conserves_particles_full_size(precision):
    """The 50^3 eighth-sphere box with every face reflecting and no object: no
    particle is ever absorbed, every deposit is exact, states stay in the box.
    A property that holds at any size, checked at the full workload's size."""
    cfg = dict(wl.OML50)
    cfg["object"] = dict(kind="none")
    cfg["particle_bc"] = ["reflect"] * 6
    sim = capi.from_config(cfg, precision=precision, inject=False, pcg_tol=1e-6, pcg_max_iter=400)
    n0 = sim.count(0) + sim.count(1)
    assert n0 == 2 * 125 * 50 ** 3
    sim.solve()
    sim.leapfrog_init()
    for _ in range(5):
        st = sim.step(1)
        assert sum(st["absorbed"]) == 0 and sum(st["collected"]) == 0
        assert sum(st["pushed"]) == n0
    assert sim.count(0) + sim.count(1) == n0
    for s in range(2):
        assert sim.node_charge(s).sum() == 2 ** 32 * sim.count(s)
    sim.close()


def test_particle_bc_errors():
    gpu, orc = make_pair("sphere16")
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    # a REFLECT face cannot inject, whichever call comes first; bad kinds and species fail
    gpu.set_particle_bc(0, ["reflect"] + ["absorb"] * 5)
    with pytest.raises(RuntimeError):
        gpu.set_injection(0, 0b000011, 1.0, 1.0, (0.0, 0.0, 0.0), 1)
    gpu.set_injection(0, 0b000010, 1.0, 1.0, (0.0, 0.0, 0.0), 1)
    with pytest.raises(RuntimeError):
        gpu.set_particle_bc(0, ["absorb", "reflect"] + ["absorb"] * 4)
    with pytest.raises(RuntimeError):
        gpu.set_particle_bc(0, [0, 1, 2, 3, 0, 0])
    with pytest.raises(RuntimeError):
        gpu.set_particle_bc(7, ["absorb"] * 6)
    gpu.close()


def test_eighth_sphere_pic_steps_match_oracle():
    """The eighth-sphere validation set-up, scaled to 12^3 cells: solved field,
    Neumann symmetry planes with reflecting particle faces at X/Y/Z_min,
    injection at X/Y/Z_max; counts and potential follow the oracle."""
    from oracle.geometry import Mesh, Sphere
    from oracle.pic import Simulation as OracleSim
    cfg = wl.oml_eighth_config(n=12, ppc=8, steps=5)
    gpu = capi.from_config(cfg, track_ids=True, pcg_tol=1e-12, pcg_max_iter=5000)
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    orc = OracleSim(m, Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"]), cfg["face_bc"],
                    cfg["dt"], tol=1e-12, maxit=5000)
    for s, sp in enumerate(cfg["species"]):
        orc.add_species(sp["q"], sp["m"], wl.macro_weight(cfg, sp))
        orc.set_particle_bc(s, cfg["particle_bc"])
        orc.load_maxwellian(s, sp["ppc"], sp["vth"], sp["drift"], cfg["seed"])
        orc.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
    gpu.solve(); orc.solve()
    assert np.abs(gpu.potential() - orc.phi).max() <= 1e-8 * np.abs(orc.phi).max()
    gpu.leapfrog_init(); orc.leapfrog_init()
    for step in range(5):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            assert sg["injected"][s] == so["injected"][s]
            assert abs(sg["collected"][s] - so["collected"][s]) <= 1
            assert abs(sg["absorbed"][s] - so["absorbed"][s]) <= 1
        rel = np.abs(gpu.potential() - orc.phi).max() / np.abs(orc.phi).max()
        assert rel <= 1e-8, (step, rel)
    for s in range(2):
        g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
        common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
        assert len(common) >= len(o["id"]) - 2
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            d = np.abs(g[k][gi] - o[k][oi]) / np.maximum(np.abs(o[k][oi]), 1.0)
            assert d.max() <= 1e-6, k
    gpu.close()
