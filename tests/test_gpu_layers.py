"""GPU layered lunar ground (pifepic_set_bedrock, PIFEPIC_OBJ_RIM_CRATER; Sec.
5.2.1: a raised-rim crater in regolith over bedrock) vs the oracle.  The set-up
and FP64 solve parity of the "lunar" cases run in test_gpu_setup.py and
test_gpu_field.py (every case of tests/pairs.py); this file adds the column
against the series capacitor, MIXED solves, the particle cycle on the
rim-crater surface, photoemission, and the error cases."""
import math

import numpy as np
import pytest

from paper_2011_10214_gb300 import capi
from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import add_species_both, by_id, explicit_particles, make_pair

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_three_layer_column_matches_oracle():
    """Plane ground over a bedrock plane, phi fixed at the bottom and the top:
    the GPU solve equals the oracle's to 1e-10."""
    from oracle.field import FieldSystem
    from oracle.geometry import Mesh, Plane, set_bedrock
    nz, h = 24, 0.5
    m = Mesh(4, 4, nz, h)
    obj = set_bedrock(Plane((0.0, 0.0, 1.0), 7.3 / h, 4.0, 1.0), m, 3.6, 10.0)
    bc = [("N",)] * 4 + [("D", 0.0), ("D", 1.0)]
    fs = FieldSystem(m, obj, bc)
    sim = capi.Simulation((4, 4, nz), h, 0.05, pcg_tol=1e-13, pcg_max_iter=5000)
    sim.set_field_bc(bc)
    sim.set_bedrock(3.6, 10.0)
    sim.set_object(capi.OBJ_PLANE, [0.0, 0.0, 1.0, 7.3 / h], 4.0, 1.0)
    q = np.zeros(len(fs.it_cell))
    phi_o, _, _ = fs.solve(np.zeros(m.nnodes), q, tol=1e-13, maxit=5000)
    sim.solve_field(np.zeros(m.nnodes), q)
    assert _rel(sim.potential(), phi_o) <= 1e-10
    assert _rel(sim.node_E(), fs.node_E(phi_o, q)) <= 1e-9
    sim.close()


@pytest.mark.parametrize("case", ["lunar", "lunar_deep"])
def test_mixed_solve_reaches_fp64_accuracy(case):
    gpu, orc = make_pair(case, precision=1)
    fs = orc.fs
    g = np.random.default_rng(5)
    F = g.normal(size=orc.mesh.nnodes)
    q = np.where(fs.it_kind == 0, g.normal(size=len(fs.it_cell)), 0.0)
    phi_o, _, _ = fs.solve(F, q, tol=1e-12, maxit=5000)
    gpu.solve_field(F, q)
    assert _rel(gpu.potential(), phi_o) <= 1e-8
    assert _rel(gpu.node_E(), fs.node_E(phi_o, q)) <= 1e-8
    gpu.close()


def _half_crater_pair(precision=0, dt=0.2):
    """The lunar case with the crater centred on the y = 0 face: that face
    reflects particles (the half-domain symmetry plane), the others absorb."""
    gpu, orc = make_pair("lunar", dt=dt, precision=precision)
    kinds = ["absorb", "absorb", "reflect", "absorb", "absorb", "absorb"]
    return gpu, orc, kinds


def test_rim_crater_particle_cycle_bit_exact():
    """Frozen field, two species, 10 steps: the rim-crater level set decides
    collection identically on both sides (particle sets, states, node charges
    and surface counts bit-exact)."""
    gpu, orc, kinds = _half_crater_pair()
    E = wl.random_node_field(orc.mesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        gpu.set_particle_bc(s, kinds)
        orc.set_particle_bc(s, kinds)
        explicit_particles(gpu, orc, s, 20000, 500 + s, 3.0 / (1 + 4 * s))
    gpu.set_external_E(E)
    orc.set_external_E(E)
    ncol = 0
    for step in range(10):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            for key in ("pushed", "absorbed", "collected"):
                assert sg[key][s] == so[key][s], (step, s, key)
            ncol += sg["collected"][s]
    assert ncol > 100
    for s in range(2):
        g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
        assert np.array_equal(g["id"], o["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.array_equal(g[k], o[k]), k
        assert np.array_equal(gpu.node_charge(s), orc.W[s])
        assert np.array_equal(gpu.surface_counts(s), orc.surf[:, s])
    gpu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_photoemission_from_the_layered_crater(precision):
    """Sun 10 degrees above the ground (as in Sec. 5.2.1): emitting tets, rates
    and every emitted particle follow the oracle; the bedrock plane emits
    nothing."""
    gpu, orc, kinds = _half_crater_pair(precision, dt=0.1)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    th = math.radians(10.0)
    sun = (-math.cos(th), 0.0, math.sin(th))
    for sim in (gpu, orc):
        sim.set_particle_bc(0, kinds)
        sim.set_photoemission(0, sun, 8.0, 1.0, 21)
    q, ne = gpu.photoemission()
    ph = orc.species[0].photo
    assert ne == len(ph.tets) > 0 and q == int(ph.Q.sum())
    assert all(int(orc.fs.it_kind[d["T"]]) == 0 for d in ph.tets)
    E = np.zeros((orc.mesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    for step in range(6):
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


def test_layered_pic_steps_follow_the_oracle():
    """Solved field with surface charging on the layered half crater: counts
    and the potential follow the oracle for a few steps."""
    gpu, orc, kinds = _half_crater_pair(dt=0.1)
    for s, (q, m, vth) in enumerate(((-1.0, 1.0, 1.0), (1.0, 25.0, 0.2))):
        add_species_both(gpu, orc, q, m, 0.01)
        gpu.set_particle_bc(s, kinds)
        orc.set_particle_bc(s, kinds)
        explicit_particles(gpu, orc, s, 15000, 700 + s, vth)
    gpu.solve(); orc.solve()
    assert _rel(gpu.potential(), orc.phi) <= 1e-8
    gpu.leapfrog_init(); orc.leapfrog_init()
    for step in range(4):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            assert abs(sg["collected"][s] - so["collected"][s]) <= 1
        assert _rel(gpu.potential(), orc.phi) <= 1e-8, step
    gpu.close()


def test_bedrock_errors():
    sim = capi.Simulation((8, 8, 8), 1.0, 0.05)
    with pytest.raises(RuntimeError):
        sim.set_bedrock(2.0, 0.0)                       # eps_bed must be positive
    sim.set_bedrock(6.5, 10.0)                          # above the ground below: outside the object
    with pytest.raises(RuntimeError):
        sim.set_object(capi.OBJ_PLANE, [0.0, 0.0, 1.0, 4.2], 4.0, 1.0)
    sim.close()
    sim = capi.Simulation((8, 8, 8), 1.0, 0.05)
    sim.set_object(capi.OBJ_PLANE, [0.0, 0.0, 1.0, 4.2], 4.0, 1.0)
    with pytest.raises(RuntimeError):
        sim.set_bedrock(2.0, 10.0)                      # after set_object
    with pytest.raises(RuntimeError):                   # r_top <= r_inner
        sim.set_object(capi.OBJ_RIM_CRATER, [4.0, 4.0, 4.0, 3.0, 3.0, 5.0, 1.0, 1.0], 4.0, 1.0)
    sim.close()
