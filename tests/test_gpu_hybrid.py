"""GPU hybrid grid (pifepic_mesh_desc.ife_refine; Sec. 2.2: the IFE mesh may
have a different resolution from the PIC mesh) vs the oracle (oracle/pic.py
refine).  Set-up and FP64 solve parity of the refined cases run in
test_gpu_setup.py and test_gpu_field.py (every case of tests/pairs.py); this
file checks the particle side: deposits on the IFE mesh, the gather at the PIC
nodes, hit cells and photoemission in IFE units."""
import math

import numpy as np
import pytest

from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import add_species_both, by_id, explicit_particles, make_pair

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", ["sphere_h2", "crater_h4"])
def test_hybrid_particle_cycle_bit_exact(case):
    """Frozen field on the IFE nodes, 10 steps: particle sets, states, IFE node
    charges and surface counts bit-exact (FP64)."""
    gpu, orc = make_pair(case, dt=0.2)
    assert orc.r > 1 and gpu.refine == orc.r
    E = wl.random_node_field(orc.fmesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        explicit_particles(gpu, orc, s, 12000, 900 + s, 2.0 / (1 + 4 * s))
    gpu.set_external_E(E)
    orc.set_external_E(E)
    ncol = 0
    for step in range(10):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            for key in ("pushed", "absorbed", "collected"):
                assert sg[key][s] == so[key][s], (step, s, key)
            ncol += sg["collected"][s]
    assert ncol > 0
    for s in range(2):
        g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
        assert np.array_equal(g["id"], o["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.array_equal(g[k], o[k]), k
        W = gpu.node_charge(s)
        assert len(W) == orc.fmesh.nnodes
        assert np.array_equal(W, orc.W[s])
        assert np.array_equal(gpu.surface_counts(s), orc.surf[:, s])
    gpu.close()


def test_hybrid_mixed_particle_cycle():
    gpu, orc = make_pair("sphere_h2", dt=0.2, precision=1)
    E = wl.random_node_field(orc.fmesh.nnodes, 3, scale=0.7)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    explicit_particles(gpu, orc, 0, 12000, 77, 2.0)
    gpu.set_external_E(E)
    orc.set_external_E(E)
    for _ in range(10):
        gpu.step(1)
        orc.step()
    g, o = by_id(gpu.particles(0)), by_id(orc.P[0])
    common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
    assert len(g["id"]) + len(o["id"]) - 2 * len(common) <= max(2, 1e-3 * len(o["id"]))
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        d = np.abs(g[k][gi] - o[k][oi]) / np.maximum(np.abs(o[k][oi]), 1.0)
        assert d.max() <= 1e-4, k
    W = gpu.node_charge(0)
    assert W.sum() == 2 ** 32 * len(g["id"])
    assert np.abs(W - orc.W[0]).max() <= 1e-4 * 2 ** 32 * 8
    gpu.close()


def test_hybrid_pic_steps_follow_the_oracle():
    """Solved field on the IFE mesh, read at the PIC nodes: counts and the
    potential follow the oracle."""
    gpu, orc = make_pair("sphere_h2", dt=0.1)
    for s, (q, m, vth) in enumerate(((-1.0, 1.0, 1.0), (1.0, 25.0, 0.2))):
        add_species_both(gpu, orc, q, m, 0.01)
        explicit_particles(gpu, orc, s, 10000, 40 + s, vth)
    gpu.solve(); orc.solve()
    assert _rel(gpu.potential(), orc.phi) <= 1e-8
    gpu.leapfrog_init(); orc.leapfrog_init()
    for step in range(4):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            assert abs(sg["collected"][s] - so["collected"][s]) <= 1
            assert abs(sg["absorbed"][s] - so["absorbed"][s]) <= 1
        assert _rel(gpu.potential(), orc.phi) <= 1e-8, step
    assert _rel(gpu.node_E(), orc.E) <= 1e-8
    gpu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_hybrid_photoemission(precision):
    """Emission from the IFE mesh's surface pieces, moved to PIC units."""
    gpu, orc = make_pair("crater_h4", dt=0.1, precision=precision)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    th = math.radians(25.0)
    sun = (-math.cos(th), 0.0, math.sin(th))
    for sim in (gpu, orc):
        sim.set_photoemission(0, sun, 4.0, 1.0, 9)
    q, ne = gpu.photoemission()
    ph = orc.species[0].photo
    assert ne == len(ph.tets) > 0 and q == int(ph.Q.sum())
    E = np.zeros((orc.fmesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    for step in range(5):
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
