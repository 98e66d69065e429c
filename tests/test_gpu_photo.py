"""GPU photoelectron emission (pifepic_set_photoemission; Sec. 5.2.2) vs the
oracle (oracle/photo.py).  Bar: the emission set-up (fixed-point rates,
emitting tets) and every count are exact integers; FP64 emitted states agree to
1e-12 (CUDA and libm transcendental functions differ in the last ulp); MIXED
stores them in FP32."""
import math

import numpy as np
import pytest

from tests.pairs import add_species_both, by_id, make_pair

pytestmark = pytest.mark.gpu

SUN = (-math.cos(math.radians(20.0)), 0.0, math.sin(math.radians(20.0)))


def _photo_pair(precision=0, dt=0.05, density=6.0, vth=1.0, seed=77):
    gpu, orc = make_pair("crater_sun", dt=dt, precision=precision)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    gpu.set_photoemission(0, SUN, density, vth, seed)
    orc.set_photoemission(0, SUN, density, vth, seed)
    return gpu, orc


def test_setup_rates_are_exact():
    gpu, orc = _photo_pair()
    q, ne = gpu.photoemission()
    ph = orc.species[0].photo
    assert ne == len(ph.tets) > 0
    assert q == int(ph.Q.sum())
    gpu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_emission_matches_oracle(precision):
    gpu, orc = _photo_pair(precision)
    E = np.zeros((orc.mesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    gpu.solve(); orc.solve()
    for step in range(8):
        sg, so = gpu.step(1), orc.step()
        assert sg["injected"][0] == so["injected"][0], step
        assert sg["inj_rejected"][0] == so["inj_rejected"][0], step
        assert sg["absorbed"][0] == so["absorbed"][0], step
        assert sg["collected"][0] == so["collected"][0], step
    assert np.array_equal(gpu.surface_counts(0), orc.surf[:, 0])
    g, o = by_id(gpu.particles(0)), by_id(orc.P[0])
    assert np.array_equal(g["id"], o["id"])
    tol = 1e-12 if precision == 0 else 2e-6
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.allclose(g[k], o[k], rtol=tol, atol=tol), k
    if precision == 0:
        assert np.array_equal(gpu.node_charge(0), orc.W[0])
    gpu.close()


def test_photo_charging_drives_the_field():
    """With the field solved, the surface charge left by the emission enters the
    flux jump: the potential follows the oracle's."""
    gpu, orc = make_pair("crater_sun", dt=0.05)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    gpu.set_photoemission(0, SUN, 6.0, 1.0, 5)
    orc.set_photoemission(0, SUN, 6.0, 1.0, 5)
    gpu.solve(); orc.solve()
    gpu.leapfrog_init(); orc.leapfrog_init()
    for _ in range(4):
        gpu.step(1); orc.step()
    phi = gpu.potential()
    assert np.abs(phi).max() > 0
    rel = np.abs(phi - orc.phi).max() / np.abs(orc.phi).max()
    assert rel <= 1e-8, rel
    gpu.close()
