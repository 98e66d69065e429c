"""GPU particle cycle vs the oracle with a frozen node field.

FP64 bar (bit-exact): particle set (ids), positions, velocities, cell indices,
absorb/collect decisions, fixed-point node charges and surface counts, over 10
steps.  Both sides follow the same IEEE operation order (no FMA contraction)."""
import numpy as np
import pytest

from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import CASES, add_species_both, by_id, explicit_particles, make_pair

pytestmark = pytest.mark.gpu


def _compare(gpu, orc, s):
    g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
    assert np.array_equal(g["id"], o["id"]), f"particle sets differ: {len(g['id'])} vs {len(o['id'])}"
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], o[k]), k
    assert np.array_equal(gpu.node_charge(s), orc.W[s])
    assert np.array_equal(gpu.surface_counts(s), orc.surf[:, s])


@pytest.mark.parametrize("case,vth,npart", [("sphere16", 1.0, 30000), ("ragged", 3.0, 20000),
                                            ("crater", 2.0, 40000), ("plane", 1.5, 5000)])
def test_frozen_field_ten_steps_bit_exact(case, vth, npart):
    gpu, orc = make_pair(case, dt=0.2)
    E = wl.random_node_field(orc.mesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        explicit_particles(gpu, orc, s, npart, 100 + s, vth / (1 + 4 * s))
    gpu.set_external_E(E)
    orc.set_external_E(E)
    for step in range(10):
        sg = gpu.step(1)
        so = orc.step()
        for s in range(2):
            assert sg["absorbed"][s] == so["absorbed"][s], (step, s)
            assert sg["collected"][s] == so["collected"][s], (step, s)
            assert sg["pushed"][s] == so["pushed"][s], (step, s)
    for s in range(2):
        _compare(gpu, orc, s)
    gpu.close()


def test_bin_overflow_spills_and_recovers():
    """All particles start in one bin and fan out: bins overflow, the spill list
    carries particles to the next step, results stay bit-exact."""
    gpu, orc = make_pair("ragged", dt=0.3)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    g = np.random.default_rng(5)
    n = 6000
    x = g.uniform(8.0, 8.9, n); y = g.uniform(8.0, 8.9, n); z = g.uniform(8.0, 8.9, n)
    v = g.normal(0, 2.0, (3, n))
    ids = np.arange(n, dtype=np.int64)
    gpu.load_particles(0, x, y, z, v[0], v[1], v[2], ids)
    orc.load_particles(0, x, y, z, v[0], v[1], v[2], ids)
    E = np.zeros((orc.mesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    # move everyone into a single far bin first: a strong uniform field is not
    # needed -- the initial load packs 6000 particles into one bin, after which
    # the rebin capacity of the bins they fan into is exceeded
    spilled = 0
    for _ in range(8):
        st = gpu.step(1)
        orc.step()
        spilled = max(spilled, st["spilled"][0])
    _compare(gpu, orc, 0)
    gpu.close()


def test_load_maxwellian_matches_oracle():
    gpu, orc = make_pair("sphere16")
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    gpu.load_maxwellian(0, 8, 1.3, (0.2, 0.0, -0.1), 99)
    orc.load_maxwellian(0, 8, 1.3, (0.2, 0.0, -0.1), 99)
    g, o = by_id(gpu.particles(0)), by_id(orc.P[0])
    assert np.array_equal(g["id"], o["id"])
    for k in ("x", "y", "z"):
        assert np.array_equal(g[k], o[k]), k        # uniforms: exact arithmetic
    for k in ("vx", "vy", "vz"):                     # Box-Muller: libm vs CUDA log/cos, last-ulp
        assert np.allclose(g[k], o[k], rtol=1e-13, atol=1e-13), k
    gpu.close()


def test_injection_matches_oracle():
    gpu, orc = make_pair("sphere16", dt=0.05)
    E = np.zeros((orc.mesh.nnodes, 3))
    for s, (q, m, vth, drift) in enumerate(((-1.0, 1.0, 1.0, (0.0, 0.0, 0.0)),
                                            (1.0, 100.0, 0.1, (0.3, 0.0, -0.4)))):
        add_species_both(gpu, orc, q, m, 0.125 / 16)
        gpu.set_injection(s, 0b111111, 1.0, vth, drift, 1234)
        orc.set_injection(s, 0b111111, 1.0, vth, drift, 1234)
        assert np.array_equal(np.array(gpu.injection_rate(s)),
                              np.array([orc.injection_rate(s, f) for f in range(6)]))
    gpu.set_external_E(E); orc.set_external_E(E)
    for _ in range(6):
        sg, so = gpu.step(1), orc.step()
        for s in range(2):
            assert sg["injected"][s] == so["injected"][s]
    for s in range(2):
        g, o = by_id(gpu.particles(s)), by_id(orc.P[s])
        assert np.array_equal(g["id"], o["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.allclose(g[k], o[k], rtol=1e-12, atol=1e-12), k
    gpu.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_deposit_with_negative_remainder_weight(precision):
    """Particles a hair above a cell face: the seven rounded weights can sum past
    2^32, so the remainder weight is negative; node sums must stay exact."""
    gpu, orc = make_pair("sphere16", dt=0.05, precision=precision)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    g = np.random.default_rng(17)
    n = 4000
    x = 3.0 + g.uniform(0, 1, n)
    y = 2.0 + g.uniform(0, 1, n)
    z = 1.0 + g.choice([1e-13, 1e-12, 2.0 ** -40, 3e-14], n)
    zero = np.zeros(n)
    ids = np.arange(n, dtype=np.int64)
    gpu.load_particles(0, x, y, z, zero, zero, zero, ids)
    orc.load_particles(0, x, y, z, zero, zero, zero, ids)
    E = np.zeros((orc.mesh.nnodes, 3))
    gpu.set_external_E(E); orc.set_external_E(E)
    gpu.step(1); orc.step()
    W = gpu.node_charge(0)
    assert W.sum() == 2 ** 32 * n
    if precision == 0:
        assert np.array_equal(W, orc.W[0])
    else:
        assert np.abs(W - orc.W[0]).max() <= 1e-4 * 2 ** 32 * 8
    gpu.close()
