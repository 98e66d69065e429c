"""Failure detection without a GPU fault: every device wait of the PCG is
bounded and reports, allocation failure is reached through the library's own
memory cap, and bad inputs are refused before they reach a kernel.

  * a grid exchange made to wait for an arrival that never comes gives up after
    its bounded wait (about a second): the call returns ETIMEOUT and the context
    then solves correctly (both persistent solvers, both precisions);
  * a memory cap below what a context needs makes its creation (or a particle
    load) return ENOMEM; the library's byte count returns to where it was when
    the contexts are destroyed;
  * particles outside the box or with NaN, and node fields or loads with NaN,
    are refused with EINVAL and change nothing.
Nothing here traps, faults or hangs the GPU."""
import numpy as np
import pytest

from tests.pairs import add_species_both, explicit_particles, make_pair

pytestmark = pytest.mark.gpu

TOL_PHI = 1e-8


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_exchange_timeout_reports_and_context_recovers(precision):
    from paper_2011_10214_gb300 import capi
    gpu, orc = make_pair("sphere16", precision=precision)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    explicit_particles(gpu, orc, 0, 4000, 3, 1.0)
    gpu.test_hold_exchange(1)
    with pytest.raises(capi.PifepicError, match="ETIMEOUT"):
        gpu.solve()
    # the hook is cleared with the counters: the same context now solves as the oracle does
    st = gpu.solve()
    orc.solve()
    assert st["pcg_converged"] == 1
    assert _rel(gpu.potential(), orc.phi) <= TOL_PHI
    gpu.leapfrog_init()
    gpu.step(2)
    gpu.close()


def test_exchange_timeout_in_the_global_memory_solver():
    """A mesh above 8 nodes per thread of the register-resident kernel runs the
    global-memory PCG; its bounded exchange wait reports the same way."""
    from paper_2011_10214_gb300 import capi
    n = (96, 96, 72)                 # 97 * 97 * 73 = 686,857 nodes
    sim = capi.Simulation(n, 0.5, 0.05, precision=capi.MIXED, pcg_tol=1e-8, pcg_max_iter=3000)
    sim.set_field_bc([("D", 0.0)] * 6)
    sim.set_object(capi.OBJ_SPHERE, [24.0, 24.0, 18.0, 6.0], 4.0, 1.0)
    F = np.random.default_rng(4).normal(size=sim.sizes()["nnodes"]) * 0.125
    sim.add_species(-1.0, 1.0, 0.01)
    sim.test_hold_exchange(1)
    with pytest.raises(capi.PifepicError, match="ETIMEOUT"):
        sim.solve()
    it, rr = sim.solve_field(F, None)
    assert rr <= 1e-8 and it > 0
    sim.close()


def test_hold_hook_rejects_bad_values():
    from paper_2011_10214_gb300 import capi
    sim = capi.Simulation((8, 8, 8), 0.5, 0.05)
    for bad in (-1, 2):
        with pytest.raises(capi.PifepicError, match="EINVAL"):
            sim.test_hold_exchange(bad)
    sim.close()


def test_memory_cap_gives_enomem_and_the_count_is_exact():
    from paper_2011_10214_gb300 import capi
    base = capi.memory_use()
    sim = capi.Simulation((32, 32, 32), 0.5, 0.05, precision=capi.MIXED)
    sim.set_object(capi.OBJ_SPHERE, [8.0, 8.0, 8.0, 3.0], 4.0, 1.0)
    held = capi.memory_use() - base
    assert held > 1 << 20
    try:
        # a second context of the same size does not fit under a cap at the first one's usage
        capi.set_memory_limit(base + held + (held // 2))
        with pytest.raises(capi.PifepicError, match="ENOMEM"):
            capi.Simulation((32, 32, 32), 0.5, 0.05, precision=capi.MIXED)
        assert capi.memory_use() == base + held           # the failed creation freed what it took
        # a particle load that would pass the cap fails the same way and leaves the species empty
        s = sim.add_species(-1.0, 1.0, 0.01)
        with pytest.raises(capi.PifepicError, match="ENOMEM"):
            sim.load_maxwellian(s, 2000, 1.0, (0.0, 0.0, 0.0), 7)
    finally:
        capi.set_memory_limit(0)
    sim.close()
    assert capi.memory_use() == base
    sim = capi.Simulation((32, 32, 32), 0.5, 0.05, precision=capi.MIXED)   # fits again without the cap
    sim.close()
    assert capi.memory_use() == base


def test_bad_particles_and_fields_are_refused():
    from paper_2011_10214_gb300 import capi
    gpu, orc = make_pair("sphere16")
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    n0 = explicit_particles(gpu, orc, 0, 1000, 9, 1.0)
    assert gpu.count(0) == n0
    x = np.array([1.5, 2.5, 3.5]); y = np.array([1.5, 1.5, 1.5]); z = np.array([0.5, 0.5, 0.5])
    v = np.zeros(3)
    for bad in ("nan_x", "outside", "at_face", "inf_v"):
        xx, yy, vv = x.copy(), y.copy(), v.copy()
        if bad == "nan_x":
            xx[1] = np.nan
        elif bad == "outside":
            yy[2] = -1e-9
        elif bad == "at_face":
            xx[0] = 16.0                                     # the box is [0, n)
        else:
            vv[0] = np.inf
        with pytest.raises(capi.PifepicError, match="EINVAL"):
            gpu.load_particles(0, xx, yy, z, vv, v, v, np.arange(3) + 10**9)
        assert gpu.count(0) == n0                            # nothing appended
    gpu.load_particles(0, x, y, z, v, v, v, np.arange(3) + 10**9)
    assert gpu.count(0) == n0 + 3
    nn = orc.mesh.nnodes
    E = np.zeros((nn, 3))
    E[5, 1] = np.nan
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        gpu.set_external_E(E)
    F = np.zeros(nn)
    F[7] = np.inf
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        gpu.solve_field(F, None)
    q = np.zeros(gpu.sizes()["n_interface_tets"])
    q[0] = np.nan
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        gpu.solve_field(np.zeros(nn), q)
    # the context still steps and solves as the oracle does
    orc.load_particles(0, x, y, z, v, v, v, np.arange(3) + 10**9)
    gpu.solve(); orc.solve()
    assert _rel(gpu.potential(), orc.phi) <= TOL_PHI
    gpu.close()
