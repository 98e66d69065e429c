"""GPU IFE field solve vs the oracle (Sec. 2.1 Eqs. 2.1-2.5, PCG level of Sec. 2.5).

Tolerance: both sides iterate to ||r|| <= 1e-12 ||b|| on the same discrete
system, so the potentials agree to about cond(A) * 1e-12; the bar is 1e-8
relative (max norm), the figure the method's FP64 path is held to."""
import numpy as np
import pytest

from tests.pairs import CASES, make_pair

pytestmark = pytest.mark.gpu

TOL_PHI = 1e-8


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", list(CASES))
def test_solve_field_matches_oracle(case):
    gpu, orc = make_pair(case)
    fs = orc.fs
    g = np.random.default_rng(11)
    F = g.normal(size=fs.mesh.nnodes) * fs.mesh.h ** 3
    q = g.normal(size=len(fs.it_cell))
    phi_o, it_o, rr_o = fs.solve(F, q, tol=1e-12, maxit=5000)
    it, rr = gpu.solve_field(F, q)
    assert rr <= 1e-12
    phi = gpu.potential()
    assert _rel(phi, phi_o) <= TOL_PHI
    E_o = fs.node_E(phi_o, q)
    assert _rel(gpu.node_E(), E_o) <= TOL_PHI
    assert abs(it - it_o) <= max(3, 0.05 * it_o)
    gpu.close()


def test_pcg_cap_and_zero_rhs():
    gpu, orc = make_pair("sphere16", maxit=3)
    F = np.random.default_rng(1).normal(size=orc.mesh.nnodes)
    it, rr = gpu.solve_field(F, None)
    assert it == 3 and rr > 1e-12
    gpu.close()
    gpu, orc = make_pair("ragged")
    it, rr = gpu.solve_field(np.zeros(orc.mesh.nnodes), np.zeros(len(orc.fs.it_cell)))
    phi_o, _, _ = orc.fs.solve(np.zeros(orc.mesh.nnodes), np.zeros(len(orc.fs.it_cell)), tol=1e-12, maxit=5000)
    assert _rel(gpu.potential(), phi_o) <= TOL_PHI
    gpu.close()


def test_sphere_with_manufactured_source_and_jump_matches_oracle():
    """The manufactured sphere's source (rho = -6) and constant flux jump
    (eps+ gamma / R^2) with zero Dirichlet faces, at 16^3 and 32^3: the CUDA
    solve equals the oracle's solve of the same discrete system.  This is a
    parity test of the solver on a sphere with a flux jump, not the O(h^2)
    convergence pin (the ABI takes one value per face, so the manufactured
    solution's own face data cannot be imposed)."""
    from paper_2011_10214_gb300 import capi
    from oracle.field import FieldSystem
    from oracle.geometry import Mesh, Sphere
    for n in (16, 32):
        h = 2.0 / n
        R, em, ep, gamma = 0.6183, 4.0, 1.0, 1.0
        sim = capi.Simulation((n, n, n), h, 0.05, origin=(-1.0, -1.0, -1.0), pcg_tol=1e-12, pcg_max_iter=5000)
        m = Mesh(n, n, n, h, origin=(-1, -1, -1))
        sim.set_field_bc([("D", 0.0)] * 6)
        sim.set_object(capi.OBJ_SPHERE, [0.0, 0.0, 0.0, R], em, ep)
        nit = sim.sizes()["n_interface_tets"]
        F = np.full(m.nnodes, -6.0 * h ** 3)
        sim.solve_field(F, np.full(nit, ep * gamma / R ** 2))
        fs = FieldSystem(m, Sphere(m, (0, 0, 0), R, em, ep), [("D", 0.0)] * 6)
        phi_o, _, _ = fs.solve(F, np.full(nit, ep * gamma / R ** 2), tol=1e-12, maxit=5000)
        assert _rel(sim.potential(), phi_o) <= TOL_PHI
        sim.close()


@pytest.mark.parametrize("n", [48, 64, 80])
def test_solve_sizes_of_every_nodes_per_thread_variant(n):
    """Meshes whose node count puts 2, 4 and 8 nodes on each thread of the
    register-resident PCG (one 512-thread block per SM): both precisions reach
    the oracle's FP64 solution at tol 1e-12."""
    from oracle.field import FieldSystem
    from oracle.geometry import Mesh, Sphere
    from paper_2011_10214_gb300 import capi
    m = Mesh(n, n, n, 0.5)
    c = n * 0.25
    R = n * 0.1
    fs = FieldSystem(m, Sphere(m, (c, c, c), R, 4.0, 1.0), [("D", 0.0)] * 6)
    g = np.random.default_rng(3)
    F = g.normal(size=m.nnodes) * m.h ** 3
    q = g.normal(size=len(fs.it_cell))
    phi_o, it_o, _ = fs.solve(F, q, tol=1e-12, maxit=5000)
    for precision in (capi.FP64, capi.MIXED):
        sim = capi.Simulation((n, n, n), 0.5, 0.05, precision=precision, pcg_tol=1e-12, pcg_max_iter=5000)
        sim.set_field_bc([("D", 0.0)] * 6)
        sim.set_object(capi.OBJ_SPHERE, [c, c, c, R], 4.0, 1.0)
        it, rr = sim.solve_field(F, q)
        assert rr <= 1e-12, (precision, rr)
        assert _rel(sim.potential(), phi_o) <= TOL_PHI, precision
        if precision == capi.FP64:
            assert abs(it - it_o) <= max(3, 0.05 * it_o), (it, it_o)
        # a second solve from the converged state (warm start) stops at once
        it2, rr2 = sim.solve_field(F, q)
        assert rr2 <= 1e-12 and it2 <= 2, (precision, it2)
        sim.close()


def test_global_memory_solver_on_a_large_crater():
    """112 x 112 x 56 cells (728k nodes, more than 8 per thread of the
    register-resident kernel): the global-memory persistent PCG, both
    precisions, reaches the oracle's FP64 solution at tol 1e-12."""
    from oracle.field import FieldSystem
    from oracle.geometry import CapCrater, Mesh
    from paper_2011_10214_gb300 import capi
    n = (112, 112, 56)
    m = Mesh(*n, 1.0)
    crater = (14.3, 56.0, 56.0, 20.0, 7.0)
    bc = [("N",)] * 5 + [("D", 0.0)]
    fs = FieldSystem(m, CapCrater(m, *crater, 4.0, 1.0), bc)
    g = np.random.default_rng(5)
    F = g.normal(size=m.nnodes)
    q = g.normal(size=len(fs.it_cell))
    phi_o, _, _ = fs.solve(F, q, tol=1e-12, maxit=20000)
    for precision, refinement in ((capi.FP64, None), (capi.MIXED, None), (capi.MIXED, (1e-3, 0.2))):
        sim = capi.Simulation(n, 1.0, 0.05, precision=precision, pcg_tol=1e-12, pcg_max_iter=20000)
        sim.set_field_bc(bc)
        sim.set_object(capi.OBJ_CAP_CRATER, list(crater), 4.0, 1.0)
        if refinement:
            sim.set_refinement(*refinement)
        it, rr = sim.solve_field(F, q)
        assert rr <= 1e-12, (precision, rr)
        assert _rel(sim.potential(), phi_o) <= TOL_PHI, precision
        sim.close()


def test_refinement_controls():
    """MIXED refinement with other inner stops (pifepic_set_refinement) still
    reaches the oracle's FP64 solution; bad controls are refused."""
    from oracle.field import FieldSystem
    from oracle.geometry import Mesh, Sphere
    from paper_2011_10214_gb300 import capi
    n = 64
    m = Mesh(n, n, n, 0.5)
    fs = FieldSystem(m, Sphere(m, (16.0, 16.0, 16.0), 6.0, 4.0, 1.0), [("D", 0.0)] * 6)
    g = np.random.default_rng(8)
    F = g.normal(size=m.nnodes) * m.h ** 3
    q = g.normal(size=len(fs.it_cell))
    phi_o, _, _ = fs.solve(F, q, tol=1e-12, maxit=5000)
    for red, margin in ((1e-3, 0.1), (1e-5, 1.0), (1e-2, 0.5)):
        sim = capi.Simulation((n, n, n), 0.5, 0.05, precision=capi.MIXED, pcg_tol=1e-12, pcg_max_iter=5000)
        sim.set_field_bc([("D", 0.0)] * 6)
        sim.set_object(capi.OBJ_SPHERE, [16.0, 16.0, 16.0, 6.0], 4.0, 1.0)
        sim.set_refinement(red, margin)
        it, rr = sim.solve_field(F, q)
        assert rr <= 1e-12, (red, margin, rr)
        assert _rel(sim.potential(), phi_o) <= TOL_PHI, (red, margin)
        sim.close()
    sim = capi.Simulation((8, 8, 8), 0.5, 0.05, precision=capi.MIXED)
    for red, margin in ((0.0, 0.5), (1.0, 0.5), (1e-4, 0.0), (1e-4, 1.5), (float("nan"), 0.5)):
        with pytest.raises(RuntimeError):
            sim.set_refinement(red, margin)
    sim.close()


@pytest.mark.parametrize("case", list(CASES))
def test_multigrid_preconditioned_solve_matches_oracle(case):
    """MIXED solve with the geometric multigrid preconditioner (Galerkin coarse
    levels, odd axes included, Dirichlet and interface rows, hybrid IFE
    meshes): the oracle's FP64 solution at tol 1e-12, in a small fraction of
    the Jacobi iterations."""
    from paper_2011_10214_gb300 import capi
    gpu, orc = make_pair(case, precision=capi.MIXED)
    gpu.set_preconditioner(capi.PRECOND_MULTIGRID)
    fs = orc.fs
    g = np.random.default_rng(11)
    F = g.normal(size=fs.mesh.nnodes) * fs.mesh.h ** 3
    q = np.where(fs.it_kind == 0, g.normal(size=len(fs.it_cell)), 0.0)
    phi_o, it_o, _ = fs.solve(F, q, tol=1e-12, maxit=5000)
    it, rr = gpu.solve_field(F, q)
    assert rr <= 1e-12
    assert _rel(gpu.potential(), phi_o) <= TOL_PHI
    assert it <= max(40, it_o // 3), (it, it_o)
    # back to Jacobi: the same solution
    gpu.set_preconditioner(capi.PRECOND_JACOBI)
    gpu.solve_field(F, q)
    assert _rel(gpu.potential(), phi_o) <= TOL_PHI
    gpu.close()


def test_preconditioner_choice_is_validated():
    from paper_2011_10214_gb300 import capi
    sim = capi.Simulation((8, 8, 8), 0.5, 0.05, precision=capi.MIXED)
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        sim.set_preconditioner(7)
    sim.close()


def test_auto_moves_to_multigrid_after_a_capped_jacobi_solve():
    """AUTO (MIXED): the crater's Jacobi solves stop at a cap of 40 unconverged
    at tol 1e-12.  The first (cold) solve changes nothing; after the second
    (warm-started) one the context runs the multigrid cycle, and its next solve
    converges within the same cap to the oracle's potential.  An explicit
    JACOBI stays capped."""
    from paper_2011_10214_gb300 import capi
    from tests.pairs import add_species_both, explicit_particles
    for precond in ("auto", "jacobi"):
        gpu, orc = make_pair("crater", precision=1, maxit=40)
        orc.maxit = 5000                      # the oracle solves to the tolerance
        if precond == "jacobi":
            gpu.set_preconditioner(capi.PRECOND_JACOBI)
        add_species_both(gpu, orc, -1.0, 1.0, 0.01)
        explicit_particles(gpu, orc, 0, 4000, 5, 1.0)
        assert gpu.solver == capi.SOLVER_REGISTERS
        st0 = gpu.solve()
        assert st0["pcg_converged"] == 0 and st0["pcg_iters"] == 40
        assert gpu.solver == capi.SOLVER_REGISTERS        # a cold start at the cap is not a reason
        st1 = gpu.solve()
        assert st1["pcg_converged"] == 0 and st1["pcg_iters"] == 40
        assert gpu.solver == (capi.SOLVER_MULTIGRID if precond == "auto" else capi.SOLVER_REGISTERS)
        st2 = gpu.solve()
        if precond == "auto":
            assert st2["pcg_converged"] == 1 and st2["pcg_iters"] < 40
            orc.solve()
            assert _rel(gpu.potential(), orc.phi) <= TOL_PHI
        else:
            assert st2["pcg_converged"] == 0 and st2["pcg_iters"] == 40
        gpu.close()
