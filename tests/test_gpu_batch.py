"""Batched steps (pifepic_batch_*): one graph launch per step over many
independent instances.  Each member's result must be the same alone and in a
mix (bit-identical: fixed-point charges, deterministic per-member reductions),
and a batched FP64 member must match the oracle like a single context does."""
import numpy as np
import pytest

from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import by_id

pytestmark = pytest.mark.gpu

MEMBERS = [wl.sphere_config(12, 1.5, 8, 5, eps_in=2.0, seed_offset=11),
           wl.sphere_config(16, 2.0, 12, 5, eps_in=4.0, seed_offset=12),
           wl.sphere_config(20, 3.0, 6, 5, eps_in=10.0, seed_offset=13)]


def _member(cfg, precision):
    from paper_2011_10214_gb300 import capi
    sim = capi.from_config(cfg, precision=precision, track_ids=True)
    sim.solve()
    sim.leapfrog_init()
    return sim


@pytest.mark.parametrize("precision,precond", [(0, None), (1, None), (1, "multigrid")])
def test_member_alone_equals_member_in_mix(precision, precond):
    """Bit-identical in a batch of one and in the mix; MIXED also with the
    multigrid clusters (hierarchies built on the first batched step)."""
    from paper_2011_10214_gb300 import capi

    def batch(sims):
        b = capi.Batch(sims)
        if precond == "multigrid":
            b.set_preconditioner(capi.PRECOND_MULTIGRID)
        return b
    alone = []
    for cfg in MEMBERS:
        s = _member(cfg, precision)
        b = batch([s])
        b.step(5)
        alone.append((s.potential(), s.node_charge(0), by_id(s.particles(1))))
        b.close(); s.close()
    sims = [_member(cfg, precision) for cfg in MEMBERS]
    b = batch(sims)
    stats = b.step(5)
    assert len(stats) == 3 and all(st["pcg_iters"] > 0 for st in stats)
    for s, (phi, W, P) in zip(sims, alone):
        assert np.array_equal(s.potential(), phi)
        assert np.array_equal(s.node_charge(0), W)
        Q = by_id(s.particles(1))
        for k in ("id", "x", "y", "z", "vx", "vy", "vz"):
            assert np.array_equal(Q[k], P[k]), k
    b.close()
    for s in sims:
        s.close()


def test_batched_fp64_member_matches_oracle():
    from paper_2011_10214_gb300 import capi
    from oracle.geometry import Mesh, Sphere
    from oracle.pic import Simulation as OracleSim
    cfg = MEMBERS[1]
    gpu = capi.from_config(cfg, precision=0, track_ids=True, pcg_tol=1e-12, pcg_max_iter=5000)
    other = capi.from_config(MEMBERS[0], precision=0, pcg_tol=1e-12, pcg_max_iter=5000)
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    orc = OracleSim(m, Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"]), cfg["face_bc"],
                    cfg["dt"], tol=1e-12, maxit=5000)
    for s, sp in enumerate(cfg["species"]):
        orc.add_species(sp["q"], sp["m"], wl.macro_weight(cfg, sp))
        orc.load_maxwellian(s, sp["ppc"], sp["vth"], sp["drift"], cfg["seed"])
        orc.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
    for sim in (gpu, other):
        sim.solve(); sim.leapfrog_init()
    orc.solve(); orc.leapfrog_init()
    b = capi.Batch([other, gpu])
    for _ in range(3):
        st = b.step(1)
        so = orc.step()
        assert st[1]["injected"] == so["injected"]
    rel = np.abs(gpu.potential() - orc.phi).max() / np.abs(orc.phi).max()
    assert rel <= 1e-8, rel
    b.remove(other)
    b.step(1)
    orc.step()
    rel = np.abs(gpu.potential() - orc.phi).max() / np.abs(orc.phi).max()
    assert rel <= 1e-8, rel
    b.close(); gpu.close(); other.close()


@pytest.mark.parametrize("overlap", [False, True])
def test_served_results_equal_alone(overlap):
    """Three requests arriving while others run (continuous batching) give the
    same potential as each run alone; with overlap the admission worker sets
    requests up on its own stream while the batch steps on another."""
    import torch
    from paper_2011_10214_gb300 import capi, serve
    cfgs = [wl.sphere_config(12, 1.5, 8, 20, eps_in=2.0, seed_offset=21),
            wl.sphere_config(14, 2.0, 6, 20, eps_in=5.0, seed_offset=22),
            wl.sphere_config(10, 1.2, 10, 20, eps_in=8.0, seed_offset=23)]
    alone = []
    for c in cfgs:
        srv = serve.Server(8 << 30, steps_per_round=5, max_steps=20, keep_phi=True, overlap=False)
        r = srv.run([c], [0.0])
        srv.close()
        alone.append(r["results"][0])
    s_batch, s_admit = torch.cuda.Stream(), torch.cuda.Stream()
    srv = serve.Server(8 << 30, steps_per_round=5, max_steps=20, keep_phi=True, overlap=overlap,
                       stream=s_batch.cuda_stream, admit_stream=s_admit.cuda_stream)
    r = srv.run(cfgs, [0.0, 0.02, 0.04])
    srv.close()
    assert r["completed"] == 3 and r["p99_s"] >= r["p50_s"] > 0
    by = {x["rid"]: x for x in r["results"]}
    for i, a in enumerate(alone):
        assert by[i]["steps"] == a["steps"]
        assert np.array_equal(by[i]["phi"], a["phi"])


@pytest.mark.parametrize("precision,precond", [(0, None), (1, "jacobi"), (1, "multigrid")])
def test_cluster_solves_match_single_instance_solves(precision, precond):
    """Members of 20^3..48^3 cells put the batched solve on clusters of 2, 4,
    8 and 16 CTAs (FP64: the largest goes to the one-CTA kernel; MIXED: Jacobi
    clusters, or multigrid clusters whose hierarchies are built on that first
    batched step).  After one step from the same state, each member's potential
    equals the same instance stepped alone (persistent single-instance solver)
    to the solver tolerance."""
    from paper_2011_10214_gb300 import capi
    cfgs = [wl.sphere_config(n, 0.2 * n * 0.5, 4, 1, eps_in=3.0, seed_offset=30 + n) for n in (20, 24, 28, 36, 48)]

    def fresh(cfg):
        s = capi.from_config(cfg, precision=precision, pcg_tol=1e-12, pcg_max_iter=5000)
        s.solve(); s.leapfrog_init()
        return s
    alone = []
    for cfg in cfgs:
        s = fresh(cfg)
        s.step(1)
        alone.append(s.potential())
        s.close()
    sims = [fresh(cfg) for cfg in cfgs]
    b = capi.Batch(sims)
    if precond is not None:
        b.set_preconditioner(capi.PRECOND_MULTIGRID if precond == "multigrid" else capi.PRECOND_JACOBI)
    st = b.step(1)
    for k, (s, phi) in enumerate(zip(sims, alone)):
        assert st[k]["pcg_converged"] == 1, k
        rel = np.abs(s.potential() - phi).max() / np.abs(phi).max()
        assert rel <= 1e-8, (cfgs[k]["n"], rel)
    b.close()
    for s in sims:
        s.close()
