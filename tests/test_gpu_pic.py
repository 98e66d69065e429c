"""Full PIC steps (scatter, IFE solve, node field, gather, push, injection,
collection) on the GPU vs the oracle, plus run-to-run determinism."""
import numpy as np
import pytest

from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import by_id

pytestmark = pytest.mark.gpu


def _pair(cfg, tol=1e-12):
    from paper_2011_10214_gb300 import capi
    from oracle.geometry import Mesh, Sphere
    from oracle.pic import Simulation as OracleSim
    gpu = capi.from_config(cfg, track_ids=True, pcg_tol=tol, pcg_max_iter=5000)
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    orc = OracleSim(m, Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"]), cfg["face_bc"],
                    cfg["dt"], tol=tol, maxit=5000)
    for s, sp in enumerate(cfg["species"]):
        orc.add_species(sp["q"], sp["m"], wl.macro_weight(cfg, sp))
        orc.load_maxwellian(s, sp["ppc"], sp["vth"], sp["drift"], cfg["seed"])
        orc.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
    return gpu, orc


def test_sphere16_pic_steps_match_oracle():
    cfg = wl.SPHERE16
    gpu, orc = _pair(cfg)
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


def test_gpu_runs_are_deterministic():
    from paper_2011_10214_gb300 import capi
    cfg = wl.SPHERE16
    out = []
    for _ in range(2):
        sim = capi.from_config(cfg, track_ids=False)
        sim.solve(); sim.leapfrog_init()
        sim.step(3)
        out.append((sim.potential(), sim.node_charge(0), sim.node_charge(1), sim.node_E()))
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
