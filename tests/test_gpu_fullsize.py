"""Full-size checks on the workloads bench.py times, in its launch configuration
(MIXED, the same set-up through capi.from_config; ids are tracked so that
particles can be matched, which adds an id array to the same kernels):

  * c2, the 64^3 sphere with 64 ppc/species (32.6M particles): one step in a
    frozen field, 10,000 particles per species sampled by id and pushed one by
    one by the oracle (FP64) from the same state and the same (FP32) node
    field, within the FP32-mode bar 1e-4; exact conservation of counts and
    exact 2^32-unit charge totals at full size; after solved steps the oracle's
    own IFE matrix and right-hand side (built from the GPU's integer charges and
    surface counts) confirm the potential's relative residual at the solve
    tolerance;
  * c4, the 64-instance batch: three sampled members (smallest, median,
    largest) give bit-identical potentials and charges in the 64-member batch
    and in a batch of their own;
  * c3, the 160x160x80 crater with photoemission (389.5M particles): exact
    conservation of counts and charge totals over two solved steps.
"""
import numpy as np
import pytest

from paper_2011_10214_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


def _oracle_field_system(cfg):
    from oracle.field import FieldSystem
    from oracle.geometry import Mesh, Sphere
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    return m, FieldSystem(m, Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"]), cfg["face_bc"])


def test_c2_frozen_field_step_sampled_against_oracle():
    from oracle import particles as pt
    from paper_2011_10214_gb300 import capi
    cfg = wl.SPHERE64
    sim = capi.from_config(cfg, precision=capi.MIXED, track_ids=True)
    sim.solve()
    sim.leapfrog_init()
    E = sim.node_E_f32().astype(np.float64)       # the FP32 field the push reads, exactly
    sim.set_external_E(E)
    m, fs = _oracle_field_system(cfg)
    obj = fs.obj
    rng = np.random.default_rng(64)
    before = [sim.particles(s) for s in range(2)]
    n0 = [len(b["id"]) for b in before]
    assert sum(n0) > 32_000_000
    st = sim.step(1)
    for s, sp in enumerate(cfg["species"]):
        after = sim.particles(s)
        n1 = len(after["id"])
        # exact bookkeeping at full size
        assert n1 == n0[s] + st["injected"][s] - st["absorbed"][s] - st["collected"][s]
        W = sim.node_charge(s)
        assert int(W.sum()) == (1 << 32) * n1
        # 10,000 sampled particles pushed one by one by the oracle
        pick = rng.choice(n0[s], 10_000, replace=False)
        P = {k: np.array(before[s][k][pick], dtype=np.float64) for k in ("x", "y", "z", "vx", "vy", "vz")}
        ids = before[s]["id"][pick]
        k = (sp["q"] / sp["m"]) * cfg["dt"]
        pt.push(m, E, P, k, cfg["dt"] / cfg["h"])
        gone = pt.outside(m, P["x"], P["y"], P["z"])
        gone |= ~gone & (obj.L(P["x"], P["y"], P["z"]) < 0.0)
        order = np.argsort(after["id"])
        pos = np.searchsorted(after["id"], ids, sorter=order)
        pos = np.minimum(pos, n1 - 1)
        found = after["id"][order[pos]] == ids
        mismatch = np.sum(found == gone)            # kept by one side only
        assert mismatch <= max(2, 1e-3 * len(ids)), mismatch
        both = found & ~gone
        assert both.sum() > 9_000
        g = order[pos[both]]
        for key in ("x", "y", "z", "vx", "vy", "vz"):
            o = P[key][both]
            d = np.abs(after[key][g] - o) / np.maximum(np.abs(o), 1.0)
            assert d.max() <= TOL32, (s, key, d.max())
    sim.close()


def test_c2_solved_steps_residual_confirmed_by_oracle():
    from paper_2011_10214_gb300 import capi
    cfg = wl.SPHERE64
    sim = capi.from_config(cfg, precision=capi.MIXED)
    sim.solve()
    sim.leapfrog_init()
    st = sim.step(3)
    assert st["pcg_converged"] == 1
    m, fs = _oracle_field_system(cfg)
    # right-hand side from the GPU's integer state: node charges and surface counts
    F = np.zeros(m.nnodes)
    Q = np.zeros(len(fs.cut_cells))
    for s, sp in enumerate(cfg["species"]):
        w = wl.macro_weight(cfg, sp)
        F += ((sp["q"] * w) / 4294967296.0) * sim.node_charge(s).astype(np.float64)
        Q += (sp["q"] * w) * sim.surface_counts(s).astype(np.float64)
    cells, _ = sim.cut_cells()
    assert np.array_equal(cells, fs.cut_cells)
    assert Q.any()                                   # charge has reached the sphere
    qT = fs.q_tets(Q)
    b = fs.load(F, qT)[fs.free] - fs.A_fd @ fs.g[fs.dirn]
    phi = sim.potential()
    r = b - fs.A_ff @ phi[fs.free]
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.01e-6, rel                       # the solve's own stopping test, checked independently
    assert np.all(phi[fs.dirn] == fs.g[fs.dirn])
    sim.close()


def test_c4_sampled_members_equal_alone():
    import torch
    from paper_2011_10214_gb300 import capi, serve
    rng = np.random.default_rng(2011102144)
    cfgs = serve.request_distribution(rng, 64, big_fraction=0.0)
    sizes = np.array([c["n"][0] ** 3 * c["species"][0]["ppc"] for c in cfgs])
    picks = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))]
    stream = torch.cuda.Stream()

    def fresh(c):
        s = capi.from_config(c, precision=capi.MIXED, stream=stream.cuda_stream)
        s.solve(); s.leapfrog_init()
        return s
    alone = {}
    for i in picks:                                  # the member in a batch of its own
        s = fresh(cfgs[i])
        b1 = capi.Batch([s], stream=stream.cuda_stream)
        b1.step(2)
        alone[i] = (s.potential(), s.node_charge(0), s.node_charge(1))
        b1.close()
        s.close()
    sims = [fresh(c) for c in cfgs]
    batch = capi.Batch(sims, stream=stream.cuda_stream)
    batch.step(2)
    for i in picks:
        got = (sims[i].potential(), sims[i].node_charge(0), sims[i].node_charge(1))
        for a, b in zip(got, alone[i]):
            assert np.array_equal(a, b), cfgs[i]["n"]
    batch.close()
    for s in sims:
        s.close()


def test_c3_crater_full_size_conservation():
    from paper_2011_10214_gb300 import capi
    cfg = wl.CRATER160
    sim = capi.from_config(cfg, precision=capi.MIXED)
    ns = len(cfg["species"]) + (1 if cfg.get("photo") else 0)
    sim.solve()
    sim.leapfrog_init()
    n0 = [sim.count(s) for s in range(ns)]
    assert sum(n0) > 380_000_000
    st = sim.step(2)
    for s in range(ns):
        n1 = sim.count(s)
        assert n1 == n0[s] + st["injected"][s] - st["absorbed"][s] - st["collected"][s], s
        assert int(sim.node_charge(s).sum()) == (1 << 32) * n1, s
        assert st["dropped"][s] == 0
    assert st["injected"][ns - 1] > 0                 # photoelectrons were emitted
    sim.close()
