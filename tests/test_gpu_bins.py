"""Particle bins of edge 8 (MIXED; pifepic_set_bin_edge) against the FP64
oracle and against bins of edge 4.

  * ten frozen-field steps with bins of 8^3 cells: positions and velocities
    within the FP32 bar 1e-4 per step, rare cell/absorb mismatches, exact
    charge totals (meshes with partial bins, an object, a hybrid IFE mesh);
  * one step from the same state with edges 4 and 8: every particle's state is
    bit-identical (the push arithmetic does not depend on the edge), counts and
    charge totals are equal, and each node charge differs by no more than the
    stayer rounding allows (2^15 units per particle touching the node: a
    stayer's weights are rounded to 2^-19 of a particle, a bin leaver's to
    2^-32, and which particles stay depends on the edge);
  * PIC steps with solves at edge 8 track the oracle's potential within 1e-4;
  * a batch whose members use both edges gives each member what it gives alone;
  * bad edges, FP64 contexts and late calls are refused.
"""
import numpy as np
import pytest

from paper_2011_10214_gb300 import workloads as wl
from tests.pairs import add_species_both, by_id, explicit_particles, make_pair

pytestmark = pytest.mark.gpu

MIXED = 1
TOL32 = 1e-4


@pytest.mark.parametrize("case,vth,npart", [("sphere16", 1.0, 30000), ("ragged", 3.0, 20000),
                                            ("crater", 2.0, 40000), ("sphere_h2", 1.0, 20000)])
def test_edge8_frozen_field_ten_steps(case, vth, npart):
    gpu, orc = make_pair(case, dt=0.2, precision=MIXED)
    gpu.set_bin_edge(8)
    assert gpu.bin_edge == 8
    fmesh = orc.fmesh if orc.r > 1 else orc.mesh   # the field and the charges live on the IFE mesh
    E = wl.random_node_field(fmesh.nnodes, 3, scale=0.7)
    for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
        add_species_both(gpu, orc, q, m, 0.01)
        explicit_particles(gpu, orc, s, npart, 100 + s, vth / (1 + 4 * s))
    gpu.set_external_E(E)
    orc.set_external_E(E)
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
        cell_rate = np.mean(np.any([np.floor(g[k][gi]) != np.floor(o[k][oi]) for k in ("x", "y", "z")], axis=0))
        assert cell_rate <= 1e-3, cell_rate
        W = gpu.node_charge(s)
        assert W.sum() == 2 ** 32 * len(g["id"])
        assert np.abs(W - orc.W[s]).max() <= TOL32 * 2 ** 32 * 8
    gpu.close()


def _touch_counts(mesh_n, P):
    """Particles whose cell has node n as a corner, per node (PIC mesh)."""
    nx, ny, nz = mesh_n
    NX, NY = nx + 1, ny + 1
    i, j, k = (np.floor(P[a]).astype(np.int64) for a in ("x", "y", "z"))
    cnt = np.zeros((nx + 1) * (ny + 1) * (nz + 1), dtype=np.int64)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                np.add.at(cnt, (i + dx) + NX * ((j + dy) + NY * (k + dz)), 1)
    return cnt


@pytest.mark.parametrize("case", ["sphere16", "ragged", "crater"])
def test_edges_4_and_8_push_alike(case):
    sims = []
    E = None
    for edge in (4, 8):
        gpu, orc = make_pair(case, dt=0.2, precision=MIXED)
        gpu.set_bin_edge(edge)
        if E is None:
            E = wl.random_node_field(orc.mesh.nnodes, 3, scale=0.7)
        for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 25.0))):
            add_species_both(gpu, orc, q, m, 0.01)
            explicit_particles(gpu, orc, s, 30000, 300 + s, 2.0 / (1 + 4 * s))
        gpu.set_external_E(E)
        sims.append((gpu, gpu.step(1)))
    (g4, st4), (g8, st8) = sims
    for key in ("pushed", "absorbed", "collected"):
        assert list(st4[key]) == list(st8[key]), key
    for s in range(2):
        a, b = by_id(g4.particles(s)), by_id(g8.particles(s))
        assert np.array_equal(a["id"], b["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.array_equal(a[k], b[k]), k
        W4, W8 = g4.node_charge(s), g8.node_charge(s)
        assert W4.sum() == W8.sum() == 2 ** 32 * len(a["id"])
        bound = (1 << 15) * _touch_counts(g4.n, a)
        assert np.all(np.abs(W4.astype(np.float64) - W8.astype(np.float64)) <= bound)
        assert np.array_equal(g4.surface_counts(s), g8.surface_counts(s))
    g4.close()
    g8.close()


def test_edge8_pic_steps_track_oracle():
    from paper_2011_10214_gb300 import capi
    from oracle.geometry import Mesh, Sphere
    from oracle.pic import Simulation as OracleSim
    cfg = wl.SPHERE16
    gpu = capi.from_config(cfg, precision=MIXED, track_ids=True, pcg_tol=1e-12, pcg_max_iter=5000, bin_edge=8)
    assert gpu.bin_edge == 8
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    orc = OracleSim(m, Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"]), cfg["face_bc"], cfg["dt"],
                    tol=1e-12, maxit=5000)
    for s, sp in enumerate(cfg["species"]):
        orc.add_species(sp["q"], sp["m"], wl.macro_weight(cfg, sp))
        orc.load_maxwellian(s, sp["ppc"], sp["vth"], sp["drift"], cfg["seed"])
        orc.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
    gpu.solve(); orc.solve()
    gpu.leapfrog_init(); orc.leapfrog_init()
    for _ in range(5):
        sg, so = gpu.step(1), orc.step()
        assert sg["pcg_converged"] == 1
        for s in range(2):
            assert sg["injected"][s] == so["injected"][s]
        rel = np.abs(gpu.potential() - orc.phi).max() / np.abs(orc.phi).max()
        assert rel <= TOL32, rel
    gpu.close()


def test_batch_with_both_edges_equals_alone():
    import torch
    from paper_2011_10214_gb300 import capi, serve
    rng = np.random.default_rng(88)
    cfgs = serve.request_distribution(rng, 4, big_fraction=0.0)
    edges = [4, 8, 8, 4]
    stream = torch.cuda.Stream()

    def fresh(c, e):
        s = capi.from_config(c, precision=MIXED, stream=stream.cuda_stream, bin_edge=e)
        s.solve(); s.leapfrog_init()
        return s
    alone = []
    for c, e in zip(cfgs, edges):   # each member in a batch of its own (the same clustered solver)
        s = fresh(c, e)
        b1 = capi.Batch([s], stream=stream.cuda_stream)
        b1.step(3)
        alone.append((s.potential(), s.node_charge(0), s.node_charge(1)))
        b1.close()
        s.close()
    sims = [fresh(c, e) for c, e in zip(cfgs, edges)]
    batch = capi.Batch(sims, stream=stream.cuda_stream)
    batch.step(3)
    for s, ref in zip(sims, alone):
        for a, b in zip((s.potential(), s.node_charge(0), s.node_charge(1)), ref):
            assert np.array_equal(a, b)
    batch.close()
    for s in sims:
        s.close()


def test_bin_edge_is_validated():
    from paper_2011_10214_gb300 import capi
    gpu, orc = make_pair("sphere16", precision=MIXED)
    for bad in (2, 6, 16, 0, -8):
        with pytest.raises(capi.PifepicError, match="EINVAL"):
            gpu.set_bin_edge(bad)
    gpu.set_bin_edge(8)
    gpu.set_bin_edge(4)
    gpu.set_bin_edge(8)
    add_species_both(gpu, orc, -1.0, 1.0, 0.01)
    with pytest.raises(capi.PifepicError, match="ESTATE"):
        gpu.set_bin_edge(4)
    assert gpu.bin_edge == 8
    gpu.close()
    g64, _ = make_pair("sphere16", precision=0)
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        g64.set_bin_edge(8)
    g64.set_bin_edge(4)
    g64.close()
