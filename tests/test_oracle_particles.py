"""Pins of oracle.particles and oracle.pic: orbits, gather, deposit, conservation,
and the statistics of the load and injection samplers."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import particles as pt
from oracle.geometry import Mesh, NoObject, Sphere
from oracle.pic import Simulation
from paper_2011_10214_gb300 import workloads as wl


def _P(x, y, z, vx, vy, vz):
    return dict(x=np.array(x, float), y=np.array(y, float), z=np.array(z, float),
                vx=np.array(vx, float), vy=np.array(vy, float), vz=np.array(vz, float))


def test_uniform_field_orbit_closed_form():
    """P5: in a uniform E, leapfrog gives v_n = v_{-1/2} + n k E and
    xi_n = xi_0 + dth (n v_{-1/2} + k E n(n+1)/2) (constant acceleration)."""
    m = Mesh(40, 40, 40, 0.5)
    E = np.tile(np.array([0.3, -0.2, 0.1]), (m.nnodes, 1))
    x0, y0, z0, v0 = 20.3, 19.7, 20.1, np.array([0.05, -0.02, 0.01])
    P = _P([x0], [y0], [z0], [v0[0]], [v0[1]], [v0[2]])
    k, dth = -0.05, 0.1
    for n in range(1, 41):
        pt.push(m, E, P, k, dth)
        vn = v0 + n * k * E[0]
        xn = np.array([x0, y0, z0]) + dth * (n * v0 + k * E[0] * n * (n + 1) / 2)
        assert np.allclose([P["vx"][0], P["vy"][0], P["vz"][0]], vn, rtol=0, atol=1e-13)
        assert np.allclose([P["x"][0], P["y"][0], P["z"][0]], xn, rtol=0, atol=1e-12)


def test_zero_field_straight_line_and_gather_linear():
    m = Mesh(8, 8, 8, 0.25)
    P = _P([1.5], [2.25], [3.75], [0.2], [0.1], [-0.3])
    for _ in range(10):
        pt.push(m, np.zeros((m.nnodes, 3)), P, 1.0, 0.5)
    assert P["x"][0] == pytest.approx(1.5 + 10 * 0.1) and P["z"][0] == pytest.approx(3.75 - 10 * 0.15)
    i, j, k = m.node_ijk()
    E = np.stack([1 + 0.5 * i, 2 - 0.25 * j + 0.1 * k, 0.3 * i - 0.2 * k], axis=1).astype(float)
    g = np.random.default_rng(1)
    x, y, z = g.uniform(0, 8, (3, 100))
    ex, ey, ez = pt.gather(m, E, x, y, z)          # trilinear reproduces trilinear data
    assert np.allclose(ex, 1 + 0.5 * x) and np.allclose(ey, 2 - 0.25 * y + 0.1 * z)
    assert np.allclose(ez, 0.3 * x - 0.2 * z)


def test_deposit_brute_force_and_exact_total():
    """Per-particle Python loop (int arithmetic) equals the vectorised deposit;
    every particle deposits exactly 2^32 units; a particle on a node puts all
    its weight there."""
    m = Mesh(5, 4, 3, 1.0)
    g = np.random.default_rng(4)
    x, y, z = g.uniform(0, 5, 300), g.uniform(0, 4, 300), g.uniform(0, 3, 300)
    x[0], y[0], z[0] = 2.0, 1.0, 1.0
    W = pt.deposit(m, x, y, z)
    ref = [0] * m.nnodes
    for p in range(len(x)):
        ci, cj, ck = int(math.floor(x[p])), int(math.floor(y[p])), int(math.floor(z[p]))
        fx, fy, fz = x[p] - ci, y[p] - cj, z[p] - ck
        ws = []
        for l in range(8):
            a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
            wl_ = ((fx if a else 1.0 - fx) * (fy if b else 1.0 - fy)) * (fz if c else 1.0 - fz)
            ws.append(int(round(wl_ * 2.0 ** 32)) if l < 7 else None)
        ws[7] = 2 ** 32 - sum(ws[:7])
        for l in range(8):
            a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
            ref[m.node(ci + a, cj + b, ck + c)] += ws[l]
    assert W.tolist() == ref
    assert W.sum() == 2 ** 32 * len(x)
    W0 = pt.deposit(m, x[:1], y[:1], z[:1])
    assert W0[m.node(2, 1, 1)] == 2 ** 32 and W0.sum() == 2 ** 32


def test_deposit_ties_round_to_even():
    m = Mesh(2, 2, 2, 1.0)
    # fx = 0.5 exactly -> weights 1/2 and 1/8 multiples; 2^32 * w are integers, no tie issue;
    # a weight of (2k+1)/2^33 is a tie: rint rounds to even
    x = np.array([0.5 + 2.0 ** -33]); y = np.array([0.0]); z = np.array([0.0])
    W = pt.deposit(m, x, y, z)
    w1 = x[0] * 2.0 ** 32
    assert W[m.node(1, 0, 0)] == int(np.rint(w1)) and W.sum() == 2 ** 32


def _small_sim(with_injection=True, steps=6):
    cfg = wl.sphere_config(8, 1.0, 4, steps)
    m = Mesh(*cfg["n"], cfg["h"])
    ob = cfg["object"]
    sim = Simulation(m, Sphere(m, ob["center"], ob["radius"], ob["eps_in"], ob["eps_out"]),
                     cfg["face_bc"], cfg["dt"], tol=1e-10, maxit=500)
    for s, sp in enumerate(cfg["species"]):
        sim.add_species(sp["q"], sp["m"], wl.macro_weight(cfg, sp))
        sim.load_maxwellian(s, sp["ppc"], sp["vth"], sp["drift"], cfg["seed"])
        if with_injection:
            sim.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
    return sim


def test_pic_conservation_counts_and_charge():
    """P6: N(t) = N_load + N_inj - N_absorbed - N_collected exactly; node sums
    equal 2^32 N; surface accumulators total the collected particles."""
    sim = _small_sim()
    n0 = sim.counts()
    sim.solve()
    sim.leapfrog_init()
    tot = dict(inj=[0, 0], ab=[0, 0], co=[0, 0], lost=[0, 0])
    for _ in range(6):
        st = sim.step()
        for s in range(2):
            tot["inj"][s] += st["injected"][s]; tot["ab"][s] += st["absorbed"][s]
            tot["co"][s] += st["collected"][s]; tot["lost"][s] += st["lost"][s]
    n = sim.counts()
    for s in range(2):
        assert n[s] == n0[s] + tot["inj"][s] - tot["ab"][s] - tot["co"][s]
        assert sim.W[s].sum() == 2 ** 32 * n[s]
        assert sim.surf[:, s].sum() + tot["lost"][s] == tot["co"][s]
        ids = sim.P[s]["id"]
        assert len(np.unique(ids)) == len(ids)
    assert sum(tot["co"]) > 0 and sum(tot["inj"]) > 0
    # every particle stays inside the box and outside the object
    for P in sim.P:
        assert not pt.outside(sim.mesh, P["x"], P["y"], P["z"]).any()
        assert (sim.obj.L(P["x"], P["y"], P["z"]) >= 0).all()


def test_flux_normal_speed_distribution():
    """Rejection sampler vs the exact CDF of v exp(-(v-s)^2/2), v > 0 (KS test)."""
    g = np.random.default_rng(9)
    for s in (0.0, 1.5, -1.0, 5.66):
        n = 40000
        U = [tuple(g.uniform(size=n) for _ in range(3)) for _ in range(pt.MAX_TRIES)]
        v, ok = pt.flux_normal_speed(U, s)
        assert ok.mean() > 0.999
        pdf = lambda t: t * np.exp(-0.5 * (t - s) ** 2)
        Z = integrate.quad(pdf, 0, np.inf)[0]
        grid = np.linspace(0, s + 12, 4001)
        cdf = np.concatenate([[0], np.cumsum([integrate.quad(pdf, a, b)[0] for a, b in zip(grid[:-1], grid[1:])])]) / Z
        res = stats.kstest(v[ok], lambda t: np.interp(t, grid, cdf))
        assert res.pvalue > 1e-3


def test_flux_density_matches_integral():
    for s in (0.0, 0.7, -1.2, 5.0):
        num = integrate.quad(lambda v: v * np.exp(-0.5 * (v - s) ** 2) / np.sqrt(2 * np.pi), 0, np.inf)[0]
        assert pt.flux_density(1.0, 1.0, s) == pytest.approx(num, rel=1e-10)
    assert pt.flux_density(2.0, 0.5, 0.0) == pytest.approx(2.0 * 0.5 / np.sqrt(2 * np.pi), rel=1e-14)


def test_load_and_inject_statistics():
    m = Mesh(10, 10, 10, 0.5)
    P = pt.load_maxwellian(m, NoObject(), 77, 0, 50, 0.3, (0.1, 0.0, -0.2))
    assert len(P["x"]) == 50000
    for c, d in zip(("vx", "vy", "vz"), (0.1, 0.0, -0.2)):
        assert abs(P[c].mean() - d) < 0.01 and abs(P[c].std() - 0.3) < 0.01
    assert stats.kstest(P["x"] - np.floor(P["x"]), "uniform").pvalue > 1e-3
    I = pt.inject_face(m, NoObject(), 5, 1, 3, 12, 20000, 1.0, (0.0, 0.0, 0.0), 0.1)
    assert I["accepted"].all()
    assert np.all(I["y0"] == 10.0) and np.all(I["vy"] < 0)                 # y+ face, inward = -y
    # flux-weighted normal speed for no drift: Rayleigh, CDF 1 - exp(-v^2/2)
    assert stats.kstest(-I["vy"], lambda v: 1 - np.exp(-0.5 * v * v)).pvalue > 1e-3
    assert abs(I["vx"].std() - 1.0) < 0.03 and abs(I["vz"].mean()) < 0.03
    assert np.allclose(I["y"], I["y0"] + I["vy"] * (I["y"] - I["y0"]) / I["vy"])
    frac = (I["y"] - I["y0"]) / (I["vy"] * 0.1)
    assert frac.min() > 0 and frac.max() < 1 and stats.kstest(frac, "uniform").pvalue > 1e-3
