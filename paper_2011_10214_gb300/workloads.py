"""Workload descriptions and seeded synthetic inputs.

This module holds none of the method's arithmetic: it only names the
problem set-ups (mesh, object, species, time step, boundary conditions) of
arXiv:2011.10214's experiments as scaled for one GPU, and draws seeded random
inputs (particle states, node fields) for parity tests.  Both the CUDA path's
tests and the CPU oracle's tests read it; nothing else is shared.

Normalisation (a reading; the paper states none): lengths in Debye lengths,
time in 1/omega_pe, potential in kT_e/e, density in n_0, eps_0 = 1.  Electrons
q/m = -1; ions q = +1, m = mass ratio.  A macro-particle carries the charge of
density * h^3 / ppc.
"""
import numpy as np

SEED_BASE = 2011102140


def sphere_config(n, radius, ppc, steps, mass_ratio=100.0, h=0.5, eps_in=4.0, dt=0.05, seed_offset=1):
    """OML sheath of a dielectric sphere (Sec. 3, scaled): box of n^3 cells,
    sphere centred, phi = 0 on all faces, Maxwellian flux injection on all faces,
    absorbing faces, e- and H+ at equal temperature."""
    L = n * h
    vti = 1.0 / np.sqrt(mass_ratio)
    return dict(
        name=f"sphere{n}",
        n=(n, n, n), h=h, origin=(0.0, 0.0, 0.0), dt=dt, steps=steps,
        object=dict(kind="sphere", center=(L / 2, L / 2, L / 2), radius=radius, eps_in=eps_in, eps_out=1.0),
        face_bc=[("D", 0.0)] * 6,
        species=[dict(name="e-", q=-1.0, m=1.0, vth=1.0, ppc=ppc, density=1.0, drift=(0.0, 0.0, 0.0)),
                 dict(name="H+", q=1.0, m=mass_ratio, vth=vti, ppc=ppc, density=1.0, drift=(0.0, 0.0, 0.0))],
        inject_faces=0b111111,
        seed=SEED_BASE + seed_offset,
    )


# 16^3 cells of 0.5 Debye length, R = 2, eps 4 inside, 16 ppc per species,
# dt = 0.05, 100 steps, plain FP64
SPHERE16 = sphere_config(16, 2.0, 16, 100, seed_offset=1)
# 64^3 cells (1.3M tets), R = 6, 64 ppc per species (~34M particles), 1000 steps
SPHERE64 = sphere_config(64, 6.0, 64, 1000, seed_offset=2)


def oml_eighth_config(n=50, h=0.1, radius=0.401, ppc=125, steps=1000, mass_ratio=1836.0, eps_in=4.0, dt=0.01,
                      seed_offset=4):
    """The paper's validation geometry (Sec. 3, the OML sheath of a dielectric
    sphere): a box of n^3 cells of h Debye lengths with the sphere centred at
    the origin, so only its positive octant lies in the domain; zero Neumann
    field faces and reflecting particle faces at X/Y/Z_min (the symmetry
    planes), phi = 0 and injecting, absorbing faces at X/Y/Z_max; e- and ions of
    the realistic mass ratio at equal temperature, ppc per species."""
    vti = 1.0 / np.sqrt(mass_ratio)
    return dict(
        name=f"oml{n}",
        n=(n, n, n), h=h, origin=(0.0, 0.0, 0.0), dt=dt, steps=steps,
        object=dict(kind="sphere", center=(0.0, 0.0, 0.0), radius=radius, eps_in=eps_in, eps_out=1.0),
        face_bc=[("N",), ("D", 0.0)] * 3,
        particle_bc=["reflect", "inject"] * 3,
        species=[dict(name="e-", q=-1.0, m=1.0, vth=1.0, ppc=ppc, density=1.0, drift=(0.0, 0.0, 0.0)),
                 dict(name="H+", q=1.0, m=mass_ratio, vth=vti, ppc=ppc, density=1.0, drift=(0.0, 0.0, 0.0))],
        inject_faces=0b101010,
        seed=SEED_BASE + seed_offset,
    )


# 50^3 cells of 0.1 Debye length (5 Debye lengths a side), 1/8 of a sphere of
# radius 0.401, eps 4, m_i/m_e = 1836, dt = 0.01, 125 ppc per species (~31M)
OML50 = oml_eighth_config()


def crater_config(nx=160, ny=160, nz=80, z_ground=20.0, rim_radius=30.0, depth=10.0, ppc=125, steps=200,
                  mass_ratio=100.0, dt=0.05, seed_offset=3):
    """Crater charging (Sec. 5, scaled to one GPU): cells of one photoelectron
    Debye length; dielectric ground (eps 4) at z_ground with a spherical-cap
    crater of the given rim radius and depth centred in x, y; phi = 0 at Z_max,
    zero Neumann on the other faces; drifting solar-wind electrons and ions
    (T_e : T_i : T_ph = 6 : 5 : 1, density 8.7/64 of the photoelectron
    reference, drift 8 ion thermal speeds at 45 degrees towards the ground in
    the X-Z plane) loaded at ppc per species in the plasma and injected on every
    face but Z_min; photoelectrons (vth 1, reference density 1) emitted from the
    sunlit, unshadowed surface, the sun opposite to the flow.  The photoelectron
    macro-particle carries the solar-wind electrons' charge."""
    n_sw = 8.7 / 64.0
    vte, vti = np.sqrt(6.0), np.sqrt(5.0 / mass_ratio)
    vd = 8.0 * vti
    c45 = np.sqrt(0.5)
    drift = (vd * c45, 0.0, -vd * c45)
    return dict(
        name=f"crater{nx}",
        n=(nx, ny, nz), h=1.0, origin=(0.0, 0.0, 0.0), dt=dt, steps=steps,
        object=dict(kind="cap_crater", z_ground=z_ground, xc=nx / 2, yc=ny / 2, rim_radius=rim_radius,
                    depth=depth, eps_in=4.0, eps_out=1.0),
        face_bc=[("N",)] * 5 + [("D", 0.0)],
        species=[dict(name="sw e-", q=-1.0, m=1.0, vth=vte, ppc=ppc, density=n_sw, drift=drift),
                 dict(name="sw H+", q=1.0, m=mass_ratio, vth=vti, ppc=ppc, density=n_sw, drift=drift)],
        photo=dict(name="photo e-", q=-1.0, m=1.0, vth=1.0, density=1.0, weight=n_sw / ppc,
                   sun=(-c45, 0.0, c45)),
        inject_faces=0b101111,
        seed=SEED_BASE + seed_offset,
    )


# 160 x 160 x 80 cells (~10M tets), crater of rim radius 30 and depth 10 in a
# ground at z = 20, 125 ppc per solar-wind species in the plasma (~384M), 200 steps
CRATER160 = crater_config()


def lunar_config(nx=200, ny=100, nz=100, z_ground=9.5, z_bed=4.5, r_inner=10.5, r_top=20.2, r_outer=30.9,
                 height=2.7, depth=4.0, ppc=125, steps=200, mass_ratio=100.0, dt=0.05, angle_deg=10.0,
                 seed_offset=8):
    """The lunar crater charging run of Sec. 5.2 on one GPU: cells of one
    photoelectron Debye length; a half crater (centred on the Y_min face, the
    symmetry plane, which reflects particles) with inner-rim, top-rim and
    outer-rim radii 10.5, 20.2, 30.9 cells in a regolith ground (eps 4) at
    z = 9.5 over bedrock (eps 10) below z = 4.5; the rim profile's height and
    depth (2.7 + 4.0 = the quoted 6.7 cells of relief) are this reading's;
    phi = 0 at Z_max, zero Neumann elsewhere; solar-wind e- and ions
    (T_e : T_i : T_ph = 6 : 5 : 1, density 8.7/64 of the photoelectron
    reference, drift 8 ion thermal speeds at 10 degrees towards the ground in
    the X-Z plane) loaded at ppc per species and injected at X_min, X_max,
    Y_max and Z_max; photoelectrons from the sunlit, unshadowed surface, the
    sun 10 degrees above the ground opposite to the flow."""
    n_sw = 8.7 / 64.0
    vte, vti = np.sqrt(6.0), np.sqrt(5.0 / mass_ratio)
    vd = 8.0 * vti
    a = np.radians(angle_deg)
    drift = (vd * np.cos(a), 0.0, -vd * np.sin(a))
    return dict(
        name=f"lunar{nx}",
        n=(nx, ny, nz), h=1.0, origin=(0.0, 0.0, 0.0), dt=dt, steps=steps,
        object=dict(kind="rim_crater", z_ground=z_ground, xc=nx / 2, yc=0.0, r_inner=r_inner, r_top=r_top,
                    r_outer=r_outer, height=height, depth=depth, eps_in=4.0, eps_out=1.0,
                    bedrock=(z_bed, 10.0)),
        face_bc=[("N",)] * 5 + [("D", 0.0)],
        particle_bc=["inject", "inject", "reflect", "inject", "absorb", "inject"],
        species=[dict(name="sw e-", q=-1.0, m=1.0, vth=vte, ppc=ppc, density=n_sw, drift=drift),
                 dict(name="sw H+", q=1.0, m=mass_ratio, vth=vti, ppc=ppc, density=n_sw, drift=drift)],
        photo=dict(name="photo e-", q=-1.0, m=1.0, vth=1.0, density=1.0, weight=n_sw / ppc,
                   sun=(-np.cos(a), 0.0, np.sin(a))),
        inject_faces=0b101011,
        seed=SEED_BASE + seed_offset,
    )


# 200 x 100 x 100 cells (10M tets) as in Sec. 5.2, 125 ppc per solar-wind species
LUNAR200 = lunar_config()


def macro_weight(cfg, sp):
    return sp["density"] * cfg["h"] ** 3 / sp["ppc"]


def random_particles(n_cells, count, seed, vth=1.0, margin=0.0):
    """Seeded uniform positions (cell units) inside the box and normal velocities."""
    g = np.random.default_rng(seed)
    nx, ny, nz = n_cells
    x = g.uniform(margin, nx - margin, count)
    y = g.uniform(margin, ny - margin, count)
    z = g.uniform(margin, nz - margin, count)
    v = g.normal(0.0, vth, (3, count))
    return x, y, z, v[0], v[1], v[2]


def random_node_field(n_nodes, seed, scale=1.0):
    """Seeded node field (n_nodes, 3) for frozen-field parity runs."""
    g = np.random.default_rng(seed)
    return g.normal(0.0, scale, (n_nodes, 3))
