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
