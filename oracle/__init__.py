"""Plain FP64 CPU oracle of the non-homogeneous IFE-PIC hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
execute anything in this package.  The CUDA library never links, imports or
calls it, and it shares no code with the CUDA path: the only module both sides
use is ``paper_2011_10214_gb300.workloads`` (seeded synthetic inputs, none of
the method's arithmetic).

Every function states the passage of arXiv:2011.10214 (PIFE-PIC) it follows.
The paper defers the IFE formulation, pusher, weighting, injection and the
preconditioner to other work; where it is silent this package takes one stated
reading, listed in the module docstrings.

Modules
-------
geometry   mesh, 5-tet split of each cube, analytic level sets, linear IFE
           local spaces on interface tetrahedra (Sec. 2.1, Eqs. 2.1-2.5)
field      assembly, right-hand side with the flux-jump term, Jacobi PCG,
           node electric field (Sec. 2.1 "field-solve"; Sec. 2.5 PCG level)
rng        Philox4x64-10 counter-based generator (published definition)
particles  load, injection, leapfrog push, boundary and object hits,
           fixed-point charge deposit (Sec. 2.1 PIC loop; Sec. 3.1.3)
pic        the PIC loop: scatter, field-solve, gather, particle-push (Fig. 1)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the load/injection velocity samplers, whose
pins are statistical (moments and Kolmogorov-Smirnov tests against the
Maxwellian and flux-weighted distributions).
"""
