"""Mesh and solver limits are refused on the host, before any device call
(pifepic_create returns EINVAL): index packing allows 2047 cells along x and
y and 1023 along z (IFE mesh, after refinement), refinement is 1, 2, 4 or 8,
sizes, h and dt must be positive, the precision one of the two modes."""
import pytest


def _create(n, h=0.5, dt=0.05, precision=0, refine=1):
    from paper_2011_10214_gb300 import capi
    return capi.Simulation(n, h, dt, precision=precision, ife_refine=refine)


@pytest.mark.parametrize("kw", [
    dict(n=(2048, 4, 4)), dict(n=(4, 2048, 4)), dict(n=(4, 4, 1024)),
    dict(n=(1024, 4, 4), refine=2), dict(n=(4, 4, 512), refine=2), dict(n=(4, 4, 4), refine=3),
    dict(n=(0, 4, 4)), dict(n=(4, -1, 4)), dict(n=(4, 4, 4), h=0.0), dict(n=(4, 4, 4), h=float("nan")),
    dict(n=(4, 4, 4), dt=0.0), dict(n=(4, 4, 4), dt=-1.0), dict(n=(4, 4, 4), precision=2),
])
def test_bad_mesh_or_solver_is_refused(kw):
    from paper_2011_10214_gb300 import capi
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        _create(**kw)
