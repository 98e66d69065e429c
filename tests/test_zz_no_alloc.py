"""pifepic_solve_field_noalloc: the field solve for callers that cannot allocate
device memory while running (serving loops whose device memory comes from a
pool they do not own, hosts that forbid allocation after start-up).  Its PCG
work vectors live in a fixed device array of the library; it must give the same
potential as pifepic_solve_field, on two calls in a row (the shared scratch
keeps the previous call's contents and must not leak into the next result).

Covered: an FP64 context, a MIXED context (the no-alloc solve runs the plain
FP64 PCG there, the allocating one the FP32 PCG inside FP64 refinement), a
hybrid grid (IFE mesh twice as fine as the PIC mesh) and a NULL flux jump on a
mesh with an object.

Collected last on purpose: a failure here comes after every other test ran."""
import numpy as np
import pytest

from tests.pairs import make_pair

pytestmark = pytest.mark.gpu

TOL_PHI = 1e-8    # the FP64 potential bar used by the other solver parity tests


@pytest.mark.parametrize("case,precision", [("sphere16", 0), ("sphere16", 1), ("sphere_h2", 0)])
def test_noalloc_solve_matches_allocating_solve_twice(case, precision):
    import torch
    gpu, orc = make_pair(case, precision=precision)
    nn = gpu.sizes()["nnodes"]
    nit = gpu.sizes()["n_interface_tets"]
    assert nit > 0
    g = np.random.default_rng(21)
    for call in range(2):
        F = g.normal(size=nn) * orc.fmesh.h ** 3
        q = g.normal(size=nit)
        gpu.solve_field(F, q)
        ref = gpu.potential()
        Fd = torch.tensor(F, dtype=torch.float64, device="cuda")
        qd = torch.tensor(q, dtype=torch.float64, device="cuda")
        phi = torch.full((nn,), float("nan"), dtype=torch.float64, device="cuda")
        it, rr = gpu.solve_field_noalloc(Fd, qd, phi)
        out = phi.cpu().numpy()
        assert rr <= 1e-12 and it > 0, call
        assert np.abs(out - ref).max() <= TOL_PHI * np.abs(ref).max(), call
        assert np.array_equal(gpu.potential(), ref)          # context state untouched
    gpu.close()


def test_noalloc_null_flux_jump_is_zero_jump():
    import torch
    gpu, orc = make_pair("sphere16")
    nn = gpu.sizes()["nnodes"]
    assert gpu.sizes()["n_interface_tets"] > 0
    F = np.random.default_rng(5).normal(size=nn) * orc.mesh.h ** 3
    gpu.solve_field(F, None)
    ref = gpu.potential()
    phi = torch.full((nn,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        it, rr = gpu.solve_field_noalloc(torch.tensor(F, dtype=torch.float64, device="cuda"), None, phi)
        assert rr <= 1e-12 and it > 0, call
        assert np.abs(phi.cpu().numpy() - ref).max() <= TOL_PHI * np.abs(ref).max(), call
    gpu.close()


def test_noalloc_rejects_meshes_beyond_the_scratch():
    import torch
    from paper_2011_10214_gb300 import capi
    sim = capi.Simulation((64, 64, 32), 0.5, 0.05)           # 65*65*33 = 139425 nodes > 131072
    sim.set_object(capi.OBJ_NONE, [], 1.0, 1.0)
    n = sim.sizes()["nnodes"]
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.PifepicError, match="EINVAL"):
        sim.solve_field_noalloc(z, None, z.clone())
    sim.close()
