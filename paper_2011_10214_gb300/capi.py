"""Python binding of libpifepic (include/pifepic.h): argument marshalling only.

Every step of the particle cycle and the field solve runs in the library's
CUDA kernels.  Importing this module loads the in-tree ``_build/libpifepic.so``
and raises ImportError if it is missing -- there is no CPU fallback.  Build it
with ``python -m paper_2011_10214_gb300.build`` or ``__graft_entry__.build()``.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpifepic.so")

FP64, MIXED = 0, 1
HOST, DEVICE = 0, 1
OBJ_NONE, OBJ_SPHERE, OBJ_CAP_CRATER, OBJ_PLANE, OBJ_RIM_CRATER = 0, 1, 2, 3, 4
SOLVER_REGISTERS, SOLVER_GLOBAL, SOLVER_MULTIGRID = 1, 2, 3
BC_DIRICHLET, BC_NEUMANN = 0, 1
PBC_ABSORB, PBC_INJECT, PBC_REFLECT = 0, 1, 2
PRECOND_AUTO, PRECOND_JACOBI, PRECOND_MULTIGRID = 0, 1, 2
_PBC_NAMES = {"absorb": PBC_ABSORB, "inject": PBC_INJECT, "reflect": PBC_REFLECT}
MAX_SPECIES = 8
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ESTATE", 4: "ECUDA", 5: "ETIMEOUT", 6: "ENOTCONV"}


class MeshDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double), ("origin", C.c_double * 3),
                ("ife_refine", C.c_int)]


class SolverDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("precision", C.c_int), ("pcg_tol", C.c_double), ("pcg_max_iter", C.c_int),
                ("track_ids", C.c_int)]


class ObjectDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.c_double * 8), ("eps_in", C.c_double), ("eps_out", C.c_double)]


class FaceBC(C.Structure):
    _fields_ = [("kind", C.c_int), ("value", C.c_double)]


_I64S = C.c_int64 * MAX_SPECIES


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("pushed", _I64S), ("count", _I64S), ("injected", _I64S),
                ("absorbed", _I64S), ("collected", _I64S), ("lost_charge", _I64S), ("inj_rejected", _I64S),
                ("spilled", _I64S), ("dropped", _I64S), ("pcg_iters_total", C.c_int64),
                ("kernel_launches", C.c_int64), ("pcg_iters", C.c_int), ("pcg_converged", C.c_int),
                ("pcg_relres", C.c_double), ("surface_charge", C.c_double), ("surface_potential", C.c_double),
                ("phase_ms", C.c_double * 8), ("pcg_outer_total", C.c_int64)]

    def as_dict(self, nspecies):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if isinstance(v, C.Array):
                v = list(v)[:nspecies] if name != "phase_ms" else list(v)
            d[name] = v
        return d


PHASES = ("push", "movers", "inject", "rebin", "rhs", "solve", "node_E", "other")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpifepic.so not built ({LIB_PATH}); run __graft_entry__.build()")
lib = C.CDLL(LIB_PATH)

_ctx = C.c_void_p
_dp = C.c_void_p          # any pointer (host or device) passed as an address
_sigs = {
    "pifepic_create": [C.POINTER(MeshDesc), C.POINTER(SolverDesc), C.c_void_p, C.POINTER(_ctx)],
    "pifepic_set_object": [_ctx, C.POINTER(ObjectDesc)],
    "pifepic_set_field_bc": [_ctx, FaceBC * 6],
    "pifepic_add_species": [_ctx, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int)],
    "pifepic_load_maxwellian": [_ctx, C.c_int, C.c_int, C.c_double, C.c_double * 3, C.c_uint64],
    "pifepic_load_particles": [_ctx, C.c_int, C.c_size_t] + [_dp] * 7 + [C.c_int],
    "pifepic_set_injection": [_ctx, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double * 3, C.c_uint64],
    "pifepic_get_injection_rate": [_ctx, C.c_int, C.c_double * 6],
    "pifepic_set_photoemission": [_ctx, C.c_int, C.c_double * 3, C.c_double, C.c_double, C.c_uint64],
    "pifepic_set_particle_bc": [_ctx, C.c_int, C.c_int * 6],
    "pifepic_set_bedrock": [_ctx, C.c_double, C.c_double],
    "pifepic_set_refinement": [_ctx, C.c_double, C.c_double],
    "pifepic_get_photoemission": [_ctx, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "pifepic_set_external_E": [_ctx, _dp, C.c_int],
    "pifepic_solve": [_ctx, C.POINTER(Stats)],
    "pifepic_leapfrog_init": [_ctx],
    "pifepic_step": [_ctx, C.c_int, C.POINTER(Stats)],
    "pifepic_get_sizes": [_ctx] + [C.POINTER(C.c_int64)] * 4,
    "pifepic_get_potential": [_ctx, _dp, C.c_int],
    "pifepic_get_node_E": [_ctx, _dp, C.c_int],
    "pifepic_get_node_E_f32": [_ctx, _dp, C.c_int],
    "pifepic_get_node_charge": [_ctx, C.c_int, _dp, C.c_int],
    "pifepic_get_surface_charge": [_ctx, C.c_int, _dp, C.c_int],
    "pifepic_get_cut_cells": [_ctx, _dp, _dp],
    "pifepic_get_cell_target": [_ctx, _dp],
    "pifepic_get_interface": [_ctx] + [_dp] * 7,
    "pifepic_get_particle_count": [_ctx, C.c_int, C.POINTER(C.c_int64)],
    "pifepic_get_particles": [_ctx, C.c_int, C.c_int64] + [_dp] * 7 + [C.POINTER(C.c_int64), C.c_int],
    "pifepic_get_stats": [_ctx, C.POINTER(Stats)],
    "pifepic_solve_field": [_ctx, _dp, _dp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "pifepic_solve_field_noalloc": [_ctx, _dp, _dp, _dp, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "pifepic_set_preconditioner": [_ctx, C.c_int],
    "pifepic_set_bin_edge": [_ctx, C.c_int],
    "pifepic_get_bin_edge": [_ctx],
    "pifepic_get_solver": [_ctx],
    "pifepic_get_memory_use": [C.POINTER(C.c_size_t)],
    "pifepic_set_memory_limit": [C.c_size_t],
    "pifepic_test_hold_exchange": [_ctx, C.c_int],
    "pifepic_batch_create": [C.POINTER(_ctx), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)],
    "pifepic_batch_add": [C.c_void_p, _ctx],
    "pifepic_batch_remove": [C.c_void_p, _ctx],
    "pifepic_batch_set_cta_nodes": [C.c_void_p, C.c_int],
    "pifepic_batch_step": [C.c_void_p, C.c_int, C.c_void_p],
    "pifepic_batch_set_preconditioner": [C.c_void_p, C.c_int],
}
for _n, _a in _sigs.items():
    _f = getattr(lib, _n)
    _f.argtypes = _a
    _f.restype = C.c_int
lib.pifepic_destroy.argtypes = [_ctx]
lib.pifepic_destroy.restype = None
lib.pifepic_last_error.argtypes = [_ctx]
lib.pifepic_last_error.restype = C.c_char_p
lib.pifepic_batch_destroy.argtypes = [C.c_void_p]
lib.pifepic_batch_destroy.restype = None
lib.pifepic_batch_last_error.argtypes = [C.c_void_p]
lib.pifepic_batch_last_error.restype = C.c_char_p
LOG_FN = C.CFUNCTYPE(None, C.c_char_p, C.c_void_p)
lib.pifepic_set_log_callback.argtypes = [LOG_FN, C.c_void_p]
lib.pifepic_set_log_callback.restype = None

EXPORTED = sorted(list(_sigs) + ["pifepic_destroy", "pifepic_last_error", "pifepic_batch_destroy",
                                 "pifepic_batch_last_error", "pifepic_set_log_callback"])

_log_keep = None   # the ctypes callback object must outlive its registration


def set_log_callback(fn):
    """Pass every error message the library records to fn(message: str)
    (pifepic_set_log_callback); None turns it off."""
    global _log_keep
    if fn is None:
        lib.pifepic_set_log_callback(LOG_FN(), None)
        _log_keep = None
        return
    cb = LOG_FN(lambda msg, user: fn(msg.decode(errors="replace")))
    lib.pifepic_set_log_callback(cb, None)
    _log_keep = cb


class PifepicError(RuntimeError):
    pass


def memory_use():
    """Bytes of device memory the library holds, process-wide (pifepic_get_memory_use)."""
    v = C.c_size_t()
    st = lib.pifepic_get_memory_use(C.byref(v))
    if st != 0:
        raise PifepicError(f"get_memory_use: {STATUS.get(st, st)}")
    return int(v.value)


def set_memory_limit(nbytes):
    """Cap the library's device memory, process-wide (0 = no cap; pifepic_set_memory_limit)."""
    st = lib.pifepic_set_memory_limit(C.c_size_t(int(nbytes)))
    if st != 0:
        raise PifepicError(f"set_memory_limit: {STATUS.get(st, st)}")


def _addr(a):
    """Address of a numpy array (host) or a torch tensor (host or device); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_dev(a):
    return (not isinstance(a, np.ndarray)) and getattr(a, "is_cuda", False)


class Simulation:
    """One IFE-PIC instance (one context) on the current CUDA device."""

    def __init__(self, n, h, dt, origin=(0.0, 0.0, 0.0), precision=FP64, pcg_tol=1e-6, pcg_max_iter=150,
                 track_ids=False, stream=None, ife_refine=1):
        """n, h: the PIC mesh; ife_refine: the IFE mesh splits each PIC cell
        ife_refine^3 times (1, 2, 4 or 8; see pifepic_mesh_desc)."""
        md = MeshDesc(int(n[0]), int(n[1]), int(n[2]), float(h), (C.c_double * 3)(*origin), int(ife_refine))
        sd = SolverDesc(float(dt), int(precision), float(pcg_tol), int(pcg_max_iter), int(bool(track_ids)))
        self._c = _ctx()
        self.n = tuple(int(v) for v in n)
        self.refine = int(ife_refine)
        self.nspecies = 0
        self.track_ids = bool(track_ids)
        st = lib.pifepic_create(C.byref(md), C.byref(sd), C.c_void_p(stream or 0), C.byref(self._c))
        if st != 0:
            msg = lib.pifepic_last_error(self._c).decode() if self._c.value else ""
            if self._c.value:
                lib.pifepic_destroy(self._c)
            self._c = None
            raise PifepicError(f"pifepic_create: {STATUS.get(st, st)} {msg}")

    def _ok(self, st, what):
        if st != 0:
            raise PifepicError(f"{what}: {STATUS.get(st, st)}: {lib.pifepic_last_error(self._c).decode()}")

    def close(self):
        if self._c is not None and self._c.value:
            lib.pifepic_destroy(self._c)
        self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -------------------------------------------------------------------
    def set_object(self, kind, params, eps_in, eps_out):
        p = list(params) + [0.0] * (8 - len(params))
        od = ObjectDesc(int(kind), (C.c_double * 8)(*p), float(eps_in), float(eps_out))
        self._ok(lib.pifepic_set_object(self._c, C.byref(od)), "set_object")

    def set_bedrock(self, z_bed, eps_bed):
        """Bedrock of permittivity eps_bed below the plane z = z_bed inside the
        object (see pifepic_set_bedrock); call before set_object."""
        self._ok(lib.pifepic_set_bedrock(self._c, float(z_bed), float(eps_bed)), "set_bedrock")

    def set_refinement(self, reduction=1e-4, margin=0.5):
        """MIXED refinement controls (see pifepic_set_refinement): an FP32 inner
        solve stops at max(margin tol |b|, reduction |r0|)."""
        self._ok(lib.pifepic_set_refinement(self._c, float(reduction), float(margin)), "set_refinement")

    def set_preconditioner(self, kind):
        """MIXED inner PCG preconditioner: PRECOND_AUTO, PRECOND_JACOBI or PRECOND_MULTIGRID."""
        self._ok(lib.pifepic_set_preconditioner(self._c, int(kind)), "set_preconditioner")

    def set_bin_edge(self, edge):
        """Particle bins of edge^3 cells, 4 or 8 (pifepic_set_bin_edge; before add_species)."""
        self._ok(lib.pifepic_set_bin_edge(self._c, int(edge)), "set_bin_edge")

    @property
    def bin_edge(self):
        return int(lib.pifepic_get_bin_edge(self._c))

    @property
    def solver(self):
        """The persistent solver of the next solve: SOLVER_REGISTERS, SOLVER_GLOBAL or SOLVER_MULTIGRID."""
        return int(lib.pifepic_get_solver(self._c))

    def set_field_bc(self, faces):
        arr = (FaceBC * 6)()
        for f, bc in enumerate(faces):
            arr[f].kind = BC_DIRICHLET if bc[0] == "D" else BC_NEUMANN
            arr[f].value = float(bc[1]) if bc[0] == "D" else 0.0
        self._ok(lib.pifepic_set_field_bc(self._c, arr), "set_field_bc")

    def add_species(self, q, m, w):
        i = C.c_int()
        self._ok(lib.pifepic_add_species(self._c, float(q), float(m), float(w), C.byref(i)), "add_species")
        self.nspecies += 1
        return i.value

    def load_maxwellian(self, s, ppc, vth, drift, seed):
        self._ok(lib.pifepic_load_maxwellian(self._c, s, int(ppc), float(vth), (C.c_double * 3)(*drift),
                                             C.c_uint64(int(seed))), "load_maxwellian")

    def load_particles(self, s, x, y, z, vx, vy, vz, ids=None):
        dev = _is_dev(x)
        arrs = [x, y, z, vx, vy, vz]
        if not dev:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
            if ids is not None:
                ids = np.ascontiguousarray(ids, dtype=np.int64)
        self._keep = (arrs, ids)
        self._ok(lib.pifepic_load_particles(self._c, s, len(arrs[0]), *[_addr(a) for a in arrs], _addr(ids),
                                            DEVICE if dev else HOST), "load_particles")

    def set_injection(self, s, face_mask, density, vth, drift, seed):
        self._ok(lib.pifepic_set_injection(self._c, s, int(face_mask), float(density), float(vth),
                                           (C.c_double * 3)(*drift), C.c_uint64(int(seed))), "set_injection")

    def set_particle_bc(self, s, face_kinds):
        """Particle boundary of faces x-, x+, y-, y+, z-, z+ for species s: each
        "absorb", "inject" or "reflect" (or PBC_* codes); see pifepic_set_particle_bc."""
        k = [_PBC_NAMES[f] if isinstance(f, str) else int(f) for f in face_kinds]
        if len(k) != 6:
            raise ValueError("six face kinds expected")
        self._ok(lib.pifepic_set_particle_bc(self._c, int(s), (C.c_int * 6)(*k)), "set_particle_bc")

    def set_photoemission(self, s, sun_dir, density, vth, seed):
        """Species s is emitted from the sunlit, unshadowed object surface (see
        pifepic_set_photoemission)."""
        self._ok(lib.pifepic_set_photoemission(self._c, int(s), (C.c_double * 3)(*sun_dir), float(density),
                                               float(vth), int(seed)), "set_photoemission")

    def photoemission(self):
        """(sum of the fixed-point rates in 2^-20 particles per step, emitting tets)."""
        q, n = C.c_int64(), C.c_int64()
        self._ok(lib.pifepic_get_photoemission(self._c, C.byref(q), C.byref(n)), "get_photoemission")
        return q.value, n.value

    def injection_rate(self, s):
        r = (C.c_double * 6)()
        self._ok(lib.pifepic_get_injection_rate(self._c, s, r), "get_injection_rate")
        return list(r)

    def set_external_E(self, E):
        if E is None:
            self._ok(lib.pifepic_set_external_E(self._c, None, HOST), "set_external_E")
            return
        dev = _is_dev(E)
        if not dev:
            E = np.ascontiguousarray(E, dtype=np.float64)
        self._ok(lib.pifepic_set_external_E(self._c, _addr(E), DEVICE if dev else HOST), "set_external_E")

    # -- run ------------------------------------------------------------------------
    def solve(self):
        st = Stats()
        self._ok(lib.pifepic_solve(self._c, C.byref(st)), "solve")
        return st.as_dict(self.nspecies)

    def leapfrog_init(self):
        self._ok(lib.pifepic_leapfrog_init(self._c), "leapfrog_init")

    def step(self, nsteps=1, stats=True):
        st = Stats()
        self._ok(lib.pifepic_step(self._c, int(nsteps), C.byref(st)), "step")
        return st.as_dict(self.nspecies)

    def solve_field(self, F, q=None):
        it = C.c_int()
        rr = C.c_double()
        dev = _is_dev(F)
        if not dev:
            F = np.ascontiguousarray(F, dtype=np.float64)
            q = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
        self._ok(lib.pifepic_solve_field(self._c, _addr(F), _addr(q), DEVICE if dev else HOST, C.byref(it),
                                         C.byref(rr)), "solve_field")
        return it.value, rr.value

    def test_hold_exchange(self, extra=1):
        """Make the next solve's first grid exchange wait in vain (pifepic_test_hold_exchange)."""
        self._ok(lib.pifepic_test_hold_exchange(self._c, int(extra)), "test_hold_exchange")

    def solve_field_noalloc(self, F, q, phi):
        """Field solve into phi without any device allocation; F, q, phi are
        CUDA tensors (q may be None).  See pifepic_solve_field_noalloc."""
        it = C.c_int()
        rr = C.c_double()
        self._ok(lib.pifepic_solve_field_noalloc(self._c, _addr(F), _addr(q), _addr(phi), C.byref(it),
                                                 C.byref(rr)), "solve_field_noalloc")
        return it.value, rr.value

    # -- read-back ----------------------------------------------------------------------
    def sizes(self):
        v = [C.c_int64() for _ in range(4)]
        self._ok(lib.pifepic_get_sizes(self._c, *[C.byref(x) for x in v]), "get_sizes")
        return dict(zip(("nnodes", "ncells", "n_interface_tets", "n_cut_cells"), [x.value for x in v]))

    def potential(self):
        out = np.empty(self.sizes()["nnodes"])
        self._ok(lib.pifepic_get_potential(self._c, _addr(out), HOST), "get_potential")
        return out

    def node_E(self):
        out = np.empty((self.sizes()["nnodes"], 3))
        self._ok(lib.pifepic_get_node_E(self._c, _addr(out), HOST), "get_node_E")
        return out

    def node_E_f32(self):
        """The FP32 node field the MIXED push gathers from (pifepic_get_node_E_f32)."""
        out = np.empty((self.sizes()["nnodes"], 3), dtype=np.float32)
        self._ok(lib.pifepic_get_node_E_f32(self._c, _addr(out), HOST), "get_node_E_f32")
        return out

    def node_charge(self, s):
        out = np.empty(self.sizes()["nnodes"], dtype=np.int64)
        self._ok(lib.pifepic_get_node_charge(self._c, s, _addr(out), HOST), "get_node_charge")
        return out

    def surface_counts(self, s):
        out = np.zeros(self.sizes()["n_cut_cells"], dtype=np.int64)
        self._ok(lib.pifepic_get_surface_charge(self._c, s, _addr(out), HOST), "get_surface_charge")
        return out

    def cut_cells(self):
        n = self.sizes()["n_cut_cells"]
        cells = np.zeros(n, dtype=np.int32)
        area = np.zeros(n)
        self._ok(lib.pifepic_get_cut_cells(self._c, _addr(cells), _addr(area)), "get_cut_cells")
        return cells, area

    def cell_target(self):
        out = np.zeros(self.sizes()["ncells"], dtype=np.int32)
        self._ok(lib.pifepic_get_cell_target(self._c, _addr(out)), "get_cell_target")
        return out

    def interface(self):
        n = self.sizes()["n_interface_tets"]
        d = dict(cell=np.zeros(n, np.int32), tet=np.zeros(n, np.int32), vol_plus=np.zeros(n),
                 vol_minus=np.zeros(n), area=np.zeros(n), K=np.zeros((n, 4, 4)), c=np.zeros((n, 4)))
        self._ok(lib.pifepic_get_interface(self._c, *[_addr(d[k]) for k in
                                                     ("cell", "tet", "vol_plus", "vol_minus", "area", "K", "c")]),
                 "get_interface")
        return d

    def count(self, s):
        n = C.c_int64()
        self._ok(lib.pifepic_get_particle_count(self._c, s, C.byref(n)), "get_particle_count")
        return n.value

    def particles(self, s):
        cap = self.count(s)
        out = {k: np.empty(cap) for k in ("x", "y", "z", "vx", "vy", "vz")}
        ids = np.empty(cap, dtype=np.int64) if self.track_ids else None
        n = C.c_int64()
        self._ok(lib.pifepic_get_particles(self._c, s, cap, *[_addr(out[k]) for k in ("x", "y", "z", "vx", "vy", "vz")],
                                           _addr(ids), C.byref(n), HOST), "get_particles")
        out = {k: v[:n.value] for k, v in out.items()}
        if ids is not None:
            out["id"] = ids[:n.value]
        return out


def from_config(cfg, precision=FP64, track_ids=False, pcg_tol=1e-6, pcg_max_iter=150, load=True, inject=True,
                stream=None, bin_edge=None):
    """Build a Simulation for a workload dict of paper_2011_10214_gb300.workloads
    (the macro-particle weights are the workload's own, workloads.macro_weight);
    bin_edge: particle bins of bin_edge^3 cells (None: the library's default)."""
    from .workloads import macro_weight
    sim = Simulation(cfg["n"], cfg["h"], cfg["dt"], cfg.get("origin", (0.0, 0.0, 0.0)), precision, pcg_tol,
                     pcg_max_iter, track_ids, stream, cfg.get("ife_refine", 1))
    if bin_edge is not None:
        sim.set_bin_edge(bin_edge)
    sim.set_field_bc(cfg["face_bc"])
    ob = cfg["object"]
    if ob.get("bedrock") is not None:
        sim.set_bedrock(*ob["bedrock"])
    if ob["kind"] == "sphere":
        sim.set_object(OBJ_SPHERE, list(ob["center"]) + [ob["radius"]], ob["eps_in"], ob["eps_out"])
    elif ob["kind"] == "cap_crater":
        sim.set_object(OBJ_CAP_CRATER, [ob["z_ground"], ob["xc"], ob["yc"], ob["rim_radius"], ob["depth"]],
                       ob["eps_in"], ob["eps_out"])
    elif ob["kind"] == "rim_crater":
        sim.set_object(OBJ_RIM_CRATER, [ob["z_ground"], ob["xc"], ob["yc"], ob["r_inner"], ob["r_top"],
                                        ob["r_outer"], ob["height"], ob["depth"]], ob["eps_in"], ob["eps_out"])
    else:
        sim.set_object(OBJ_NONE, [], 1.0, 1.0)
    pbc = cfg.get("particle_bc")
    for sp in cfg["species"]:
        s = sim.add_species(sp["q"], sp["m"], macro_weight(cfg, sp))
        if pbc is not None:
            sim.set_particle_bc(s, pbc)
        if load:
            sim.load_maxwellian(s, sp["ppc"], sp["vth"], sp["drift"], cfg["seed"])
        if inject:
            sim.set_injection(s, cfg["inject_faces"], sp["density"], sp["vth"], sp["drift"], cfg["seed"])
    ph = cfg.get("photo")
    if ph is not None:
        s = sim.add_species(ph["q"], ph["m"], ph["weight"])
        if pbc is not None:
            sim.set_particle_bc(s, pbc)
        if inject:
            sim.set_photoemission(s, ph["sun"], ph["density"], ph["vth"], cfg["seed"])
    return sim


class Batch:
    """Many Simulations advanced together, one CUDA graph launch per step
    (pifepic_batch_*).  Members keep their own state; results of a member do
    not depend on the others."""

    def __init__(self, sims=(), stream=None):
        self._b = C.c_void_p()
        self.members = []
        st = lib.pifepic_batch_create(None, 0, C.c_void_p(stream or 0), C.byref(self._b))
        if st != 0:
            raise PifepicError(f"pifepic_batch_create: {STATUS.get(st, st)}")
        for s in sims:
            self.add(s)

    def _ok(self, st, what):
        if st != 0:
            raise PifepicError(f"{what}: {STATUS.get(st, st)}: {lib.pifepic_batch_last_error(self._b).decode()}")

    def add(self, sim):
        self._ok(lib.pifepic_batch_add(self._b, sim._c), "batch_add")
        self.members.append(sim)

    def remove(self, sim):
        self._ok(lib.pifepic_batch_remove(self._b, sim._c), "batch_remove")
        self.members.remove(sim)

    def set_preconditioner(self, kind):
        """The batched MIXED solves' preconditioner (pifepic_batch_set_preconditioner)."""
        self._ok(lib.pifepic_batch_set_preconditioner(self._b, int(kind)), "batch_set_preconditioner")

    def set_cta_nodes(self, cta_nodes):
        """Preferred nodes per CTA of the clustered field solves (a power of two, 2048 to 65536)."""
        self._ok(lib.pifepic_batch_set_cta_nodes(self._b, int(cta_nodes)), "batch_set_cta_nodes")

    def step(self, nsteps=1, stats=True):
        n = len(self.members)
        arr = (Stats * max(n, 1))() if stats else None
        self._ok(lib.pifepic_batch_step(self._b, int(nsteps), C.cast(arr, C.c_void_p) if arr is not None else None),
                 "batch_step")
        if not stats:
            return None
        return [arr[i].as_dict(m.nspecies) for i, m in enumerate(self.members)]

    def close(self):
        if self._b is not None and self._b.value:
            lib.pifepic_batch_destroy(self._b)
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
